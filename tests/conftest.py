import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs on the GB300 box)")


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.build()
    return oracle


def read_golden(name):
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return rows


@pytest.fixture(scope="session")
def dev():
    """The DFGT library on cuda:0 (GPU tests only)."""
    import paper_1102_2878_gb300 as dfgt

    dfgt.build()
    ctx = dfgt.Context(0)
    yield ctx
    ctx.close()


def to_cuda(x):
    import torch

    return torch.from_numpy(x).cuda()
