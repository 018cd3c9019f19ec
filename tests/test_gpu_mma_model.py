"""The tensor cores' rounding that the bound of the D >= 6 tensor-core exact
sums rests on (base_hd_forms.cuh): mma.sync m16n8k16 and m16n8k8 with
float16 operands and a float32 C, checked on the device against float64
sums.  Both fragment layouts must give every element (no element off by
more than 64u), and the accumulation error must stay within the 8u of the
sum of |terms| that the bound allows per chained step (u = 2^-24)."""
import os
import re
import shutil
import subprocess

import pytest

from conftest import ROOT

pytestmark = pytest.mark.gpu


def test_mma_layouts_and_accumulation_error(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "mma_accum_probe")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                    os.path.join(ROOT, "tests", "mma_accum_probe.cu")], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=120).stdout
    rows = re.findall(r"(m16n8k\d+) status=(\d+) worst_c0=([\d.]+) worst_cancel=([\d.]+) "
                      r"worst_random=([\d.]+) off=(\d+)", out)
    assert {r[0] for r in rows} == {"m16n8k16", "m16n8k8"}, out
    for shape, status, c0, cancel, rand, off in rows:
        assert int(status) == 0, (shape, out)
        assert int(off) == 0, (shape, out)
        assert max(float(c0), float(cancel), float(rand)) <= 8.0, (shape, out)
