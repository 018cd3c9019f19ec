"""The tensor cores' layout and rounding that the tensor-core exact sums for
D >= 6 rest on (base_hd_forms.cuh, base_tc.cu): tcgen05.mma kind::f16 with
M = N = 128, float16 operands K-major in 8 x 16-byte core matrices without
swizzle, float32 D in tensor memory.  Every element must match its float64
sum (no element off by more than 64u, which a wrong layout would break),
and the accumulation error must stay within the 4u of the sum of
|products| per chained K16 step that the bound allows (u = 2^-24), for
K = 32, 64 and 112 (the K of D = 8, 16 and 32) with random and with
cancelling operands."""
import os
import re
import shutil
import subprocess

import pytest

from conftest import ROOT

pytestmark = pytest.mark.gpu


def test_tcgen05_layout_and_accumulation_error(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "tcgen05_accum_probe")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                    os.path.join(ROOT, "tests", "tcgen05_accum_probe.cu")], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=120).stdout
    rows = re.findall(r"K=(\d+) status=(\d+) wait=(\d+) worst_random=([\d.]+) worst_cancel=([\d.]+) "
                      r"off=(\d+) steps=(\d+)", out)
    assert {int(r[0]) for r in rows} == {32, 64, 112}, out
    for K, status, wait, rnd, cancel, off, steps in rows:
        assert int(status) == 0 and int(wait) == 0, (K, out)
        assert int(off) == 0, (K, out)
        assert max(float(rnd), float(cancel)) <= 4.0 * int(steps), (K, out)
