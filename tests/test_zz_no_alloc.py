"""The allocation-free brute-force entry point (dfgt_sum_bruteforce_static).

It exists for callers that must not allocate device memory (code running
under CUDA graph capture, hosts with a fixed memory budget, loops that
cannot afford an allocation's synchronisation).  Its scratch is a static
device array shared by every call, so the test makes two calls in a row
with different sizes and checks both against the context-based entry
point.  This file is collected last so that a failure here cannot hide
failures elsewhere.
"""
import numpy as np
import pytest
import torch

import paper_1102_2878_gb300 as dfgt
from paper_1102_2878_gb300 import _lib, datagen

pytestmark = pytest.mark.gpu

TOL = 1e-5  # the brute-force tolerance of the other GPU tests


def test_static_scratch_entry_matches_bruteforce_twice():
    dfgt.build()
    ctx = dfgt.Context(0)
    cases = [(3000, 40_000, 3, list(datagen.logspace_bandwidths(0.01, 0.5, 10))),
             (700, 9_000, 5, [0.05, 0.2])]
    for nq, nr, D, hs in cases:
        q = torch.from_numpy(datagen.isotropic_mixture(nq, D, 4, 0.08, seed=nq)).cuda()
        r = torch.from_numpy(datagen.isotropic_mixture(nr, D, 4, 0.08, seed=nr)).cuda()
        want = dfgt.kde_sum_bruteforce(ctx, q, r, hs)
        out = torch.full((len(hs), nq), float("nan"), dtype=torch.float64, device="cuda")
        dfgt.kde_sum_bruteforce_static(q, r, hs, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref = want.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.all(np.abs(got - ref) <= TOL * ref), (nq, nr, D)
    ctx.close()


def test_static_scratch_entry_rejects_oversize_requests():
    q = torch.zeros((600_000, 2), dtype=torch.float32, device="cuda")
    out = torch.empty((2, 600_000), dtype=torch.float64, device="cuda")
    with pytest.raises(dfgt.DFGTError, match="ECAPACITY"):
        dfgt.kde_sum_bruteforce_static(q, q, [0.1, 0.2], out)
    lib = _lib.load()
    assert lib.dfgt_sum_bruteforce_static(None, 1, None, 1, 2, None, 1, None, None) == 1  # EINVAL
