"""The allocation-free brute-force entry point (dfgt_sum_bruteforce_static).

Some callers cannot let the library allocate device memory: hosts that hand
it a fixed memory budget, code running while a CUDA graph is captured, and
loops where an allocation's implicit synchronisation is not acceptable.
This entry point keeps its scratch in a static device array shared by every
call, so the tests make calls in a row with different sizes (the array keeps
the previous call's contents) and check each against the FP64 oracle within
the float32 tolerance of the other brute-force GPU tests.  The cases cover the
split-reference path with the D <= 5 kernels and the generic kernel
(D = 8), a reference set of one tile (nr <= 128) and a query set large
enough to skip the split.  This file is collected last so that a failure
here cannot hide failures elsewhere.
"""
import numpy as np
import pytest
import torch

import paper_1102_2878_gb300 as dfgt
from paper_1102_2878_gb300 import _lib, datagen

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


def float32_tolerance(q64, r64, h):
    """The brute-force tolerance of the other GPU tests: each float32 term
    exp(-x) carries 2^-21 (ex2) plus (D+4) u x (its exponent from D
    coordinate differences), and the compensated sum 2^-20 of G."""
    D = q64.shape[1]
    tol = np.empty(len(q64))
    G = np.empty(len(q64))
    for i, q in enumerate(q64):
        x = ((r64 - q) ** 2).sum(1) / (2 * h * h)
        K = np.exp(-x)
        tol[i] = (K * (2.0 ** -21 + (D + 4) * U * x)).sum()
        G[i] = K.sum()
    return tol + 2.0 ** -20 * G


CASES = [  # nq, nr, D, bandwidths
    (3000, 40_000, 3, list(datagen.logspace_bandwidths(0.01, 0.5, 10))),
    (700, 9_000, 5, [0.05, 0.2]),
    (1500, 12_000, 8, [0.1, 0.3, 1.0]),
    (900, 100, 3, [0.02, 0.3]),
    (50_000, 1_500, 4, [0.05, 0.2, 0.8]),
]


def _points(n, d, seed):
    return datagen.isotropic_mixture(n, d, 4, 0.08, seed=seed)


def test_static_scratch_entry_matches_oracle_on_calls_in_a_row(orc):
    dfgt.build()
    for nq, nr, D, hs in CASES:
        q = _points(nq, D, nq + D)
        r = _points(nr, D, nr + D)
        qd, rd = torch.from_numpy(q).cuda(), torch.from_numpy(r).cuda()
        out = torch.full((len(hs), nq), float("nan"), dtype=torch.float64, device="cuda")
        dfgt.kde_sum_bruteforce_static(qd, rd, hs, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.isfinite(got).all(), (nq, nr, D)
        q64, r64 = q.astype(np.float64), r.astype(np.float64)
        sample = np.random.default_rng(nq).choice(nq, size=min(nq, 400), replace=False)
        for i, h in enumerate(hs):
            ref = orc.naive_kde(q64[sample], r64, h)
            tol = float32_tolerance(q64[sample], r64, h)
            pos = ref > 1e-30  # the float32 range of the exact terms
            err = np.abs(got[i][sample] - ref)
            assert np.all(err[pos] <= tol[pos]), (nq, nr, D, h)
            assert np.all(np.abs(got[i][sample][~pos]) <= 1e-30), (nq, nr, D, h)


def test_static_scratch_entry_allocates_nothing():
    q = torch.from_numpy(_points(2000, 3, 5)).cuda()
    r = torch.from_numpy(_points(30_000, 3, 6)).cuda()
    hs = [0.03, 0.3]
    out = torch.empty((2, 2000), dtype=torch.float64, device="cuda")
    dfgt.kde_sum_bruteforce_static(q, r, hs, out)  # loads the kernels and looks up the array
    torch.cuda.synchronize()
    first = out.clone()
    free0, _ = torch.cuda.mem_get_info()
    dfgt.kde_sum_bruteforce_static(q, r, hs, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.equal(out, first)


def test_static_scratch_entry_rejects_bad_requests():
    # a split request past the static array's limit
    q = torch.zeros((30_000, 2), dtype=torch.float32, device="cuda")
    hs = list(np.linspace(0.1, 1.0, 40))
    out = torch.empty((40, 30_000), dtype=torch.float64, device="cuda")
    with pytest.raises(dfgt.DFGTError, match="ECAPACITY"):
        dfgt.kde_sum_bruteforce_static(q, q, hs, out)
    lib = _lib.load()
    assert lib.dfgt_sum_bruteforce_static(None, 1, None, 1, 2, None, 1, None, None) == 1  # EINVAL
    # the wrapper checks what the C entry point cannot see
    small = torch.empty((40, 100), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        dfgt.kde_sum_bruteforce_static(q, q, hs, small)
    with pytest.raises(ValueError):
        dfgt.kde_sum_bruteforce_static(q, q, hs, out.float())
    with pytest.raises(ValueError):
        dfgt.kde_sum_bruteforce_static(q, torch.zeros((10, 3), device="cuda"), hs, out)
    with pytest.raises(ValueError):
        dfgt.kde_sum_bruteforce_static(q.t(), q, hs, out)
