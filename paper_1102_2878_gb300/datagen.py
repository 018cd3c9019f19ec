"""Seeded synthetic point sets shaped like the paper's workloads.

This module holds no part of the kernel-summation method: it only draws
coordinates.  Both the CUDA path and the CPU oracle are fed from here, so
every comparison runs on bit-identical inputs.

The paper evaluates on astronomy (2-D, 3-D) and pharmaceutical (5-D) point
sets (Section 4, experiment tables).  Those datasets are not available, so
clustered Gaussian mixtures stand in for them; every recipe below is one
named workload with fixed sizes.  Points are drawn in float64, clipped to
the unit cube and rounded to float32 (the GPU storage type); callers that
need float64 get the float32 values widened, so both sides see the same
numbers.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "isotropic_mixture",
    "anisotropic_mixture",
    "mixture_with_background",
    "manifold_points",
    "uneven_query_batches",
    "workload",
    "WORKLOADS",
    "bichromatic",
    "BICHROMATIC",
    "logspace_bandwidths",
]


def _finish(x: np.ndarray) -> np.ndarray:
    """Clip to [0,1]^D and round to float32 (row-major, contiguous)."""
    return np.ascontiguousarray(np.clip(x, 0.0, 1.0).astype(np.float32))


def isotropic_mixture(n: int, d: int, k: int, sigma, seed: int, draw_seed: int | None = None) -> np.ndarray:
    """n points from k isotropic Gaussians with means uniform in [0,1]^d.

    ``sigma`` is either one standard deviation for all components or a pair
    (lo, hi) from which each component's deviation is drawn log-uniformly.
    Components have equal weight.  The mixture comes from ``seed``; with
    ``draw_seed`` the points are an independent draw from that same mixture.
    """
    rng = np.random.default_rng(seed)
    means = rng.random((k, d))
    if np.isscalar(sigma):
        sig = np.full(k, float(sigma))
    else:
        lo, hi = sigma
        sig = np.exp(rng.uniform(np.log(lo), np.log(hi), size=k))
    if draw_seed is not None:
        rng = np.random.default_rng(draw_seed)
    comp = rng.integers(0, k, size=n)
    x = means[comp] + rng.standard_normal((n, d)) * sig[comp, None]
    return _finish(x)


def anisotropic_mixture(n: int, d: int, k: int, eig_lo: float, eig_hi: float,
                        seed: int) -> np.ndarray:
    """n points from k Gaussians with random SPD covariances U diag(l) U^T.

    U is Haar-random (QR of a Gaussian matrix with sign fix) and the
    eigenvalues l are log-uniform in [eig_lo, eig_hi].
    """
    rng = np.random.default_rng(seed)
    means = rng.random((k, d))
    chol = np.empty((k, d, d))
    for c in range(k):
        a = rng.standard_normal((d, d))
        qm, rm = np.linalg.qr(a)
        qm = qm * np.sign(np.diag(rm))[None, :]
        lam = np.exp(rng.uniform(np.log(eig_lo), np.log(eig_hi), size=d))
        chol[c] = qm * np.sqrt(lam)[None, :]
    comp = rng.integers(0, k, size=n)
    z = rng.standard_normal((n, d))
    x = means[comp] + np.einsum("nij,nj->ni", chol[comp], z)
    return _finish(x)


def mixture_with_background(n: int, d: int, k: int, sigma_lo: float,
                            sigma_hi: float, background: float,
                            seed: int) -> np.ndarray:
    """Isotropic mixture plus a fraction ``background`` of uniform points."""
    rng = np.random.default_rng(seed)
    nb = int(round(n * background))
    fg = isotropic_mixture(n - nb, d, k, (sigma_lo, sigma_hi), seed + 1000)
    bg = rng.random((nb, d)).astype(np.float32)
    x = np.concatenate([fg, bg], axis=0)
    return np.ascontiguousarray(x[rng.permutation(n)])


def manifold_points(n: int, d: int, latent: int, noise: float,
                    seed: int) -> np.ndarray:
    """Points on a smooth latent-dimensional manifold in [0,1]^d plus noise.

    x = 0.5 + 0.45 sin(W u + b), u ~ U[0,1]^latent, W ~ N(0, pi^2).
    """
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((d, latent)) * np.pi
    b = rng.uniform(0, 2 * np.pi, size=d)
    u = rng.random((n, latent))
    x = 0.5 + 0.45 * np.sin(u @ w.T + b) + rng.standard_normal((n, d)) * noise
    return _finish(x)


def uneven_query_batches(nbatch: int, lo: int, hi: int, seed: int):
    """Batch sizes floor(exp(U[ln lo, ln hi])) for uneven query sets."""
    rng = np.random.default_rng(seed)
    return np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi), size=nbatch))).astype(np.int64)


def logspace_bandwidths(lo: float, hi: float, n: int) -> np.ndarray:
    return np.exp(np.linspace(np.log(lo), np.log(hi), n))


# Named workloads.  "Q=R" means the query set is the reference set itself
# (the cross-validation setting of the paper's introduction).
WORKLOADS = {
    # D=2, N=1e4, 8 isotropic components, sigma 0.05, one bandwidth.
    "kde2d_n1e4": dict(d=2, n=10_000, h=[0.02], eps=1e-2,
                       gen=lambda: isotropic_mixture(10_000, 2, 8, 0.05, seed=1)),
    # D=3, N=2e5, 32 anisotropic components, 10 bandwidths in [1e-3, 1].
    "kde3d_n2e5_sweep10": dict(d=3, n=200_000,
                               h=list(logspace_bandwidths(1e-3, 1.0, 10)), eps=1e-2,
                               gen=lambda: anisotropic_mixture(200_000, 3, 32, 1e-4, 1e-2, seed=2)),
    # D=5, N=5e5, 64 isotropic components + 10% uniform background.
    "kde5d_n5e5": dict(d=5, n=500_000, h=[0.01, 0.05, 0.2], eps=1e-3,
                       gen=lambda: mixture_with_background(500_000, 5, 64, 0.02, 0.1, 0.1, seed=3)),
    # D=16, N=1e6, 4-dim manifold, 8 bandwidths in [0.01, 1].
    "kde16d_n1e6_sweep8": dict(d=16, n=1_000_000,
                               h=list(logspace_bandwidths(0.01, 1.0, 8)), eps=1e-2,
                               gen=lambda: manifold_points(1_000_000, 16, 4, 0.01, seed=4)),
}


# Bichromatic workloads: a reference set and separately drawn query batches
# from the same mixture.
BICHROMATIC = {
    # D=32, |R|=1e6 from 128 isotropic components (sigma log-uniform in
    # [0.02, 0.1]); 64 query batches of sizes log-uniform in [1e3, 2e5] from
    # the same mixture; 16 bandwidths in [0.01, 1]; eps 1e-2 and 1e-3.
    "kde32d_r1e6_q64batches": dict(d=32, nr=1_000_000, k=128, sigma=(0.02, 0.1), nbatch=64,
                                   batch_lo=1_000, batch_hi=200_000,
                                   h=list(logspace_bandwidths(0.01, 1.0, 16)), eps=[1e-2, 1e-3], seed=5),
}


def bichromatic(name: str, nr: int | None = None, nbatch: int | None = None,
                batch_hi: int | None = None):
    """Return (references float32 [nr,D], list of query batches, bandwidths,
    eps values) for a named bichromatic workload.  ``nr``, ``nbatch`` and
    ``batch_hi`` give a smaller case of the same recipe."""
    w = BICHROMATIC[name]
    nr = w["nr"] if nr is None else nr
    nbatch = w["nbatch"] if nbatch is None else nbatch
    hi = w["batch_hi"] if batch_hi is None else batch_hi
    refs = isotropic_mixture(nr, w["d"], w["k"], w["sigma"], w["seed"])
    sizes = uneven_query_batches(nbatch, w["batch_lo"], hi, w["seed"] + 100)
    batches = [isotropic_mixture(int(m), w["d"], w["k"], w["sigma"], w["seed"], draw_seed=1000 * w["seed"] + b)
               for b, m in enumerate(sizes)]
    return refs, batches, list(w["h"]), list(w["eps"])


def workload(name: str, n: int | None = None):
    """Return (points float32 [n,D], bandwidths list, eps) for a named workload.

    ``n`` truncates the point set (the first n rows of the full draw), which
    keeps the distribution of a smaller case identical to the full one.
    """
    w = WORKLOADS[name]
    x = w["gen"]()
    if n is not None:
        x = np.ascontiguousarray(x[:n])
    return x, list(w["h"]), w["eps"]
