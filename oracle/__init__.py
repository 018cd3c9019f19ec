"""FP64 CPU oracle for the Dual-Tree Fast Gauss Transform (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library
and its Python binding) never imports it, and it never imports them.

``build()`` compiles ``oracle.c`` with gcc into ``liboracle.so`` beside it.
Every wrapper takes and returns float64 numpy arrays.  Citations to the
paper sit beside each routine in ``oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

INF_ORDER = -1
METHOD_F, METHOD_D, METHOD_T, METHOD_E = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, -O2, OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                        "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = C.CDLL(_LIB)
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int)
    i64 = C.c_int64
    lib.orc_naive_kde.argtypes = [dp, i64, dp, i64, C.c_int, C.c_double, dp]
    lib.orc_log_naive_kde.argtypes = [dp, i64, dp, i64, C.c_int, C.c_double, dp]
    lib.orc_num_threads.argtypes = []
    lib.orc_num_threads.restype = C.c_int
    lib.orc_hermite_functions.argtypes = [C.c_double, C.c_int, dp]
    lib.orc_gauss_volume.argtypes = [C.c_int, C.c_double]
    lib.orc_gauss_volume.restype = C.c_double
    lib.orc_loo_sums.argtypes = [dp, i64, C.c_int, C.c_double, dp]
    lib.orc_cv_lk.argtypes = [dp, i64, C.c_int, C.c_double]
    lib.orc_cv_lk.restype = C.c_double
    lib.orc_cv_ls.argtypes = [dp, i64, C.c_int, C.c_double]
    lib.orc_cv_ls.restype = C.c_double
    lib.orc_cv_lk_grad.argtypes = [dp, i64, C.c_int, C.c_double, dp, dp]
    lib.orc_cv_lk_grad.restype = None
    lib.orc_pmax.argtypes = [C.c_int]
    lib.orc_pmax.restype = C.c_int
    lib.orc_multi_to_pos.argtypes = [ip, C.c_int, C.c_int]
    lib.orc_multi_to_pos.restype = C.c_int
    lib.orc_pos_to_multi.argtypes = [C.c_int, C.c_int, C.c_int, ip]
    lib.orc_farfield_moments.argtypes = [dp, i64, C.c_int, dp, C.c_double, C.c_int, C.c_int, dp]
    lib.orc_eval_farfield.argtypes = [dp, C.c_int, C.c_int, C.c_int, dp, C.c_double, dp]
    lib.orc_eval_farfield.restype = C.c_double
    lib.orc_direct_local.argtypes = [dp, i64, C.c_int, dp, C.c_double, C.c_int, C.c_int, dp]
    lib.orc_far_to_local.argtypes = [dp, C.c_int, C.c_int, C.c_int, dp, dp, C.c_double, dp]
    lib.orc_far_to_far.argtypes = [dp, C.c_int, C.c_int, C.c_int, dp, dp, C.c_double, dp]
    lib.orc_local_to_local.argtypes = [dp, C.c_int, C.c_int, C.c_int, dp, dp, C.c_double, dp]
    lib.orc_eval_local.argtypes = [dp, C.c_int, C.c_int, C.c_int, dp, C.c_double, dp]
    lib.orc_eval_local.restype = C.c_double
    for f in ("orc_bound_farfield", "orc_bound_local", "orc_bound_f2l"):
        getattr(lib, f).argtypes = [C.c_double, C.c_int, C.c_double, C.c_int]
        getattr(lib, f).restype = C.c_double
    lib.orc_order_farfield.argtypes = [dp, dp, C.c_double, C.c_int, C.c_double, C.c_double, C.c_int]
    lib.orc_order_farfield.restype = C.c_int
    lib.orc_order_local.argtypes = [dp, dp, C.c_double, C.c_int, C.c_double, C.c_double, C.c_int]
    lib.orc_order_local.restype = C.c_int
    lib.orc_order_f2l.argtypes = [dp, dp, dp, dp, C.c_double, C.c_int, C.c_double, C.c_double, C.c_int]
    lib.orc_order_f2l.restype = C.c_int
    lib.orc_dist_bounds.argtypes = [dp, dp, dp, dp, C.c_int, dp, dp]
    lib.orc_choose_best_method.argtypes = [dp, dp, C.c_double, dp, dp, C.c_double, C.c_int,
                                           C.c_double, C.c_double, C.c_int, ip]
    lib.orc_choose_best_method.restype = C.c_int
    lib.orc_dfgt.argtypes = [dp, i64, dp, i64, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int,
                             dp, dp, dp, dp, C.POINTER(C.c_longlong)]
    lib.orc_dfgt.restype = C.c_int
    _lib = lib
    return lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(C.POINTER(C.c_int))


def _vec(x, D):
    x = np.ascontiguousarray(np.broadcast_to(np.asarray(x, dtype=np.float64), (D,)))
    return _d(x)


# ---------------------------------------------------------------- exact sum
def naive_kde(Q, R, h):
    """Exact G(q_i) = sum_j exp(-||q_i - r_j||^2 / 2h^2) (Eq. 5, Algorithm 1)."""
    lib = _load()
    Q, qp = _d(np.atleast_2d(Q))
    R, rp = _d(np.atleast_2d(R))
    D = Q.shape[1]
    assert R.shape[1] == D
    G = np.empty(Q.shape[0])
    gp = G.ctypes.data_as(C.POINTER(C.c_double))
    lib.orc_naive_kde(qp, Q.shape[0], rp, R.shape[0], D, float(h), gp)
    return G


def log_naive_kde(Q, R, h):
    """log G(q_i) of Eq. 5 by log-sum-exp with the per-query shift
    m = min_j ||q_i - r_j||^2 / 2h^2 (finite where G underflows)."""
    lib = _load()
    Q, qp = _d(np.atleast_2d(Q))
    R, rp = _d(np.atleast_2d(R))
    D = Q.shape[1]
    assert R.shape[1] == D
    L = np.empty(Q.shape[0])
    lib.orc_log_naive_kde(qp, Q.shape[0], rp, R.shape[0], D, float(h), L.ctypes.data_as(C.POINTER(C.c_double)))
    return L


def num_threads() -> int:
    """Host threads the oracle's parallel loops use."""
    return int(_load().orc_num_threads())


# ---------------------------------------------------------- multi-indices
def gauss_volume(D, h):
    """V_{D,h} of Eq. 1 for the Gaussian kernel."""
    return _load().orc_gauss_volume(int(D), float(h))


def loo_sums(X, h):
    """Leave-one-out sums S_j = sum_{i != j} exp(-|x_j - x_i|^2 / 2h^2)."""
    X, xp = _d(X)
    n, D = X.shape
    S, sp = _d(np.empty(n))
    _load().orc_loo_sums(xp, n, D, float(h), sp)
    return S


def cv_lk(X, h):
    """Likelihood cross-validation score CV_LK(h) of the introduction."""
    X, xp = _d(X)
    return _load().orc_cv_lk(xp, X.shape[0], X.shape[1], float(h))


def cv_lk_grad(X, h):
    """(dCV_LK/dlog h, dCV_LK/dx [n][D]) from the derivative of the definition."""
    X, xp = _d(X)
    n, D = X.shape
    assert D <= 64
    dx, dxp = _d(np.empty((n, D)))
    g = C.c_double()
    _load().orc_cv_lk_grad(xp, n, D, float(h), C.byref(g), dxp)
    return g.value, dx


def cv_ls(X, h):
    """Least-squares cross-validation score CV_LS(h) of the introduction."""
    X, xp = _d(X)
    return _load().orc_cv_ls(xp, X.shape[0], X.shape[1], float(h))


def pmax(D: int) -> int:
    return _load().orc_pmax(D)


def multi_to_pos(alpha, p):
    a, ap = _i(alpha)
    return _load().orc_multi_to_pos(ap, p, len(a))


def pos_to_multi(i, p, D):
    a = np.zeros(D, dtype=np.int32)
    _load().orc_pos_to_multi(i, p, D, a.ctypes.data_as(C.POINTER(C.c_int)))
    return a


def hermite_functions(t, n):
    """[h_0(t), ..., h_{n-1}(t)] with h_k = e^{-t^2} H_k(t)."""
    out = np.zeros(n)
    _load().orc_hermite_functions(float(t), n, out.ctypes.data_as(C.POINTER(C.c_double)))
    return out


# ------------------------------------------------------------ expansions
def farfield_moments(R, c, h, p, pm=None):
    R, rp = _d(np.atleast_2d(R))
    D = R.shape[1]
    pm = p if pm is None else pm
    c, cp = _vec(c, D)
    M = np.zeros(pm ** D)
    _load().orc_farfield_moments(rp, R.shape[0], D, cp, float(h), pm, p,
                                 M.ctypes.data_as(C.POINTER(C.c_double)))
    return M


def eval_farfield(M, c, h, p, q, pm=None):
    q = np.asarray(q, dtype=np.float64)
    D = q.shape[-1]
    pm = p if pm is None else pm
    M, mp = _d(M)
    c, cp = _vec(c, D)
    qq = np.atleast_2d(q)
    out = np.empty(qq.shape[0])
    lib = _load()
    for i in range(qq.shape[0]):
        x, xp = _d(qq[i])
        out[i] = lib.orc_eval_farfield(mp, D, pm, p, cp, float(h), xp)
    return out if q.ndim > 1 else out[0]


def direct_local(R, c, h, p, pm=None, L=None):
    R, rp = _d(np.atleast_2d(R))
    D = R.shape[1]
    pm = p if pm is None else pm
    c, cp = _vec(c, D)
    L = np.zeros(pm ** D) if L is None else np.ascontiguousarray(L, dtype=np.float64)
    _load().orc_direct_local(rp, R.shape[0], D, cp, float(h), pm, p,
                             L.ctypes.data_as(C.POINTER(C.c_double)))
    return L


def far_to_local(M, cR, cQ, h, p, pm=None, L=None):
    D = np.asarray(cR).shape[-1]
    pm = p if pm is None else pm
    M, mp = _d(M)
    cR, crp = _vec(cR, D)
    cQ, cqp = _vec(cQ, D)
    L = np.zeros(pm ** D) if L is None else np.ascontiguousarray(L, dtype=np.float64)
    _load().orc_far_to_local(mp, D, pm, p, crp, cqp, float(h), L.ctypes.data_as(C.POINTER(C.c_double)))
    return L


def far_to_far(M, c_old, c_new, h, p, pm=None, out=None):
    D = np.asarray(c_old).shape[-1]
    pm = p if pm is None else pm
    M, mp = _d(M)
    c0, c0p = _vec(c_old, D)
    c1, c1p = _vec(c_new, D)
    out = np.zeros(pm ** D) if out is None else np.ascontiguousarray(out, dtype=np.float64)
    _load().orc_far_to_far(mp, D, pm, p, c0p, c1p, float(h), out.ctypes.data_as(C.POINTER(C.c_double)))
    return out


def local_to_local(L, c_old, c_new, h, p, pm=None, out=None):
    D = np.asarray(c_old).shape[-1]
    pm = p if pm is None else pm
    L, lp = _d(L)
    c0, c0p = _vec(c_old, D)
    c1, c1p = _vec(c_new, D)
    out = np.zeros(pm ** D) if out is None else np.ascontiguousarray(out, dtype=np.float64)
    _load().orc_local_to_local(lp, D, pm, p, c0p, c1p, float(h), out.ctypes.data_as(C.POINTER(C.c_double)))
    return out


def eval_local(L, c, h, p, q, pm=None):
    q = np.asarray(q, dtype=np.float64)
    D = q.shape[-1]
    pm = p if pm is None else pm
    L, lp = _d(L)
    c, cp = _vec(c, D)
    qq = np.atleast_2d(q)
    out = np.empty(qq.shape[0])
    lib = _load()
    for i in range(qq.shape[0]):
        x, xp = _d(qq[i])
        out[i] = lib.orc_eval_local(lp, D, pm, p, cp, float(h), xp)
    return out if q.ndim > 1 else out[0]


# ---------------------------------------------------------------- bounds
def bound_farfield(nR, D, r, p):
    return _load().orc_bound_farfield(float(nR), D, float(r), p)


def bound_local(nR, D, r, p):
    return _load().orc_bound_local(float(nR), D, float(r), p)


def bound_f2l(nR, D, r, p):
    return _load().orc_bound_f2l(float(nR), D, float(r), p)


def order_farfield(Rlo, Rhi, nR, h, tau, pm):
    lo, lp = _d(Rlo)
    hi, hp = _d(Rhi)
    return _load().orc_order_farfield(lp, hp, float(nR), len(lo), float(h), float(tau), pm)


def order_local(Qlo, Qhi, nR, h, tau, pm):
    lo, lp = _d(Qlo)
    hi, hp = _d(Qhi)
    return _load().orc_order_local(lp, hp, float(nR), len(lo), float(h), float(tau), pm)


def order_f2l(Qlo, Qhi, Rlo, Rhi, nR, h, tau, pm):
    a, ap = _d(Qlo)
    b, bp = _d(Qhi)
    c, cp = _d(Rlo)
    d, dp = _d(Rhi)
    return _load().orc_order_f2l(ap, bp, cp, dp, float(nR), len(a), float(h), float(tau), pm)


def dist_bounds(Qlo, Qhi, Rlo, Rhi):
    a, ap = _d(Qlo)
    b, bp = _d(Qhi)
    c, cp = _d(Rlo)
    d, dpp = _d(Rhi)
    lo = C.c_double()
    hi = C.c_double()
    _load().orc_dist_bounds(ap, bp, cp, dpp, len(a), C.byref(lo), C.byref(hi))
    return lo.value, hi.value


def choose_best_method(Qlo, Qhi, nQ, Rlo, Rhi, nR, h, tau, pm):
    a, ap = _d(Qlo)
    b, bp = _d(Qhi)
    c, cp = _d(Rlo)
    d, dpp = _d(Rhi)
    order = C.c_int()
    m = _load().orc_choose_best_method(ap, bp, float(nQ), cp, dpp, float(nR), len(a), float(h),
                                       float(tau), pm, C.byref(order))
    return m, order.value


# ------------------------------------------------------------ traversal
def dfgt(Q, R, h, eps, leaf=32, pm=0, want_bounds=False, want_acct=False):
    """The paper's recursive DFGTMain in FP64.

    Returns G~ (and, when asked, the per-query bounds, the number of
    reference points accounted per query, and the stats
    [prune, F, D, T, base pairs, DFGT calls])."""
    lib = _load()
    Q, qp = _d(np.atleast_2d(Q))
    R, rp = _d(np.atleast_2d(R))
    nq, D = Q.shape
    G = np.zeros(nq)
    Gl = np.zeros(nq) if want_bounds else None
    Gu = np.zeros(nq) if want_bounds else None
    acct = np.zeros(nq) if want_acct else None
    stats = (C.c_longlong * 6)()
    null = C.POINTER(C.c_double)()

    def ptr(a):
        return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else null

    rc = lib.orc_dfgt(qp, nq, rp, R.shape[0], D, float(h), float(eps), int(leaf), int(pm),
                      ptr(G), ptr(Gl), ptr(Gu), ptr(acct), stats)
    if rc != 0:
        raise ValueError("orc_dfgt: invalid arguments")
    out = {"G": G, "stats": list(stats)}
    if want_bounds:
        out["Gl"], out["Gu"] = Gl, Gu
    if want_acct:
        out["acct"] = acct
    return out
