"""GB300-native dual-tree fast Gauss transform (Lee, Gray & Moore).

Python face of ``libdfgt.so``.  PyTorch provides device memory and the
stream; every step of the computation runs in the library's CUDA kernels.

    ctx = Context()                       # device 0, a private CUDA stream
    tree = Tree(ctx, points)              # points: float32 CUDA tensor [n, d]
    G, stats = kde_sum(ctx, tree, tree, [0.01, 0.1], eps=1e-2)   # [nh, n] float64
    Gx = kde_sum_bruteforce(ctx, points, points, [0.01, 0.1])    # exact sums
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib

__all__ = ["Context", "Tree", "DFGTError", "kde_sum", "kde_sum_loo", "kde_sum_batches", "kde_sum_bruteforce",
           "kde_sum_bruteforce_static", "kde_host", "apply_pairs", "cv_scores", "cv_grad", "cv_likelihood",
           "autotune", "build"]


class DFGTError(RuntimeError):
    def __init__(self, status, message):
        self.status = _lib.STATUS.get(status, str(status))
        super().__init__(f"{self.status}: {message}")


def build(force: bool = False) -> str:
    from .build_ext import build as _b

    return _b(force=force)


def _torch():
    import torch

    return torch


class Context:
    """A device, a CUDA stream (a torch stream the library runs on) and the
    library's cached workspace.  Calls wait for the caller's current torch
    stream before they start, and return after their own work finished."""

    def __init__(self, device: int = 0):
        torch = _torch()
        self.lib = _lib.load()
        self.device = device
        self.stream = torch.cuda.Stream(device=device)
        h = C.c_void_p()
        st = self.lib.dfgt_create(C.byref(h), device, C.c_void_p(self.stream.cuda_stream))
        if st != 0:
            raise DFGTError(st, "dfgt_create failed")
        self.h = h

    def check(self, st, what):
        if st != 0:
            msg = self.lib.dfgt_last_error(self.h)
            raise DFGTError(st, f"{what}: {msg.decode() if msg else ''}")

    def set_capacity(self, frontier_pairs: int, list_items: int):
        """Initial work-list capacities (pairs per frontier, items per list)."""
        self.check(self.lib.dfgt_set_capacity(self.h, int(frontier_pairs), int(list_items)),
                   "dfgt_set_capacity")

    def launch_count(self) -> int:
        """Kernels this context launched so far."""
        return int(self.lib.dfgt_launch_count(self.h))

    def test_wait_timeout(self, on: bool):
        """Make every grid-barrier wait of this context's cooperative launches
        run out (on) or restore the normal waits (off); see
        dfgt_test_wait_timeout in include/dfgt.h."""
        self.check(self.lib.dfgt_test_wait_timeout(self.h, 1 if on else 0), "dfgt_test_wait_timeout")

    def order_after_torch(self):
        torch = _torch()
        self.stream.wait_stream(torch.cuda.current_stream(self.device))

    def close(self):
        if getattr(self, "h", None):
            self.lib.dfgt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _opts(leaf_size=0, p_max=0, eps_fp=0.0, base_block=0):
    return _lib.Opts(int(leaf_size), int(p_max), float(eps_fp), int(base_block))


class Tree:
    """The mid-point kd-tree of Algorithm 2 over float32 points [n, d] on
    the context's device, with the raw far-field moments of every node."""

    def __init__(self, ctx: Context, points, leaf_size: int = 0, p_max: int = 0, eps_fp: float = 0.0,
                 base_block: int = 0):
        torch = _torch()
        if not (isinstance(points, torch.Tensor) and points.is_cuda and points.dtype == torch.float32
                and points.dim() == 2):
            raise TypeError("points must be a float32 CUDA tensor [n, d]")
        self.ctx = ctx
        self.points = points.contiguous()
        self.n, self.d = self.points.shape
        opts = _opts(leaf_size, p_max, eps_fp, base_block)
        h = C.c_void_p()
        ctx.order_after_torch()
        st = ctx.lib.dfgt_build(ctx.h, C.c_void_p(self.points.data_ptr()), self.n, self.d,
                                C.byref(opts), C.byref(h))
        ctx.check(st, "dfgt_build")
        self.h = h

    def info(self) -> dict:
        inf = _lib.TreeInfo()
        self.ctx.check(self.ctx.lib.dfgt_tree_get_info(self.h, C.byref(inf)), "dfgt_tree_get_info")
        return {k: getattr(inf, k) for k, _ in inf._fields_}

    def export(self) -> dict:
        inf = self.info()
        nn, d, P = inf["n_nodes"], inf["d"], inf["n_coeff"]
        out = {"perm": np.empty(self.n, np.int32), "lo": np.empty((nn, d), np.float32),
               "hi": np.empty((nn, d), np.float32), "begin": np.empty(nn, np.int32),
               "count": np.empty(nn, np.int32), "left": np.empty(nn, np.int32),
               "moments": np.empty((nn, P), np.float64), "radius": np.empty(nn, np.float32)}
        ptr = [C.c_void_p(out[k].ctypes.data) for k in ("perm", "lo", "hi", "begin", "count", "left", "moments",
                                                         "radius")]
        self.ctx.check(self.ctx.lib.dfgt_tree_export(self.h, *ptr), "dfgt_tree_export")
        out["info"] = inf
        return out

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.dfgt_tree_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _hs(hs):
    a = np.ascontiguousarray(np.atleast_1d(np.asarray(hs, dtype=np.float64)))
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def kde_sum(ctx: Context, qtree: Tree, rtree: Tree, hs, eps: float, out=None):
    """G~ [nh, nq] float64 (CUDA) within relative error eps of Eq. 5, and work stats."""
    torch = _torch()
    ha, hp = _hs(hs)
    if out is None:
        out = torch.empty((len(ha), qtree.n), dtype=torch.float64, device=f"cuda:{ctx.device}")
    stats = _lib.Stats()
    ctx.order_after_torch()
    st = ctx.lib.dfgt_sum(ctx.h, qtree.h, rtree.h, hp, len(ha), float(eps), C.c_void_p(out.data_ptr()),
                          C.byref(stats))
    ctx.check(st, "dfgt_sum")
    return out, stats.as_dict()


def kde_sum_log(ctx: Context, qtree: Tree, rtree: Tree, hs, eps: float):
    """dfgt_sum_log: G~ and log G~ [nh, nq] float64 (CUDA) with
    |exp(log G~ - log G) - 1| <= eps for every query, including sums below
    the float range, and work stats."""
    torch = _torch()
    ha, hp = _hs(hs)
    out = torch.empty((len(ha), qtree.n), dtype=torch.float64, device=f"cuda:{ctx.device}")
    lout = torch.empty_like(out)
    stats = _lib.Stats()
    ctx.order_after_torch()
    st = ctx.lib.dfgt_sum_log(ctx.h, qtree.h, rtree.h, hp, len(ha), float(eps), C.c_void_p(out.data_ptr()),
                              C.c_void_p(lout.data_ptr()), C.byref(stats))
    ctx.check(st, "dfgt_sum_log")
    return out, lout, stats.as_dict()


def kde_sum_loo(ctx: Context, tree: Tree, hs, eps: float, out=None):
    """dfgt_sum_loo: leave-one-out sums S~ [nh, n] float64 (CUDA) over the
    tree's points, |S~ - S| <= eps S, and work stats."""
    torch = _torch()
    ha, hp = _hs(hs)
    if out is None:
        out = torch.empty((len(ha), tree.n), dtype=torch.float64, device=f"cuda:{ctx.device}")
    stats = _lib.Stats()
    ctx.order_after_torch()
    st = ctx.lib.dfgt_sum_loo(ctx.h, tree.h, hp, len(ha), float(eps), C.c_void_p(out.data_ptr()),
                              C.byref(stats))
    ctx.check(st, "dfgt_sum_loo")
    return out, stats.as_dict()


def kde_sum_batches(ctx: Context, query_batches, rtree: Tree, hs, eps: float, leaf_size: int = 0,
                    base_block: int = 0, eps_fp: float = 0.0, max_queries: int = 1 << 18, log: bool = False):
    """Sums for several query batches against one reference tree.  A query's
    sum does not depend on the other queries, so consecutive batches are
    concatenated into groups of at most ``max_queries`` queries (a larger
    batch is a group of its own), each group into one query tree summed in
    one call; a group whose frontier would pass the context's capacity
    (DFGT_ECAPACITY) is halved and retried.  Returns one [nh, n_b] float64
    tensor per batch (with ``log``: (G, log G) pairs from dfgt_sum_log) and
    the summed work statistics."""
    torch = _torch()
    sizes = [int(b.shape[0]) for b in query_batches]
    groups, cur, cnt = [], [], 0
    for i, m in enumerate(sizes):
        if cur and cnt + m > max_queries:
            groups.append(cur)
            cur, cnt = [], 0
        cur.append(i)
        cnt += m
    if cur:
        groups.append(cur)
    outs = [None] * len(sizes)
    total = {}

    def group_points(idx):
        # consecutive batches that already lie back to back in one tensor
        # (e.g. splits of one array) are used in place; others are copied
        bs = [query_batches[i] for i in idx]
        if all(b.is_contiguous() and b.dim() == 2 for b in bs) and all(
                bs[k + 1].data_ptr() == bs[k].data_ptr() + bs[k].numel() * bs[k].element_size()
                for k in range(len(bs) - 1)):
            first = bs[0]
            rows = sum(int(b.shape[0]) for b in bs)
            return first.as_strided((rows, first.shape[1]), (first.shape[1], 1))
        return torch.cat([b.contiguous() for b in bs], dim=0)

    def run(idx):
        q = group_points(idx)
        qt = Tree(ctx, q, leaf_size=leaf_size, base_block=base_block, eps_fp=eps_fp)
        try:
            if log:
                G, L, st = kde_sum_log(ctx, qt, rtree, hs, eps)
            else:
                G, st = kde_sum(ctx, qt, rtree, hs, eps)
        except DFGTError as e:
            qt.close()
            if e.status != "DFGT_ECAPACITY" or len(idx) == 1:
                raise
            run(idx[: len(idx) // 2])
            run(idx[len(idx) // 2:])
            return
        qt.close()
        parts = torch.split(G, [sizes[i] for i in idx], dim=1)
        lparts = torch.split(L, [sizes[i] for i in idx], dim=1) if log else [None] * len(idx)
        for i, g, lg in zip(idx, parts, lparts):
            outs[i] = (g, lg) if log else g
        for k, v in st.items():
            if isinstance(v, (int, float)):
                total[k] = total.get(k, 0) + v

    for idx in groups:
        run(idx)
    return outs, total


def cv_scores(ctx: Context, tree: Tree, hs, eps: float):
    """dfgt_cv_scores: CV_LK and CV_LS for each bandwidth over the tree's
    point set, with bounds on their error; returns a dict of numpy arrays."""
    ha, hp = _hs(hs)
    nh = len(ha)
    outs = {k: np.empty(nh) for k in ("cv_lk", "cv_ls", "lk_bound", "ls_bound")}
    ptr = {k: v.ctypes.data_as(C.POINTER(C.c_double)) for k, v in outs.items()}
    stats = _lib.Stats()
    ctx.order_after_torch()
    st = ctx.lib.dfgt_cv_scores(ctx.h, tree.h, hp, nh, float(eps), ptr["cv_lk"], ptr["cv_ls"],
                                ptr["lk_bound"], ptr["ls_bound"], C.byref(stats))
    ctx.check(st, "dfgt_cv_scores")
    outs["stats"] = stats.as_dict()
    return outs


def cv_grad(ctx: Context, points, hs, want_points: bool = True):
    """dfgt_cv_grad: CV_LK, dCV_LK/dlog h (numpy [nh]) and dCV_LK/dx (float64
    CUDA tensor [nh, n, d], or None) over the points, from exact sums."""
    torch = _torch()
    if not (isinstance(points, torch.Tensor) and points.is_cuda and points.dtype == torch.float32
            and points.dim() == 2):
        raise TypeError("points must be a float32 CUDA tensor [n, d]")
    x = points.contiguous()
    n, d = x.shape
    ha, hp = _hs(hs)
    nh = len(ha)
    cv, dlogh = np.empty(nh), np.empty(nh)
    dx = torch.empty((nh, n, d), dtype=torch.float64, device=x.device) if want_points else None
    ctx.order_after_torch()
    st = ctx.lib.dfgt_cv_grad(ctx.h, C.c_void_p(x.data_ptr()), n, d, hp, nh,
                              cv.ctypes.data_as(C.POINTER(C.c_double)),
                              dlogh.ctypes.data_as(C.POINTER(C.c_double)),
                              C.c_void_p(dx.data_ptr() if dx is not None else 0))
    ctx.check(st, "dfgt_cv_grad")
    return cv, dlogh, dx


def cv_likelihood(ctx: Context, points, log_h):
    """CV_LK at the bandwidths exp(log_h) as a differentiable function of
    the points (float32 CUDA [n, d]) and of log_h (float64 tensor [nh]):
    the backward pass is the hand-written adjoint of dfgt_cv_grad."""
    torch = _torch()

    class _CVLikelihood(torch.autograd.Function):
        @staticmethod
        def forward(fctx, x, lh):
            hs = torch.exp(lh.detach().double()).cpu().numpy()
            cv, dlogh, dx = cv_grad(ctx, x.detach(), hs, want_points=x.requires_grad)
            fctx.save_for_backward(torch.from_numpy(dlogh), dx if dx is not None else torch.empty(0))
            fctx.has_dx = dx is not None
            return torch.from_numpy(cv).to(lh.device)

        @staticmethod
        def backward(fctx, g):
            dlogh, dx = fctx.saved_tensors
            g64 = g.double()
            gl = (g64.cpu() * dlogh).to(g.device)
            gx = None
            if fctx.has_dx:
                gx = torch.einsum("k,knd->nd", g64.to(dx.device), dx).float()
            return gx, gl

    return _CVLikelihood.apply(points, log_h)


def autotune(ctx: Context, points, hs, eps: float, trials: int = 2, p_max: int = 0, eps_fp: float = 0.0):
    """dfgt_autotune: the leaf size, exact-sum threshold and expansion order
    limit that make a build + sum of these points fastest; returns (options
    dict, ms).  p_max > 0 fixes the order instead of searching it."""
    torch = _torch()
    if not (isinstance(points, torch.Tensor) and points.is_cuda and points.dtype == torch.float32
            and points.dim() == 2):
        raise TypeError("points must be a float32 CUDA tensor [n, d]")
    p = points.contiguous()
    ha, hp = _hs(hs)
    opts = _opts(0, p_max, eps_fp, 0)
    ms = C.c_double(0.0)
    ctx.order_after_torch()
    st = ctx.lib.dfgt_autotune(ctx.h, C.c_void_p(p.data_ptr()), p.shape[0], p.shape[1], hp, len(ha),
                               float(eps), int(trials), C.byref(opts), C.byref(ms))
    ctx.check(st, "dfgt_autotune")
    return {"leaf_size": opts.leaf_size, "base_block": opts.base_block, "p_max": opts.p_max,
            "eps_fp": opts.eps_fp}, ms.value


def kde_sum_bruteforce(ctx: Context, q, r, hs, out=None):
    """Exact G [nh, nq] float64 (CUDA) by the all-pairs sum."""
    torch = _torch()
    ha, hp = _hs(hs)
    q = q.contiguous()
    r = r.contiguous()
    if out is None:
        out = torch.empty((len(ha), q.shape[0]), dtype=torch.float64, device=f"cuda:{ctx.device}")
    ctx.order_after_torch()
    st = ctx.lib.dfgt_sum_bruteforce(ctx.h, C.c_void_p(q.data_ptr()), q.shape[0], C.c_void_p(r.data_ptr()),
                                     r.shape[0], q.shape[1], hp, len(ha), C.c_void_p(out.data_ptr()))
    ctx.check(st, "dfgt_sum_bruteforce")
    return out


def kde_sum_bruteforce_static(q, r, hs, out, stream=None):
    """Exact G [nh, nq] into a preallocated float64 CUDA tensor `out`,
    without any device allocation by the library (static scratch; see
    dfgt_sum_bruteforce_static in include/dfgt.h for the limit and the
    rule that overlapping calls race).  q and r must be contiguous float32
    CUDA tensors [n, d] on one device (no copy is made: a copy would be an
    allocation, and one on another stream could be freed while the kernels
    still read it).  Runs on `stream` (a torch CUDA stream, default: the
    current one) and returns without waiting."""
    torch = _torch()
    lib = _lib.load()
    for name, t in (("q", q), ("r", r)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.dim() == 2):
            raise ValueError(f"{name} must be a float32 CUDA tensor [n, d]")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if q.shape[1] != r.shape[1] or q.device != r.device:
        raise ValueError("q and r must have the same dimension and device")
    ha, hp = _hs(hs)
    if not (isinstance(out, torch.Tensor) and out.is_cuda and out.dtype == torch.float64 and out.is_contiguous()
            and tuple(out.shape) == (len(ha), q.shape[0]) and out.device == q.device):
        raise ValueError("out must be a contiguous float64 CUDA tensor [len(hs), nq] on q's device")
    with torch.cuda.device(q.device):
        stream = torch.cuda.current_stream(q.device) if stream is None else stream
        st = lib.dfgt_sum_bruteforce_static(C.c_void_p(q.data_ptr()), q.shape[0], C.c_void_p(r.data_ptr()),
                                            r.shape[0], q.shape[1], hp, len(ha), C.c_void_p(out.data_ptr()),
                                            C.c_void_p(stream.cuda_stream))
    if st != 0:
        raise DFGTError(st, "dfgt_sum_bruteforce_static failed")
    return out


def kde_host(ctx: Context, q: np.ndarray, r: np.ndarray | None, hs, eps: float, leaf_size=0, p_max=0,
             eps_fp=0.0, out: np.ndarray | None = None):
    """End to end on host arrays: G~ [nh, nq] float64 (numpy).  Pass r=None
    (or r is q) for the cross-validation setting Q = R (one tree)."""
    q = np.ascontiguousarray(q, dtype=np.float32)
    same = r is None or r is q
    r = q if same else np.ascontiguousarray(r, dtype=np.float32)
    ha, hp = _hs(hs)
    if out is None:
        out = np.empty((len(ha), q.shape[0]), dtype=np.float64)
    opts = _opts(leaf_size, p_max, eps_fp)
    stats = _lib.Stats()
    st = ctx.lib.dfgt_kde_host(ctx.h, C.c_void_p(q.ctypes.data), q.shape[0], C.c_void_p(r.ctypes.data),
                               r.shape[0], q.shape[1], hp, len(ha), float(eps), C.byref(opts),
                               C.c_void_p(out.ctypes.data), C.byref(stats))
    ctx.check(st, "dfgt_kde_host")
    return out, stats.as_dict()


def apply_pairs(ctx: Context, qtree: Tree, rtree: Tree, qnode, rnode, action, order, h: float, out=None,
                with_stats: bool = False):
    """Contributions of explicit (Q, R, action, order) items for one bandwidth
    (and, with with_stats, the exact sums' work counters)."""
    torch = _torch()
    arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.int32)) for a in (qnode, rnode, action, order)]
    n = len(arrs[0])
    if out is None:
        out = torch.empty(qtree.n, dtype=torch.float64, device=f"cuda:{ctx.device}")
    ctx.order_after_torch()
    stats = _lib.Stats()
    st = ctx.lib.dfgt_apply_pairs(ctx.h, qtree.h, rtree.h, *[C.c_void_p(a.ctypes.data) for a in arrs], n,
                                  float(h), C.c_void_p(out.data_ptr()), C.byref(stats))
    ctx.check(st, "dfgt_apply_pairs")
    return (out, stats.as_dict()) if with_stats else out
