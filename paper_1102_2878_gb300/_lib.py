"""ctypes binding of ``libdfgt.so`` (argument marshalling only).

Every entry point of ``include/dfgt.h`` is declared here with the same
name.  Loading fails loudly if the library is missing: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libdfgt.so")

STATUS = {0: "DFGT_OK", 1: "DFGT_EINVAL", 2: "DFGT_ENOMEM", 3: "DFGT_ECUDA",
          4: "DFGT_ECAPACITY", 5: "DFGT_ETIMEOUT", 6: "DFGT_EUNSUPPORTED"}

ACT_PRUNE, ACT_FARFIELD, ACT_LOCAL, ACT_F2L, ACT_BASE = 0, 1, 2, 3, 4


class Opts(C.Structure):
    _fields_ = [("leaf_size", C.c_int), ("p_max", C.c_int), ("eps_fp", C.c_double),
                ("base_block", C.c_longlong)]


class Stats(C.Structure):
    _fields_ = [("pairs_visited", C.c_longlong), ("n_prune", C.c_longlong),
                ("n_farfield", C.c_longlong), ("n_local", C.c_longlong),
                ("n_f2l", C.c_longlong), ("n_base", C.c_longlong),
                ("base_interactions", C.c_longlong), ("kernel_launches", C.c_longlong),
                ("rounds", C.c_int), ("list_flushes", C.c_int),
                ("ms_traverse", C.c_double), ("ms_classify", C.c_double), ("ms_actions", C.c_double),
                ("ms_post", C.c_double),
                ("ms_base", C.c_double), ("ms_farfield", C.c_double), ("ms_local", C.c_double),
                ("ms_f2l", C.c_double), ("base_expanded", C.c_longlong),
                ("farfield_terms", C.c_longlong), ("local_terms", C.c_longlong),
                ("f2l_terms", C.c_longlong), ("log_queries", C.c_longlong), ("ms_log", C.c_double),
                ("ms_base_tc", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TreeInfo(C.Structure):
    _fields_ = [("n_points", C.c_int64), ("d", C.c_int), ("n_nodes", C.c_int),
                ("n_leaves", C.c_int), ("depth", C.c_int), ("leaf_size", C.c_int),
                ("p_max", C.c_int), ("n_coeff", C.c_int), ("ms_levels", C.c_double),
                ("ms_moments", C.c_double)]


# name -> (restype, argtypes)
SIGNATURES = {
    "dfgt_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_void_p]),
    "dfgt_destroy": (None, [C.c_void_p]),
    "dfgt_set_capacity": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64]),
    "dfgt_last_error": (C.c_char_p, [C.c_void_p]),
    "dfgt_launch_count": (C.c_longlong, [C.c_void_p]),
    "dfgt_test_wait_timeout": (C.c_int, [C.c_void_p, C.c_int]),
    "dfgt_build": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.POINTER(Opts),
                             C.POINTER(C.c_void_p)]),
    "dfgt_tree_destroy": (None, [C.c_void_p]),
    "dfgt_sum": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.c_int,
                           C.c_double, C.c_void_p, C.POINTER(Stats)]),
    "dfgt_sum_log": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.c_int,
                               C.c_double, C.c_void_p, C.c_void_p, C.POINTER(Stats)]),
    "dfgt_sum_bruteforce": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                      C.c_int, C.POINTER(C.c_double), C.c_int, C.c_void_p]),
    "dfgt_sum_bruteforce_static": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int,
                                             C.POINTER(C.c_double), C.c_int, C.c_void_p, C.c_void_p]),
    "dfgt_kde_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int,
                                C.POINTER(C.c_double), C.c_int, C.c_double, C.POINTER(Opts),
                                C.c_void_p, C.POINTER(Stats)]),
    "dfgt_tree_get_info": (C.c_int, [C.c_void_p, C.POINTER(TreeInfo)]),
    "dfgt_tree_export": (C.c_int, [C.c_void_p] + [C.c_void_p] * 8),
    "dfgt_apply_pairs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p] + [C.c_void_p] * 4 +
                         [C.c_int, C.c_double, C.c_void_p, C.POINTER(Stats)]),
    "dfgt_cv_scores": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.c_int, C.c_double,
                                 C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                 C.POINTER(C.c_double), C.POINTER(Stats)]),
    "dfgt_sum_loo": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.c_int, C.c_double,
                               C.c_void_p, C.POINTER(Stats)]),
    "dfgt_cv_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.POINTER(C.c_double), C.c_int,
                               C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p]),
    "dfgt_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.POINTER(C.c_double), C.c_int,
                            C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p]),
    "dfgt_autotune": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.POINTER(C.c_double), C.c_int,
                                C.c_double, C.c_int, C.POINTER(Opts), C.POINTER(C.c_double)]),
}

_lib = None


def load():
    """Load libdfgt.so (built by ``build_ext.build()``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() first "
                           "(the DFGT path has no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
