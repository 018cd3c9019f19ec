"""The C-ABI library loads and exports every entry point the header declares
(no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def lib():
    from paper_1102_2878_gb300 import _lib, build_ext

    build_ext.build()
    return _lib.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "dfgt.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dfgt_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("dfgt_create", "dfgt_destroy", "dfgt_build", "dfgt_sum", "dfgt_sum_bruteforce",
                 "dfgt_kde_host", "dfgt_last_error", "dfgt_tree_destroy"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_the_header(lib):
    from paper_1102_2878_gb300 import _lib

    assert set(declared_functions()) == set(_lib.SIGNATURES)


def test_invalid_arguments_rejected_without_a_device(lib):
    # argument checks run before any CUDA call
    assert lib.dfgt_create(None, 0, None) == 1          # DFGT_EINVAL
    assert lib.dfgt_build(None, None, 0, 0, None, None) == 1
    assert lib.dfgt_sum(None, None, None, None, 0, 0.0, None, None) == 1
    assert lib.dfgt_grad(None, None, 0, 0, None, 0, None, None, None) == 1
    assert lib.dfgt_cv_grad(None, None, 0, 0, None, 0, None, None, None) == 1
    lib.dfgt_destroy(None)
    lib.dfgt_tree_destroy(None)
    assert lib.dfgt_last_error(None) == b"null context"


def test_library_is_built_for_sm_103a():
    from paper_1102_2878_gb300 import build_ext

    assert "arch=compute_103a,code=sm_103a" in build_ext.ARCH
