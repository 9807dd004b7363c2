"""The C-ABI library builds, loads and exports every declared symbol (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    with open(os.path.join(ROOT, "include", "wd.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|const char \*)\s*\*?\s*(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_0710_1988_gb300 import build
    build.build()
    import paper_0710_1988_gb300 as pkg
    return pkg.lib()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for fn in ("wd_create", "wd_apply", "gmresdr_solve", "dbicgstab_solve", "wd_destroy",
               "wd_error_string", "wd_last_error_detail"):
        assert fn in names


def test_every_declared_symbol_is_exported(lib):
    from paper_0710_1988_gb300 import _lib
    names = _declared_functions()
    for fn in names:
        assert hasattr(lib, fn), fn
    # the binding declares exactly the header's functions
    assert sorted(_lib.SIGNATURES) == names


def test_error_strings(lib):
    assert lib.wd_error_string(0) == b"ok"
    assert lib.wd_error_string(2) == b"not converged"
    assert lib.wd_error_string(99) == b"unknown status"


def test_argument_checks_need_no_gpu(lib):
    from paper_0710_1988_gb300 import _lib
    h = ctypes.c_void_p()
    bad = (ctypes.c_int * 4)(4, 0, 4, 4)
    assert lib.wd_create(bad, ctypes.c_void_p(1), 0.1, 0.0, ctypes.byref(h)) == _lib.WD_BAD_ARG
    assert "extents" in _lib.last_error()
    assert lib.wd_apply(None, None, None, 1, 0, None) == _lib.WD_BAD_ARG
    assert lib.gmresdr_solve(None, None, None, 20, 6, 1e-10, 100, None, None, None, None,
                             None) == _lib.WD_BAD_ARG
    assert lib.dbicgstab_solve(None, None, None, 1, None, None, 0, 1e-10, 10, None,
                               None) == _lib.WD_BAD_ARG
    lib.wd_destroy(None)
    lib.wd_deflation_destroy(None)


def test_stats_struct_layout():
    from paper_0710_1988_gb300._lib import WdStats
    # long long x2, int x5, (pad), double x3
    assert ctypes.sizeof(WdStats) == 8 * 2 + 4 * 5 + 4 + 8 * 3


def test_new_entry_points_reject_bad_arguments_without_a_gpu(lib):
    """The contraction, history, probe and setter entry points check their
    arguments before touching the device."""
    from paper_0710_1988_gb300 import _lib
    # wd_tsgemm: NULL pointers, bad sizes, bad mode, kv beyond the tensor-core limit
    assert lib.wd_tsgemm(None, 4, None, 8, 8, None, None, 0, 1.0, 100, 1, None) == _lib.WD_BAD_ARG
    p = ctypes.c_void_p(16)
    assert lib.wd_tsgemm(p, 0, p, 8, 8, None, p, 0, 1.0, 100, 1, None) == _lib.WD_BAD_ARG
    assert lib.wd_tsgemm(p, 4, p, 4, 8, None, p, 0, 1.0, 100, 1, None) == _lib.WD_BAD_ARG  # ldy < ncol
    assert lib.wd_tsgemm(p, 4, p, 8, 8, None, p, 0, 1.0, 100, 2, None) == _lib.WD_BAD_ARG
    assert lib.wd_tsgemm(p, 89, p, 8, 8, None, p, 0, 1.0, 100, 1, None) == _lib.WD_BAD_ARG
    assert "88" in _lib.last_error()
    assert lib.wd_tsgemm(p, 129, p, 8, 8, None, p, 0, 1.0, 100, 0, None) == _lib.WD_BAD_ARG
    assert lib.wd_tsgemm(p, 4, p, 8, 8, None, p, 1, 1.0, 100, 1, None) == _lib.WD_BAD_ARG  # IN NULL
    # gmresdr_history: NULL handle or negative length
    assert lib.gmresdr_history(None, None, 0) == -_lib.WD_BAD_ARG
    # wd_set_contraction: NULL handle
    assert lib.wd_set_contraction(None, 1) == _lib.WD_BAD_ARG
    # wd_set_eigen_estimates: NULL handle
    assert lib.wd_set_eigen_estimates(None, 1) == _lib.WD_BAD_ARG
    # probes: bad sizes
    out = ctypes.c_double()
    assert lib.wd_probe_fp64_peak(0, 1, ctypes.byref(out), None, None) == _lib.WD_BAD_ARG
    assert lib.wd_probe_bf16_mma_peak(1, 0, ctypes.byref(out), None, None) == _lib.WD_BAD_ARG
    assert lib.wd_probe_bf16_mma_peak(1, 1, None, None, None) == _lib.WD_BAD_ARG
