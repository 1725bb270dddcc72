"""The C-ABI library loads on a CPU-only host and exports what cdfns.h
declares; argument errors that need no device are reported as such."""
import ctypes
import os

import pytest

import paper_2506_06805_gb300 as P


def _lib_or_skip():
    if not os.path.exists(P.LIB_PATH):
        pytest.skip("libcdfns.so not built (run __graft_entry__.build())")
    return P.lib()


def test_header_symbols_are_exported():
    L = _lib_or_skip()
    names = P.header_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n


def test_null_arguments_rejected_without_device():
    L = _lib_or_skip()
    out = ctypes.c_void_p()
    assert L.cc_init(1, 1, 1, None, None, ctypes.byref(out)) == -1
    assert L.cc_ladder_dev(None, None, None) == -1
    assert L.cc_residual_dev(None, None, None, None, None) == -1
    assert L.ipeom_sigma_dev(None, 1, None, None) == -1
    assert L.ccsd_solve(None, 1e-8, 10, None, None) == -1
    assert L.cc_set_precision(None, 0) == -1
    assert L.cc_dump_integrals(None, 9, None) == -1
    assert L.cc_set_memory_limit(None, ctypes.c_size_t(1 << 30)) == -1
    assert L.cc_cholesky_dev(0, 1, None, 1e-6, 1, None, None, None) == -1
    assert L.ipeom_solve_lr(None, 1, 1e-7, 10, None, None, None, None, None) == -1
    assert L.ipeom_left_sigma_dev(None, 1, None, None) == -1


def test_allocator_pair_must_be_complete():
    L = _lib_or_skip()
    cb = P._ALLOC(lambda n, u: None)
    assert L.cc_set_default_allocator(cb, P._FREE(0), None) == -1
    assert L.cc_set_default_allocator(P._ALLOC(0), P._FREE(0), None) == 0
