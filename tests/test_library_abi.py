"""CPU-only checks of the C ABI: the library builds, loads, exports every
symbol declared in include/ipeps_ctm.h, and validates arguments before any
CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ipeps_ctm.h")).read()
    return sorted(set(re.findall(r"\b(ipeps_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1711_04798_gb300 import build
    path = build.LIB
    if not os.path.exists(path):
        build.build()
    from paper_1711_04798_gb300 import load_library
    return load_library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_argument_validation_without_gpu(lib):
    from paper_1711_04798_gb300.binding import Cell, Options
    cell = Cell()
    cell.Lx = cell.Ly = 2
    for i in range(4):
        cell.pattern[i] = i
    cell.n_tensors, cell.d, cell.D, cell.dtype = 4, 8, 4, 1
    ptrs = (ctypes.c_void_p * 4)(1, 1, 1, 1)
    cell.tensors = ctypes.cast(ptrs, ctypes.POINTER(ctypes.c_void_p))
    opt = Options()
    lib.ipeps_default_options(ctypes.byref(opt))
    assert opt.svd_cutoff == 0.0 and opt.rsvd_oversample == 16  # 0: chosen by precision
    opt.chi = 8  # < D^2 = 16
    n = ctypes.c_size_t()
    assert lib.ipeps_ctm_workspace_size(ctypes.byref(cell), ctypes.byref(opt), ctypes.byref(n)) == 1
    assert b"chi" in lib.ipeps_last_error()
    opt.chi = 64
    assert lib.ipeps_ctm_workspace_size(ctypes.byref(cell), ctypes.byref(opt), ctypes.byref(n)) == 0
    assert n.value > 64 * 16 * 64 * 16 * 16  # at least the four enlarged corners
    cell.pattern[3] = 7
    h = ctypes.c_void_p()
    assert lib.ipeps_ctm_create(ctypes.byref(cell), ctypes.byref(opt), ctypes.byref(h)) == 1
