"""The allocation-free corner spectrum (ipeps_corner_spectrum_noalloc).

Some callers cannot call cudaMalloc -- their device memory belongs to another
allocator, or their loop must not take the device synchronisation that
cudaMalloc/cudaFree imply.  This entry point serves them: it computes one
corner's normalised singular values with all intermediates in a fixed device
array inside the library.  Here it is called through the C ABI on the corners
of a real environment and compared with ipeps_ctm_spectra, on two calls in a
row (the second call reuses the array the first one left behind).

This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import synth
from gpu_common import gpu_ctm

pytestmark = pytest.mark.gpu


def _lib():
    from paper_1711_04798_gb300 import load_library
    lib = load_library()
    f = lib.ipeps_corner_spectrum_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return lib, f


def test_noalloc_corner_spectrum_matches_spectra_twice():
    import torch
    lib, f = _lib()
    w = synth.workload("real", seed=11, chi=16)
    g = gpu_ctm(w["tensors"], w["pattern"], 16)
    g.sweep(2)
    s_ref = g.spectra()  # existing entry point, [4][Ly][Lx][chi]
    stream = torch.cuda.current_stream()
    # two calls in a row, on two different corners
    for (role, x, y) in [(0, 0, 0), (2, 1, 1)]:
        C = g.env(role, x, y)  # host copy of the corner
        Cd = torch.from_numpy(C.view(np.float64).copy()).cuda()
        sd = torch.full((16,), -1.0, dtype=torch.float64, device="cuda")
        st = f(Cd.data_ptr(), 16, sd.data_ptr(), stream.cuda_stream)
        assert st == 0, lib.ipeps_last_error()
        s = sd.cpu().numpy()
        ref = s_ref[role, y, x]
        assert np.max(np.abs(s - ref)) < 1e-10, (s, ref)
    # sizes beyond the fixed array are refused before any GPU work
    st = f(Cd.data_ptr(), 257, sd.data_ptr(), stream.cuda_stream)
    assert st == 1 and b"1..256" in lib.ipeps_last_error()
