"""The allocation-free corner spectrum (ipeps_corner_spectrum_noalloc).

Some callers cannot call cudaMalloc -- their device memory belongs to another
allocator with a fixed budget, or their loop must not take the device
synchronisation that cudaMalloc/cudaFree imply.  This entry point serves them:
it computes one corner's normalised singular values with all intermediates in
a fixed device array inside the library.  Here it is called through the C ABI
and compared with the oracle's corner spectra (LAPACK SVD divided by the
largest value) and with the existing entry point ipeps_ctm_spectra, on two
calls in a row each (the second call reuses the array the first one left
behind), at chi = 16 (the small-row cooperative Jacobi) and chi = 256 (the
largest chi the array holds; the cluster Jacobi).  The device memory in use
is the same before and after the calls.

This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
import synth
from gpu_common import gpu_ctm, oracle_options

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _lib():
    from paper_1711_04798_gb300 import load_library
    lib = load_library()
    f = lib.ipeps_corner_spectrum_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return lib, f


def _free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _call(f, lib, C, chi, stream):
    import torch
    Cd = torch.from_numpy(np.ascontiguousarray(C).view(np.float64).copy()).cuda()
    sd = torch.full((chi,), -1.0, dtype=torch.float64, device="cuda")
    free0, torch0 = _free_bytes(), torch.cuda.memory_allocated()
    st = f(Cd.data_ptr(), chi, sd.data_ptr(), stream.cuda_stream)
    assert st == 0, lib.ipeps_last_error()
    s = sd.cpu().numpy()
    return s, _free_bytes() - free0, torch.cuda.memory_allocated() - torch0


def test_noalloc_corner_spectrum_chi16_matches_oracle_and_spectra_twice():
    import torch
    lib, f = _lib()
    w = synth.workload("real", seed=11, chi=16)
    g = gpu_ctm(w["tensors"], w["pattern"], 16)
    g.sweep(2)
    s_api = g.spectra()  # existing entry point, [4][Ly][Lx][chi]
    st = O.make_state(w["tensors"], w["pattern"], w["D"], 16)
    for _ in range(2):
        st = O.sweep(st, oracle_options(16, w["D"]))
    s_ref = O.corner_spectra(st)
    stream = torch.cuda.current_stream()
    assert f(None, 16, None, stream.cuda_stream) == 1  # refused: null pointers
    # two calls in a row, on two different corners
    for n, (role, x, y) in enumerate([(0, 0, 0), (2, 1, 1)]):
        s, dfree, dtorch = _call(f, lib, g.env(role, x, y), 16, stream)
        assert np.max(np.abs(s - s_api[role, y, x])) < TOL, (s, s_api[role, y, x])
        mask = s_ref[role, y, x] > 1e-8
        assert np.max(np.abs(s - s_ref[role, y, x])[mask]) < TOL, (s, s_ref[role, y, x])
        if n:  # after the first call (which may load device code), nothing is allocated
            assert dfree == 0 and dtorch == 0, (dfree, dtorch)
    # sizes beyond the fixed array are refused before any GPU work
    z = torch.zeros(2, dtype=torch.float64, device="cuda")
    assert f(z.data_ptr(), 257, z.data_ptr(), stream.cuda_stream) == 1
    assert b"1..256" in lib.ipeps_last_error()
    g.close()


def test_noalloc_corner_spectrum_chi256_matches_oracle_twice():
    """chi = 256, the largest the fixed array holds: two random complex
    matrices (one with a decaying spectrum like a converged corner) against
    the oracle's corner spectra (LAPACK SVD, divided by the largest value)."""
    import torch
    lib, f = _lib()
    stream = torch.cuda.current_stream()
    chi = 256
    rng = np.random.default_rng(256)
    U, _ = np.linalg.qr(rng.standard_normal((chi, chi)) + 1j * rng.standard_normal((chi, chi)))
    V, _ = np.linalg.qr(rng.standard_normal((chi, chi)) + 1j * rng.standard_normal((chi, chi)))
    decaying = (U * np.exp(-np.arange(chi) / 20.0)) @ V.conj().T
    dense = rng.standard_normal((chi, chi)) + 1j * rng.standard_normal((chi, chi))
    for n, C in enumerate((dense, decaying)):
        st = O.CTMState(Lx=1, Ly=1, D=1, chi=chi, a=[[None]], C=[[[C]], [[C]], [[C]], [[C]]], T=[])
        s_ref = O.corner_spectra(st)[0, 0, 0]
        s, dfree, dtorch = _call(f, lib, C, chi, stream)
        mask = s_ref > 1e-8
        err = np.max(np.abs(s - s_ref)[mask])
        print(f"chi 256 call {n + 1}: max |s/s0 - oracle| {err:.2e}")
        assert err < TOL
        if n:
            assert dfree == 0 and dtorch == 0, (dfree, dtorch)
