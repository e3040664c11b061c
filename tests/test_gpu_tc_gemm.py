"""tcgen05 GEMM of the precision form (TF32, split-BF16 x3 and x6) against
numpy's complex128 product, through ipeps_zgemm, on ragged shapes that span
several tiles, the split-K path and every operand op.  The error bound is
relative to sum_k |A_ik| |B_kj| (the scale of each output element): 2^-10 for
TF32 inputs (two roundings to 11 bits), 2^-15 for the BF16 hi/lo split (each
input kept to about 16 bits) plus FP32 accumulation, 2^-17 for the three-part
BF16 split: its inputs carry 24 bits (the dropped products lie below 2^-22 of
each term), so the FP32 accumulation sets the error -- about sqrt(n) 2^-24
for a sum of n = 2K real terms in one K split (measured 2.2e-6 for K = 1500
without splits, 1e-7 to 5e-7 where K is split).

Precision code 4 is the FP64-accurate tensor-core product of the projector
step (exact base-256 digit splitting, digit-plane products summed exactly):
held to 1e-15 of the scale, and to the FP64 CUDA-core kernel (code 0)."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = {0: 1e-13, 1: 2.0 ** -10, 2: 2.0 ** -15, 3: 2.0 ** -17, 4: 1e-15}


def _zgemm(prec, A, opA, B, opB, M, N, K):
    from paper_1711_04798_gb300 import load_library
    lib = load_library()
    f = lib.ipeps_zgemm
    P = ctypes.POINTER(ctypes.c_double)
    f.argtypes = [ctypes.c_int] * 4 + [P, ctypes.c_int, P, ctypes.c_int, P]
    f.restype = ctypes.c_int
    C = np.zeros((M, N), dtype=np.complex128)
    A = np.ascontiguousarray(A)
    B = np.ascontiguousarray(B)
    st = f(prec, M, N, K, A.ctypes.data_as(P), opA, B.ctypes.data_as(P), opB, C.ctypes.data_as(P))
    assert st == 0, lib.ipeps_last_error()
    return C


def _op(X, op):
    if op & 1:
        X = X.T
    if op & 2:
        X = X.conj()
    return X


@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("shape", [(130, 77, 300), (1, 1000, 700), (116, 600, 2500), (300, 129, 33)])
@pytest.mark.parametrize("ops", [(0, 0), (1, 3), (2, 1), (3, 2)])
def test_tc_gemm_matches_complex128(prec, shape, ops):
    M, N, K = shape
    rng = np.random.default_rng(M * 7 + N + K + prec)
    opA, opB = ops
    Ast = rng.standard_normal((K, M) if opA & 1 else (M, K)) + 1j * rng.standard_normal((K, M) if opA & 1 else (M, K))
    Bst = rng.standard_normal((N, K) if opB & 1 else (K, N)) + 1j * rng.standard_normal((N, K) if opB & 1 else (K, N))
    C = _zgemm(prec, Ast, opA, Bst, opB, M, N, K)
    Aop, Bop = _op(Ast, opA), _op(Bst, opB)
    ref = Aop @ Bop
    scale = np.abs(Aop) @ np.abs(Bop)
    err = np.max(np.abs(C - ref) / scale)
    print(f"prec {prec} shape {shape} ops {ops}: max error / scale {err:.2e}")
    assert err < TOL[prec], err


def _zgemm_tile(prec, bn, splits, A, opA, B, opB, M, N, K):
    from paper_1711_04798_gb300 import load_library
    lib = load_library()
    f = lib.ipeps_zgemm_tile
    P = ctypes.POINTER(ctypes.c_double)
    f.argtypes = [ctypes.c_int] * 6 + [P, ctypes.c_int, P, ctypes.c_int, P]
    f.restype = ctypes.c_int
    C = np.zeros((M, N), dtype=np.complex128)
    st = f(prec, bn, splits, M, N, K, np.ascontiguousarray(A).ctypes.data_as(P), opA,
           np.ascontiguousarray(B).ctypes.data_as(P), opB, C.ctypes.data_as(P))
    assert st == 0, lib.ipeps_last_error()
    return C


@pytest.mark.parametrize("prec", [1, 2, 3])
@pytest.mark.parametrize("bn", [128, 256])
@pytest.mark.parametrize("splits", [1, 3, 8, 40])
def test_every_tile_choice_matches_complex128(prec, bn, splits):
    """Each (tile width, K split) the autotuner can pick gives the same product."""
    M, N, K = 200, 333, 1500
    rng = np.random.default_rng(bn + splits + 10 * prec)
    A = rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))
    B = rng.standard_normal((N, K)) + 1j * rng.standard_normal((N, K))  # op T
    C = _zgemm_tile(prec, bn, splits, A, 0, B, 1, M, N, K)
    ref = A @ B.T
    scale = np.abs(A) @ np.abs(B.T)
    assert np.max(np.abs(C - ref) / scale) < TOL[prec]


@pytest.mark.parametrize("shape,ops", [((116, 116, 2500), (2, 1)), ((116, 2500, 116), (1, 0)),
                                       ((116, 116, 116), (1, 1)), ((33, 77, 1000), (3, 2))])
def test_fp64_tensor_core_product_matches_the_fp64_kernel(shape, ops):
    """The projector step's shapes (a Hermitian Gram of k x K rows, a
    triangular apply, a k x k core product): the digit-split tensor-core
    product against the FP64 CUDA-core kernel and against numpy."""
    M, N, K = shape
    opA, opB = ops
    rng = np.random.default_rng(M + 3 * N + 7 * K)
    Ast = rng.standard_normal((K, M) if opA & 1 else (M, K)) + 1j * rng.standard_normal((K, M) if opA & 1 else (M, K))
    Bst = rng.standard_normal((N, K) if opB & 1 else (K, N)) + 1j * rng.standard_normal((N, K) if opB & 1 else (K, N))
    C4 = _zgemm(4, Ast, opA, Bst, opB, M, N, K)
    C0 = _zgemm(0, Ast, opA, Bst, opB, M, N, K)
    Aop, Bop = _op(Ast, opA), _op(Bst, opB)
    scale = np.abs(Aop) @ np.abs(Bop)
    e_ref = np.max(np.abs(C4 - Aop @ Bop) / scale)
    e_fp64 = np.max(np.abs(C4 - C0) / scale)
    print(f"shape {shape} ops {ops}: digit-split vs numpy {e_ref:.2e}, vs FP64 kernel {e_fp64:.2e}")
    assert e_ref < 1e-15 and e_fp64 < 1e-15


def test_fp64_tensor_core_wide_product():
    """The shape of the enlarged corner's dominant product at D = 5, chi = 100
    (chi^2 x D^4 x D^4 = 10^4 x 625 x 625): whole waves of 128 x 32 tiles
    without K splits, against numpy on every element, 1e-15 of the scale."""
    M, N, K = 10000, 625, 625
    rng = np.random.default_rng(11)
    A = rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))
    B = rng.standard_normal((K, N)) + 1j * rng.standard_normal((K, N))
    C4 = _zgemm(4, A, 0, B, 0, M, N, K)
    scale = np.abs(A) @ np.abs(B)
    e_ref = np.max(np.abs(C4 - A @ B) / scale)
    print(f"wide digit-split product vs numpy {e_ref:.2e}")
    assert e_ref < 1e-15
