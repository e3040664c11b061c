// Tensor-core (tcgen05) complex GEMM of the precision form: TF32 or
// split-BF16 (hi*hi + hi*lo + lo*hi) with FP32 accumulation in TMEM.
#pragma once
#include "ctm_internal.h"

// C[M,N] = alpha * opA(A) opB(B) with complex FP64 storage of A, B, C; the
// operands are packed (permuted, converted, real-embedded) into `scratch`
// above scratch_top.  Returns cudaErrorNotSupported when the precision or the
// shape has no tensor-core kernel.
cudaError_t tc_zgemm(cudaStream_t s, int prec, int M, int N, int K, cplx alpha, const cplx* A,
                     long long lda, int opA, const cplx* B, long long ldb, int opB, cplx* C,
                     long long ldc, cplx* scratch, long long scratch_elems, long long scratch_top);

// number of bounded-wait timeouts inside tensor-core kernels since the last
// call (resets the counter); synchronous.
int tc_take_errors();
