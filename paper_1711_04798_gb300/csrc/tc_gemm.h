// Tensor-core (tcgen05) complex GEMM of the precision form: TF32, split-BF16x3
// (hi*hi + hi*lo + lo*hi) or split-BF16x6 (three parts, the six products of
// combined order <= 2) with FP32 accumulation in TMEM.
#pragma once
#include <cuda.h>

#include "ctm_internal.h"

// C[M,N] = alpha * opA(A) opB(B) with complex FP64 storage of A, B, C; the
// operands are packed (permuted, converted, real-embedded) into `scratch`
// above scratch_top.  Returns cudaErrorNotSupported when the precision or the
// shape has no tensor-core kernel.  `timeouts` (device int, required) counts
// the bounded waits inside the kernel that ran out; the caller owns it and
// reads it after the stream has drained (each handle passes its own slot).
struct TcTuner;
struct TcChoice;

// Optional timing probe of one product (measurement support): events recorded
// on the launching stream before the main tensor-core kernel, after it, and
// after the split-K reduction; the call fills in the padded shape and tile
// choice it ran, so the caller can credit algorithmic flops and bytes.
struct TcProbe {
  cudaEvent_t ev[3];
  long long Mp, Nrp, Krp;  // padded real-embedded shape
  int splits, bn, parts, elem_bytes;
  bool packed_b;           // B came pre-packed (not repacked by this call)
};

// An operand read through a strided view instead of a permuted copy: element
// (r, c) is p[roff(r) + coff(c)], roff / coff sums of per-axis strides over
// up to four axes each (the last axis fastest), conjugated when conj.  For
// the A role rows are m and columns k; for the B role rows are n and columns
// k (the transpose of op(B)).
struct TcView {
  const cplx* p;
  int nr, nc;
  int rdim[4], cdim[4];
  long long rstr[4], cstr[4];
  int conj;
};
// force: a fixed tile choice instead of the tuner's or the default one
cudaError_t tc_zgemm(cudaStream_t s, int prec, int M, int N, int K, cplx alpha, const cplx* A,
                     long long lda, int opA, const cplx* B, long long ldb, int opB, cplx* C,
                     long long ldc, cplx* scratch, long long scratch_elems, long long scratch_top,
                     int* timeouts, TcTuner* tuner = nullptr, const TcChoice* force = nullptr,
                     TcProbe* probe = nullptr);

// A B-role operand (op(B) is K x N complex) packed once as Br^T (2N x 2K real,
// K-major, padded), reusable across products.
struct TcPacked {
  int prec;
  long long N, K;
  void* b0;  // TF32 values, or the leading BF16 part
  void* b1;  // second BF16 part (== b0 for TF32)
  void* b2;  // third BF16 part of BF16x6 (== b1 otherwise)
};
size_t tc_packed_bytes(int prec, int N, int K);
cudaError_t tc_pack_b(cudaStream_t s, int prec, const cplx* B, long long ldb, int opB, int N, int K, void* mem,
                      TcPacked* out);
// C = alpha opA(A) B  (or its complex conjugate when conj_out), B pre-packed
cudaError_t tc_zgemm_packed(cudaStream_t s, int prec, int M, cplx alpha, const cplx* A, long long lda, int opA,
                            const TcPacked& B, cplx* C, long long ldc, bool conj_out, cplx* scratch,
                            long long scratch_elems, long long scratch_top, int* timeouts,
                            TcTuner* tuner = nullptr, TcProbe* probe = nullptr);

// Tile choice of one product: output tile 128 x bn (bn = 128 or 256 real
// columns) and the number of K splits (FP32 partials summed in a fixed order).
struct TcChoice {
  int bn;
  int splits;
};

// Autotuner table (shape -> tile choice).  Products run through a tuner use
// its choice for their shape; while measuring, a shape not yet in the table is
// timed with every candidate choice (CUDA events, synchronising) and the
// fastest is recorded.  Without a tuner, or for unknown shapes when not
// measuring, the default heuristic applies.  Not thread-safe.
TcTuner* tc_tuner_create();
void tc_tuner_destroy(TcTuner* t);
void tc_tuner_set_measuring(TcTuner* t, bool on);
int tc_tuner_size(const TcTuner* t);
// entry i: fields = {prec, M, N, K, bn, splits}; us = {best time, default-choice time}
bool tc_tuner_entry(const TcTuner* t, int i, int fields[6], double us[2]);

// one-time setup (kernel attributes, driver entry point); called before any
// stream capture so that captured products make no such calls.
cudaError_t tc_init();

// C[M,N] = alpha A B with either operand given as a view (the other, when the
// view pointer is null, as (ptr, ld, op) like tc_zgemm): the operand packing
// gathers straight from the source tensor (a fused permute-and-pack).
cudaError_t tc_zgemm_views(cudaStream_t s, int prec, int M, int N, int K, cplx alpha, const TcView* va,
                           const cplx* A, long long lda, int opA, const TcView* vb, const cplx* B, long long ldb,
                           int opB, cplx* C, long long ldc, cplx* scratch, long long scratch_elems,
                           long long scratch_top, int* timeouts, TcTuner* tuner = nullptr,
                           TcProbe* probe = nullptr);

// 2D tensor map of a K-major BF16 operand [rows x kcols] with boxes of
// box_rows x 64 elements (128 bytes, 128-byte swizzle), for the tcgen05 kernels.
cudaError_t tc_encode_bf16_map(CUtensorMap* map, void* base, long long rows, long long kcols, int box_rows);

// FP64-accurate complex GEMM on the tensor cores (ozaki.cu): C = opA(A) opB(B)
// (complex FP64 storage, alpha 1, beta 0).  `work` (device, work_bytes) holds
// the digit planes, row scales and split partials: oz_work_bytes(M, N, K).
size_t oz_work_bytes(int M, int N, int K);
cudaError_t oz_zgemm(cudaStream_t s, int M, int N, int K, const cplx* A, long long lda, int opA, const cplx* B,
                     long long ldb, int opB, cplx* C, long long ldc, void* work, size_t work_bytes, int* timeouts);
