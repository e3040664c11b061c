// Internal declarations shared by the CUDA translation units of the library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <string>
#include <vector>

typedef double2 cplx;  // (re, im), 16-byte aligned

// ---------------------------------------------------------------------------
// IEEE-754 binary64 <-> binary32 conversions and sign flips on the integer
// pipe.  GB300 issues FP64 instructions (conversions included) at a small
// fraction of its integer / FP32 rate, so data-movement kernels that touched
// every element with one became bound by the FP64 unit.
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
// binary64 -> binary32, mantissa truncated to 23 bits; |x| below 2^-126
// becomes a signed zero, beyond the binary32 range an infinity (NaN too).
__device__ __forceinline__ float d2f_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7FF) - 1023 + 127;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7F800000u);
  return __uint_as_float(sign | ((unsigned)e << 23) | (unsigned)((b >> 29) & 0x7FFFFFu));
}
// binary32 -> binary64, exact for normal numbers (subnormals become zero)
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned e = (u >> 23) & 0xFFu;
  const unsigned long long mant = (unsigned long long)(u & 0x7FFFFFu) << 29;
  if (e == 0) return __longlong_as_double((long long)sign);
  if (e == 255) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull | mant));
  return __longlong_as_double((long long)(sign | ((unsigned long long)(e - 127 + 1023) << 52) | mant));
}
__device__ __forceinline__ double neg_bits(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
}

// One complex Jacobi rotation of a row pair (a, b) (Hestenes; Demmel and
// Veselic 1992), with phi the phase of the inner product a^H b:
//   a' = c a - s e^{-i phi} b,   b' = s e^{i phi} a + c b
// (sq = s e^{-i phi}, sp = s e^{i phi}).  This form tends to the identity as
// s -> 0, so rows keep their phases through small rotations and a start that
// already diagonalises is left in place (a warm start stays a warm start).
__device__ __forceinline__ void jac_rotate(cplx& a, cplx& b, double c, cplx sq, cplx sp) {
  const cplx x = a, y = b;
  a = make_double2(c * x.x - (sq.x * y.x - sq.y * y.y), c * x.y - (sq.x * y.y + sq.y * y.x));
  b = make_double2(c * y.x + (sp.x * x.x - sp.y * x.y), c * y.y + (sp.x * x.y + sp.y * x.x));
}
#endif

// ---------------------------------------------------------------------------
// error plumbing: every launcher returns cudaError_t; the API layer converts.
// ---------------------------------------------------------------------------
struct DevStatus {
  // written by kernels that can run out of an iteration budget
  int jacobi_unconverged;  // number of Jacobi calls that hit the sweep budget
  int nonfinite;           // a NaN/Inf met in a norm
  int jacobi_sweeps;       // sweeps used by all Jacobi calls (accounting)
  int jacobi_calls;
  int tc_timeouts;         // bounded waits inside tensor-core GEMMs that ran out
  int barrier_timeouts;    // grid-barrier waits (small-row Jacobi) that ran out
};

// ---------------------------------------------------------------------------
// GEMM operand ops (row-major storage):
//   A op N: element (m,k) at A[m*lda + k];  op T: at A[k*lda + m]
//   B op N: element (k,n) at B[k*ldb + n];  op T: at B[n*ldb + k]
//   OP_C flag conjugates the element.
// ---------------------------------------------------------------------------
enum { OP_N = 0, OP_T = 1, OP_CONJ = 2, OP_C = OP_N | OP_CONJ, OP_H = OP_T | OP_CONJ };

struct GemmBatch {
  int count;
  long long sA, sB, sC;  // element strides between batch entries
};

// C[M,N] = alpha * opA(A) opB(B) + beta * C   (complex FP64, CUDA cores).  With a
// workspace, products with few output tiles split K (partials summed in order).
// flags: ZG_UPPER_TILES (M == N; tiles below the diagonal are not computed and,
// when K is split, returned as zero: for Hermitian results read by their upper
// triangle), ZG_A_LOWER (opA(A) is lower triangular: k-tiles beyond a tile
// row's diagonal are skipped).
enum { ZG_UPPER_TILES = 1, ZG_A_LOWER = 2 };
cudaError_t zgemm(cudaStream_t s, int M, int N, int K, cplx alpha, const cplx* A, long long lda,
                  int opA, const cplx* B, long long ldb, int opB, cplx beta, cplx* C,
                  long long ldc, GemmBatch batch = {1, 0, 0, 0}, cplx* work = nullptr,
                  long long work_elems = 0, int flags = 0);
// sigma[i] = ||row i|| of G (n rows of length m, stride ldg)
cudaError_t row_norms(cudaStream_t s, const cplx* G, int n, int m, long long ldg, double* sigma);

// out = alpha * (conj?) permute(in): out axis i is in axis perm[i].
cudaError_t permute(cudaStream_t s, const cplx* in, cplx* out, int nd, const int* in_dims,
                    const int* perm, bool conj, cplx alpha);

// ---------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------
cudaError_t double_layer(cudaStream_t s, const cplx* A, const cplx* B, cplx* a, int d, int D);
cudaError_t rotate_a(cudaStream_t s, const cplx* a, cplx* out, int D2);
// trace init of one environment tensor from a double-layer tensor (role 0..7)
cudaError_t trace_init_tensor(cudaStream_t s, const cplx* a, cplx* out, int role, int D, int chi);
// x *= 1/||x||_F (FP64 reduction); work holds >= 1024 doubles
cudaError_t normalize(cudaStream_t s, cplx* x, long long n, double* work, DevStatus* st);
cudaError_t fill_omega_t(cudaStream_t s, cplx* omt, int k, int K, uint64_t seed);
cudaError_t set_zero(cudaStream_t s, cplx* x, long long n);

// One-sided (Hestenes) Jacobi on the n rows of G (row length m, row stride ldg):
// rotates row pairs until mutually orthogonal; optional Vt (n x n) accumulates the
// same rotations starting from the identity.  sigma[i] = ||row i|| on return.
// counters: 4 ints of scratch (sweep counters and, for m <= 256, a grid barrier);
// work: 1 double of scratch.
// rotlog (optional, jacobi_log_elems(n, max_sweeps) complex slots): lets the
// cluster path rebuild Vt from logged rotations instead of holding it.
// wait_cycles: limit of each grid-barrier wait of the small-row kernel (<= 0:
// about 2 s of clock); a wait that runs out is counted in st->barrier_timeouts
// and its CTA stops.
// warm_v: Vt holds a unitary n x n start V0^T on entry (the rotations are
// accumulated onto it, Vt = J^T V0^T) instead of starting from the identity.
// dfloat: where the cluster path rebuilds Vt from the rotation log, hold,
// dot and rotate the rows in double-float arithmetic (about 48 bits; the
// rotations themselves and Vt stay FP64), for the precision form.
cudaError_t jacobi_rows(cudaStream_t s, cplx* G, int n, int m, long long ldg, cplx* Vt,
                        double* sigma, int max_sweeps, double* work, int* counters,
                        DevStatus* st, cplx* rotlog = nullptr, long long rotlog_elems = 0,
                        long long wait_cycles = 0, bool warm_v = false, bool dfloat = false);
// V (n x n) = identity
cudaError_t set_identity(cudaStream_t s, cplx* V, int n);
// rows of G scaled to unit norm where sigma > tol*max(sigma), zero otherwise
cudaError_t orth_rows_finish(cudaStream_t s, cplx* G, int n, int m, long long ldg,
                             const double* sigma, double tol);
// descending selection of the top chi of sigma[0..n) above cutoff*max:
// perm[0..chi) (or -1), s_sel[0..chi) (or 0)
cudaError_t select_top(cudaStream_t s, const double* sigma, int n, int chi, double cutoff,
                       int* perm, double* s_sel);
// out[a, :] = scale_a * in[perm[a], :] (row length m); scale_a = 1/sigma[perm[a]] if
// normalize_by_sigma, else 1; rows with perm[a] < 0 are zero.
cudaError_t gather_rows(cudaStream_t s, const cplx* in, long long ldi, cplx* out,
                        long long ldo, const int* perm, const double* sigma, int rows, int m,
                        bool normalize_by_sigma);
// rows a < chi of X scaled by s_sel[a]^(-1/2) (0 where s_sel == 0)
cudaError_t scale_rows_isqrt(cudaStream_t s, cplx* X, int rows, int m, long long ld,
                             const double* s_sel);
// out = sum_{ij} rho[i,j] * H[j,i]  (real part), accumulated with weight w into acc[idx]
cudaError_t trace_product(cudaStream_t s, const cplx* rho, const cplx* H, int n, double* acc,
                          int idx, double w);
cudaError_t trace_normalize(cudaStream_t s, cplx* rho, int n, double* work);

// Cholesky with dropped pivots (d <= tol * max diagonal) of the Hermitian n x n G:
// R upper triangular (dropped rows zero); work: n*n scratch.  One CTA.
cudaError_t chol_drop(cudaStream_t s, const cplx* G, cplx* work, cplx* R, int n, double tol);
// inverse of upper-triangular R on its kept block (zero where R[i,i] == 0)
cudaError_t tri_inv(cudaStream_t s, const cplx* R, cplx* Rinv, int n);
// G += coef * tr(G) * I for the Hermitian n x n Gram G (device): the diagonal
// shift of shifted CholeskyQR
cudaError_t gram_shift(cudaStream_t s, cplx* G, int n, double coef);

// ---------------------------------------------------------------------------
// Krylov readout of the boundary density operator (lanczos.cu)
// ---------------------------------------------------------------------------
struct LanczosResult {
  int iters;       // Lanczos steps taken (size of the tridiagonal)
  int converged;   // leading Ritz values with residual <= tol * largest
  int breakdown;   // an invariant subspace was reached (Ritz values exact)
  int indefinite;  // a negative B-norm met: B is not positive definite
};
// *out = sum conj(x) y over n entries (fixed order); partial: 512 double2
cudaError_t zdotc_dev(cudaStream_t s, const cplx* x, const cplx* y, long long n, double2* partial, double2* out);
// y = A x for a dense n x n row-major A; fp32_products: products on the FP32
// pipe, FP64 accumulation of groups of four (for precision-form operators)
cudaError_t zgemv_dense(cudaStream_t s, const cplx* A, long long n, const cplx* x, cplx* y, bool fp32_products);
// complex elements of work lanczos_leading needs
long long lanczos_work_elems(long long n, int max_iter);
// Leading k eigenvalues of M = A B (A, B Hermitian, B positive definite) by
// Lanczos in the B inner product with full reorthogonalisation; on return
// s_sel[0..k) holds the Ritz values, descending (device).  fp32_products:
// mat-vecs with FP32 products (operators built in the precision form).
cudaError_t lanczos_leading(cudaStream_t s, const cplx* A, const cplx* B, long long n, int k, int max_iter,
                            double tol, uint64_t seed, cplx* work, long long work_elems, double* s_sel,
                            bool fp32_products, LanczosResult* res);
// lam = theta / Re tr(A B) (k values) and out = {-sum lam ln lam, 1 - sum lam}
cudaError_t topk_finish(cudaStream_t s, const cplx* A, const cplx* B, long long n, const double* theta, int k,
                        double2* partial, double2* trd, double* lam, double* out);

// one-time queries of the kernels' launch limits; called before any stream capture
cudaError_t kernels_init();

// FP64 Jacobi / Cholesky on one thread-block cluster (cluster_fp64.cu): rows
// in distributed shared memory, hardware cluster barriers between steps.
cudaError_t fp64_cluster_init();
bool jacobi_cluster_fits(int n, int m, bool vt_in_smem);
// With rotlog (jacobi_log_elems(n, max_sweeps) complex slots) and sweeps_used
// (one int), Vt is not held in the cluster: the rotations are logged and
// replayed onto the identity (onto Vt itself with warm_v) by one CTA per
// column afterwards.
cudaError_t jacobi_cluster(cudaStream_t s, cplx* G, int n, int m, long long ldg, cplx* Vt, int max_sweeps,
                           DevStatus* st, cplx* rotlog, int* sweeps_used, bool warm_v = false,
                           bool dfloat = false);
long long jacobi_log_elems(int n, int max_sweeps);
bool chol_cluster_fits(int n);
cudaError_t chol_cluster(cudaStream_t s, const cplx* G, cplx* R, int n, double tol);

// launch accounting (host counter incremented by every launcher)
void count_launch(int n = 1);
uint64_t launch_counter();
