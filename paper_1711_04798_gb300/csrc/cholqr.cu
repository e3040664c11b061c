// Cholesky QR pieces of the precision-form projector step (FP64):
//   G = Y^H Y (a GEMM elsewhere), G = R^H R with pivots below tol * max
//   diagonal dropped (row of R set to zero), R^{-1} of the kept block, so that
//   Q = Y R^{-1} has orthonormal columns on the kept directions and zero
//   columns on the dropped ones (CholeskyQR, Yamamoto et al. 2015; applied
//   twice it is backward stable below condition 1e8).
#include "ctm_internal.h"

namespace {

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One CTA: right-looking Cholesky of the Hermitian n x n G (upper triangle
// used), in place in W (a copy), R written upper triangular (zero rows for
// dropped pivots).
__global__ void __launch_bounds__(1024) chol_drop_kernel(const cplx* __restrict__ G, cplx* __restrict__ W,
                                                         cplx* __restrict__ R, int n, double tol) {
  __shared__ double s_piv;
  __shared__ double s_max;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (long long e = tid; e < (long long)n * n; e += nt) {
    W[e] = G[e];
    R[e] = make_double2(0.0, 0.0);
  }
  __syncthreads();
  if (tid == 0) {
    double m = 0.0;
    for (int i = 0; i < n; ++i) m = fmax(m, W[(long long)i * n + i].x);
    s_max = m;
  }
  __syncthreads();
  const double thr = tol * s_max;
  for (int j = 0; j < n; ++j) {
    if (tid == 0) s_piv = W[(long long)j * n + j].x;
    __syncthreads();
    const double d = s_piv;
    if (!(d > thr)) {  // dropped direction: row j of R stays zero
      __syncthreads();
      continue;
    }
    const double rjj = sqrt(d), inv = 1.0 / rjj;
    // row j of R
    for (int l = j + tid; l < n; l += nt) {
      const cplx g = W[(long long)j * n + l];
      R[(long long)j * n + l] = make_double2(l == j ? rjj : g.x * inv, l == j ? 0.0 : g.y * inv);
    }
    __syncthreads();
    // trailing update of the upper triangle: W[i,l] -= conj(R[j,i]) R[j,l], j < i <= l
    const int m = n - j - 1;
    const long long cnt = (long long)m * m;
    for (long long e = tid; e < cnt; e += nt) {
      const int i = j + 1 + (int)(e / m), l = j + 1 + (int)(e % m);
      if (l < i) continue;
      const cplx a = R[(long long)j * n + i], b = R[(long long)j * n + l];
      cplx* w = W + (long long)i * n + l;
      // conj(a) * b
      w->x -= a.x * b.x + a.y * b.y;
      w->y -= a.x * b.y - a.y * b.x;
    }
    __syncthreads();
  }
}

// Rinv = inverse of the upper-triangular R on its kept block (zero rows and
// columns where R[i,i] == 0).  One warp per column c: back substitution
// R x = e_c, x_i for i = c .. 0, with x held in the warp's slice of shared
// memory (each step reads the entries the previous steps wrote) and written
// to Rinv at the end.
constexpr int TRI_WARPS = 4;
__global__ void tri_inv_kernel(const cplx* __restrict__ R, cplx* __restrict__ Rinv, int n) {
  extern __shared__ cplx xs_all[];  // [TRI_WARPS][n] solution columns, then [n] reciprocal diagonal
  double* rinv = (double*)(xs_all + (long long)TRI_WARPS * n);
  const int w = threadIdx.x >> 5;
  const int c = blockIdx.x * TRI_WARPS + w;
  const int lane = threadIdx.x & 31;
  // the diagonal's reciprocals once per block, off the substitution's serial chain
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double d = R[(long long)i * n + i].x;
    rinv[i] = d != 0.0 ? 1.0 / d : 0.0;
  }
  __syncthreads();
  if (c >= n) return;
  cplx* xs = xs_all + (long long)w * n;
  for (int i = lane; i < n; i += 32) xs[i] = make_double2(0.0, 0.0);
  __syncwarp();
  if (R[(long long)c * n + c].x != 0.0) {
    for (int i = c; i >= 0; --i) {
      const cplx* Ri = R + (long long)i * n;
      double sr = 0.0, si = 0.0;
      for (int j = i + 1 + lane; j <= c; j += 32) {
        const cplx a = Ri[j], x = xs[j];
        sr += a.x * x.x - a.y * x.y;
        si += a.x * x.y + a.y * x.x;
      }
      sr = warp_sum_d(sr);
      si = warp_sum_d(si);
      if (lane == 0) {
        const double ri = rinv[i];  // 0 for a dropped direction
        xs[i] = make_double2(((i == c ? 1.0 : 0.0) - sr) * ri, -si * ri);
      }
      __syncwarp();
    }
  }
  for (int i = lane; i < n; i += 32) Rinv[(long long)i * n + c] = xs[i];
}

// G += coef * tr(G) I (one CTA): the shift of shifted CholeskyQR (Fukaya,
// Kannan, Nakatsukasa, Yamamoto and Yanagisawa 2020), with the trace of the
// Gram (the squared Frobenius norm of Y) bounding the squared 2-norm.
__global__ void __launch_bounds__(256) gram_shift_kernel(cplx* __restrict__ G, int n, double coef) {
  __shared__ double s_part[8];
  double t = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) t += G[(long long)i * n + i].x;
  t = warp_sum_d(t);
  if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = t;
  __syncthreads();
  double tr = 0.0;
#pragma unroll
  for (int w = 0; w < 8; ++w) tr += s_part[w];
  const double shift = coef * tr;
  for (int i = threadIdx.x; i < n; i += blockDim.x) G[(long long)i * n + i].x += shift;
}

}  // namespace

cudaError_t gram_shift(cudaStream_t s, cplx* G, int n, double coef) {
  gram_shift_kernel<<<1, 256, 0, s>>>(G, n, coef);
  count_launch();
  return cudaGetLastError();
}

cudaError_t chol_drop(cudaStream_t s, const cplx* G, cplx* work, cplx* R, int n, double tol) {
  cudaError_t e;
  if ((e = kernels_init()) != cudaSuccess) return e;
  if (chol_cluster_fits(n)) return chol_cluster(s, G, R, n, tol);
  chol_drop_kernel<<<1, 1024, 0, s>>>(G, work, R, n, tol);
  count_launch();
  return cudaGetLastError();
}

cudaError_t tri_inv(cudaStream_t s, const cplx* R, cplx* Rinv, int n) {
  const size_t smem = (size_t)TRI_WARPS * n * sizeof(cplx) + (size_t)n * sizeof(double);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;  // n above about 3000
  static size_t attr = 48 * 1024;
  if (smem > attr) {
    cudaError_t e = cudaFuncSetAttribute(tri_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr = 200 * 1024;
  }
  tri_inv_kernel<<<(n + TRI_WARPS - 1) / TRI_WARPS, TRI_WARPS * 32, smem, s>>>(R, Rinv, n);
  count_launch();
  return cudaGetLastError();
}
