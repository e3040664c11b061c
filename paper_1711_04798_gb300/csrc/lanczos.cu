// Krylov readout of the boundary density operator on long cylinders (Sec. IV).
//
// The spectrum of the half-cylinder density operator is that of
// M = sigma_L^T sigma_R (the identity after Eq. "rho").  For circumferences
// whose D^Nv is too large for a dense eigensolver only the leading eigenvalues
// are wanted; they come from a Lanczos iteration.  With A = sigma_L^T and
// B = sigma_R Hermitian and B positive definite, M = A B is self-adjoint in
// the inner product <x, y>_B = x^H B y:
//     <x, M y>_B = x^H B A B y = <M x, y>_B,
// so the three-term recurrence of Hermitian Lanczos applies with B-inner
// products.  Every Krylov vector v_j is stored with u_j = B v_j, so that one
// product with A and one with B per step suffice:
//     w = A u_j,  alpha_j = u_j^H w,  r = w - alpha_j v_j - beta_j v_{j-1},
//     r -= V (U^H r)  (twice: full reorthogonalisation in the B product),
//     s = B r,  beta_{j+1} = sqrt(r^H s),  v_{j+1} = r / beta,  u_{j+1} = s / beta.
// The Ritz values are the eigenvalues of the tridiagonal T(alpha, beta),
// found by bisection on Sturm counts; the residual of Ritz pair i is
// beta_m |y_i[m-1]| (Parlett, "The Symmetric Eigenvalue Problem", ch. 13),
// the last component from inverse iteration.
// Everything is FP64; A and B are dense row-major complex matrices.
#include "ctm_internal.h"

namespace {

constexpr int DOT_BLOCKS = 512;
constexpr int MAX_KRYLOV = 1024;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sum over a block of 256 threads, fixed order; result valid in thread 0
__device__ double block_sum_256(double v, double* sh) {
  v = warp_sum_d(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < 8; ++w) t += sh[w];
  __syncthreads();
  return t;
}

__device__ __forceinline__ double beta_of(double2 d) { return d.x > 0.0 ? sqrt(d.x) : 0.0; }

// y = A x, A dense n x n row-major: one warp per row, A streamed once (cache
// streaming loads), x re-read from L2; four loads in flight per lane.
__global__ void __launch_bounds__(256) zgemv_kernel(const cplx* __restrict__ A, long long n,
                                                    const cplx* __restrict__ x, cplx* __restrict__ y) {
  const long long row = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const cplx* a = A + row * n;
  double re0 = 0.0, im0 = 0.0, re1 = 0.0, im1 = 0.0;
  long long t = lane;
  for (; t + 96 < n; t += 128) {
    const cplx a0 = __ldcs(a + t), a1 = __ldcs(a + t + 32), a2 = __ldcs(a + t + 64), a3 = __ldcs(a + t + 96);
    const cplx x0 = x[t], x1 = x[t + 32], x2 = x[t + 64], x3 = x[t + 96];
    re0 += a0.x * x0.x - a0.y * x0.y;
    im0 += a0.x * x0.y + a0.y * x0.x;
    re1 += a1.x * x1.x - a1.y * x1.y;
    im1 += a1.x * x1.y + a1.y * x1.x;
    re0 += a2.x * x2.x - a2.y * x2.y;
    im0 += a2.x * x2.y + a2.y * x2.x;
    re1 += a3.x * x3.x - a3.y * x3.y;
    im1 += a3.x * x3.y + a3.y * x3.x;
  }
  for (; t < n; t += 32) {
    const cplx a0 = __ldcs(a + t), x0 = x[t];
    re0 += a0.x * x0.x - a0.y * x0.y;
    im0 += a0.x * x0.y + a0.y * x0.x;
  }
  const double re = warp_sum_d(re0 + re1), im = warp_sum_d(im0 + im1);
  if (lane == 0) y[row] = make_double2(re, im);
}

// y = A x as zgemv_kernel, with the products on the FP32 pipe: A is read as
// FP64 and narrowed on the integer pipe, x is narrowed once per element,
// four products are summed in FP32 and every such group is added in FP64.
// For operators built in the precision form (their entries carry ~1e-6
// relative error); GB300 issues FP64 too slowly for an HBM-rate mat-vec.
__global__ void __launch_bounds__(256) zgemv_mixed_kernel(const cplx* __restrict__ A, long long n,
                                                          const cplx* __restrict__ x, cplx* __restrict__ y) {
  const long long row = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const cplx* a = A + row * n;
  double re = 0.0, im = 0.0;
  long long t = lane;
  for (; t + 96 < n; t += 128) {
    const cplx a0 = __ldcs(a + t), a1 = __ldcs(a + t + 32), a2 = __ldcs(a + t + 64), a3 = __ldcs(a + t + 96);
    const cplx x0 = x[t], x1 = x[t + 32], x2 = x[t + 64], x3 = x[t + 96];
    float r = 0.f, i = 0.f;
    const float ar0 = d2f_bits(a0.x), ai0 = d2f_bits(a0.y), xr0 = d2f_bits(x0.x), xi0 = d2f_bits(x0.y);
    const float ar1 = d2f_bits(a1.x), ai1 = d2f_bits(a1.y), xr1 = d2f_bits(x1.x), xi1 = d2f_bits(x1.y);
    const float ar2 = d2f_bits(a2.x), ai2 = d2f_bits(a2.y), xr2 = d2f_bits(x2.x), xi2 = d2f_bits(x2.y);
    const float ar3 = d2f_bits(a3.x), ai3 = d2f_bits(a3.y), xr3 = d2f_bits(x3.x), xi3 = d2f_bits(x3.y);
    r = fmaf(ar0, xr0, r); r = fmaf(-ai0, xi0, r); i = fmaf(ar0, xi0, i); i = fmaf(ai0, xr0, i);
    r = fmaf(ar1, xr1, r); r = fmaf(-ai1, xi1, r); i = fmaf(ar1, xi1, i); i = fmaf(ai1, xr1, i);
    r = fmaf(ar2, xr2, r); r = fmaf(-ai2, xi2, r); i = fmaf(ar2, xi2, i); i = fmaf(ai2, xr2, i);
    r = fmaf(ar3, xr3, r); r = fmaf(-ai3, xi3, r); i = fmaf(ar3, xi3, i); i = fmaf(ai3, xr3, i);
    re += f2d_bits(r);
    im += f2d_bits(i);
  }
  for (; t < n; t += 32) {
    const cplx a0 = __ldcs(a + t), x0 = x[t];
    const float ar = d2f_bits(a0.x), ai = d2f_bits(a0.y), xr = d2f_bits(x0.x), xi = d2f_bits(x0.y);
    re += f2d_bits(fmaf(ar, xr, -ai * xi));
    im += f2d_bits(fmaf(ar, xi, ai * xr));
  }
  re = warp_sum_d(re);
  im = warp_sum_d(im);
  if (lane == 0) y[row] = make_double2(re, im);
}

// partial[b] = sum over block b's grid-stride slice of conj(x) y
__global__ void __launch_bounds__(256) zdotc_partial_kernel(const cplx* __restrict__ x, const cplx* __restrict__ y,
                                                            long long n, double2* __restrict__ partial) {
  __shared__ double sh[8];
  double re = 0.0, im = 0.0;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    const cplx a = x[i], b = y[i];
    re += a.x * b.x + a.y * b.y;
    im += a.x * b.y - a.y * b.x;
  }
  re = block_sum_256(re, sh);
  im = block_sum_256(im, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = make_double2(re, im);
}

// out = sum of the DOT_BLOCKS partials in a fixed order
__global__ void __launch_bounds__(256) zdotc_final_kernel(const double2* __restrict__ partial, double2* out) {
  __shared__ double sh[8];
  double re = 0.0, im = 0.0;
  for (int i = threadIdx.x; i < DOT_BLOCKS; i += 256) {
    re += partial[i].x;
    im += partial[i].y;
  }
  re = block_sum_256(re, sh);
  im = block_sum_256(im, sh);
  if (threadIdx.x == 0) *out = make_double2(re, im);
}

// r = w - alpha_j v_j - beta_j v_{j-1}
__global__ void lanczos_update_kernel(const cplx* __restrict__ w, const cplx* __restrict__ vj,
                                      const cplx* __restrict__ vjm1, const double2* __restrict__ adot,
                                      const double2* __restrict__ bdot, int j, long long n, cplx* __restrict__ r) {
  const double al = adot[j].x, be = j > 0 ? beta_of(bdot[j]) : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    cplx v = w[i];
    const cplx a = vj[i];
    v.x -= al * a.x;
    v.y -= al * a.y;
    if (j > 0) {
      const cplx b = vjm1[i];
      v.x -= be * b.x;
      v.y -= be * b.y;
    }
    r[i] = v;
  }
}

// c[i] = u_i^H r for the m stored vectors (one block per i)
__global__ void __launch_bounds__(256) proj_coeff_kernel(const cplx* __restrict__ U, long long n,
                                                         const cplx* __restrict__ r, cplx* __restrict__ c) {
  __shared__ double sh[8];
  const cplx* u = U + (long long)blockIdx.x * n;
  double re = 0.0, im = 0.0;
  for (long long t = threadIdx.x; t < n; t += 256) {
    const cplx a = u[t], b = r[t];
    re += a.x * b.x + a.y * b.y;
    im += a.x * b.y - a.y * b.x;
  }
  re = block_sum_256(re, sh);
  im = block_sum_256(im, sh);
  if (threadIdx.x == 0) c[blockIdx.x] = make_double2(re, im);
}

// r -= sum_{i<m} c[i] v_i
__global__ void __launch_bounds__(256) sub_proj_kernel(const cplx* __restrict__ V, long long n, int m,
                                                       const cplx* __restrict__ c, cplx* __restrict__ r) {
  __shared__ cplx cs[MAX_KRYLOV + 1];
  for (int i = threadIdx.x; i < m; i += blockDim.x) cs[i] = c[i];
  __syncthreads();
  for (long long t = blockIdx.x * 256LL + threadIdx.x; t < n; t += (long long)gridDim.x * 256) {
    double re = 0.0, im = 0.0;
    for (int i = 0; i < m; ++i) {
      const cplx v = V[(long long)i * n + t], a = cs[i];
      re += a.x * v.x - a.y * v.y;
      im += a.x * v.y + a.y * v.x;
    }
    cplx x = r[t];
    x.x -= re;
    x.y -= im;
    r[t] = x;
  }
}

// v = r / beta, u = s / beta with beta = sqrt(r^H s) (zero where beta == 0)
__global__ void scale_pair_kernel(const cplx* __restrict__ r, const cplx* __restrict__ s,
                                  const double2* __restrict__ bd, long long n, cplx* __restrict__ v,
                                  cplx* __restrict__ u) {
  const double be = beta_of(*bd);
  const double inv = be > 0.0 ? 1.0 / be : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const cplx a = r[i], b = s[i];
    v[i] = make_double2(a.x * inv, a.y * inv);
    u[i] = make_double2(b.x * inv, b.y * inv);
  }
}

// Leading k eigenvalues of the symmetric tridiagonal T (diagonal alpha_i =
// adot[i].x, off-diagonal beta_i = sqrt(bdot[i].x), i = 1..m-1) and the
// residual estimates beta_m |y_i[m-1]| of their Ritz pairs.  Block a finds the
// a-th largest eigenvalue by bisection on Sturm counts (the number of negative
// pivots of T - x I is the number of eigenvalues below x; Wilkinson, "The
// Algebraic Eigenvalue Problem", ch. 5), then the eigenvector's last
// component by inverse iteration with (T - theta I) factored without pivoting
// (a tiny shift guards exact singularity).  One lane per block computes.
__device__ int sturm_below(const double2* __restrict__ adot, const double2* __restrict__ bdot, int m, double x,
                           double pivmin) {
  int cnt = 0;
  double q = adot[0].x - x;
  if (fabs(q) < pivmin) q = -pivmin;
  cnt += q < 0.0;
  for (int i = 1; i < m; ++i) {
    const double b2 = bdot[i].x > 0.0 ? bdot[i].x : 0.0;
    q = (adot[i].x - x) - b2 / q;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += q < 0.0;
  }
  return cnt;
}

__global__ void tridiag_topk_kernel(const double2* __restrict__ adot, const double2* __restrict__ bdot, int m, int k,
                                    double* __restrict__ theta, double* __restrict__ resid, double* __restrict__ work) {
  const int a = blockIdx.x;
  if (threadIdx.x != 0 || a >= k) return;
  // Gershgorin interval
  double lo = 1e300, hi = -1e300, bmax = 0.0;
  for (int i = 0; i < m; ++i) {
    const double bl = i > 0 ? beta_of(bdot[i]) : 0.0, br = i + 1 < m ? beta_of(bdot[i + 1]) : 0.0;
    lo = fmin(lo, adot[i].x - bl - br);
    hi = fmax(hi, adot[i].x + bl + br);
    bmax = fmax(bmax, bl);
  }
  const double scale = fmax(fabs(lo), fabs(hi));
  const double pivmin = fmax(1e-300, 1e-30 * scale * scale) / fmax(scale, 1e-300);
  // the (m - 1 - a)-th smallest = the a-th largest
  const int target = m - a;  // eigenvalue with exactly target - 1 below it
  double l = lo, h = hi;
  for (int it = 0; it < 200 && h - l > 2.2e-16 * fmax(fabs(l), fabs(h)) + 1e-300; ++it) {
    const double mid = 0.5 * (l + h);
    if (sturm_below(adot, bdot, m, mid, pivmin) >= target) h = mid; else l = mid;
  }
  const double th = 0.5 * (l + h);
  theta[a] = th;
  // inverse iteration on (T - s I), s = th + tiny: y <- solve, normalise
  double* dd = work + (long long)a * 3 * m;  // pivots
  double* y = dd + m;
  double* lw = y + m;  // multipliers
  const double shift = th + 1e-14 * fmax(scale, 1e-300);
  for (int i = 0; i < m; ++i) y[i] = 1.0;
  double last = 0.0;
  for (int pass = 0; pass < 3; ++pass) {
    // LU of T - shift I without pivoting: d_0 = a_0 - s, l_i = b_i / d_{i-1}, d_i = a_i - s - l_i b_i
    double d = adot[0].x - shift;
    if (fabs(d) < pivmin) d = pivmin;
    dd[0] = d;
    for (int i = 1; i < m; ++i) {
      const double b = beta_of(bdot[i]);
      const double li = b / dd[i - 1];
      lw[i] = li;
      double di = (adot[i].x - shift) - li * b;
      if (fabs(di) < pivmin) di = pivmin;
      dd[i] = di;
    }
    // forward (L z = y), backward (U x = z), U = diag(d) + superdiag(b)
    for (int i = 1; i < m; ++i) y[i] -= lw[i] * y[i - 1];
    y[m - 1] /= dd[m - 1];
    for (int i = m - 2; i >= 0; --i) y[i] = (y[i] - beta_of(bdot[i + 1]) * y[i + 1]) / dd[i];
    double nrm = 0.0;
    for (int i = 0; i < m; ++i) nrm += y[i] * y[i];
    nrm = sqrt(nrm);
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    for (int i = 0; i < m; ++i) y[i] *= inv;
    last = y[m - 1];
  }
  resid[a] = beta_of(bdot[m]) * fabs(last);
}

// lam = theta / tr M (k values, descending); out = {S = -sum lam ln lam, 1 - sum lam}
__global__ void topk_finish_kernel(const double* __restrict__ theta, int k, const double2* __restrict__ trd,
                                   double* __restrict__ lam, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  const double tr = trd->x;
  double S = 0.0, sum = 0.0;
  for (int i = 0; i < k; ++i) {
    const double l = tr != 0.0 ? theta[i] / tr : 0.0;
    lam[i] = l;
    sum += l;
    if (l > 0.0) S -= l * log(l);
  }
  out[0] = S;
  out[1] = 1.0 - sum;
}

unsigned blocks_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

// sum conj(x) y over n entries into *out (device), fixed summation order
cudaError_t zdotc_dev(cudaStream_t s, const cplx* x, const cplx* y, long long n, double2* partial, double2* out) {
  zdotc_partial_kernel<<<DOT_BLOCKS, 256, 0, s>>>(x, y, n, partial);
  zdotc_final_kernel<<<1, 256, 0, s>>>(partial, out);
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t zgemv_dense(cudaStream_t s, const cplx* A, long long n, const cplx* x, cplx* y, bool fp32_products) {
  if (fp32_products)
    zgemv_mixed_kernel<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(A, n, x, y);
  else
    zgemv_kernel<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(A, n, x, y);
  count_launch();
  return cudaGetLastError();
}

long long lanczos_work_elems(long long n, int max_iter) {
  const long long M = max_iter;
  return 2 * (M + 1) * n + 3 * n + 2 * M * M + 5 * M + 8 + DOT_BLOCKS;
}

cudaError_t lanczos_leading(cudaStream_t s, const cplx* A, const cplx* B, long long n, int k, int max_iter,
                            double tol, uint64_t seed, cplx* work, long long work_elems, double* s_sel,
                            bool fp32_products, LanczosResult* res) {
  res->iters = 0;
  res->converged = 0;
  res->breakdown = 0;
  res->indefinite = 0;
  if (k < 1 || max_iter < k || max_iter > MAX_KRYLOV || max_iter > n) return cudaErrorInvalidValue;
  if (work_elems < lanczos_work_elems(n, max_iter)) return cudaErrorMemoryAllocation;
  const long long M = max_iter;
  cplx* V = work;
  cplx* U = V + (M + 1) * n;
  cplx* w = U + (M + 1) * n;
  cplx* r = w + n;
  cplx* sv = r + n;
  cplx* T = sv + n;  // 2 M^2 complex slots: work of the tridiagonal eigensolver
  cplx* c = T + 2 * M * M;
  double2* adot = (double2*)(c + M);
  double2* bdot = adot + M;
  double* resid = (double*)(bdot + M + 1);  // M doubles
  double2* partial = (double2*)(c + 5 * M + 8);  // past resid
  cudaError_t e;
  const unsigned gb = blocks_for(n);
  auto check = [&]() { return cudaGetLastError(); };

  // v0: uniform random entries (the range-finder generator), B-normalised
  if ((e = fill_omega_t(s, r, 1, (int)n, seed)) != cudaSuccess) return e;
  if ((e = zgemv_dense(s, B, n, r, sv, fp32_products)) != cudaSuccess) return e;
  if ((e = zdotc_dev(s, r, sv, n, partial, &bdot[0])) != cudaSuccess) return e;
  scale_pair_kernel<<<gb, 256, 0, s>>>(r, sv, &bdot[0], n, V, U);
  count_launch();
  if ((e = check()) != cudaSuccess) return e;

  double amax = 0.0;
  int m = 0;
  for (int j = 0; j < max_iter; ++j) {
    cplx* vj = V + (long long)j * n;
    cplx* uj = U + (long long)j * n;
    if ((e = zgemv_dense(s, A, n, uj, w, fp32_products)) != cudaSuccess) return e;
    if ((e = zdotc_dev(s, uj, w, n, partial, &adot[j])) != cudaSuccess) return e;
    lanczos_update_kernel<<<gb, 256, 0, s>>>(w, vj, j > 0 ? vj - n : vj, adot, bdot, j, n, r);
    count_launch();
    for (int pass = 0; pass < 2; ++pass) {
      proj_coeff_kernel<<<j + 1, 256, 0, s>>>(U, n, r, c);
      sub_proj_kernel<<<gb, 256, 0, s>>>(V, n, j + 1, c, r);
      count_launch(2);
    }
    if ((e = check()) != cudaSuccess) return e;
    if ((e = zgemv_dense(s, B, n, r, sv, fp32_products)) != cudaSuccess) return e;
    if ((e = zdotc_dev(s, r, sv, n, partial, &bdot[j + 1])) != cudaSuccess) return e;
    scale_pair_kernel<<<gb, 256, 0, s>>>(r, sv, &bdot[j + 1], n, V + (long long)(j + 1) * n,
                                         U + (long long)(j + 1) * n);
    count_launch();
    if ((e = check()) != cudaSuccess) return e;
    // host control: the new beta^2 and alpha decide breakdown and indefiniteness
    double2 hb[2];
    if ((e = cudaMemcpyAsync(&hb[0], &adot[j], sizeof(double2), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(&hb[1], &bdot[j + 1], sizeof(double2), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    amax = fmax(amax, fabs(hb[0].x));
    m = j + 1;
    const double b2 = hb[1].x;
    if (b2 < 0.0 && -b2 > 1e-20 * amax * amax) {  // r^H B r < 0: B is not positive definite
      res->indefinite = 1;
      break;
    }
    if (b2 <= 1e-26 * amax * amax) {  // invariant Krylov subspace: the Ritz values are exact
      res->breakdown = 1;
      break;
    }
    // Ritz check every 10 steps once k + 10 values exist (the end is handled below)
    if (m >= k + 10 && m % 10 == 0 && m < max_iter) {
      tridiag_topk_kernel<<<k, 32, 0, s>>>(adot, bdot, m, k, s_sel, resid, (double*)T);
      count_launch();
      if ((e = check()) != cudaSuccess) return e;
      double th0 = 0.0;
      std::vector<double> rs(k);
      if ((e = cudaMemcpyAsync(&th0, s_sel, sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
      if ((e = cudaMemcpyAsync(rs.data(), resid, k * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return e;
      if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
      int conv = 0;
      for (int a = 0; a < k; ++a) conv += rs[a] <= tol * th0;
      res->converged = conv;
      if (conv == k) break;
    }
  }
  res->iters = m;
  // final Ritz values from the last complete tridiagonal (m steps)
  if (m < k) {
    // fewer steps than requested values (breakdown): all m Ritz values are exact
    res->converged = m;
  }
  const int kk = m < k ? m : k;  // after an early breakdown only m Ritz values exist
  if (kk < k) {
    if ((e = cudaMemsetAsync(s_sel, 0, k * sizeof(double), s)) != cudaSuccess) return e;
  }
  tridiag_topk_kernel<<<kk, 32, 0, s>>>(adot, bdot, m, kk, s_sel, resid, (double*)T);
  count_launch();
  if ((e = check()) != cudaSuccess) return e;
  if (res->breakdown) {
    res->converged = kk;
  } else {
    if ((e = check()) != cudaSuccess) return e;
    double th0 = 0.0;
    std::vector<double> rs(k);
    if ((e = cudaMemcpyAsync(&th0, s_sel, sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(rs.data(), resid, k * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    int conv = 0;
    for (int a = 0; a < k; ++a) conv += rs[a] <= tol * th0;
    res->converged = conv;
  }
  return cudaSuccess;
}

// lam[0..k) = theta / Re tr(A B) and out = {S, 1 - sum lam}; tr(A B) = sum
// A_ij B_ji = sum conj(B_ij) A_ij for Hermitian B (one pass over both)
cudaError_t topk_finish(cudaStream_t s, const cplx* A, const cplx* B, long long n, const double* theta, int k,
                        double2* partial, double2* trd, double* lam, double* out) {
  cudaError_t e;
  if ((e = zdotc_dev(s, B, A, n * n, partial, trd)) != cudaSuccess) return e;
  topk_finish_kernel<<<1, 32, 0, s>>>(theta, k, trd, lam, out);
  count_launch();
  return cudaGetLastError();
}
