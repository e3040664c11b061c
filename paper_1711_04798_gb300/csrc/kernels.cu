// Element-wise / reduction kernels of the CTM path: double layer (Fig. 3a),
// trace initialisation, Frobenius normalisation, the range-finder test
// matrix, and the one-sided Jacobi SVD used by the projectors.
#include <cooperative_groups.h>

#include "ctm_internal.h"

namespace cg = cooperative_groups;

namespace {

__device__ __forceinline__ cplx cmul(cplx a, cplx b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Block-wide sum of NV doubles; every thread gets the totals.  blockDim <= 1024.
template <int NV>
__device__ void block_sum(double (&v)[NV], double* sh /* >= 32*NV */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[q * 32 + warp] = v[q];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += sh[q * 32 + w];  // fixed order: deterministic
    v[q] = t;
  }
  __syncthreads();
}

// a[(u u'),(l l'),(d d'),(r r')] = sum_p A[p,u,l,d,r] conj(B[p,u',l',d',r'])
__global__ void double_layer_kernel(const cplx* __restrict__ A, const cplx* __restrict__ B,
                                    cplx* __restrict__ a, int d, int D) {
  const int D2 = D * D, D4 = D2 * D2;
  const long long total = (long long)D4 * D4;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    // output index (u,u',l,l',d,d',r,r') with the last fastest
    long long t = i;
    const int rp = t % D; t /= D;
    const int r = t % D; t /= D;
    const int dp = t % D; t /= D;
    const int dd = t % D; t /= D;
    const int lp = t % D; t /= D;
    const int l = t % D; t /= D;
    const int up = t % D; t /= D;
    const int u = (int)t;
    const long long ik = (((long long)u * D + l) * D + dd) * D + r;
    const long long ib = (((long long)up * D + lp) * D + dp) * D + rp;
    double sr = 0.0, si = 0.0;
    for (int p = 0; p < d; ++p) {
      const cplx x = A[(long long)p * D4 + ik];
      const cplx y = B[(long long)p * D4 + ib];
      sr += x.x * y.x + x.y * y.y;
      si += x.y * y.x - x.x * y.y;
    }
    a[i] = make_double2(sr, si);
  }
}

// One environment tensor of the trace initialisation, padded to chi.
// role 0..3 = C1..C4, 4..7 = T1..T4 (leg orders as in the public header).
__global__ void trace_init_kernel(const cplx* __restrict__ a, cplx* __restrict__ out, int role,
                                  int D, int chi) {
  const int D2 = D * D;
  const bool isC = role < 4;
  const long long total = isC ? (long long)chi * chi : (long long)chi * D2 * chi;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int i0, i1, i2 = 0;
    if (isC) {
      i0 = (int)(i / chi);
      i1 = (int)(i % chi);
    } else {
      i0 = (int)(i / ((long long)D2 * chi));
      i1 = (int)((i / chi) % D2);
      i2 = (int)(i % chi);
    }
    cplx v = make_double2(0.0, 0.0);
    // chi-legs beyond D^2 are padding
    bool pad;
    if (isC) pad = (i0 >= D2) || (i1 >= D2);
    else pad = (i0 >= D2) || (i2 >= D2);
    if (!pad) {
      // a index (u, l, d, r), each in [0, D2); diagonal legs summed over t in [0, D)
      double sr = 0.0, si = 0.0;
      if (isC) {
        for (int t1 = 0; t1 < D; ++t1)
          for (int t2 = 0; t2 < D; ++t2) {
            const int g1 = t1 * D + t1, g2 = t2 * D + t2;
            int u, l, dd, r;
            switch (role) {
              case 0: u = g1; l = g2; dd = i0; r = i1; break;   // C1[d,r]: u,l traced
              case 1: u = g1; r = g2; l = i0; dd = i1; break;   // C2[l,d]: u,r traced
              case 2: dd = g1; r = g2; u = i0; l = i1; break;   // C3[u,l]: d,r traced
              default: l = g1; dd = g2; r = i0; u = i1; break;  // C4[r,u]: l,d traced
            }
            const cplx x = a[(((long long)u * D2 + l) * D2 + dd) * D2 + r];
            sr += x.x;
            si += x.y;
          }
      } else {
        for (int t1 = 0; t1 < D; ++t1) {
          const int g = t1 * D + t1;
          int u, l, dd, r;
          switch (role) {
            case 4: u = g; l = i0; dd = i1; r = i2; break;    // T1[l,d,r]: u traced
            case 5: r = g; u = i0; l = i1; dd = i2; break;    // T2[u,l,d]: r traced
            case 6: dd = g; r = i0; u = i1; l = i2; break;    // T3[r,u,l]: d traced
            default: l = g; dd = i0; r = i1; u = i2; break;   // T4[d,r,u]: l traced
          }
          const cplx x = a[(((long long)u * D2 + l) * D2 + dd) * D2 + r];
          sr += x.x;
          si += x.y;
        }
      }
      v = make_double2(sr, si);
    }
    out[i] = v;
  }
}

constexpr int NORM_BLOCKS = 256;

__global__ void sumsq_kernel(const cplx* __restrict__ x, long long n, double* partial) {
  __shared__ double sh[32];
  double v[1] = {0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    v[0] += x[i].x * x[i].x + x[i].y * x[i].y;
  block_sum<1>(v, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = v[0];
}

__global__ void scale_by_inv_norm_kernel(cplx* __restrict__ x, long long n,
                                         const double* partial, DevStatus* st) {
  __shared__ double sh[32];
  double v[1] = {0.0};
  for (int i = threadIdx.x; i < NORM_BLOCKS; i += blockDim.x) v[0] += partial[i];
  block_sum<1>(v, sh);
  const double nrm = sqrt(v[0]);
  if (!(nrm > 0.0) || !isfinite(nrm)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&st->nonfinite, 1);
    return;
  }
  const double s = 1.0 / nrm;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    x[i].x *= s;
    x[i].y *= s;
  }
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t n) {
  uint64_t z = seed + (n + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// omt[j*K + i] = Omega[i, j]; Omega entries (2u-1) + i (2u'-1) with u, u' the
// uniform53 draws of counters 2c, 2c+1, c = i*k + j.
__global__ void omega_kernel(cplx* __restrict__ omt, int k, int K, uint64_t seed) {
  const long long total = (long long)k * K;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long j = e / K, i = e % K;
    const uint64_t c = (uint64_t)(i * k + j);
    const double u1 = (double)(splitmix64(seed, 2 * c) >> 11) * 0x1.0p-53;
    const double u2 = (double)(splitmix64(seed, 2 * c + 1) >> 11) * 0x1.0p-53;
    omt[e] = make_double2(2.0 * u1 - 1.0, 2.0 * u2 - 1.0);
  }
}

__global__ void zero_kernel(cplx* x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = make_double2(0.0, 0.0);
}

// ---------------------------------------------------------------------------
// One-sided Jacobi (Hestenes 1958) on row vectors, parallel round-robin
// ordering; one CTA per row pair, grid-wide barrier between rounds.
// ---------------------------------------------------------------------------
constexpr int JAC_THREADS = 256;

__global__ void __launch_bounds__(JAC_THREADS)
    jacobi_rows_kernel(cplx* __restrict__ G, int n, int m, long long ldg, cplx* __restrict__ Vt,
                       int max_sweeps, double tol, int* counters, double* fro2, DevStatus* st) {
  cg::grid_group grid = cg::this_grid();
  __shared__ double sh[32 * 4];
  // squared Frobenius norm of G: rows below 1e-15 ||G||_F are rounding noise
  // and take part in no rotation (otherwise noise rows, re-contaminated by
  // every rotation of the others, never test orthogonal).
  {
    double v[1] = {0.0};
    for (int i = blockIdx.x; i < n; i += gridDim.x)
      for (int t = threadIdx.x; t < m; t += blockDim.x) {
        const cplx x = G[(long long)i * ldg + t];
        v[0] += x.x * x.x + x.y * x.y;
      }
    block_sum<1>(v, sh);
    if (threadIdx.x == 0) atomicAdd(fro2, v[0]);
  }
  grid.sync();
  const double negligible = *((volatile double*)fro2) * 1e-30;
  const int np = (n + 1) & ~1;  // even number of players (last may be a dummy)
  const int rounds = np - 1, npairs = np / 2;
  bool converged = false;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    for (int r = 0; r < rounds; ++r) {
      for (int p = blockIdx.x; p < npairs; p += gridDim.x) {
        int i, j;
        if (p == 0) {
          i = np - 1;
          j = r;
        } else {
          i = (r + p) % rounds;
          j = (r - p + rounds) % rounds;
        }
        if (i > j) { const int t = i; i = j; j = t; }
        if (j >= n) continue;  // pair with the dummy player
        cplx* gi = G + (long long)i * ldg;
        cplx* gj = G + (long long)j * ldg;
        double v[4] = {0.0, 0.0, 0.0, 0.0};  // alpha, beta, Re gamma, Im gamma
        for (int t = threadIdx.x; t < m; t += blockDim.x) {
          const cplx x = gi[t], y = gj[t];
          v[0] += x.x * x.x + x.y * x.y;
          v[1] += y.x * y.x + y.y * y.y;
          v[2] += x.x * y.x + x.y * y.y;  // conj(x) * y
          v[3] += x.x * y.y - x.y * y.x;
        }
        block_sum<4>(v, sh);
        const double al = v[0], be = v[1];
        const double g = hypot(v[2], v[3]);
        if (al > negligible && be > negligible && g > tol * sqrt(al * be)) {
          const double zeta = (be - al) / (2.0 * g);
          const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
          const cplx ph = make_double2(v[2] / g, -v[3] / g);  // exp(-i phi)
          const cplx sq = make_double2(s * ph.x, s * ph.y), sp = make_double2(s * ph.x, -s * ph.y);
          for (int q = threadIdx.x; q < m; q += blockDim.x) jac_rotate(gi[q], gj[q], c, sq, sp);
          if (Vt) {
            cplx* vi = Vt + (long long)i * n;
            cplx* vj = Vt + (long long)j * n;
            for (int q = threadIdx.x; q < n; q += blockDim.x) jac_rotate(vi[q], vj[q], c, sq, sp);
          }
          if (threadIdx.x == 0) atomicAdd(&counters[sweep & 1], 1);
        }
        __syncthreads();
      }
      grid.sync();
    }
    const int cnt = *((volatile int*)&counters[sweep & 1]);
    if (blockIdx.x == 0 && threadIdx.x == 0) counters[(sweep + 1) & 1] = 0;
    grid.sync();
    if (cnt == 0) {
      converged = true;
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&st->jacobi_sweeps, sweep + 1);
      break;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    atomicAdd(&st->jacobi_calls, 1);
    if (!converged) {
      atomicAdd(&st->jacobi_unconverged, 1);
      atomicAdd(&st->jacobi_sweeps, max_sweeps);
    }
  }
}


// ---------------------------------------------------------------------------
// One-sided Jacobi for short rows (m <= 256): one warp per row pair, one pair
// per CTA, warp-shuffle reductions only, and a light generation barrier
// between rounds (bounded spin; all CTAs are co-resident by cooperative launch).
// ---------------------------------------------------------------------------
constexpr long long BARRIER_WAIT_CYCLES = 4000000000LL;  // default limit: ~2 s at 2 GHz

__device__ __forceinline__ bool grid_barrier(unsigned* count, volatile unsigned* gen, unsigned nblocks,
                                             unsigned& my_gen, long long limit) {
  __syncwarp();
  bool ok = true;
  if ((threadIdx.x & 31) == 0) {
    __threadfence();
    const unsigned g0 = my_gen;
    if (atomicAdd(count, 1u) == nblocks - 1) {
      *count = 0;
      __threadfence();
      atomicExch((unsigned*)gen, g0 + 1);
    } else {
      const long long t0 = clock64();
      while (*gen == g0) {
        if (clock64() - t0 > limit) { ok = false; break; }
      }
    }
    __threadfence();
  }
  my_gen += 1;
  ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
  __syncwarp();
  return ok;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(32)
    jacobi_small_kernel(cplx* __restrict__ G, int n, int m, long long ldg, cplx* __restrict__ Vt,
                        int max_sweeps, double tol, int* counters, double* fro2, unsigned* bar,
                        DevStatus* st, long long wait_limit) {
  const int lane = threadIdx.x;
  unsigned my_gen = 0;
  const unsigned nb = gridDim.x;
  bool alive = true;
  {
    double v = 0.0;
    for (int i = blockIdx.x; i < n; i += gridDim.x)
      for (int t = lane; t < m; t += 32) {
        const cplx x = G[(long long)i * ldg + t];
        v += x.x * x.x + x.y * x.y;
      }
    v = warp_sum(v);
    if (lane == 0) atomicAdd(fro2, v);
  }
  alive = grid_barrier(bar, bar + 1, nb, my_gen, wait_limit);
  const double negligible = *((volatile double*)fro2) * 1e-30;
  const int np = (n + 1) & ~1;
  const int rounds = np - 1, npairs = np / 2;
  bool converged = false;
  int sweep = 0;
  for (; sweep < max_sweeps && alive; ++sweep) {
    for (int r = 0; r < rounds && alive; ++r) {
      for (int p = blockIdx.x; p < npairs; p += gridDim.x) {
        int i, j;
        if (p == 0) {
          i = np - 1;
          j = r;
        } else {
          i = (r + p) % rounds;
          j = (r - p + rounds) % rounds;
        }
        if (i > j) { const int t = i; i = j; j = t; }
        if (j >= n) continue;
        cplx* gi = G + (long long)i * ldg;
        cplx* gj = G + (long long)j * ldg;
        double al = 0.0, be = 0.0, gr = 0.0, gim = 0.0;
        for (int t = lane; t < m; t += 32) {
          const cplx x = gi[t], y = gj[t];
          al += x.x * x.x + x.y * x.y;
          be += y.x * y.x + y.y * y.y;
          gr += x.x * y.x + x.y * y.y;
          gim += x.x * y.y - x.y * y.x;
        }
        al = warp_sum(al);
        be = warp_sum(be);
        gr = warp_sum(gr);
        gim = warp_sum(gim);
        const double g = hypot(gr, gim);
        if (al > negligible && be > negligible && g > tol * sqrt(al * be)) {
          const double zeta = (be - al) / (2.0 * g);
          const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
          const cplx ph = make_double2(gr / g, -gim / g);  // exp(-i phi)
          const cplx sq = make_double2(s * ph.x, s * ph.y), sp = make_double2(s * ph.x, -s * ph.y);
          for (int q = lane; q < m; q += 32) jac_rotate(gi[q], gj[q], c, sq, sp);
          if (Vt) {
            cplx* vi = Vt + (long long)i * n;
            cplx* vj = Vt + (long long)j * n;
            for (int q = lane; q < n; q += 32) jac_rotate(vi[q], vj[q], c, sq, sp);
          }
          if (lane == 0) atomicAdd(&counters[sweep & 1], 1);
        }
      }
      alive = grid_barrier(bar, bar + 1, nb, my_gen, wait_limit);
    }
    if (!alive) break;
    const int cnt = *((volatile int*)&counters[sweep & 1]);
    if (blockIdx.x == 0 && lane == 0) counters[(sweep + 1) & 1] = 0;
    alive = grid_barrier(bar, bar + 1, nb, my_gen, wait_limit);
    if (cnt == 0) {
      converged = true;
      break;
    }
  }
  if (!alive && lane == 0) atomicAdd(&st->barrier_timeouts, 1);  // this CTA gave up waiting
  if (blockIdx.x == 0 && lane == 0) {
    atomicAdd(&st->jacobi_calls, 1);
    atomicAdd(&st->jacobi_sweeps, converged ? sweep + 1 : max_sweeps);
    if (!converged && alive) atomicAdd(&st->jacobi_unconverged, 1);
  }
}

__global__ void row_norms_kernel(const cplx* __restrict__ G, int n, int m, long long ldg,
                                 double* sigma) {
  __shared__ double sh[32];
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    double v[1] = {0.0};
    const cplx* g = G + (long long)i * ldg;
    for (int t = threadIdx.x; t < m; t += blockDim.x) v[0] += g[t].x * g[t].x + g[t].y * g[t].y;
    block_sum<1>(v, sh);
    if (threadIdx.x == 0) sigma[i] = sqrt(v[0]);
  }
}

__global__ void init_identity_kernel(cplx* V, int n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * n;
       e += (long long)gridDim.x * blockDim.x)
    V[e] = make_double2((e / n) == (e % n) ? 1.0 : 0.0, 0.0);
}

__device__ double block_max(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < nw; ++w) t = fmax(t, sh[w]);
  __syncthreads();
  return t;
}

__global__ void orth_finish_kernel(cplx* __restrict__ G, int n, int m, long long ldg,
                                   const double* __restrict__ sigma, double tol) {
  __shared__ double sh[32];
  double mx = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, sigma[i]);
  mx = block_max(mx, sh);
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const double s = sigma[i];
    const double f = (mx > 0.0 && s > tol * mx) ? 1.0 / s : 0.0;
    cplx* g = G + (long long)i * ldg;
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
      g[t].x *= f;
      g[t].y *= f;
    }
  }
}

__global__ void select_top_kernel(const double* __restrict__ sigma, int n, int chi,
                                  double cutoff, int* perm, double* s_sel) {
  __shared__ double sh[32];
  __shared__ int cnt_sh;
  double mx = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, sigma[i]);
  mx = block_max(mx, sh);
  if (threadIdx.x == 0) cnt_sh = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (mx > 0.0 && sigma[i] > cutoff * mx) atomicAdd(&cnt_sh, 1);
  __syncthreads();
  const int keep = min(chi, cnt_sh);
  for (int a = threadIdx.x; a < chi; a += blockDim.x) {
    perm[a] = -1;
    s_sel[a] = 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double si = sigma[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double sj = sigma[j];
      rank += (sj > si) || (sj == si && j < i);
    }
    if (rank < keep) {
      perm[rank] = i;
      s_sel[rank] = si;
    }
  }
}

__global__ void gather_rows_kernel(const cplx* __restrict__ in, long long ldi,
                                   cplx* __restrict__ out, long long ldo,
                                   const int* __restrict__ perm, const double* __restrict__ sigma,
                                   int rows, int m, int norm) {
  for (int a = blockIdx.x; a < rows; a += gridDim.x) {
    const int src = perm[a];
    double f = 0.0;
    if (src >= 0) f = norm ? 1.0 / sigma[src] : 1.0;
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
      cplx v = make_double2(0.0, 0.0);
      if (src >= 0) {
        v = in[(long long)src * ldi + t];
        v.x *= f;
        v.y *= f;
      }
      out[(long long)a * ldo + t] = v;
    }
  }
}

__global__ void scale_rows_isqrt_kernel(cplx* __restrict__ X, int rows, int m, long long ld,
                                        const double* __restrict__ s_sel) {
  for (int a = blockIdx.x; a < rows; a += gridDim.x) {
    const double s = s_sel[a];
    const double f = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
      X[(long long)a * ld + t].x *= f;
      X[(long long)a * ld + t].y *= f;
    }
  }
}

// acc[idx] += w * Re sum_{ij} rho[i,j] H[j,i]
__global__ void trace_product_kernel(const cplx* __restrict__ rho, const cplx* __restrict__ H,
                                     int n, double* acc, int idx, double w) {
  __shared__ double sh[32];
  double v[1] = {0.0};
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    const cplx x = rho[e], y = H[(long long)j * n + i];
    v[0] += x.x * y.x - x.y * y.y;
  }
  block_sum<1>(v, sh);
  if (threadIdx.x == 0) acc[idx] += w * v[0];
}

__global__ void trace_normalize_kernel(cplx* rho, int n) {
  __shared__ double sh[64];
  double v[2] = {0.0, 0.0};
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    v[0] += rho[(long long)i * n + i].x;
    v[1] += rho[(long long)i * n + i].y;
  }
  block_sum<2>(v, sh);
  const double den = v[0] * v[0] + v[1] * v[1];
  const cplx inv = make_double2(v[0] / den, -v[1] / den);
  for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) rho[e] = cmul(rho[e], inv);
}

unsigned grid_for(long long n, int threads = 256) {
  long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 152 * 16) b = 152 * 16;
  return (unsigned)b;
}

}  // namespace

cudaError_t double_layer(cudaStream_t s, const cplx* A, const cplx* B, cplx* a, int d, int D) {
  const long long n = (long long)D * D * D * D * D * D * D * D;
  double_layer_kernel<<<grid_for(n), 256, 0, s>>>(A, B, a, d, D);
  count_launch();
  return cudaGetLastError();
}

cudaError_t rotate_a(cudaStream_t s, const cplx* a, cplx* out, int D2) {
  const int dims[4] = {D2, D2, D2, D2};
  const int perm[4] = {3, 0, 1, 2};
  return permute(s, a, out, 4, dims, perm, false, make_double2(1.0, 0.0));
}

cudaError_t trace_init_tensor(cudaStream_t s, const cplx* a, cplx* out, int role, int D, int chi) {
  const long long n = role < 4 ? (long long)chi * chi : (long long)chi * D * D * chi;
  trace_init_kernel<<<grid_for(n), 256, 0, s>>>(a, out, role, D, chi);
  count_launch();
  return cudaGetLastError();
}

cudaError_t normalize(cudaStream_t s, cplx* x, long long n, double* work, DevStatus* st) {
  sumsq_kernel<<<NORM_BLOCKS, 256, 0, s>>>(x, n, work);
  scale_by_inv_norm_kernel<<<grid_for(n), 256, 0, s>>>(x, n, work, st);
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t fill_omega_t(cudaStream_t s, cplx* omt, int k, int K, uint64_t seed) {
  omega_kernel<<<grid_for((long long)k * K), 256, 0, s>>>(omt, k, K, seed);
  count_launch();
  return cudaGetLastError();
}

cudaError_t set_zero(cudaStream_t s, cplx* x, long long n) {
  zero_kernel<<<grid_for(n), 256, 0, s>>>(x, n);
  count_launch();
  return cudaGetLastError();
}

// co-resident CTA limits of the cooperative Jacobi kernels (queried once)
static int max_small = 0, max_coresident = 0;

cudaError_t kernels_init() {
  if (max_small > 0 && max_coresident > 0) return cudaSuccess;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_small_kernel, 32, 0)) != cudaSuccess)
    return e;
  max_small = sms * (per_sm > 0 ? per_sm : 1);
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_rows_kernel, JAC_THREADS, 0)) !=
      cudaSuccess)
    return e;
  max_coresident = sms * (per_sm > 0 ? per_sm : 1);
  return fp64_cluster_init();
}

cudaError_t jacobi_rows(cudaStream_t s, cplx* G, int n, int m, long long ldg, cplx* Vt,
                        double* sigma, int max_sweeps, double* work, int* counters,
                        DevStatus* st, cplx* rotlog, long long rotlog_elems, long long wait_cycles, bool warm_v,
                        bool dfloat) {
  if (n <= 0) return cudaSuccess;
  cudaError_t e;
  if ((e = kernels_init()) != cudaSuccess) return e;
  const bool logged = Vt && rotlog && n <= 2048 && rotlog_elems >= jacobi_log_elems(n, max_sweeps);
  if (jacobi_cluster_fits(n, m, Vt != nullptr && !logged)) {
    // rows (and Vt unless logged) fit in one cluster's shared memory: no grid-wide barrier
    if ((e = jacobi_cluster(s, G, n, m, ldg, Vt, max_sweeps, st, logged ? rotlog : nullptr,
                            logged ? counters : nullptr, warm_v, dfloat)) != cudaSuccess)
      return e;
    row_norms_kernel<<<n < 1024 ? n : 1024, 256, 0, s>>>(G, n, m, ldg, sigma);
    count_launch();
    return cudaGetLastError();
  }
  if (Vt && !warm_v) {
    init_identity_kernel<<<grid_for((long long)n * n), 256, 0, s>>>(Vt, n);
    count_launch();
  }
  e = cudaMemsetAsync(counters, 0, 2 * sizeof(int), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(work, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  if (n >= 2 && m <= 256 && n <= 2 * 1024) {
    // counters[2..3] hold the barrier (count, generation)
    e = cudaMemsetAsync(counters + 2, 0, 2 * sizeof(int), s);
    if (e != cudaSuccess) return e;
    if ((e = kernels_init()) != cudaSuccess) return e;
    const int npairs = ((n + 1) & ~1) / 2;
    int grid = npairs < max_small ? npairs : max_small;
    double tol = (double)m * 2.220446049250313e-16;
    unsigned* bar = (unsigned*)(counters + 2);
    long long limit = wait_cycles > 0 ? wait_cycles : BARRIER_WAIT_CYCLES;
    void* args[] = {&G, &n, &m, &ldg, &Vt, &max_sweeps, &tol, &counters, &work, &bar, &st, &limit};
    e = cudaLaunchCooperativeKernel((const void*)jacobi_small_kernel, dim3(grid), dim3(32), args, 0, s);
    count_launch();
    if (e != cudaSuccess) return e;
  } else if (n >= 2) {
    if ((e = kernels_init()) != cudaSuccess) return e;
    const int npairs = ((n + 1) & ~1) / 2;
    int grid = npairs < max_coresident ? npairs : max_coresident;
    // m * eps: an orthogonality a computed dot product of length m always resolves
    double tol = (double)m * 2.220446049250313e-16;
    void* args[] = {&G, &n, &m, &ldg, &Vt, &max_sweeps, &tol, &counters, &work, &st};
    e = cudaLaunchCooperativeKernel((const void*)jacobi_rows_kernel, dim3(grid), dim3(JAC_THREADS),
                                    args, 0, s);
    count_launch();
    if (e != cudaSuccess) return e;
  }
  row_norms_kernel<<<n < 1024 ? n : 1024, 256, 0, s>>>(G, n, m, ldg, sigma);
  count_launch();
  return cudaGetLastError();
}

cudaError_t set_identity(cudaStream_t s, cplx* V, int n) {
  init_identity_kernel<<<grid_for((long long)n * n), 256, 0, s>>>(V, n);
  count_launch();
  return cudaGetLastError();
}

cudaError_t orth_rows_finish(cudaStream_t s, cplx* G, int n, int m, long long ldg,
                             const double* sigma, double tol) {
  orth_finish_kernel<<<n < 1024 ? n : 1024, 256, 0, s>>>(G, n, m, ldg, sigma, tol);
  count_launch();
  return cudaGetLastError();
}

cudaError_t select_top(cudaStream_t s, const double* sigma, int n, int chi, double cutoff,
                       int* perm, double* s_sel) {
  select_top_kernel<<<1, 1024, 0, s>>>(sigma, n, chi, cutoff, perm, s_sel);
  count_launch();
  return cudaGetLastError();
}

cudaError_t gather_rows(cudaStream_t s, const cplx* in, long long ldi, cplx* out, long long ldo,
                        const int* perm, const double* sigma, int rows, int m,
                        bool normalize_by_sigma) {
  gather_rows_kernel<<<rows < 1024 ? rows : 1024, 256, 0, s>>>(in, ldi, out, ldo, perm, sigma,
                                                               rows, m, normalize_by_sigma);
  count_launch();
  return cudaGetLastError();
}

cudaError_t scale_rows_isqrt(cudaStream_t s, cplx* X, int rows, int m, long long ld,
                             const double* s_sel) {
  scale_rows_isqrt_kernel<<<rows < 1024 ? rows : 1024, 256, 0, s>>>(X, rows, m, ld, s_sel);
  count_launch();
  return cudaGetLastError();
}

cudaError_t trace_product(cudaStream_t s, const cplx* rho, const cplx* H, int n, double* acc,
                          int idx, double w) {
  trace_product_kernel<<<1, 1024, 0, s>>>(rho, H, n, acc, idx, w);
  count_launch();
  return cudaGetLastError();
}

cudaError_t trace_normalize(cudaStream_t s, cplx* rho, int n, double* work) {
  (void)work;
  trace_normalize_kernel<<<1, 1024, 0, s>>>(rho, n);
  count_launch();
  return cudaGetLastError();
}

cudaError_t row_norms(cudaStream_t s, const cplx* G, int n, int m, long long ldg, double* sigma) {
  row_norms_kernel<<<n < 1024 ? n : 1024, 256, 0, s>>>(G, n, m, ldg, sigma);
  count_launch();
  return cudaGetLastError();
}

