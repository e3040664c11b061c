// Complex FP64 GEMM on the CUDA cores (the plain-FP64 path of the CTM
// contractions) and the generic index permutation that feeds it.
#include "ctm_internal.h"

#include <algorithm>
#include <atomic>
#include <cmath>

static std::atomic<uint64_t> g_launches{0};
void count_launch(int n) { g_launches += (uint64_t)n; }
uint64_t launch_counter() { return g_launches.load(); }

namespace {

constexpr int BK = 16;
constexpr cplx ONE_C = {1.0, 0.0};
constexpr cplx ZERO_C = {0.0, 0.0};

__device__ __forceinline__ cplx ld_op(const cplx* p, bool cj) {
  cplx v = *p;
  if (cj) v.y = neg_bits(v.y);
  return v;
}

// TM x TN output tile per CTA (64 x 64 with 256 threads, or 32 x 32 with 64
// threads for small outputs), each thread a 4x4 block of outputs strided by
// TM/4 (TN/4) so that shared-memory reads are broadcast / conflict-free.
template <int TM, int TN>
__global__ void __launch_bounds__((TM / 4) * (TN / 4)) zgemm_kernel(int M, int N, int K, cplx alpha,
                                                   const cplx* __restrict__ A, long long lda,
                                                   int opA, const cplx* __restrict__ B,
                                                   long long ldb, int opB, cplx beta,
                                                   cplx* __restrict__ C, long long ldc,
                                                   long long sA, long long sB, long long sC,
                                                   int ksplit, int flags) {
  constexpr int BM = TM, BN = TN, NT = (TM / 4) * (TN / 4), SX = TN / 4, SY = TM / 4;
  __shared__ cplx As[BK][BM + 1];
  __shared__ cplx Bs[BK][BN + 1];
  const long long bz = blockIdx.z;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  if ((flags & ZG_UPPER_TILES) && blockIdx.y > blockIdx.x) return;  // tile below the diagonal: not needed
  const int tx = threadIdx.x % SX, ty = threadIdx.x / SX;
  const bool tA = opA & OP_T, cA = opA & OP_CONJ;
  const bool tB = opB & OP_T, cB = opB & OP_CONJ;
  if (ksplit > 0) {
    // split-K: entry z sums k in [z*ksplit, min(K, (z+1)*ksplit)) into its own C slice
    const long long kb = bz * (long long)ksplit;
    A += tA ? kb * lda : kb;
    B += tB ? kb : kb * ldb;
    K = (int)min((long long)ksplit, (long long)K - kb);
    if (flags & ZG_A_LOWER) K = (int)max(0LL, min((long long)K, (long long)(m0 + BM) - kb));
    C += bz * sC;
  } else {
    if (flags & ZG_A_LOWER) K = min(K, m0 + BM);  // A[m, k] = 0 for k > m: later k-tiles add nothing
    A += bz * sA;
    B += bz * sB;
    C += bz * sC;
  }
  double cr[4][4], ci[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) cr[i][j] = ci[i][j] = 0.0;

  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int e = threadIdx.x; e < BM * BK; e += NT) {
      int mm, kk;
      if (tA) { mm = e % BM; kk = e / BM; } else { kk = e % BK; mm = e / BK; }
      const int m = m0 + mm, k = k0 + kk;
      cplx v = make_double2(0.0, 0.0);
      if (m < M && k < K) v = ld_op(tA ? A + (long long)k * lda + m : A + (long long)m * lda + k, cA);
      As[kk][mm] = v;
    }
    for (int e = threadIdx.x; e < BN * BK; e += NT) {
      int nn, kk;
      if (tB) { kk = e % BK; nn = e / BK; } else { nn = e % BN; kk = e / BN; }
      const int n = n0 + nn, k = k0 + kk;
      cplx v = make_double2(0.0, 0.0);
      if (n < N && k < K) v = ld_op(tB ? B + (long long)n * ldb + k : B + (long long)k * ldb + n, cB);
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      cplx a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + SY * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + SX * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          cr[i][j] = fma(a[i].x, b[j].x, cr[i][j]);
          cr[i][j] = fma(-a[i].y, b[j].y, cr[i][j]);
          ci[i][j] = fma(a[i].x, b[j].y, ci[i][j]);
          ci[i][j] = fma(a[i].y, b[j].x, ci[i][j]);
        }
    }
    __syncthreads();
  }
  const bool use_beta = (beta.x != 0.0 || beta.y != 0.0);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + SY * i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx + SX * j;
      if (n >= N) continue;
      cplx* cp = C + (long long)m * ldc + n;
      double r = alpha.x * cr[i][j] - alpha.y * ci[i][j];
      double im = alpha.x * ci[i][j] + alpha.y * cr[i][j];
      if (use_beta) {
        const cplx o = *cp;
        r += beta.x * o.x - beta.y * o.y;
        im += beta.x * o.y + beta.y * o.x;
      }
      *cp = make_double2(r, im);
    }
  }
}

// C = alpha * sum_z W[z] (+ beta C), fixed summation order
__global__ void splitk_sum_kernel(const cplx* __restrict__ W, int S, int M, int N, cplx alpha, cplx beta,
                                  cplx* __restrict__ C, long long ldc, int flags, int tm, int tn) {
  const long long total = (long long)M * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    if ((flags & ZG_UPPER_TILES) && ((int)(e / N)) / tm > ((int)(e % N)) / tn) {
      C[(long long)(e / N) * ldc + (e % N)] = make_double2(0.0, 0.0);  // tile not computed
      continue;
    }
    double r = 0.0, im = 0.0;
    for (int z = 0; z < S; ++z) {
      r += W[z * total + e].x;
      im += W[z * total + e].y;
    }
    const int m = (int)(e / N), n = (int)(e % N);
    cplx* cp = C + (long long)m * ldc + n;
    double orr = alpha.x * r - alpha.y * im, oi = alpha.x * im + alpha.y * r;
    if (beta.x != 0.0 || beta.y != 0.0) {
      const cplx o = *cp;
      orr += beta.x * o.x - beta.y * o.y;
      oi += beta.x * o.y + beta.y * o.x;
    }
    *cp = make_double2(orr, oi);
  }
}

struct PermParams {
  int nd;
  long long odims[8];
  long long istr[8];
};

template <typename Idx>
__global__ void permute_kernel(const cplx* __restrict__ in, cplx* __restrict__ out,
                               long long total, PermParams p, int conj, cplx alpha, int unit) {
  for (Idx i = (Idx)blockIdx.x * (Idx)blockDim.x + threadIdx.x; i < (Idx)total; i += (Idx)gridDim.x * blockDim.x) {
    Idx r = i, off = 0;
    for (int a = p.nd - 1; a >= 0; --a) {
      const Idx d = (Idx)p.odims[a];
      const Idx q = r / d;
      off += (r - q * d) * (Idx)p.istr[a];
      r = q;
    }
    cplx v = in[off];
    if (conj) v.y = neg_bits(v.y);
    if (unit) {
      out[i] = v;  // no FP64 arithmetic for the usual alpha = 1
    } else {
      out[i] = make_double2(alpha.x * v.x - alpha.y * v.y, alpha.x * v.y + alpha.y * v.x);
    }
  }
}

}  // namespace

cudaError_t zgemm(cudaStream_t s, int M, int N, int K, cplx alpha, const cplx* A, long long lda,
                  int opA, const cplx* B, long long ldb, int opB, cplx beta, cplx* C,
                  long long ldc, GemmBatch batch, cplx* work, long long work_elems, int flags) {
  if (M <= 0 || N <= 0 || batch.count <= 0) return cudaSuccess;
  if ((flags & ZG_UPPER_TILES) && M != N) return cudaErrorInvalidValue;
  // Tile size and K split from a cost model of the FP64 pipe: every SM's FP64
  // units carry the product; an SM runs at full rate with >= 16 resident warps
  // and, measured on GB300, at 0.61x with one 8-warp CTA (rate ~ (warps/16)^0.72
  // below 16).  Cost = k-tiles per CTA x CTAs on the busiest SM x tile work /
  // rate; splits keep whole k-tiles.
  const long long kb = (K + BK - 1) / BK;
  int best_T = 64;
  long long best_S = 1;
  double best_cost = -1.0;
  for (int T : {64, 32}) {
    if (batch.count != 1 && T != 64) continue;
    const long long tm = (M + T - 1) / T, tn = (N + T - 1) / T;
    const long long tiles = (flags & ZG_UPPER_TILES) ? tm * (tm + 1) / 2 : tm * tn;
    const double unit = T == 64 ? 1.0 : 0.25;
    const int warps = T == 64 ? 8 : 2;
    const bool can_split = batch.count == 1 && work && K >= 2 * BK;
    for (long long S = 1; S <= (can_split ? 160 : 1) && S <= kb; ++S) {
      const long long kps = (kb + S - 1) / S, Se = (kb + kps - 1) / kps;
      if (Se > 1 && Se * M * N > work_elems) break;
      const long long busy = (tiles * Se * batch.count + 151) / 152;
      const double rate = std::min(1.0, std::pow((double)(busy * warps) / 16.0, 0.72));
      const double cost = (double)kps * (double)busy * unit / rate + 1e-4 * (double)Se;
      if (best_cost < 0.0 || cost < best_cost) {
        best_cost = cost;
        best_S = Se;
        best_T = T;
      }
    }
  }
  const int T = best_T;
  const long long tm = (M + T - 1) / T, tn = (N + T - 1) / T;
  auto launch = [&](dim3 grid, cplx al, cplx be, cplx* out, long long ldo, long long sC, int ksplit, int fl) {
    if (T == 64)
      zgemm_kernel<64, 64><<<grid, 256, 0, s>>>(M, N, K, al, A, lda, opA, B, ldb, opB, be, out, ldo, batch.sA,
                                                batch.sB, sC, ksplit, fl);
    else
      zgemm_kernel<32, 32><<<grid, 64, 0, s>>>(M, N, K, al, A, lda, opA, B, ldb, opB, be, out, ldo, batch.sA,
                                               batch.sB, sC, ksplit, fl);
  };
  if (best_S >= 2) {
    const long long kps = (kb + best_S - 1) / best_S;
    const int ksplit = (int)(kps * BK);
    const long long S = (K + ksplit - 1) / ksplit;
    launch(dim3((unsigned)tn, (unsigned)tm, (unsigned)S), ONE_C, ZERO_C, work, N, (long long)M * N, ksplit, flags);
    long long blocks = ((long long)M * N + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    splitk_sum_kernel<<<(unsigned)blocks, 256, 0, s>>>(work, (int)S, M, N, alpha, beta, C, ldc, flags, T, T);
    count_launch(2);
    return cudaGetLastError();
  }
  if (flags & ZG_UPPER_TILES) flags &= ~ZG_UPPER_TILES;  // unsplit: full tiles (lower ones are cheap here)
  dim3 grid((unsigned)tn, (unsigned)tm, batch.count);
  if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
  launch(grid, alpha, beta, C, ldc, batch.sC, 0, flags);
  count_launch();
  return cudaGetLastError();
}

cudaError_t permute(cudaStream_t s, const cplx* in, cplx* out, int nd, const int* in_dims,
                    const int* perm, bool conj, cplx alpha) {
  if (nd < 1 || nd > 8) return cudaErrorInvalidValue;
  PermParams p;
  p.nd = nd;
  long long istride[8];
  long long acc = 1;
  for (int a = nd - 1; a >= 0; --a) {
    istride[a] = acc;
    acc *= in_dims[a];
  }
  // output axes that stay adjacent and in order in the input merge into one
  // (fewer divisions per element)
  p.nd = 0;
  for (int i = 0; i < nd; ++i) {
    if (p.nd > 0 && perm[i] == perm[i - 1] + 1) {
      p.odims[p.nd - 1] *= in_dims[perm[i]];
      p.istr[p.nd - 1] = istride[perm[i]];
    } else {
      p.odims[p.nd] = in_dims[perm[i]];
      p.istr[p.nd] = istride[perm[i]];
      ++p.nd;
    }
  }
  const long long total = acc;
  if (total == 0) return cudaSuccess;
  long long blocks = (total + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  const int unit = alpha.x == 1.0 && alpha.y == 0.0;
  if (total < (1LL << 31))  // 32-bit index arithmetic (offsets are below total)
    permute_kernel<unsigned><<<(unsigned)blocks, 256, 0, s>>>(in, out, total, p, conj ? 1 : 0, alpha, unit);
  else
    permute_kernel<unsigned long long><<<(unsigned)blocks, 256, 0, s>>>(in, out, total, p, conj ? 1 : 0, alpha,
                                                                         unit);
  count_launch();
  return cudaGetLastError();
}
