// Tensor-core GEMM of the precision form (sm_103a, tcgen05 + TMA + TMEM).
//
// A complex GEMM C = alpha opA(A) opB(B) (complex128 storage) runs as one real
// GEMM through the real embedding
//     Ar[m, 2k+c]      = (Re, Im)[c] of A[m,k]                       (M x 2K)
//     Br^T[2n+b, 2k+a] = [[Re, Im], [-Im, Re]][a][b] of B[k,n]        (2N x 2K)
//     Cr[m, 2n+b]      = (Re, Im)[b] of C[m,n]
// Both packed operands are K-major, in TF32 (one array), in BF16 hi/lo pairs
// (x = hi + lo, three products hi*hi + hi*lo + lo*hi accumulated in FP32 in
// tensor memory: 16 significand bits per operand) or in BF16 hi/mid/lo
// triples (x = p0 + p1 + p2, the six products p_i q_j with i + j <= 2: 24
// significand bits, the FP32 class).  One CTA computes a 128 x BN tile of Cr: warp 0
// issues the TMA loads (128-byte swizzle), warp 1 issues tcgen05.mma, all four
// warps drain the accumulator with tcgen05.ld.  Thin products (few output
// tiles) split K over the grid's z dimension into FP32 partials, summed in a
// fixed order by a second kernel.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "tc_gemm.h"
#include "tc_ptx.h"

#include <algorithm>
#include <map>
#include <tuple>
#include <type_traits>
#include <vector>

namespace {

// N of every packed B operand padded to NPAD; 256-wide tiles only where the
// padded N is a multiple of 256
constexpr int BM = 128, NPAD = 128;
constexpr int NTHREADS = 192;        // main kernel: producer warp, MMA warp, four epilogue warps
constexpr int PREC_TF32 = 1, PREC_BF16X3 = 2, PREC_BF16X6 = 3;



// Tile configuration: 128 x BN output tile (BN = 128 or 256), k-blocks of 128
// bytes (64 for BF16x6), as many pipeline stages as fit in ~220 KB of shared
// memory.  NOPS parts per operand (1 TF32, 2 BF16 hi/lo, 3 BF16 hi/mid/lo);
// BF16x6 takes 64-byte k-blocks (64-byte swizzle) so that its three A and
// three B parts fit four stages at BN = 128 and three at BN = 256.
template <int PREC, int BN_>
struct Cfg {
  static constexpr int BN = BN_;
  static constexpr int ELEM = PREC == PREC_TF32 ? 4 : 2;
  static constexpr int KB_BYTES = PREC == PREC_BF16X6 ? 64 : 128;  // bytes of a k-block row
  static constexpr int BK = KB_BYTES / ELEM;                        // elements per k-block
  static constexpr int NOPS = PREC == PREC_TF32 ? 1 : (PREC == PREC_BF16X3 ? 2 : 3);
  static constexpr int A_BYTES = BM * KB_BYTES;
  static constexpr int B_BYTES = BN * KB_BYTES;
  static constexpr int STAGE_BYTES = NOPS * (A_BYTES + B_BYTES);
  static constexpr int STAGES = (220 * 1024) / STAGE_BYTES;
  static_assert(STAGES >= 2, "at least two pipeline stages");
  static constexpr int UMMA_K = PREC == PREC_TF32 ? 8 : 16;  // K of one MMA
  static constexpr int KSTEPS = BK / UMMA_K;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 256;
  // instruction descriptor: FP32 accumulate, K-major A and B, N = BN, M = 128
  static constexpr uint32_t IDESC = (1u << 4) | ((PREC == PREC_TF32 ? 2u : 1u) << 7) |
                                    ((PREC == PREC_TF32 ? 2u : 1u) << 10) |
                                    ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
};

template <int PREC, uint32_t IDESC>
__device__ __forceinline__ void umma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t accum) {
  if (PREC == PREC_TF32) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(IDESC), "r"(accum)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(IDESC), "r"(accum)
        : "memory");
  }
}

// Persistent main kernel: CTA b takes the output tiles t = b, b + grid, ...
// (t = n_tile + n_tiles * (m_tile + m_tiles * split)).  Warp 0 streams the
// k-blocks of its tiles through the shared-memory stages (TMA), warp 1 issues
// the MMAs of tile i into accumulator set i % 2 (tensor-memory columns
// BN (i % 2) ..), warps 2..5 drain set i % 2 to global memory while the MMAs
// of tile i + 1 run in the other set.
template <int PREC, int BN>
__global__ void __launch_bounds__(NTHREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
                   const __grid_constant__ CUtensorMap mA2, const __grid_constant__ CUtensorMap mB0,
                   const __grid_constant__ CUtensorMap mB1, const __grid_constant__ CUtensorMap mB2,
                   int kb_total, int kb_per_split, int n_tiles, int m_tiles, int tiles, int M, int Nr, cplx alpha,
                   cplx* __restrict__ C, long long ldc, float* __restrict__ partial, int Nrp, long long pstride,
                   int conj_out, int unit_alpha, int* __restrict__ timeouts) {
  using K_ = Cfg<PREC, BN>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + K_::STAGES * K_::STAGE_BYTES);
  uint64_t* empty = full + K_::STAGES;
  uint64_t* acc_full = empty + K_::STAGES;  // [2], per accumulator set
  uint64_t* acc_empty = acc_full + 2;      // [2]
  uint64_t* mma_done = acc_empty + 2;
  uint32_t* tmem_slot = (uint32_t*)(mma_done + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto kblocks = [&](int t, int* kb0) {
    const int split = t / (n_tiles * m_tiles);
    *kb0 = split * kb_per_split;
    return min(kb_total, *kb0 + kb_per_split) - *kb0;  // >= 1 by construction
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < K_::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);  // one arrival per epilogue warp
    }
    mbar_init(mma_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer: one k-block per stage, the stages cycling across tiles
    int q = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
      int kb0;
      const int nkb = kblocks(t, &kb0);
      const int n_tile = t % n_tiles, m_tile = (t / n_tiles) % m_tiles;
      for (int i = 0; i < nkb; ++i, ++q) {
        const int s = q % K_::STAGES, r = q / K_::STAGES;
        if (!mbar_wait(&empty[s], (r & 1) ^ 1)) {
          atomicAdd(timeouts, 1);
          ok = false;
          break;
        }
        unsigned char* st = smem + s * K_::STAGE_BYTES;
        mbar_expect_tx(&full[s], K_::STAGE_BYTES);
        const int kx = (kb0 + i) * K_::BK;
        unsigned char* sb = st + K_::NOPS * K_::A_BYTES;
        tma_load_2d(st, &mA0, &full[s], kx, m_tile * BM);
        tma_load_2d(sb, &mB0, &full[s], kx, n_tile * BN);
        if (K_::NOPS >= 2) {
          tma_load_2d(st + K_::A_BYTES, &mA1, &full[s], kx, m_tile * BM);
          tma_load_2d(sb + K_::B_BYTES, &mB1, &full[s], kx, n_tile * BN);
        }
        if (K_::NOPS == 3) {
          tma_load_2d(st + 2 * K_::A_BYTES, &mA2, &full[s], kx, m_tile * BM);
          tma_load_2d(sb + 2 * K_::B_BYTES, &mB2, &full[s], kx, n_tile * BN);
        }
      }
    }
    // the last loads of every stage have landed before the CTA can leave
    // (they are what an MMA issuer that gave up may not have waited for)
    for (int j = max(0, q - K_::STAGES); j < q; ++j)
      if (!mbar_wait(&full[j % K_::STAGES], (j / K_::STAGES) & 1)) atomicAdd(timeouts, 1);
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    int q = 0, it = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++it) {
      int kb0;
      const int nkb = kblocks(t, &kb0);
      const int b = it & 1;
      // the set was drained: tile it - 2 was that set's drain number it/2 - 1
      if (it >= 2 && !mbar_wait(&acc_empty[b], ((it >> 1) - 1) & 1)) {
        atomicAdd(timeouts, 1);
        ok = false;
        break;
      }
      fence_after();
      const uint32_t d = tmem + (uint32_t)(b * BN);
      for (int i = 0; i < nkb; ++i, ++q) {
        const int s = q % K_::STAGES, r = q / K_::STAGES;
        if (!mbar_wait(&full[s], r & 1)) {
          atomicAdd(timeouts, 1);
          ok = false;
          break;
        }
        fence_after();
        const uint32_t base = smem_u32(smem + s * K_::STAGE_BYTES);
        const uint32_t a0 = base, a1 = base + K_::A_BYTES, a2 = base + 2 * K_::A_BYTES;
        const uint32_t b0 = base + K_::NOPS * K_::A_BYTES, b1 = b0 + K_::B_BYTES, b2 = b0 + 2 * K_::B_BYTES;
#pragma unroll
        for (int j = 0; j < K_::KSTEPS; ++j) {
          const uint32_t ko = j * 32;  // bytes of one MMA's K inside the k-block row
          const uint32_t acc = (i > 0 || j > 0) ? 1u : 0u;
          if (K_::NOPS == 3) {
            // smallest parts first: p_i q_j with i + j = 2, then 1, then 0
            umma<PREC, K_::IDESC>(d, sdesc_kb<K_::KB_BYTES>(a0 + ko), sdesc_kb<K_::KB_BYTES>(b2 + ko), acc);
            umma<PREC, K_::IDESC>(d, sdesc_kb<K_::KB_BYTES>(a1 + ko), sdesc_kb<K_::KB_BYTES>(b1 + ko), 1u);
            umma<PREC, K_::IDESC>(d, sdesc_kb<K_::KB_BYTES>(a2 + ko), sdesc_kb<K_::KB_BYTES>(b0 + ko), 1u);
            umma<PREC, K_::IDESC>(d, sdesc_kb<K_::KB_BYTES>(a0 + ko), sdesc_kb<K_::KB_BYTES>(b1 + ko), 1u);
            umma<PREC, K_::IDESC>(d, sdesc_kb<K_::KB_BYTES>(a1 + ko), sdesc_kb<K_::KB_BYTES>(b0 + ko), 1u);
            umma<PREC, K_::IDESC>(d, sdesc_kb<K_::KB_BYTES>(a0 + ko), sdesc_kb<K_::KB_BYTES>(b0 + ko), 1u);
          } else {
            umma<PREC, K_::IDESC>(d, sdesc_kb<K_::KB_BYTES>(a0 + ko), sdesc_kb<K_::KB_BYTES>(b0 + ko), acc);
            if (K_::NOPS == 2) {
              umma<PREC, K_::IDESC>(d, sdesc_kb<K_::KB_BYTES>(a0 + ko), sdesc_kb<K_::KB_BYTES>(b1 + ko), 1u);
              umma<PREC, K_::IDESC>(d, sdesc_kb<K_::KB_BYTES>(a1 + ko), sdesc_kb<K_::KB_BYTES>(b0 + ko), 1u);
            }
          }
        }
        umma_commit(&empty[s]);  // frees the stage when these MMAs are done
      }
      if (ok) umma_commit(&acc_full[b]);
    }
    // every MMA issued has completed before the accumulators are released
    umma_commit(mma_done);
    if (!mbar_wait(mma_done, 0)) atomicAdd(timeouts, 1);
  } else if (warp >= 2) {
    // epilogue: warp w drains tensor-memory lanes 32 (w % 4) .. (the rows of its quarter)
    const int quad = warp & 3;
    int it = 0;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++it) {
      const int split = t / (n_tiles * m_tiles);
      const int n_tile = t % n_tiles, m_tile = (t / n_tiles) % m_tiles;
      const int b = it & 1;
      // every lane saw the set complete, or the warp stops (a wait that ran out)
      const bool ready = __all_sync(0xffffffffu, mbar_wait(&acc_full[b], (it >> 1) & 1));
      if (!ready) {
        if (lane == 0) atomicAdd(timeouts, 1);
        break;
      }
      fence_after();
      const int row = m_tile * BM + quad * 32 + lane;
      const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * BN);
      for (int c0 = 0; c0 < BN; c0 += 16) {
        float v[16];
        tmem_ld16(trow + c0, v);
        const int col = n_tile * BN + c0;  // real column
        if (partial) {
          float4* dst = (float4*)(partial + split * pstride + (long long)row * Nrp + col);
#pragma unroll
          for (int q = 0; q < 4; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        } else if (row < M) {
          if (unit_alpha) {
            // alpha = 1: exact FP32 -> FP64 widening on the integer pipe
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              if (col + 2 * u < Nr) {
                const double re = f2d_bits(v[2 * u]), im = f2d_bits(v[2 * u + 1]);
                C[(long long)row * ldc + (col >> 1) + u] = make_double2(re, conj_out ? neg_bits(im) : im);
              }
            }
          } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              if (col + 2 * u < Nr) {
                const double re = v[2 * u], im = v[2 * u + 1];
                const double orr = alpha.x * re - alpha.y * im, oi = alpha.x * im + alpha.y * re;
                C[(long long)row * ldc + (col >> 1) + u] = make_double2(orr, conj_out ? -oi : oi);
              }
            }
          }
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[b]);
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN) : "memory");
  }
}

// C[m,n] = alpha * sum_z P[z][m][2n .. 2n+1]  (fixed summation order)
__global__ void splitk_reduce_kernel(const float* __restrict__ P, int S, long long pstride, int Nrp, int M,
                                     int N, cplx alpha, cplx* __restrict__ C, long long ldc, int conj_out,
                                     int unit_alpha) {
  const long long total = (long long)M * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(e / N), n = (int)(e % N);
    if (unit_alpha) {
      // FP32 sum of the partials (the products carry ~16 significant bits),
      // widened to FP64 on the integer pipe
      float re = 0.0f, im = 0.0f;
      for (int z = 0; z < S; ++z) {
        const float2 p = *(const float2*)(P + z * pstride + (long long)m * Nrp + 2 * n);
        re += p.x;
        im += p.y;
      }
      const double dr = f2d_bits(re), di = f2d_bits(im);
      C[(long long)m * ldc + n] = make_double2(dr, conj_out ? neg_bits(di) : di);
      continue;
    }
    double re = 0.0, im = 0.0;
    for (int z = 0; z < S; ++z) {
      const float2 p = *(const float2*)(P + z * pstride + (long long)m * Nrp + 2 * n);
      re += p.x;
      im += p.y;
    }
    const double oi = alpha.x * im + alpha.y * re;
    C[(long long)m * ldc + n] = make_double2(alpha.x * re - alpha.y * im, conj_out ? -oi : oi);
  }
}

// The same with a warp per output for many splits: lane l sums splits
// l, l + 32, ... in order, then the lanes' sums meet in a fixed butterfly.
__global__ void splitk_reduce_warp_kernel(const float* __restrict__ P, int S, long long pstride, int Nrp, int M,
                                          int N, cplx alpha, cplx* __restrict__ C, long long ldc, int conj_out,
                                          int unit_alpha) {
  const int lane = threadIdx.x & 31;
  const long long total = (long long)M * N;
  for (long long e = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; e < total;
       e += ((long long)gridDim.x * blockDim.x) >> 5) {
    const int m = (int)(e / N), n = (int)(e % N);
    float re = 0.0f, im = 0.0f;
    for (int z = lane; z < S; z += 32) {
      const float2 p = *(const float2*)(P + z * pstride + (long long)m * Nrp + 2 * n);
      re += p.x;
      im += p.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane != 0) continue;
    if (unit_alpha) {
      const double dr = f2d_bits(re), di = f2d_bits(im);
      C[(long long)m * ldc + n] = make_double2(dr, conj_out ? neg_bits(di) : di);
    } else {
      const double r = re, i = im;
      const double oi = alpha.x * i + alpha.y * r;
      C[(long long)m * ldc + n] = make_double2(alpha.x * r - alpha.y * i, conj_out ? -oi : oi);
    }
  }
}

__device__ __forceinline__ cplx load_op(const cplx* X, long long ld, int op, int r, int c) {
  // element (r, c) of the operand in its GEMM role (A: (m,k); B: (k,n))
  cplx v = (op & OP_T) ? X[(long long)c * ld + r] : X[(long long)r * ld + c];
  if (op & OP_CONJ) v.y = neg_bits(v.y);
  return v;
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return u;
}

// binary64 -> binary32 rounded to nearest (ties away from zero) on the
// integer pipe: half an FP32 ulp is added to the magnitude bits before the
// truncation of d2f_bits (a carry into the exponent is the correct rounding).
__device__ __forceinline__ float d2f_rn_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned long long mag = b & 0x7FFFFFFFFFFFFFFFull;
  if (mag >= 0x7FF0000000000000ull) return d2f_bits(x);  // Inf / NaN
  return d2f_bits(__longlong_as_double((long long)((b & 0x8000000000000000ull) | (mag + (1ull << 28)))));
}

// x = p0 + p1 + p2 exactly for the FP32 value f (24 significand bits): each
// part is the BF16 rounding of the remainder the previous parts leave
__device__ __forceinline__ void split3(float f, __nv_bfloat16& p0, __nv_bfloat16& p1, __nv_bfloat16& p2) {
  p0 = __float2bfloat16_rn(f);
  const float r1 = f - __bfloat162float(p0);
  p1 = __float2bfloat16_rn(r1);
  p2 = __float2bfloat16_rn(r1 - __bfloat162float(p1));
}

__device__ __forceinline__ void store_pair(int prec, long long e, double x0, double x1, void* o0, void* o1,
                                           void* o2) {
  // two consecutive packed reals at element e (e even)
  if (prec == PREC_TF32) {
    ((uint2*)o0)[e >> 1] = make_uint2(to_tf32(d2f_bits(x0)), to_tf32(d2f_bits(x1)));
  } else if (prec == PREC_BF16X6) {
    __nv_bfloat16 a0, a1, a2, c0, c1, c2;
    split3(d2f_rn_bits(x0), a0, a1, a2);
    split3(d2f_rn_bits(x1), c0, c1, c2);
    ((__nv_bfloat162*)o0)[e >> 1] = __halves2bfloat162(a0, c0);
    ((__nv_bfloat162*)o1)[e >> 1] = __halves2bfloat162(a1, c1);
    ((__nv_bfloat162*)o2)[e >> 1] = __halves2bfloat162(a2, c2);
  } else {
    const float f0 = d2f_bits(x0), f1 = d2f_bits(x1);
    const __nv_bfloat16 h0 = __float2bfloat16_rn(f0), h1 = __float2bfloat16_rn(f1);
    const __nv_bfloat16 l0 = __float2bfloat16_rn(f0 - __bfloat162float(h0));
    const __nv_bfloat16 l1 = __float2bfloat16_rn(f1 - __bfloat162float(h1));
    ((__nv_bfloat162*)o0)[e >> 1] = __halves2bfloat162(h0, h1);
    ((__nv_bfloat162*)o1)[e >> 1] = __halves2bfloat162(l0, l1);
  }
}

// Ar[m, kr], padded to Mp x Krp (K-major)
template <int PREC, typename Idx>
__global__ void pack_a_kernel(const cplx* __restrict__ A, long long lda, int opA, int M, int K, int Mp, int Krp,
                              void* __restrict__ o0, void* __restrict__ o1, void* __restrict__ o2) {
  // one thread per complex element: its (Re, Im) pair stored together
  const Idx kc = (Idx)(Krp >> 1), total = (Idx)Mp * kc;
  for (Idx e = (Idx)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (Idx)gridDim.x * blockDim.x) {
    const Idx m = e / kc, k = e - m * kc;
    cplx v = make_double2(0.0, 0.0);
    if ((int)m < M && (int)k < K) v = load_op(A, lda, opA, (int)m, (int)k);
    store_pair(PREC, (long long)m * Krp + 2 * (long long)k, v.x, v.y, o0, o1, o2);
  }
}

// Br^T[nr, kr] = [[Re, Im], [-Im, Re]][kr%2][nr%2] of B[kr/2, nr/2], padded to Nrp x Krp
template <int PREC, typename Idx>
__global__ void pack_b_kernel(const cplx* __restrict__ B, long long ldb, int opB, int N, int K, int Nrp, int Krp,
                              void* __restrict__ o0, void* __restrict__ o1, void* __restrict__ o2) {
  // one thread per complex element B[k, n]: rows 2n (Re, -Im) and 2n+1 (Im, Re)
  const Idx kc = (Idx)(Krp >> 1), total = (Idx)(Nrp >> 1) * kc;
  for (Idx e = (Idx)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (Idx)gridDim.x * blockDim.x) {
    const Idx n = e / kc, k = e - n * kc;
    cplx v = make_double2(0.0, 0.0);
    if ((int)n < N && (int)k < K) v = load_op(B, ldb, opB, (int)k, (int)n);
    const long long r0 = (long long)(2 * n) * Krp + 2 * (long long)k;
    store_pair(PREC, r0, v.x, neg_bits(v.y), o0, o1, o2);
    store_pair(PREC, r0 + Krp, v.y, v.x, o0, o1, o2);
  }
}

// Br^T[nr, kr] for an op-N (or op-C) operand B[k, n] (row-major, k x n):
// 32 x 32 complex tiles through shared memory so reads run along n and
// writes along kr (the plain kernel would read with stride ldb).
template <int PREC>
__global__ void pack_b_tr_kernel(const cplx* __restrict__ B, long long ldb, int conj, int N, int K, int Nrp,
                                 int Krp, void* __restrict__ o0, void* __restrict__ o1, void* __restrict__ o2) {
  __shared__ cplx tile[32][33];
  const int k0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int k = k0 + i, n = n0 + threadIdx.x;
    cplx v = make_double2(0.0, 0.0);
    if (k < K && n < N) {
      v = B[(long long)k * ldb + n];
      if (conj) v.y = neg_bits(v.y);
    }
    tile[i][threadIdx.x] = v;
  }
  __syncthreads();
  // thread x writes the real pair of complex column k0 + x on each of the
  // 64 real rows: a warp stores 128 contiguous bytes per part
  const int k = k0 + threadIdx.x;
  if (2 * k >= Krp) return;
  for (int r = threadIdx.y; r < 64; r += blockDim.y) {
    const int nr = 2 * n0 + r;
    if (nr >= Nrp) break;
    const cplx v = tile[threadIdx.x][r >> 1];
    const long long e = (long long)nr * Krp + 2 * (long long)k;
    if (r & 1)
      store_pair(PREC, e, v.y, v.x, o0, o1, o2);  // row 2n+1: (Im, Re)
    else
      store_pair(PREC, e, v.x, neg_bits(v.y), o0, o1, o2);  // row 2n: (Re, -Im)
  }
}

__device__ __forceinline__ long long view_off(unsigned idx, int n, const int* dim, const long long* str) {
  long long off = 0;
  for (int a = n - 1; a >= 0; --a) {
    const unsigned d = (unsigned)dim[a];
    const unsigned q = idx / d;
    off += (long long)(idx - q * d) * str[a];
    idx = q;
  }
  return off;
}


// Ar[m, kr] gathered through a view (rows m, columns k): a fused
// permute-and-pack of the A operand, padded to Mp x Krp, by 32 x 32 complex
// tiles.  The view offsets of the tile's 32 rows and 32 columns are computed
// once per tile (the divisions of the index arithmetic would otherwise bound
// the kernel); reads run along whichever of m or k is contiguous in the
// source (row_contig: m), writes along k.
template <int PREC>
__global__ void pack_a_tiled_kernel(TcView V, int M, int K, int Mp, int Krp, int row_contig, void* __restrict__ o0,
                                    void* __restrict__ o1, void* __restrict__ o2) {
  __shared__ cplx tile[32][33];
  __shared__ long long roff[32], coff[32];
  const int k0 = blockIdx.x * 32, m0 = blockIdx.y * 32;
  if (threadIdx.y == 0) {
    const int m = m0 + threadIdx.x, k = k0 + threadIdx.x;
    roff[threadIdx.x] = m < M ? view_off((unsigned)m, V.nr, V.rdim, V.rstr) : -1;
    coff[threadIdx.x] = k < K ? view_off((unsigned)k, V.nc, V.cdim, V.cstr) : -1;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int mi = row_contig ? (int)threadIdx.x : i, ki = row_contig ? i : (int)threadIdx.x;
    cplx v = make_double2(0.0, 0.0);
    if (roff[mi] >= 0 && coff[ki] >= 0) {
      v = V.p[roff[mi] + coff[ki]];
      if (V.conj) v.y = neg_bits(v.y);
    }
    tile[ki][mi] = v;
  }
  __syncthreads();
  const int k = k0 + threadIdx.x;
  if (2 * k >= Krp) return;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int m = m0 + r;
    if (m >= Mp) break;
    const cplx v = tile[threadIdx.x][r];
    store_pair(PREC, (long long)m * Krp + 2 * (long long)k, v.x, v.y, o0, o1, o2);
  }
}

// Br^T[nr, kr] gathered through a view (rows n, columns k), padded to Nrp x Krp,
// by 32 x 32 complex tiles as pack_a_tiled_kernel: complex (n, k) gives rows
// 2n: (Re, -Im) and 2n+1: (Im, Re) at columns 2k, 2k+1
template <int PREC>
__global__ void pack_b_tiled_kernel(TcView V, int N, int K, int Nrp, int Krp, int row_contig, void* __restrict__ o0,
                                    void* __restrict__ o1, void* __restrict__ o2) {
  __shared__ cplx tile[32][33];
  __shared__ long long roff[32], coff[32];
  const int k0 = blockIdx.x * 32, n0 = blockIdx.y * 32;
  if (threadIdx.y == 0) {
    const int n = n0 + threadIdx.x, k = k0 + threadIdx.x;
    roff[threadIdx.x] = n < N ? view_off((unsigned)n, V.nr, V.rdim, V.rstr) : -1;
    coff[threadIdx.x] = k < K ? view_off((unsigned)k, V.nc, V.cdim, V.cstr) : -1;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int ni = row_contig ? (int)threadIdx.x : i, ki = row_contig ? i : (int)threadIdx.x;
    cplx v = make_double2(0.0, 0.0);
    if (roff[ni] >= 0 && coff[ki] >= 0) {
      v = V.p[roff[ni] + coff[ki]];
      if (V.conj) v.y = neg_bits(v.y);
    }
    tile[ki][ni] = v;
  }
  __syncthreads();
  const int k = k0 + threadIdx.x;
  if (2 * k >= Krp) return;
  for (int r = threadIdx.y; r < 64; r += blockDim.y) {
    const int nr = 2 * n0 + r;
    if (nr >= Nrp) break;
    const cplx v = tile[threadIdx.x][r >> 1];
    const long long e = (long long)nr * Krp + 2 * (long long)k;
    if (r & 1)
      store_pair(PREC, e, v.y, v.x, o0, o1, o2);  // row 2n+1: (Im, Re)
    else
      store_pair(PREC, e, v.x, neg_bits(v.y), o0, o1, o2);  // row 2n: (Re, -Im)
  }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

cudaError_t get_encoder() {
  if (g_encode) return cudaSuccess;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess) return e;
  if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
  g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  return cudaSuccess;
}

// K-major [rows x kcols] operand, box of box_rows x (128 bytes)
cudaError_t make_map(CUtensorMap* map, void* base, int prec, long long rows, long long kcols, int box_rows,
                     int kb_bytes = 128) {
  const bool tf = prec == PREC_TF32;
  const int esz = tf ? 4 : 2;
  const cuuint64_t dims[2] = {(cuuint64_t)kcols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(kcols * esz)};
  const cuuint32_t box[2] = {(cuuint32_t)(kb_bytes / esz), (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(map, tf ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        kb_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

unsigned grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 152 * 16) b = 152 * 16;
  return (unsigned)b;
}

template <int PREC>
cudaError_t pack_b_any(cudaStream_t s, const cplx* B, long long ldb, int opB, int N, int K, long long Nrp,
                       long long Krp, void* b0, void* b1, void* b2) {
  if (opB & OP_T) {
    if (Nrp * Krp < (1LL << 31))
      pack_b_kernel<PREC, unsigned><<<grid_for(Nrp * Krp / 4), 256, 0, s>>>(B, ldb, opB, N, K, (int)Nrp, (int)Krp, b0, b1,
                                                                          b2);
    else
      pack_b_kernel<PREC, unsigned long long><<<grid_for(Nrp * Krp / 4), 256, 0, s>>>(B, ldb, opB, N, K, (int)Nrp,
                                                                                   (int)Krp, b0, b1, b2);
  } else {
    dim3 grid((unsigned)((Nrp / 2 + 31) / 32), (unsigned)((Krp / 2 + 31) / 32));
    pack_b_tr_kernel<PREC><<<grid, dim3(32, 8), 0, s>>>(B, ldb, (opB & OP_CONJ) ? 1 : 0, N, K, (int)Nrp, (int)Krp,
                                                        b0, b1, b2);
  }
  count_launch();
  return cudaGetLastError();
}

template <int PREC>
void padded(int N, int K, long long* Nrp, long long* Krp) {
  // BF16 operands (x3 and x6 alike) are padded to 64-element k-blocks, so that
  // a corner packed once serves either mode's kernel
  constexpr int BK = Cfg<PREC == PREC_BF16X6 ? PREC_BF16X3 : PREC, 128>::BK;
  *Krp = (2LL * K + BK - 1) / BK * BK;
  *Nrp = (2LL * N + NPAD - 1) / NPAD * NPAD;
}

constexpr int NSM = 152;  // SMs of the part (one CTA of the main kernel per SM)

// Default tile choice: 256-wide tiles; a product with fewer output tiles than
// SMs splits K into at most two whole waves of CTAs.
TcChoice heuristic(long long Mp, long long Nrp, int kb_total) {
  const int bn = Nrp % 256 == 0 ? 256 : 128;
  const long long tiles = (Mp / BM) * (Nrp / bn);
  int S = 1;
  if (tiles < NSM) {
    S = (int)((2 * NSM) / tiles);
    if (S > kb_total / 2) S = kb_total / 2;
    if (S < 1) S = 1;
  }
  return TcChoice{bn, S};
}

// effective number of splits (every split gets at least one k-block)
int eff_splits(int kb_total, int S) {
  if (S < 1) S = 1;
  if (S > kb_total) S = kb_total;
  const int kps = (kb_total + S - 1) / S;
  return (kb_total + kps - 1) / kps;
}

// The packed operands of one product, ready for the main kernel.
struct Operands {
  void *a0, *a1, *a2, *b0, *b1, *b2;
  long long Mp, Nrp, Krp;
  int kb_total;
};

// one-time kernel attribute (dynamic shared memory above 48 KB)
template <int PREC, int BN>
cudaError_t ensure_attr() {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<PREC, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         Cfg<PREC, BN>::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  return cudaSuccess;
}

template <int PREC, int BN>
cudaError_t launch_main(cudaStream_t s, const Operands& o, int S, int M, int N, cplx alpha, cplx* C, long long ldc,
                        float* part, bool conj_out, int* timeouts, TcProbe* probe) {
  using K_ = Cfg<PREC, BN>;
  cudaError_t e;
  if ((e = ensure_attr<PREC, BN>()) != cudaSuccess) return e;
  if ((e = get_encoder()) != cudaSuccess) return e;
  CUtensorMap mA0, mA1, mA2, mB0, mB1, mB2;
  constexpr int KB = K_::KB_BYTES;
  if ((e = make_map(&mA0, o.a0, PREC, o.Mp, o.Krp, BM, KB)) != cudaSuccess) return e;
  if ((e = make_map(&mB0, o.b0, PREC, o.Nrp, o.Krp, BN, KB)) != cudaSuccess) return e;
  mA1 = mA2 = mA0;
  mB1 = mB2 = mB0;
  if (K_::NOPS >= 2) {
    if ((e = make_map(&mA1, o.a1, PREC, o.Mp, o.Krp, BM, KB)) != cudaSuccess) return e;
    if ((e = make_map(&mB1, o.b1, PREC, o.Nrp, o.Krp, BN, KB)) != cudaSuccess) return e;
  }
  if (K_::NOPS == 3) {
    if ((e = make_map(&mA2, o.a2, PREC, o.Mp, o.Krp, BM, KB)) != cudaSuccess) return e;
    if ((e = make_map(&mB2, o.b2, PREC, o.Nrp, o.Krp, BN, KB)) != cudaSuccess) return e;
  }
  S = eff_splits(o.kb_total, S);
  const int kps = (o.kb_total + S - 1) / S;
  const int n_tiles = (int)(o.Nrp / BN), m_tiles = (int)(o.Mp / BM);
  const long long tiles = (long long)n_tiles * m_tiles * S;
  if (tiles >= (1LL << 31)) return cudaErrorInvalidValue;
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  }
  const unsigned grid = (unsigned)std::min<long long>(tiles, nsm);
  const int unit = alpha.x == 1.0 && alpha.y == 0.0;
  if (probe) {
    probe->Mp = o.Mp;
    probe->Nrp = o.Nrp;
    probe->Krp = o.Krp;
    probe->splits = S;
    probe->bn = BN;
    probe->parts = K_::NOPS;
    probe->elem_bytes = K_::ELEM;
    if ((e = cudaEventRecord(probe->ev[0], s)) != cudaSuccess) return e;
  }
  tc_gemm_kernel<PREC, BN><<<grid, NTHREADS, K_::SMEM, s>>>(mA0, mA1, mA2, mB0, mB1, mB2, o.kb_total, kps, n_tiles,
                                                             m_tiles, (int)tiles, M, 2 * N, alpha, C, ldc,
                                                             S > 1 ? part : nullptr, (int)o.Nrp, o.Mp * o.Nrp,
                                                             conj_out ? 1 : 0, unit, timeouts);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (probe && (e = cudaEventRecord(probe->ev[1], s)) != cudaSuccess) return e;
  if (S > 1) {
    if (S >= 64)
      splitk_reduce_warp_kernel<<<grid_for(32LL * M * N), 256, 0, s>>>(part, S, o.Mp * o.Nrp, (int)o.Nrp, M, N, alpha,
                                                                      C, ldc, conj_out ? 1 : 0, unit);
    else
      splitk_reduce_kernel<<<grid_for((long long)M * N), 256, 0, s>>>(part, S, o.Mp * o.Nrp, (int)o.Nrp, M, N,
                                                                      alpha, C, ldc, conj_out ? 1 : 0, unit);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (probe && (e = cudaEventRecord(probe->ev[2], s)) != cudaSuccess) return e;
  return cudaSuccess;
}

template <int PREC>
cudaError_t launch_choice(cudaStream_t s, const Operands& o, TcChoice c, int M, int N, cplx alpha, cplx* C,
                          long long ldc, float* part, bool conj_out, int* timeouts, TcProbe* probe = nullptr) {
  if (c.bn == 128 || o.Nrp % 256 != 0)
    return launch_main<PREC, 128>(s, o, c.splits, M, N, alpha, C, ldc, part, conj_out, timeouts, probe);
  return launch_main<PREC, 256>(s, o, c.splits, M, N, alpha, C, ldc, part, conj_out, timeouts, probe);
}

}  // namespace

// ---------------------------------------------------------------------------
// autotuner: shape -> tile choice, filled by timing every candidate once
// ---------------------------------------------------------------------------
struct TcTuner {
  struct Key {
    int prec, M, N, K;
    bool operator<(const Key& o) const {
      return std::tie(prec, M, N, K) < std::tie(o.prec, o.M, o.N, o.K);
    }
  };
  struct Entry {
    TcChoice choice;
    double us, heuristic_us;
    int candidates;
  };
  std::map<Key, Entry> table;
  std::vector<Key> order;  // insertion order, for reporting
  bool measuring = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};

TcTuner* tc_tuner_create() {
  TcTuner* t = new TcTuner();
  if (cudaEventCreate(&t->e0) != cudaSuccess || cudaEventCreate(&t->e1) != cudaSuccess) {
    delete t;
    return nullptr;
  }
  return t;
}

void tc_tuner_destroy(TcTuner* t) {
  if (!t) return;
  if (t->e0) cudaEventDestroy(t->e0);
  if (t->e1) cudaEventDestroy(t->e1);
  delete t;
}

void tc_tuner_set_measuring(TcTuner* t, bool on) {
  if (t) t->measuring = on;
}

int tc_tuner_size(const TcTuner* t) { return t ? (int)t->order.size() : 0; }

bool tc_tuner_entry(const TcTuner* t, int i, int fields[6], double us[2]) {
  if (!t || i < 0 || i >= (int)t->order.size()) return false;
  const TcTuner::Key& k = t->order[i];
  const TcTuner::Entry& e = t->table.at(k);
  fields[0] = k.prec;
  fields[1] = k.M;
  fields[2] = k.N;
  fields[3] = k.K;
  fields[4] = e.choice.bn;
  fields[5] = e.choice.splits;
  us[0] = e.us;
  us[1] = e.heuristic_us;
  return true;
}

namespace {

template <int PREC>
cudaError_t run(cudaStream_t s, int M, int N, int K, cplx alpha, const cplx* A, long long lda, int opA,
                const cplx* B, long long ldb, int opB, const TcPacked* pre, cplx* C, long long ldc, bool conj_out,
                char* scratch, size_t scratch_bytes, TcTuner* tuner, const TcChoice* force, int* timeouts,
                TcProbe* probe, const TcView* va = nullptr, const TcView* vb = nullptr) {
  if (!timeouts) return cudaErrorInvalidValue;
  using K_ = Cfg<PREC, 128>;  // element size, k-block and parts do not depend on the tile width
  Operands o;
  o.Mp = (M + BM - 1) / BM * BM;
  padded<PREC>(N, K, &o.Nrp, &o.Krp);
  o.kb_total = (int)(o.Krp / K_::BK);
  auto al = [](size_t x) { return (x + 1023) & ~(size_t)1023; };
  const size_t abytes = al((size_t)o.Mp * o.Krp * K_::ELEM);
  const size_t bbytes = pre ? 0 : al((size_t)o.Nrp * o.Krp * K_::ELEM);
  const size_t fixed = K_::NOPS * (abytes + bbytes) + 1024;
  if (fixed > scratch_bytes) return cudaErrorMemoryAllocation;
  const size_t part_room = scratch_bytes - fixed;
  auto part_bytes = [&](int S) { return S > 1 ? al((size_t)S * o.Mp * o.Nrp * 4) : (size_t)0; };
  char* p = (char*)(((uintptr_t)scratch + 1023) & ~(uintptr_t)1023);
  o.a0 = p;
  o.a1 = p + abytes;
  o.a2 = p + 2 * abytes;
  o.b0 = p + K_::NOPS * abytes;
  o.b1 = (char*)o.b0 + bbytes;
  o.b2 = (char*)o.b0 + 2 * bbytes;
  float* part = (float*)((char*)o.b0 + K_::NOPS * bbytes);

  TcChoice choice = heuristic(o.Mp, o.Nrp, o.kb_total);
  const TcTuner::Key key{PREC, M, N, K};
  bool tune_now = false;
  if (tuner) {
    auto it = tuner->table.find(key);
    if (it != tuner->table.end())
      choice = it->second.choice;
    else
      tune_now = tuner->measuring;
  }
  if (force) {
    if (force->bn != 128 && force->bn != 256) return cudaErrorInvalidValue;
    choice = TcChoice{force->bn, eff_splits(o.kb_total, force->splits)};
    tune_now = false;
  }
  if (part_bytes(eff_splits(o.kb_total, choice.splits)) > part_room) return cudaErrorMemoryAllocation;

  // the A operand: a view, or a plain operand as a view (rows m, columns k of op(A))
  TcView pa;
  if (!va) {
    const bool t = (opA & OP_T) != 0;
    pa.p = A;
    pa.conj = (opA & OP_CONJ) ? 1 : 0;
    pa.nr = pa.nc = 1;
    pa.rdim[0] = M;
    pa.cdim[0] = K;
    pa.rstr[0] = t ? 1 : lda;
    pa.cstr[0] = t ? lda : 1;
  }
  const TcView& av = va ? *va : pa;
  if (o.Mp / 32 <= 65535 && o.Mp * o.Krp < (1LL << 40)) {
    const int row_contig = av.rstr[av.nr - 1] == 1 && av.cstr[av.nc - 1] != 1;
    pack_a_tiled_kernel<PREC><<<dim3((unsigned)((o.Krp / 2 + 31) / 32), (unsigned)(o.Mp / 32)), dim3(32, 8), 0, s>>>(
        av, M, K, (int)o.Mp, (int)o.Krp, row_contig, o.a0, o.a1, o.a2);
  } else if (va) {
    return cudaErrorNotSupported;
  } else {
    pack_a_kernel<PREC, unsigned long long><<<grid_for(o.Mp * o.Krp / 2), 256, 0, s>>>(A, lda, opA, M, K, (int)o.Mp,
                                                                                   (int)o.Krp, o.a0, o.a1, o.a2);
  }
  count_launch();
  cudaError_t e;
  if (pre) {
    if (pre->prec != PREC || pre->N != N || pre->K != K) return cudaErrorInvalidValue;
    o.b0 = pre->b0;
    o.b1 = pre->b1;
    o.b2 = pre->b2;
  } else if (vb) {
    if (o.Nrp / 64 > 65535) return cudaErrorNotSupported;
    const int row_contig = vb->rstr[vb->nr - 1] == 1 && vb->cstr[vb->nc - 1] != 1;
    pack_b_tiled_kernel<PREC><<<dim3((unsigned)((o.Krp / 2 + 31) / 32), (unsigned)(o.Nrp / 64)), dim3(32, 8), 0, s>>>(
        *vb, N, K, (int)o.Nrp, (int)o.Krp, row_contig, o.b0, o.b1, o.b2);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  } else if ((e = pack_b_any<PREC>(s, B, ldb, opB, N, K, o.Nrp, o.Krp, o.b0, o.b1, o.b2)) != cudaSuccess) {
    return e;
  }
  if (tune_now) {
    // time every candidate (best of two runs each) on the packed operands
    auto time_one = [&](TcChoice c, double* us) -> cudaError_t {
      double best = 1e30;
      for (int rep = 0; rep < 2; ++rep) {
        cudaError_t r;
        if ((r = cudaEventRecord(tuner->e0, s)) != cudaSuccess) return r;
        if ((r = launch_choice<PREC>(s, o, c, M, N, alpha, C, ldc, part, conj_out, timeouts)) != cudaSuccess)
          return r;
        if ((r = cudaEventRecord(tuner->e1, s)) != cudaSuccess) return r;
        if ((r = cudaEventSynchronize(tuner->e1)) != cudaSuccess) return r;
        float ms = 0;
        if ((r = cudaEventElapsedTime(&ms, tuner->e0, tuner->e1)) != cudaSuccess) return r;
        best = std::min(best, 1e3 * (double)ms);
      }
      *us = best;
      return cudaSuccess;
    };
    TcTuner::Entry ent{choice, 0.0, 0.0, 0};
    if ((e = time_one(choice, &ent.heuristic_us)) != cudaSuccess) return e;
    ent.us = ent.heuristic_us;
    ent.candidates = 1;
    static const int bns[2] = {128, 256};
    for (int bn : bns) {
      if (o.Nrp % bn != 0) continue;
      // powers of two, and the counts that fill one to four whole waves
      const long long tiles = (o.Mp / BM) * (o.Nrp / bn);
      std::vector<int> splits = {1, 2, 4, 8, 16, 32};
      for (int w = 1; w <= 4; ++w) {
        const int S = (int)((long long)w * NSM / tiles);
        if (S > 1 && std::find(splits.begin(), splits.end(), S) == splits.end()) splits.push_back(S);
      }
      for (int S0 : splits) {
        const int S = eff_splits(o.kb_total, S0);
        if (S != S0 && S0 != 1) continue;        // duplicate of a smaller split count
        if (S > 1 && o.kb_total / S < 2) continue;  // splits of a single k-block
        if (part_bytes(S) > part_room) continue;
        const TcChoice c{bn, S};
        if (c.bn == ent.choice.bn && c.splits == eff_splits(o.kb_total, choice.splits)) continue;
        double us = 0;
        if ((e = time_one(c, &us)) != cudaSuccess) return e;
        ++ent.candidates;
        if (us < ent.us) {
          ent.us = us;
          ent.choice = c;
        }
      }
    }
    tuner->table[key] = ent;
    tuner->order.push_back(key);
    choice = ent.choice;
  }
  if (probe) probe->packed_b = pre != nullptr;
  return launch_choice<PREC>(s, o, choice, M, N, alpha, C, ldc, part, conj_out, timeouts, probe);
}


}  // namespace

cudaError_t tc_encode_bf16_map(CUtensorMap* map, void* base, long long rows, long long kcols, int box_rows) {
  cudaError_t e = get_encoder();
  if (e != cudaSuccess) return e;
  return make_map(map, base, PREC_BF16X3, rows, kcols, box_rows);
}

namespace {

// dispatch on the precision mode (a run<> instantiation per mode)
template <typename F>
cudaError_t by_prec(int prec, F&& f) {
  switch (prec) {
    case PREC_TF32:
      return f(std::integral_constant<int, PREC_TF32>());
    case PREC_BF16X3:
      return f(std::integral_constant<int, PREC_BF16X3>());
    case PREC_BF16X6:
      return f(std::integral_constant<int, PREC_BF16X6>());
    default:
      return cudaErrorNotSupported;
  }
}

}  // namespace

cudaError_t tc_zgemm(cudaStream_t s, int prec, int M, int N, int K, cplx alpha, const cplx* A, long long lda,
                     int opA, const cplx* B, long long ldb, int opB, cplx* C, long long ldc, cplx* scratch,
                     long long scratch_elems, long long scratch_top, int* timeouts, TcTuner* tuner,
                     const TcChoice* force, TcProbe* probe) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaErrorNotSupported;
  char* base = (char*)(scratch + scratch_top);
  const size_t bytes = (size_t)(scratch_elems - scratch_top) * sizeof(cplx);
  return by_prec(prec, [&](auto P) {
    return run<decltype(P)::value>(s, M, N, K, alpha, A, lda, opA, B, ldb, opB, nullptr, C, ldc, false, base, bytes,
                                   tuner, force, timeouts, probe);
  });
}

cudaError_t tc_zgemm_views(cudaStream_t s, int prec, int M, int N, int K, cplx alpha, const TcView* va,
                           const cplx* A, long long lda, int opA, const TcView* vb, const cplx* B, long long ldb,
                           int opB, cplx* C, long long ldc, cplx* scratch, long long scratch_elems,
                           long long scratch_top, int* timeouts, TcTuner* tuner, TcProbe* probe) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaErrorNotSupported;
  char* base = (char*)(scratch + scratch_top);
  const size_t bytes = (size_t)(scratch_elems - scratch_top) * sizeof(cplx);
  return by_prec(prec, [&](auto P) {
    return run<decltype(P)::value>(s, M, N, K, alpha, A, lda, opA, B, ldb, opB, nullptr, C, ldc, false, base, bytes,
                                   tuner, nullptr, timeouts, probe, va, vb);
  });
}

static int n_parts(int prec) { return prec == PREC_TF32 ? 1 : (prec == PREC_BF16X3 ? 2 : 3); }

size_t tc_packed_bytes(int prec, int N, int K) {
  long long Nrp, Krp;
  if (prec == PREC_TF32) {
    padded<PREC_TF32>(N, K, &Nrp, &Krp);
    return (size_t)Nrp * Krp * 4 + 2048;
  }
  padded<PREC_BF16X3>(N, K, &Nrp, &Krp);  // BF16 k-blocks: the same padding for x3 and x6
  return (size_t)n_parts(prec) * ((size_t)Nrp * Krp * 2 + 1024) + 2048;
}

cudaError_t tc_pack_b(cudaStream_t s, int prec, const cplx* B, long long ldb, int opB, int N, int K, void* mem,
                      TcPacked* out) {
  long long Nrp, Krp;
  char* p = (char*)(((uintptr_t)mem + 1023) & ~(uintptr_t)1023);
  out->prec = prec;
  out->N = N;
  out->K = K;
  if (prec == PREC_TF32) {
    padded<PREC_TF32>(N, K, &Nrp, &Krp);
    out->b0 = out->b1 = out->b2 = p;
    return pack_b_any<PREC_TF32>(s, B, ldb, opB, N, K, Nrp, Krp, out->b0, out->b1, out->b2);
  }
  if (prec == PREC_BF16X3 || prec == PREC_BF16X6) {
    padded<PREC_BF16X3>(N, K, &Nrp, &Krp);
    const size_t part = ((size_t)Nrp * Krp * 2 + 1023) & ~(size_t)1023;
    out->b0 = p;
    out->b1 = p + part;
    out->b2 = prec == PREC_BF16X6 ? p + 2 * part : out->b1;
    if (prec == PREC_BF16X3) return pack_b_any<PREC_BF16X3>(s, B, ldb, opB, N, K, Nrp, Krp, out->b0, out->b1, out->b2);
    return pack_b_any<PREC_BF16X6>(s, B, ldb, opB, N, K, Nrp, Krp, out->b0, out->b1, out->b2);
  }
  return cudaErrorNotSupported;
}

cudaError_t tc_zgemm_packed(cudaStream_t s, int prec, int M, cplx alpha, const cplx* A, long long lda, int opA,
                            const TcPacked& B, cplx* C, long long ldc, bool conj_out, cplx* scratch,
                            long long scratch_elems, long long scratch_top, int* timeouts, TcTuner* tuner,
                            TcProbe* probe) {
  if (M <= 0) return cudaSuccess;
  char* base = (char*)(scratch + scratch_top);
  const size_t bytes = (size_t)(scratch_elems - scratch_top) * sizeof(cplx);
  return by_prec(prec, [&](auto P) {
    return run<decltype(P)::value>(s, M, (int)B.N, (int)B.K, alpha, A, lda, opA, nullptr, 0, 0, &B, C, ldc, conj_out,
                                   base, bytes, tuner, nullptr, timeouts, probe);
  });
}

cudaError_t tc_init() {
  cudaError_t e;
  if ((e = ensure_attr<PREC_TF32, 128>()) != cudaSuccess) return e;
  if ((e = ensure_attr<PREC_TF32, 256>()) != cudaSuccess) return e;
  if ((e = ensure_attr<PREC_BF16X3, 128>()) != cudaSuccess) return e;
  if ((e = ensure_attr<PREC_BF16X3, 256>()) != cudaSuccess) return e;
  if ((e = ensure_attr<PREC_BF16X6, 128>()) != cudaSuccess) return e;
  return get_encoder();
}
