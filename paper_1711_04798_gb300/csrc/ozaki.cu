// FP64-accurate complex GEMM on the tcgen05 tensor cores.
//
// GB300 runs FP64 at a small fraction of its tensor-core rate, so the FP64
// products of the projector step (CholeskyQR Grams and applies of k x K
// matrices), and in the FP64-accurate form every contraction product, are
// computed here by exact splitting into integer digit planes,
// after the error-free splitting of Ozaki, Ogita, Oishi and Rump (2012),
// arranged for BF16 tensor cores with FP32 accumulation:
//
//  * the complex product is the real product of the embedding of tc_gemm.cu:
//    Ar (M x 2K) and Br^T (2N x 2K), both K-major;
//  * every row r of Ar and of Br^T gets a power-of-two bound 2^e_r above its
//    largest magnitude, and each element is rounded to 55 fraction bits below
//    it, x = 2^e_r sum_{s<7} d_s 2^(-7-8s), with balanced base-256 digits d_s
//    in [-128, 128] (exact in BF16), taken from the FP64 bit pattern with
//    integer operations;
//  * the digit-plane products P_st = sum_k dA_s dB_t are sums of integers below
//    2^14 in magnitude; those of equal weight g = s + t accumulate in one FP32
//    accumulator, and over a chunk of 128 reals of K a group (at most 7 pairs)
//    stays below 2^24, so the tensor cores' FP32 sums are exact.  The 28
//    pairs with s + t <= 6 are computed; the others weigh below 2^-53 of the
//    terms' scale;
//  * after each chunk the seven group sums leave tensor memory: groups 0..3
//    combine exactly in 64-bit integers, I += 2^24 P_0 + 2^16 P_1 + 2^8 P_2 +
//    P_3 (below 2^49 per chunk), groups 4..6 (weight 2^-32 and below) in FP32,
//    u += P_4 + 2^-8 (P_5 + 2^-8 P_6), whose rounding weighs below 2^-56;
//  * Cr = 2^(ea + eb - 38) (I + 2^-8 u): the only rounding to FP64 is the last.
//
// The error is that of the 55-bit rounding of each element relative to its
// row's bound (and the dropped digit pairs), i.e. relative to max|a| max|b|
// of the rows involved rather than to sum |a||b|: FP64-level for rows
// without a wide spread of magnitudes, as the projector step's are.
//
// One CTA computes a 128 x 32 or 128 x 64 tile of Cr over a range of K
// chunks: warp 0 issues the TMA loads (per stage one A digit plane and the B
// planes it pairs with), warp 1 the tcgen05.mma, the other warps (four or
// eight) drain the seven group accumulators after each chunk.  Ranges of K
// are split over the grid; the exact partials (I, u) are summed by a second
// kernel.
#include <cuda_bf16.h>

#include "tc_gemm.h"
#include "tc_ptx.h"

namespace {

constexpr int OZ_DIGITS = 7;                          // base-256 digits per element
constexpr int OZ_GROUPS = 7;                          // weights g = s + t = 0..6
constexpr int OZ_BM = 128;                            // output tile rows
constexpr int OZ_BK = 64;                             // bf16 elements per k-block (128 bytes)
constexpr int OZ_CHUNK = 128;                         // reals of K per exact FP32 chunk
constexpr int OZ_KB_PER_CHUNK = OZ_CHUNK / OZ_BK;     // 2
constexpr int OZ_A_BYTES = OZ_BM * 128;               // one A plane k-block: 16 KB
constexpr int OZ_TMEM_COLS = 512;
static_assert(OZ_GROUPS == OZ_DIGITS, "weights 0..6 of the digit pairs s + t <= 6");

// Output tiles of 128 x BN real columns.  BN = 32: two sets of the seven group
// accumulators (224 of 256 columns each), so that a chunk's products run
// while the epilogue drains the previous chunk; four 44 KB stages; four
// epilogue warps.  BN = 64: one set (448 columns), the products of a chunk
// wait for the previous chunk's drain, but each MMA does twice the work (the
// narrow MMAs' issue bounds the 32-wide tile); three 72 KB stages; eight
// epilogue warps (two per lane quarter, 32 columns each).
template <int BN>
struct OzTile {
  static constexpr int B_BYTES = BN * 128;                       // one B plane k-block
  static constexpr int STAGE = OZ_A_BYTES + OZ_DIGITS * B_BYTES;  // 44 KB / 72 KB
  static constexpr int STAGES = BN == 32 ? 4 : 3;
  static constexpr int SETS = BN == 32 ? 2 : 1;
  static constexpr int ACC_COLS = BN == 32 ? 256 : 512;          // columns per accumulator set
  static constexpr int EPI_WARPS = BN / 8;
  static constexpr int THREADS = 64 + 32 * EPI_WARPS;            // producer, MMA issuer, epilogue
  static constexpr int SMEM = STAGES * STAGE + 1024 + 256;
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                    ((uint32_t)(OZ_BM >> 4) << 24);  // FP32 += BF16 x BF16, K-major
  static_assert(OZ_GROUPS * BN <= ACC_COLS && SETS * ACC_COLS <= OZ_TMEM_COLS, "accumulators fit");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

__device__ __forceinline__ void umma_bf16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}

// The same MMA with the A operand kept in the tensor core's collector buffer
// across consecutive MMAs that share it: FILL reads A from shared memory and
// keeps it, USE takes the kept A, LAST takes it and releases the buffer.
enum { COLL_FILL = 1, COLL_USE = 2, COLL_LAST = 3 };
template <int COLL>
__device__ __forceinline__ void umma_bf16_coll(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc,
                                               uint32_t accum) {
  if constexpr (COLL == COLL_FILL)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
  else if constexpr (COLL == COLL_USE)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16.collector::a::use [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
}

// 2^k for k in the normal range, built from its bit pattern
__device__ __forceinline__ double pow2(int k) {
  k = k < -1022 ? -1022 : (k > 1023 ? 1023 : k);
  return __longlong_as_double((long long)(k + 1023) << 52);
}

// biased binary64 exponent of x (0 for zero and subnormals)
__device__ __forceinline__ int bexp(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }

// balanced base-256 digits of x / 2^e (|x| < 2^e), rounded to 55 fraction bits:
// x = 2^e sum_s d[s] 2^(-7-8s), d[s] in [-128, 128]
__device__ __forceinline__ void digits7(double x, int e, int (&d)[OZ_DIGITS]) {
  const long long b = __double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  long long v = 0;
  if (E != 0) {
    const long long m = (b & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
    const int shift = (E - 1023) - e + 3;  // v = x 2^(55 - e) = m 2^shift, shift <= 2
    if (shift >= 0)
      v = m << shift;
    else if (shift > -60)
      v = (m + (1LL << (-shift - 1))) >> (-shift);
    if (b < 0) v = -v;
  }
#pragma unroll
  for (int s = OZ_DIGITS - 1; s >= 1; --s) {
    const int dd = (int)(((v + 128) & 255) - 128);
    d[s] = dd;
    v = (v - dd) >> 8;  // exact: v - dd is a multiple of 256
  }
  d[0] = (int)v;
}

__device__ __forceinline__ cplx oz_load(const cplx* X, long long ld, int op, int r, int c) {
  // element (r, c) of op(X)
  cplx v = (op & OP_T) ? X[(long long)c * ld + r] : X[(long long)r * ld + c];
  if (op & OP_CONJ) v.y = -v.y;
  return v;
}

// Both operands' exponents and digit planes in one launch.  Block b < Mp takes
// row b of op(A) (M x K complex): e = (largest biased exponent of the row) -
// 1022, the power-of-two bound of that row of Ar (0 for rows at or beyond M
// and for zero rows), and digit plane s of Ar is [Mp x Krp] bf16 at
// pa + s * Mp * Krp.  Block Mp + n takes column n of op(B) (K x N) the same
// way: its bound goes to rows 2n and 2n+1 of Br^T, and complex (k, n) gives
// row 2n (Re, -Im) and row 2n+1 (Im, Re) at columns 2k, 2k+1 of each plane of
// Br^T [Nrp x Krp].  The block first reduces the row's largest exponent, then
// writes its digits; the row is read twice, the second time from cache.
constexpr int OZ_PREP_THREADS = 128;
__global__ void __launch_bounds__(OZ_PREP_THREADS)
    oz_prep_kernel(const cplx* __restrict__ A, long long lda, int opA, const cplx* __restrict__ B, long long ldb,
                   int opB, int M, int N, int K, int Mp, int Nrp, int Krp, int* __restrict__ ea, int* __restrict__ eb,
                   __nv_bfloat16* __restrict__ pa, __nv_bfloat16* __restrict__ pb) {
  __shared__ int s_e[OZ_PREP_THREADS / 32];
  const bool is_a = (int)blockIdx.x < Mp;
  const int r = is_a ? (int)blockIdx.x : (int)blockIdx.x - Mp;  // row of op(A), or column of op(B)
  const bool live = is_a ? r < M : r < N;
  auto load = [&](int c) {
    return is_a ? oz_load(A, lda, opA, r, c) : oz_load(B, ldb, opB, c, r);
  };
  int E = 0;
  if (live)
    for (int c = threadIdx.x; c < K; c += OZ_PREP_THREADS) {
      const cplx v = load(c);
      E = max(E, max(bexp(v.x), bexp(v.y)));
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) E = max(E, __shfl_xor_sync(0xffffffffu, E, o));
  if ((threadIdx.x & 31) == 0) s_e[threadIdx.x >> 5] = E;
  __syncthreads();
  E = s_e[0];
#pragma unroll
  for (int w = 1; w < OZ_PREP_THREADS / 32; ++w) E = max(E, s_e[w]);
  const int e = E ? E - 1022 : 0;
  if (threadIdx.x == 0) {
    if (is_a)
      ea[r] = e;
    else
      eb[2 * r] = eb[2 * r + 1] = e;
  }
  const long long kc = Krp / 2;
  const long long plane = is_a ? (long long)Mp * Krp : (long long)Nrp * Krp;
  for (int c = threadIdx.x; c < kc; c += OZ_PREP_THREADS) {
    cplx v = make_double2(0.0, 0.0);
    if (live && c < K) v = load(c);
    int dr[OZ_DIGITS], di[OZ_DIGITS];
    digits7(v.x, e, dr);
    digits7(v.y, e, di);
    if (is_a) {
      __nv_bfloat162* out = (__nv_bfloat162*)(pa + (long long)r * Krp + 2LL * c);
#pragma unroll
      for (int s = 0; s < OZ_DIGITS; ++s)
        out[s * plane / 2] = __halves2bfloat162(__float2bfloat16_rn((float)dr[s]), __float2bfloat16_rn((float)di[s]));
    } else {
      __nv_bfloat162* r0 = (__nv_bfloat162*)(pb + (long long)(2 * r) * Krp + 2LL * c);
      __nv_bfloat162* r1 = (__nv_bfloat162*)(pb + (long long)(2 * r + 1) * Krp + 2LL * c);
#pragma unroll
      for (int s = 0; s < OZ_DIGITS; ++s) {
        const __nv_bfloat16 re = __float2bfloat16_rn((float)dr[s]), im = __float2bfloat16_rn((float)di[s]);
        r0[s * plane / 2] = __halves2bfloat162(re, __float2bfloat16_rn((float)-di[s]));
        r1[s * plane / 2] = __halves2bfloat162(im, re);
      }
    }
  }
}

// Cr element from its exact sums: 2^(ea + eb - 38) (I + 2^-8 u)
__device__ __forceinline__ double oz_value(long long I, float u, int ea, int eb) {
  return ((double)I + (double)u * (1.0 / 256.0)) * pow2(ea + eb - 38);
}

template <int BN>
__global__ void __launch_bounds__(OzTile<BN>::THREADS, 1)
    oz_gemm_kernel(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB, int Mp, int Nrp,
                   int chunks_total, int chunks_per_split, int M, int N, const int* __restrict__ ea,
                   const int* __restrict__ eb, cplx* __restrict__ C, long long ldc, long long* __restrict__ pI,
                   float* __restrict__ pU, int* __restrict__ timeouts) {
  using T = OzTile<BN>;
  constexpr int OZ_STAGES = T::STAGES, OZ_STAGE = T::STAGE, OZ_B_BYTES = T::B_BYTES, SETS = T::SETS;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + OZ_STAGES * OZ_STAGE);
  uint64_t* empty = full + OZ_STAGES;
  uint64_t* acc_full = empty + OZ_STAGES;  // [2], per accumulator set
  uint64_t* acc_empty = acc_full + 2;      // [2]
  uint64_t* mma_done = acc_empty + 2;
  uint32_t* tmem_slot = (uint32_t*)(mma_done + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_tile = blockIdx.x, m_tile = blockIdx.y, split = blockIdx.z;
  const int c0 = split * chunks_per_split;
  const int nch = min(chunks_total, c0 + chunks_per_split) - c0;  // >= 1 by construction
  const int nstage = nch * OZ_KB_PER_CHUNK * OZ_DIGITS;             // (chunk, k-block, A digit)

  if (threadIdx.x == 0) {
    for (int s = 0; s < OZ_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], T::EPI_WARPS);  // one arrival per epilogue warp
    }
    mbar_init(mma_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(OZ_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer: stage q = (chunk, k-block, s) holds A plane s and B planes 0..6-s
    int issued = 0;
    for (int q = 0; q < nstage; ++q) {
      const int slot = q % OZ_STAGES, round = q / OZ_STAGES;
      const int s = q % OZ_DIGITS, kb = (c0 * OZ_KB_PER_CHUNK) + q / OZ_DIGITS;
      if (!mbar_wait(&empty[slot], (round & 1) ^ 1)) {
        atomicAdd(timeouts, 1);
        break;
      }
      unsigned char* st = smem + slot * OZ_STAGE;
      mbar_expect_tx(&full[slot], OZ_A_BYTES + (OZ_DIGITS - s) * OZ_B_BYTES);
      tma_load_2d(st, &mA, &full[slot], kb * OZ_BK, s * Mp + m_tile * OZ_BM);
      for (int t = 0; t < OZ_DIGITS - s; ++t)
        tma_load_2d(st + OZ_A_BYTES + t * OZ_B_BYTES, &mB, &full[slot], kb * OZ_BK, t * Nrp + n_tile * BN);
      issued = q + 1;
    }
    // the last loads of every slot have landed before the CTA can leave
    for (int q = max(0, issued - OZ_STAGES); q < issued; ++q)
      if (!mbar_wait(&full[q % OZ_STAGES], (q / OZ_STAGES) & 1)) atomicAdd(timeouts, 1);
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: group g = s + t of chunk c accumulates in tensor-memory
    // columns ACC_COLS (c % SETS) + BN g .. (with two sets chunk c's products
    // run while the epilogue drains chunk c - 1)
    bool ok = true;
    for (int q = 0; q < nstage && ok; ++q) {
      const int slot = q % OZ_STAGES, round = q / OZ_STAGES;
      const int s = q % OZ_DIGITS, kbc = (q / OZ_DIGITS) % OZ_KB_PER_CHUNK, c = q / (OZ_DIGITS * OZ_KB_PER_CHUNK);
      const bool chunk_start = kbc == 0 && s == 0;
      // the set was drained: chunk c - SETS was that set's drain number c/SETS - 1
      if (chunk_start && c >= SETS && !mbar_wait(&acc_empty[c % SETS], ((c / SETS) - 1) & 1)) {
        atomicAdd(timeouts, 1);
        ok = false;
        break;
      }
      if (!mbar_wait(&full[slot], round & 1)) {
        atomicAdd(timeouts, 1);
        ok = false;
        break;
      }
      fence_after();
      const uint32_t a = smem_u32(smem + slot * OZ_STAGE);
      // per k-step, A plane s meets the B planes t = 0 .. 6 - s in turn (group
      // s + t each): A is read from shared memory once per k-step and kept in
      // the collector buffer for the other B planes
      const int nt = OZ_DIGITS - s;
      const uint32_t d0 = tmem + (uint32_t)((c % SETS) * T::ACC_COLS + s * BN);
#pragma unroll
      for (int ks = 0; ks < OZ_BK / 16; ++ks) {
        const uint64_t ad = sdesc(a + ks * 32);
        const uint32_t acc = (chunk_start && ks == 0) ? 0u : 1u;
        const uint32_t b0 = a + OZ_A_BYTES + ks * 32;
        if (nt == 1) {
          umma_bf16(d0, ad, sdesc(b0), T::IDESC, acc);
          continue;
        }
        umma_bf16_coll<COLL_FILL>(d0, ad, sdesc(b0), T::IDESC, acc);
        for (int t = 1; t < nt - 1; ++t)
          umma_bf16_coll<COLL_USE>(d0 + t * BN, ad, sdesc(b0 + t * OZ_B_BYTES), T::IDESC, acc);
        umma_bf16_coll<COLL_LAST>(d0 + (nt - 1) * BN, ad, sdesc(b0 + (nt - 1) * OZ_B_BYTES), T::IDESC, acc);
      }
      umma_commit(&empty[slot]);  // frees the slot when these MMAs are done
      if (kbc == OZ_KB_PER_CHUNK - 1 && s == OZ_DIGITS - 1) umma_commit(&acc_full[c % SETS]);
    }
    // every MMA issued has completed before the accumulators are released
    umma_commit(mma_done);
    if (!mbar_wait(mma_done, 0)) atomicAdd(timeouts, 1);
  } else if (warp >= 2) {
    // epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. (the rows of its
    // quarter), columns 32 h .. 32 h + 31 of each group (h = 0, and 1 for the
    // second four epilogue warps of BN = 64)
    constexpr int EC = 32;  // columns per epilogue thread
    const int q4 = warp & 3, h = (warp - 2) >> 2;
    const int row = m_tile * OZ_BM + 32 * q4 + lane;
    const uint32_t trow = tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(EC * h);
    long long I[EC];
    float u[EC];
#pragma unroll
    for (int j = 0; j < EC; ++j) {
      I[j] = 0;
      u[j] = 0.0f;
    }
    bool ok = true;
    for (int c = 0; c < nch; ++c) {
      const bool ready = mbar_wait(&acc_full[c % SETS], (c / SETS) & 1);
      if (!ready) {
        if (lane == 0) atomicAdd(timeouts, 1);
        ok = false;
        break;
      }
      fence_after();
      const uint32_t tset = trow + (uint32_t)((c % SETS) * T::ACC_COLS);
      // two halves of 16 columns (fewer live registers beside the running sums)
#pragma unroll
      for (int hf = 0; hf < 2; ++hf) {
        float v[16], t[16];
        // groups 0..3: exact integers (below 2^24) into the 64-bit sum
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          tmem_ld16(tset + g * BN + 16 * hf, v);
#pragma unroll
          for (int j = 0; j < 16; ++j) I[16 * hf + j] += (long long)__float2int_rn(v[j]) << (8 * (3 - g));
        }
        // groups 4..6 (weight 2^-32 and below relative to group 0): FP32
        tmem_ld16(tset + 6 * BN + 16 * hf, t);
        tmem_ld16(tset + 5 * BN + 16 * hf, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) t[j] = fmaf(t[j], 1.0f / 256.0f, v[j]);
        tmem_ld16(tset + 4 * BN + 16 * hf, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) u[16 * hf + j] += fmaf(t[j], 1.0f / 256.0f, v[j]);
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[c % SETS]);
    }
    if (ok) {
      const int col0 = n_tile * BN + EC * h;
      if (pI) {
        // exact partial sums of this K range
        const long long base = ((long long)split * Mp + row) * Nrp + col0;
#pragma unroll
        for (int j = 0; j < EC; ++j) {
          pI[base + j] = I[j];
          pU[base + j] = u[j];
        }
      } else if (row < M) {
        const int er = ea[row];
#pragma unroll
        for (int j = 0; j < EC; j += 2) {
          const int n = (col0 + j) >> 1;
          if (n < N)
            C[(long long)row * ldc + n] = make_double2(oz_value(I[j], u[j], er, eb[col0 + j]),
                                                       oz_value(I[j + 1], u[j + 1], er, eb[col0 + j + 1]));
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS) : "memory");
  }
}

// C[m, n] from the S exact partials of (I, u) (integer sums are exact; u in FP32)
__global__ void oz_reduce_kernel(const long long* __restrict__ pI, const float* __restrict__ pU, int S, int Mp,
                                 int Nrp, int M, int N, const int* __restrict__ ea, const int* __restrict__ eb,
                                 cplx* __restrict__ C, long long ldc) {
  const long long total = (long long)M * N, pstride = (long long)Mp * Nrp;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(e / N), n = (int)(e - (long long)m * N);
    long long I0 = 0, I1 = 0;
    float u0 = 0.0f, u1 = 0.0f;
    for (int z = 0; z < S; ++z) {
      const long long o = z * pstride + (long long)m * Nrp + 2 * n;
      I0 += pI[o];
      I1 += pI[o + 1];
      u0 += pU[o];
      u1 += pU[o + 1];
    }
    C[(long long)m * ldc + n] = make_double2(oz_value(I0, u0, ea[m], eb[2 * n]), oz_value(I1, u1, ea[m], eb[2 * n + 1]));
  }
}

unsigned oz_grid(long long n) {
  long long b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 152 * 16) b = 152 * 16;
  return (unsigned)b;
}

struct OzLayout {
  int Mp, Nrp, Krp, chunks, S, cps, bn;
  size_t off_ea, off_eb, off_a, off_b, off_pi, off_pu, total;
};

OzLayout oz_layout(int M, int N, int K) {
  OzLayout L;
  L.Mp = (M + OZ_BM - 1) / OZ_BM * OZ_BM;
  L.Krp = (2 * K + OZ_CHUNK - 1) / OZ_CHUNK * OZ_CHUNK;
  L.chunks = L.Krp / OZ_CHUNK;
  // tile width and chunks per CTA: the fewest chunk-times over whole waves of
  // CTAs (152 SMs, one CTA each), counting a CTA's start (barriers, tensor
  // memory, the pipeline's fill) as one chunk-time and, for K splits, the
  // exact partials' round trip through memory (24 bytes per output element
  // and split, about 16 MB per chunk-time).  A chunk of a 64-wide tile takes
  // about the time of a 32-wide one (measured: its MMAs do twice the work at
  // the same issue rate, its drain is not overlapped).  Ties: the wider tile,
  // the fewer K splits.
  double best = -1.0;
  for (int bn = 64; bn >= 32; bn -= 32) {
    const int Nrp = (2 * N + bn - 1) / bn * bn;
    const long long tiles = (long long)(L.Mp / OZ_BM) * (Nrp / bn);
    for (int cps = L.chunks; cps >= 1; --cps) {
      const long long S = (L.chunks + cps - 1) / cps;
      const double partials = S > 1 ? 24.0 * (double)S * L.Mp * Nrp / 16.0e6 : 0.0;
      const double cost = (double)((tiles * S + 151) / 152) * (cps + 1) + partials;
      if (best < 0 || cost < best) {
        best = cost;
        L.bn = bn;
        L.Nrp = Nrp;
        L.cps = cps;
      }
    }
  }
  L.S = (L.chunks + L.cps - 1) / L.cps;
  auto al = [](size_t x) { return (x + 1023) & ~(size_t)1023; };
  size_t o = 0;
  L.off_ea = o;
  o += al(sizeof(int) * L.Mp);
  L.off_eb = o;
  o += al(sizeof(int) * L.Nrp);
  L.off_a = o;
  o += al((size_t)OZ_DIGITS * L.Mp * L.Krp * 2);
  L.off_b = o;
  o += al((size_t)OZ_DIGITS * L.Nrp * L.Krp * 2);
  L.off_pi = o;
  o += L.S > 1 ? al((size_t)L.S * L.Mp * L.Nrp * 8) : 0;
  L.off_pu = o;
  o += L.S > 1 ? al((size_t)L.S * L.Mp * L.Nrp * 4) : 0;
  L.total = o + 1024;
  return L;
}

}  // namespace

size_t oz_work_bytes(int M, int N, int K) { return oz_layout(M, N, K).total; }

cudaError_t oz_zgemm(cudaStream_t s, int M, int N, int K, const cplx* A, long long lda, int opA, const cplx* B,
                     long long ldb, int opB, cplx* C, long long ldc, void* work, size_t work_bytes, int* timeouts) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  if (!timeouts) return cudaErrorInvalidValue;
  const OzLayout L = oz_layout(M, N, K);
  if (!work || work_bytes < L.total) return cudaErrorMemoryAllocation;
  static bool attr = false;
  cudaError_t e;
  if (!attr) {
    if ((e = cudaFuncSetAttribute(oz_gemm_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  OzTile<32>::SMEM)) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(oz_gemm_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  OzTile<64>::SMEM)) != cudaSuccess)
      return e;
    attr = true;
  }
  char* base = (char*)(((uintptr_t)work + 1023) & ~(uintptr_t)1023);
  int* ea = (int*)(base + L.off_ea);
  int* eb = (int*)(base + L.off_eb);
  __nv_bfloat16* pa = (__nv_bfloat16*)(base + L.off_a);
  __nv_bfloat16* pb = (__nv_bfloat16*)(base + L.off_b);
  long long* pI = L.S > 1 ? (long long*)(base + L.off_pi) : nullptr;
  float* pU = L.S > 1 ? (float*)(base + L.off_pu) : nullptr;
  oz_prep_kernel<<<(unsigned)(L.Mp + L.Nrp / 2), OZ_PREP_THREADS, 0, s>>>(A, lda, opA, B, ldb, opB, M, N, K, L.Mp,
                                                                          L.Nrp, L.Krp, ea, eb, pa, pb);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  CUtensorMap mA, mB;
  if ((e = tc_encode_bf16_map(&mA, pa, (long long)OZ_DIGITS * L.Mp, L.Krp, OZ_BM)) != cudaSuccess) return e;
  if ((e = tc_encode_bf16_map(&mB, pb, (long long)OZ_DIGITS * L.Nrp, L.Krp, L.bn)) != cudaSuccess) return e;
  dim3 grid((unsigned)(L.Nrp / L.bn), (unsigned)(L.Mp / OZ_BM), (unsigned)L.S);
  if (L.bn == 64)
    oz_gemm_kernel<64><<<grid, OzTile<64>::THREADS, OzTile<64>::SMEM, s>>>(mA, mB, L.Mp, L.Nrp, L.chunks, L.cps, M,
                                                                          N, ea, eb, C, ldc, pI, pU, timeouts);
  else
    oz_gemm_kernel<32><<<grid, OzTile<32>::THREADS, OzTile<32>::SMEM, s>>>(mA, mB, L.Mp, L.Nrp, L.chunks, L.cps, M,
                                                                          N, ea, eb, C, ldc, pI, pU, timeouts);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (L.S > 1) {
    oz_reduce_kernel<<<oz_grid((long long)M * N), 256, 0, s>>>(pI, pU, L.S, L.Mp, L.Nrp, M, N, ea, eb, C, ldc);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}
