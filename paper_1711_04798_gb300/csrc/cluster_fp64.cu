// FP64 pieces of the projector step on one thread-block cluster.
//
// GB300 executes FP64 at a small fraction of its FP32 rate per SM, so a
// k x k Jacobi SVD or Cholesky factorisation on a single CTA is bound by one
// SM's FP64 units, while spreading it over a grid pays a global-memory
// barrier per step.  Here the rows are distributed over the CTAs of one
// cluster (row i lives in the shared memory of CTA i mod csize), warps read
// and write partner rows through distributed shared memory, and steps are
// separated by the hardware cluster barrier.  The pair schedule and the
// arithmetic are those of the grid-wide kernels (kernels.cu, cholqr.cu).
#include <cooperative_groups.h>

#include "ctm_internal.h"

namespace cg = cooperative_groups;

namespace {

constexpr int CL_THREADS = 256;         // 8 warps per CTA (Cholesky): FP64 pipe occupancy
constexpr int JC_THREADS = 256;         // Jacobi: 8 warps per CTA, two per row pair
constexpr int CL_SMEM = 200 * 1024;     // dynamic shared memory bound per CTA
int g_csize = 0;                        // CTAs per cluster (16 if schedulable, else 8)

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sums of four values over a warp with 6 FP64 additions per lane instead of
// 20: the first two butterfly levels halve the values each lane carries.  On
// return lane 0 holds the total of a, lane 8 of b, lane 16 of c, lane 24 of d.
__device__ __forceinline__ double warp_sum4(double a, double b, double c, double d) {
  const int lane = threadIdx.x & 31;
  const bool up = lane & 16;
  double k1 = up ? c : a, k2 = up ? d : b;
  k1 += __shfl_xor_sync(0xffffffffu, up ? a : c, 16);
  k2 += __shfl_xor_sync(0xffffffffu, up ? b : d, 16);
  const bool b3 = lane & 8;
  double k = b3 ? k2 : k1;
  k += __shfl_xor_sync(0xffffffffu, b3 ? k1 : k2, 8);
  k += __shfl_xor_sync(0xffffffffu, k, 4);
  k += __shfl_xor_sync(0xffffffffu, k, 2);
  k += __shfl_xor_sync(0xffffffffu, k, 1);
  return k;
}

__device__ __forceinline__ void pair_of(int r, int p, int np, int rounds, int* i, int* j) {
  int a, b;
  if (p == 0) {
    a = np - 1;
    b = r;
  } else {
    a = (r + p) % rounds;
    b = (r - p + rounds) % rounds;
  }
  if (a > b) { const int t = a; a = b; b = t; }
  *i = a;
  *j = b;
}

// ---------------------------------------------------------------------------
// Double-float arithmetic (a value is an unevaluated sum hi + lo of two FP32
// numbers, about 48 significand bits; Dekker 1971, Knuth's TwoSum): the
// precision form's Jacobi runs its dot products and row rotations on the
// FP32 pipe, which this part executes at 64 times its FP64 rate.  The
// intrinsics below are never contracted into fused multiply-adds, which the
// error-free transformations rely on.
// ---------------------------------------------------------------------------
struct df2 {
  float h, l;
};

__device__ __forceinline__ df2 df_of(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ double df_val(df2 a) { return (double)a.h + (double)a.l; }

// s + e = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fadd_rn(s, -a);
  e = __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -bb)), __fadd_rn(b, -bb));
}

// acc += a b: the leading product exactly (its rounding error by an FMA), the
// cross terms and the tails in FP32, the leading sum's rounding error carried
// into acc.l
__device__ __forceinline__ void acc_mul(df2& acc, df2 a, df2 b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  float s, t;
  two_sum(acc.h, p, s, t);
  acc.h = s;
  acc.l = __fadd_rn(acc.l, __fadd_rn(t, e));
}

__device__ __forceinline__ df2 df_norm(df2 a) {
  df2 r;
  two_sum(a.h, a.l, r.h, r.l);
  return r;
}

__device__ __forceinline__ df2 df_negate(df2 a) { return {-a.h, -a.l}; }

// a complex element of a row: (Re hi, Re lo, Im hi, Im lo)
__device__ __forceinline__ float4 df_elem(cplx x) {
  const df2 r = df_of(x.x), i = df_of(x.y);
  return make_float4(r.h, r.l, i.h, i.l);
}

__device__ __forceinline__ df2 warp_sum_df(df2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, v.h, o), ol = __shfl_xor_sync(0xffffffffu, v.l, o);
    float s, t;
    two_sum(v.h, oh, s, t);
    v.h = s;
    v.l = __fadd_rn(v.l, __fadd_rn(ol, t));
  }
  return df_norm(v);
}

// One-sided Jacobi on the n rows of G (length m): rows and, with Vt, the rows
// of the accumulated rotation (length n, from the identity, or from Vt itself
// with warm) in the cluster's shared memory.  DF: the rows are held, dotted
// and rotated in double-float arithmetic (the rotation angles stay FP64;
// only with a rotation log, Vt being rebuilt from it in FP64).
template <bool DF>
__global__ void __launch_bounds__(JC_THREADS, 1)
    jacobi_cluster_kernel(cplx* __restrict__ G, int n, int m, long long ldg, cplx* __restrict__ Vt, int max_sweeps,
                          double tol, double4_16a* __restrict__ log, int* sweeps_used, DevStatus* st, int warm) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), cs = (int)cl.num_blocks();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = JC_THREADS / 32;
  const int R = (n + cs - 1) / cs;  // row slots per CTA
  extern __shared__ cplx sm[];      // [R x m] rows of G, then [R x n] rows of Vt
  __shared__ double s_fro;
  __shared__ int s_rot, s_big;
  __shared__ double s_part[JC_THREADS / 64][2][4];  // [pair slot][half][al, be, Re g, Im g]
  __shared__ double s_rp[JC_THREADS / 64][4];       // [pair slot][c, s, Re ph, Im ph]
  __shared__ float s_rf[JC_THREADS / 64][6];        // DF: c, Re sq, Im sq as double-float pairs
  __shared__ int s_rr[JC_THREADS / 64];             // [pair slot] rotated
  cplx* gl = sm;
  cplx* vl = sm + (long long)R * m;
  double f = 0.0;
  for (int l = 0; l < R; ++l) {
    const int i = l * cs + rank;
    if (i >= n) break;
    for (int t = threadIdx.x; t < m; t += JC_THREADS) {
      const cplx x = G[(long long)i * ldg + t];
      if constexpr (DF)
        ((float4*)gl)[(long long)l * m + t] = df_elem(x);
      else
        gl[(long long)l * m + t] = x;
      f += x.x * x.x + x.y * x.y;
    }
    if (Vt)
      for (int t = threadIdx.x; t < n; t += JC_THREADS)
        vl[(long long)l * n + t] = warm ? Vt[(long long)i * n + t] : make_double2(t == i ? 1.0 : 0.0, 0.0);
  }
  f = warp_sum(f);
  __shared__ double s_w[JC_THREADS / 32];
  if (lane == 0) s_w[warp] = f;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < nwarps; ++w) t += s_w[w];
    s_fro = t;
    s_rot = 0;
    s_big = 0;
  }
  cl.sync();
  double fro2 = 0.0;
  for (int r = 0; r < cs; ++r) fro2 += *cl.map_shared_rank(&s_fro, r);
  const double negligible = fro2 * 1e-30;
  auto grow = [&](int i) { return cl.map_shared_rank(gl, i % cs) + (long long)(i / cs) * m; };
  auto vrow = [&](int i) { return cl.map_shared_rank(vl, i % cs) + (long long)(i / cs) * n; };
  const int np = (n + 1) & ~1;
  const int rounds = np - 1, npairs = np / 2;
  bool converged = false;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    for (int r = 0; r < rounds; ++r) {
      // two warps per pair: warp (slot, half) takes the columns of 32-wide
      // chunks 2j + half; the halves' sums meet in shared memory (fixed order)
      for (int p0 = rank * (nwarps / 2); p0 < npairs; p0 += cs * (nwarps / 2)) {
        const int slot = warp % (nwarps / 2), half = warp / (nwarps / 2);
        const int p = p0 + slot;
        int i = 0, j = n;
        if (p < npairs) pair_of(r, p, np, rounds, &i, &j);
        const bool active = p < npairs && j < n;
        cplx* gi = active ? grow(i) : nullptr;
        cplx* gj = active ? grow(j) : nullptr;
        if (active && DF) {
          df2 al = {0.f, 0.f}, be = {0.f, 0.f}, gr = {0.f, 0.f}, gim = {0.f, 0.f};
          const float4* fi = (const float4*)gi;
          const float4* fj = (const float4*)gj;
          for (int t = lane + 32 * half; t < m; t += 64) {
            const float4 x4 = fi[t], y4 = fj[t];
            const df2 xr = {x4.x, x4.y}, xi = {x4.z, x4.w}, yr = {y4.x, y4.y}, yi = {y4.z, y4.w};
            acc_mul(al, xr, xr);
            acc_mul(al, xi, xi);
            acc_mul(be, yr, yr);
            acc_mul(be, yi, yi);
            acc_mul(gr, xr, yr);
            acc_mul(gr, xi, yi);
            acc_mul(gim, xr, yi);
            acc_mul(gim, df_negate(xi), yr);
          }
          al = warp_sum_df(al);
          be = warp_sum_df(be);
          gr = warp_sum_df(gr);
          gim = warp_sum_df(gim);
          if (lane == 0) {
            s_part[slot][half][0] = df_val(al);
            s_part[slot][half][1] = df_val(be);
            s_part[slot][half][2] = df_val(gr);
            s_part[slot][half][3] = df_val(gim);
          }
        } else if (active) {
          double al = 0.0, be = 0.0, gr = 0.0, gim = 0.0;
          for (int t = lane + 32 * half; t < m; t += 64) {
            const cplx x = gi[t], y = gj[t];
            al += x.x * x.x + x.y * x.y;
            be += y.x * y.x + y.y * y.y;
            gr += x.x * y.x + x.y * y.y;
            gim += x.x * y.y - x.y * y.x;
          }
          const double tot = warp_sum4(al, be, gr, gim);
          if ((lane & 7) == 0) s_part[slot][half][lane >> 3] = tot;
        }
        __syncthreads();
        // the pair's rotation, by one thread of the pair (a lone FP64
        // instruction occupies the sub-partition's FP64 unit as long as a
        // full warp's).  c = 1/sqrt(1 + t^2) and the phase g/|g| in FP64, so
        // that c^2 + s^2 = 1 and |ph| = 1 to FP64 rounding; the tangent t in
        // FP32 for double-float rows (their angles only steer a convergence
        // judged at 48 bits), in FP64 otherwise (an FP32 tangent raised the
        // FP64 path's corner-spectrum noise from 2e-11 to 1e-10)
        if (active && half == 0 && lane == 0) {
          double c = 1.0, sn = 0.0, phr = 1.0, phi = 0.0;
          int rot = 0;
          const double al = s_part[slot][0][0] + s_part[slot][1][0], be = s_part[slot][0][1] + s_part[slot][1][1];
          const double gr = s_part[slot][0][2] + s_part[slot][1][2], gim = s_part[slot][0][3] + s_part[slot][1][3];
          const double g2 = gr * gr + gim * gim;
          if (al > negligible && be > negligible && g2 > tol * tol * al * be) {
            const double ig = rsqrt(g2);
            const double zeta = 0.5 * (be - al) * ig;
            double t;
            if (!DF) {
              t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            } else if (fabs(zeta) < 1e15) {
              const float zf = (float)zeta;
              t = (double)(copysignf(1.0f, zf) / (fabsf(zf) + sqrtf(fmaf(zf, zf, 1.0f))));
            } else {
              t = 0.5 / zeta;  // t -> 1/(2 zeta)
            }
            c = rsqrt(fma(t, t, 1.0));
            sn = c * t;
            phr = gr * ig;
            phi = -gim * ig;
            rot = 1;
            atomicAdd(&s_rot, 1);
            // a rotation with off-orthogonality or angle above 1e-8 keeps
            // the sweep from being the last one
            if (g2 > 1e-16 * al * be || fabs(sn) > 1e-8) s_big = 1;
          }
          s_rp[slot][0] = c;
          s_rp[slot][1] = sn;
          s_rp[slot][2] = phr;
          s_rp[slot][3] = phi;
          s_rr[slot] = rot;
          if (DF) {
            // the rotation's double-float factors once here, not in every thread
            const df2 cd = df_of(c), qr = df_of(sn * phr), qi = df_of(sn * phi);
            s_rf[slot][0] = cd.h;
            s_rf[slot][1] = cd.l;
            s_rf[slot][2] = qr.h;
            s_rf[slot][3] = qr.l;
            s_rf[slot][4] = qi.h;
            s_rf[slot][5] = qi.l;
          }
          if (log)
            log[((long long)sweep * rounds + r) * npairs + p] = rot ? make_double4_16a(c, sn, phr, phi)
                                                                   : make_double4_16a(2.0, 0.0, 0.0, 0.0);
        } else if (!active && lane == 0 && half == 0) {
          s_rr[slot] = 0;
          if (log && p < npairs)
            log[((long long)sweep * rounds + r) * npairs + p] = make_double4_16a(2.0, 0.0, 0.0, 0.0);
        }
        __syncthreads();  // the rotation is published; partial sums read before the next pair overwrites them
        if (s_rr[slot]) {
          if constexpr (DF) {
            // a' = c a - sq b, b' = c b + sp a (the form of jac_rotate), sp = conj(sq)
            const df2 cd = {s_rf[slot][0], s_rf[slot][1]}, qr = {s_rf[slot][2], s_rf[slot][3]},
                      qi = {s_rf[slot][4], s_rf[slot][5]}, pr = qr, pi = df_negate(qi);
            float4* fi = (float4*)gi;
            float4* fj = (float4*)gj;
            for (int q = lane + 32 * half; q < m; q += 64) {
              const float4 x4 = fi[q], y4 = fj[q];
              const df2 xr = {x4.x, x4.y}, xi = {x4.z, x4.w}, yr = {y4.x, y4.y}, yi = {y4.z, y4.w};
              df2 ar = {0.f, 0.f}, ai = {0.f, 0.f}, br = {0.f, 0.f}, bi = {0.f, 0.f};
              acc_mul(ar, cd, xr);
              acc_mul(ar, df_negate(qr), yr);
              acc_mul(ar, qi, yi);
              acc_mul(ai, cd, xi);
              acc_mul(ai, df_negate(qr), yi);
              acc_mul(ai, df_negate(qi), yr);
              acc_mul(br, cd, yr);
              acc_mul(br, pr, xr);
              acc_mul(br, df_negate(pi), xi);
              acc_mul(bi, cd, yi);
              acc_mul(bi, pr, xi);
              acc_mul(bi, pi, xr);
              ar = df_norm(ar);
              ai = df_norm(ai);
              br = df_norm(br);
              bi = df_norm(bi);
              fi[q] = make_float4(ar.h, ar.l, ai.h, ai.l);
              fj[q] = make_float4(br.h, br.l, bi.h, bi.l);
            }
          } else {
            const double c = s_rp[slot][0], sn = s_rp[slot][1];
            const cplx ph = make_double2(s_rp[slot][2], s_rp[slot][3]);
            const cplx sq = make_double2(sn * ph.x, sn * ph.y), sp = make_double2(sn * ph.x, -sn * ph.y);
            for (int q = lane + 32 * half; q < m; q += 64) jac_rotate(gi[q], gj[q], c, sq, sp);
            if (Vt) {
              cplx* vi = vrow(i);
              cplx* vj = vrow(j);
              for (int q = lane + 32 * half; q < n; q += 64) jac_rotate(vi[q], vj[q], c, sq, sp);
            }
          }
        }
      }
      cl.sync();
    }
    int total = 0, big = 0;
    for (int r = 0; r < cs; ++r) {
      total += *cl.map_shared_rank(&s_rot, r);
      big |= *cl.map_shared_rank(&s_big, r);
    }
    cl.sync();  // every CTA has read every count
    if (threadIdx.x == 0) {
      s_rot = 0;
      s_big = 0;
    }
    cl.sync();
    // No rotation: converged.  Only rotations with off-orthogonality and angle
    // <= 1e-8: each later rotation changed an earlier pair's inner product by at
    // most 1e-16 relative, so the rows are orthogonal to ~k * 1e-16 (the
    // m * eps tolerance) and the confirming sweep is skipped.
    if (total == 0 || big == 0) {
      converged = true;
      break;
    }
  }
  for (int l = 0; l < R; ++l) {
    const int i = l * cs + rank;
    if (i >= n) break;
    for (int t = threadIdx.x; t < m; t += JC_THREADS) {
      if constexpr (DF) {
        const float4 x4 = ((const float4*)gl)[(long long)l * m + t];
        G[(long long)i * ldg + t] = make_double2(df_val({x4.x, x4.y}), df_val({x4.z, x4.w}));
      } else {
        G[(long long)i * ldg + t] = gl[(long long)l * m + t];
      }
    }
    if (Vt)
      for (int t = threadIdx.x; t < n; t += JC_THREADS) Vt[(long long)i * n + t] = vl[(long long)l * n + t];
  }
  if (rank == 0 && threadIdx.x == 0) {
    if (sweeps_used) *sweeps_used = converged ? sweep + 1 : max_sweeps;
    atomicAdd(&st->jacobi_calls, 1);
    atomicAdd(&st->jacobi_sweeps, converged ? sweep + 1 : max_sweeps);
    if (!converged) atomicAdd(&st->jacobi_unconverged, 1);
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

// Vt (n x n) = the logged rotations applied to the identity (warm: to Vt as
// it is, in place), one CTA per column q (columns are independent: a CTA
// reads and writes its own column only): thread p applies pair p of every
// round, rounds in order, the column held in shared memory.  Rotation c = 2
// marks a pair that was not rotated.  DF (the precision form): the column in
// double-float arithmetic on the FP32 pipe; the unitarity of V then holds to
// about 2^-48 per rotation instead of 2^-53, some 1e-12 after thousands of
// visits of a cut, far below the precision form's 1e-6 truncation.
template <bool DF>
__global__ void jacobi_replay_kernel(cplx* __restrict__ Vt, int n, const double4_16a* __restrict__ log,
                                     const int* __restrict__ sweeps_used, int warm) {
  extern __shared__ cplx col[];  // DF: (Re hi, Re lo, Im hi, Im lo) per element, the same 16 bytes
  float4* colf = (float4*)col;
  const int q = blockIdx.x;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const cplx v = warm ? Vt[(long long)i * n + q] : make_double2(i == q ? 1.0 : 0.0, 0.0);
    if constexpr (DF)
      colf[i] = df_elem(v);
    else
      col[i] = v;
  }
  __syncthreads();
  const int sweeps = *sweeps_used;
  const int np = (n + 1) & ~1;
  const int rounds = np - 1, npairs = np / 2;
  const int p = threadIdx.x;
  const long long steps = (long long)sweeps * rounds;
  // the next round's record is loaded while this round's rotation runs
  double4_16a next = make_double4_16a(2.0, 0.0, 0.0, 0.0);
  if (p < npairs && steps > 0) next = log[p];
  for (long long st = 0; st < steps; ++st) {
    const int r = (int)(st % rounds);
    const double4_16a rec = next;
    if (p < npairs && st + 1 < steps) next = log[(st + 1) * npairs + p];
    if (p < npairs && rec.x < 1.5) {
      int i, j;
      pair_of(r, p, np, rounds, &i, &j);
      const double c = rec.x, s = rec.y;
      if constexpr (DF) {
        const df2 cd = df_of(c), qr = df_of(s * rec.z), qi = df_of(s * rec.w), pr = qr, pi = df_negate(qi);
        const float4 x4 = colf[i], y4 = colf[j];
        const df2 xr = {x4.x, x4.y}, xi = {x4.z, x4.w}, yr = {y4.x, y4.y}, yi = {y4.z, y4.w};
        df2 ar = {0.f, 0.f}, ai = {0.f, 0.f}, br = {0.f, 0.f}, bi = {0.f, 0.f};
        acc_mul(ar, cd, xr);
        acc_mul(ar, df_negate(qr), yr);
        acc_mul(ar, qi, yi);
        acc_mul(ai, cd, xi);
        acc_mul(ai, df_negate(qr), yi);
        acc_mul(ai, df_negate(qi), yr);
        acc_mul(br, cd, yr);
        acc_mul(br, pr, xr);
        acc_mul(br, df_negate(pi), xi);
        acc_mul(bi, cd, yi);
        acc_mul(bi, pr, xi);
        acc_mul(bi, pi, xr);
        ar = df_norm(ar);
        ai = df_norm(ai);
        br = df_norm(br);
        bi = df_norm(bi);
        colf[i] = make_float4(ar.h, ar.l, ai.h, ai.l);
        colf[j] = make_float4(br.h, br.l, bi.h, bi.l);
      } else {
        jac_rotate(col[i], col[j], c, make_double2(s * rec.z, s * rec.w), make_double2(s * rec.z, -s * rec.w));
      }
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    if constexpr (DF) {
      const float4 x4 = colf[i];
      Vt[(long long)i * n + q] = make_double2(df_val({x4.x, x4.y}), df_val({x4.z, x4.w}));
    } else {
      Vt[(long long)i * n + q] = col[i];
    }
  }
}

// Right-looking Cholesky of the Hermitian n x n G (upper triangle used) with
// dropped pivots (d <= tol * max diagonal: row of R zero), blocked by CH_NB
// rows.  Rows of the working copy W live in the cluster's shared memory (row
// i in CTA i mod csize).  For the block of rows j0 .. j0+nb-1 each CTA
// factors the nb x nb diagonal block (every CTA the same arithmetic, so the
// same pivots) and, for the columns l >= j0+nb it owns (l mod csize = rank),
// the block's entries of R; after a cluster barrier every CTA gathers the
// block's rows of R and updates its own rows below the block, W[i,l] -=
// conj(R[j,i]) R[j,l] for l >= i, j in order.  The operations and their order
// per element are those of the column-by-column algorithm.
constexpr int CH_NB = 8;

__global__ void __launch_bounds__(CL_THREADS)
    chol_cluster_kernel(const cplx* __restrict__ G, cplx* __restrict__ Rout, int n, double tol) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), cs = (int)cl.num_blocks();
  const int R = (n + cs - 1) / cs;
  extern __shared__ cplx sm[];  // [R x n] own rows of W, then [CH_NB x n] the block's rows of W, then of R
  cplx* pan = sm + (long long)R * n;
  cplx* rpan = pan + (long long)CH_NB * n;
  __shared__ double s_max, s_rjj[CH_NB], s_inv[CH_NB];
  for (int l = 0; l < R; ++l) {
    const int i = l * cs + rank;
    if (i >= n) break;
    for (int t = threadIdx.x; t < n; t += CL_THREADS) sm[(long long)l * n + t] = G[(long long)i * n + t];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int l = 0; l < R; ++l) {
      const int i = l * cs + rank;
      if (i >= n) break;
      mx = fmax(mx, sm[(long long)l * n + i].x);
    }
    s_max = mx;
  }
  cl.sync();
  double dmax = 0.0;
  for (int r = 0; r < cs; ++r) dmax = fmax(dmax, *cl.map_shared_rank(&s_max, r));
  const double thr = tol * dmax;
  // columns of the block this CTA works on: the diagonal block (c < nb), then
  // its own columns l >= j0 + nb (c >= nb: l = j0 + nb + (c - nb) * cs + off)
  for (int j0 = 0; j0 < n; j0 += CH_NB) {
    const int nb = min(CH_NB, n - j0), jn = j0 + nb;
    const int off = ((rank - jn) % cs + cs) % cs;  // first own column at or after jn is jn + off
    const int nown = jn + off < n ? (n - 1 - (jn + off)) / cs + 1 : 0;
    const int ncol = nb + nown;
    auto col = [&](int c) { return c < nb ? j0 + c : jn + off + (c - nb) * cs; };
    // the block's rows of W on those columns, from their owners
    for (int e = threadIdx.x; e < nb * ncol; e += CL_THREADS) {
      const int jj = e / ncol, l = col(e % ncol), j = j0 + jj;
      pan[(long long)jj * n + l] = cl.map_shared_rank(sm, j % cs)[(long long)(j / cs) * n + l];
    }
    __syncthreads();
    for (int jj = 0; jj < nb; ++jj) {
      const int j = j0 + jj;
      cplx* pj = pan + (long long)jj * n;
      // the pivot's reciprocal root once, r = d / sqrt(d) from it (FP64
      // roots and divides are slow on this part, a lone thread's the more)
      if (threadIdx.x == 0) {
        const double d = pj[j].x;
        const bool keep = d > thr;
        const double inv = keep ? rsqrt(d) : 0.0;
        s_inv[jj] = inv;
        s_rjj[jj] = keep ? d * inv : 0.0;
      }
      __syncthreads();
      const double rjj = s_rjj[jj], inv = s_inv[jj];
      const bool keep = rjj > 0.0;
      // row j of R on the CTA's columns into its own buffer (zero left of the
      // diagonal, and for a dropped direction), and in the same phase the
      // block's rows i > j: W[i,l] -= conj(R[j,i]) R[j,l] for l >= i, with
      // R[j,.] = W[j,.] / r formed from row j of W, which this phase only reads
      for (int c = threadIdx.x; c < ncol; c += CL_THREADS) {
        const int l = col(c);
        cplx v = make_double2(0.0, 0.0);
        if (keep && l >= j) {
          const cplx g = pj[l];
          v = l == j ? make_double2(rjj, 0.0) : make_double2(g.x * inv, g.y * inv);
        }
        rpan[(long long)jj * n + l] = v;
      }
      if (keep) {
        for (int e = threadIdx.x; e < (nb - 1 - jj) * ncol; e += CL_THREADS) {
          const int i = j + 1 + e / ncol, l = col(e % ncol);
          if (l < i) continue;
          const cplx a = make_double2(pj[i].x * inv, pj[i].y * inv), b = make_double2(pj[l].x * inv, pj[l].y * inv);
          cplx* wi = pan + (long long)(i - j0) * n;
          wi[l].x -= a.x * b.x + a.y * b.y;
          wi[l].y -= a.x * b.y - a.y * b.x;
        }
      }
      __syncthreads();
    }
    cl.sync();  // every CTA's columns of the block's rows of R are final
    // the other CTAs' columns of those rows
    for (int e = threadIdx.x; e < nb * (n - jn); e += CL_THREADS) {
      const int jj = e / (n - jn), l = jn + e % (n - jn);
      const int o = l % cs;
      if (o != rank) rpan[(long long)jj * n + l] = cl.map_shared_rank(rpan, o)[(long long)jj * n + l];
    }
    __syncthreads();
    // the owners store their rows of R
    for (int jj = 0; jj < nb; ++jj) {
      const int j = j0 + jj;
      if (j % cs != rank) continue;
      for (int l = threadIdx.x; l < n; l += CL_THREADS)
        Rout[(long long)j * n + l] = l < j0 ? make_double2(0.0, 0.0) : rpan[(long long)jj * n + l];
    }
    // own rows below the block
    for (int l0 = 0; l0 < R; ++l0) {
      const int i = l0 * cs + rank;
      if (i >= n) break;
      if (i < jn) continue;
      cplx* wi = sm + (long long)l0 * n;
      for (int l = i + threadIdx.x; l < n; l += CL_THREADS) {
        cplx v = wi[l];
        for (int jj = 0; jj < nb; ++jj) {
          if (s_rjj[jj] == 0.0) continue;  // dropped direction: no update
          const cplx a = rpan[(long long)jj * n + i], b = rpan[(long long)jj * n + l];
          v.x -= a.x * b.x + a.y * b.y;
          v.y -= a.x * b.y - a.y * b.x;
        }
        wi[l] = v;
      }
    }
    cl.sync();  // rows updated before they are read as the next block; gathers done before rpan is rewritten
  }
}

}  // namespace

static cudaError_t cluster_init() {
  if (g_csize) return cudaSuccess;
  cudaError_t e;
  const void* fns[3] = {(const void*)jacobi_cluster_kernel<false>, (const void*)jacobi_cluster_kernel<true>,
                        (const void*)chol_cluster_kernel};
  for (const void* f : fns) {
    if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, CL_SMEM)) != cudaSuccess) return e;
  }
  // 16 CTAs per cluster when the hardware can place such a cluster, else 8
  int csize = 8;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = 16;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.gridDim = dim3(16);
  cfg.blockDim = dim3(CL_THREADS);
  cfg.dynamicSmemBytes = CL_SMEM;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, (const void*)jacobi_cluster_kernel<false>, &cfg) == cudaSuccess &&
      nclusters >= 1)
    csize = 16;
  cudaGetLastError();  // a refused query leaves no error behind
  g_csize = csize;
  return cudaSuccess;
}

cudaError_t fp64_cluster_init() { return cluster_init(); }

static cudaError_t launch_cluster(const void* fn, void** args, size_t smem, cudaStream_t s,
                                  int threads = CL_THREADS) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = g_csize;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.gridDim = dim3(g_csize);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

bool jacobi_cluster_fits(int n, int m, bool vt_in_smem) {
  if (n < 32) return false;
  if (cluster_init() != cudaSuccess) return false;
  const long long R = (n + g_csize - 1) / g_csize;
  return R * ((long long)m + (vt_in_smem ? n : 0)) * (long long)sizeof(cplx) <= CL_SMEM;
}

long long jacobi_log_elems(int n, int max_sweeps) {
  const long long np = (n + 1) & ~1;
  return (long long)max_sweeps * (np - 1) * (np / 2) * 2;  // one double4_16a = two complex slots per pair
}

cudaError_t jacobi_cluster(cudaStream_t s, cplx* G, int n, int m, long long ldg, cplx* Vt, int max_sweeps,
                           DevStatus* st, cplx* rotlog, int* sweeps_used, bool warm_v, bool dfloat) {
  cudaError_t e;
  if ((e = cluster_init()) != cudaSuccess) return e;
  const bool replay = Vt && rotlog && sweeps_used && n <= 2048;
  cplx* Vin = replay ? nullptr : Vt;  // with a log, Vt is rebuilt afterwards across the GPU
  double4_16a* logp = replay ? (double4_16a*)rotlog : nullptr;
  int* su = replay ? sweeps_used : nullptr;
  const long long R = (n + g_csize - 1) / g_csize;
  const size_t smem = (size_t)(R * ((long long)m + (Vin ? n : 0)) * sizeof(cplx));
  // double-float rows only where Vt is rebuilt from the log in FP64; their
  // dot products resolve orthogonality to about m 2^-48, so pairs are left
  // alone below m 2^-44 (FP64: m eps)
  const bool df = dfloat && replay;
  double tol = df ? (double)m * 0x1p-44 : (double)m * 2.220446049250313e-16;
  int warm = warm_v && Vin ? 1 : 0;
  void* args[] = {&G, &n, &m, &ldg, &Vin, &max_sweeps, &tol, &logp, &su, &st, &warm};
  e = launch_cluster(df ? (const void*)jacobi_cluster_kernel<true> : (const void*)jacobi_cluster_kernel<false>, args,
                     smem, s, JC_THREADS);
  count_launch();
  if (e != cudaSuccess || !replay) return e;
  const int npairs = ((n + 1) & ~1) / 2;
  const int threads = (npairs + 31) / 32 * 32;
  if (df)
    jacobi_replay_kernel<true><<<n, threads, n * sizeof(cplx), s>>>(Vt, n, (const double4_16a*)rotlog, sweeps_used,
                                                                  warm_v ? 1 : 0);
  else
    jacobi_replay_kernel<false><<<n, threads, n * sizeof(cplx), s>>>(Vt, n, (const double4_16a*)rotlog, sweeps_used,
                                                                   warm_v ? 1 : 0);
  count_launch();
  return cudaGetLastError();
}

bool chol_cluster_fits(int n) {
  if (n < 32) return false;
  if (cluster_init() != cudaSuccess) return false;
  const long long R = (n + g_csize - 1) / g_csize;
  return (R + 2 * CH_NB) * n * (long long)sizeof(cplx) <= CL_SMEM;
}

cudaError_t chol_cluster(cudaStream_t s, const cplx* G, cplx* R, int n, double tol) {
  cudaError_t e;
  if ((e = cluster_init()) != cudaSuccess) return e;
  const long long rows = (n + g_csize - 1) / g_csize;
  const size_t smem = (size_t)((rows + 2 * CH_NB) * n * sizeof(cplx));
  void* args[] = {&G, &R, &n, &tol};
  e = launch_cluster((const void*)chol_cluster_kernel, args, smem, s);
  count_launch();
  return e;
}
