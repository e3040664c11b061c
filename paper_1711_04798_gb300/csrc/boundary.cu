// Kernels of the boundary density operator readout (Sec. IV, Eq. "rho"):
// phase-fixing and Hermitising sigma_L / sigma_R, the |sigma_L^T|^(1/2)
// factor scaling, and the normalised spectrum with its von Neumann entropy.
#include "ctm_internal.h"

namespace {

__global__ void trace_kernel(const cplx* S, int n, double* out) {
  __shared__ double sr[1024], si[1024];
  double a = 0, b = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    a += S[(long long)i * n + i].x;
    b += S[(long long)i * n + i].y;
  }
  sr[threadIdx.x] = a;
  si[threadIdx.x] = b;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sr[threadIdx.x] += sr[threadIdx.x + o];
      si[threadIdx.x] += si[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sr[0];
    out[1] = si[0];
  }
}

// S <- Herm(ph * S), ph = conj(tr S)/|tr S|; optionally stored transposed
// (the transpose of a Hermitian matrix is its complex conjugate).
__global__ void phase_herm_kernel(cplx* S, int n, int transpose_out, const double* tr) {
  const double m = hypot(tr[0], tr[1]);
  const double pr = m > 0 ? tr[0] / m : 1.0, pi = m > 0 ? -tr[1] / m : 0.0;
  const long long total = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    if (i > j) continue;
    const cplx x = S[(long long)i * n + j], y = S[(long long)j * n + i];
    const double ar = pr * x.x - pi * x.y, ai = pr * x.y + pi * x.x;  // ph * S[i,j]
    const double br = pr * y.x - pi * y.y, bi = pr * y.y + pi * y.x;  // ph * S[j,i]
    double hr = 0.5 * (ar + br), hi = 0.5 * (ai - bi);                 // H[i,j]
    if (i == j) hi = 0.0;
    if (transpose_out) hi = -hi;  // (H^T)[i,j] = H[j,i] = conj(H[i,j])
    S[(long long)i * n + j] = make_double2(hr, hi);
    S[(long long)j * n + i] = make_double2(hr, -hi);
  }
}

__global__ void scale_cols_kernel(cplx* G, int n, const double* sigma) {
  const long long total = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e % n);
    const double s = sigma[j];
    const double f = s > 1e-300 ? 1.0 / sqrt(s) : 0.0;
    G[e].x *= f;
    G[e].y *= f;
  }
}

// lam = sigma sorted descending / sum; S_vn = -sum lam ln lam (lam > 0)
__global__ void spectrum_finish_kernel(const double* sigma, int n, double* lam, double* S_vn) {
  __shared__ double red[1024];
  double t = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) t += sigma[i];
  red[threadIdx.x] = t;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double tot = red[0];
  __syncthreads();
  double ent = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double si = sigma[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double sj = sigma[j];
      rank += (sj > si) || (sj == si && j < i);
    }
    const double l = tot > 0 ? si / tot : 0.0;
    lam[rank] = l;
    if (l > 0) ent -= l * log(l);
  }
  red[threadIdx.x] = ent;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *S_vn = red[0];
}

// partial[2b], partial[2b+1] = Re, Im of the sum of M[i][j] M[j][i] over the
// 32 x 32 tile pairs block b visits (tiles staged in shared memory so that both
// reads run along rows); tr(M^2) is the sum over all blocks.
__global__ void purity_partial_kernel(const cplx* __restrict__ M, int n, double* __restrict__ partial) {
  __shared__ cplx ta[32][33], tb[32][33];
  __shared__ double red[2][256];
  double sr = 0.0, si = 0.0;
  const int nt = (n + 31) / 32;
  const long long tiles = (long long)nt * nt;
  for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int ti = (int)(t / nt), tj = (int)(t % nt);
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
      const int i = ti * 32 + r, j = tj * 32 + threadIdx.x;
      ta[r][threadIdx.x] = (i < n && j < n) ? M[(long long)i * n + j] : make_double2(0.0, 0.0);
      const int i2 = tj * 32 + r, j2 = ti * 32 + threadIdx.x;
      tb[r][threadIdx.x] = (i2 < n && j2 < n) ? M[(long long)i2 * n + j2] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    // M[i][j] M[j][i] with i = ti*32 + r, j = tj*32 + c: ta[r][c] * tb[c][r]
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
      const cplx x = ta[r][threadIdx.x], y = tb[threadIdx.x][r];
      sr += x.x * y.x - x.y * y.y;
      si += x.x * y.y + x.y * y.x;
    }
  }
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  red[0][tid] = sr;
  red[1][tid] = si;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (tid < o) {
      red[0][tid] += red[0][tid + o];
      red[1][tid] += red[1][tid + o];
    }
    __syncthreads();
  }
  if (tid == 0) {
    partial[2 * blockIdx.x] = red[0][0];
    partial[2 * blockIdx.x + 1] = red[1][0];
  }
}

// out = {Re tr M, Im tr M, Re tr M^2, Im tr M^2}: the block partials summed in a fixed order
__global__ void purity_finish_kernel(const double* __restrict__ partial, int nb, const double* __restrict__ tr,
                                     double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int i = 0; i < nb; ++i) {
    a += partial[2 * i];
    b += partial[2 * i + 1];
  }
  out[0] = tr[0];
  out[1] = tr[1];
  out[2] = a;
  out[3] = b;
}

// ring operator S[(k_1..k_Nv), (b_1..b_Nv)] <-> vector v[(k_1 b_1) .. (k_Nv b_Nv)]
// (base-D digits; to_vector selects the direction)
__global__ void interleave_kernel(const cplx* __restrict__ in, cplx* __restrict__ out, int D, int Nv,
                                  long long total, int to_vector) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    // e indexes the vector form: digits (k_1 b_1 ... k_Nv b_Nv), most significant first
    long long rest = e, K = 0, B = 0, pw = 1;
    for (int i = Nv - 1; i >= 0; --i) {
      const long long b = rest % D;
      rest /= D;
      const long long k = rest % D;
      rest /= D;
      K += k * pw;
      B += b * pw;
      pw *= D;
    }
    const long long o = K * pw + B;  // pw = D^Nv: the operator's row length
    if (to_vector)
      out[e] = in[o];
    else
      out[o] = in[e];
  }
}

// out = sum |a - b|^2 (fixed-order block partials, then one block)
__global__ void diff_norm2_kernel(const cplx* __restrict__ a, const cplx* __restrict__ b, long long n,
                                  double* __restrict__ partial) {
  __shared__ double red[256];
  double s = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double dr = a[e].x - b[e].x, di = a[e].y - b[e].y;
    s += dr * dr + di * di;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void sum_partials_kernel(const double* __restrict__ partial, int nb, double* __restrict__ out) {
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < nb; ++i) s += partial[i];
    *out = s;
  }
}

}  // namespace

namespace bnd {
void launch_interleave(cudaStream_t s, const cplx* in, cplx* out, int D, int Nv, bool to_vector) {
  long long total = 1;
  for (int i = 0; i < 2 * Nv; ++i) total *= D;
  long long blocks = (total + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  interleave_kernel<<<(unsigned)blocks, 256, 0, s>>>(in, out, D, Nv, total, to_vector ? 1 : 0);
}
// *out = sum |a - b|^2; work >= 513 doubles
void launch_diff_norm2(cudaStream_t s, const cplx* a, const cplx* b, long long n, double* work, double* out) {
  diff_norm2_kernel<<<512, 256, 0, s>>>(a, b, n, work);
  sum_partials_kernel<<<1, 32, 0, s>>>(work, 512, out);
}
// out[0..3] = tr M and tr M^2 (re, im) of the dense n x n M; work >= 2 + 2 * 1216 doubles
void launch_purity(cudaStream_t s, const cplx* M, int n, double* work, double* out) {
  const int nb = 1216;  // 152 SMs x 8
  trace_kernel<<<1, 1024, 0, s>>>(M, n, work);
  purity_partial_kernel<<<nb, dim3(32, 8), 0, s>>>(M, n, work + 2);
  purity_finish_kernel<<<1, 32, 0, s>>>(work + 2, nb, work, out);
}
void launch_phase_herm(cudaStream_t s, cplx* S, int n, bool transpose_out, double* work) {
  trace_kernel<<<1, 1024, 0, s>>>(S, n, work);
  long long total = (long long)n * n;
  long long blocks = (total + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  phase_herm_kernel<<<(unsigned)blocks, 256, 0, s>>>(S, n, transpose_out ? 1 : 0, work);
}
void launch_scale_cols(cudaStream_t s, cplx* G, int n, const double* sigma) {
  long long total = (long long)n * n;
  long long blocks = (total + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  scale_cols_kernel<<<(unsigned)blocks, 256, 0, s>>>(G, n, sigma);
}
void launch_spectrum_finish(cudaStream_t s, const double* sigma, int n, double* lam, double* S_vn) {
  spectrum_finish_kernel<<<1, 1024, 0, s>>>(sigma, n, lam, S_vn);
}
}  // namespace bnd
