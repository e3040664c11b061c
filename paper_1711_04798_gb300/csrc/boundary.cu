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

}  // namespace

namespace bnd {
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
