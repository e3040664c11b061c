// Corner spectrum without any device allocation.
//
// Some callers cannot call cudaMalloc: a process whose device memory is all
// owned by another allocator (for instance a framework's caching allocator
// with a fixed budget), or a latency-critical loop in which the implicit
// device synchronisation of cudaMalloc / cudaFree is not allowed.  For them
// ipeps_corner_spectrum_noalloc computes the singular values of one chi x chi
// corner matrix with the same Jacobi SVD kernel as ipeps_ctm_spectra, keeping
// every intermediate in the fixed file-scope device array below.
#include <cstdio>

#include "../../include/ipeps_ctm.h"
#include "ctm_internal.h"

void set_last_error_message(const char* msg);  // defined with ipeps_last_error

namespace {

constexpr int NOALLOC_MAX_CHI = 256;
// working copy of the matrix + singular values + selection + counters/status
constexpr size_t OFF_WORK = 0;
constexpr size_t OFF_SIGMA = OFF_WORK + sizeof(cplx) * NOALLOC_MAX_CHI * NOALLOC_MAX_CHI;
constexpr size_t OFF_SEL = OFF_SIGMA + sizeof(double) * NOALLOC_MAX_CHI;
constexpr size_t OFF_PERM = OFF_SEL + sizeof(double) * NOALLOC_MAX_CHI;
constexpr size_t OFF_FRO2 = OFF_PERM + sizeof(int) * NOALLOC_MAX_CHI;
constexpr size_t OFF_COUNT = OFF_FRO2 + 256;
constexpr size_t OFF_STATUS = OFF_COUNT + 256;
constexpr size_t NOALLOC_SCRATCH_BYTES = OFF_STATUS + 256;  // about 1.01 MiB

// Shared by every call in the process; each device that loads the library
// holds its own copy until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

thread_local char g_msg_buf[256];  // formatted here, then handed to ipeps_last_error()

// s_out[a] = s_sel[a] / s_sel[0] (zero when s_sel[0] == 0)
__global__ void normalise_by_first_kernel(const double* s_sel, int n, double* s_out) {
  const double s0 = s_sel[0];
  for (int a = threadIdx.x; a < n; a += blockDim.x) s_out[a] = s0 > 0.0 ? s_sel[a] / s0 : 0.0;
}

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in; its device address is looked
// up on every call, with the caller's device current, so that it stays right
// after a device reset or on a context created later (the first lookup on a
// device also loads this library's device code there).
ipeps_status scratch_address(unsigned char** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    snprintf(g_msg_buf, sizeof g_msg_buf, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
    set_last_error_message(g_msg_buf);
    return IPEPS_ECUDA;
  }
  *out = (unsigned char*)p;
  return IPEPS_OK;
}

}  // namespace

extern "C" ipeps_status ipeps_corner_spectrum_noalloc(const double* C_dev, int chi, double* s_dev,
                                                      void* stream) {
  if (!C_dev || !s_dev) {
    snprintf(g_msg_buf, sizeof g_msg_buf, "null device pointer");
    set_last_error_message(g_msg_buf);
    return IPEPS_EINVAL;
  }
  if (chi < 1 || chi > NOALLOC_MAX_CHI) {
    snprintf(g_msg_buf, sizeof g_msg_buf, "chi = %d outside 1..%d (the fixed scratch holds one %dx%d matrix)",
             chi, NOALLOC_MAX_CHI, NOALLOC_MAX_CHI, NOALLOC_MAX_CHI);
    set_last_error_message(g_msg_buf);
    return IPEPS_EINVAL;
  }
  unsigned char* base = nullptr;
  ipeps_status st = scratch_address(&base);
  if (st != IPEPS_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cplx* work = (cplx*)(base + OFF_WORK);
  double* sigma = (double*)(base + OFF_SIGMA);
  double* sel = (double*)(base + OFF_SEL);
  int* perm = (int*)(base + OFF_PERM);
  double* fro2 = (double*)(base + OFF_FRO2);
  int* counters = (int*)(base + OFF_COUNT);
  DevStatus* dst = (DevStatus*)(base + OFF_STATUS);
  const size_t mbytes = (size_t)chi * chi * sizeof(cplx);
  cudaError_t e = cudaMemsetAsync(dst, 0, sizeof(DevStatus), s);  // status must start at zero
  if (e == cudaSuccess) e = cudaMemcpyAsync(work, C_dev, mbytes, cudaMemcpyDeviceToDevice, s);
  // jacobi_rows clears its own counters and Frobenius accumulator
  if (e == cudaSuccess) e = jacobi_rows(s, work, chi, chi, chi, nullptr, sigma, 40, fro2, counters, dst);
  if (e == cudaSuccess) e = select_top(s, sigma, chi, chi, 0.0, perm, sel);
  if (e == cudaSuccess) {
    normalise_by_first_kernel<<<1, 256, 0, s>>>(sel, chi, s_dev);
    count_launch();
    e = cudaGetLastError();
  }
  DevStatus h_st = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_st, dst, sizeof h_st, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    snprintf(g_msg_buf, sizeof g_msg_buf, "CUDA error: %s", cudaGetErrorString(e));
    set_last_error_message(g_msg_buf);
    return IPEPS_ECUDA;
  }
  if (h_st.jacobi_unconverged) {
    snprintf(g_msg_buf, sizeof g_msg_buf, "Jacobi SVD hit its sweep budget");
    set_last_error_message(g_msg_buf);
    return IPEPS_ETIMEOUT;
  }
  return IPEPS_OK;
}

