// C ABI of the CTM library: handle, device arena, the directional move
// (enlarged corners -> projectors -> renormalisation, paper Sec. II.C) and the
// readouts (RDMs/energy App. A, kappa/fidelity Sec. III, boundary rho Sec. IV).
//
// Every contraction runs in this library's kernels (complex FP64 GEMM or the
// tensor-core GEMMs, index permutation, Jacobi SVD); the host only plans and
// launches.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/ipeps_ctm.h"
#include "ctm_internal.h"
#include "tc_gemm.h"

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

static ipeps_status fail(ipeps_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(IPEPS_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                  __FILE__, __LINE__);                                                 \
  } while (0)

#define CKS(call)                     \
  do {                                \
    ipeps_status s_ = (call);         \
    if (s_ != IPEPS_OK) return s_;    \
  } while (0)

extern "C" const char* ipeps_last_error(void) { return g_err.c_str(); }

void set_last_error_message(const char* msg) { g_err = msg; }

static const cplx ONE = {1.0, 0.0};
static const cplx ZERO = {0.0, 0.0};

// ---------------------------------------------------------------------------
// handle
// ---------------------------------------------------------------------------
struct TV {  // contiguous row-major tensor view
  cplx* p;
  int nd;
  int dims[8];
  long long size() const {
    long long s = 1;
    for (int i = 0; i < nd; ++i) s *= dims[i];
    return s;
  }
};

static TV tv(cplx* p, std::initializer_list<int> dims) {
  TV t;
  t.p = p;
  t.nd = 0;
  for (int d : dims) t.dims[t.nd++] = d;
  return t;
}

// Resources of one projector computation.  The two cuts of a unit-cell
// column are independent; the second one runs on its own stream with its own
// copy of these buffers, swapped into the handle while it is being enqueued.
struct Lane {
  cudaStream_t stream;
  cplx* Q[4];
  TcPacked Qp[4][2];
  void* Qpmem[4][2];
  cplx* thin[4];
  cplx* Vt;
  cplx* Gsel;
  double* sigma;
  double* s_sel;
  int* perm;
  int* counters;
  double* dwork;
  cplx* scratch;
  long long scratch_elems, scratch_top;
};

struct ipeps_ctm_s {
  int Lx, Ly, d, D, D2, chi, K, k, ntens;
  int pattern[4];
  int leg[4][4];      // host tensor leg sizes (u, l, d, r) per tensor: D, or 1 for a trivial bond
  bool mixed;
  int dtype;
  ipeps_options opt;
  cudaStream_t stream;
  bool own_mem;
  char* base;
  size_t bytes, used;
  // device data
  cplx* A[4][4];      // [rotation][tensor] ket tensors A[p,u,l,d,r] in each frame
  cplx* Bt[4][4];     // bra tensors (== A unless mixed)
  cplx* a[4][4];      // [rotation][tensor] double layers
  cplx* C[4][4];      // [role][y*Lx + x], original frame
  cplx* T[4][4];
  cplx* spareC[2][2]; // replacement buffers for renormalised C1 / C4, per row
  cplx* spareT[2];    // replacement T4 per row
  cplx* Q[4];
  TcPacked Qp[4][2];  // precision form: corners packed once per cut, [op N, op T]
  void* Qpmem[4][2];
  cplx* omt;
  cplx* thin[4];      // k x K work
  cplx* PT[2];        // chi x K, projector P transposed, per cut row
  cplx* Ptil[2];      // chi x K
  cplx* Vt;           // k x k
  cplx* Gsel;         // chi x k
  // precision forms: per cut (frame, position), the right singular vectors of
  // the core found at the previous visit (k x k, rows = columns of V), the
  // start of the next Jacobi SVD of that cut
  cplx* Vwarm[4][4];
  cplx* Hbond[4];     // 64x64 ruby bond operators: H_r, H_l, H_u, H_d
  double* sigma;
  double* s_sel;
  int* perm;
  int* counters;
  double* dwork;      // 4096 doubles
  double* dacc;       // 64 doubles
  cplx* scalar;       // 16 complex
  DevStatus* st;
  cplx* scratch;      // bump-allocated per operation
  long long scratch_elems, scratch_top;
  uint64_t launches_at_create;
  bool has_alt;       // second lane available (Ly or Lx == 2)
  bool no_alt;        // run the two cuts of a column one after the other
  Lane alt;
  TcTuner* tuner;     // tile choices of the tensor-core products, or null
  bool own_tuner;     // created by ipeps_ctm_autotune (else owned by a batch)
  cudaEvent_t ev_fork, ev_join;
  // CUDA graphs of the moves: one per direction (and one per sweep), captured
  // on the private stream cap_stream at first use, launched on `stream`
  cudaStream_t cap_stream;
  cudaGraphExec_t exec[5];
  int exec_kernels[5];  // kernels inside each graph (launch accounting)
  // optional per-kernel-class timing (CUDA events on the handle's stream)
  bool profiling;
  long long jac_sweeps, jac_calls;  // accumulated while profiling
  struct Rec {
    cudaEvent_t a, b;
    double flops;
    int kind;
    bool own_a = true, own_b = true;  // events shared between records belong to one of them
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
};

static cudaEvent_t pool_event(ipeps_ctm h) {
  if (!h->pool.empty()) {
    cudaEvent_t e = h->pool.back();
    h->pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

// kind 0: contraction GEMMs, 1: Jacobi SVDs
static void prof_begin(ipeps_ctm h, cudaEvent_t* a) {
  if (!h->profiling) return;
  *a = pool_event(h);
  cudaEventRecord(*a, h->stream);
}
static void prof_end(ipeps_ctm h, cudaEvent_t a, double flops, int kind) {
  if (!h->profiling) return;
  cudaEvent_t b = pool_event(h);
  cudaEventRecord(b, h->stream);
  h->recs.push_back({a, b, flops, kind});
}

// Tensor-core products, timed apart from their operand packing: kind 5 the
// main kernel of wide products (more than 256 output rows: enlarged corners,
// absorption, readouts; algorithmic flops), kind 6 the main kernel of thin
// products (at most 256 rows: the range finder and projector assembly;
// algorithmic flops) and kind 7 the same launches as kind 6 with the bytes the
// kernel must move (packed operands read once, output written once), kind 8
// the split-K reductions (bytes of partials read and output written).
static TcProbe* tc_probe_begin(ipeps_ctm h, TcProbe* p) {
  if (!h->profiling) return nullptr;
  for (int i = 0; i < 3; ++i) p->ev[i] = pool_event(h);
  return p;
}
static void tc_probe_end(ipeps_ctm h, TcProbe* p, int M, int N, int K) {
  if (!p) return;
  const double flops = 8.0 * (double)M * (double)N * (double)K;
  const bool thin = M <= 256;
  h->recs.push_back({p->ev[0], p->ev[1], flops, thin ? 6 : 5, true, true});
  if (thin) {
    const double ab = (double)p->Mp * p->Krp * p->elem_bytes * p->parts;
    const double bb = (double)p->Nrp * p->Krp * p->elem_bytes * p->parts;
    const double out = p->splits > 1 ? (double)p->splits * p->Mp * p->Nrp * 4.0 : (double)M * N * 16.0;
    h->recs.push_back({p->ev[0], p->ev[1], ab + bb + out, 7, false, false});
  }
  if (p->splits > 1)
    h->recs.push_back({p->ev[1], p->ev[2], (double)p->splits * p->Mp * p->Nrp * 4.0 + (double)M * N * 16.0, 8,
                       false, true});
  else
    h->pool.push_back(p->ev[2]);
}

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// NVTX range over a host scope (a move direction, a readout), so profilers can
// select or group the kernels it enqueues; a no-op when no tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// cudaMalloc that leaves no error behind when it fails: a failed allocation is
// also recorded as the runtime's last error, which the launch checks of every
// later call would otherwise report as their own failure.
static cudaError_t dev_alloc(void** p, size_t bytes) {
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
  }
  return e;
}

// swap the handle's active projector resources with the second lane
static void swap_lane(ipeps_ctm h) {
  std::swap(h->stream, h->alt.stream);
  for (int i = 0; i < 4; ++i) {
    std::swap(h->Q[i], h->alt.Q[i]);
    std::swap(h->thin[i], h->alt.thin[i]);
    for (int v = 0; v < 2; ++v) {
      std::swap(h->Qp[i][v], h->alt.Qp[i][v]);
      std::swap(h->Qpmem[i][v], h->alt.Qpmem[i][v]);
    }
  }
  std::swap(h->Vt, h->alt.Vt);
  std::swap(h->Gsel, h->alt.Gsel);
  std::swap(h->sigma, h->alt.sigma);
  std::swap(h->s_sel, h->alt.s_sel);
  std::swap(h->perm, h->alt.perm);
  std::swap(h->counters, h->alt.counters);
  std::swap(h->dwork, h->alt.dwork);
  std::swap(h->scratch, h->alt.scratch);
  std::swap(h->scratch_elems, h->alt.scratch_elems);
  std::swap(h->scratch_top, h->alt.scratch_top);
}

template <class Tp>
static Tp* carve(ipeps_ctm h, size_t count) {
  const size_t b = align_up(count * sizeof(Tp));
  if (h->used + b > h->bytes) return nullptr;
  Tp* p = (Tp*)(h->base + h->used);
  h->used += b;
  return p;
}

static cplx* scratch_alloc(ipeps_ctm h, long long n) {
  const long long nn = (n + 15) & ~15LL;
  if (h->scratch_top + nn > h->scratch_elems) return nullptr;
  cplx* p = h->scratch + h->scratch_top;
  h->scratch_top += nn;
  return p;
}

// the precision forms whose contraction products run on the BF16/TF32 tensor
// cores (FP32 accumulation); IPEPS_PREC_FP64TC runs every other step as the
// FP64 path does and only its products on the tensor cores, FP64-accurate
static bool tc_form(int prec) {
  return prec == IPEPS_PREC_TF32 || prec == IPEPS_PREC_BF16X3 || prec == IPEPS_PREC_BF16X6;
}

// sizes of everything a handle carves from its memory
struct Sizes {
  long long tens, a, C, T, Q, thin, proj, scratch;
  size_t total;
};

static Sizes plan_sizes(int Lx, int Ly, int d, int D, int chi, int k, int ntens, int prec) {
  Sizes s;
  const long long D2 = (long long)D * D, K = chi * D2;
  s.tens = (long long)d * D2 * D2;
  s.a = D2 * D2 * D2 * D2;
  s.C = (long long)chi * chi;
  s.T = (long long)chi * D2 * chi;
  s.Q = K * K;
  s.thin = (long long)k * K;
  s.proj = (long long)chi * K;
  // largest intermediates: RDM halves (chi^2 D^4 d, three of them) and the
  // enlarged-corner chain (a few K^2); boundary rings are below these.
  // rdm: L2, L3, L4 and two contraction temporaries of chi^2 D^4 d, the halves
  const long long rdm = 6 * (long long)chi * chi * D2 * D2 * d + 3 * (long long)chi * chi * D2 * d * d;
  s.scratch = std::max(6 * s.Q, rdm) + (1 << 16);
  // packed tensor-core operands (padded to 128 x 256 tiles) and split-K partials
  if (tc_form(prec)) s.scratch = s.scratch * (prec == IPEPS_PREC_BF16X6 ? 2 : 3) / 2 + (1 << 22);
  // digit planes of the FP64-accurate products: 28 B per complex element of
  // the A side, 56 B of the B side, and the exact split partials
  if (prec == IPEPS_PREC_FP64TC) s.scratch = s.scratch * 3 + (1 << 22);
  size_t tot = 0;
  auto add = [&](long long n, size_t el) { tot += align_up((size_t)n * el); };
  for (int i = 0; i < 2 * 4 * ntens; ++i) add(s.tens, 16);
  for (int i = 0; i < 4 * ntens; ++i) add(s.a, 16);
  for (int i = 0; i < 4 * Lx * Ly; ++i) { add(s.C, 16); add(s.T, 16); }
  for (int i = 0; i < 4; ++i) add(s.C, 16);
  for (int i = 0; i < 2; ++i) add(s.T, 16);
  for (int i = 0; i < 4; ++i) add(s.Q, 16);
  if (tc_form(prec))
    for (int i = 0; i < 8; ++i) tot += align_up(tc_packed_bytes(prec, (int)K, (int)K));
  add(s.thin, 16);
  for (int i = 0; i < 4; ++i) add(s.thin, 16);
  for (int i = 0; i < 4; ++i) add(s.proj, 16);
  add((long long)k * k, 16);
  add((long long)chi * k, 16);
  for (int i = 0; i < 4; ++i) add(64 * 64, 16);
  add(std::max(k, 4096), 8);
  add(std::max(k, 4096), 8);
  add(std::max(k, 4096), 4);
  add(4, 4);
  add(4096, 8);
  add(64, 8);
  add(16, 16);
  add(1, sizeof(DevStatus));
  add(s.scratch, 16);
  // second projector lane (the other cut of a column runs concurrently)
  for (int i = 0; i < 4; ++i) add(s.Q, 16);
  if (tc_form(prec))
    for (int i = 0; i < 8; ++i) tot += align_up(tc_packed_bytes(prec, (int)K, (int)K));
  for (int i = 0; i < 4; ++i) add(s.thin, 16);
  add((long long)k * k, 16);
  add((long long)chi * k, 16);
  add(std::max(k, 4096), 8);
  add(std::max(k, 4096), 8);
  add(std::max(k, 4096), 4);
  add(4, 4);
  add(4096, 8);
  if (prec != IPEPS_PREC_FP64)
    for (int i = 0; i < 4 * Lx * Ly; ++i) add((long long)k * k, 16);
  s.total = tot + 4096;
  return s;
}

// ---------------------------------------------------------------------------
// frames: frame f is the network rotated f times by 90 degrees counter-
// clockwise; environment role j of frame f is role (j+f) mod 4 of frame 0.
// ---------------------------------------------------------------------------
static void frame_dims(ipeps_ctm h, int f, int* Lx, int* Ly) {
  *Lx = (f & 1) ? h->Ly : h->Lx;
  *Ly = (f & 1) ? h->Lx : h->Ly;
}

// frame-f coordinates -> frame-0 coordinates
static void to_orig(ipeps_ctm h, int f, int x, int y, int* ox, int* oy) {
  int lx, ly;
  frame_dims(h, f, &lx, &ly);
  x = ((x % lx) + lx) % lx;
  y = ((y % ly) + ly) % ly;
  for (int g = f; g > 0; --g) {
    // frame g (dims lx, ly) -> frame g-1 (dims ly, lx): x_prev = -y, y_prev = x
    const int plx = ly, ply = lx;
    const int nx = ((-y) % plx + plx) % plx, ny = x % ply;
    x = nx;
    y = ny;
    lx = plx;
    ly = ply;
  }
  *ox = x;
  *oy = y;
}

static int cell_index(ipeps_ctm h, int f, int x, int y) {
  int ox, oy;
  to_orig(h, f, x, y, &ox, &oy);
  return oy * h->Lx + ox;
}

static cplx*& envC(ipeps_ctm h, int f, int j, int x, int y) {
  return h->C[(j + f) & 3][cell_index(h, f, x, y)];
}
static cplx*& envT(ipeps_ctm h, int f, int j, int x, int y) {
  return h->T[(j + f) & 3][cell_index(h, f, x, y)];
}
static int tensor_id(ipeps_ctm h, int f, int x, int y) {
  return h->pattern[cell_index(h, f, x, y)];
}
static cplx* site_a(ipeps_ctm h, int f, int x, int y) { return h->a[f][tensor_id(h, f, x, y)]; }

// ---------------------------------------------------------------------------
// contraction planner: C[labels] = alpha * A[labels] B[labels], every label of
// C appearing in exactly one operand, shared labels summed (transpose/permute
// into GEMM form, one complex GEMM, permute out if needed).
// ---------------------------------------------------------------------------
struct Plan {
  std::string la, lb, lc;
};

static ipeps_status gemm_dispatch_raw(ipeps_ctm h, int M, int N, int K, const cplx* A, long long lda,
                                      int opA, const cplx* B, long long ldb, int opB, cplx* C,
                                      long long ldc, cplx alpha);

static ipeps_status gemm_dispatch(ipeps_ctm h, int M, int N, int K, const cplx* A, long long lda,
                                  int opA, const cplx* B, long long ldb, int opB, cplx* C,
                                  long long ldc, cplx alpha) {
  cudaEvent_t a = nullptr;
  prof_begin(h, &a);
  ipeps_status st = gemm_dispatch_raw(h, M, N, K, A, lda, opA, B, ldb, opB, C, ldc, alpha);
  prof_end(h, a, 8.0 * (double)M * (double)N * (double)K, 0);
  return st;
}

static ipeps_status gemm_dispatch_raw(ipeps_ctm h, int M, int N, int K, const cplx* A, long long lda,
                                      int opA, const cplx* B, long long ldb, int opB, cplx* C,
                                      long long ldc, cplx alpha) {
  // FP64-accurate tensor-core products (unit alpha, the digit planes within
  // the scratch left); smaller products and the rest on the FP64 CUDA cores
  if (h->opt.prec == IPEPS_PREC_FP64TC && M >= 64 && N >= 32 && K >= 16 && alpha.x == 1.0 && alpha.y == 0.0 &&
      oz_work_bytes(M, N, K) <= (size_t)(h->scratch_elems - h->scratch_top) * sizeof(cplx)) {
    CK(oz_zgemm(h->stream, M, N, K, A, lda, opA, B, ldb, opB, C, ldc, h->scratch + h->scratch_top,
                (size_t)(h->scratch_elems - h->scratch_top) * sizeof(cplx), &h->st->tc_timeouts));
    return IPEPS_OK;
  }
  // small products (a few tiles of zero padding would dominate) stay FP64
  if (tc_form(h->opt.prec) && M >= 64 && N >= 32 && K >= 16) {
    TcProbe pr;
    TcProbe* p = tc_probe_begin(h, &pr);
    cudaError_t e = tc_zgemm(h->stream, (int)h->opt.prec, M, N, K, alpha, A, lda, opA, B, ldb,
                             opB, C, ldc, h->scratch, h->scratch_elems, h->scratch_top, &h->st->tc_timeouts,
                             h->tuner, nullptr, p);
    if (e == cudaSuccess) tc_probe_end(h, p, M, N, K);
    if (e == cudaErrorNotSupported) return fail(IPEPS_EUNSUPPORTED, "tensor-core GEMM unavailable for this shape");
    CK(e);
    return IPEPS_OK;
  }
  CK(zgemm(h->stream, M, N, K, alpha, A, lda, opA, B, ldb, opB, ZERO, C, ldc, GemmBatch{1, 0, 0, 0},
           h->scratch + h->scratch_top, h->scratch_elems - h->scratch_top));
  return IPEPS_OK;
}

// View of tensor X (labels lx) with rows over labels `rows` and columns over
// labels `cols` (each in the given order); adjacent axes contiguous in X are
// merged.  False when either side needs more than four axes.
static bool make_view(const TV& X, const std::string& lx, const std::string& rows, const std::string& cols,
                      bool cj, TcView* v) {
  long long str[8];
  long long acc = 1;
  for (int a = X.nd - 1; a >= 0; --a) {
    str[a] = acc;
    acc *= X.dims[a];
  }
  auto side = [&](const std::string& labs, int* n, int* dim, long long* st) {
    *n = 0;
    for (char c : labs) {
      const int a = (int)lx.find(c);
      if (*n > 0 && st[*n - 1] == str[a] * X.dims[a]) {  // contiguous with the previous axis: merge
        dim[*n - 1] *= X.dims[a];
        st[*n - 1] = str[a];
        continue;
      }
      if (*n == 4) return false;
      dim[*n] = X.dims[a];
      st[*n] = str[a];
      ++*n;
    }
    return true;
  };
  v->p = X.p;
  v->conj = cj ? 1 : 0;
  if (!side(rows, &v->nr, v->rdim, v->rstr) || !side(cols, &v->nc, v->cdim, v->cstr)) return false;
  if (v->nr == 0) { v->nr = 1; v->rdim[0] = 1; v->rstr[0] = 0; }
  if (v->nc == 0) { v->nc = 1; v->cdim[0] = 1; v->cstr[0] = 0; }
  return true;
}

static ipeps_status contract(ipeps_ctm h, const char* spec, TV A, bool conjA, TV B, bool conjB,
                             TV C, cplx alpha = ONE) {
  std::string s(spec);
  const size_t c1 = s.find(','), ar = s.find("->");
  if (c1 == std::string::npos || ar == std::string::npos)
    return fail(IPEPS_EINVAL, "bad contraction spec %s", spec);
  std::string la = s.substr(0, c1), lb = s.substr(c1 + 1, ar - c1 - 1), lc = s.substr(ar + 2);
  if ((int)la.size() != A.nd || (int)lb.size() != B.nd || (int)lc.size() != C.nd)
    return fail(IPEPS_EINVAL, "rank mismatch in %s", spec);
  auto dimA = [&](char c) { return A.dims[la.find(c)]; };
  auto dimB = [&](char c) { return B.dims[lb.find(c)]; };
  std::string fa, fb, kc;
  for (char c : la) (lb.find(c) == std::string::npos ? fa : kc) += c;
  for (char c : lb)
    if (la.find(c) == std::string::npos) fb += c;
  for (char c : kc)
    if (dimA(c) != dimB(c)) return fail(IPEPS_EINVAL, "dim mismatch on %c in %s", c, spec);
  for (char c : lc)
    if (la.find(c) == std::string::npos && lb.find(c) == std::string::npos)
      return fail(IPEPS_EINVAL, "output label %c not in inputs (%s)", c, spec);
  if (fa.size() + fb.size() != lc.size()) return fail(IPEPS_EINVAL, "batch labels unsupported: %s", spec);

  // output order: C = [fa', fb'] directly, or [fb', fa'] with the operands swapped
  bool swap = false, direct = false;
  std::string Mo, No;
  {
    std::string head = lc.substr(0, fa.size()), tail = lc.substr(fa.size());
    std::string sh = head, sf = fa;
    std::sort(sh.begin(), sh.end());
    std::sort(sf.begin(), sf.end());
    if (sh == sf) {
      direct = true;
      Mo = head;
      No = tail;
    } else {
      std::string head2 = lc.substr(0, fb.size()), tail2 = lc.substr(fb.size());
      std::string s2 = head2, sfb = fb;
      std::sort(s2.begin(), s2.end());
      std::sort(sfb.begin(), sfb.end());
      if (s2 == sfb) {
        direct = true;
        swap = true;
        Mo = tail2;   // rows of the A-side product are A's free labels ...
        No = head2;   // ... but C is stored [fb, fa]: compute C = B' A'
      } else {
        Mo = fa;
        No = fb;
      }
    }
  }
  long long M = 1, N = 1, Kd = 1;
  for (char c : fa) M *= dimA(c);
  for (char c : fb) N *= dimB(c);
  for (char c : kc) Kd *= dimA(c);

  const long long mark = h->scratch_top;
  // Tensor-core products: an operand that is not already in GEMM form is
  // gathered by the operand packing through a view (fused permute-and-pack)
  // instead of being permuted into a copy first.
  const bool tc = tc_form(h->opt.prec) &&
                  ((direct && swap) ? (N >= 64 && M >= 32 && Kd >= 16) : (M >= 64 && N >= 32 && Kd >= 16)) &&
                  (2 * std::max(M, N) + 512) * (2 * Kd + 128) < (1LL << 31);  // gathers index in 32 bits
  // arrange one operand as [free..., k...] (op N) or [k..., free...] (op T)
  auto arrange = [&](TV X, const std::string& lx, bool cj, const std::string& fo,
                     const std::string& ko, const cplx** out, long long* ld, int* op) -> ipeps_status {
    long long fdim = 1, kdim = 1;
    for (char c : fo) fdim *= X.dims[lx.find(c)];
    for (char c : ko) kdim *= X.dims[lx.find(c)];
    if (lx == fo + ko) {
      *out = X.p; *ld = kdim; *op = OP_N | (cj ? OP_CONJ : 0);
      return IPEPS_OK;
    }
    if (lx == ko + fo) {
      *out = X.p; *ld = fdim; *op = OP_T | (cj ? OP_CONJ : 0);
      return IPEPS_OK;
    }
    std::string want = fo + ko;
    int perm[8];
    for (size_t i = 0; i < want.size(); ++i) perm[i] = (int)lx.find(want[i]);
    cplx* t = scratch_alloc(h, X.size());
    if (!t) return fail(IPEPS_ENOMEM, "scratch exhausted in %s", spec);
    CK(permute(h->stream, X.p, t, X.nd, X.dims, perm, cj, ONE));
    *out = t; *ld = kdim; *op = OP_N;
    return IPEPS_OK;
  };
  // choose the contracted-label order from an operand that is already in GEMM form
  auto is_form = [](const std::string& lx, const std::string& f, const std::string& k) {
    return lx == f + k || lx == k + f;
  };
  std::string ko = kc;  // order as in A
  {
    std::string kb;
    for (char c : lb)
      if (la.find(c) != std::string::npos) kb += c;
    // prefer the order that leaves an operand untouched
    if (!is_form(la, swap ? Mo : Mo, kc) && !is_form(la, Mo, kc)) {
      if (is_form(lb, No, kb)) ko = kb;
    }
    if (!is_form(la, Mo, ko) && is_form(lb, No, kb)) ko = kb;
  }
  const cplx *pa = nullptr, *pb = nullptr;
  long long lda = 0, ldb = 0;
  int opa = OP_N, opb = OP_N;
  TcView va, vb;
  bool use_va = false, use_vb = false;
  if (tc && !is_form(la, Mo, ko)) use_va = make_view(A, la, Mo, ko, conjA, &va);
  if (!use_va) CKS(arrange(A, la, conjA, Mo, ko, &pa, &lda, &opa));
  // B must be [ko, No] (op N) or [No, ko] (op T); arrange() returns [No, ko] forms
  {
    long long fdim = 1, kdim = 1;
    for (char c : No) fdim *= dimB(c);
    for (char c : ko) kdim *= dimB(c);
    if (lb == ko + No) {
      pb = B.p; ldb = fdim; opb = OP_N | (conjB ? OP_CONJ : 0);
    } else if (lb == No + ko) {
      pb = B.p; ldb = kdim; opb = OP_T | (conjB ? OP_CONJ : 0);
    } else if (tc && make_view(B, lb, No, ko, conjB, &vb)) {
      use_vb = true;
    } else {
      std::string want = ko + No;
      int perm[8];
      for (size_t i = 0; i < want.size(); ++i) perm[i] = (int)lb.find(want[i]);
      cplx* t = scratch_alloc(h, B.size());
      if (!t) return fail(IPEPS_ENOMEM, "scratch exhausted in %s", spec);
      CK(permute(h->stream, B.p, t, B.nd, B.dims, perm, conjB, ONE));
      pb = t; ldb = fdim; opb = OP_N;
    }
  }
  // a plain operand as a view, for the products that take one view
  auto plain_view = [&](const cplx* p, long long ld, int op, int rows, int cols, bool as_b, TcView* v) {
    // A role: element (m, k) of op(A); B role: element (n, k) of op(B)^T
    const bool t = (op & OP_T) != 0;
    v->p = p;
    v->conj = (op & OP_CONJ) ? 1 : 0;
    v->nr = v->nc = 1;
    v->rdim[0] = rows;
    v->cdim[0] = cols;
    const bool row_major_rows = as_b ? t : !t;  // rows stride ld, columns stride 1
    v->rstr[0] = row_major_rows ? ld : 1;
    v->cstr[0] = row_major_rows ? 1 : ld;
  };
  if (use_va || use_vb) {
    // at least one gathered operand: one tensor-core product with views
    const TcView* VA = use_va ? &va : nullptr;
    const TcView* VB = use_vb ? &vb : nullptr;
    cudaEvent_t ev = nullptr;
    if (direct && swap) {
      // C[No, Mo] = B' A'^T: the B operand takes the A role, A the B role
      TcView xa, xb;
      if (VB) xa = *VB; else plain_view(pb, ldb, opb ^ OP_T, (int)N, (int)Kd, false, &xa);
      if (VA) xb = *VA; else plain_view(pa, lda, opa ^ OP_T, (int)M, (int)Kd, true, &xb);
      prof_begin(h, &ev);
      TcProbe pr;
      TcProbe* p = tc_probe_begin(h, &pr);
      cudaError_t e = tc_zgemm_views(h->stream, (int)h->opt.prec, (int)N, (int)M, (int)Kd, alpha, &xa, nullptr, 0, 0,
                                     &xb, nullptr, 0, 0, C.p, M, h->scratch, h->scratch_elems, h->scratch_top,
                                     &h->st->tc_timeouts, h->tuner, p);
      prof_end(h, ev, 8.0 * (double)M * (double)N * (double)Kd, 0);
      if (e == cudaSuccess) tc_probe_end(h, p, (int)N, (int)M, (int)Kd);
      CK(e);
    } else {
      cplx* out = C.p;
      cplx* t = nullptr;
      if (!direct) {
        t = scratch_alloc(h, M * N);
        if (!t) return fail(IPEPS_ENOMEM, "scratch exhausted in %s", spec);
        out = t;
      }
      prof_begin(h, &ev);
      TcProbe pr;
      TcProbe* p = tc_probe_begin(h, &pr);
      cudaError_t e = tc_zgemm_views(h->stream, (int)h->opt.prec, (int)M, (int)N, (int)Kd, direct ? alpha : ONE, VA,
                                     pa, lda, opa, VB, pb, ldb, opb, out, N, h->scratch, h->scratch_elems,
                                     h->scratch_top, &h->st->tc_timeouts, h->tuner, p);
      prof_end(h, ev, 8.0 * (double)M * (double)N * (double)Kd, 0);
      if (e == cudaSuccess) tc_probe_end(h, p, (int)M, (int)N, (int)Kd);
      CK(e);
      if (!direct) {
        std::string have = Mo + No;
        int dims[8], perm[8];
        for (size_t i = 0; i < have.size(); ++i)
          dims[i] = la.find(have[i]) != std::string::npos ? dimA(have[i]) : dimB(have[i]);
        for (size_t i = 0; i < lc.size(); ++i) perm[i] = (int)have.find(lc[i]);
        CK(permute(h->stream, t, C.p, (int)have.size(), dims, perm, false, alpha));
      }
    }
    h->scratch_top = mark;
    return IPEPS_OK;
  }
  if (direct && !swap) {
    CKS(gemm_dispatch(h, (int)M, (int)N, (int)Kd, pa, lda, opa, pb, ldb, opb, C.p, N, alpha));
  } else if (direct && swap) {
    // C[No, Mo] = (A' B')^T = B'^T A'^T
    auto flip = [](int op) { return op ^ OP_T; };
    CKS(gemm_dispatch(h, (int)N, (int)M, (int)Kd, pb, ldb, flip(opb), pa, lda, flip(opa), C.p, M, alpha));
  } else {
    cplx* t = scratch_alloc(h, M * N);
    if (!t) return fail(IPEPS_ENOMEM, "scratch exhausted in %s", spec);
    CKS(gemm_dispatch(h, (int)M, (int)N, (int)Kd, pa, lda, opa, pb, ldb, opb, t, N, ONE));
    // t has labels Mo+No; permute to lc
    std::string have = Mo + No;
    int dims[8], perm[8];
    for (size_t i = 0; i < have.size(); ++i)
      dims[i] = la.find(have[i]) != std::string::npos ? dimA(have[i]) : dimB(have[i]);
    for (size_t i = 0; i < lc.size(); ++i) perm[i] = (int)have.find(lc[i]);
    CK(permute(h->stream, t, C.p, (int)have.size(), dims, perm, false, alpha));
  }
  h->scratch_top = mark;
  return IPEPS_OK;
}

// ---------------------------------------------------------------------------
// host tables: ruby bond operators of App. A (block-site basis p = 4b1+2b2+b3,
// b = 0 meaning sigma^z = +1), each sigma^a sigma^a link weighted by -J_a.
// ---------------------------------------------------------------------------
struct CM {  // small dense complex matrix on the host
  int n;
  std::vector<double> re, im;
  explicit CM(int n_) : n(n_), re(n_ * n_, 0.0), im(n_ * n_, 0.0) {}
};

static CM kron(const CM& A, const CM& B) {
  CM R(A.n * B.n);
  for (int i = 0; i < A.n; ++i)
    for (int j = 0; j < A.n; ++j)
      for (int k = 0; k < B.n; ++k)
        for (int l = 0; l < B.n; ++l) {
          const int r = i * B.n + k, c = j * B.n + l;
          const double ar = A.re[i * A.n + j], ai = A.im[i * A.n + j];
          const double br = B.re[k * B.n + l], bi = B.im[k * B.n + l];
          R.re[r * R.n + c] = ar * br - ai * bi;
          R.im[r * R.n + c] = ar * bi + ai * br;
        }
  return R;
}

static CM matmul(const CM& A, const CM& B) {
  CM R(A.n);
  for (int i = 0; i < A.n; ++i)
    for (int j = 0; j < A.n; ++j) {
      double sr = 0, si = 0;
      for (int k = 0; k < A.n; ++k) {
        const double ar = A.re[i * A.n + k], ai = A.im[i * A.n + k];
        const double br = B.re[k * A.n + j], bi = B.im[k * A.n + j];
        sr += ar * br - ai * bi;
        si += ar * bi + ai * br;
      }
      R.re[i * A.n + j] = sr;
      R.im[i * A.n + j] = si;
    }
  return R;
}

static void axpy(CM& Y, double a, const CM& X) {
  for (size_t i = 0; i < Y.re.size(); ++i) {
    Y.re[i] += a * X.re[i];
    Y.im[i] += a * X.im[i];
  }
}

// sigma^alpha on spin k (1..3) of a block site, 8x8
static CM spin_op(char alpha, int k) {
  CM s(2), I2(2);
  I2.re[0] = I2.re[3] = 1.0;
  if (alpha == 'x') { s.re[1] = s.re[2] = 1.0; }
  if (alpha == 'y') { s.im[1] = -1.0; s.im[2] = 1.0; }
  if (alpha == 'z') { s.re[0] = 1.0; s.re[3] = -1.0; }
  const CM& f1 = k == 1 ? s : I2;
  const CM& f2 = k == 2 ? s : I2;
  const CM& f3 = k == 3 ? s : I2;
  return kron(kron(f1, f2), f3);
}

static void ruby_bonds(const double J[3], CM* Hr, CM* Hv) {
  CM I8(8);
  for (int i = 0; i < 8; ++i) I8.re[i * 8 + i] = 1.0;
  CM hs(8);
  axpy(hs, -J[2], matmul(spin_op('z', 1), spin_op('z', 2)));
  axpy(hs, -J[2], matmul(spin_op('z', 1), spin_op('z', 3)));
  axpy(hs, -J[2], matmul(spin_op('z', 2), spin_op('z', 3)));
  *Hr = CM(64);
  axpy(*Hr, -J[0], kron(spin_op('x', 1), spin_op('x', 1)));
  axpy(*Hr, -J[1], kron(spin_op('y', 3), spin_op('y', 3)));
  *Hv = CM(64);
  axpy(*Hv, 0.5, kron(hs, I8));
  axpy(*Hv, 0.5, kron(I8, hs));
  axpy(*Hv, -J[0], kron(spin_op('x', 3), spin_op('x', 2)));
  axpy(*Hv, -J[1], kron(spin_op('y', 2), spin_op('y', 1)));
}

// ---------------------------------------------------------------------------
// create / destroy
// ---------------------------------------------------------------------------
extern "C" void ipeps_default_options(ipeps_options* o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->chi = 0;
  o->prec = IPEPS_PREC_FP64;
  o->rsvd_oversample = 16;
  o->rsvd_power = 2;
  o->svd_cutoff = 0.0;  // automatic by precision
  o->orth_tol = 1e-14;
  o->omega_seed = 7;
  o->jacobi_max_sweeps = 40;
  o->corners = 4;
}

static ipeps_status validate(const ipeps_cell* c, const ipeps_options* o) {
  if (!c || !o) return fail(IPEPS_EINVAL, "null cell or options");
  if (c->Lx < 1 || c->Lx > 2 || c->Ly < 1 || c->Ly > 2) return fail(IPEPS_EINVAL, "Lx, Ly must be 1 or 2");
  if (c->n_tensors < 1 || c->n_tensors > 4) return fail(IPEPS_EINVAL, "n_tensors must be 1..4");
  for (int i = 0; i < c->Lx * c->Ly; ++i)
    if (c->pattern[i] < 0 || c->pattern[i] >= c->n_tensors) return fail(IPEPS_EINVAL, "pattern id out of range");
  if (c->d < 1 || c->d > 64 || c->D < 1 || c->D > 12) return fail(IPEPS_EINVAL, "d in 1..64, D in 1..12");
  if (c->dtype != IPEPS_REAL64 && c->dtype != IPEPS_COMPLEX128) return fail(IPEPS_EINVAL, "bad dtype");
  if (!c->tensors) return fail(IPEPS_EINVAL, "null tensors");
  if (c->leg_dims)
    for (int i = 0; i < 4 * c->n_tensors; ++i)
      if (c->leg_dims[i] != 1 && c->leg_dims[i] != c->D)
        return fail(IPEPS_EINVAL, "leg_dims[%d] = %d: legs are 1 (trivial) or D", i, c->leg_dims[i]);
  if (o->chi < c->D * c->D) return fail(IPEPS_EINVAL, "chi (%d) must be >= D*D (%d)", o->chi, c->D * c->D);
  if (o->chi > 1024) return fail(IPEPS_EINVAL, "chi > 1024");
  if (o->rsvd_oversample < 0 || o->rsvd_power < 0) return fail(IPEPS_EINVAL, "bad rsvd options");
  if (o->chi + o->rsvd_oversample > 1024) return fail(IPEPS_EINVAL, "chi + oversample > 1024");
  if (o->prec < IPEPS_PREC_FP64 || o->prec > IPEPS_PREC_FP64TC) return fail(IPEPS_EINVAL, "bad prec");
  if (o->jacobi_max_sweeps < 1) return fail(IPEPS_EINVAL, "jacobi_max_sweeps >= 1");
  if (o->corners != 0 && o->corners != 2 && o->corners != 4) return fail(IPEPS_EINVAL, "corners must be 2 or 4");
  return IPEPS_OK;
}

extern "C" ipeps_status ipeps_ctm_workspace_size(const ipeps_cell* c, const ipeps_options* o,
                                                 size_t* bytes) {
  CKS(validate(c, o));
  if (!bytes) return fail(IPEPS_EINVAL, "null bytes");
  Sizes s = plan_sizes(c->Lx, c->Ly, c->d, c->D, o->chi, o->chi + o->rsvd_oversample, c->n_tensors, o->prec);
  *bytes = s.total;
  return IPEPS_OK;
}

static ipeps_status build_layers(ipeps_ctm h) {
  // rotated site tensors: A'[p,u,l,d,r] = A[p,l,d,r,u] per counter-clockwise turn
  const int dims5[5] = {h->d, h->D, h->D, h->D, h->D};
  const int rot5[5] = {0, 4, 1, 2, 3};
  for (int t = 0; t < h->ntens; ++t) {
    for (int f = 1; f < 4; ++f) {
      CK(permute(h->stream, h->A[f - 1][t], h->A[f][t], 5, dims5, rot5, false, ONE));
      CK(permute(h->stream, h->Bt[f - 1][t], h->Bt[f][t], 5, dims5, rot5, false, ONE));
    }
    CK(double_layer(h->stream, h->A[0][t], h->Bt[0][t], h->a[0][t], h->d, h->D));
    for (int f = 1; f < 4; ++f) CK(rotate_a(h->stream, h->a[f - 1][t], h->a[f][t], h->D2));
  }
  return IPEPS_OK;
}

static ipeps_status trace_init_env(ipeps_ctm h) {
  // a fresh environment starts every cut's Jacobi SVD from the identity again
  for (int f = 0; f < 4; ++f)
    for (int i = 0; i < 4; ++i)
      if (h->Vwarm[f][i]) CK(set_identity(h->stream, h->Vwarm[f][i], h->k));
  // role -> neighbouring site offset (frame 0)
  static const int off[8][2] = {{-1, -1}, {1, -1}, {1, 1}, {-1, 1}, {0, -1}, {1, 0}, {0, 1}, {-1, 0}};
  for (int y = 0; y < h->Ly; ++y)
    for (int x = 0; x < h->Lx; ++x)
      for (int r = 0; r < 8; ++r) {
        const int sx = ((x + off[r][0]) % h->Lx + h->Lx) % h->Lx;
        const int sy = ((y + off[r][1]) % h->Ly + h->Ly) % h->Ly;
        const cplx* a = h->a[0][h->pattern[sy * h->Lx + sx]];
        cplx* out = r < 4 ? h->C[r][y * h->Lx + x] : h->T[r - 4][y * h->Lx + x];
        CK(trace_init_tensor(h->stream, a, out, r, h->D, h->chi));
        const long long n = r < 4 ? (long long)h->chi * h->chi : (long long)h->chi * h->D2 * h->chi;
        CK(normalize(h->stream, out, n, h->dwork, h->st));
      }
  return IPEPS_OK;
}

static ipeps_status upload_one(ipeps_ctm h, const void* src, cplx* dst, std::vector<double>& buf, int t);

static ipeps_status check_status(ipeps_ctm h) {
  DevStatus st;
  CK(cudaMemcpyAsync(&st, h->st, sizeof st, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (h->profiling) {
    h->jac_sweeps += st.jacobi_sweeps;
    h->jac_calls += st.jacobi_calls;
  }
  if (st.nonfinite) return fail(IPEPS_ENUMERIC, "non-finite or zero norm met (%d times)", st.nonfinite);
  if (st.barrier_timeouts)  // before the sweep budget: a CTA that gave up leaves its SVD unconverged too
    return fail(IPEPS_ETIMEOUT, "%d grid-barrier waits of the Jacobi SVD ran out", st.barrier_timeouts);
  if (st.jacobi_unconverged)
    return fail(IPEPS_ETIMEOUT, "%d Jacobi SVDs hit the sweep budget", st.jacobi_unconverged);
  if (st.tc_timeouts) return fail(IPEPS_ETIMEOUT, "%d tensor-core GEMM waits timed out", st.tc_timeouts);
  return IPEPS_OK;
}

// Called where every operation starts.  The scratch arenas are bump-allocated
// per operation: an operation that failed part way may have left its
// allocations in place, so they are released here as well.
static ipeps_status reset_status(ipeps_ctm h) {
  h->scratch_top = 0;
  h->alt.scratch_top = 0;
  CK(cudaMemsetAsync(h->st, 0, sizeof(DevStatus), h->stream));
  return IPEPS_OK;
}

// The second lane's stream and its fork/join events: each released if it was
// created (creation can stop part way, leaving has_alt false).
static void drop_graphs(ipeps_ctm h) {
  for (int d = 0; d < 5; ++d)
    if (h->exec[d]) {
      cudaGraphExecDestroy(h->exec[d]);
      h->exec[d] = nullptr;
    }
}

static void release_lane(ipeps_ctm h) {
  drop_graphs(h);
  if (h->cap_stream) {
    cudaStreamDestroy(h->cap_stream);
    h->cap_stream = nullptr;
  }
  if (h->alt.stream) {
    cudaStreamSynchronize(h->alt.stream);
    cudaStreamDestroy(h->alt.stream);
    h->alt.stream = nullptr;
  }
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  h->ev_fork = h->ev_join = nullptr;
  h->has_alt = false;
}

extern "C" ipeps_status ipeps_ctm_create(const ipeps_cell* c, const ipeps_options* o, ipeps_ctm* out) {
  CKS(validate(c, o));
  if (!out) return fail(IPEPS_EINVAL, "null out");
  ipeps_ctm h = new ipeps_ctm_s();
  h->Lx = c->Lx; h->Ly = c->Ly; h->d = c->d; h->D = c->D; h->D2 = c->D * c->D;
  h->chi = o->chi; h->K = o->chi * h->D2; h->k = o->chi + o->rsvd_oversample;
  h->ntens = c->n_tensors;
  for (int i = 0; i < 4; ++i) h->pattern[i] = i < c->Lx * c->Ly ? c->pattern[i] : 0;
  h->mixed = c->tensors_bra != nullptr;
  for (int t = 0; t < 4; ++t)
    for (int q = 0; q < 4; ++q) h->leg[t][q] = (c->leg_dims && t < c->n_tensors) ? c->leg_dims[4 * t + q] : c->D;
  h->dtype = c->dtype;
  h->opt = *o;
  if (!(h->opt.svd_cutoff > 0.0))  // automatic: above the noise floor of the contraction arithmetic
    h->opt.svd_cutoff = !tc_form(o->prec) ? 1e-8 : (o->prec == IPEPS_PREC_TF32 ? 1e-5 : 1e-6);
  h->stream = (cudaStream_t)o->stream;
  Sizes sz = plan_sizes(h->Lx, h->Ly, h->d, h->D, h->chi, h->k, h->ntens, o->prec);
  if (o->workspace) {
    if (o->workspace_bytes < sz.total) {
      delete h;
      return fail(IPEPS_ENOMEM, "workspace too small: %zu < %zu bytes", o->workspace_bytes, sz.total);
    }
    h->base = (char*)o->workspace;
    h->bytes = o->workspace_bytes;
    h->own_mem = false;
  } else {
    cudaError_t e = dev_alloc((void**)&h->base, sz.total);
    if (e != cudaSuccess) {
      delete h;
      return fail(IPEPS_ENOMEM, "cudaMalloc(%zu) failed: %s", sz.total, cudaGetErrorString(e));
    }
    h->bytes = sz.total;
    h->own_mem = true;
  }
  h->used = 0;
  bool ok = true;
  auto need = [&](void* p) { if (!p) ok = false; };
  for (int f = 0; f < 4; ++f)
    for (int t = 0; t < h->ntens; ++t) {
      need(h->A[f][t] = carve<cplx>(h, sz.tens));
      need(h->Bt[f][t] = carve<cplx>(h, sz.tens));
      need(h->a[f][t] = carve<cplx>(h, sz.a));
    }
  for (int j = 0; j < 4; ++j)
    for (int i = 0; i < h->Lx * h->Ly; ++i) {
      need(h->C[j][i] = carve<cplx>(h, sz.C));
      need(h->T[j][i] = carve<cplx>(h, sz.T));
    }
  for (int i = 0; i < 2; ++i) {
    need(h->spareC[0][i] = carve<cplx>(h, sz.C));
    need(h->spareC[1][i] = carve<cplx>(h, sz.C));
    need(h->spareT[i] = carve<cplx>(h, sz.T));
  }
  for (int i = 0; i < 4; ++i) need(h->Q[i] = carve<cplx>(h, sz.Q));
  if (tc_form(o->prec))
    for (int i = 0; i < 4; ++i)
      for (int v = 0; v < 2; ++v) need(h->Qpmem[i][v] = carve<char>(h, tc_packed_bytes(o->prec, h->K, h->K)));
  need(h->omt = carve<cplx>(h, sz.thin));
  for (int i = 0; i < 4; ++i) need(h->thin[i] = carve<cplx>(h, sz.thin));
  for (int i = 0; i < 2; ++i) {
    need(h->PT[i] = carve<cplx>(h, sz.proj));
    need(h->Ptil[i] = carve<cplx>(h, sz.proj));
  }
  need(h->Vt = carve<cplx>(h, (size_t)h->k * h->k));
  need(h->Gsel = carve<cplx>(h, (size_t)h->chi * h->k));
  for (int i = 0; i < 4; ++i) need(h->Hbond[i] = carve<cplx>(h, 64 * 64));
  need(h->sigma = carve<double>(h, std::max(h->k, 4096)));
  need(h->s_sel = carve<double>(h, std::max(h->k, 4096)));
  need(h->perm = carve<int>(h, std::max(h->k, 4096)));
  need(h->counters = carve<int>(h, 4));
  need(h->dwork = carve<double>(h, 4096));
  need(h->dacc = carve<double>(h, 64));
  need(h->scalar = carve<cplx>(h, 16));
  need(h->st = carve<DevStatus>(h, 1));
  need(h->scratch = carve<cplx>(h, sz.scratch));
  h->scratch_elems = sz.scratch;
  h->scratch_top = 0;
  for (int i = 0; i < 4; ++i) need(h->alt.Q[i] = carve<cplx>(h, sz.Q));
  if (tc_form(o->prec))
    for (int i = 0; i < 4; ++i)
      for (int v = 0; v < 2; ++v) need(h->alt.Qpmem[i][v] = carve<char>(h, tc_packed_bytes(o->prec, h->K, h->K)));
  for (int i = 0; i < 4; ++i) need(h->alt.thin[i] = carve<cplx>(h, sz.thin));
  need(h->alt.Vt = carve<cplx>(h, (size_t)h->k * h->k));
  need(h->alt.Gsel = carve<cplx>(h, (size_t)h->chi * h->k));
  need(h->alt.sigma = carve<double>(h, std::max(h->k, 4096)));
  need(h->alt.s_sel = carve<double>(h, std::max(h->k, 4096)));
  need(h->alt.perm = carve<int>(h, std::max(h->k, 4096)));
  need(h->alt.counters = carve<int>(h, 4));
  need(h->alt.dwork = carve<double>(h, 4096));
  for (int f = 0; f < 4; ++f)
    for (int i = 0; i < 4; ++i)
      h->Vwarm[f][i] = (o->prec != IPEPS_PREC_FP64 && i < h->Lx * h->Ly) ? carve<cplx>(h, (size_t)h->k * h->k) : nullptr;
  for (int f = 0; f < 4 && o->prec != IPEPS_PREC_FP64; ++f)
    for (int i = 0; i < h->Lx * h->Ly; ++i) need(h->Vwarm[f][i]);
  if (!ok) {
    if (h->own_mem) cudaFree(h->base);
    delete h;
    return fail(IPEPS_ENOMEM, "arena layout exceeded (internal)");
  }
  h->launches_at_create = launch_counter();
  ipeps_status st = IPEPS_OK;
  h->has_alt = false;
  if (cudaStreamCreateWithFlags(&h->alt.stream, cudaStreamNonBlocking) == cudaSuccess &&
      cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
      cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) == cudaSuccess)
    h->has_alt = true;
  if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    h->cap_stream = nullptr;  // moves then run without graphs
  }
  // host -> device copies of the tensors (real inputs promoted to complex)
  std::vector<double> buf;
  for (int t = 0; t < h->ntens && st == IPEPS_OK; ++t) {
    const void* ket = c->tensors[t];
    const void* bra = h->mixed ? c->tensors_bra[t] : c->tensors[t];
    if (!ket || !bra) { st = fail(IPEPS_EINVAL, "null tensor pointer %d", t); break; }
    st = upload_one(h, ket, h->A[0][t], buf, t);
    if (st == IPEPS_OK) st = upload_one(h, bra, h->Bt[0][t], buf, t);
  }
  if (st == IPEPS_OK) st = reset_status(h);
  if (st == IPEPS_OK) st = build_layers(h);
  if (st == IPEPS_OK) {
    cudaError_t e = fill_omega_t(h->stream, h->omt, h->k, h->K, o->omega_seed);
    if (e != cudaSuccess) st = fail(IPEPS_ECUDA, "omega: %s", cudaGetErrorString(e));
  }
  if (st == IPEPS_OK) st = trace_init_env(h);
  if (st == IPEPS_OK) st = check_status(h);
  if (st != IPEPS_OK) {
    release_lane(h);
    if (h->own_mem) cudaFree(h->base);
    delete h;
    return st;
  }
  *out = h;
  return IPEPS_OK;
}

extern "C" ipeps_status ipeps_ctm_profile(ipeps_ctm h, int enable) {
  if (!h) return fail(IPEPS_EINVAL, "null handle");
  CK(cudaStreamSynchronize(h->stream));
  for (auto& r : h->recs) {
    if (r.own_a) h->pool.push_back(r.a);
    if (r.own_b) h->pool.push_back(r.b);
  }
  h->recs.clear();
  h->profiling = enable != 0;
  h->jac_sweeps = h->jac_calls = 0;
  return IPEPS_OK;
}

extern "C" ipeps_status ipeps_ctm_profile_read(ipeps_ctm h, int kind, double* total_ms,
                                               uint64_t* launches, double* flops) {
  if (!h) return fail(IPEPS_EINVAL, "null handle");
  CK(cudaStreamSynchronize(h->stream));
  double ms = 0, fl = 0;
  uint64_t n = 0;
  for (auto& r : h->recs) {
    if (r.kind != kind) continue;
    float t = 0;
    CK(cudaEventElapsedTime(&t, r.a, r.b));
    ms += t;
    fl += r.flops;
    ++n;
  }
  if (kind == 1) fl = h->jac_calls ? (double)h->jac_sweeps / (double)h->jac_calls : 0.0;
  if (total_ms) *total_ms = ms;
  if (launches) *launches = n;
  if (flops) *flops = fl;
  return IPEPS_OK;
}

extern "C" void ipeps_ctm_destroy(ipeps_ctm h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  for (auto& r : h->recs) {
    if (r.own_a) cudaEventDestroy(r.a);
    if (r.own_b) cudaEventDestroy(r.b);
  }
  for (auto e : h->pool) cudaEventDestroy(e);
  release_lane(h);
  if (h->own_tuner) tc_tuner_destroy(h->tuner);
  if (h->own_mem) cudaFree(h->base);
  delete h;
}

extern "C" ipeps_status ipeps_ctm_sync(ipeps_ctm h) {
  if (!h) return fail(IPEPS_EINVAL, "null handle");
  CK(cudaStreamSynchronize(h->stream));
  return IPEPS_OK;
}

extern "C" uint64_t ipeps_ctm_launch_count(ipeps_ctm h) {
  return h ? launch_counter() - h->launches_at_create : 0;
}

static ipeps_status upload_one(ipeps_ctm h, const void* src, cplx* dst, std::vector<double>& buf, int t) {
  const long long n = (long long)h->d * h->D2 * h->D2;
  const double* sp = (const double*)src;
  const int* L = h->leg[t];
  const bool trivial = L[0] < h->D || L[1] < h->D || L[2] < h->D || L[3] < h->D;
  if (h->dtype == IPEPS_REAL64 || trivial) {
    // host-side promotion of real inputs; legs of size 1 embedded at index 0 of a D leg
    buf.assign(2 * n, 0.0);
    const int cw = h->dtype == IPEPS_REAL64 ? 1 : 2;  // doubles per input element
    long long i = 0;
    for (int p = 0; p < h->d; ++p)
      for (int u = 0; u < L[0]; ++u)
        for (int l = 0; l < L[1]; ++l)
          for (int dd = 0; dd < L[2]; ++dd)
            for (int r = 0; r < L[3]; ++r, ++i) {
              const long long o = (((long long)p * h->D + u) * h->D + l) * h->D2 + (long long)dd * h->D + r;
              buf[2 * o] = sp[cw * i];
              buf[2 * o + 1] = cw == 2 ? sp[cw * i + 1] : 0.0;
            }
    sp = buf.data();
  }
  CK(cudaMemcpyAsync(dst, sp, n * sizeof(cplx), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));  // the staging buffer is reused
  return IPEPS_OK;
}

extern "C" ipeps_status ipeps_ctm_set_tensors(ipeps_ctm h, const void* const* tensors,
                                              const void* const* tensors_bra) {
  if (!h) return fail(IPEPS_EINVAL, "null handle");
  if (!tensors) {  // rebuild the double layers from the device-resident tensors
    CKS(build_layers(h));
    return IPEPS_OK;
  }
  if ((tensors_bra != nullptr) != h->mixed) return fail(IPEPS_EINVAL, "bra tensors must match create");
  std::vector<double> buf;
  for (int t = 0; t < h->ntens; ++t) {
    if (!tensors[t] || (h->mixed && !tensors_bra[t])) return fail(IPEPS_EINVAL, "null tensor %d", t);
    CKS(upload_one(h, tensors[t], h->A[0][t], buf, t));
    CKS(upload_one(h, h->mixed ? tensors_bra[t] : tensors[t], h->Bt[0][t], buf, t));
  }
  CKS(build_layers(h));
  CK(cudaStreamSynchronize(h->stream));
  return IPEPS_OK;
}

extern "C" ipeps_status ipeps_ctm_reset_env(ipeps_ctm h) {
  if (!h) return fail(IPEPS_EINVAL, "null handle");
  CKS(reset_status(h));
  CKS(trace_init_env(h));
  return check_status(h);
}

// ---------------------------------------------------------------------------
// the move
// ---------------------------------------------------------------------------
// Enlarged corners of the plaquette with upper-left site (x,y) in frame f:
//   Q1[(d_T4,d_a),(r_T1,r_a)]  Q2[(l_T1,l_a),(d_T2,d_a)]
//   Q3[(u_T2,u_a),(l_T3,l_a)]  Q4[(u_T4,u_a),(r_T3,r_a)]
// the two-corner projector (ipeps_options.corners = 2): X = Q1^T Q4
static bool two_corners(ipeps_ctm h) { return h->opt.corners == 2; }

static ipeps_status enlarged_corners(ipeps_ctm h, int f, int x, int y) {
  const int c = h->chi, D2 = h->D2;
  const long long entry = h->scratch_top;
  cplx* w1 = scratch_alloc(h, (long long)c * D2 * c);
  cplx* w2 = scratch_alloc(h, (long long)h->K * h->K);
  if (!w1 || !w2) return fail(IPEPS_ENOMEM, "scratch exhausted (corners)");
  const long long mark = h->scratch_top;
  // Q1 = ((C1 T1) T4) a
  CKS(contract(h, "ab,bcr->acr", tv(envC(h, f, 0, x, y), {c, c}), false,
               tv(envT(h, f, 0, x, y), {c, D2, c}), false, tv(w1, {c, D2, c})));
  CKS(contract(h, "dea,acr->decr", tv(envT(h, f, 3, x, y), {c, D2, c}), false, tv(w1, {c, D2, c}),
               false, tv(w2, {c, D2, D2, c})));
  CKS(contract(h, "decr,ceDR->dDrR", tv(w2, {c, D2, D2, c}), false,
               tv(site_a(h, f, x, y), {D2, D2, D2, D2}), false, tv(h->Q[0], {c, D2, c, D2})));
  h->scratch_top = mark;
  if (two_corners(h)) goto lower_left;  // Q2 and Q3 are not part of the two-corner ring
  // Q2 = ((T1 C2) T2) a
  CKS(contract(h, "Ltg,gh->Lth", tv(envT(h, f, 0, x + 1, y), {c, D2, c}), false,
               tv(envC(h, f, 1, x + 1, y), {c, c}), false, tv(w1, {c, D2, c})));
  CKS(contract(h, "Lth,hmE->LtmE", tv(w1, {c, D2, c}), false, tv(envT(h, f, 1, x + 1, y), {c, D2, c}),
               false, tv(w2, {c, D2, D2, c})));
  CKS(contract(h, "LtmE,tKem->LKEe", tv(w2, {c, D2, D2, c}), false,
               tv(site_a(h, f, x + 1, y), {D2, D2, D2, D2}), false, tv(h->Q[1], {c, D2, c, D2})));
  h->scratch_top = mark;
  // Q3 = ((T2 C3) T3) a
  CKS(contract(h, "Umh,hg->Umg", tv(envT(h, f, 1, x + 1, y + 1), {c, D2, c}), false,
               tv(envC(h, f, 2, x + 1, y + 1), {c, c}), false, tv(w1, {c, D2, c})));
  CKS(contract(h, "Umg,gtL->UmtL", tv(w1, {c, D2, c}), false,
               tv(envT(h, f, 2, x + 1, y + 1), {c, D2, c}), false, tv(w2, {c, D2, D2, c})));
  CKS(contract(h, "UmtL,uKtm->UuLK", tv(w2, {c, D2, D2, c}), false,
               tv(site_a(h, f, x + 1, y + 1), {D2, D2, D2, D2}), false, tv(h->Q[2], {c, D2, c, D2})));
  h->scratch_top = mark;
lower_left:
  // Q4 = ((C4 T4) T3) a
  CKS(contract(h, "gh,hmU->gmU", tv(envC(h, f, 3, x, y + 1), {c, c}), false,
               tv(envT(h, f, 3, x, y + 1), {c, D2, c}), false, tv(w1, {c, D2, c})));
  CKS(contract(h, "gmU,Rtg->mUtR", tv(w1, {c, D2, c}), false, tv(envT(h, f, 2, x, y + 1), {c, D2, c}),
               false, tv(w2, {D2, c, D2, c})));
  CKS(contract(h, "mUtR,umtr->UuRr", tv(w2, {D2, c, D2, c}), false,
               tv(site_a(h, f, x, y + 1), {D2, D2, D2, D2}), false, tv(h->Q[3], {c, D2, c, D2})));
  h->scratch_top = entry;
  return IPEPS_OK;
}

// thin (k x K, row-major = transposed K x k) times one corner
static ipeps_status thin_mul(ipeps_ctm h, const cplx* in, int opin, cplx* out, const cplx* Qm, int opQ,
                             int rows) {
  return gemm_dispatch(h, rows, h->K, h->K, in, h->K, opin, Qm, h->K, opQ, out, h->K, ONE);
}

// precision form: in (op opin) times the pre-packed corner q in variant v
// (0: Q, 1: Q^T); the result is conjugated when conj_out.
static ipeps_status thin_mul_packed(ipeps_ctm h, const cplx* in, int opin, cplx* out, int q, int v, int rows,
                                    bool conj_out) {
  cudaEvent_t a = nullptr;
  prof_begin(h, &a);
  TcProbe pr;
  TcProbe* p = tc_probe_begin(h, &pr);
  cudaError_t e = tc_zgemm_packed(h->stream, (int)h->opt.prec, rows, ONE, in, h->K, opin, h->Qp[q][v], out, h->K,
                                  conj_out, h->scratch, h->scratch_elems, h->scratch_top, &h->st->tc_timeouts,
                                  h->tuner, p);
  prof_end(h, a, 8.0 * (double)rows * (double)h->K * (double)h->K, 0);
  if (e == cudaSuccess) tc_probe_end(h, p, rows, h->K, h->K);
  CK(e);
  return IPEPS_OK;
}

static ipeps_status pack_corners(ipeps_ctm h) {
  for (int q = 0; q < 4; ++q) {
    if (two_corners(h) && (q == 1 || q == 2)) continue;
    for (int v = 0; v < 2; ++v)
      CK(tc_pack_b(h->stream, (int)h->opt.prec, h->Q[q], h->K, v ? OP_T : OP_N, h->K, h->K, h->Qpmem[q][v],
                   &h->Qp[q][v]));
  }
  return IPEPS_OK;
}

static bool packed_path(ipeps_ctm h) { return tc_form(h->opt.prec); }

// Yt = In * Q3 * Q4^T * Q1 * Q2      (the transpose of X * In^T)
// two corners: Yt = In * Q4^T * Q1
static ipeps_status apply_XT(ipeps_ctm h, const cplx* in, cplx* out, int rows) {
  if (two_corners(h)) {
    if (packed_path(h)) {
      CKS(thin_mul_packed(h, in, OP_N, h->thin[2], 3, 1, rows, false));
      CKS(thin_mul_packed(h, h->thin[2], OP_N, out, 0, 0, rows, false));
    } else {
      CKS(thin_mul(h, in, OP_N, h->thin[2], h->Q[3], OP_T, rows));
      CKS(thin_mul(h, h->thin[2], OP_N, out, h->Q[0], OP_N, rows));
    }
    return IPEPS_OK;
  }
  if (packed_path(h)) {
    CKS(thin_mul_packed(h, in, OP_N, h->thin[2], 2, 0, rows, false));
    CKS(thin_mul_packed(h, h->thin[2], OP_N, h->thin[3], 3, 1, rows, false));
    CKS(thin_mul_packed(h, h->thin[3], OP_N, h->thin[2], 0, 0, rows, false));
    CKS(thin_mul_packed(h, h->thin[2], OP_N, out, 1, 0, rows, false));
    return IPEPS_OK;
  }
  CKS(thin_mul(h, in, OP_N, h->thin[2], h->Q[2], OP_N, rows));
  CKS(thin_mul(h, h->thin[2], OP_N, h->thin[3], h->Q[3], OP_T, rows));
  CKS(thin_mul(h, h->thin[3], OP_N, h->thin[2], h->Q[0], OP_N, rows));
  CKS(thin_mul(h, h->thin[2], OP_N, out, h->Q[1], OP_N, rows));
  return IPEPS_OK;
}
// Zt = In * Q2^H * Q1^H * conj(Q4) * Q3^H   (the transpose of X^H * In^T)
//    = conj( conj(In) * Q2^T * Q1^T * Q4 * Q3^T )
// two corners: Zt = In * Q1^H * conj(Q4) = conj( conj(In) * Q1^T * Q4 )
static ipeps_status apply_XHT(ipeps_ctm h, const cplx* in, cplx* out, int rows) {
  if (two_corners(h)) {
    if (packed_path(h)) {
      CKS(thin_mul_packed(h, in, OP_C, h->thin[2], 0, 1, rows, false));
      CKS(thin_mul_packed(h, h->thin[2], OP_N, out, 3, 0, rows, true));
    } else {
      CKS(thin_mul(h, in, OP_N, h->thin[2], h->Q[0], OP_H, rows));
      CKS(thin_mul(h, h->thin[2], OP_N, out, h->Q[3], OP_C, rows));
    }
    return IPEPS_OK;
  }
  if (packed_path(h)) {
    CKS(thin_mul_packed(h, in, OP_C, h->thin[2], 1, 1, rows, false));
    CKS(thin_mul_packed(h, h->thin[2], OP_N, h->thin[3], 0, 1, rows, false));
    CKS(thin_mul_packed(h, h->thin[3], OP_N, h->thin[2], 3, 0, rows, false));
    CKS(thin_mul_packed(h, h->thin[2], OP_N, out, 2, 1, rows, true));
    return IPEPS_OK;
  }
  CKS(thin_mul(h, in, OP_N, h->thin[2], h->Q[1], OP_H, rows));
  CKS(thin_mul(h, h->thin[2], OP_N, h->thin[3], h->Q[0], OP_H, rows));
  CKS(thin_mul(h, h->thin[3], OP_N, h->thin[2], h->Q[3], OP_C, rows));
  CKS(thin_mul(h, h->thin[2], OP_N, out, h->Q[2], OP_H, rows));
  return IPEPS_OK;
}

static ipeps_status orth(ipeps_ctm h, cplx* G) {
  cudaEvent_t a = nullptr;
  prof_begin(h, &a);
  CK(jacobi_rows(h->stream, G, h->k, h->K, h->K, nullptr, h->sigma, h->opt.jacobi_max_sweeps,
                 h->dwork, h->counters, h->st, nullptr, 0, h->opt.wait_cycles));
  prof_end(h, a, 0.0, 1);
  CK(orth_rows_finish(h->stream, G, h->k, h->K, h->K, h->sigma, h->opt.orth_tol));
  return IPEPS_OK;
}

// FP64 GEMM of the precision form's projector step (CholeskyQR Grams and
// applies, the core products): FP64-accurate products on the tensor cores
// (exact digit splitting, ozaki.cu), bracketed as profiling class 2 with
// their algorithmic flops (structure-aware: a Hermitian Gram counts its upper
// triangle, a triangular factor its nonzero part; the digit products compute
// the full rectangle, so `flags` only states the structure).
static cudaError_t proj_zgemm(ipeps_ctm h, double flops, int M, int N, int K, const cplx* A, long long lda,
                              int opA, const cplx* B, long long ldb, int opB, cplx* C, long long ldc, int flags) {
  (void)flags;
  cudaEvent_t ev = nullptr;
  prof_begin(h, &ev);
  cudaError_t e = oz_zgemm(h->stream, M, N, K, A, lda, opA, B, ldb, opB, C, ldc, h->scratch + h->scratch_top,
                           (size_t)(h->scratch_elems - h->scratch_top) * sizeof(cplx), &h->st->tc_timeouts);
  prof_end(h, ev, flops, 2);
  return e;
}

// Precision form, one CholeskyQR pass on the k rows of `in` (length K):
// G = conj(in) in^T (FP64), G = R^H R (dropped pivots below tol * max), out =
// R^{-T} in (rows orthonormal on the kept directions, zero elsewhere).  R is
// left in Rout (k x k) when given.
static ipeps_status cholqr_pass(ipeps_ctm h, const cplx* in, cplx* out, cplx* Rout, double tol,
                                bool apply = true, bool shifted = false) {
  const int k = h->k, K = h->K;
  const long long mark = h->scratch_top;
  cplx* G = scratch_alloc(h, (long long)k * k);
  cplx* W = scratch_alloc(h, (long long)k * k);
  cplx* R = Rout ? Rout : scratch_alloc(h, (long long)k * k);
  cplx* Ri = scratch_alloc(h, (long long)k * k);
  if (!G || !W || !R || !Ri) return fail(IPEPS_ENOMEM, "scratch exhausted (cholqr)");
  // Hermitian Gram: the Cholesky reads its upper triangle only
  CK(proj_zgemm(h, 8.0 * K * (0.5 * k * (k + 1)), k, k, K, in, K, OP_C, in, K, OP_T, G, k, ZG_UPPER_TILES));
  // shifted CholeskyQR: s = 11 (m n + n (n + 1)) u ||Y||^2 with u = 2^-53
  if (shifted) CK(gram_shift(h->stream, G, k, 11.0 * ((double)K * k + (double)k * (k + 1)) * 0x1p-53));
  CK(chol_drop(h->stream, G, W, R, k, tol));
  if (apply) {
    CK(tri_inv(h->stream, R, Ri, k));
    // Q = Y R^{-1}  ->  Q^T = R^{-T} Y^T
    CK(proj_zgemm(h, 8.0 * K * (0.5 * k * (k + 1)), k, K, k, Ri, k, OP_T, in, K, OP_N, out, K, ZG_A_LOWER));
  }
  h->scratch_top = mark;
  return IPEPS_OK;
}

// Precision form orthonormalisation: CholeskyQR2 (directions below ~1e-7 of
// the largest singular value dropped in the first pass).
static ipeps_status orth_chol(ipeps_ctm h, cplx* Y, cplx* tmp, bool twice) {
  if (h->opt.prec == IPEPS_PREC_FP64TC) {
    // FP64-accurate form: no direction of the basis is dropped for being
    // small.  Shifted CholeskyQR (the shift keeps the Cholesky defined at any
    // condition number; the result spans the same space with condition below
    // about 1e5) and then one CholeskyQR pass (intermediate bases of the
    // subspace iteration) or two (the final basis: shifted CholeskyQR3), whose
    // pivots are dropped only where the shifted pass left rounding noise.
    CKS(cholqr_pass(h, Y, tmp, nullptr, 0.0, true, true));
    CKS(cholqr_pass(h, tmp, Y, nullptr, 1e-14));
    if (twice) {
      CKS(cholqr_pass(h, Y, tmp, nullptr, 1e-14));
      CK(cudaMemcpyAsync(Y, tmp, (size_t)h->k * h->K * sizeof(cplx), cudaMemcpyDeviceToDevice, h->stream));
    }
    return IPEPS_OK;
  }
  if (!twice) {
    // intermediate bases of the subspace iteration only need to stay well
    // conditioned: one pass (orthogonality ~ eps cond^2 below the dropped 1e-7)
    CKS(cholqr_pass(h, Y, tmp, nullptr, 1e-14));
    CK(cudaMemcpyAsync(Y, tmp, (size_t)h->k * h->K * sizeof(cplx), cudaMemcpyDeviceToDevice, h->stream));
    return IPEPS_OK;
  }
  CKS(cholqr_pass(h, Y, tmp, nullptr, 1e-14));
  CKS(cholqr_pass(h, tmp, Y, nullptr, 1e-14));
  return IPEPS_OK;
}

// Precision form SVD of W (K x k, stored as the k rows Wt): W = Q R by
// CholeskyQR2 (R = R2 R1, backward stable), one-sided Jacobi on the columns of
// the k x k R (R V = U_R S), then out rows = (W v_i)^T = s_i u_i^T, sigma = s,
// Vt rows = columns of V.
//
// Vt holds on entry the V this cut's SVD found at its previous visit (the
// identity at the first): the Jacobi starts from R V_prev and accumulates its
// rotations onto V_prev.  Between CTM iterations R changes little, so the
// rotated core is already nearly column-orthogonal and the sweeps converge
// quadratically from there; the SVD found is the same (the Jacobi stops on
// the same orthogonality test whatever its start).  The unitarity of the
// accumulated V degrades like sqrt(rotations) x 2^-48 (the rotations are
// replayed in double-float arithmetic), ~1e-12 after thousands of visits, far
// below the 1e-6 truncation of the precision forms.
static ipeps_status svd_rows_chol(ipeps_ctm h, const cplx* Wt, cplx* out, cplx* Vt) {
  const int k = h->k, K = h->K;
  const long long mark = h->scratch_top;
  cplx* R1 = scratch_alloc(h, (long long)k * k);
  cplx* R2 = scratch_alloc(h, (long long)k * k);
  cplx* Rt = scratch_alloc(h, (long long)k * k);
  if (!R1 || !R2 || !Rt) return fail(IPEPS_ENOMEM, "scratch exhausted (svd chol)");
  const bool fp64tc = h->opt.prec == IPEPS_PREC_FP64TC;
  cplx* Q3 = nullptr;
  if (fp64tc) {
    // shifted CholeskyQR3: W = Q3 R3 R2 R1 (no direction dropped for being small)
    cplx* R3 = scratch_alloc(h, (long long)k * k);
    cplx* Q2 = scratch_alloc(h, (long long)k * K);
    cplx* R21 = scratch_alloc(h, (long long)k * k);
    Q3 = scratch_alloc(h, (long long)k * K);
    if (!R3 || !Q2 || !R21 || !Q3) return fail(IPEPS_ENOMEM, "scratch exhausted (svd chol)");
    CKS(cholqr_pass(h, Wt, out, R1, 0.0, true, true));
    CKS(cholqr_pass(h, out, Q2, R2, 1e-14));
    CKS(cholqr_pass(h, Q2, Q3, R3, 1e-14));
    // Rt = (R3 R2 R1)^T = (R2 R1)^T R3^T
    CK(proj_zgemm(h, 8.0 * k * (k + 1.0) * (k + 2.0) / 6.0, k, k, k, R1, k, OP_T, R2, k, OP_T, R21, k, ZG_A_LOWER));
    CK(proj_zgemm(h, 8.0 * k * (k + 1.0) * (k + 2.0) / 6.0, k, k, k, R21, k, OP_N, R3, k, OP_T, Rt, k, ZG_A_LOWER));
  } else {
    CKS(cholqr_pass(h, Wt, out, R1, 1e-14));
    CKS(cholqr_pass(h, out, nullptr, R2, 1e-14, false));  // only R2 is needed
    // Rt = (R2 R1)^T: rows of Rt are the columns of R
    CK(proj_zgemm(h, 8.0 * k * (k + 1.0) * (k + 2.0) / 6.0, k, k, k, R1, k, OP_T, R2, k, OP_T, Rt, k, ZG_A_LOWER));
  }
  // R1 = V_prev^T Rt: rows are the columns of R V_prev
  CK(proj_zgemm(h, 8.0 * k * (double)k * k, k, k, k, Vt, k, OP_N, Rt, k, OP_N, R1, k, 0));
  {
    cudaEvent_t a = nullptr;
    prof_begin(h, &a);
    const long long nlog = jacobi_log_elems(k, h->opt.jacobi_max_sweeps);
    cplx* rotlog = scratch_alloc(h, nlog);
    if (!rotlog) return fail(IPEPS_ENOMEM, "scratch exhausted (rotation log)");
    CK(jacobi_rows(h->stream, R1, k, k, k, Vt, h->sigma, h->opt.jacobi_max_sweeps, h->dwork, h->counters,
                   h->st, rotlog, nlog, h->opt.wait_cycles, true, !fp64tc));
    prof_end(h, a, 0.0, 1);
  }
  if (fp64tc) {
    // out = R1 Q3^T: rows (Q3 R v_i)^T = s_i (Q3 u_R,i)^T.  The left singular
    // vectors of W as the orthonormal basis Q3 times those of the core, rather
    // than W v_i / s_i, whose division by a small s_i magnifies the rounding
    // of W v_i (FP64-level agreement with the exact SVD needs the former).
    CK(proj_zgemm(h, 8.0 * k * (double)K * k, k, K, k, R1, k, OP_N, Q3, K, OP_N, out, K, 0));
  } else {
    // out = V^T Wt  (rows (W v_i)^T)
    CK(proj_zgemm(h, 8.0 * k * (double)K * k, k, K, k, Vt, k, OP_N, Wt, K, OP_N, out, K, 0));
  }
  CK(row_norms(h->stream, out, k, K, K, h->sigma));
  h->scratch_top = mark;
  return IPEPS_OK;
}

// Projectors of the left cut of plaquette (x,y): PT = P^T, Ptil (both chi x K).
static ipeps_status projectors(ipeps_ctm h, int f, int x, int y, cplx* PT, cplx* Ptil) {
  CKS(enlarged_corners(h, f, x, y));
  const int k = h->k, K = h->K, chi = h->chi;
  // the FP64 path orthonormalises by Jacobi; the other forms by CholeskyQR on
  // FP64-accurate Grams (FP64TC: its products unpacked, on the digit planes)
  const bool fp64 = h->opt.prec == IPEPS_PREC_FP64;
  if (packed_path(h)) CKS(pack_corners(h));
  cplx* Qt = h->thin[0];
  cplx* Zt = h->thin[1];
  auto orth_any = [&](cplx* Y, bool last) -> ipeps_status {
    return fp64 ? orth(h, Y) : orth_chol(h, Y, h->thin[2], last);
  };
  const int q = h->opt.rsvd_power;
  CKS(apply_XT(h, h->omt, Qt, k));
  CKS(orth_any(Qt, q == 0));
  for (int it = 0; it < q; ++it) {
    CKS(apply_XHT(h, Qt, Zt, k));
    CKS(orth_any(Zt, false));
    CKS(apply_XT(h, Zt, Qt, k));
    CKS(orth_any(Qt, it == q - 1));
  }
  // W = X^H Q (K x k) stored as Wt; its SVD W = U_w S V_w^H gives X ~ (Q V_w) S U_w^H
  CKS(apply_XHT(h, Qt, Zt, k));
  cplx* Wrot;  // rows sigma_i u_i^T
  cplx* Vt = h->Vt;  // rows = columns of V
  if (fp64) {
    cudaEvent_t a = nullptr;
    prof_begin(h, &a);
    CK(jacobi_rows(h->stream, Zt, k, K, K, h->Vt, h->sigma, h->opt.jacobi_max_sweeps, h->dwork,
                   h->counters, h->st, nullptr, 0, h->opt.wait_cycles));
    prof_end(h, a, 0.0, 1);
    Wrot = Zt;
  } else {
    int lx, ly;
    frame_dims(h, f, &lx, &ly);
    Vt = h->Vwarm[f][y * lx + x];
    CKS(svd_rows_chol(h, Zt, h->thin[2], Vt));
    Wrot = h->thin[2];
  }
  cplx* Vt_chi = (Wrot == Zt) ? h->thin[2] : Zt;
  cplx* Ut_chi = h->thin[3];
  cplx* tmp = (Wrot == Zt) ? Zt : h->thin[2];  // free once Vt_chi has been gathered
  CK(select_top(h->stream, h->sigma, k, chi, h->opt.svd_cutoff, h->perm, h->s_sel));
  // V_chi^T rows = selected columns of U_w (normalised rows of Wrot)
  CK(gather_rows(h->stream, Wrot, K, Vt_chi, K, h->perm, h->sigma, chi, K, true));
  // U_chi^T = (V_w[:, sel])^T Q^T
  CK(gather_rows(h->stream, Vt, k, h->Gsel, k, h->perm, h->sigma, chi, k, false));
  CKS(gemm_dispatch(h, chi, K, k, h->Gsel, k, OP_N, Qt, K, OP_N, Ut_chi, K, ONE));
  // P^T = S^-1/2 V^T Q3 Q4^T ;  Ptil = S^-1/2 U^H Q2^T Q1^T
  // (two corners: P^T = S^-1/2 V^T Q4^T ;  Ptil = S^-1/2 U^H Q1^T)
  if (two_corners(h)) {
    if (packed_path(h))
      CKS(thin_mul_packed(h, Vt_chi, OP_N, PT, 3, 1, chi, false));
    else
      CKS(thin_mul(h, Vt_chi, OP_N, PT, h->Q[3], OP_T, chi));
  } else if (packed_path(h)) {
    CKS(thin_mul_packed(h, Vt_chi, OP_N, tmp, 2, 0, chi, false));
    CKS(thin_mul_packed(h, tmp, OP_N, PT, 3, 1, chi, false));
  } else {
    CKS(thin_mul(h, Vt_chi, OP_N, tmp, h->Q[2], OP_N, chi));
    CKS(thin_mul(h, tmp, OP_N, PT, h->Q[3], OP_T, chi));
  }
  CK(scale_rows_isqrt(h->stream, PT, chi, K, K, h->s_sel));
  if (two_corners(h)) {
    if (packed_path(h))
      CKS(thin_mul_packed(h, Ut_chi, OP_C, Ptil, 0, 1, chi, false));
    else
      CKS(thin_mul(h, Ut_chi, OP_C, Ptil, h->Q[0], OP_T, chi));
  } else if (packed_path(h)) {
    CKS(thin_mul_packed(h, Ut_chi, OP_C, tmp, 1, 1, chi, false));
    CKS(thin_mul_packed(h, tmp, OP_N, Ptil, 0, 1, chi, false));
  } else {
    CKS(thin_mul(h, Ut_chi, OP_C, tmp, h->Q[1], OP_T, chi));
    CKS(thin_mul(h, tmp, OP_N, Ptil, h->Q[0], OP_T, chi));
  }
  CK(scale_rows_isqrt(h->stream, Ptil, chi, K, K, h->s_sel));
  return IPEPS_OK;
}

static ipeps_status left_move(ipeps_ctm h, int f) {
  int Lx, Ly;
  frame_dims(h, f, &Lx, &Ly);
  const int c = h->chi, D2 = h->D2;
  for (int x = 0; x < Lx; ++x) {
    if (Ly == 2 && h->has_alt && !h->no_alt) {
      // fork: cut y = 0 on the handle's stream, cut y = 1 on the second lane
      const long long full = h->scratch_elems, half = (full / 2) & ~1023LL;
      CK(cudaEventRecord(h->ev_fork, h->stream));
      CK(cudaStreamWaitEvent(h->alt.stream, h->ev_fork, 0));
      h->scratch_elems = half;
      h->alt.scratch = h->scratch + half;
      h->alt.scratch_elems = full - half;
      h->alt.scratch_top = 0;
      ipeps_status s0 = projectors(h, f, x, 0, h->PT[0], h->Ptil[0]);
      ipeps_status s1 = IPEPS_OK;
      if (s0 == IPEPS_OK) {
        swap_lane(h);
        s1 = projectors(h, f, x, 1, h->PT[1], h->Ptil[1]);
        swap_lane(h);
      }
      h->scratch_elems = full;
      CK(cudaEventRecord(h->ev_join, h->alt.stream));
      CK(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
      CKS(s0);
      CKS(s1);
    } else {
      for (int y = 0; y < Ly; ++y) CKS(projectors(h, f, x, y, h->PT[y], h->Ptil[y]));
    }
    for (int y = 0; y < Ly; ++y) {
      const int ym = (y - 1 + Ly) % Ly;
      cplx* w1 = scratch_alloc(h, (long long)c * D2 * c);
      cplx* w2 = scratch_alloc(h, (long long)c * D2 * c * D2);
      if (!w1 || !w2) return fail(IPEPS_ENOMEM, "scratch exhausted (absorb)");
      // C1'[n,r] = sum P[(a,s),n] (C1 T1)[a,s,r]
      CKS(contract(h, "ab,bsr->asr", tv(envC(h, f, 0, x, y), {c, c}), false,
                   tv(envT(h, f, 0, x, y), {c, D2, c}), false, tv(w1, {c, D2, c})));
      CKS(contract(h, "nas,asr->nr", tv(h->PT[ym], {c, c, D2}), false, tv(w1, {c, D2, c}), false,
                   tv(h->spareC[0][y], {c, c})));
      // T4'[b,r,a] = sum P[(e,h),b] T4[e,m,f] a[g,m,h,r] Ptil[a,(f,g)]
      CKS(contract(h, "emf,beh->mfhb", tv(envT(h, f, 3, x, y), {c, D2, c}), false,
                   tv(h->PT[y], {c, c, D2}), false, tv(w2, {D2, c, D2, c})));
      cplx* w3 = scratch_alloc(h, (long long)c * D2 * c * D2);
      if (!w3) return fail(IPEPS_ENOMEM, "scratch exhausted (absorb)");
      CKS(contract(h, "mfhb,gmhr->fbgr", tv(w2, {D2, c, D2, c}), false,
                   tv(site_a(h, f, x, y), {D2, D2, D2, D2}), false, tv(w3, {c, c, D2, D2})));
      CKS(contract(h, "fbgr,afg->bra", tv(w3, {c, c, D2, D2}), false, tv(h->Ptil[ym], {c, c, D2}),
                   false, tv(h->spareT[y], {c, D2, c})));
      // C4'[r,a] = sum (C4 T3)[r,s,u] Ptil[a,(u,s)]
      CKS(contract(h, "gu,rsg->rsu", tv(envC(h, f, 3, x, y), {c, c}), false,
                   tv(envT(h, f, 2, x, y), {c, D2, c}), false, tv(w1, {c, D2, c})));
      CKS(contract(h, "rsu,aus->ra", tv(w1, {c, D2, c}), false, tv(h->Ptil[y], {c, c, D2}), false,
                   tv(h->spareC[1][y], {c, c})));
      h->scratch_top = 0;
      CK(normalize(h->stream, h->spareC[0][y], (long long)c * c, h->dwork, h->st));
      CK(normalize(h->stream, h->spareT[y], (long long)c * D2 * c, h->dwork, h->st));
      CK(normalize(h->stream, h->spareC[1][y], (long long)c * c, h->dwork, h->st));
    }
    // install the renormalised tensors at column x+1.  Device copies keep the
    // buffer of every environment tensor fixed, so a captured CUDA graph of a
    // move stays valid for every replay.
    const size_t cb = (size_t)c * c * sizeof(cplx), tb = (size_t)c * D2 * c * sizeof(cplx);
    for (int y = 0; y < Ly; ++y) {
      CK(cudaMemcpyAsync(envC(h, f, 0, x + 1, y), h->spareC[0][y], cb, cudaMemcpyDeviceToDevice, h->stream));
      CK(cudaMemcpyAsync(envT(h, f, 3, x + 1, y), h->spareT[y], tb, cudaMemcpyDeviceToDevice, h->stream));
      CK(cudaMemcpyAsync(envC(h, f, 3, x + 1, y), h->spareC[1][y], cb, cudaMemcpyDeviceToDevice, h->stream));
    }
  }
  return IPEPS_OK;
}

// Enqueue one move (or one sweep) on the handle's stream without waiting for
// the device or reading its status: the work a batch captures in a graph.
ipeps_status ctm_enqueue_move(ipeps_ctm h, int dir) {
  static const int sweep[4] = {IPEPS_MOVE_LEFT, IPEPS_MOVE_RIGHT, IPEPS_MOVE_UP, IPEPS_MOVE_DOWN};
  static const char* names[4] = {"ctm move L", "ctm move U", "ctm move R", "ctm move D"};
  if (dir == IPEPS_SWEEP) {
    for (int i = 0; i < 4; ++i) {
      NvtxRange r(names[sweep[i]]);
      CKS(left_move(h, sweep[i]));
    }
    return IPEPS_OK;
  }
  NvtxRange r(names[dir]);
  return left_move(h, dir);
}

// Capture the move (or sweep) `dir` as a CUDA graph: the work is enqueued on
// the private capture stream (the second projector lane joins the capture
// through the fork/join events), so the graph can be launched on any stream,
// the legacy default stream included.  Every buffer a move touches keeps its
// address for the life of the handle, so the graph stays valid until the
// tile choices change (autotuning), which drops it.
static ipeps_status capture_move(ipeps_ctm h, int dir) {
  CK(kernels_init());
  CK(fp64_cluster_init());
  if (h->opt.prec != IPEPS_PREC_FP64) CK(tc_init());
  cudaStream_t user = h->stream;
  const uint64_t l0 = launch_counter();
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeRelaxed));
  h->stream = h->cap_stream;
  ipeps_status st = ctm_enqueue_move(h, dir);
  h->stream = user;
  const cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
  h->scratch_top = 0;
  h->alt.scratch_top = 0;
  h->exec_kernels[dir] = (int)(launch_counter() - l0);
  count_launch(-h->exec_kernels[dir]);  // counted at each launch instead
  if (st != IPEPS_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    if (st != IPEPS_OK) return st;
    return fail(IPEPS_ECUDA, "move capture: %s", cudaGetErrorString(e));
  }
  const cudaError_t e2 = cudaGraphInstantiate(&h->exec[dir], g, 0);
  cudaGraphDestroy(g);
  if (e2 != cudaSuccess) {
    h->exec[dir] = nullptr;
    return fail(IPEPS_ECUDA, "move graph: %s", cudaGetErrorString(e2));
  }
  return IPEPS_OK;
}

extern "C" ipeps_status ipeps_ctm_move(ipeps_ctm h, int dir, int count) {
  if (!h) return fail(IPEPS_EINVAL, "null handle");
  if (dir < 0 || dir > 4 || count < 0) return fail(IPEPS_EINVAL, "bad dir/count");
  CKS(reset_status(h));
  // graphs unless per-kernel timing is on (its events are per launch)
  if (count > 0 && h->cap_stream && !h->profiling) {
    if (!h->exec[dir]) CKS(capture_move(h, dir));
    for (int n = 0; n < count; ++n) {
      CK(cudaGraphLaunch(h->exec[dir], h->stream));
      count_launch(h->exec_kernels[dir]);
    }
    return check_status(h);
  }
  for (int n = 0; n < count; ++n) CKS(ctm_enqueue_move(h, dir));
  return check_status(h);
}

static ipeps_status all_rdms(ipeps_ctm h, cplx* rh, cplx* rv);
static ipeps_status rdm_buffers(ipeps_ctm h, cplx** rh, cplx** rv);

extern "C" ipeps_status ipeps_ctm_autotune(ipeps_ctm h) {
  if (!h) return fail(IPEPS_EINVAL, "null handle");
  if (!tc_form(h->opt.prec)) return IPEPS_OK;  // no tiled tensor-core products to tune
  CK(kernels_init());
  CK(tc_init());
  if (!h->tuner) {
    h->tuner = tc_tuner_create();
    if (!h->tuner) return fail(IPEPS_ECUDA, "tuner events");
    h->own_tuner = true;
  }
  drop_graphs(h);  // captured with the previous tile choices
  // snapshot of the environment and of the cuts' Jacobi starts, restored
  // after the tuning sweep (later results do not depend on the tuning)
  const int ncell = h->Lx * h->Ly;
  const size_t cb = (size_t)h->chi * h->chi * sizeof(cplx), tb = (size_t)h->chi * h->D2 * h->chi * sizeof(cplx);
  const size_t vb = (size_t)h->k * h->k * sizeof(cplx), env_bytes = 4 * ncell * (cb + tb);
  char* snap = nullptr;
  CK(dev_alloc((void**)&snap, env_bytes + 4 * ncell * vb));
  for (int j = 0; j < 4; ++j)
    for (int i = 0; i < ncell; ++i) {
      CK(cudaMemcpyAsync(snap + (j * ncell + i) * (cb + tb), h->C[j][i], cb, cudaMemcpyDeviceToDevice, h->stream));
      CK(cudaMemcpyAsync(snap + (j * ncell + i) * (cb + tb) + cb, h->T[j][i], tb, cudaMemcpyDeviceToDevice,
                         h->stream));
      CK(cudaMemcpyAsync(snap + env_bytes + (j * ncell + i) * vb, h->Vwarm[j][i], vb, cudaMemcpyDeviceToDevice,
                         h->stream));
    }
  tc_tuner_set_measuring(h->tuner, true);
  h->no_alt = true;  // cuts in sequence: timings unperturbed by the other lane
  ipeps_status st = reset_status(h);
  if (st == IPEPS_OK) st = ctm_enqueue_move(h, IPEPS_SWEEP);
  if (st == IPEPS_OK) {
    // the bond readout's products too (the environment is left as it is)
    cplx *rh, *rv;
    st = rdm_buffers(h, &rh, &rv);
    const long long n2 = (long long)h->d * h->d * h->d * h->d * h->Lx * h->Ly;
    const long long save = h->scratch_elems;
    h->scratch_elems -= 2 * n2;
    if (st == IPEPS_OK) st = all_rdms(h, rh, rv);
    h->scratch_elems = save;
  }
  if (st == IPEPS_OK) st = check_status(h);
  h->no_alt = false;
  tc_tuner_set_measuring(h->tuner, false);
  for (int j = 0; j < 4; ++j)
    for (int i = 0; i < ncell; ++i) {
      cudaMemcpyAsync(h->C[j][i], snap + (j * ncell + i) * (cb + tb), cb, cudaMemcpyDeviceToDevice, h->stream);
      cudaMemcpyAsync(h->T[j][i], snap + (j * ncell + i) * (cb + tb) + cb, tb, cudaMemcpyDeviceToDevice, h->stream);
      cudaMemcpyAsync(h->Vwarm[j][i], snap + env_bytes + (j * ncell + i) * vb, vb, cudaMemcpyDeviceToDevice,
                      h->stream);
    }
  cudaError_t e = cudaStreamSynchronize(h->stream);
  cudaFree(snap);
  CKS(st);
  CK(e);
  return IPEPS_OK;
}

extern "C" int ipeps_ctm_tuning_size(ipeps_ctm h) { return h ? tc_tuner_size(h->tuner) : 0; }

// handle internals used by the batch module (batch.cu)
cudaStream_t ctm_stream(ipeps_ctm h) { return h->stream; }
ipeps_status ctm_reset_status(ipeps_ctm h) { return reset_status(h); }
ipeps_status ctm_check_status(ipeps_ctm h) { return check_status(h); }
ipeps_status ctm_reinit_env(ipeps_ctm h) { return trace_init_env(h); }
void ctm_set_tuner(ipeps_ctm h, TcTuner* t) {
  drop_graphs(h);
  h->tuner = t;
}
void ctm_set_sequential_cuts(ipeps_ctm h, bool on) {
  if (h->no_alt != on) drop_graphs(h);
  h->no_alt = on;
}

// ---------------------------------------------------------------------------
// spectra / convergence
// ---------------------------------------------------------------------------
static ipeps_status spectra_device(ipeps_ctm h, double* host) {
  const int c = h->chi;
  cplx* w = scratch_alloc(h, (long long)c * c);
  if (!w) return fail(IPEPS_ENOMEM, "scratch exhausted (spectra)");
  const int ncell = h->Lx * h->Ly;
  for (int j = 0; j < 4; ++j)
    for (int i = 0; i < ncell; ++i) {
      CK(cudaMemcpyAsync(w, h->C[j][i], (size_t)c * c * sizeof(cplx), cudaMemcpyDeviceToDevice, h->stream));
      CK(jacobi_rows(h->stream, w, c, c, c, nullptr, h->sigma, h->opt.jacobi_max_sweeps, h->dwork,
                     h->counters, h->st, nullptr, 0, h->opt.wait_cycles));
      CK(select_top(h->stream, h->sigma, c, c, 0.0, h->perm, h->s_sel));
      CK(cudaMemcpyAsync(host + (size_t)(j * ncell + i) * c, h->s_sel, c * sizeof(double),
                         cudaMemcpyDeviceToHost, h->stream));
    }
  h->scratch_top = 0;
  CK(cudaStreamSynchronize(h->stream));
  for (int q = 0; q < 4 * ncell; ++q) {
    double* s = host + (size_t)q * c;
    const double s0 = s[0];
    if (s0 > 0)
      for (int a = 0; a < c; ++a) s[a] /= s0;
  }
  return IPEPS_OK;
}

extern "C" ipeps_status ipeps_ctm_spectra(ipeps_ctm h, double* s_out) {
  if (!h || !s_out) return fail(IPEPS_EINVAL, "null argument");
  NvtxRange range("corner spectra");
  CKS(reset_status(h));
  CKS(spectra_device(h, s_out));
  return check_status(h);
}

extern "C" ipeps_status ipeps_ctm_converge(ipeps_ctm h, double tol, int max_sweeps, int* sweeps,
                                           double* delta) {
  if (!h) return fail(IPEPS_EINVAL, "null handle");
  const size_t n = (size_t)4 * h->Lx * h->Ly * h->chi;
  std::vector<double> s_old(n), s_new(n);
  CKS(ipeps_ctm_spectra(h, s_old.data()));
  double dl = INFINITY;
  int it = 0;
  while (it < max_sweeps) {
    CKS(ipeps_ctm_move(h, IPEPS_SWEEP, 1));
    ++it;
    CKS(ipeps_ctm_spectra(h, s_new.data()));
    dl = 0.0;
    for (size_t q = 0; q < n / h->chi; ++q) {
      double acc = 0.0;
      for (int a = 0; a < h->chi; ++a) {
        const double t = s_new[q * h->chi + a] - s_old[q * h->chi + a];
        acc += t * t;
      }
      dl = std::max(dl, sqrt(acc));
    }
    s_old.swap(s_new);
    if (dl < tol) break;
  }
  if (sweeps) *sweeps = it;
  if (delta) *delta = dl;
  if (!(dl < tol)) return fail(IPEPS_ENOCONV, "not converged after %d sweeps (delta %.3e)", it, dl);
  return IPEPS_OK;
}

// ---------------------------------------------------------------------------
// RDMs and energy (frame f horizontal bond (x,y)-(x+1,y))
// ---------------------------------------------------------------------------
// Left half of the window of site (x,y) in frame f, its physical legs open:
// C1 T1 / T4 [A, A*] / C4 T3 contracted into left[h, r, s, k, p, q] with h
// T1's right leg, (r, s) the site's right double leg (ket, bra), k T3's right
// leg and (p, q) the physical (ket, bra) pair.  L2, L3, L4, small are work.
static ipeps_status rdm_left_half(ipeps_ctm h, int f, int x, int y, cplx* L2, cplx* L3, cplx* L4, cplx* small,
                                  cplx* left) {
  const int c = h->chi, D = h->D, d = h->d;
  const cplx* Aa = h->A[f][tensor_id(h, f, x, y)];
  CKS(contract(h, "ab,bUVh->aUVh", tv(envC(h, f, 0, x, y), {c, c}), false,
               tv(envT(h, f, 0, x, y), {c, D, D, c}), false, tv(small, {c, D, D, c})));
  CKS(contract(h, "eLMa,aUVh->eLMUVh", tv(envT(h, f, 3, x, y), {c, D, D, c}), false,
               tv(small, {c, D, D, c}), false, tv(L2, {c, D, D, D, D, c})));
  CKS(contract(h, "eLMUVh,pULSr->eMVhpSr", tv(L2, {c, D, D, D, D, c}), false,
               tv((cplx*)Aa, {d, D, D, D, D}), false, tv(L3, {c, D, D, c, d, D, D})));
  CKS(contract(h, "ge,kSTg->ekST", tv(envC(h, f, 3, x, y), {c, c}), false,
               tv(envT(h, f, 2, x, y), {c, D, D, c}), false, tv(small, {c, c, D, D})));
  CKS(contract(h, "eMVhpSr,ekST->MVhprkT", tv(L3, {c, D, D, c, d, D, D}), false,
               tv(small, {c, c, D, D}), false, tv(L4, {D, D, c, d, D, c, D})));
  CKS(contract(h, "MVhprkT,qVMTs->hrskpq", tv(L4, {D, D, c, d, D, c, D}), false,
               tv((cplx*)Aa, {d, D, D, D, D}), true, tv(left, {c, D, D, c, d, d})));
  return IPEPS_OK;
}

static ipeps_status rdm_horizontal(ipeps_ctm h, int f, int x, int y, cplx* rho) {
  const int c = h->chi, D = h->D, d = h->d;
  const cplx* Ab = h->A[f][tensor_id(h, f, x + 1, y)];
  const long long big = (long long)c * c * D * D * D * D * d;
  cplx* L2 = scratch_alloc(h, (long long)c * c * D * D * D * D);
  cplx* L3 = scratch_alloc(h, big);
  cplx* L4 = scratch_alloc(h, big);
  cplx* left = scratch_alloc(h, (long long)c * c * D * D * d * d);
  cplx* right = scratch_alloc(h, (long long)c * c * D * D * d * d);
  cplx* small = scratch_alloc(h, (long long)c * c * D * D);
  if (!L2 || !L3 || !L4 || !left || !right || !small) return fail(IPEPS_ENOMEM, "scratch exhausted (rdm)");
  CKS(rdm_left_half(h, f, x, y, L2, L3, L4, small, left));
  // right half
  CKS(contract(h, "hUVc,cf->hUVf", tv(envT(h, f, 0, x + 1, y), {c, D, D, c}), false,
               tv(envC(h, f, 1, x + 1, y), {c, c}), false, tv(small, {c, D, D, c})));
  CKS(contract(h, "hUVf,fRSg->hUVRSg", tv(small, {c, D, D, c}), false,
               tv(envT(h, f, 1, x + 1, y), {c, D, D, c}), false, tv(L2, {c, D, D, D, D, c})));
  CKS(contract(h, "hUVRSg,pUlXR->hVSgplX", tv(L2, {c, D, D, D, D, c}), false,
               tv((cplx*)Ab, {d, D, D, D, D}), false, tv(L3, {c, D, D, c, d, D, D})));
  CKS(contract(h, "gi,iXYk->gXYk", tv(envC(h, f, 2, x + 1, y), {c, c}), false,
               tv(envT(h, f, 2, x + 1, y), {c, D, D, c}), false, tv(small, {c, D, D, c})));
  CKS(contract(h, "hVSgplX,gXYk->hVSplYk", tv(L3, {c, D, D, c, d, D, D}), false,
               tv(small, {c, D, D, c}), false, tv(L4, {c, D, D, d, D, D, c})));
  CKS(contract(h, "hVSplYk,qVmYS->hlmkpq", tv(L4, {c, D, D, d, D, D, c}), false,
               tv((cplx*)Ab, {d, D, D, D, D}), true, tv(right, {c, D, D, c, d, d})));
  CKS(contract(h, "hrskpq,hrskPQ->pPqQ", tv(left, {c, D, D, c, d, d}), false,
               tv(right, {c, D, D, c, d, d}), false, tv(rho, {d, d, d, d})));
  CK(trace_normalize(h->stream, rho, d * d, h->dwork));
  h->scratch_top = 0;
  return IPEPS_OK;
}

// One-site RDM at (x,y) (frame 0): the left half closed by the site's own
// right column C2 T2 C3 (col[h, r, s, k]).
static ipeps_status rdm_site(ipeps_ctm h, int x, int y, cplx* rho) {
  const int c = h->chi, D = h->D, d = h->d;
  const long long big = (long long)c * c * D * D * D * D * d;
  cplx* L2 = scratch_alloc(h, (long long)c * c * D * D * D * D);
  cplx* L3 = scratch_alloc(h, big);
  cplx* L4 = scratch_alloc(h, big);
  cplx* left = scratch_alloc(h, (long long)c * c * D * D * d * d);
  cplx* small = scratch_alloc(h, (long long)c * c * D * D);
  cplx* col = scratch_alloc(h, (long long)c * c * D * D);
  if (!L2 || !L3 || !L4 || !left || !small || !col) return fail(IPEPS_ENOMEM, "scratch exhausted (site rdm)");
  CKS(rdm_left_half(h, 0, x, y, L2, L3, L4, small, left));
  CKS(contract(h, "hf,fRSg->hRSg", tv(envC(h, 0, 1, x, y), {c, c}), false,
               tv(envT(h, 0, 1, x, y), {c, D, D, c}), false, tv(small, {c, D, D, c})));
  CKS(contract(h, "hRSg,gk->hRSk", tv(small, {c, D, D, c}), false, tv(envC(h, 0, 2, x, y), {c, c}), false,
               tv(col, {c, D, D, c})));
  CKS(contract(h, "hrskpq,hrsk->pq", tv(left, {c, D, D, c, d, d}), false, tv(col, {c, D, D, c}), false,
               tv(rho, {d, d})));
  CK(trace_normalize(h->stream, rho, d, h->dwork));
  h->scratch_top = 0;
  return IPEPS_OK;
}

extern "C" ipeps_status ipeps_rdm_site(ipeps_ctm h, double* rho_s) {
  if (!h || !rho_s) return fail(IPEPS_EINVAL, "null argument");
  NvtxRange range("rdm sites");
  CKS(reset_status(h));
  const long long n1 = (long long)h->d * h->d;
  const long long n = n1 * h->Lx * h->Ly;
  // results at the top of the scratch arena, below them the per-site work
  cplx* rs = h->scratch + h->scratch_elems - n;
  const long long save = h->scratch_elems;
  h->scratch_elems -= n;
  ipeps_status st = IPEPS_OK;
  for (int y = 0; y < h->Ly && st == IPEPS_OK; ++y)
    for (int x = 0; x < h->Lx && st == IPEPS_OK; ++x) st = rdm_site(h, x, y, rs + (y * h->Lx + x) * n1);
  h->scratch_elems = save;
  CKS(st);
  CK(cudaMemcpyAsync(rho_s, rs, n * sizeof(cplx), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return check_status(h);
}

// all bond RDMs into device buffers rh, rv ([Ly][Lx][d^2][d^2] each)
static ipeps_status all_rdms(ipeps_ctm h, cplx* rh, cplx* rv) {
  const long long n2 = (long long)h->d * h->d * h->d * h->d;
  // both kinds of bond: horizontal bonds on the handle's stream, vertical ones
  // on the second lane, each lane with half of the scratch arena, when half
  // holds one bond's intermediates (the halves' six-leg tensors, the
  // contraction temporaries and the packed tensor-core operands)
  const long long c = h->chi, D = h->D, d = h->d;
  const long long big = c * c * D * D * D * D * d;
  const long long need = c * c * D * D * D * D + 4 * big + 2 * c * c * D * D * d * d + c * c * D * D + (1LL << 22);
  const long long full = h->scratch_elems, half = (full / 2) & ~1023LL;
  if (rh && rv && h->has_alt && !h->no_alt && tc_form(h->opt.prec) && half >= need) {
    CK(cudaEventRecord(h->ev_fork, h->stream));
    CK(cudaStreamWaitEvent(h->alt.stream, h->ev_fork, 0));
    h->scratch_elems = half;
    h->alt.scratch = h->scratch + half;
    h->alt.scratch_elems = full - half;
    h->alt.scratch_top = 0;
    ipeps_status s0 = IPEPS_OK, s1 = IPEPS_OK;
    for (int y = 0; y < h->Ly && s0 == IPEPS_OK; ++y)
      for (int x = 0; x < h->Lx && s0 == IPEPS_OK; ++x)
        s0 = rdm_horizontal(h, 0, x, y, rh + (long long)(y * h->Lx + x) * n2);
    if (s0 == IPEPS_OK) {
      swap_lane(h);
      for (int y = 0; y < h->Ly && s1 == IPEPS_OK; ++y)
        for (int x = 0; x < h->Lx && s1 == IPEPS_OK; ++x)
          s1 = rdm_horizontal(h, 1, y, -x, rv + (long long)(y * h->Lx + x) * n2);  // (x,y)-(x,y+1) in frame 1
      swap_lane(h);
    }
    h->scratch_elems = full;
    CK(cudaEventRecord(h->ev_join, h->alt.stream));
    CK(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
    CKS(s0);
    CKS(s1);
    return IPEPS_OK;
  }
  for (int y = 0; y < h->Ly; ++y)
    for (int x = 0; x < h->Lx; ++x) {
      const long long o = (long long)(y * h->Lx + x) * n2;
      if (rh) CKS(rdm_horizontal(h, 0, x, y, rh + o));
      // vertical bond (x,y)-(x,y+1) is horizontal in frame 1 at (y, -x)
      if (rv) CKS(rdm_horizontal(h, 1, y, -x, rv + o));
    }
  return IPEPS_OK;
}

static ipeps_status rdm_buffers(ipeps_ctm h, cplx** rh, cplx** rv) {
  const long long n2 = (long long)h->d * h->d * h->d * h->d * h->Lx * h->Ly;
  // keep the RDMs at the top of the scratch arena, below the per-bond work
  *rh = h->scratch + h->scratch_elems - 2 * n2;
  *rv = *rh + n2;
  return IPEPS_OK;
}

extern "C" ipeps_status ipeps_rdm(ipeps_ctm h, double* rho_h, double* rho_v) {
  if (!h) return fail(IPEPS_EINVAL, "null handle");
  NvtxRange range("rdm bonds");
  CKS(reset_status(h));
  cplx *rh, *rv;
  CKS(rdm_buffers(h, &rh, &rv));
  const long long n2 = (long long)h->d * h->d * h->d * h->d * h->Lx * h->Ly;
  const long long save = h->scratch_elems;
  h->scratch_elems -= 2 * n2;
  ipeps_status st = all_rdms(h, rho_h ? rh : nullptr, rho_v ? rv : nullptr);
  h->scratch_elems = save;
  CKS(st);
  if (rho_h) CK(cudaMemcpyAsync(rho_h, rh, n2 * sizeof(cplx), cudaMemcpyDeviceToHost, h->stream));
  if (rho_v) CK(cudaMemcpyAsync(rho_v, rv, n2 * sizeof(cplx), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return check_status(h);
}

// Star lattice (App. B) with Heisenberg couplings, one reading of its block
// structure (the figure is not in the text): the three spins of a triangle
// block site link to the left (spin 1), right (spin 2) and vertical (spin 3)
// neighbours of the brick wall, A sites (x + y even) downwards, B sites
// upwards, so the vertical bond with B on top is the trivial (D = 1) edge.
// h_t = J_t (s1.s2 + s1.s3 + s2.s3) inside each triangle (half on each
// horizontal bond), J_e s.s on the links between triangles; s = Pauli matrices.
static CM dot_pair(int a, int b) {  // s_a (left/upper site) . s_b (right/lower site)
  CM m(64);
  for (char al : {'x', 'y', 'z'}) axpy(m, 1.0, kron(spin_op(al, a), spin_op(al, b)));
  return m;
}
static void star_bonds(const double J[2], CM* Hh, CM* Hv) {
  CM I8(8);
  for (int i = 0; i < 8; ++i) I8.re[i * 8 + i] = 1.0;
  CM ht(8);
  const int pairs[3][2] = {{1, 2}, {1, 3}, {2, 3}};
  for (const auto& pr : pairs)
    for (char al : {'x', 'y', 'z'}) axpy(ht, J[0], matmul(spin_op(al, pr[0]), spin_op(al, pr[1])));
  *Hh = CM(64);
  axpy(*Hh, 0.5, kron(ht, I8));
  axpy(*Hh, 0.5, kron(I8, ht));
  axpy(*Hh, J[1], dot_pair(2, 1));
  *Hv = CM(64);
  axpy(*Hv, J[1], dot_pair(3, 3));
}

// bond operators H_r, H_l, H_u, H_d (64 x 64 complex, NULL = 0) to the device
static ipeps_status upload_ops(ipeps_ctm h, const CM* const mats[4]) {
  std::vector<double> buf(2 * 64 * 64);
  for (int m = 0; m < 4; ++m) {
    for (int i = 0; i < 64 * 64; ++i) {
      buf[2 * i] = mats[m] ? mats[m]->re[i] : 0.0;
      buf[2 * i + 1] = mats[m] ? mats[m]->im[i] : 0.0;
    }
    CK(cudaMemcpyAsync(h->Hbond[m], buf.data(), buf.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  return IPEPS_OK;
}

// energy per spin = (1/12) sum over the cell's 8 bonds of Re tr(rho_b H_b), with
// the operators of upload_ops: H_r / H_l for horizontal bonds with the A / B
// site on the left, H_u / H_d for vertical bonds with A / B on top
static ipeps_status energy_of_ops(ipeps_ctm h, double* e) {
  cplx *rh, *rv;
  CKS(rdm_buffers(h, &rh, &rv));
  const long long n2 = 64LL * 64 * 4;
  const long long save = h->scratch_elems;
  h->scratch_elems -= 2 * n2;
  ipeps_status st = all_rdms(h, rh, rv);
  h->scratch_elems = save;
  CKS(st);
  CK(cudaMemsetAsync(h->dacc, 0, sizeof(double), h->stream));
  for (int y = 0; y < 2; ++y)
    for (int x = 0; x < 2; ++x) {
      const bool siteA = ((x + y) % 2) == 0;
      const long long o = (long long)(y * 2 + x) * 64 * 64;
      CK(trace_product(h->stream, rh + o, h->Hbond[siteA ? 0 : 1], 64, h->dacc, 0, 1.0 / 12.0));
      CK(trace_product(h->stream, rv + o, h->Hbond[siteA ? 2 : 3], 64, h->dacc, 0, 1.0 / 12.0));
    }
  CK(cudaMemcpyAsync(e, h->dacc, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return check_status(h);
}

extern "C" ipeps_status ipeps_energy(ipeps_ctm h, const double J[3], double* e) {
  if (!h || !J || !e) return fail(IPEPS_EINVAL, "null argument");
  if (h->d != 8 || h->Lx != 2 || h->Ly != 2)
    return fail(IPEPS_EINVAL, "the ruby energy needs a 2x2 cell of d = 8 block sites");
  NvtxRange range("energy");
  CKS(reset_status(h));
  CM Hr(64), Hv(64);
  ruby_bonds(J, &Hr, &Hv);
  const CM* mats[4] = {&Hr, nullptr, &Hv, &Hv};  // H_r, H_l (= 0), H_u, H_d
  CKS(upload_ops(h, mats));
  return energy_of_ops(h, e);
}

extern "C" ipeps_status ipeps_energy_star(ipeps_ctm h, const double J[2], double* e) {
  if (!h || !J || !e) return fail(IPEPS_EINVAL, "null argument");
  if (h->d != 8 || h->Lx != 2 || h->Ly != 2)
    return fail(IPEPS_EINVAL, "the star-lattice energy needs a 2x2 cell of d = 8 block sites");
  NvtxRange range("energy star");
  CKS(reset_status(h));
  CM Hh(64), Hv(64);
  star_bonds(J, &Hh, &Hv);
  const CM* mats[4] = {&Hh, &Hh, &Hv, nullptr};  // H_r, H_l, H_u, H_d (the trivial edge)
  CKS(upload_ops(h, mats));
  return energy_of_ops(h, e);
}

// ---------------------------------------------------------------------------
// kappa (Sec. III): window at (0,0) contracted row by row, labels generated
// ---------------------------------------------------------------------------
struct Lab {
  int next = 0;
  char fresh() {
    static const char pool[] = "abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ";
    return pool[(next++) % 52];
  }
};

// The 2x2 window of sites at (0,0) (cell indices mod Lx, Ly), contracted with
// its environment.  rows/cols select which of the window's two rows (T4 ..
// T2) and two columns (T1 .. T3) are present; the corners always are.  The
// full window (rows and cols) is the trace of the ring of enlarged corners,
// sum_{i,k} (Q1 Q2)[i,k] (Q4 Q3^T)[i,k]; the others are contracted row by row.
static ipeps_status window_contract(ipeps_ctm h, bool rows, bool cols, cplx* result) {
  const int c = h->chi, D2 = h->D2, Lx = h->Lx, Ly = h->Ly, W = 2;
  const long long mark = h->scratch_top;
  if (rows && cols) {
    CKS(enlarged_corners(h, 0, 0, 0));
    const long long K = h->K;
    cplx* Rup = scratch_alloc(h, K * K);
    cplx* Rdn = scratch_alloc(h, K * K);
    if (!Rup || !Rdn) return fail(IPEPS_ENOMEM, "scratch exhausted (kappa)");
    CKS(gemm_dispatch(h, (int)K, (int)K, (int)K, h->Q[0], K, OP_N, h->Q[1], K, OP_N, Rup, K, ONE));
    CKS(gemm_dispatch(h, (int)K, (int)K, (int)K, h->Q[3], K, OP_N, h->Q[2], K, OP_T, Rdn, K, ONE));
    TV out; out.p = result; out.nd = 0;
    CKS(contract(h, "ik,ik->", tv(Rup, {(int)K, (int)K}), false, tv(Rdn, {(int)K, (int)K}), false, out));
    h->scratch_top = mark;
    return IPEPS_OK;
  }
  const int n = cols ? W : 0;
  const int xr = (W - 1) % Lx, yb = (W - 1) % Ly;
  auto Cp = [&](int role, int x, int y) { return h->C[role][(y % Ly) * Lx + (x % Lx)]; };
  auto Tp = [&](int role, int x, int y) { return h->T[role][(y % Ly) * Lx + (x % Lx)]; };
  Lab L;
  std::string bl;
  std::vector<int> bd;
  const long long cap = (long long)c * D2 * D2 * c + (long long)c * c * D2;
  cplx* cur = scratch_alloc(h, cap);
  cplx* nxt = scratch_alloc(h, cap);
  if (!cur || !nxt) return fail(IPEPS_ENOMEM, "scratch exhausted (kappa)");
  auto view = [&](cplx* p, const std::vector<int>& dims) {
    TV t; t.p = p; t.nd = (int)dims.size();
    for (int i = 0; i < t.nd; ++i) t.dims[i] = dims[i];
    return t;
  };
  auto step = [&](cplx* op, const std::string& lop, const std::vector<int>& dop,
                  const std::string& lout) -> ipeps_status {
    std::vector<int> dout;
    long long sz = 1;
    for (char ch : lout) {
      size_t p = bl.find(ch);
      dout.push_back(p != std::string::npos ? bd[p] : dop[lop.find(ch)]);
      sz *= dout.back();
    }
    if (sz > cap) return fail(IPEPS_ENOMEM, "kappa intermediate too large");
    std::string spec = bl + "," + lop + "->" + lout;
    CKS(contract(h, spec.c_str(), view(cur, bd), false, view(op, dop), false, view(nxt, dout)));
    std::swap(cur, nxt);
    bl = lout;
    bd = dout;
    return IPEPS_OK;
  };
  {  // top: C1 [vl, h]
    char vl = L.fresh(), hh = L.fresh();
    CK(cudaMemcpyAsync(cur, Cp(0, 0, 0), (size_t)c * c * sizeof(cplx), cudaMemcpyDeviceToDevice, h->stream));
    bl = std::string() + vl + hh;
    bd = {c, c};
  }
  for (int x = 0; x < n; ++x) {  // T1[l, d, r]
    char v = L.fresh(), hn = L.fresh();
    CKS(step(Tp(0, x, 0), std::string() + bl.back() + v + hn, {c, D2, c}, bl.substr(0, bl.size() - 1) + v + hn));
  }
  {  // C2[l, d]
    char vr = L.fresh();
    CKS(step(Cp(1, xr, 0), std::string() + bl.back() + vr, {c, c}, bl.substr(0, bl.size() - 1) + vr));
  }
  for (int y = 0; y < (rows ? W : 0); ++y) {  // rows only when there are no columns
    char dn = L.fresh(), hr = L.fresh();
    CKS(step(Tp(3, 0, y), std::string() + dn + hr + bl[0], {c, D2, c}, std::string() + dn + hr + bl.substr(1)));
    char hx = bl[1], vr = bl[2], dd = L.fresh();
    CKS(step(Tp(1, xr, y), std::string() + vr + hx + dd, {c, D2, c}, bl.substr(0, 1) + dd));
  }
  {  // C4[r, u]
    char hb = L.fresh();
    CKS(step(Cp(3, 0, yb), std::string() + hb + bl[0], {c, c}, std::string() + hb + bl.substr(1)));
  }
  for (int x = 0; x < n; ++x) {  // T3[r, u, l]
    char hb = bl[0], vx = bl[1], rr = L.fresh();
    CKS(step(Tp(2, x, yb), std::string() + rr + vx + hb, {c, D2, c}, std::string() + rr + bl.substr(2)));
  }
  {  // C3[u=vr, l=hb] -> scalar
    std::string lop = std::string() + bl[1] + bl[0];
    std::string spec = bl + "," + lop + "->";
    TV out; out.p = result; out.nd = 0;
    CKS(contract(h, spec.c_str(), view(cur, bd), false, tv(Cp(2, xr, yb), {c, c}), false, out));
  }
  h->scratch_top = mark;
  return IPEPS_OK;
}

static ipeps_status kappa_host(ipeps_ctm h, double* kre, double* kim) {
  CKS(window_contract(h, true, true, h->scalar + 0));
  CKS(window_contract(h, false, false, h->scalar + 1));
  CKS(window_contract(h, false, true, h->scalar + 2));
  CKS(window_contract(h, true, false, h->scalar + 3));
  cplx z[4];
  CK(cudaMemcpyAsync(z, h->scalar, sizeof z, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  // kappa = Z_cell Z_00 / (Z_cols Z_rows)
  const double nr = z[0].x * z[1].x - z[0].y * z[1].y, ni = z[0].x * z[1].y + z[0].y * z[1].x;
  const double dr = z[2].x * z[3].x - z[2].y * z[3].y, di = z[2].x * z[3].y + z[2].y * z[3].x;
  const double den = dr * dr + di * di;
  if (!(den > 0)) return fail(IPEPS_ENUMERIC, "zero partition ratio denominator");
  *kre = (nr * dr + ni * di) / den;
  *kim = (ni * dr - nr * di) / den;
  return IPEPS_OK;
}

extern "C" ipeps_status ipeps_kappa(ipeps_ctm h, double* k) {
  if (!h || !k) return fail(IPEPS_EINVAL, "null argument");
  NvtxRange range("kappa");
  CKS(reset_status(h));
  CKS(kappa_host(h, k, k + 1));
  return check_status(h);
}

// Fidelity per block site from the kappas of the mixed and the two plain
// networks (Eq. "fidelity" with the normalisation of each state divided out):
// d = (|k12| / sqrt(|k11| |k22|))^(1/4) on the 2x2 window, per spin d^(1/3).
void fidelity_from_kappa(const double k12[2], const double k11[2], const double k22[2], double* d_block,
                         double* d_spin) {
  const int ns = 4;  // sites of the 2x2 window kappa is taken on
  const double l12 = log(hypot(k12[0], k12[1])), l11 = log(hypot(k11[0], k11[1]));
  const double l22 = log(hypot(k22[0], k22[1]));
  const double db = exp((l12 - 0.5 * (l11 + l22)) / ns);
  if (d_block) *d_block = db;
  if (d_spin) *d_spin = pow(db, 1.0 / 3.0);
}

extern "C" ipeps_status ipeps_fidelity(ipeps_ctm h12, ipeps_ctm h11, ipeps_ctm h22, double* d_block,
                                       double* d_spin) {
  if (!h12 || !h11 || !h22) return fail(IPEPS_EINVAL, "null handle");
  if (h12->Lx != h11->Lx || h12->Ly != h11->Ly || h22->Lx != h11->Lx || h22->Ly != h11->Ly)
    return fail(IPEPS_EINVAL, "cells differ");
  double k[3][2];
  CKS(ipeps_kappa(h12, k[0]));
  CKS(ipeps_kappa(h11, k[1]));
  CKS(ipeps_kappa(h22, k[2]));
  fidelity_from_kappa(k[0], k[1], k[2], d_block, d_spin);
  return IPEPS_OK;
}

void ctm_cell(ipeps_ctm h, int* Lx, int* Ly) {
  *Lx = h->Lx;
  *Ly = h->Ly;
}

// ---------------------------------------------------------------------------
// boundary density operator (Sec. IV)
// ---------------------------------------------------------------------------
// half ring of `len` edge tensors starting at row y0 of column xc in role
// `role` (T2: [u,(k,b),d] going down; T4: [d,(k,b),u] going down) -> out
// [c_first, K, B, c_last] with K, B the fused ket / bra multi-indices.
static ipeps_status half_ring(ipeps_ctm h, int role, int xc, int y0, int len, cplx* out, cplx* tmp) {
  const int c = h->chi, D = h->D;
  auto Tptr = [&](int i) { return h->T[role][((y0 + i) % h->Ly) * h->Lx + xc]; };
  long long Kd = D;
  // first tensor as [c0, k, b, c1]
  if (role == 1) {
    CK(cudaMemcpyAsync(out, Tptr(0), (size_t)c * D * D * c * sizeof(cplx), cudaMemcpyDeviceToDevice, h->stream));
  } else {
    const int dims[4] = {c, D, D, c};
    const int perm[4] = {3, 1, 2, 0};
    CK(permute(h->stream, Tptr(0), out, 4, dims, perm, false, ONE));
  }
  for (int i = 1; i < len; ++i) {
    // R[a, K, B, c] T[c, k, b, e] -> [a, K, k, B, b, e]
    if (role == 1)
      CKS(contract(h, "aKBc,ckbe->aKkBbe", tv(out, {c, (int)Kd, (int)Kd, c}), false,
                   tv(Tptr(i), {c, D, D, c}), false, tv(tmp, {c, (int)Kd, D, (int)Kd, D, c})));
    else
      CKS(contract(h, "aKBc,ekbc->aKkBbe", tv(out, {c, (int)Kd, (int)Kd, c}), false,
                   tv(Tptr(i), {c, D, D, c}), false, tv(tmp, {c, (int)Kd, D, (int)Kd, D, c})));
    Kd *= D;
    CK(cudaMemcpyAsync(out, tmp, (size_t)c * Kd * Kd * c * sizeof(cplx), cudaMemcpyDeviceToDevice, h->stream));
  }
  return IPEPS_OK;
}

static ipeps_status ring_sigma(ipeps_ctm h, int role, int xc, int Nv, cplx* sigma) {
  const int c = h->chi, D = h->D;
  const int h1 = Nv / 2, h2 = Nv - h1;
  long long K1 = 1, K2 = 1;
  for (int i = 0; i < h1; ++i) K1 *= D;
  for (int i = 0; i < h2; ++i) K2 *= D;
  cplx* H1 = scratch_alloc(h, (long long)c * K1 * K1 * c);
  cplx* H2 = scratch_alloc(h, (long long)c * K2 * K2 * c);
  cplx* tmp = scratch_alloc(h, (long long)c * K2 * K2 * c);
  if (!H1 || !H2 || !tmp) return fail(IPEPS_ENOMEM, "scratch exhausted (ring)");
  if (h1 > 0) CKS(half_ring(h, role, xc, 0, h1, H1, tmp));
  CKS(half_ring(h, role, xc, h1, h2, H2, tmp));
  if (h1 == 0) {
    // single tensor ring: trace its two chi legs
    return fail(IPEPS_EINVAL, "Nv must be >= 2");
  }
  // sigma[(K1 K2),(B1 B2)] = sum_{a,m} H1[a,K1,B1,m] H2[m,K2,B2,a]
  CKS(contract(h, "aKBm,mLEa->KLBE", tv(H1, {c, (int)K1, (int)K1, c}), false,
               tv(H2, {c, (int)K2, (int)K2, c}), false, tv(sigma, {(int)K1, (int)K2, (int)K1, (int)K2})));
  return IPEPS_OK;
}

namespace bnd {
void launch_phase_herm(cudaStream_t s, cplx* S, int n, bool transpose_out, double* work);
void launch_spectrum_finish(cudaStream_t s, const double* sigma, int n, double* lam, double* S_vn);
void launch_scale_cols(cudaStream_t s, cplx* G, int n, const double* sigma);
}  // namespace bnd

// Dense boundary spectrum of the rings sL, sR (n x n operators, overwritten):
// phase-fix by the trace and Hermitise (sL replaced by sigma_L^T), the
// |sigma_L^T|^(1/2) factor from a Jacobi SVD, the similar operator and its
// singular values, normalised, with their entropy.  G, Hm, Vt: n^2 work each.
static ipeps_status spectrum_of_rings_dev(ipeps_ctm h, cplx* sL, cplx* sR, int nn, cplx* G, cplx* Hm, cplx* Vt,
                                          double* eig_out, double* S_vn) {
  const long long n = nn;
  bnd::launch_phase_herm(h->stream, sL, nn, true, h->dwork);
  bnd::launch_phase_herm(h->stream, sR, nn, false, h->dwork);
  count_launch(2);
  CK(cudaGetLastError());
  // |sigma_L^T|^(1/2) factor: Jacobi on the rows of sigma_L^T gives rows
  // lambda_i w_i^H; G = (rows)^H scaled by sigma_i^(-1/2) column-wise.
  CK(cudaMemcpyAsync(G, sL, n * n * sizeof(cplx), cudaMemcpyDeviceToDevice, h->stream));
  CK(jacobi_rows(h->stream, G, nn, nn, nn, nullptr, h->sigma, h->opt.jacobi_max_sweeps, h->dwork,
                 h->counters, h->st, nullptr, 0, h->opt.wait_cycles));
  // Gm = G^H (n x n), columns scaled
  {
    const int dims[2] = {nn, nn}, perm[2] = {1, 0};
    CK(permute(h->stream, G, Hm, 2, dims, perm, true, ONE));
  }
  bnd::launch_scale_cols(h->stream, Hm, nn, h->sigma);
  count_launch();
  CK(cudaGetLastError());
  // H = Gm^H sR Gm
  CK(zgemm(h->stream, nn, nn, nn, ONE, sR, nn, OP_N, Hm, nn, OP_N, ZERO, G, nn));
  CK(zgemm(h->stream, nn, nn, nn, ONE, Hm, nn, OP_H, G, nn, OP_N, ZERO, Vt, nn));
  CK(jacobi_rows(h->stream, Vt, nn, nn, nn, nullptr, h->sigma, h->opt.jacobi_max_sweeps, h->dwork,
                 h->counters, h->st, nullptr, 0, h->opt.wait_cycles));
  bnd::launch_spectrum_finish(h->stream, h->sigma, nn, h->s_sel, h->dacc);
  count_launch();
  CK(cudaGetLastError());
  if (eig_out) CK(cudaMemcpyAsync(eig_out, h->s_sel, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  double S = 0;
  CK(cudaMemcpyAsync(&S, h->dacc, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (S_vn) *S_vn = S;
  return IPEPS_OK;
}

extern "C" ipeps_status ipeps_boundary_rho(ipeps_ctm h, int x, int Nv, double* eig_out, int* n_out,
                                           double* S_vn) {
  if (!h) return fail(IPEPS_EINVAL, "null handle");
  if (Nv < 2 || Nv % h->Ly) return fail(IPEPS_EINVAL, "Nv must be a multiple of Ly and >= 2");
  long long n = 1;
  for (int i = 0; i < Nv; ++i) n *= h->D;
  if (n > 4096) return fail(IPEPS_EINVAL, "D^Nv = %lld > 4096", n);
  NvtxRange range("boundary rho");
  CKS(reset_status(h));
  const int nn = (int)n;
  const long long mark = h->scratch_top;
  cplx* sL = scratch_alloc(h, n * n);
  cplx* sR = scratch_alloc(h, n * n);
  cplx* G = scratch_alloc(h, n * n);
  cplx* Hm = scratch_alloc(h, n * n);
  cplx* Vt = scratch_alloc(h, n * n);
  if (!sL || !sR || !G || !Hm || !Vt) return fail(IPEPS_ENOMEM, "scratch exhausted (boundary rho)");
  const long long inner = h->scratch_top;
  const int xl = ((x + 1) % h->Lx + h->Lx) % h->Lx, xr = ((x % h->Lx) + h->Lx) % h->Lx;
  CKS(ring_sigma(h, 3, xl, Nv, sL));
  h->scratch_top = inner;
  CKS(ring_sigma(h, 1, xr, Nv, sR));
  h->scratch_top = inner;
  CKS(spectrum_of_rings_dev(h, sL, sR, nn, G, Hm, Vt, eig_out, S_vn));
  h->scratch_top = mark;
  if (n_out) *n_out = nn;
  return check_status(h);
}

namespace bnd {
void launch_interleave(cudaStream_t s, const cplx* in, cplx* out, int D, int Nv, bool to_vector);
void launch_diff_norm2(cudaStream_t s, const cplx* a, const cplx* b, long long n, double* work, double* out);
}  // namespace bnd

// One column of the cylinder's transfer matrix (rows 0..Nv-1 of column col,
// periodic vertically) applied to a boundary vector v (one D^2 index per row):
// right = true: out(l) = sum_{r,u} prod_i a_i[u_i, l_i, u_{i+1}, r_i] v(r);
// right = false: the same with the roles of l and r exchanged (v from the left).
// Rows are absorbed one at a time; the open u leg of row 0 (A) is traced with
// the last row's d leg at the end.  w0, w1: D^(2 Nv + 4) complex each.
static ipeps_status column_apply(ipeps_ctm h, int col, int Nv, const cplx* v, cplx* out, bool right, cplx* w0,
                                 cplx* w1, const cplx* ident) {
  const int D2 = h->D2;
  long long Rn = 1;
  for (int i = 0; i < Nv - 1; ++i) Rn *= D2;
  cplx* wa = w0;
  cplx* wb = w1;
  CKS(contract(h, right ? "ulvr,rR->ulvR" : "ulvr,lR->urvR", tv(site_a(h, 0, col, 0), {D2, D2, D2, D2}), false,
               tv((cplx*)v, {D2, (int)Rn}), false, tv(wa, {D2, D2, D2, (int)Rn})));
  long long Ld = D2;
  for (int i = 1; i < Nv; ++i) {
    Rn /= D2;
    CKS(contract(h, right ? "ALurR,ulvr->ALlvR" : "ALulR,ulvr->ALrvR",
                 tv(wa, {D2, (int)Ld, D2, D2, (int)Rn}), false, tv(site_a(h, 0, col, i), {D2, D2, D2, D2}), false,
                 tv(wb, {D2, (int)Ld, D2, D2, (int)Rn})));
    Ld *= D2;
    std::swap(wa, wb);
  }
  CKS(contract(h, "ALB,AB->L", tv(wa, {D2, (int)Ld, D2}), false, tv((cplx*)ident, {D2, D2}), false,
               tv(out, {(int)Ld})));
  return IPEPS_OK;
}

// Sec. IV beyond the ring approximation: sigma_L, sigma_R refined by power
// iteration with the exact column transfer matrices of one cell period,
// starting from the CTM rings; then the dense boundary spectrum.
extern "C" ipeps_status ipeps_boundary_rho_refined(ipeps_ctm h, int x, int Nv, int iters, double tol,
                                                   double* eig_out, int* n_out, double* S_vn, int* iters_used,
                                                   double* change) {
  if (!h) return fail(IPEPS_EINVAL, "null handle");
  if (Nv < 2 || Nv % h->Ly) return fail(IPEPS_EINVAL, "Nv must be a multiple of Ly and >= 2");
  if (iters < 0) return fail(IPEPS_EINVAL, "iters must be >= 0");
  long long n = 1;
  for (int i = 0; i < Nv; ++i) n *= h->D;
  if (n > 4096) return fail(IPEPS_EINVAL, "D^Nv = %lld > 4096", n);
  const long long n2 = n * n, big = n2 * h->D2 * h->D2;
  if (big > (1LL << 28)) return fail(IPEPS_EINVAL, "D^(2 Nv + 4) = %lld above 2^28", big);
  NvtxRange range("boundary rho refined");
  CKS(reset_status(h));
  // region: vectors vL, vR, res, tmp (n^2 each), identity, w0, w1 (big each),
  // spectrum work (5 n^2), contraction scratch (the rest)
  const long long D4 = (long long)h->D2 * h->D2;
  const long long id_elems = (D4 + 15) & ~15LL;
  const long long fixed = 4 * n2 + id_elems + 2 * big + 5 * n2;
  const long long region_elems = fixed + 3 * big + 4 * (long long)h->chi * h->chi * (n + 64) + (1LL << 22);
  cplx* mem = nullptr;
  cudaError_t e = dev_alloc((void**)&mem, (size_t)region_elems * sizeof(cplx));
  if (e != cudaSuccess)
    return fail(IPEPS_ENOMEM, "boundary rho refined: cudaMalloc of %.1f GB failed: %s",
                (double)region_elems * 16e-9, cudaGetErrorString(e));
  cplx* vec[2] = {mem, mem + n2};  // [0] = sigma_L, [1] = sigma_R
  cplx* res = mem + 2 * n2;
  cplx* tmp = mem + 3 * n2;
  cplx* ident = mem + 4 * n2;
  cplx* w0 = ident + id_elems;
  cplx* w1 = w0 + big;
  cplx* sL = w1 + big;
  cplx* sR = sL + n2;
  cplx* G = sR + n2;
  cplx* Hm = G + n2;
  cplx* Vt = Hm + n2;
  cplx* save_scratch = h->scratch;
  const long long save_elems = h->scratch_elems, save_top = h->scratch_top;
  h->scratch = mem + fixed;
  h->scratch_elems = region_elems - fixed;
  h->scratch_top = 0;
  auto body = [&]() -> ipeps_status {
    std::vector<double> id(2 * D4, 0.0);
    for (int i = 0; i < h->D2; ++i) id[2 * (i * h->D2 + i)] = 1.0;
    CK(cudaMemcpyAsync(ident, id.data(), id.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    const int xl = ((x + 1) % h->Lx + h->Lx) % h->Lx, xr = ((x % h->Lx) + h->Lx) % h->Lx;
    CKS(ring_sigma(h, 3, xl, Nv, sL));
    h->scratch_top = 0;
    CKS(ring_sigma(h, 1, xr, Nv, sR));
    h->scratch_top = 0;
    bnd::launch_interleave(h->stream, sL, vec[0], h->D, Nv, true);
    bnd::launch_interleave(h->stream, sR, vec[1], h->D, Nv, true);
    count_launch(2);
    CK(cudaGetLastError());
    for (int q = 0; q < 2; ++q) CK(normalize(h->stream, vec[q], n2, h->dwork, h->st));
    double2* partial = (double2*)(h->dwork + 2048);  // 512 double2 after the norm work
    double2* ovd = (double2*)(h->dwork + 3072);
    double* d2 = h->dwork + 3080;
    int it = 0;
    double ch = INFINITY;
    while (it < iters) {
      ch = 0.0;
      for (int q = 0; q < 2; ++q) {
        const bool right = q == 1;
        // one cell period: sigma_R <- E_{x+1} .. E_{x+Lx} sigma_R; sigma_L <- sigma_L E_{x-Lx+1} .. E_x
        const cplx* in = vec[q];
        cplx* bufs[2] = {res, tmp};
        int nb = 0;
        for (int c = 0; c < h->Lx; ++c) {
          const int col = right ? ((x + h->Lx - c) % h->Lx + h->Lx) % h->Lx : ((x - h->Lx + 1 + c) % h->Lx + h->Lx) % h->Lx;
          cplx* out = bufs[nb];
          CKS(column_apply(h, col, Nv, in, out, right, w0, w1, ident));
          h->scratch_top = 0;
          in = out;
          nb ^= 1;
        }
        cplx* nv = (cplx*)in;
        CK(normalize(h->stream, nv, n2, h->dwork, h->st));
        CK(zdotc_dev(h->stream, vec[q], nv, n2, partial, ovd));
        double2 ov;
        CK(cudaMemcpyAsync(&ov, ovd, sizeof ov, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        const double m = hypot(ov.x, ov.y);
        if (!(m > 0)) return fail(IPEPS_ENUMERIC, "boundary rho refined: orthogonal iterates");
        const int dims1[1] = {(int)n2}, perm1[1] = {0};
        CK(permute(h->stream, nv, nv, 1, dims1, perm1, false, make_double2(ov.x / m, -ov.y / m)));
        bnd::launch_diff_norm2(h->stream, nv, vec[q], n2, h->dwork, d2);
        count_launch(2);
        double dd = 0.0;
        CK(cudaMemcpyAsync(&dd, d2, sizeof dd, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaMemcpyAsync(vec[q], nv, n2 * sizeof(cplx), cudaMemcpyDeviceToDevice, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        ch = std::max(ch, sqrt(dd));
      }
      ++it;
      if (ch < tol) break;
    }
    bnd::launch_interleave(h->stream, vec[0], sL, h->D, Nv, false);
    bnd::launch_interleave(h->stream, vec[1], sR, h->D, Nv, false);
    count_launch(2);
    CK(cudaGetLastError());
    CKS(spectrum_of_rings_dev(h, sL, sR, (int)n, G, Hm, Vt, eig_out, S_vn));
    if (iters_used) *iters_used = it;
    if (change) *change = ch;
    return IPEPS_OK;
  };
  const ipeps_status st = body();
  h->scratch = save_scratch;
  h->scratch_elems = save_elems;
  h->scratch_top = save_top;
  cudaStreamSynchronize(h->stream);
  cudaFree(mem);
  CKS(st);
  if (n_out) *n_out = (int)n;
  return check_status(h);
}

// ---------------------------------------------------------------------------
// Long cylinders (Sec. IV): the rings as dense operators built by one product
// of two half rings laid out for it, and the leading spectrum by Lanczos.
// ---------------------------------------------------------------------------
// Half ring of `len` edge tensors (role T2 = 1 or T4 = 3) at column xc from
// row y0 down, inner chi legs contracted, written in the layout the ring
// product reads directly (no operand permutation):
//   upper: out[K, B, a, m]  (a: open chi leg at the top, m: at the bottom)
//   lower: out[a, m, K, B]  (m: open chi leg at the top, a: at the bottom)
// K / B fuse the ket / bra legs of the len sites, the first site slowest.
static ipeps_status half_ring_layout(ipeps_ctm h, int role, int xc, int y0, int len, bool upper, cplx* out) {
  const int c = h->chi, D = h->D;
  auto Tptr = [&](int i) { return h->T[role][((y0 + i) % h->Ly) * h->Lx + xc]; };
  const long long mark = h->scratch_top;
  // working form R[c0, K, B, c1] of the first tensor
  cplx* cur = Tptr(0);
  if (role != 1) {
    cur = scratch_alloc(h, (long long)c * D * D * c);
    if (!cur) return fail(IPEPS_ENOMEM, "scratch exhausted (half ring)");
    const int dims[4] = {c, D, D, c}, perm[4] = {3, 1, 2, 0};
    CK(permute(h->stream, Tptr(0), cur, 4, dims, perm, false, ONE));
  }
  long long Kd = D;
  if (len == 1) {
    const int dims[4] = {c, D, D, c};
    const int pu[4] = {1, 2, 0, 3}, pl[4] = {3, 0, 1, 2};
    CK(permute(h->stream, cur, out, 4, dims, upper ? pu : pl, false, ONE));
    h->scratch_top = mark;
    return IPEPS_OK;
  }
  const char* in_spec = role == 1 ? "aKBc,ckbe" : "aKBc,ekbc";
  for (int i = 1; i < len; ++i) {
    const TV R = tv(cur, {c, (int)Kd, (int)Kd, c});
    const TV T = tv(Tptr(i), {c, D, D, c});
    if (i < len - 1) {
      cplx* nxt = scratch_alloc(h, (long long)c * Kd * D * Kd * D * c);
      if (!nxt) return fail(IPEPS_ENOMEM, "scratch exhausted (half ring)");
      CKS(contract(h, (std::string(in_spec) + "->aKkBbe").c_str(), R, false, T, false,
                   tv(nxt, {c, (int)Kd, D, (int)Kd, D, c})));
      cur = nxt;
      Kd *= D;
    } else if (upper) {
      CKS(contract(h, (std::string(in_spec) + "->KkBbae").c_str(), R, false, T, false,
                   tv(out, {(int)Kd, D, (int)Kd, D, c, c})));
    } else {
      CKS(contract(h, (std::string(in_spec) + "->eaKkBb").c_str(), R, false, T, false,
                   tv(out, {c, c, (int)Kd, D, (int)Kd, D})));
    }
  }
  h->scratch_top = mark;
  return IPEPS_OK;
}

// sigma[(K1 K2), (B1 B2)] of the ring of Nv edge tensors (role, column xc):
// t[(K1 B1), (K2 B2)] = H1[(K1 B1), (a m)] H2[(a m), (K2 B2)] in the handle's
// contraction arithmetic, then one permutation into sigma.  Uses the handle's
// scratch from its current top: t first, then the half rings and the
// product's own work.  sigma must not overlap t.
// complex elements of scratch the ring product's packed tensor-core operands
// take, per n chi^2 (A: n x 2 chi^2 reals, B: 2n x 2 chi^2 reals, 2-byte parts:
// two parts for BF16x3, three for BF16x6, one 4-byte part for TF32), with margin
static double ring_pack_factor(ipeps_ctm h) { return h->opt.prec == IPEPS_PREC_BF16X6 ? 2.4 : 1.6; }

static ipeps_status ring_sigma_dense(ipeps_ctm h, int role, int xc, int Nv, cplx* sigma) {
  const int c = h->chi, D = h->D;
  const int h1 = Nv / 2, h2 = Nv - h1;
  long long K1 = 1, K2 = 1;
  for (int i = 0; i < h1; ++i) K1 *= D;
  for (int i = 0; i < h2; ++i) K2 *= D;
  const long long mark = h->scratch_top;
  cplx* t = scratch_alloc(h, K1 * K1 * K2 * K2);
  cplx* H1 = scratch_alloc(h, K1 * K1 * c * c);
  cplx* H2 = scratch_alloc(h, K2 * K2 * c * c);
  if (!t || !H1 || !H2) return fail(IPEPS_ENOMEM, "scratch exhausted (ring)");
  CKS(half_ring_layout(h, role, xc, 0, h1, true, H1));
  CKS(half_ring_layout(h, role, xc, h1, h2, false, H2));
  CKS(gemm_dispatch(h, (int)(K1 * K1), (int)(K2 * K2), c * c, H1, (long long)c * c, OP_N, H2, K2 * K2, OP_N, t,
                    K2 * K2, ONE));
  const int dims[4] = {(int)K1, (int)K1, (int)K2, (int)K2}, perm[4] = {0, 2, 1, 3};
  CK(permute(h->stream, t, sigma, 4, dims, perm, false, ONE));
  h->scratch_top = mark;
  return IPEPS_OK;
}

extern "C" ipeps_status ipeps_boundary_rho_topk(ipeps_ctm h, int x, int Nv, int k, int max_iter, double tol,
                                                double* eig_out, int* n_conv, double* S_vn, double* rest) {
  if (!h) return fail(IPEPS_EINVAL, "null handle");
  if (Nv < 2 || Nv % h->Ly) return fail(IPEPS_EINVAL, "Nv must be a multiple of Ly and >= 2");
  long long n = 1;
  for (int i = 0; i < Nv; ++i) {
    n *= h->D;
    if (n > 200000) return fail(IPEPS_EINVAL, "D^Nv above 200000");
  }
  if (k < 1 || max_iter < k || max_iter > 1024 || max_iter > n)
    return fail(IPEPS_EINVAL, "need 1 <= k <= max_iter <= min(1024, D^Nv)");
  if (!(tol > 0.0)) return fail(IPEPS_EINVAL, "tol must be positive");
  NvtxRange range("boundary rho leading");
  CKS(reset_status(h));
  const long long c2 = (long long)h->chi * h->chi;
  long long K1 = 1, K2 = 1;
  for (int i = 0; i < Nv / 2; ++i) K1 *= h->D;
  for (int i = 0; i < Nv - Nv / 2; ++i) K2 *= h->D;
  // region: [t | H1 | H2 | work of the half rings and of the ring product]
  // while a ring is built; [. | sigma_R | Lanczos work] afterwards
  const long long n2 = n * n;
  // half rings: the last step's product output (chi^2 K^2) plus small
  // intermediates; ring product: its packed tensor-core operands (~1.5 n chi^2)
  const long long ring_work = std::max(c2 * std::max(K1 * K1, K2 * K2) * 5 / 4,
                                       (long long)(ring_pack_factor(h) * (double)n * (double)c2)) + (1LL << 24);
  const long long ring_phase = n2 + c2 * (K1 * K1 + K2 * K2) + ring_work;
  const long long krylov_phase = 2 * n2 + lanczos_work_elems(n, max_iter) + 1024;
  const long long region_elems = std::max(ring_phase, krylov_phase);
  cplx* mem = nullptr;
  cudaError_t e = dev_alloc((void**)&mem, (size_t)(n2 + region_elems) * sizeof(cplx));
  if (e != cudaSuccess)
    return fail(IPEPS_ENOMEM, "boundary rho: cudaMalloc of %.1f GB failed: %s",
                (double)(n2 + region_elems) * 16e-9, cudaGetErrorString(e));
  cplx* sL = mem;
  cplx* region = mem + n2;
  cplx* sR = region + n2;  // written over the dead half rings after the ring product
  cplx* save_scratch = h->scratch;
  const long long save_elems = h->scratch_elems, save_top = h->scratch_top;
  h->scratch = region;
  h->scratch_elems = region_elems;
  h->scratch_top = 0;
  const int xl = ((x + 1) % h->Lx + h->Lx) % h->Lx, xr = ((x % h->Lx) + h->Lx) % h->Lx;
  cudaEvent_t pr = nullptr;
  prof_begin(h, &pr);
  ipeps_status st = ring_sigma_dense(h, 3, xl, Nv, sL);
  if (st == IPEPS_OK) st = ring_sigma_dense(h, 1, xr, Nv, sR);
  prof_end(h, pr, 2.0 * 8.0 * (double)n * (double)n * (double)c2, 3);
  h->scratch = save_scratch;
  h->scratch_elems = save_elems;
  h->scratch_top = save_top;
  LanczosResult res{0, 0, 0, 0};
  double out2[2] = {0.0, 0.0};
  if (st == IPEPS_OK) {
    // phase-fix by the trace, Hermitise; sL is replaced by sigma_L^T
    bnd::launch_phase_herm(h->stream, sL, (int)n, true, h->dwork);
    bnd::launch_phase_herm(h->stream, sR, (int)n, false, h->dwork);
    count_launch(4);
    cplx* work = region + 2 * n2;
    const long long work_elems = region_elems - 2 * n2;
    e = cudaGetLastError();
    cudaEvent_t pl = nullptr;
    prof_begin(h, &pl);
    if (e == cudaSuccess)
      e = lanczos_leading(h->stream, sL, sR, n, k, max_iter, tol, h->opt.omega_seed ^ 0x5bd1e995ULL, work,
                          work_elems, h->s_sel, tc_form(h->opt.prec), &res);
    prof_end(h, pl, (double)res.iters, 4);
    double2* partial = (double2*)work;
    double2* trd = partial + 512;
    double* lam = (double*)(trd + 1);
    double* dout = lam + k + 1;
    if (e == cudaSuccess) e = topk_finish(h->stream, sL, sR, n, h->s_sel, k, partial, trd, lam, dout);
    if (e == cudaSuccess && eig_out)
      e = cudaMemcpyAsync(eig_out, lam, k * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out2, dout, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) st = fail(IPEPS_ECUDA, "boundary rho (Lanczos): %s", cudaGetErrorString(e));
  }
  cudaStreamSynchronize(h->stream);
  cudaFree(mem);
  CKS(st);
  if (res.indefinite) return fail(IPEPS_ENUMERIC, "sigma_R is not positive definite (negative norm in Lanczos)");
  if (n_conv) *n_conv = res.converged;
  if (S_vn) *S_vn = out2[0];
  if (rest) *rest = out2[1];
  return check_status(h);
}

namespace bnd {
void launch_purity(cudaStream_t s, const cplx* M, int n, double* work, double* out);
}

// Second Renyi entropy of the boundary density operator from traces of the
// dense product M = sigma_L^T sigma_R (Sec. IV): purity tr(M^2)/(tr M)^2.
extern "C" ipeps_status ipeps_boundary_renyi2(ipeps_ctm h, int x, int Nv, double* S2, double* purity) {
  if (!h) return fail(IPEPS_EINVAL, "null handle");
  if (Nv < 2 || Nv % h->Ly) return fail(IPEPS_EINVAL, "Nv must be a multiple of Ly and >= 2");
  const long long n_max = !tc_form(h->opt.prec) ? 4096 : 200000;
  long long n = 1;
  for (int i = 0; i < Nv; ++i) {
    n *= h->D;
    if (n > n_max) return fail(IPEPS_EINVAL, "D^Nv above %lld for this precision", n_max);
  }
  NvtxRange range("boundary renyi2");
  CKS(reset_status(h));
  const long long c2 = (long long)h->chi * h->chi, n2 = n * n;
  long long K1 = 1, K2 = 1;
  for (int i = 0; i < Nv / 2; ++i) K1 *= h->D;
  for (int i = 0; i < Nv - Nv / 2; ++i) K2 *= h->D;
  const long long ring_work = std::max(c2 * std::max(K1 * K1, K2 * K2) * 5 / 4,
                                       (long long)(ring_pack_factor(h) * (double)n * (double)c2)) + (1LL << 24);
  const long long ring_phase = n2 + c2 * (K1 * K1 + K2 * K2) + ring_work;
  // product phase: sigma_R, M and the product's packed operands (BF16x6: 2.25 n^2)
  const long long product_phase = 2 * n2 + (!tc_form(h->opt.prec) ? n2 : (9 * n2) / 4) + (1LL << 24);
  const long long region_elems = std::max(ring_phase, product_phase);
  cplx* mem = nullptr;
  cudaError_t e = dev_alloc((void**)&mem, (size_t)(n2 + region_elems) * sizeof(cplx));
  if (e != cudaSuccess)
    return fail(IPEPS_ENOMEM, "boundary renyi2: cudaMalloc of %.1f GB failed: %s",
                (double)(n2 + region_elems) * 16e-9, cudaGetErrorString(e));
  cplx* sL = mem;
  cplx* region = mem + n2;
  cplx* sR = region + n2;
  cplx* save_scratch = h->scratch;
  const long long save_elems = h->scratch_elems, save_top = h->scratch_top;
  h->scratch = region;
  h->scratch_elems = region_elems;
  h->scratch_top = 0;
  const int xl = ((x + 1) % h->Lx + h->Lx) % h->Lx, xr = ((x % h->Lx) + h->Lx) % h->Lx;
  ipeps_status st = ring_sigma_dense(h, 3, xl, Nv, sL);
  if (st == IPEPS_OK) st = ring_sigma_dense(h, 1, xr, Nv, sR);
  double tr[4] = {0.0, 0.0, 0.0, 0.0};
  if (st == IPEPS_OK) {
    bnd::launch_phase_herm(h->stream, sL, (int)n, true, h->dwork);  // sL <- sigma_L^T
    bnd::launch_phase_herm(h->stream, sR, (int)n, false, h->dwork);
    count_launch(4);
    cplx* M = region;  // the half rings are dead: M takes their place, sigma_R stays after it
    h->scratch = region + 2 * n2;
    h->scratch_elems = region_elems - 2 * n2;
    h->scratch_top = 0;
    cudaEvent_t pr = nullptr;
    prof_begin(h, &pr);
    st = gemm_dispatch(h, (int)n, (int)n, (int)n, sL, n, OP_N, sR, n, OP_N, M, n, ONE);
    prof_end(h, pr, 8.0 * (double)n * (double)n * (double)n, 3);
    if (st == IPEPS_OK) {
      double* out = h->dwork + 4000;  // after the block partials (dwork[2 .. 2434))
      bnd::launch_purity(h->stream, M, (int)n, h->dwork, out);
      count_launch(3);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaMemcpyAsync(tr, out, sizeof tr, cudaMemcpyDeviceToHost, h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
      if (e != cudaSuccess) st = fail(IPEPS_ECUDA, "boundary renyi2: %s", cudaGetErrorString(e));
    }
  }
  h->scratch = save_scratch;
  h->scratch_elems = save_elems;
  h->scratch_top = save_top;
  cudaStreamSynchronize(h->stream);
  cudaFree(mem);
  CKS(st);
  if (!(tr[0] != 0.0) || !std::isfinite(tr[2])) return fail(IPEPS_ENUMERIC, "boundary renyi2: tr M = %g", tr[0]);
  const double p = tr[2] / (tr[0] * tr[0]);
  if (purity) *purity = p;
  if (S2) *S2 = -log(p);
  return check_status(h);
}

extern "C" ipeps_status ipeps_ctm_env_get(ipeps_ctm h, int role, int x, int y, double* out) {
  if (!h || !out) return fail(IPEPS_EINVAL, "null argument");
  if (role < 0 || role > 7 || x < 0 || x >= h->Lx || y < 0 || y >= h->Ly)
    return fail(IPEPS_EINVAL, "bad role/position");
  const long long n = role < 4 ? (long long)h->chi * h->chi : (long long)h->chi * h->D2 * h->chi;
  const cplx* src = role < 4 ? h->C[role][y * h->Lx + x] : h->T[role - 4][y * h->Lx + x];
  CK(cudaMemcpyAsync(out, src, n * sizeof(cplx), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return IPEPS_OK;
}

extern "C" ipeps_status ipeps_ctm_env_set(ipeps_ctm h, int role, int x, int y, const double* in) {
  if (!h || !in) return fail(IPEPS_EINVAL, "null argument");
  if (role < 0 || role > 7 || x < 0 || x >= h->Lx || y < 0 || y >= h->Ly)
    return fail(IPEPS_EINVAL, "bad role/position");
  const long long n = role < 4 ? (long long)h->chi * h->chi : (long long)h->chi * h->D2 * h->chi;
  cplx* dst = role < 4 ? h->C[role][y * h->Lx + x] : h->T[role - 4][y * h->Lx + x];
  CK(cudaMemcpyAsync(dst, in, n * sizeof(cplx), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return IPEPS_OK;
}

extern "C" ipeps_status ipeps_ctm_env_copy(ipeps_ctm dst, ipeps_ctm src) {
  if (!dst || !src) return fail(IPEPS_EINVAL, "null handle");
  if (dst == src) return IPEPS_OK;
  if (dst->Lx != src->Lx || dst->Ly != src->Ly || dst->D != src->D || dst->chi != src->chi)
    return fail(IPEPS_EINVAL, "env copy: the handles differ in Lx, Ly, D or chi");
  // the copies run on dst's stream after everything queued on src's
  cudaEvent_t ev = nullptr, done = nullptr;
  CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
  CK(cudaEventRecord(ev, src->stream));
  CK(cudaStreamWaitEvent(dst->stream, ev, 0));
  const long long nc = (long long)dst->chi * dst->chi, nt = (long long)dst->chi * dst->D2 * dst->chi;
  for (int role = 0; role < 4; ++role)
    for (int i = 0; i < dst->Lx * dst->Ly; ++i) {
      CK(cudaMemcpyAsync(dst->C[role][i], src->C[role][i], nc * sizeof(cplx), cudaMemcpyDeviceToDevice,
                         dst->stream));
      CK(cudaMemcpyAsync(dst->T[role][i], src->T[role][i], nt * sizeof(cplx), cudaMemcpyDeviceToDevice,
                         dst->stream));
    }
  // src may be used (or destroyed) once its copies are done
  CK(cudaEventRecord(done, dst->stream));
  CK(cudaStreamWaitEvent(src->stream, done, 0));
  cudaEventDestroy(ev);  // released by the runtime once complete
  cudaEventDestroy(done);
  return IPEPS_OK;
}

// geometry for the checkpoint module: Lx, Ly, d, D, chi, n_tensors, pattern[4]
void ctm_geometry(ipeps_ctm h, int g[10]) {
  g[0] = h->Lx; g[1] = h->Ly; g[2] = h->d; g[3] = h->D; g[4] = h->chi; g[5] = h->ntens;
  for (int i = 0; i < 4; ++i) g[6 + i] = h->pattern[i];
}

// ---------------------------------------------------------------------------
// stand-alone complex GEMM (building block, host buffers) for unit tests
// ---------------------------------------------------------------------------
// prec code of ipeps_zgemm for the FP64-accurate tensor-core GEMM (ozaki.cu)
constexpr int ZGEMM_FP64_TC = IPEPS_PREC_FP64TC;

static ipeps_status zgemm_host(int prec, int M, int N, int K, const double* A, int opA, const double* B, int opB,
                               double* C, const TcChoice* force);

extern "C" ipeps_status ipeps_zgemm(int prec, int M, int N, int K, const double* A, int opA, const double* B,
                                    int opB, double* C) {
  return zgemm_host(prec, M, N, K, A, opA, B, opB, C, nullptr);
}

extern "C" ipeps_status ipeps_zgemm_tile(int prec, int bn, int splits, int M, int N, int K, const double* A, int opA,
                                         const double* B, int opB, double* C) {
  if (prec != IPEPS_PREC_TF32 && prec != IPEPS_PREC_BF16X3 && prec != IPEPS_PREC_BF16X6)
    return fail(IPEPS_EINVAL, "tile choice needs TF32/BF16X3/BF16X6");
  if ((bn != 128 && bn != 256) || splits < 1)
    return fail(IPEPS_EINVAL, "bad tile choice");
  const TcChoice c{bn, splits};
  return zgemm_host(prec, M, N, K, A, opA, B, opB, C, &c);
}

static ipeps_status zgemm_host(int prec, int M, int N, int K, const double* A, int opA, const double* B, int opB,
                               double* C, const TcChoice* force) {
  if (M <= 0 || N <= 0 || K <= 0 || !A || !B || !C) return fail(IPEPS_EINVAL, "bad GEMM arguments");
  if (prec < 0 || prec > ZGEMM_FP64_TC || opA < 0 || opA > 3 || opB < 0 || opB > 3)
    return fail(IPEPS_EINVAL, "bad prec/op");
  const size_t na = (size_t)M * K, nb = (size_t)K * N, nc = (size_t)M * N;
  size_t scratch_elems = 4 * (na + nb) + 8 * nc + (force ? 4 * (size_t)force->splits * (nc + 256 * (size_t)M) : 0) +
                         (1 << 20);
  if (prec == ZGEMM_FP64_TC) scratch_elems = oz_work_bytes(M, N, K) / sizeof(cplx) + 1024;
  cplx *dA = nullptr, *dB = nullptr, *dC = nullptr, *dS = nullptr;
  int* dT = nullptr;  // tensor-core wait timeouts of this call
  ipeps_status st = IPEPS_OK;
  auto cleanup = [&]() { cudaFree(dA); cudaFree(dB); cudaFree(dC); cudaFree(dS); cudaFree(dT); };
  cudaError_t e = dev_alloc((void**)&dT, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(dT, 0, sizeof(int));
  if (e == cudaSuccess) e = dev_alloc((void**)&dA, na * sizeof(cplx));
  if (e == cudaSuccess) e = dev_alloc((void**)&dB, nb * sizeof(cplx));
  if (e == cudaSuccess) e = dev_alloc((void**)&dC, nc * sizeof(cplx));
  if (e == cudaSuccess && prec) e = dev_alloc((void**)&dS, scratch_elems * sizeof(cplx));
  if (e == cudaSuccess) e = cudaMemcpy(dA, A, na * sizeof(cplx), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dB, B, nb * sizeof(cplx), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { cleanup(); return fail(IPEPS_ECUDA, "zgemm setup: %s", cudaGetErrorString(e)); }
  const long long lda = (opA & OP_T) ? M : K, ldb = (opB & OP_T) ? K : N;
  if (prec == 0) e = zgemm(0, M, N, K, ONE, dA, lda, opA, dB, ldb, opB, ZERO, dC, N);
  else if (prec == ZGEMM_FP64_TC) e = oz_zgemm(0, M, N, K, dA, lda, opA, dB, ldb, opB, dC, N, dS, scratch_elems * sizeof(cplx), dT);
  else e = tc_zgemm(0, prec, M, N, K, ONE, dA, lda, opA, dB, ldb, opB, dC, N, dS, (long long)scratch_elems, 0, dT,
                    nullptr, force);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(C, dC, nc * sizeof(cplx), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) st = fail(IPEPS_ECUDA, "zgemm: %s", cudaGetErrorString(e));
  if (st == IPEPS_OK && prec) {
    int n = 0;
    e = cudaMemcpy(&n, dT, sizeof n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) st = fail(IPEPS_ECUDA, "zgemm: %s", cudaGetErrorString(e));
    else if (n) st = fail(IPEPS_ETIMEOUT, "%d tensor-core GEMM waits timed out", n);
  }
  cleanup();
  return st;
}
