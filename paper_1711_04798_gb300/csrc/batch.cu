// Batched scan: many independent CTM instances (a phase-diagram scan of
// coupling points with uneven D and chi) advanced together.
//
// Every instance is an ordinary handle with its own device memory and its own
// stream.  A batch move is captured once per direction as one CUDA graph in
// which each instance is a branch forked from the batch stream (and, inside an
// instance, the two cuts of a column are two sub-branches), so a replay is a
// single graph launch that lets the GPU overlap the small contractions of all
// instances.  The tensor-core products of every distinct shape take the tile
// choice (n-tile width, K splits) that the autotuner measured for that shape.
#include <stdarg.h>
#include <stdio.h>

#include <string>
#include <vector>

#include "../../include/ipeps_ctm.h"
#include "ctm_internal.h"
#include "tc_gemm.h"

// internals of the single-instance handle (ctm_api.cu)
ipeps_status ctm_enqueue_move(ipeps_ctm h, int dir);
cudaStream_t ctm_stream(ipeps_ctm h);
ipeps_status ctm_reset_status(ipeps_ctm h);
ipeps_status ctm_check_status(ipeps_ctm h);
ipeps_status ctm_reinit_env(ipeps_ctm h);
void ctm_set_tuner(ipeps_ctm h, TcTuner* t);
void ctm_set_sequential_cuts(ipeps_ctm h, bool on);
void set_last_error_message(const char* msg);
void fidelity_from_kappa(const double k12[2], const double k11[2], const double k22[2], double* d_block,
                         double* d_spin);
void ctm_cell(ipeps_ctm h, int* Lx, int* Ly);

namespace {

ipeps_status bfail(ipeps_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_last_error_message(buf);
  return st;
}

}  // namespace

struct ipeps_batch_s {
  int n;
  std::vector<ipeps_ctm> inst;
  std::vector<cudaStream_t> streams;  // one per instance (owned)
  std::vector<cudaEvent_t> join;      // one per instance
  cudaStream_t origin;                // batch stream: graphs are launched here (owned)
  cudaEvent_t fork;
  cudaGraphExec_t exec[5];            // per ipeps_dir, captured on first use
  int kernels[5];                     // kernels inside each graph (launch accounting)
  TcTuner* tuner;
  uint64_t launches_at_create;
  int graphs;                         // number of captured graphs
};

static void batch_free(ipeps_batch b) {
  if (!b) return;
  if (b->origin) cudaStreamSynchronize(b->origin);
  for (int d = 0; d < 5; ++d)
    if (b->exec[d]) cudaGraphExecDestroy(b->exec[d]);
  for (ipeps_ctm h : b->inst) ipeps_ctm_destroy(h);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->join) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->origin) cudaStreamDestroy(b->origin);
  tc_tuner_destroy(b->tuner);
  delete b;
}

extern "C" ipeps_status ipeps_batch_create(int n, const ipeps_cell* cells, const ipeps_options* opts, int tune,
                                           ipeps_batch* out) {
  if (n <= 0 || !cells || !opts || !out) return bfail(IPEPS_EINVAL, "batch: bad arguments");
  ipeps_batch b = new ipeps_batch_s();
  b->n = n;
  b->origin = nullptr;
  b->fork = nullptr;
  for (int d = 0; d < 5; ++d) {
    b->exec[d] = nullptr;
    b->kernels[d] = 0;
  }
  b->tuner = nullptr;
  b->graphs = 0;
  b->launches_at_create = launch_counter();
  auto cuda_fail = [&](cudaError_t e, const char* what) {
    batch_free(b);
    return bfail(IPEPS_ECUDA, "batch: %s: %s", what, cudaGetErrorString(e));
  };
  cudaError_t e;
  if ((e = kernels_init()) != cudaSuccess) return cuda_fail(e, "kernel limits");
  if ((e = tc_init()) != cudaSuccess) return cuda_fail(e, "tensor-core setup");
  if ((e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(e, "stream");
  if ((e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(e, "event");
  b->tuner = tc_tuner_create();
  if (!b->tuner) {
    batch_free(b);
    return bfail(IPEPS_ECUDA, "batch: tuner events");
  }
  for (int i = 0; i < n; ++i) {
    cudaStream_t s;
    cudaEvent_t j;
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e, "stream");
    b->streams.push_back(s);
    if ((e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(e, "event");
    b->join.push_back(j);
    ipeps_options o = opts[i];
    o.stream = s;
    o.workspace = nullptr;
    o.workspace_bytes = 0;
    ipeps_ctm h = nullptr;
    ipeps_status st = ipeps_ctm_create(&cells[i], &o, &h);
    if (st != IPEPS_OK) {
      std::string msg = std::string("batch instance ") + std::to_string(i) + ": " + ipeps_last_error();
      batch_free(b);
      set_last_error_message(msg.c_str());
      return st;
    }
    ctm_set_tuner(h, b->tuner);
    b->inst.push_back(h);
  }
  if (tune) {
    // one sweep per instance, cuts in sequence so that timings are not
    // perturbed by a concurrent lane; then back to the trace initialisation
    tc_tuner_set_measuring(b->tuner, true);
    for (int i = 0; i < n; ++i) {
      ipeps_ctm h = b->inst[i];
      ctm_set_sequential_cuts(h, true);
      ipeps_status st = ctm_reset_status(h);
      if (st == IPEPS_OK) st = ctm_enqueue_move(h, IPEPS_SWEEP);
      if (st == IPEPS_OK) st = ctm_check_status(h);
      if (st == IPEPS_OK) st = ctm_reset_status(h);
      if (st == IPEPS_OK) st = ctm_reinit_env(h);
      if (st == IPEPS_OK) st = ctm_check_status(h);
      ctm_set_sequential_cuts(h, false);
      if (st != IPEPS_OK) {
        std::string msg = std::string("batch tuning, instance ") + std::to_string(i) + ": " + ipeps_last_error();
        batch_free(b);
        set_last_error_message(msg.c_str());
        return st;
      }
    }
    tc_tuner_set_measuring(b->tuner, false);
  }
  *out = b;
  return IPEPS_OK;
}

// Capture one graph of `dir` over all instances.
static ipeps_status capture(ipeps_batch b, int dir) {
  cudaGraph_t g = nullptr;
  const uint64_t l0 = launch_counter();
  cudaError_t e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return bfail(IPEPS_ECUDA, "batch: begin capture: %s", cudaGetErrorString(e));
  ipeps_status st = IPEPS_OK;
  e = cudaEventRecord(b->fork, b->origin);
  for (int i = 0; i < b->n && e == cudaSuccess && st == IPEPS_OK; ++i) {
    e = cudaStreamWaitEvent(b->streams[i], b->fork, 0);
    if (e != cudaSuccess) break;
    st = ctm_enqueue_move(b->inst[i], dir);
    if (st != IPEPS_OK) break;
    e = cudaEventRecord(b->join[i], b->streams[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, b->join[i], 0);
  }
  cudaError_t e2 = cudaStreamEndCapture(b->origin, &g);
  // captured launches did not run: they are counted at each replay instead
  b->kernels[dir] = (int)(launch_counter() - l0);
  count_launch(-b->kernels[dir]);
  if (st != IPEPS_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return bfail(IPEPS_ECUDA, "batch: capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(&b->exec[dir], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    b->exec[dir] = nullptr;
    return bfail(IPEPS_ECUDA, "batch: instantiate: %s", cudaGetErrorString(e));
  }
  ++b->graphs;
  return IPEPS_OK;
}

extern "C" ipeps_status ipeps_batch_move(ipeps_batch b, int dir, int count) {
  if (!b) return bfail(IPEPS_EINVAL, "null batch");
  if (dir < 0 || dir > 4 || count < 0) return bfail(IPEPS_EINVAL, "bad dir/count");
  if (count == 0) return IPEPS_OK;
  // status words cleared before the replays (ordered: same instance streams)
  for (ipeps_ctm h : b->inst) {
    ipeps_status st = ctm_reset_status(h);
    if (st != IPEPS_OK) return st;
  }
  cudaError_t e;
  for (int i = 0; i < b->n; ++i) {
    if ((e = cudaEventRecord(b->join[i], b->streams[i])) != cudaSuccess ||
        (e = cudaStreamWaitEvent(b->origin, b->join[i], 0)) != cudaSuccess)
      return bfail(IPEPS_ECUDA, "batch: ordering: %s", cudaGetErrorString(e));
  }
  if (!b->exec[dir]) {
    ipeps_status st = capture(b, dir);
    if (st != IPEPS_OK) return st;
  }
  for (int c = 0; c < count; ++c) {
    if ((e = cudaGraphLaunch(b->exec[dir], b->origin)) != cudaSuccess)
      return bfail(IPEPS_ECUDA, "batch: graph launch: %s", cudaGetErrorString(e));
    count_launch(b->kernels[dir]);
  }
  // instance streams wait for the replays before any later per-instance work
  if ((e = cudaEventRecord(b->fork, b->origin)) != cudaSuccess)
    return bfail(IPEPS_ECUDA, "batch: ordering: %s", cudaGetErrorString(e));
  for (int i = 0; i < b->n; ++i)
    if ((e = cudaStreamWaitEvent(b->streams[i], b->fork, 0)) != cudaSuccess)
      return bfail(IPEPS_ECUDA, "batch: ordering: %s", cudaGetErrorString(e));
  ipeps_status worst = IPEPS_OK;
  std::string msg;
  for (int i = 0; i < b->n; ++i) {
    ipeps_status st = ctm_check_status(b->inst[i]);
    if (st != IPEPS_OK && worst == IPEPS_OK) {
      worst = st;
      msg = std::string("batch instance ") + std::to_string(i) + ": " + ipeps_last_error();
    }
  }
  if (worst != IPEPS_OK) set_last_error_message(msg.c_str());
  return worst;
}

extern "C" ipeps_status ipeps_batch_energy(ipeps_batch b, const double* J, double* e_out) {
  if (!b || !J || !e_out) return bfail(IPEPS_EINVAL, "batch energy: null argument");
  for (int i = 0; i < b->n; ++i) {
    ipeps_status st = ipeps_energy(b->inst[i], J + 3 * i, e_out + i);
    if (st != IPEPS_OK) return st;
  }
  return IPEPS_OK;
}

// Fidelity surface (Sec. VI): kappa of every instance the pairs name, each
// computed once, then the fidelity per site of each pair.
extern "C" ipeps_status ipeps_batch_fidelity(ipeps_batch b, int n_pairs, const int* i12, const int* i11,
                                             const int* i22, double* d_block, double* d_spin) {
  if (!b || n_pairs < 0 || (n_pairs && (!i12 || !i11 || !i22 || !d_block)))
    return bfail(IPEPS_EINVAL, "batch fidelity: bad arguments");
  std::vector<int> need(b->n, 0);
  for (int p = 0; p < n_pairs; ++p) {
    const int idx[3] = {i12[p], i11[p], i22[p]};
    for (int q = 0; q < 3; ++q) {
      if (idx[q] < 0 || idx[q] >= b->n) return bfail(IPEPS_EINVAL, "batch fidelity: pair %d names instance %d", p, idx[q]);
      need[idx[q]] = 1;
    }
    int lx[3], ly[3];
    for (int q = 0; q < 3; ++q) ctm_cell(b->inst[idx[q]], &lx[q], &ly[q]);
    if (lx[0] != lx[1] || lx[0] != lx[2] || ly[0] != ly[1] || ly[0] != ly[2])
      return bfail(IPEPS_EINVAL, "batch fidelity: pair %d: cells differ", p);
  }
  std::vector<double> k(2 * (size_t)b->n, 0.0);
  for (int i = 0; i < b->n; ++i) {
    if (!need[i]) continue;
    const ipeps_status st = ipeps_kappa(b->inst[i], &k[2 * i]);
    if (st != IPEPS_OK) {
      const std::string msg = std::string("batch instance ") + std::to_string(i) + ": " + ipeps_last_error();
      set_last_error_message(msg.c_str());
      return st;
    }
  }
  for (int p = 0; p < n_pairs; ++p)
    fidelity_from_kappa(&k[2 * i12[p]], &k[2 * i11[p]], &k[2 * i22[p]], d_block + p, d_spin ? d_spin + p : nullptr);
  return IPEPS_OK;
}

extern "C" ipeps_ctm ipeps_batch_instance(ipeps_batch b, int i) {
  if (!b || i < 0 || i >= b->n) return nullptr;
  return b->inst[i];
}

extern "C" int ipeps_batch_tuning_size(ipeps_batch b) { return b ? tc_tuner_size(b->tuner) : 0; }

extern "C" ipeps_status ipeps_batch_tuning_entry(ipeps_batch b, int i, int fields[6], double us[2]) {
  if (!b || !fields || !us) return bfail(IPEPS_EINVAL, "batch tuning: null argument");
  if (!tc_tuner_entry(b->tuner, i, fields, us)) return bfail(IPEPS_EINVAL, "batch tuning: no entry %d", i);
  return IPEPS_OK;
}

extern "C" uint64_t ipeps_batch_launch_count(ipeps_batch b) {
  return b ? launch_counter() - b->launches_at_create : 0;
}

extern "C" ipeps_status ipeps_batch_sync(ipeps_batch b) {
  if (!b) return bfail(IPEPS_EINVAL, "null batch");
  cudaError_t e = cudaStreamSynchronize(b->origin);
  for (int i = 0; i < b->n && e == cudaSuccess; ++i) e = cudaStreamSynchronize(b->streams[i]);
  if (e != cudaSuccess) return bfail(IPEPS_ECUDA, "batch sync: %s", cudaGetErrorString(e));
  return IPEPS_OK;
}

extern "C" void* ipeps_batch_stream(ipeps_batch b) { return b ? (void*)b->origin : nullptr; }

extern "C" void ipeps_batch_destroy(ipeps_batch b) { batch_free(b); }
