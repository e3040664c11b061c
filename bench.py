"""Benchmark of the CTM hot path on GB300.

One step = rebuild of the double layers (Fig. 3a) + one CTM sweep (moves L,
R, U, D: enlarged corners, projectors, renormalisation, normalisation) + the
eight nearest-neighbour RDMs and the ruby energy, on the D=5, chi=100, 2x2
complex workload.  value = CTM moves per second over the whole job
(4 moves per step and rank).  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "CTM moves/s & TFLOP/s at D=5 χ=100: mixed-prec/batched vs FP64, |ΔE|≤1e-6"
MOVES_PER_STEP = 4


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=4)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--prec", default="bf16x6", choices=["fp64", "tf32", "bf16x3", "bf16x6", "fp64tc"])
    p.add_argument("--no-fp64-check", action="store_true",
                   help="skip the FP64 comparison run (moves/s and |dE| of the plain FP64 GPU path)")
    p.add_argument("--D", type=int, default=5)
    p.add_argument("--chi", type=int, default=100)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--workload", default="single", choices=["single", "scan", "cylinder", "fidelity"],
                   help="single: one D=5 chi=100 instance; scan: 64-instance batched phase-diagram scan; "
                        "cylinder: D=6 chi=144 environment, boundary spectrum at Nv = 2, 4, 6; "
                        "fidelity: fidelity surface of a coupling line on the batch engine")
    p.add_argument("--points", type=int, default=8, help="fidelity: points on the coupling line")
    p.add_argument("--sweeps", type=int, default=12, help="cylinder: CTM sweeps before the readout")
    p.add_argument("--topk", type=int, default=64, help="cylinder: leading eigenvalues at Nv = 6")
    p.add_argument("--instances", type=int, default=64)
    p.add_argument("--no-tune", action="store_true")
    return p.parse_args()


def workload(D, chi, seed):
    import synth
    return synth.workload("product_noise", seed=seed, D=D, chi=chi)


def config_desc(args, prec):
    return {
        "workload": f"2x2 ruby block-site cell, d=8, D={args.D}, chi={args.chi}, complex product state "
                    f"+ 0.1 complex-normal noise, rSVD projectors k=chi+16, q=2",
        "step": "double-layer rebuild + 1 sweep (L,R,U,D) + 8 bond RDMs + energy",
        "prec": prec,
        "cell": "2x2",
        "l2": "working set > L2 (four enlarged corners of (chi D^2)^2 complex128 = 400 MB)",
    }


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            return json.load(open(path)), "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def zgemm_peak_tflops(torch):
    """Complex128 GEMM throughput of cuBLAS on this GPU (FP64 reference peak)."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.complex128, device="cuda")
    b = torch.randn(n, n, dtype=torch.complex128, device="cuda")
    best = 0.0
    for _ in range(4):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        a @ b
        e1.record()
        torch.cuda.synchronize()
        best = max(best, 8.0 * n ** 3 / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    del a, b
    return best


def oracle_move_seconds(D, chi, n_moves=1):
    """The oracle as it stands: one left move of the same workload on the host cores."""
    import oracle as O
    import synth
    w = workload(D, chi, 0)
    st = O.make_state(w["tensors"], w["pattern"], D, chi)
    K, k = chi * D * D, chi + 16
    opt = O.CTMOptions(chi=chi, proj="rsvd", omega=synth.omega(7, K, k))
    t0 = time.perf_counter()
    for _ in range(n_moves):
        st = O.move(st, "L", opt)
    return (time.perf_counter() - t0) / n_moves


def oracle_column_seconds_one_thread(D, chi):
    """The oracle on one host thread (BLAS thread pools pinned to one in a
    fresh interpreter): one column of a left move of the same workload (its
    two cuts' corners and projectors and their absorption), half a move."""
    code = (
        "import sys, time\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "import bench, oracle as O, synth\n"
        f"D, chi = {int(D)}, {int(chi)}\n"
        "w = bench.workload(D, chi, 0)\n"
        "st = O.make_state(w['tensors'], w['pattern'], D, chi)\n"
        "K, k = chi * D * D, chi + 16\n"
        "opt = O.CTMOptions(chi=chi, proj='rsvd', omega=synth.omega(7, K, k))\n"
        "t0 = time.perf_counter()\n"
        "O.left_move(st, opt, columns=[0])\n"
        "print(time.perf_counter() - t0)\n")
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-400:])
    return float(out.stdout.strip().splitlines()[-1])


# ---------------------------------------------------------------------------
# multi-rank bookkeeping (replicas: one independent instance per rank, no
# collective on the data path; only the timing is reduced)
# ---------------------------------------------------------------------------
def init_dist(world):
    """torch.distributed for world > 1: NCCL with GPUs, else gloo (CPU tests)."""
    if world <= 1:
        return None
    import torch
    import torch.distributed as dist
    dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return dist


def max_over_ranks(x, dist):
    """Largest value of x over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world, seconds_max):
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * units_per_rank / seconds_max


def rank_seed(rank):
    """Workload seed of a replica: each rank contracts its own synthetic state."""
    return rank


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def run_reference(args, rank, world):
    if rank != 0:
        return
    secs = []
    for i in range(args.warmup + args.steps):
        t = oracle_move_seconds(args.D, args.chi)
        if i >= args.warmup:
            secs.append(t)
    mean = sum(secs) / len(secs)
    v = 1.0 / mean
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "moves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_desc(args, "fp64 numpy oracle"),
        "cpu_baseline": {"value": v, "unit": "moves/s", "cores": host_cores(), "kind": "oracle",
                         "sample": "one left move (of the 4 per sweep) per step, numpy/LAPACK FP64"},
        "e2e": {"value": v, "unit": "moves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


GOLDEN = os.path.join(ROOT, "tests", "golden")
PASSES = {"fp64": 1, "tf32": 1, "bf16x3": 3, "bf16x6": 6, "fp64tc": 28}  # tensor-core products per product
DTYPE = {"fp64": "f64", "tf32": "tf32", "bf16x3": "bf16x3", "bf16x6": "bf16x6", "fp64tc": "f64"}


def stored_oracle(D, chi, seed, cutoff):
    """The FP64 oracle's converged state of this workload, when tests/golden
    holds it (written by tests/golden/make_golden.py from oracle/ alone)."""
    name = {(5, 100, 0, 1e-6): "product_noise_D5_chi100_cut6"}.get((D, chi, seed, cutoff))
    path = os.path.join(GOLDEN, f"{name}.npz") if name else None
    if not path or not os.path.exists(path):
        return None
    with np.load(path) as z:
        return {k: z[k] for k in z.files} if "E_conv" in z.files else None


def kernel_classes(g, prec, ms_step, steps, peaks, peak_src, zpk):
    """Per-class roofline records from one profiled pass (library CUDA events
    on the stream each kernel runs on)."""
    classes = []
    rd = {k: g.profile_read(k) for k in (1, 2, 5, 6, 7, 8)}
    bf16 = peaks.get("bf16_tflops_sustained", 1700.0)
    hbm = peaks.get("hbm_gbs", 6800.0)
    zsrc = "cuBLAS complex128 GEMM measured in this run (no FP64 entry in the peaks file)"
    if prec == "fp64":
        c0 = g.profile_read(0)
        classes.append({"kernel": "zgemm_kernel (complex FP64 GEMM, CUDA cores): contractions", "bound": "alu",
                        "ms": c0["ms"], "work": c0["flops"] / 1e12, "launches": c0["launches"], "peak": zpk,
                        "unit": "TFLOP/s", "peak_source": zsrc})
    elif prec == "fp64tc":
        c0 = g.profile_read(0)
        classes.append({"kernel": "oz_gemm_kernel with its digit preparation and exact reduction (FP64-accurate "
                                  "digit-split products on tcgen05): contractions, range finder, readouts",
                        "bound": "tensor", "ms": c0["ms"], "work": c0["flops"] * PASSES[prec] / 1e12,
                        "launches": c0["launches"], "peak": bf16, "unit": "TFLOP/s",
                        "peak_source": f"bf16 dense sustained ({peak_src}); executed flops = 8MNK algorithmic x 28 "
                                       "digit-plane products (tile padding not counted)",
                        "fp64_equivalent_tflops": c0["flops"] / (c0["ms"] * 1e-3) / 1e12 if c0["ms"] else None})
    else:
        npass = PASSES[prec]
        # a contraction takes the peak of its own dtype: BF16 dense (measured); TF32 at half of it
        pk = bf16 if prec != "tf32" else bf16 / 2.0
        classes.append({"kernel": f"tc_gemm_kernel (tcgen05 {prec}), wide products: enlarged corners, absorption, "
                                  "readouts", "bound": "tensor", "ms": rd[5]["ms"],
                        "work": rd[5]["flops"] * npass / 1e12, "launches": rd[5]["launches"], "peak": pk,
                        "unit": "TFLOP/s",
                        "peak_source": f"bf16 dense sustained ({peak_src}){' x 1/2 for TF32' if prec == 'tf32' else ''};"
                                       f" executed flops = 8MNK algorithmic x {npass} products"})
        classes.append({"kernel": f"tc_gemm_kernel (tcgen05 {prec}), thin products: range finder and projector "
                                  "assembly", "bound": "hbm", "ms": rd[7]["ms"], "work": rd[7]["flops"] / 1e9,
                        "launches": rd[7]["launches"], "peak": hbm, "unit": "GB/s",
                        "peak_source": f"HBM copy ({peak_src}); bytes = packed operands read once + output written",
                        "algorithmic_tflops": rd[6]["flops"] / (rd[6]["ms"] * 1e-3) / 1e12 if rd[6]["ms"] else None})
        classes.append({"kernel": "splitk_reduce_kernel (FP32 partial sums)", "bound": "hbm", "ms": rd[8]["ms"],
                        "work": rd[8]["flops"] / 1e9, "launches": rd[8]["launches"], "peak": hbm, "unit": "GB/s",
                        "peak_source": f"HBM copy ({peak_src})"})
    if prec != "fp64":
        classes.append({"kernel": "oz_gemm_kernel with its digit preparation and exact reduction (FP64-accurate "
                                  "digit-split products on tcgen05): CholeskyQR Grams/applies and core products "
                                  "of the projectors",
                        "bound": "latency", "ms": rd[2]["ms"], "work": rd[2]["flops"] / 1e12,
                        "launches": rd[2]["launches"], "peak": zpk, "unit": "TFLOP/s",
                        "peak_source": zsrc + "; the FP64-pipe rate these products replace (frac > 1: faster than "
                                              "that pipe can run them); algorithmic FP64 flops"})
    classes.append({"kernel": "Jacobi SVD kernels (FP64, projector cores and orthonormalisation)", "bound": "alu",
                    "ms": rd[1]["ms"], "work": None, "launches": rd[1]["launches"], "peak": None, "unit": None,
                    "peak_source": "latency-bound FP64 rotations; mean sweeps per call "
                                   f"{rd[1]['flops']:.2f}", "mean_sweeps_per_call": rd[1]["flops"]})
    for c in classes:
        c["achieved"] = c["work"] / (c["ms"] * 1e-3) if c["ms"] and c["work"] else None
        c["frac"] = c["achieved"] / c["peak"] if c["achieved"] and c["peak"] else None
        c["share_of_step"] = c["ms"] / (ms_step * steps) if ms_step else None
        c["ms_per_launch"] = c["ms"] / c["launches"] if c["launches"] else None
    return classes


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1711_04798_gb300 import CTM
    torch.cuda.set_device(local_rank)
    dist = init_dist(world)
    stream = torch.cuda.current_stream()
    w = workload(args.D, args.chi, seed=rank_seed(rank))
    J = w["J"]
    g = CTM(w["tensors"], w["pattern"], args.chi, prec=args.prec, stream=stream.cuda_stream)
    tuned = 0 if args.no_tune else g.autotune()

    def step():
        g.rebuild()
        g.sweep(1)
        return g.energy(J)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    l0 = g.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        energies = [step() for _ in range(args.steps)]
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = g.launch_count() - l0
    ms_max = max_over_ranks(ms, dist)
    value = job_value(args.steps * MOVES_PER_STEP, world, ms_max * 1e-3)

    # the step's parts in a separate pass of the same handle (CUDA events on
    # the stream): the sweep of four moves and the bond readout with the energy
    def part_ms(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(args.steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / args.steps

    breakdown = {"sweep_ms": part_ms(lambda: g.sweep(1)), "readout_ms": part_ms(lambda: g.energy(J)),
                 "rebuild_ms": part_ms(g.rebuild)}
    breakdown["sweep_moves_per_s"] = MOVES_PER_STEP / (breakdown["sweep_ms"] * 1e-3)

    # end to end through the public API: host tensors in, energy out, every step
    host_tensors = w["tensors"]
    h2d = sum(a.nbytes for a in host_tensors)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        g.set_tensors(host_tensors)
        g.sweep(1)
        g.energy(J)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value = job_value(args.steps * MOVES_PER_STEP, world, max_over_ranks(e2e_s, dist))

    if rank != 0:
        g.close()
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    # profiled pass (the same steps, kernels launched one by one and bracketed
    # by the library's CUDA events): per-class times for the roofline
    g.profile(True)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(args.steps):
        step()
    p1.record(stream)
    torch.cuda.synchronize()
    ms_prof = p0.elapsed_time(p1) / args.steps
    peaks, peak_src = measured_peaks()
    zpk = zgemm_peak_tflops(torch)
    classes = kernel_classes(g, args.prec, ms_prof, args.steps, peaks, peak_src, zpk)
    g.profile(False)
    timed = [c for c in classes if c["achieved"]]
    dom = max(timed, key=lambda c: c["ms"])
    roof = {"bound": dom["bound"], "achieved": dom["achieved"], "peak": dom["peak"], "unit": dom["unit"],
            "frac": dom["frac"], "traffic": TRAFFIC.get((args.prec, dom["bound"])), "kernel": dom["kernel"],
            "peak_source": dom["peak_source"],
            "dominant_by": "CUDA-event time per kernel class in a profiled pass of the same steps "
                           f"({ms_prof:.1f} ms per step with per-launch events, vs {ms_max / args.steps:.1f} ms "
                           "as CUDA graphs)",
            "by_class": [{k: c[k] for k in ("kernel", "bound", "achieved", "peak", "unit", "frac", "share_of_step",
                                            "launches", "ms_per_launch", "mean_sweeps_per_call", "fp64_equivalent_tflops",
                                            "algorithmic_tflops") if k in c}
                         for c in classes]}
    fp64_cmp = None
    if args.prec != "fp64" and not args.no_fp64_check:
        fp64_cmp = fp64_comparison(args, w, J, stream, torch, value)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        secs = oracle_move_seconds(args.D, args.chi)
        cpu = {"value": 1.0 / secs, "unit": "moves/s", "cores": host_cores(), "kind": "oracle",
               "sample": "one left move of the same workload (numpy/LAPACK FP64, all host cores)"}
        col = oracle_column_seconds_one_thread(args.D, args.chi)
        cpu["one_thread"] = {"value": 1.0 / (2.0 * col), "unit": "moves/s", "cores": 1,
                             "sample": "one column of a left move (half a move) on one thread, "
                                       "BLAS thread pools pinned to one"}
    line = {
        "metric": METRIC, "value": value, "unit": "moves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[args.prec],
        "data": "synthetic", "config": config_desc(args, args.prec),
        "tflops": MOVES_PER_STEP * flops_per_move(args.D, args.chi) / (ms_max / args.steps * 1e-3) / 1e12,
        "autotuned_shapes": tuned,
        "energy_per_spin": energies[-1],
        "roofline": roof, "cpu_baseline": cpu, "fp64_comparison": fp64_cmp,
        "e2e": {"value": e2e_value, "unit": "moves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 8},
        "gpu_launches": launches, "host_graph_launches_per_step": MOVES_PER_STEP // 4,
        "step_breakdown": breakdown,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    g.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


# DRAM bytes per launch of the dominant class from one ncu capture of the
# current kernel (the mean of the wide-product launches in the profile summary
# of the default workload), keyed by (precision, bound); absent where no
# capture of the current kernel exists
TRAFFIC = {("bf16x6", "tensor"): 93.6e6}


def flops_per_move(D, chi, q=2, over=16):
    """Algorithmic real flops of one move (the survey's count: 16 enlarged
    corners, the range finder and projector assembly of four cuts, and the
    absorption of two columns; complex = 8 real flops per multiply-add)."""
    D2, N, k = D * D, chi * D * D, chi + over
    Q = chi ** 3 * D2 + chi ** 3 * D2 ** 2 + chi ** 2 * D2 ** 4
    return 8.0 * (16 * Q + 4 * ((2 * q + 2) * 4 * N * N * k + 2 * N * N * chi) + 8 * 2 * chi ** 3 * D2
                  + 4 * (2 * chi ** 3 * D2 ** 2 + chi ** 2 * D2 ** 4))


def fp64_comparison(args, w, J, stream, torch, value):
    """The precision form against FP64: the plain FP64 GPU path's speed over one
    sweep, and -- where the stored oracle record of this workload exists --
    the converged precision-form energy, RDMs and corner spectra against the
    FP64 oracle's converged values at the same truncation cutoff."""
    from paper_1711_04798_gb300 import CTM
    gf = CTM(w["tensors"], w["pattern"], args.chi, prec="fp64", stream=stream.cuda_stream)
    gf.sweep(1)  # capture
    gf.reset_env()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    gf.sweep(1)
    f1.record(stream)
    torch.cuda.synchronize()
    out = {"fp64_moves_per_s": 4 / (f0.elapsed_time(f1) * 1e-3)}
    out["speedup_vs_fp64"] = value / out["fp64_moves_per_s"]
    gf.close()
    # the FP64-accurate tensor-core form (FP64 results, digit-split products)
    gt = CTM(w["tensors"], w["pattern"], args.chi, prec="fp64tc", stream=stream.cuda_stream)
    gt.sweep(1)
    gt.reset_env()
    torch.cuda.synchronize()
    f0.record(stream)
    gt.sweep(1)
    f1.record(stream)
    torch.cuda.synchronize()
    out["fp64tc_moves_per_s"] = 4 / (f0.elapsed_time(f1) * 1e-3)
    out["fp64tc_vs_fp64"] = out["fp64tc_moves_per_s"] / out["fp64_moves_per_s"]
    gt.close()
    cut = 1e-6
    ref = stored_oracle(args.D, args.chi, 0, cut) if rank_seed(0) == 0 else None
    if ref is None:
        out["converged"] = None
        return out
    gm = CTM(w["tensors"], w["pattern"], args.chi, prec=args.prec, cutoff=cut, stream=stream.cuda_stream)
    n, delta, ok = gm.converge(1e-8, 40)
    r = gm.rdms()
    e = gm.energy(J)
    s = gm.spectra()
    sref = ref["spectra_conv"]
    mask = sref > 1e-5

    def errors(e, r, s):
        return {"abs_dE": abs(e - float(ref["E_conv"])),
                "max_abs_drho": float(max(np.max(np.abs(r["h"] - ref["rho_h_conv"])),
                                          np.max(np.abs(r["v"] - ref["rho_v_conv"])))),
                "max_spectrum_err": float(np.max(np.abs(s - sref)[mask]))}

    # polish: FP64-accurate tensor-core sweeps from the precision form's environment
    gp = CTM(w["tensors"], w["pattern"], args.chi, prec="fp64tc", cutoff=cut, stream=stream.cuda_stream)
    gp.copy_env_from(gm)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n2, delta2, ok2 = gp.converge(1e-10, 30)
    torch.cuda.synchronize()
    t_pol = time.perf_counter() - t0
    polished = {"form": "FP64-accurate tensor-core sweeps (fp64tc) started from the precision form's converged "
                        "environment, to 1e-10 in the corner spectra",
                "sweeps": n2, "delta": delta2, "converged_to_1e-10": ok2, "seconds": t_pol}
    polished.update(errors(gp.energy(J), gp.rdms(), gp.spectra()))
    gp.close()
    out["converged"] = {
        "reference": "FP64 oracle (exact truncated SVD), converged to 1e-10 in the corner spectra, cutoff 1e-6, "
                     f"{int(ref['sweeps'])} sweeps; stored by tests/golden/make_golden.py",
        "sweeps": n, "delta": delta, "converged_to_1e-8": ok, "cutoff": cut,
        "energy": e, "energy_oracle": float(ref["E_conv"]),
        **errors(e, r, s),
        "targets": {"abs_dE": 1e-6, "max_abs_drho": 1e-6, "max_spectrum_err": 1e-5},
        "polished": polished,
    }
    gm.close()
    return out


SCAN_DESC = ("batched scan: {n} independent instances on the line Jx=Jy=(2-Jz)/2, Jz_k=2k/{n1}; "
             "D_k in {{3,4,5}} and chi_k in {{32,48,64,100}} round-robin (r = seed mod 12); 2x2 cell, d=8, "
             "complex product state + 0.1 complex-normal noise per instance")


def run_scan(args, rank, world, local_rank):
    """Batched scan: every instance advanced by one graph launch per sweep."""
    import torch
    import synth
    from paper_1711_04798_gb300 import Batch, CTM
    torch.cuda.set_device(local_rank)
    dist = init_dist(world)
    insts = synth.scan(seed=rank_seed(rank), n=args.instances)
    t0 = time.perf_counter()
    b = Batch(insts, tune=not args.no_tune, prec=args.prec)
    create_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    b.sweep(1)  # captures the sweep graph
    capture_s = time.perf_counter() - t0
    for _ in range(max(args.warmup - 1, 0)):
        b.sweep(1)
    s = torch.cuda.ExternalStream(b.stream())
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    l0 = b.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        e0.record(s)
        for _ in range(args.steps):
            b.sweep(1)
        e1.record(s)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = b.launch_count() - l0
    ms_max = max_over_ranks(ms, dist)
    n = len(insts)
    value = job_value(n * MOVES_PER_STEP * args.steps, world, ms_max * 1e-3)
    energies = b.energies([i["J"] for i in insts])
    tuning = b.tuning()
    b.close()
    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    # one representative per (D, chi) class, one sweep each, run alone:
    # sequential estimates for the same precision and for the plain FP64 path
    classes = {}
    for i in insts:
        classes.setdefault((i["D"], i["chi"]), []).append(i)
    stream = torch.cuda.current_stream()
    seq_prec = seq_fp64 = 0.0
    dE = 0.0
    per_class = []
    for (D, chi), members in sorted(classes.items()):
        rep = members[0]
        times, es = {}, {}
        for prec in (args.prec, "fp64"):
            # the same truncation cutoff on both sides (the precision form's)
            g = CTM(rep["tensors"], rep["pattern"], chi, prec=prec, cutoff=1e-6, stream=stream.cuda_stream)
            torch.cuda.synchronize()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            g.sweep(1)
            f1.record(stream)
            torch.cuda.synchronize()
            times[prec] = f0.elapsed_time(f1) * 1e-3
            es[prec] = g.energy(rep["J"])
            g.close()
        seq_prec += len(members) * times[args.prec]
        seq_fp64 += len(members) * times["fp64"]
        dE = max(dE, abs(es[args.prec] - es["fp64"]))
        per_class.append({"D": D, "chi": chi, "count": len(members), "sweep_s_" + args.prec: times[args.prec],
                          "sweep_s_fp64": times["fp64"], "abs_dE_1sweep": abs(es[args.prec] - es["fp64"])})
    seq_prec_rate = n * MOVES_PER_STEP / seq_prec
    seq_fp64_rate = n * MOVES_PER_STEP / seq_fp64
    line = {
        "metric": METRIC, "value": value, "unit": "instance-moves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.prec],
        "data": "synthetic",
        "config": {"workload": SCAN_DESC.format(n=n, n1=n - 1), "step": "one sweep (L,R,U,D) of every instance",
                   "prec": args.prec, "autotune": not args.no_tune,
                   "l2": "working set > L2 (the enlarged corners of all instances, tens of GB)"},
        "scan": {"instances": n, "create_s": create_s, "first_sweep_with_capture_s": capture_s,
                 "tuned_shapes": len(tuning),
                 "tuned_speedup_vs_default": (sum(t["default_us"] for t in tuning) / sum(t["us"] for t in tuning))
                 if tuning else None,
                 "sequential_same_prec_inst_moves_per_s": seq_prec_rate,
                 "sequential_fp64_inst_moves_per_s": seq_fp64_rate,
                 "speedup_vs_sequential_same_prec": value / seq_prec_rate,
                 "speedup_vs_sequential_fp64": value / seq_fp64_rate,
                 "max_abs_dE_vs_fp64_one_sweep": dE, "classes": per_class,
                 "energy_range": [float(min(energies)), float(max(energies))]},
        "gpu_launches": launches, "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_cylinder(args, rank, world, local_rank):
    """Long-cylinder readout: environment at D=6 chi=144, boundary spectrum and
    entanglement entropy on cylinders of Nv = 2, 4 (dense) and 6 (Lanczos)."""
    import torch
    import synth
    from paper_1711_04798_gb300 import CTM
    torch.cuda.set_device(local_rank)
    D = args.D if args.D != 5 else 6
    chi = args.chi if args.chi != 100 else 144
    w = synth.workload("product_noise", seed=rank_seed(rank), D=D, chi=chi)
    stream = torch.cuda.current_stream()
    g = CTM(w["tensors"], w["pattern"], chi, prec=args.prec, stream=stream.cuda_stream)

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1) * 1e-3

    g.sweep(1)  # warm-up
    with ClockSampler(local_rank) as clk:
        _, ctm_s = timed(lambda: g.sweep(args.sweeps))
        spectra = g.spectra()
        readouts = []
        for Nv in (2, 4):
            (lam, S), t = timed(lambda: g.boundary_rho(0, Nv))
            readouts.append({"Nv": Nv, "route": "dense", "dim": int(D ** Nv), "S_vn": S, "seconds": t,
                             "lam_top4": [float(v) for v in lam[:4]]})
        Nv = 6
        k = min(args.topk, D ** Nv)
        g.profile(True)
        (lam, S, rest, nconv), t = timed(lambda: g.boundary_rho_topk(0, Nv, k, max_iter=min(8 * k, 1024),
                                                                     tol=1e-8))
        ring, lz = g.profile_read(3), g.profile_read(4)
        g.profile(False)
        (S2, purity), t2 = timed(lambda: g.boundary_renyi2(0, Nv))
        readouts.append({"Nv": Nv, "route": "renyi2 from traces of the dense product sigma_L^T sigma_R",
                         "S_renyi2": S2, "purity": purity, "seconds": t2})
        readouts.append({"Nv": Nv, "route": "lanczos", "dim": int(D ** Nv), "k": k, "converged": nconv,
                         "S_vn_topk": S, "rest_weight": rest, "seconds": t,
                         "ring_build_s": ring["ms"] * 1e-3,
                         "ring_products_tflops": ring["flops"] / (ring["ms"] * 1e-3) / 1e12 if ring["ms"] else None,
                         "lanczos_s": lz["ms"] * 1e-3, "lanczos_steps": int(lz["flops"]),
                         "lam_top4": [float(v) for v in lam[:4]]})
    e = g.energy(w["J"])
    g.close()
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": 4 * args.sweeps / ctm_s, "unit": "moves/s", "n_gpus": world,
        "steps": args.sweeps, "warmup": 1, "ms_per_step": 1e3 * ctm_s / args.sweeps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[args.prec], "data": "synthetic",
        "config": {"workload": f"cylinder readout: 2x2 cell, d=8, D={D}, chi={chi}, complex product state + 0.1 "
                               f"noise; {args.sweeps} sweeps then boundary rho at Nv=2,4,6",
                   "prec": args.prec},
        "readouts": readouts, "energy_per_spin": e,
        "corner_spectrum_tail": float(np.min(spectra[spectra > 0])), "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


FID_DESC = ("fidelity surface: {n} points of a synthetic coupling line (all-up product + 0.1 x (cos t N1 + sin t "
            "N2), t in [0, pi/2]), 2x2 cell, d=8, D={D}, chi={chi}; {n} plain + {m} mixed networks advanced "
            "together on the batch engine, then the fidelity per site of every pair")


def run_fidelity(args, rank, world, local_rank):
    """NEXT-row fidelity surface: the plain network of every point and the mixed
    network of every pair of points of a coupling line, swept together by the
    batch engine's graph launches; throughput in pairs per second."""
    import itertools
    import torch
    import synth
    from paper_1711_04798_gb300 import Batch
    torch.cuda.set_device(local_rank)
    D = 3 if args.D == 5 else args.D
    chi = 24 if args.chi == 100 else args.chi
    line = synth.fidelity_line(seed=rank_seed(rank), n=args.points, D=D)
    pat = [[0, 1], [2, 3]]
    insts = [{"tensors": ts, "pattern": pat, "chi": chi} for ts in line]
    pairs = []
    for a, b in itertools.combinations(range(args.points), 2):
        pairs.append((len(insts), a, b))
        insts.append({"tensors": line[a], "bra": line[b], "pattern": pat, "chi": chi})
    b = Batch(insts, tune=not args.no_tune, prec=args.prec)
    b.sweep(1)  # capture
    s = torch.cuda.ExternalStream(b.stream())
    sweeps = max(args.steps, 1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        t0 = time.perf_counter()
        e0.record(s)
        b.sweep(sweeps)
        e1.record(s)
        torch.cuda.synchronize()
        d_block, d_spin = b.fidelity(pairs)
        wall = time.perf_counter() - t0
    ms = e0.elapsed_time(e1)
    b.close()
    if rank != 0:
        return
    surf = np.eye(args.points)
    for (i12, a, c), d in zip(pairs, d_block):
        surf[a, c] = surf[c, a] = d
    line_out = {
        "metric": METRIC, "value": len(pairs) / wall, "unit": "fidelity pairs/s", "n_gpus": world,
        "steps": sweeps, "warmup": 1, "ms_per_step": ms / sweeps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE[args.prec], "data": "synthetic",
        "config": {"workload": FID_DESC.format(n=args.points, D=D, chi=chi, m=len(pairs)), "prec": args.prec,
                   "sweeps": sweeps},
        "fidelity": {"pairs": len(pairs), "instances": len(insts), "sweeps_ms": ms,
                     "instance_moves_per_s": 4 * sweeps * len(insts) / (ms * 1e-3),
                     "surface_d_block": [[round(float(v), 12) for v in row] for row in surf]},
        "clocks": clk.summary(),
    }
    print(json.dumps(line_out), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "scan":
        run_scan(args, rank, world, local_rank)
    elif args.workload == "cylinder":
        run_cylinder(args, rank, world, local_rank)
    elif args.workload == "fidelity":
        run_fidelity(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
