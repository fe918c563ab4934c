#!/usr/bin/env python3
"""Benchmark of libloopnest's hot path.

One step = one pass of the chained product E = (A B) C, F = alpha E + beta D
on 2048 x 2048 FP32 matrices (alpha = 1.5, beta = 1.2, entries U[-1,1],
seed 0), the polybench 2mm loop nest of the paper's evaluation, through the
C ABI (ln_gemm_chain) in the internalized tensor-core form with the 3xBF16
split (hi*hi + hi*lo + lo*hi, FP32 accumulation), the gated precision.

Reported (one JSON line from rank 0):
  value        GFLOP/s of the internalized form, algorithmic flops 4 n^3 per
               step, device time from CUDA events around each step (one
               CUDA graph replay of the captured ln_gemm_chain call), L2
               flushed (256 MiB write) between steps outside the timed events
  plain        GFLOP/s of the plain one-thread-per-output form, same work
  fp32_tiled   GFLOP/s of the exact-FP32 shared-memory tiled form
  roofline     the tcgen05 contraction kernel: algorithmic flops per launch
               (2 n^3) / its mean launch time (CUDA events the library
               records on the launch stream), against the measured BF16
               peak divided by the 3 MMA products of the split
  e2e          same metric through ln_gemm_chain called on pinned host
               buffers: its kernels read A, B, C, D and write E, F in host
               memory over the host link inside the timed region (the staged
               variant, explicit copies around a device-buffer call, is
               reported beside it)
  cpu_baseline the FP64 oracle on this host's cores over a bounded sample of
               rows of the same workload; its rows also give rel_err, the
               sampled relative Frobenius error of E against the oracle
  clocks       nvidia-smi samples taken while the steps ran

`--impl reference` times the oracle alone (the reference arm of this
project: the paper publishes no code), on bounded samples of the workload.
With --gpus N under torchrun every rank runs its own replica (no data-path
collective); value is the sum over ranks, timed by the slowest rank.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 2048
WORKLOAD = {
    "workload": "polybench 2mm chain E=(A*B)*C, F=alpha*E+beta*D, 2048x2048 FP32, alpha=1.5, beta=1.2, "
                "U[-1,1] seed 0",
    "n": N,
    "form": "internalized",
    "precision": "3xbf16",
    "l2": "flushed between timed steps (256 MiB write outside the step events)",
    "launch": "one CUDA graph per timed step, captured from the public ln_gemm_chain call",
}
METRIC = "GFLOP/s & roofline fraction, internalized vs plain kernels, at <=1e-5 rel error"
FLOPS = 4.0 * N ** 3          # two N^3 multiply-adds per step
FLOPS_PER_UMMA = 2.0 * N ** 3
PRODUCTS = 3                   # MMA products per multiply-add in the 3xBF16 split
TF32_RATIO = 1.1 / 2.25        # nominal dense TF32 / BF16 tensor throughput


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["own", "reference"], default="own")
    ap.add_argument("--plain-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="target wall time of the CPU baseline sample")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline (profiling runs)")
    ap.add_argument("--no-suite", action="store_true",
                    help="skip the per-workload suite object of the benchmark line (profiling runs)")
    ap.add_argument("--suite", action="store_true", help="measure every workload and form, one JSON line each")
    ap.add_argument("--only", default="",
                    help="suite: comma-separated workloads (gemm,chain,3mm,cov,batched,backward,gramschmidt)")
    ap.add_argument("--modes", default="", help="suite: comma-separated form/precision pairs, e.g. internalized/3xbf16")
    return ap.parse_args()


UMMA_SOURCES = ["ln_umma_kernel.cuh", "ln_umma_general.cu", "ln_umma_sym.cu", "ln_umma_pair.cu", "ln_umma_tf32.cu", "ln_umma_tf32_pair.cu", "ln_split.cuh",
                "ln_epilogue.cuh", "ln_async.cuh", "ln_pack_stream.cuh", "ln_internal.h"]


def umma_traffic():
    """DRAM bytes per launch of the tcgen05 contraction from the committed ncu
    summary, or None when the kernel's sources changed since that capture."""
    import hashlib

    try:
        with open(os.path.join(ROOT, "profiles", "k_umma_traffic.json")) as f:
            d = json.load(f)
        h = hashlib.sha256()
        for name in d["sources"]:
            with open(os.path.join(ROOT, "paper_2312_13170_gb300", "csrc", name), "rb") as g:
                h.update(g.read())
        return float(d["dram_bytes_per_launch_mean"]) if h.hexdigest() == d["sources_sha256"] else None
    except Exception:
        return None


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["bf16_tflops"]), float(d.get("hbm_gbs", 6800.0)), "measured"
    except Exception:
        return 1900.0, 6800.0, "fallback"


# ---------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.proc = None
        self.path = None
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 7:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- distributed
def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------- CPU (oracle) leg
def host_cores():
    """Cores this process may run on (its CPU affinity mask)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_sample(d, target_s, rows_max=N):
    """Time the FP64 oracle on the first R rows of the chain (E rows depend
    only on the same rows of A and D), on every core of this process's
    affinity mask (R calibrated to ~target_s) and on one core (a smaller
    sample, ~target_s / 3)."""
    import oracle

    oracle.build()
    cores = host_cores()

    def calibrated(threads, seconds):
        oracle.set_threads(threads)
        r = 4
        t0 = time.perf_counter()
        oracle.gemm_chain(d["A"][:r], d["B"], d["C"], d["D"][:r], d["alpha"], d["beta"])
        dt = max(time.perf_counter() - t0, 1e-4)
        R = int(min(rows_max, max(r, r * seconds / dt)))
        t0 = time.perf_counter()
        E_rows, F_rows = oracle.gemm_chain(d["A"][:R], d["B"], d["C"], d["D"][:R], d["alpha"], d["beta"])
        return R, time.perf_counter() - t0, E_rows, F_rows

    R, dt, E_rows, F_rows = calibrated(cores, target_s)
    R1, dt1, _, _ = calibrated(1, target_s / 3.0)
    oracle.set_threads(cores)
    base = {"value": 4.0 * R * N * N / dt / 1e9, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
            "sample": f"first {R} of {N} rows of E and F (4*{R}*{N}^2 flops), {dt:.2f} s on {cores} cores",
            "seconds": dt,
            "one_core": {"value": 4.0 * R1 * N * N / dt1 / 1e9, "unit": "GFLOP/s", "cores": 1,
                         "sample": f"first {R1} of {N} rows, {dt1:.2f} s"}}
    return base, R, E_rows, F_rows


def run_reference(args):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return 0
    from paper_2312_13170_gb300 import inputs
    import oracle

    oracle.build()
    d = inputs.chain_inputs(N, seed=0)
    cores = host_cores()
    oracle.set_threads(cores)
    # calibrate a per-step sample of about 1 s
    r = 4
    t0 = time.perf_counter()
    oracle.gemm_chain(d["A"][:r], d["B"], d["C"], d["D"][:r], d["alpha"], d["beta"])
    dt = max(time.perf_counter() - t0, 1e-4)
    R = int(min(N, max(1, r * 1.0 / dt)))
    for _ in range(args.warmup):
        oracle.gemm_chain(d["A"][:R], d["B"], d["C"], d["D"][:R], d["alpha"], d["beta"])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.gemm_chain(d["A"][:R], d["B"], d["C"], d["D"][:R], d["alpha"], d["beta"])
    total = time.perf_counter() - t0
    ms = total / max(args.steps, 1) * 1e3
    gflops = 4.0 * R * N * N / (ms / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": gflops, "unit": "GFLOP/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(WORKLOAD, parallelism=f"replicas x{ws}"), "impl": "reference",
        "cpu_baseline": {"value": gflops, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": f"first {R} of {N} rows of E and F per step"},
        "e2e": {"value": gflops, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- replicas
def max_over_ranks(ms, dist=None, device="cpu"):
    """The slowest rank's step time; every rank receives it (one replica per
    GPU, so the job is as fast as its slowest replica)."""
    if dist is None:
        return float(ms)
    import torch

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gflops(flops_per_replica_step, world_size, ms_max):
    """Whole-job throughput: every replica does one step's work per ms_max."""
    return flops_per_replica_step * world_size / (ms_max / 1e3) / 1e9


# ---------------------------------------------------------------- GPU leg
def run_own(args):
    import torch

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    import __graft_entry__

    __graft_entry__.build()
    from paper_2312_13170_gb300 import api, inputs

    d = inputs.chain_inputs(N, seed=0)
    dev = torch.device("cuda", local)
    T = {k: torch.from_numpy(d[k]).to(dev) for k in "ABCD"}
    E = torch.empty((N, N), dtype=torch.float32, device=dev)
    F = torch.empty_like(E)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    alpha, beta = d["alpha"], d["beta"]

    def step(form="internalized", prec="3xbf16"):
        api.gemm_chain(T["A"], T["B"], T["C"], T["D"], alpha, beta, form=form, prec=prec, out=(E, F))

    def graph_steps(nsteps, form, prec):
        """One CUDA graph per step, each capturing one ln_gemm_chain call through
        the public binding (a deployed, graph-launched call)."""
        cap = torch.cuda.Stream()
        cap.wait_stream(torch.cuda.current_stream())
        graphs, pool = [], None
        for _ in range(nsteps):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, pool=pool, stream=cap):
                step(form, prec)
            pool = g.pool()
            graphs.append(g)
        for g in graphs:  # the first replay uploads the graph
            g.replay()
        barrier()
        return graphs

    def replay_timed(graphs):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in graphs]
        barrier()
        for g, (s, e) in zip(graphs, evs):
            flush.zero_()
            s.record()
            g.replay()
            e.record()
        barrier()
        return sum(s.elapsed_time(e) for s, e in evs) / max(len(graphs), 1)

    def timed(nsteps, warm, form, prec, with_timing=False):
        """Steps replay their own graphs. With timing, two more timed passes
        replay graphs captured with the library's launch-timing event nodes
        (the step time comes from the first pass, the kernel durations from
        these): "span" (timing mode 2: the chain's two contractions, launched
        back to back with programmatic overlap, share one event pair, so the
        second starts as it does in the timed step) and "bracketed" (mode 1:
        an event pair around every launch, which delays the second
        contraction until the first has finished)."""
        for _ in range(warm):
            step(form, prec)
        api.stream_check()
        l0 = api.launch_count()
        graphs = graph_steps(nsteps, form, prec)
        launches = (api.launch_count() - l0) // max(nsteps, 1) * nsteps
        ms = replay_timed(graphs)
        del graphs
        fams = {}
        for tag, mode in (("span", 2), ("bracketed", 1)) if with_timing else ():
            api.timing_enable(mode)
            for fam in ("umma", "pack", "simt", "plain", "stats"):
                api.timing_read(fam)
            graphs = graph_steps(nsteps, form, prec)  # event nodes are captured here
            api.timing_enable(0)
            # each graph's event nodes are re-recorded by the timed replay below
            # (overwriting the upload replay's), then read once
            ms_t = replay_timed(graphs)
            fams[tag] = {fam: api.timing_read(fam) for fam in ("umma", "pack")}
            fams[tag]["step_ms_with_events"] = ms_t
            del graphs
        api.stream_check()
        return ms, launches, fams

    clocks = Clocks(local)
    ms, launches, fams = timed(args.steps, args.warmup, "internalized", "3xbf16", with_timing=True)
    clk = clocks.stop()
    E_int = E.clone()
    ms_max = max_over_ranks(ms, dist, dev)
    value = whole_job_gflops(FLOPS, ws, ms_max)

    # plain and exact-FP32 tiled forms: same work, fewer steps
    ms_plain, _, _ = timed(args.plain_steps, 1, "plain", "fp32")
    ms_tiled, _, _ = timed(max(args.plain_steps, 5), 1, "internalized", "fp32")

    # end to end through the public API with host buffers: the chain call takes
    # the pinned host operands and outputs directly (its kernels read A..D and
    # write E, F over the host link; no staging copies), every step
    hostA = {k: torch.from_numpy(d[k]).pin_memory() for k in "ABCD"}
    hostE = torch.empty((N, N), dtype=torch.float32).pin_memory()
    hostF = torch.empty((N, N), dtype=torch.float32).pin_memory()
    h2d = sum(v.numel() * 4 for v in hostA.values())
    d2h = 2 * N * N * 4

    def e2e_step():
        api.gemm_chain(hostA["A"], hostA["B"], hostA["C"], hostA["D"], alpha, beta, form="internalized",
                       prec="3xbf16", out=(hostE, hostF))

    def staged_step():  # the same through explicit copies to and from device buffers
        for k in "ABCD":
            T[k].copy_(hostA[k], non_blocking=True)
        step()
        hostE.copy_(E, non_blocking=True)
        hostF.copy_(F, non_blocking=True)

    def time_host(fn, n):
        for _ in range(3):
            fn()
        barrier()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for s, e in evs:
            s.record()
            fn()
            e.record()
        barrier()
        return sum(s.elapsed_time(e) for s, e in evs) / max(n, 1)

    ms_staged = time_host(staged_step, args.e2e_steps)
    ms_e2e = time_host(e2e_step, args.e2e_steps)
    e2e_err = float((hostE - E_int.cpu()).abs().max())  # zero-copy result equals the device-resident one

    bf16_peak, hbm, peak_src = peaks()
    span, brk = fams.get("span", {}), fams.get("bracketed", {})
    umma_ms, umma_n = span.get("umma", (0.0, 0))
    achieved = FLOPS_PER_UMMA / (umma_ms / umma_n / 1e3) / 1e12 if umma_n else None
    brk_ms, brk_n = brk.get("umma", (0.0, 0))
    peak = bf16_peak / PRODUCTS
    line = {
        "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16",
        "precision": "3xBF16 split (hi*hi + hi*lo + lo*hi), FP32 accumulation",
        "data": "synthetic (seeded U[-1,1], shapes of the paper's polybench 2mm at the 2048 workload)",
        "config": dict(WORKLOAD, parallelism=f"replicas x{ws}"),
        "plain": {"value": FLOPS / (ms_plain / 1e3) / 1e9, "unit": "GFLOP/s", "ms_per_step": ms_plain,
                  "form": "plain", "precision": "fp32"},
        "fp32_tiled": {"value": FLOPS / (ms_tiled / 1e3) / 1e9, "unit": "GFLOP/s", "ms_per_step": ms_tiled,
                       "form": "internalized", "precision": "fp32"},
        "speedup_vs_plain": ms_plain / ms,
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": umma_traffic(),
                     "traffic_unit": "DRAM bytes per launch (ncu, profiles/k_umma_traffic.json)",
                     "kernel": "k_umma<2,0> (tcgen05 3xBF16 contraction)",
                     "peak_note": f"{peak_src} bf16 burst {bf16_peak} TFLOP/s / {PRODUCTS} products",
                     "launches": umma_n, "ms_per_launch": (umma_ms / umma_n) if umma_n else None,
                     "pack_ms_per_step": span.get("pack", (0.0, 0))[0] / max(args.steps, 1),
                     "timing_pass": "timed pass of the same steps, graphs captured with the library's launch "
                                    "event nodes in span mode: one pair around each step's two back-to-back "
                                    "contractions (ms_per_launch = span / 2), one pair around each other launch",
                     "timing_pass_ms_per_step": span.get("step_ms_with_events"),
                     "bracketed": {"ms_per_launch": (brk_ms / brk_n) if brk_n else None, "launches": brk_n,
                                   "frac": (FLOPS_PER_UMMA / (brk_ms / brk_n / 1e3) / 1e12 / peak) if brk_n else None,
                                   "timing_pass_ms_per_step": brk.get("step_ms_with_events"),
                                   "note": "an event pair around every launch: the second contraction waits for "
                                           "the first to finish"}},
        "e2e": {"value": FLOPS / (ms_e2e / 1e3) / 1e9, "unit": "GFLOP/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e,
                "path": "ln_gemm_chain on pinned host buffers (kernels read A..D and write E, F over the host link)",
                "max_abs_diff_vs_device_path": e2e_err,
                "staged_copies": {"value": FLOPS / (ms_staged / 1e3) / 1e9, "ms_per_step": ms_staged,
                                  "path": "H2D of A..D, ln_gemm_chain on device buffers, D2H of E, F"}},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if rank == 0 and not args.no_suite:
        # every gated workload measured in this same run (after the timed
        # steps above, so it does not disturb them): plain FP32, tiled FP32 and
        # the gated 3xBF16 tensor-core form
        records = []
        t_suite = time.perf_counter()
        suite_lines(SUITE_MODES, ALL_WORKLOADS, 5, records.append)
        line["suite"] = suite_summary(records)
        line["suite_seconds"] = round(time.perf_counter() - t_suite, 1)
        line["probes"] = peak_probes(api, bf16_peak, hbm)
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu, R, E_rows, F_rows = cpu_sample(d, args.cpu_seconds)
        line["cpu_baseline"] = cpu
        got = E_int[:R].cpu().numpy()
        line["rel_err"] = {"value": inputs.rel_fro(got, E_rows), "gate": 1e-5,
                           "sample": f"rows 0..{R - 1} of E against the FP64 oracle"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------- suite: every workload, every form
def suite_lines(modes, only, reps, sink):
    """Measures every workload of `only` in every (form, precision) of `modes`
    and hands one record per entry to sink: GFLOP/s, the roofline fraction
    (roofline time = max(flops / peak of the mode, bytes / HBM bandwidth)),
    and the relative Frobenius error on sampled outputs against the FP64
    oracle, computed in that entry's CPU-baseline leg."""
    import torch

    import oracle
    from paper_2312_13170_gb300 import api, inputs

    oracle.build()
    bf16_peak, hbm, peak_src = peaks()
    fp32_peak = fp32_simt_peak()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def peak_of(prec):
        """Peak of a mode: FP32 from unit counts; the measured BF16 peak divided
        by the products; TF32 modes from the BF16 peak scaled by the nominal
        dense TF32 / BF16 ratio (1.1 / 2.25 PFLOP/s)."""
        if prec == "fp32":
            return fp32_peak
        if prec in ("tf32", "3xtf32"):
            return bf16_peak * TF32_RATIO / (3 if prec == "3xtf32" else 1)
        return bf16_peak / {"bf16": 1, "3xbf16": 3, "6xbf16": 6}[prec]

    def time_it(fn, n=reps, graph=True):
        """Median and mean device time of fn over n repetitions, L2 flushed
        before each. With graph (the default, as in the main benchmark) every
        repetition replays its own CUDA graph of fn, so host launch gaps are
        not timed; fn must then be capturable."""
        fn()
        torch.cuda.synchronize()
        if graph:
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):  # warm-up off the default stream (autograd capture)
                fn()
            torch.cuda.current_stream().wait_stream(side)
            torch.cuda.synchronize()
            graphs, pool = [], None
            for _ in range(n):
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, pool=pool):
                    fn()
                pool = g.pool()
                graphs.append(g)
            for g in graphs:
                g.replay()
            torch.cuda.synchronize()
            run = iter([g.replay for g in graphs])
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for a, b in evs:
            f = next(run) if graph else fn
            flush.zero_()
            a.record()
            f()
            b.record()
        torch.cuda.synchronize()
        t = sorted(a.elapsed_time(b) for a, b in evs)
        return float(np.median(t)), float(np.mean(t))

    def emit(work, op, form, prec, flops, nbytes, ms, err, cpu):
        roof_ms = max(flops / (peak_of(prec) * 1e12), nbytes / (hbm * 1e9)) * 1e3
        line = {"suite": True, "workload": work, "op": op, "form": form, "precision": prec,
                "launch": "one CUDA graph replay per timed step, L2 flushed before each",
                "ms_median": ms[0], "ms_mean": ms[1], "gflops": flops / (ms[0] / 1e3) / 1e9,
                "roofline_ms": roof_ms, "roofline_frac": roof_ms / ms[0],
                "bound": "tensor" if (prec != "fp32" and flops / peak_of(prec) / 1e12 > nbytes / hbm / 1e9)
                else ("alu" if flops / peak_of(prec) / 1e12 > nbytes / hbm / 1e9 else "hbm"),
                "peak": {"tflops": peak_of(prec), "hbm_gbs": hbm, "source": peak_src},
                "rel_err": err, "cpu_baseline": cpu}
        sink(line)

    cores = host_cores()
    oracle.set_threads(cores)
    run_gemm_256(only, modes, api, inputs, oracle, cores, time_it, emit)
    run_chain_2048(only, modes, api, inputs, oracle, cores, time_it, emit, reps)
    run_3mm(only, modes, api, inputs, oracle, cores, time_it, emit, reps)
    run_cov(only, modes, api, inputs, oracle, cores, time_it, emit, reps, hbm, sink)
    run_batched(only, modes, api, inputs, oracle, cores, time_it, emit, reps)
    run_backward(only, modes, api, inputs, oracle, cores, time_it, emit, reps)
    run_gramschmidt(only, modes, api, inputs, oracle, cores, time_it, reps, fp32_peak, sink)


ALL_WORKLOADS = {"gemm", "chain", "3mm", "cov", "batched", "backward", "gramschmidt"}
SUITE_MODES = [("plain", "fp32"), ("internalized", "fp32"), ("internalized", "3xbf16"), ("internalized", "3xtf32")]
ALL_MODES = [("plain", "fp32"), ("internalized", "fp32"), ("internalized", "bf16"), ("internalized", "3xbf16"),
             ("internalized", "6xbf16"), ("internalized", "tf32"), ("internalized", "3xtf32")]


def run_suite(args):
    """--suite: one JSON line per (workload, operation, form, precision)."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)
    modes = [tuple(x.split("/")) for x in args.modes.split(",")] if args.modes else ALL_MODES
    only = set(args.only.split(",")) if args.only else ALL_WORKLOADS
    suite_lines(modes, only, max(args.steps // 20, 5), lambda line: print(json.dumps(line), flush=True))
    return 0


def suite_summary(records):
    """The suite records of the benchmark line, one entry per workload and
    operation: per form/precision the device time, GFLOP/s, roofline fraction
    and sampled error, and the internalized 3xBF16 and FP32 speedups over the
    plain form."""
    out = {}
    for r in records:
        key = f"{r['op']}: {r['workload']}"
        e = out.setdefault(key, {})
        ent = {"ms": round(r["ms_median"], 5), "rel_err": r.get("rel_err")}
        if "gflops" in r:
            ent["gflops"] = round(r["gflops"], 1)
        for k in ("roofline_frac", "hbm_gbs", "fp32_frac", "bound"):
            if k in r:
                ent[k] = round(r[k], 4) if isinstance(r[k], float) else r[k]
        e[f"{r['form']}/{r['precision']}"] = ent
    for e in out.values():
        plain = e.get("plain/fp32") or e.get("plain/fp64")
        for mode in ("internalized/3xbf16", "internalized/fp32", "internalized/fp64"):
            if plain and mode in e and e[mode]["ms"] > 0:
                e["speedup_" + mode.split("/")[1] + "_vs_plain"] = round(plain["ms"] / e[mode]["ms"], 2)
    return out


def run_gemm_256(only, modes, api, inputs, oracle, cores, time_it, emit):
    import torch

    if "gemm" not in only:
        return
    d = inputs.gemm_inputs(256, 256, 256, seed=0)
    t0 = time.perf_counter()
    ref = oracle.gemm(d["A"], d["B"], d["C"], d["alpha"], d["beta"])
    cpu = {"kind": "oracle", "cores": cores, "seconds": time.perf_counter() - t0, "sample": "whole problem",
           "gflops": 2 * 256 ** 3 / (time.perf_counter() - t0) / 1e9}
    T = {k: torch.from_numpy(d[k]).cuda() for k in "ABC"}
    for form, prec in modes:
        C = T["C"].clone()
        api.gemm(T["A"], T["B"], C, d["alpha"], d["beta"], form=form, prec=prec)
        err = inputs.rel_fro(C.cpu().numpy(), ref)
        Cw = T["C"].clone()
        ms = time_it(lambda: api.gemm(T["A"], T["B"], Cw, d["alpha"], d["beta"], form=form, prec=prec))
        emit("gemm 256^3 alpha=1.5 beta=1.2", "gemm", form, prec, 2 * 256 ** 3, 4 * 4 * 256 * 256, ms, err, cpu)



def run_chain_2048(only, modes, api, inputs, oracle, cores, time_it, emit, reps):
    import torch

    if "chain" not in only:
        return
    n = 2048
    d = inputs.chain_inputs(n, seed=0)
    rows = 64
    t0 = time.perf_counter()
    Er, Fr = oracle.gemm_chain(d["A"][:rows], d["B"], d["C"], d["D"][:rows], d["alpha"], d["beta"])
    dt = time.perf_counter() - t0
    cpu = {"kind": "oracle", "cores": cores, "seconds": dt, "sample": f"first {rows} rows of E, F",
           "gflops": 4 * rows * n * n / dt / 1e9}
    T = {k: torch.from_numpy(d[k]).cuda() for k in "ABCD"}
    for form, prec in modes:
        E, F = api.gemm_chain(T["A"], T["B"], T["C"], T["D"], d["alpha"], d["beta"], form=form, prec=prec)
        err = max(inputs.rel_fro(E[:rows].cpu().numpy(), Er), inputs.rel_fro(F[:rows].cpu().numpy(), Fr))
        out = (E, F)
        ms = time_it(lambda: api.gemm_chain(T["A"], T["B"], T["C"], T["D"], d["alpha"], d["beta"], form=form,
                                            prec=prec, out=out), n=3 if form == "plain" else reps)
        emit("chain 2048^2", "gemm_chain", form, prec, 4.0 * n ** 3, 6 * 4 * n * n, ms, err, cpu)



def run_3mm(only, modes, api, inputs, oracle, cores, time_it, emit, reps):
    """Polybench 3mm, G = (A B)(C D), at the paper's problem size (1024) and at
    2048; entries U[-1,1], seed 0, drawn in the order A, B, C, D. At 1024 also
    its adjoint (dA, dB, dC, dD for an upstream gradient U[-1,1], seed 1)."""
    import torch

    if "3mm" not in only:
        return
    for n in (1024, 2048):
        rng = np.random.default_rng(0)
        A, B, C, D = (rng.uniform(-1.0, 1.0, size=(n, n)).astype(np.float32) for _ in range(4))
        rows = 64
        t0 = time.perf_counter()
        Gr = oracle.three_mm(A[:rows], B, C, D)  # full F = C D, then the sampled rows of G
        dt = time.perf_counter() - t0
        cpu = {"kind": "oracle", "cores": cores, "seconds": dt, "sample": f"first {rows} rows of G (with all of F)",
               "gflops": 2.0 * (rows * n * n + n ** 3 + rows * n * n) / dt / 1e9}
        T = [torch.from_numpy(x).cuda() for x in (A, B, C, D)]
        for form, prec in modes:
            if form == "plain" and n > 1024:
                continue
            G = api.three_mm(*T, form=form, prec=prec)
            err = inputs.rel_fro(G[:rows].cpu().numpy(), Gr)
            ms = time_it(lambda: api.three_mm(*T, form=form, prec=prec, out=G), n=3 if form == "plain" else reps)
            emit(f"3mm {n}^3 (G = (A*B)*(C*D))", "3mm", form, prec, 6.0 * n ** 3, 5 * 4 * n * n, ms, err, cpu)
        if n != 1024:
            continue
        # the adjoint at the paper's size: upstream gradient U[-1,1] (seed 1)
        Gb = np.random.default_rng(1).uniform(-1.0, 1.0, size=(n, n)).astype(np.float32)
        t0 = time.perf_counter()
        ref = oracle.three_mm_vjp(A, B, C, D, Gb)
        dt = time.perf_counter() - t0
        cpu_b = {"kind": "oracle", "cores": cores, "seconds": dt, "sample": "the whole adjoint (8 products)",
                 "gflops": 16.0 * n ** 3 / dt / 1e9}
        Gbt = torch.from_numpy(Gb).cuda()
        for form, prec in modes:
            grads = api.three_mm_bwd(*T, Gbt, form=form, prec=prec)
            err = max(inputs.rel_fro(g.cpu().numpy(), r) for g, r in zip(grads, ref))
            ms = time_it(lambda: api.three_mm_bwd(*T, Gbt, form=form, prec=prec), n=3 if form == "plain" else reps)
            emit(f"3mm adjoint {n}^3 (dA, dB, dC, dD)", "3mm_bwd", form, prec, 16.0 * n ** 3, 9 * 4 * n * n, ms, err,
                 cpu_b)


def run_cov(only, modes, api, inputs, oracle, cores, time_it, emit, reps, hbm, sink):
    import torch

    if "cov" not in only:
        return
    ns, m = 8192, 2048
    X = inputs.cov_inputs(ns, m, seed=0)["X"]
    Xt = torch.from_numpy(X).cuda()
    rows_s = [0, 100, 1000, 2047]
    t0 = time.perf_counter()
    cov_r = oracle.cov_rows(X, rows_s)
    corr_r = oracle.cov_rows(X, rows_s, corr=True)
    dt = time.perf_counter() - t0
    cpu = {"kind": "oracle", "cores": cores, "seconds": dt, "sample": f"rows {rows_s} of cov and corr",
           "gflops": 2 * 2 * len(rows_s) * ns * m / dt / 1e9}
    flops = float(ns) * m * (m + 1)
    for form in ("plain", "internalized"):
        mean, ss = api.col_stats(Xt, form=form)
        ms = time_it(lambda: api.col_stats(Xt, form=form))
        mr, sr = oracle.col_stats(X)
        err = max(inputs.rel_fro(mean.cpu().numpy(), mr), inputs.rel_fro(ss.cpu().numpy(), sr))
        line = {"suite": True, "workload": "column statistics 8192x2048", "op": "col_stats", "form": form,
                "precision": "fp64", "ms_median": ms[0], "ms_mean": ms[1],
                "hbm_gbs": 2 * 4 * ns * m / (ms[0] / 1e3) / 1e9,
                "roofline_frac": (2 * 4 * ns * m / (hbm * 1e9) * 1e3) / ms[0], "bound": "hbm", "rel_err": err}
        sink(line)
    for form, prec in modes:
        if form == "plain":
            reps_here = 2
        else:
            reps_here = reps
        cv = api.covariance(Xt, form=form, prec=prec)
        cr = api.correlation(Xt, form=form, prec=prec)
        err_c = inputs.rel_fro(cv[rows_s].cpu().numpy(), cov_r)
        err_r = inputs.rel_fro(cr[rows_s].cpu().numpy(), corr_r)
        ms = time_it(lambda: api.covariance(Xt, form=form, prec=prec, out=cv), n=reps_here)
        emit("covariance 8192x2048", "covariance", form, prec, flops, (2 * 4 * ns * m + 4 * m * m), ms, err_c, cpu)
        ms = time_it(lambda: api.correlation(Xt, form=form, prec=prec, out=cr), n=reps_here)
        emit("correlation 8192x2048", "correlation", form, prec, flops, (3 * 4 * ns * m + 4 * m * m), ms, err_r, cpu)



def run_batched(only, modes, api, inputs, oracle, cores, time_it, emit, reps):
    import torch

    if "batched" not in only:
        return
    b = inputs.sym_batch_inputs(512, 32, 1536, seed=0)
    inst = b["instances"]
    nk = [(x["n"], x["k"]) for x in inst]
    As = [torch.from_numpy(x["A"]).cuda() for x in inst]
    Bs = [torch.from_numpy(x["B"]).cuda() for x in inst]
    C0 = [torch.from_numpy(x["C"]).cuda() for x in inst]
    rng = np.random.default_rng(5)
    samp = [(i, int(rng.integers(inst[i]["n"]))) for i in rng.choice(512, size=16, replace=False)]
    for two in (False, True):
        op = "syr2k_batched" if two else "syrk_batched"
        fl = sum((2.0 if two else 1.0) * n_ * (n_ + 1) * k_ for n_, k_ in nk)
        by = sum((8.0 if two else 4.0) * n_ * k_ + 8.0 * n_ * n_ for n_, k_ in nk)
        t0 = time.perf_counter()
        refs = {}
        for i, r in samp:
            x = inst[i]
            if two:
                v = oracle.gemm(x["A"][r:r + 1], x["B"].T, x["C"][r:r + 1], b["alpha"], b["beta"])
                v += oracle.gemm(x["B"][r:r + 1], x["A"].T, None, b["alpha"], 0.0)
            else:
                v = oracle.gemm(x["A"][r:r + 1], x["A"].T, x["C"][r:r + 1], b["alpha"], b["beta"])
            refs[(i, r)] = v
        dt = time.perf_counter() - t0
        cpu = {"kind": "oracle", "cores": cores, "seconds": dt, "sample": "16 sampled rows of 16 instances"}
        for form, prec in modes:
            Cs = [c.clone() for c in C0]
            batch = api.SymBatch(As, Cs, Bs if two else None, b["alpha"], b["beta"], form=form, prec=prec)
            batch.run()
            torch.cuda.synchronize()
            got = np.concatenate([Cs[i][r:r + 1].cpu().numpy() for i, r in samp], axis=1)
            want = np.concatenate([refs[(i, r)] for i, r in samp], axis=1)
            err = inputs.rel_fro(got, want)
            g = torch.cuda.CUDAGraph()
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                batch.run(s)
            torch.cuda.current_stream().wait_stream(s)
            with torch.cuda.graph(g):
                batch.run()
            ms = time_it(g.replay, n=2 if form == "plain" else reps, graph=False)
            emit("512 uneven instances, n,k log-uniform [32,1536], CUDA graph", op, form, prec, fl, by, ms, err, cpu)



def run_backward(only, modes, api, inputs, oracle, cores, time_it, emit, reps):
    import torch

    if "backward" not in only:
        return
    d = inputs.backward_inputs(4096, 1024, 1024, seed=0)
    Xb = torch.from_numpy(d["X"]).cuda()
    W = torch.from_numpy(d["W"]).cuda()
    A, B, C = (torch.from_numpy(d[k]).cuda() for k in "ABC")
    t0 = time.perf_counter()
    dx_ref = oracle.correlation_vjp(d["X"][:, :], d["W"])
    dt = time.perf_counter() - t0
    cpu = {"kind": "oracle", "cores": cores, "seconds": dt, "sample": "whole correlation VJP"}
    p, nb, mb = 1024, 4096, 1024
    # corr forward (triangle) + dZ = Z (W + W^T) + chain forward 4p^3 + chain adjoint 10p^3 (T reused)
    fl = float(nb) * mb * (mb + 1) + 2.0 * nb * mb * mb + 14.0 * p ** 3
    for form, prec in [m for m in modes if m[1] in ("fp32", "3xbf16")]:
        def step():
            Xg = Xb.detach().requires_grad_(True)
            Ag, Bg, Cg = (t.detach().requires_grad_(True) for t in (A, B, C))
            R = api.CorrelationFn.apply(Xg, form, prec, True)
            E = api.GemmChainFn.apply(Ag, Bg, Cg, form, prec)
            ((W * R).sum() + (E * E).sum()).backward()
            return Xg.grad
        gx = step()
        err = inputs.rel_fro(gx.cpu().numpy(), dx_ref)
        ms = time_it(step, n=2 if form == "plain" else reps)
        emit("backward: X 4096x1024, W/A/B/C 1024^2", "fwd+bwd", form, prec, fl,
             4.0 * (5 * nb * mb + 2 * mb * mb + 10 * p * p), ms, err, cpu)


def fp32_simt_peak():
    """FP32 FFMA peak from unit counts: SMs x 128 lanes x 2 flops x max SM clock."""
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    try:
        out = subprocess.run(["nvidia-smi", "-i", "0", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                             capture_output=True, text=True, timeout=20).stdout.strip()
        mhz = float(out.splitlines()[0])
    except Exception:
        mhz = 2070.0
    return sms * 128 * 2 * mhz * 1e6 / 1e12


def peak_probes(api, bf16_peak, hbm):
    """The library's peak probes on this GPU (median of 5 event-timed launches
    each, after one warm-up launch): tcgen05 BF16 and TF32 MMA issue loops,
    FFMA chains and a 1 GiB streaming copy. Context for the roofline
    denominators above, which stay the measured copy and cuBLAS figures."""
    import torch

    def rate(kind, iters, src=None, dst=None):
        api.peak_probe(kind, iters, src, dst)
        torch.cuda.synchronize()
        out = []
        for _ in range(5):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            work = api.peak_probe(kind, iters, src, dst)
            e.record()
            e.synchronize()
            out.append(work / (s.elapsed_time(e) / 1e3))
        return sorted(out)[2]

    err = torch.zeros(4, dtype=torch.int32, device="cuda")
    bf16 = rate("mma_bf16", 16384, dst=err) / 1e12
    tf32 = rate("mma_tf32", 16384, dst=err) / 1e12
    timed_out = int(err[0])
    ffma = rate("ffma", 4096, dst=torch.zeros(1, device="cuda")) / 1e12
    src = torch.empty(1 << 28, device="cuda").fill_(1.0)  # 1 GiB each way
    dst = torch.empty_like(src)
    copy = rate("copy", 0, src, dst) / 1e9
    del src, dst
    api.stream_check()
    return {"mma_bf16_tflops": bf16, "mma_tf32_tflops": tf32, "ffma_tflops": ffma, "copy_gbs": copy,
            "mma_timed_out": timed_out,
            "vs_denominators": {"mma_bf16 / measured cuBLAS bf16": bf16 / bf16_peak,
                                "mma_tf32 / (measured cuBLAS bf16 x 1.1/2.25)": tf32 / (bf16_peak * TF32_RATIO),
                                "ffma / (SMs x 128 lanes x 2 x max SM clock)": ffma / fp32_simt_peak(),
                                "copy / measured copy": copy / hbm},
            "kernels": "k_peak_mma<TF> (one CTA per SM, M=128 N=256, operands in shared memory), k_peak_ffma, "
                       "k_peak_copy (ln_peak_probe)"}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.suite:
        return run_suite(args)
    return run_own(args)


def run_gramschmidt(only, modes, api, inputs, oracle, cores, time_it, reps, fp32_peak, sink):
    """Polybench Gram-Schmidt QR at the paper's size (1024 x 1024, U[-1,1]),
    the FP32 forms among `modes`. Flops as the loop nest counts them: per
    column k, 2m for the norm, m for the scaling and 4m per later column."""
    import torch

    forms = [f for f, p in modes if p == "fp32"]
    if "gramschmidt" not in only or not forms:
        return
    m = n = 1024
    A = inputs.gramschmidt_inputs(m, n, seed=0)["A"]
    t0 = time.perf_counter()
    Qo, Ro = oracle.gramschmidt(A)
    dt = time.perf_counter() - t0
    flops = sum(3.0 * m + 4.0 * m * (n - k - 1) for k in range(n))
    cpu = {"kind": "oracle", "cores": cores, "seconds": dt, "sample": "the whole 1024 x 1024 factorisation",
           "gflops": flops / dt / 1e9}
    kappa = float(np.linalg.cond(A.astype(np.float64)))
    Ad = torch.from_numpy(A).cuda()
    Q = torch.empty_like(Ad)
    R = torch.empty((n, n), dtype=torch.float32, device="cuda")
    for form in forms:
        api.gramschmidt(Ad, form=form, Q=Q, R=R)
        errR = inputs.rel_fro(R.cpu().numpy(), Ro)
        errQ = inputs.rel_fro(Q.cpu().numpy(), Qo)
        ms = time_it(lambda: api.gramschmidt(Ad, form=form, Q=Q, R=R), n=3 if form == "plain" else reps)
        gflops = flops / (ms[0] / 1e3) / 1e9
        line = {"suite": True, "workload": "Gram-Schmidt QR 1024 x 1024 (modified, polybench order)",
                "op": "gramschmidt", "form": form, "precision": "fp32",
                "launch": "one CUDA graph replay per timed step, L2 flushed before each",
                "launches_per_call": 3 * n if form == "plain" else 2 * ((n + 31) // 32) - 1,
                "ms_median": ms[0], "ms_mean": ms[1], "gflops": gflops,
                "bound": "latency",
                "bound_note": "n dependent column steps, each a reduction over all m rows; "
                              "the FP32 fraction below is of the whole GPU's FP32 rate",
                "fp32_frac": gflops / 1e3 / fp32_peak,
                "rel_err": errR, "rel_err_Q": errQ, "kappa": kappa, "Q_bound": max(1e-5, kappa * 2.0 ** -24),
                "cpu_baseline": cpu}
        sink(line)


if __name__ == "__main__":
    sys.exit(main())
