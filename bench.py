#!/usr/bin/env python
"""Benchmark of the D-iteration hot path on GB300.

One step = one complete solve of X = P X + B (PageRank form, d = 0.85) by the
threshold-frontier D-iteration, from F = B to the exact FP64 stop
|B + P H - H|_1 <= 1e-8 |B|_1, on a seeded synthetic web-like graph.
Metric: solves per second to that tolerance (the reciprocal of the time to
tolerance, summed over replicas); the line also carries the time to
tolerance, edge diffusions per second (the paper's elementary cost unit,
Sec. 2.4) and the normalised iterations (edge diffusions / L).  The default
run adds the N = 2^24 stress workload (stress_16m) and the learned warm start
as specified (warmstart_cfg5: 200 training graphs, 32 held-out N = 3e6
graphs), each checked against the CPU oracle.

Default workload: N = 1,000,000 nodes, mean out-degree 10 (non-dangling),
10% dangling, +-64 locality window, FP32 fluid with FP64 history, exact
FP64 residual when |F|_1 fell 1024-fold.  Inputs are resident in HBM for the
device timing; L2 is flushed (256 MiB write) before every timed step.

Arms:
  --impl native     (default) the CUDA library through its C ABI;
  --impl reference  the CPU oracle, timed as it stands on the host cores.
Multi-GPU (torchrun): independent replicas, one solve per rank per step,
no collective on the data path ("scaling": "weak").
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

import numpy as np

REPO = os.path.dirname(os.path.abspath(__file__))
if REPO not in sys.path:
    sys.path.insert(0, REPO)

from paper_1202_6168_gb300 import graphgen as gg  # noqa: E402

D = 0.85
WORKLOADS = {
    "web-1m": (gg.WEB_1M, "web-like N=1e6, m=10, +-64 window, seed 0"),
    "stress-16m": (gg.STRESS_16M, "web-like N=2^24, m=16, +-256 window, seed 0"),
    "web-10k": (gg.SMALL_10K, "web-like N=1e4, m=8, +-64 window, seed 0"),
    "web-4m": (gg.MID_4M, "web-like N=2^22, m=16, +-256 window, seed 0"),
    "warmstart": (None, "learned warm start: trained on seeded web-like graphs (N log-uniform in [1e5, 1e6], "
                        "m=10, seeds 1000..), evaluated on held-out N=3e6, m=10 graphs (seeds 2000..)"),
    "kpid-1m": (gg.WEB_1M, "K-PID asynchronous D-iteration (Secs. 2.3-2.6) on the web-like N=1e6, m=10 graph, "
                           "K = 1, 2, 4, 8, uniform and cost-balanced ranges"),
    "batch-64x4": (None, "64 web-like graphs, N log-uniform in [1e4, 2e6], m ~ U[6, 14], seeds 0..63; "
                         "4 personalised right-hand sides each (B = 0.15 e_s), 256 solves per step"),
    "kpid-sim": (gg.GraphSpec(n=100_000, mean_deg=10.0, window=64, seed=0),
                 "time-stepped simulation of K PIDs (Secs. 2.3-2.6, Sec. 3) on the host cores: web-like N=1e5, "
                 "m=10, PID_Speed = L/K, target error r/(1-d) <= 1/N, K = 1..64, uniform and cost-balanced "
                 "ranges, Delay_Proba 0 / 0.5 / 0.8 at K = 8"),
}
# algorithmic bytes of the level kernel: per edge diffusion, per node
# diffusion, and per node scanned (the fluid read of the selection)
EDGE_BYTES = {"f32": 12, "f64": 20}   # 4 B column index + target fluid read + write
NODE_BYTES = {"f32": 40, "f64": 48}   # row_ptr pair, fluid exchange, FP64 history RMW, frontier write + read
SCAN_BYTES = {"f32": 4, "f64": 8}     # fluid read of every node, every level


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["native", "reference"], default="native")
    p.add_argument("--workload", choices=sorted(WORKLOADS), default="web-1m")
    p.add_argument("--fp64", action="store_true", help="FP64 fluid instead of FP32")
    p.add_argument("--no-extras", action="store_true", help="skip e2e, roofline and CPU baseline legs")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline and the oracle check only")
    p.add_argument("--alpha", type=float, default=None, help="threshold decay (library default if unset)")
    p.add_argument("--recompute-every", type=int, default=None,
                   help="exact FP64 residual every this many levels (stress-16m: 8, its configuration's rule)")
    p.add_argument("--recompute-drop", type=float, default=None,
                   help="exact FP64 residual when |F|_1 fell by this factor (library default 1024; stress-16m: off)")
    p.add_argument("--no-l2-window", action="store_true", help="no L2 access-policy windows")
    p.add_argument("--propagation", type=int, default=None,
                   help="0 auto/binned gather, 1 auto/flat gather, 2 push only, 3 asynchronous push, "
                        "4 asynchronous push with warp-level tiles, 5 fused select + push, "
                        "6 node-ordered chunks with on-chip window and hot slots, 7 persistent level loop")
    p.add_argument("--push-ratio", type=int, default=None, help="dense-level threshold of the auto modes")
    p.add_argument("--resweeps", type=int, default=None,
                   help="propagations 3-7: re-selections at the same threshold before T <- T/alpha")
    p.add_argument("--slice-sweeps", type=int, default=None,
                   help="propagations 3 and 7: sweeps of each push CTA's node slice at the level's threshold "
                        "after the frontier (nodes that crossed T while the level pushed), 0 = off")
    p.add_argument("--exact-residual", type=int, default=None,
                   help="exact FP64 residual: 0 auto, 1 binned gather, 2 source-blocked gather")
    p.add_argument("--autotune", action="store_true", help="single solves: choose the push shape by timing first")
    p.add_argument("--dangling", action="store_true",
                   help="complete the dangling columns by 1/N (standard PageRank normalisation)")
    p.add_argument("--weighted", action="store_true",
                   help="select on |F_i| / ((in_i + 1)(out_i + 1)) (the score of the paper's ideal order)")
    p.add_argument("--ws-train", type=int, default=200, help="warm start: training graphs")
    p.add_argument("--ws-eval", type=int, default=32, help="warm start: held-out evaluation graphs")
    p.add_argument("--ws-epochs", type=int, default=8, help="warm start: training epochs")
    p.add_argument("--ws-lr", type=float, default=1e-3, help="warm start: Adam learning rate")
    p.add_argument("--no-stress", action="store_true", help="skip the N=2^24 stress sub-object")
    p.add_argument("--no-cfg5", action="store_true", help="skip the learned warm-start study sub-object")
    p.add_argument("--host-loop", action="store_true",
                   help="host-driven levels with per-kernel events (profilers cannot see kernels in "
                        "graphs with conditional nodes)")
    return p.parse_args()


def aggregate_over_ranks(secs: float, units: float, world: int, device: str) -> tuple[float, float]:
    """Whole-job figures of replicas: the slowest rank's time (max) and the
    units all ranks processed (sum).  No data-path collective: this is the
    only exchange, after the timed region."""
    if world <= 1:
        return float(secs), float(units)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(secs)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def measured_hbm_peak():
    path = os.path.join(REPO, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def level_traffic(workload: str, prec: str, propagation: int, slice_sweeps: int):
    """DRAM bytes (read + write) of one level's kernels (selection + push),
    averaged over the levels of one solve, from the ncu capture summarised in
    profiles/level_traffic.txt (lines: workload precision propagation
    slice_sweeps bytes); None when no capture of this configuration is
    recorded."""
    path = os.path.join(REPO, "profiles", "level_traffic.txt")
    try:
        with open(path) as f:
            for line in f:
                parts = line.split()
                if len(parts) == 5 and not line.startswith("#") and parts[0] == workload and parts[1] == prec \
                        and parts[2] == str(propagation) and parts[3] == str(slice_sweeps):
                    return float(parts[4])
    except OSError:
        return None
    return None


def cpu_baseline(rp, col, b, tol, dangling=False):
    """The CPU oracle as it stands, on one host core, one full solve."""
    from oracle import diter as od
    t0 = time.perf_counter()
    r = od.d_iteration(rp, col, b, D, tol=tol, dangling=dangling)
    dt = time.perf_counter() - t0
    return {"value": 1.0 / dt, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"one full sequential FP64 solve of the same graph to the same tol "
                      f"({r.levels} levels, {r.edge_diffusions} edge diffusions, {dt:.2f} s)",
            "seconds": dt, "edge_diffusions_per_s": r.edge_diffusions / dt,
            "normalised_iterations": r.edge_diffusions / len(col)}


def run_reference(args, world, rank):
    if rank != 0:
        return
    spec, desc = WORKLOADS[args.workload]
    if args.workload == "kpid-1m":
        run_reference_kpid(args, desc)
        return
    if spec is None:
        run_reference_multi(args, desc)
        return
    rp, col = gg.generate(spec)
    b = gg.uniform_b(spec.n, D)
    tol = 1e-8 * b.sum()
    from oracle import diter as od
    for _ in range(args.warmup):
        od.d_iteration(rp, col, b, D, tol=tol)
    edges, secs = 0, 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = od.d_iteration(rp, col, b, D, tol=tol)
        secs += time.perf_counter() - t0
        edges += r.edge_diffusions
    value = args.steps / secs
    line = {"impl": "reference", "metric": "solves_per_s_to_tol", "value": value,
            "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "n": spec.n, "nnz": int(len(col)), "tol": tol,
                       "oracle": "sequential cyclic-threshold D-iteration, FP64, 1 core"},
            "time_to_tol_ms": 1e3 * secs / args.steps, "edge_diffusions_per_s": edges / secs,
            "normalised_iterations": edges / args.steps / len(col),
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} full solves of the workload"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_kpid(args, desc):
    """Reference arm of the K-PID workload: the oracle's emulation of 8 PIDs
    (cost-balanced ranges) on a bounded sample, a web-like graph of N = 1e5
    (N = 2e4 with the 1/N completion, whose completed columns cost the
    sequential emulation O(N) each)."""
    from oracle import kpid as ok
    n_sample = 20_000 if args.dangling else 100_000
    sp = gg.GraphSpec(n=n_sample, mean_deg=10.0, window=64, seed=0)
    rp, col = gg.generate(sp)
    b = gg.uniform_b(sp.n, D)
    tol = 1e-8 * b.sum()
    L = int(len(col))
    costs, secs = [], 0.0
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = ok.kpid(rp, col, b, D, tol=tol, bounds=ok.cb_bounds(rp, 8), dangling=bool(args.dangling))
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            secs += dt
            costs.append(float(r.ops.max()) / L)
    value = statistics.mean(costs)
    line = {"impl": "reference", "metric": "max_pid_normalised_iterations", "value": value,
            "unit": "iterations (ops/L)", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / max(args.steps, 1), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "sample": f"web-like N={n_sample:.0e}, m=10, K=8 cost-balanced ranges",
                       "oracle": "sequential emulation of K PIDs, FP64, 1 core",
                       "dangling": ["zero columns", "uniform 1/N completion"][int(bool(args.dangling))]},
            "cpu_baseline": {"value": value, "unit": "iterations (ops/L)", "cores": 1, "kind": "oracle",
                             "sample": f"K=8 cost-balanced ranges on a web-like N={n_sample:.0e} graph"},
            "e2e": {"value": value, "unit": "iterations (ops/L)", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_kpid_sim(args, world, rank, local):
    """Reference arm of the K-PID simulation: the oracle's lock-step emulation
    (one sweep per PID per round) on the same graph and target, K = 1 and
    K = 64 cost-balanced; its speed-up is the one-PID cost over the largest
    per-PID cost (the emulation has no time steps)."""
    from oracle import kpid as ok
    spec, desc = WORKLOADS["kpid-sim"]
    rp, col = gg.generate(spec)
    n, L = spec.n, int(len(col))
    b = gg.uniform_b(n, D)
    tol = (1.0 - D) / n
    t0 = time.perf_counter()
    one = ok.kpid(rp, col, b, D, tol=tol, K=1)
    many = ok.kpid(rp, col, b, D, tol=tol, bounds=ok.cb_bounds(rp, 64))
    secs = time.perf_counter() - t0
    value = float(one.ops.max()) / float(many.ops.max())
    print(json.dumps({"impl": "reference", "metric": "kpid_speedup", "value": value,
                      "unit": "x (1-PID time / K-PID time)", "n_gpus": 0, "steps": 2, "warmup": 0,
                      "ms_per_step": 1e3 * secs / 2, "higher_is_better": True, "scaling": "weak",
                      "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": desc, "sample": "K = 1 and K = 64 cost-balanced, lock-step emulation",
                                 "oracle": "sequential emulation of K PIDs, FP64, 1 core"},
                      "cpu_baseline": {"value": value, "unit": "x (1-PID time / K-PID time)", "cores": 1,
                                       "kind": "oracle", "sample": "K = 1 and K = 64 cost-balanced"},
                      "e2e": {"value": value, "unit": "x (1-PID time / K-PID time)", "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}), flush=True)


def run_reference_multi(args, desc):
    """Reference arm of the batched and warm-start workloads: the oracle's cold
    solves of a bounded sample of their items, on one host core."""
    from oracle import diter as od
    if args.workload == "batch-64x4":
        specs, csrs, rhs = batch_inputs()
        order = sorted(range(len(specs)), key=lambda g: specs[g].n)
        items = [(csrs[gi], gg.personalised_b(specs[gi].n, src, D)) for gi in order for (g2, src) in rhs if g2 == gi]
        sample = "items of the smallest graphs"
    else:
        sp = gg.warmstart_specs("eval", 1)[0]
        items = [(gg.generate(sp), gg.uniform_b(sp.n, D))]
        sample = "the cold solve of one held-out N=3e6 graph"
    edges, secs, done = 0, 0.0, 0
    for step in range(args.warmup + args.steps):
        for (rp, col), b in items[:max(1, len(items) // 8)]:
            t0 = time.perf_counter()
            r = od.d_iteration(rp, col, b, D, tol=1e-8 * b.sum())
            if step >= args.warmup:
                secs += time.perf_counter() - t0
                edges += r.edge_diffusions
                done += 1
    if args.workload == "batch-64x4":
        # the native line's metric: edge diffusions per second
        metric, unit, value, hib = "edge_diffusions_per_s", "edge_diffusions/s", edges / secs, True
    else:
        # the native line's metric: time to tol of one held-out graph (the zero start)
        metric, unit, value, hib = "time_to_tol_ms", "ms", 1e3 * secs / max(done, 1), False
    print(json.dumps({"impl": "reference", "metric": metric, "value": value,
                      "unit": unit, "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": 1e3 * secs / max(args.steps, 1), "higher_is_better": hib, "scaling": "weak",
                      "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": desc, "oracle": "sequential cyclic-threshold D-iteration, FP64, 1 core"},
                      "cpu_baseline": {"value": value, "unit": unit, "cores": 1, "kind": "oracle",
                                       "sample": f"{done} solves: {sample}"},
                      "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}), flush=True)


def phase_roofline(di, g, B, H, tol, opts, prec, n, flush, stream, workload, reps=3):
    """Roofline of the level kernels of propagation 3 (selection, then the
    asynchronous push), with every phase timed on the device: the persistent
    level loop (propagation 7) runs the same selection and push code and
    reads %globaltimer at its grid barriers, so the times are those of the
    phases inside a running solve, with no host launch in between.  Each
    phase's time includes its closing grid barrier, which makes the
    fractions conservative.  Algorithmic bytes: 4 B (FP64: 8 B) of fluid per
    node and selection pass; 12 B (20 B) per edge diffusion and 40 B (48 B)
    per node diffusion for the push."""
    popt = di.opts_copy(opts, propagation=7, timing=0)
    sel_s = push_s = 0.0
    passes = nodes = edges = reds = 0
    sweeps = 0
    for _ in range(reps):
        flush.zero_()
        _, st = di.di_solve(g, B, D, tol, H, None, popt)
        sweeps = st.slice_sweeps
        sel_s += st.select_seconds
        push_s += st.level_seconds - st.select_seconds
        passes += st.level_launches
        nodes += st.node_diffusions
        edges += st.edge_diffusions
        reds += st.red_ops
    peak, peak_src = measured_hbm_peak()
    sel_b = SCAN_BYTES[prec] * n * passes
    # the push's slice sweeps read the fluid once more per sweep
    push_b = EDGE_BYTES[prec] * edges + NODE_BYTES[prec] * nodes + SCAN_BYTES[prec] * n * passes * sweeps
    achieved = (sel_b + push_b) / (sel_s + push_s) / 1e9
    traffic = level_traffic(workload, prec, 3, sweeps) \
        if not (opts.selection or opts.dangling) and opts.resweeps == 0 else None
    out = {"bound": "hbm", "kernel": "selection + asynchronous push of a level (propagation 3's code)",
           "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "peak_source": f"{peak_src} (hbm_gbs)", "traffic": traffic,
           "alg_bytes_per_launch": (sel_b + push_b) / max(passes, 1),
           "avg_launch_us": 1e6 * (sel_s + push_s) / max(passes, 1),
           "phases": {"select": {"seconds": sel_s, "alg_bytes": sel_b, "achieved": sel_b / sel_s / 1e9,
                                 "frac": sel_b / sel_s / 1e9 / peak},
                      "push": {"seconds": push_s, "alg_bytes": push_b, "achieved": push_b / push_s / 1e9,
                               "frac": push_b / push_s / 1e9 / peak}},
           "passes": passes, "solves": reps,
           "measured_by": "device %globaltimer at the grid barriers of the persistent level loop "
                          "(propagation 7: the same selection and push code, one launch per segment)"}
    if reds:
        red_peak, _ = di.probe_l2("red_f32" if prec == "f32" else "red_f64", 1 << 24, 1 << 28, stream)
        out_red = {"achieved": reds / push_s, "peak": red_peak, "unit": "red sectors/s",
                   "frac": reds / push_s / red_peak, "red_sectors_per_edge": reds / max(edges, 1),
                   "peak_source": "di_probe_l2 scattered red over 2^24 words, this run",
                   "kernel": "push phase"}
        return out, out_red
    return out, None


def stress_leg(args, di, stream, flush):
    """The N = 2^24, m = 16, +-256 window workload: FP32 fluid, FP64 history, an
    exact FP64 residual every 8 levels (the workload's schedule), the library's
    default level (one slice sweep per level); time to tolerance, the phase
    roofline, and the error of H against the oracle's X (the oracle solved to
    1e-10 |B|_1, so its own error is <= 6.7e-10 |X|_1)."""
    import torch
    from oracle import diter as od
    sp = gg.STRESS_16M
    t0 = time.perf_counter()
    rp, col = gg.generate(sp)
    gen_s = time.perf_counter() - t0
    n, nnz = sp.n, int(len(col))
    b = gg.uniform_b(n, D)
    tol = 1e-8 * b.sum()
    g = di.Graph.create(rp, col, stream=stream)
    B = torch.from_numpy(b).cuda()
    H = torch.zeros(n, dtype=torch.float64, device="cuda")
    opts = di.opts_default(stream=stream.cuda_stream, recompute_every=8, recompute_drop=0.0)
    di.di_solve(g, B, D, tol, H, None, opts)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    times, st = [], None
    for _ in range(3):
        flush.zero_()
        ev[0].record(stream)
        _, st = di.di_solve(g, B, D, tol, H, None, opts)
        ev[1].record(stream)
        torch.cuda.synchronize()
        times.append(ev[0].elapsed_time(ev[1]))
    ms = statistics.median(times)
    roof, red = phase_roofline(di, g, B, H, tol, opts, "f32", n, flush, stream, "stress-16m")
    h = H.cpu().numpy()
    g.close()
    del B, H
    t0 = time.perf_counter()
    x = od.d_iteration(rp, col, b, D, tol=1e-10 * b.sum()).H
    oracle_s = time.perf_counter() - t0
    _, r_cpu = od.residual(rp, col, b, D, h)
    out = {"workload": WORKLOADS["stress-16m"][1], "n": n, "nnz": nnz, "time_to_tol_ms": ms,
           "solves_per_s": 1e3 / ms, "edge_diffusions_per_s": st.edge_diffusions / (ms * 1e-3),
           "normalised_iterations": st.edge_diffusions / nnz, "levels": st.levels,
           "passes": st.body_iterations, "recomputes": st.recomputes,
           "options": {"propagation": "asynchronous push (3)", "resweeps": 0, "slice_sweeps": st.slice_sweeps,
                       "recompute_every": 8, "fluid": "f32", "history": "f64"},
           "roofline": roof,
           "check": {"rel_l1_err_vs_oracle_x": float(np.abs(h - x).sum() / np.abs(x).sum()),
                     "resid_l1_oracle_fp64": r_cpu, "tol": tol, "stop_ok": bool(r_cpu <= tol * (1 + 1e-9)),
                     "oracle_tol": "1e-10 |B|_1", "oracle_seconds": oracle_s},
           "setup_seconds": {"generate": gen_s}}
    if red:
        out["l2_red"] = red
    return out


def warmstart_study(args, di, stream, flush, n_train, n_eval, epochs, lr, reps=2, warmup=1):
    """The learned warm start as the workload specifies it: train on n_train
    seeded graphs (N log-uniform in [1e5, 1e6], m = 10) with targets from the
    plain solver, then time to |F|_1 <= 1e-8 |B|_1 on n_eval held-out N = 3e6
    graphs - warm (features + network + F0 + solve, all timed) against the
    zero start on the same GPU - with the fallback count."""
    import torch
    t_gen = time.perf_counter()
    graphs, Bs, Xs = [], [], []
    train_nodes = 0
    for sp in gg.warmstart_specs("train", n_train):
        rp, col = gg.generate(sp)
        g = di.Graph.create(rp, col, stream=stream)
        b = torch.full((sp.n,), (1.0 - D) / sp.n, dtype=torch.float64, device="cuda")
        h = torch.zeros(sp.n, dtype=torch.float64, device="cuda")
        di.di_solve(g, b, D, 1e-8 * (1.0 - D), h, None, di.opts_default(stream=stream.cuda_stream))
        graphs.append(g)
        Bs.append(b)
        Xs.append(h)
        train_nodes += sp.n
    t_gen = time.perf_counter() - t_gen
    model = di.Model.create(7)
    t0 = time.perf_counter()
    loss = model.train(graphs, Bs, Xs, di.train_opts_default(epochs=epochs, batch=65536, lr=lr,
                                                             stream=stream.cuda_stream))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    for g in graphs:
        g.close()
    del Bs, Xs
    rows = []
    opts_c = di.opts_default(stream=stream.cuda_stream)
    opts_w = di.opts_default(stream=stream.cuda_stream, warm_start=1)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    infer_parts = None
    for sp in gg.warmstart_specs("eval", n_eval):
        rp, col = gg.generate(sp)
        g = di.Graph.create(rp, col, stream=stream)
        n = sp.n
        b = torch.full((n,), (1.0 - D) / n, dtype=torch.float64, device="cuda")
        tol = 1e-8 * (1.0 - D)
        H = torch.zeros(n, dtype=torch.float64, device="cuda")
        res = {}
        for label in ("cold", "warm"):
            times = []
            for rep in range(warmup + reps):
                flush.zero_()
                ev[0].record(stream)
                if label == "warm":
                    model.infer(g, b, H, stream)
                    _, st = di.di_solve(g, b, D, tol, H, None, opts_w)
                else:
                    _, st = di.di_solve(g, b, D, tol, H, None, opts_c)
                ev[1].record(stream)
                torch.cuda.synchronize()
                if rep >= warmup:
                    times.append(ev[0].elapsed_time(ev[1]))
            res[label] = {"ms": statistics.median(times), "edges": st.edge_diffusions, "levels": st.levels,
                          "warm_used": st.warm_used, "f0_over_b": st.f0_l1 / st.b_l1, "resid": st.resid_l1}
        if infer_parts is None:
            # the inference parts alone on the first held-out graph: features and the network
            feat = torch.empty((n, 9), dtype=torch.float32, device="cuda")
            yv = torch.empty(n, dtype=torch.float32, device="cuda")
            t_feat, t_fwd = [], []
            for rep in range(5):
                flush.zero_()
                ev[0].record(stream)
                model.features(g, b, feat, stream)
                ev[1].record(stream)
                torch.cuda.synchronize()
                t_feat.append(ev[0].elapsed_time(ev[1]))
                flush.zero_()
                ev[0].record(stream)
                model.forward(feat, n, yv, stream)
                ev[1].record(stream)
                torch.cuda.synchronize()
                t_fwd.append(ev[0].elapsed_time(ev[1]))
            fwd_s = statistics.median(t_fwd[1:]) * 1e-3
            peak, peak_src = measured_hbm_peak()
            infer_parts = {"features_ms": statistics.median(t_feat[1:]), "network_ms": fwd_s * 1e3,
                           "network_roofline": {"bound": "hbm", "kernel": "k_mlp_fwd (BF16 mma.sync)",
                                                "achieved": (36 + 4) * n / fwd_s / 1e9, "peak": peak,
                                                "unit": "GB/s", "frac": (36 + 4) * n / fwd_s / 1e9 / peak,
                                                "peak_source": f"{peak_src} (hbm_gbs)",
                                                "tflops": 2 * (16 * 64 + 64 * 64 + 64) * n / fwd_s / 1e12,
                                                "bytes_per_node": "36 B features in, 4 B prediction out"}}
            del feat, yv
        rows.append(res)
        g.close()
        del H, b
    cold = [r["cold"]["ms"] for r in rows]
    warm = [r["warm"]["ms"] for r in rows]
    ratios = [c / w for c, w in zip(cold, warm)]
    model.close()
    return {"workload": WORKLOADS["warmstart"][1], "train_graphs": n_train, "train_nodes": train_nodes,
            "eval_graphs": n_eval, "epochs": epochs, "lr": lr, "tol": "1e-8 |B|_1",
            "timed": "warm: features + network + F0 + solve; cold: solve; L2 flushed before each",
            "cold_ms": statistics.mean(cold), "warm_ms": statistics.mean(warm),
            "speedup": statistics.mean(cold) / statistics.mean(warm),
            "speedup_per_graph": {"mean": statistics.mean(ratios), "min": min(ratios), "max": max(ratios),
                                  "stdev": statistics.pstdev(ratios)},
            "fallbacks": sum(1 - r["warm"]["warm_used"] for r in rows),
            "f0_over_b_mean": statistics.mean(r["warm"]["f0_over_b"] for r in rows),
            "edges_cold": statistics.mean(r["cold"]["edges"] for r in rows),
            "edges_warm": statistics.mean(r["warm"]["edges"] for r in rows),
            "levels_cold": statistics.mean(r["cold"]["levels"] for r in rows),
            "levels_warm": statistics.mean(r["warm"]["levels"] for r in rows),
            "inference": infer_parts,
            "train": {"loss_last_epoch": loss, "seconds": t_train, "generate_and_solve_s": t_gen},
            "per_graph": rows}


def run_native(args, world, rank, local):
    import torch
    import torch.distributed as dist
    from paper_1202_6168_gb300 import binding as di

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    spec, desc = WORKLOADS[args.workload]
    rp, col = gg.generate(spec)
    n, nnz = spec.n, int(len(col))
    b = gg.uniform_b(n, D)
    tol = 1e-8 * b.sum()
    prec = "f64" if args.fp64 else "f32"
    stream = torch.cuda.current_stream()
    opts = di.opts_default(fluid_fp64=1 if args.fp64 else 0, stream=stream.cuda_stream,
                           timing=1 if args.host_loop else 0, l2_window=0 if args.no_l2_window else 1)
    if args.alpha is not None:
        opts.alpha = args.alpha
    if args.workload == "stress-16m":
        # this workload fixes the refinement schedule: an exact FP64 residual every 8 levels
        opts.recompute_every, opts.recompute_drop = 8, 0.0
    if args.recompute_every is not None:
        opts.recompute_every = args.recompute_every
    if args.recompute_drop is not None:
        opts.recompute_drop = args.recompute_drop
    if args.propagation is not None:
        opts.propagation = args.propagation
    if args.push_ratio is not None:
        opts.push_ratio = args.push_ratio
    if args.resweeps is not None:
        opts.resweeps = args.resweeps
    if args.slice_sweeps is not None:
        opts.slice_sweeps = args.slice_sweeps
    if args.exact_residual is not None:
        opts.exact_residual = args.exact_residual
    if args.weighted:
        opts.selection = 1
    if args.dangling:
        opts.dangling = 1

    g = di.Graph.create(rp, col, stream=stream)
    B = torch.from_numpy(b).cuda()
    H = torch.zeros(n, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > 129 MB of L2
    if args.autotune:
        di.autotune(g, B, D, tol, opts)
    shape = di.get_tune(g).as_dict()

    for _ in range(max(args.warmup, 0)):
        di.di_solve(g, B, D, tol, H, None, opts)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    edges = nodes = launches = 0
    levels = []
    for k in range(args.steps):
        flush.zero_()
        ev0[k].record(stream)
        _, st = di.di_solve(g, B, D, tol, H, None, opts)
        ev1[k].record(stream)
        edges += st.edge_diffusions
        nodes += st.node_diffusions
        launches += st.gpu_launches
        levels.append(st.levels)
    barrier()
    clocks = sampler.stop()
    secs = sum(a.elapsed_time(c) for a, c in zip(ev0, ev1)) * 1e-3
    last = st

    secs_max, edges_all = aggregate_over_ranks(secs, edges, world, "cuda")
    solves_all = world * args.steps   # every rank makes args.steps solves

    extras = {}
    if rank == 0 and not args.no_extras:
        if opts.propagation in (3, 7) and not args.fp64:
            # the dominant kernels (selection + push), phases timed on the device
            extras["roofline"], red = phase_roofline(di, g, B, H, tol, opts, prec, n, flush, stream, args.workload)
            if red:
                extras["l2_red"] = red
        else:
            # other modes: CUDA events around every level kernel of host-driven solves
            topt = di.opts_default(fluid_fp64=opts.fluid_fp64, stream=stream.cuda_stream, timing=1,
                                   alpha=opts.alpha, recompute_every=opts.recompute_every,
                                   recompute_drop=opts.recompute_drop,
                                   l2_window=opts.l2_window, propagation=opts.propagation,
                                   push_ratio=opts.push_ratio, exact_residual=opts.exact_residual,
                                   selection=opts.selection, dangling=opts.dangling, resweeps=opts.resweeps,
                                   slice_sweeps=opts.slice_sweeps)
            te = tn = 0
            tpush = trec = tsel = 0.0
            npush = 0
            reps = min(3, max(args.steps, 1))
            for _ in range(reps):
                flush.zero_()
                _, ts = di.di_solve(g, B, D, tol, H, None, topt)
                te += ts.edge_diffusions
                tn += ts.node_diffusions
                tpush += ts.level_seconds
                trec += ts.recompute_seconds
                tsel += ts.select_seconds
                npush += ts.level_launches
            alg_bytes = EDGE_BYTES[prec] * te + NODE_BYTES[prec] * tn + SCAN_BYTES[prec] * n * npush
            achieved = alg_bytes / tpush / 1e9
            peak, peak_src = measured_hbm_peak()
            extras["roofline"] = {"bound": "hbm", "kernel": "level kernels (selection + push)",
                                  "achieved": achieved, "peak": peak, "unit": "GB/s",
                                  "frac": achieved / peak, "peak_source": f"{peak_src} (hbm_gbs)",
                                  "traffic": None, "alg_bytes_per_launch": alg_bytes / max(npush, 1),
                                  "avg_launch_us": 1e6 * tpush / max(npush, 1),
                                  "seconds": {"level": tpush, "of_which_selection": tsel,
                                              "recompute_and_empty_launches": trec},
                                  "measured_by": "CUDA events around every level kernel of host-driven solves"}
        # end to end through the host-buffer entry point: H2D of B, D2H of H
        Bh = torch.from_numpy(b).pin_memory()
        Hh = torch.zeros(n, dtype=torch.float64).pin_memory()
        for _ in range(2):
            di.di_solve_host(g, Bh.data_ptr(), D, tol, Hh.data_ptr(), None, opts)
        torch.cuda.synchronize()
        e_edges, e_secs = 0, 0.0
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, es = di.di_solve_host(g, Bh.data_ptr(), D, tol, Hh.data_ptr(), None, opts)
            e_secs += time.perf_counter() - t0
            e_edges += es.edge_diffusions
        extras["e2e"] = {"value": args.steps / e_secs, "unit": "solves/s",
                         "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n,
                         "ms_per_step": 1e3 * e_secs / args.steps, "edge_diffusions_per_s": e_edges / e_secs,
                         "api": "di_solve_host (pinned host B in, H out; graph resident)"}
        if not args.no_cpu:
            # error of the result against the exact residual bound, and the CPU oracle
            h = H.cpu().numpy()
            from oracle import diter as od
            dang = bool(opts.dangling)
            _, r_cpu = od.residual(rp, col, b, D, h, dangling=dang)
            extras["check"] = {"resid_l1_oracle_fp64": r_cpu, "tol": tol,
                               "stop_ok": bool(r_cpu <= tol * (1 + 1e-9)),
                               "err_bound_rel": r_cpu / (1 - D) / max(h.sum(), 1e-300)}
            # the oracle spreads a dangling diffusion over all N nodes one by one,
            # which is too slow beyond small graphs: no oracle solve then
            if not dang or n <= 100_000:
                # error against the oracle's FP64 solution (solved to 1e-12 |B|_1)
                x = od.d_iteration(rp, col, b, D, tol=1e-12 * b.sum(), dangling=dang).H
                extras["check"]["rel_l1_err_vs_oracle_x"] = float(np.abs(h - x).sum() / np.abs(x).sum())
                extras["cpu_baseline"] = cpu_baseline(rp, col, b, tol, dang)
        if args.workload == "web-1m" and not args.no_stress:
            extras["stress_16m"] = stress_leg(args, di, stream, flush)
        if args.workload == "web-1m" and not args.no_cfg5:
            extras["warmstart_cfg5"] = warmstart_study(args, di, stream, flush, args.ws_train, args.ws_eval,
                                                       args.ws_epochs, args.ws_lr)

    if rank == 0:
        info = g.info()
        ms = 1e3 * secs_max / args.steps
        line = {"metric": "solves_per_s_to_tol", "value": solves_all / secs_max, "unit": "solves/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": prec, "data": "synthetic",
                "config": {"workload": desc, "n": n, "nnz": nnz, "n_dangling": info["n_dangling"],
                           "n_hot_targets": info["n_hot"], "d": D, "tol": tol, "tol_rel_b_l1": 1e-8,
                           "fluid": prec, "history": "f64", "recompute_every": opts.recompute_every,
                           "recompute_drop": opts.recompute_drop,
                           "alpha": opts.alpha, "l2": "flushed (256 MiB write) before each timed step",
                           "l2_window": bool(opts.l2_window),
                           "propagation": ["auto: binned gather / push", "auto: flat gather / push",
                                           "push only", "asynchronous push",
                                           "asynchronous push, warp-level tiles",
                                           "fused select + push, one launch per level",
                                           "node-ordered chunks, on-chip window and hot slots, one launch "
                                           "per level",
                                           "asynchronous push, persistent cooperative level loop"][opts.propagation],
                           "push_ratio": opts.push_ratio, "resweeps": opts.resweeps, "slice_sweeps": last.slice_sweeps,
                           "push_shape": dict(shape, chosen_by="di_autotune" if args.autotune else "default"),
                           "exact_residual": ["auto", "binned gather", "source-blocked gather"][opts.exact_residual],
                           "selection": ["|F_i| >= T", "|F_i| / ((in_i+1)(out_i+1)) >= T"][opts.selection],
                           "dangling": ["zero columns", "uniform 1/N completion"][opts.dangling],
                           "level_loop": "host-driven" if args.host_loop else "CUDA graph (WHILE/IF nodes)",
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
                "time_to_tol_ms": ms,
                "edge_diffusions_per_s": edges_all / secs_max,
                "edge_diffusions_per_step": edges / args.steps,
                "normalised_iterations": edges / args.steps / nnz,
                "levels": levels[-1], "passes": last.body_iterations, "recomputes": last.recomputes,
                "gpu_launches": launches, "clocks": clocks}
        line.update(extras)
        print(json.dumps(line), flush=True)
    g.close()
    if world > 1:
        dist.destroy_process_group()


def batch_inputs():
    specs = gg.batch_specs(64, seed=0)
    csrs = [gg.generate(sp) for sp in specs]
    rhs = []
    for sp in specs:
        for src in gg.batch_sources(sp.n, 4, seed=sp.seed):
            rhs.append((len(rhs) // 4, int(src)))
    return specs, csrs, rhs


def run_batch(args, world, rank, local):
    """One step = di_solve_batched over all 256 (graph, source) items."""
    import torch
    import torch.distributed as dist
    from paper_1202_6168_gb300 import binding as di

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    specs, csrs, rhs = batch_inputs()
    stream = torch.cuda.current_stream()
    prec = "f64" if args.fp64 else "f32"
    opts = di.opts_default(fluid_fp64=1 if args.fp64 else 0, stream=stream.cuda_stream)
    if args.slice_sweeps is not None:
        opts.slice_sweeps = args.slice_sweeps
    graphs = [di.Graph.create(rp, col, stream=stream) for rp, col in csrs]
    batch = di.Batch(graphs, [4] * len(graphs), stream=stream)
    B, H, tols = [], [], []
    for gi, src in rhs:
        n = specs[gi].n
        b = torch.zeros(n, dtype=torch.float64, device="cuda")
        b[src] = 1.0 - D
        B.append(b)
        H.append(torch.zeros(n, dtype=torch.float64, device="cuda"))
        tols.append(1e-8 * (1.0 - D))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    # frontier tile shape of the batched push, chosen by timing (the autotuner)
    tune, tune_s = di.batch_autotune(batch, B, D, tols, H, opts)
    for _ in range(max(args.warmup, 0)):
        di.di_solve_batched(batch, B, D, tols, H, opts)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    torch.cuda.synchronize()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    edges = launches = nodes = levels_sum = 0
    for k in range(args.steps):
        flush.zero_()
        ev0[k].record(stream)
        _, st, tot = di.di_solve_batched(batch, B, D, tols, H, opts)
        ev1[k].record(stream)
        edges += tot.edge_diffusions
        nodes += tot.node_diffusions
        levels_sum += tot.body_iterations
        launches += tot.gpu_launches
    torch.cuda.synchronize()
    clocks = sampler.stop()
    secs = sum(a.elapsed_time(c) for a, c in zip(ev0, ev1)) * 1e-3
    secs_rank = secs
    secs, edges_all = aggregate_over_ranks(secs, edges, world, "cuda")
    extras = {}
    if rank == 0:
        # whole-solve roofline: every launch of the batched solve, algorithmic bytes
        # of the level kernels (per edge, per node, and a scan of the union per level)
        n_union = batch.info()["n_union"]
        alg = EDGE_BYTES[prec] * edges + NODE_BYTES[prec] * nodes + SCAN_BYTES[prec] * n_union * levels_sum
        peak, peak_src = measured_hbm_peak()
        extras["roofline"] = {"bound": "hbm", "kernel": "whole batched solve (k_bscan_level + k_bpush + "
                                                        "exact residuals, all launches)",
                              "achieved": alg / secs_rank / 1e9, "peak": peak, "unit": "GB/s",
                              "frac": alg / secs_rank / 1e9 / peak, "peak_source": f"{peak_src} (hbm_gbs)",
                              "traffic": None, "alg_bytes_per_step": alg / args.steps,
                              "measured_by": "CUDA events around every timed di_solve_batched"}
    if rank == 0 and not args.no_extras:
        # the same 256 solves one di_solve call at a time
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        seq_edges = 0
        for (gi, _), b, h, tol in zip(rhs, B, H, tols):
            _, s1 = di.di_solve(graphs[gi], b, D, tol, h, None, opts)
            seq_edges += s1.edge_diffusions
        torch.cuda.synchronize()
        seq = time.perf_counter() - t0
        extras["sequential_di_solve"] = {"seconds": seq, "edge_diffusions": seq_edges,
                                         "value": seq_edges / seq, "unit": "edge_diffusions/s"}
        # exactness of every item: the oracle's residual of the returned H
        from oracle import diter as od
        worst = 0.0
        _, st, _ = di.di_solve_batched(batch, B, D, tols, H, opts)
        for (gi, src), h, tol in zip(rhs, H, tols):
            rp, col = csrs[gi]
            b = gg.personalised_b(specs[gi].n, src, D)
            _, r = od.residual(rp, col, b, D, h.cpu().numpy())
            worst = max(worst, r / tol)
        extras["check"] = {"max_resid_over_tol_oracle_fp64": worst, "stop_ok": bool(worst <= 1 + 1e-9)}
        # the oracle on a bounded sample: the items of the smallest graphs
        order = sorted(range(len(specs)), key=lambda g: specs[g].n)
        t0 = time.perf_counter()
        cpu_edges, items_done = 0, 0
        for gi in order:
            rp, col = csrs[gi]
            for (g2, src) in rhs:
                if g2 != gi:
                    continue
                r = od.d_iteration(rp, col, gg.personalised_b(specs[gi].n, src, D), D, tol=1e-8 * (1.0 - D))
                cpu_edges += r.edge_diffusions
                items_done += 1
            if time.perf_counter() - t0 > 15.0:
                break
        dt = time.perf_counter() - t0
        extras["cpu_baseline"] = {"value": cpu_edges / dt, "unit": "edge_diffusions/s", "cores": 1,
                                  "kind": "oracle", "sample": f"{items_done} items of the smallest graphs, "
                                                              f"{dt:.1f} s"}
    if rank == 0:
        info = batch.info()
        line = {"metric": "edge_diffusions_per_s", "value": edges_all / secs, "unit": "edge_diffusions/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": prec, "data": "synthetic",
                "config": {"workload": WORKLOADS["batch-64x4"][1], "items": info["n_items"],
                           "n_union": info["n_union"], "nnz_union": info["nnz_union"],
                           "tol": "1e-8 |B|_1 per item", "l2": "flushed (256 MiB write) before each timed step",
                           "recompute_every": opts.recompute_every, "recompute_drop": opts.recompute_drop,
                           "push_shape": dict(tune.as_dict(), chosen_by="di_batch_autotune", best_s=tune_s),
                           "level_loop": "CUDA graph (WHILE/IF nodes)",
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
                "time_to_tol_ms": 1e3 * secs / args.steps, "gpu_launches": launches, "clocks": clocks}
        line.update(extras)
        print(json.dumps(line), flush=True)
    batch.close()
    for g in graphs:
        g.close()
    if world > 1:
        dist.destroy_process_group()


def run_warmstart(args, world, rank, local):
    """Time to |F|_1 <= 1e-8 |B|_1 with the learned warm start (features, network,
    F0 and the solve, all timed) against the zero start, on held-out graphs."""
    import torch
    from paper_1202_6168_gb300 import binding as di

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    r = warmstart_study(args, di, stream, flush, args.ws_train, args.ws_eval, args.ws_epochs, args.ws_lr,
                        reps=max(args.steps, 1), warmup=max(args.warmup, 1))
    line = {"metric": "time_to_tol_ms", "value": r["warm_ms"], "unit": "ms",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["warm_ms"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {k: r[k] for k in ("workload", "train_graphs", "train_nodes", "eval_graphs", "epochs", "lr",
                                         "tol", "timed")}}
    line.update({k: v for k, v in r.items() if k not in line["config"]})
    print(json.dumps(line), flush=True)


def run_kpid_sim(args, world, rank, local):
    """The paper's evaluation of its distributed scheme (Sec. 3), on the host
    cores: time in normalised iterations (steps x PID_Speed / L) to the target
    error 1/N for K = 1..64 PIDs, uniform and cost-balanced ranges; the
    speed-up over one PID, each PID's operations and the idle share, and the
    impact of Delay_Proba at K = 8."""
    from paper_1202_6168_gb300 import kpid_sim as ks
    spec, desc = WORKLOADS["kpid-sim"]
    rp, col = gg.generate(spec)
    n, L = spec.n, int(len(col))
    b = gg.uniform_b(n, D)
    tol = (1.0 - D) / n                      # r / (1 - d) <= 1 / N
    rows, secs = [], 0.0
    one = None
    grid = [(1, "uniform", 0.0)] + [(K, kind, 0.0) for K in (2, 4, 8, 16, 32, 64) for kind in ("uniform", "cb")]
    grid += [(8, kind, p) for p in (0.5, 0.8) for kind in ("uniform", "cb")]
    for K, kind, p in grid:
        bounds = ks.uniform_bounds(n, K) if kind == "uniform" else ks.cb_bounds(rp, K)
        t0 = time.perf_counter()
        r = ks.simulate(rp, col, b, D, tol=tol, bounds=bounds, delay_proba=p, seed=7)
        secs += time.perf_counter() - t0
        if one is None:
            one = r.normalised_time
        rows.append({"K": K, "partition": kind, "delay_proba": p, "status": r.status,
                     "normalised_time": r.normalised_time, "speedup": one / r.normalised_time,
                     "steps": r.steps, "max_pid_cost": float(r.ops.max()) / L, "total_cost": float(r.ops.sum()) / L,
                     "idle_share": r.idle_share, "transmissions": int(r.sends.sum()), "resid": r.resid_l1})
    best = max((row for row in rows if row["delay_proba"] == 0.0), key=lambda row: row["speedup"])
    line = {"metric": "kpid_speedup", "value": best["speedup"], "unit": "x (1-PID time / K-PID time)",
            "n_gpus": 0, "steps": len(rows), "warmup": 0, "ms_per_step": 1e3 * secs / len(rows),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "n": n, "nnz": L, "tol": tol, "best": {"K": best["K"],
                       "partition": best["partition"]}, "cores": os.cpu_count(),
                       "timed": "wall clock of every simulation (host cores, OpenMP over the PIDs)"},
            "rows": rows, "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def run_kpid(args, world, rank, local):
    """K-PID asynchronous D-iteration: for every K and partition, the time to
    tol and each PID's elementary diffusions normalised by L (the paper's
    normalised iterations, Sec. 2.4), against the one-PID solve."""
    import torch
    from paper_1202_6168_gb300 import binding as di

    torch.cuda.set_device(local)
    spec, desc = WORKLOADS[args.workload]
    rp, col = gg.generate(spec)
    n, nnz = spec.n, int(len(col))
    b = gg.uniform_b(n, D)
    tol = 1e-8 * b.sum()
    stream = torch.cuda.current_stream()
    g = di.Graph.create(rp, col, stream=stream)
    B = torch.from_numpy(b).cuda()
    H = torch.zeros(n, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    opts = di.opts_default(stream=stream.cuda_stream, dangling=1 if args.dangling else 0)
    rows = []
    for K, kind in ((1, 0), (2, 0), (2, 1), (4, 0), (4, 1), (8, 0), (8, 1)):
        times = []
        for rep in range(max(args.warmup, 1) + max(args.steps, 1)):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, st, ops, sends = di.di_solve_partitioned(g, B, D, tol, H, K, kind, None, opts)
            dt = time.perf_counter() - t0
            if rep >= max(args.warmup, 1):
                times.append(dt)
        rows.append({"K": K, "partition": ["uniform", "cost-balanced"][kind], "ms": 1e3 * statistics.median(times),
                     "rounds": st.body_iterations, "recomputes": st.recomputes,
                     "normalised_cost_per_pid": [float(v) / nnz for v in ops],
                     "max_pid_cost": float(ops.max()) / nnz, "total_cost": float(ops.sum()) / nnz,
                     "transmissions": [int(v) for v in sends], "resid": st.resid_l1,
                     "gpu_launches": st.gpu_launches})
    g.close()
    one = rows[0]["max_pid_cost"]
    best = min(rows[1:], key=lambda r: r["max_pid_cost"])
    line = {"metric": "max_pid_normalised_iterations", "value": best["max_pid_cost"], "unit": "iterations (ops/L)",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": best["ms"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": desc, "n": n, "nnz": nnz, "tol": "1e-8 |B|_1", "best": {"K": best["K"],
                       "partition": best["partition"]}, "level_loop": "CUDA graph (WHILE/IF nodes), one round per level",
                       "dangling": ["zero columns", "uniform 1/N completion"][opts.dangling],
                       "timed": "wall clock around each di_solve_partitioned (synchronous)",
                       "l2": "flushed (256 MiB write) before each timed solve"},
            "one_pid_cost": one, "cost_split": best["max_pid_cost"] / one, "rows": rows,
            "gpu_launches": best["gpu_launches"]}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.workload == "kpid-sim":
        # a host-core simulation in both arms: the reference arm runs the oracle's
        # lock-step emulation (see run_reference_kpid_sim)
        if rank == 0:
            (run_reference_kpid_sim if args.impl == "reference" else run_kpid_sim)(args, world, rank, local)
    elif args.workload == "kpid-1m" and args.impl != "reference":
        if rank == 0:
            run_kpid(args, world, rank, local)
    elif args.workload == "warmstart" and args.impl != "reference":
        if rank == 0:
            run_warmstart(args, world, rank, local)
    elif args.workload == "batch-64x4" and args.impl != "reference":
        run_batch(args, world, rank, local)
    elif args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_native(args, world, rank, local)


if __name__ == "__main__":
    main()
