#!/usr/bin/env python
"""Benchmark of the multi-body Nystrom solve on B300.

One step = one full mixed-precision solve of a seeded scene: self-block
assembly for the wavenumber, incident right-hand sides, GMRES with the FP32
operator inside FP64 iterative refinement to ||b - A mu|| <= 1e-10 ||b|| (the
metric asks for 1e-8 relative error; the error against the FP64 solve is
reported), and
the far field on 200 x 200 directions.  Geometry (qams_set_bodies) is
resident before the timed region; the e2e figure repeats the step through
the C ABI starting from host descriptors and ending with the densities and
far field copied back to host memory.

value = Nystrom pair-interactions per second over the whole step: the
pair-sum evaluations of every operator apply in the solve (N^2 - sum n_b^2
per apply and right-hand side) divided by the step time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Nyström pair-interactions/s, solves/s at 1e-8 rel err; p50/p99 solve latency"
UNIT = "pair-interactions/s"
FAR_DIRS = 200  # 200 x 200 far-field directions (Sec. 6)


def far_directions(n=FAR_DIRS):
    import numpy as np
    th = (np.arange(n) + 0.5) * math.pi / n
    ph = np.arange(n) * 2 * math.pi / n
    T, P = np.meshgrid(th, ph, indexing="ij")
    return np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1).reshape(-1, 3)


class ClockSampler:
    """nvidia-smi samples of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


def fp64_peak_tflops(torch):
    """Dense FP64 rate measured on this GPU (cuBLAS DGEMM 8192^3, best of 5)."""
    n = 8192
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    del a, b
    return 2.0 * n ** 3 / best / 1e12


# FP32 pair (R = 1): 34 FP32 operations + 4 MUFU (rsqrt, rcp, sin, cos) + 4 FMA per
# right-hand side; FP64 pair: 44 FP64 operations + rsqrt (counted as 4) incl. the
# table-driven e^{ik rho} (15) -- counted from the kernel sources.
FP32_OPS_PER_PAIR = 34
FP64_OPS_PER_PAIR = 48
# float-float pair: ~640 FP32 operations (the e^{ik rho} evaluation ~195, the
# accumulation 72 per right-hand side) -- counted from the kernel source
FF_OPS_PER_PAIR = 640


def _time_ms(torch, fn, reps=5):
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def kernel_rooflines(torch, q, ctx, sc, N, R, pairs, device):
    """Pair sums (ALU: FP32 pipe + MUFU, FP64 pipe) and block products (HBM),
    each timed alone with CUDA events on the current stream."""
    props = torch.cuda.get_device_properties(device)
    sms = props.multi_processor_count
    f = 2.032e9  # maximum SM clock (the sampled clock sits there under this load)
    hbm = measured_peaks()[0]["hbm_gbs"]
    s32 = torch.randn((N, R), dtype=torch.complex64, device="cuda")
    y32 = torch.empty_like(s32)
    s64 = s32.to(torch.complex128)
    y64 = torch.empty_like(s64)
    t32 = _time_ms(torch, lambda: ctx.pairsum(s32, y32, q.PREC_FP32))
    t64 = _time_ms(torch, lambda: ctx.pairsum(s64, y64, q.PREC_FP64), reps=2)
    yff = torch.empty_like(s64)
    tff = _time_ms(torch, lambda: ctx.pairsum(s64, yff, q.PREC_FF), reps=3)
    ff_diff = float(torch.linalg.norm(yff - y64) / torch.linalg.norm(y64))
    peakff = 128 * sms * f / (FF_OPS_PER_PAIR + 72 * (R - 1))
    # FP32: min over the FP32 pipe (128 lanes/SM/clk) and MUFU (16/SM/clk, 4 per pair)
    peak32 = min(128 * sms * f / (FP32_OPS_PER_PAIR + 4 * R), 16 * sms * f / 4)
    peak64 = 2 * sms * f / (FP64_OPS_PER_PAIR + 4 * (R - 1))  # FP64 pipe: 2 lanes/SM/clk
    entries = sum(b.n_nodes ** 2 for b in sc.bodies)
    tb32 = _time_ms(torch, lambda: ctx.selfblock_apply(s32, y32, q.PREC_FP32))
    tb64 = _time_ms(torch, lambda: ctx.selfblock_apply(s64, y64, q.PREC_FP64))
    reps16 = (R + 15) // 16
    gb32 = entries * 8 * reps16 / (tb32 / 1e3) / 1e9
    gb64 = entries * 16 * reps16 / (tb64 / 1e3) / 1e9
    return {
        "pairsum_f32_kernel": {"ms": t32, "pairs_per_s": pairs / (t32 / 1e3), "bound": "alu",
                               "peak_pairs_per_s": peak32, "frac": pairs / (t32 / 1e3) / peak32},
        "pairsum_f64_kernel": {"ms": t64, "pairs_per_s": pairs / (t64 / 1e3), "bound": "alu (FP64 pipe)",
                               "peak_pairs_per_s": peak64, "frac": pairs / (t64 / 1e3) / peak64},
        "pairsum_ff_kernel": {"ms": tff, "pairs_per_s": pairs / (tff / 1e3), "bound": "alu (FP32 pipe)",
                              "peak_pairs_per_s": peakff, "frac": pairs / (tff / 1e3) / peakff,
                              "rel_diff_vs_fp64_kernel": ff_diff},
        "block_apply_kernel<float2>": {"ms": tb32, "achieved": gb32, "peak": hbm, "unit": "GB/s",
                                       "bound": "hbm", "frac": gb32 / hbm},
        # complex128 entries: 4 FP64 operations per entry and right-hand side put the
        # FP64 pipe (2 lanes/SM/clk) below the HBM stream
        "block_apply_kernel<double2>": {"ms": tb64, "achieved": entries * R / (tb64 / 1e3), "unit": "entries/s",
                                        "bound": "alu (FP64 pipe)", "peak": 2 * sms * f / 4,
                                        "frac": entries * R / (tb64 / 1e3) / (2 * sms * f / 4),
                                        "hbm_gbs": gb64},
        "note": "pair peaks from the op counts above at the maximum SM clock; HBM peak of measured",
    }


def assembly_flops(scene, counts):
    """Algorithmic FP64 operations of one self-block assembly, counted from the
    kernel's dense loops: per modal outer node the cosine transforms,
    convolutions, theta-coefficients and accumulation; per far outer node the
    azimuthal samples and accumulation; per row and near panel the inverse
    DFT.  ``counts`` = (modal, far) outer nodes reported by the library.
    Transcendental calls, the Q recursions and index arithmetic are not
    counted, so this undercounts the work."""
    n_modal, n_far = counts
    per_node = per_far = flush = 0.0
    wsum = 0.0
    for b in scene.bodies:
        order, nth, npan = b.order, b.n_theta, b.n_panels
        N = nth // 2
        if getattr(b, "kind", 0) == 1:
            rmax = sum(abs(A) + abs(B) for (_, A, B) in b.series[3])
        else:
            rmax = b.base_radius * (1 + sum(abs(x) for x in b.mode_cos) + sum(abs(x) for x in b.mode_sin))
        n1 = math.ceil(1.3 * scene.k * rmax + 16.0)
        M2 = n1 + 8
        w = b.n_nodes
        wsum += w
        # cosine DFTs of 3 smooth factors, three convolutions (modes 0..N+1, one to N+2),
        # theta-coefficients of the two integrands, accumulation
        per_node += w * (6 * (n1 + 2) * (M2 - 1) + 2 * (3 * (N + 2) + 1) * (2 * n1 + 1) + 40 * nth
                         + 8 * order * nth)
        per_far += w * (30 * nth + 8 * order * nth)
        # every row: inverse DFT per near panel
        near = sum(min(npan - 1, p + 1) - max(0, p - 1) + 1 for p in range(npan)) * order * nth
        flush += near * 8 * order * nth * nth
    return n_modal * per_node / wsum + n_far * per_far / wsum + flush


def max_over_ranks(x: float, dist, device: str) -> float:
    """Largest value of x over all ranks (the job is as slow as its slowest rank)."""
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(pair_evals_per_rank: float, world: int, elapsed_max: float) -> float:
    """Whole-job pair-interactions/s: every rank solves its own request of the
    same size (replicas, weak scaling), timed by the slowest rank."""
    return pair_evals_per_rank * world / elapsed_max


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    import paper_2606_31380_b300 as q
    import scenes

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    sc = scenes.config(args.config, request_id=rank)  # replicas: independent request per rank
    if args.bodies:
        # a smaller case of the same workload (profiling captures)
        sc = scenes.Scene(sc.name + f" (first {args.bodies} bodies)", sc.bodies[:args.bodies], sc.k, sc.eta,
                          sc.directions)
    R = sc.n_rhs
    xh = far_directions()
    M = xh.shape[0]
    ctx = q.Context(local_rank)
    ctx.set_bodies(sc.bodies)
    ctx.set_wavenumber(sc.k, sc.eta)
    N = ctx.N
    pairs = sc.pair_count()
    b = torch.zeros((N, R), dtype=torch.complex128, device="cuda")
    mu = torch.zeros_like(b)
    u = torch.zeros((M, R), dtype=torch.complex128, device="cuda")
    stream = torch.cuda.current_stream()

    def step(record=None):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record()
        ctx.assemble()
        ev[1].record()
        ctx.incident_plane(sc.directions, b)
        st = ctx.solve(b, mu, q.PREC_FP32, tol=args.tol)
        ev[2].record()
        ctx.farfield(mu, xh, u)
        ev[3].record()
        if record is not None:
            record.append((ev, st))
        return st

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    launches0 = q.kernel_launches()
    recs = []
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record()
    for _ in range(args.steps):
        step(recs)
    t1.record()
    torch.cuda.synchronize()
    launches = q.kernel_launches() - launches0
    clk = clocks.stop()
    elapsed = t0.elapsed_time(t1) / 1e3
    if dist:
        elapsed = max_over_ranks(elapsed, dist, "cuda")
        dist.barrier()
    step_ms = [r[0][0].elapsed_time(r[0][3]) for r in recs]
    asm_ms = [r[0][0].elapsed_time(r[0][1]) for r in recs]
    solve_ms = [r[0][1].elapsed_time(r[0][2]) for r in recs]
    ff_ms = [r[0][2].elapsed_time(r[0][3]) for r in recs]
    applies = [r[1]["applies_fp32"] + r[1]["applies_fp64"] for r in recs]
    pair_evals = sum(a * pairs * R for a in applies)
    value = job_value(pair_evals, world, elapsed)

    # accuracy of the mixed result against the plain FP64 GPU solve of the same scene
    mu64 = torch.zeros_like(b)
    ctx.solve(b, mu64, q.PREC_FP64, tol=1e-12)
    rel_err = float(torch.linalg.norm(mu - mu64) / torch.linalg.norm(mu64))

    # dominant kernel: self-block assembly (FP64 ALU) -- time it alone with events
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ctx.assemble()
    e1.record()
    torch.cuda.synchronize()
    asm_alone = e0.elapsed_time(e1) / 1e3
    asm_counts = ctx.assembly_counts()
    flops = assembly_flops(sc, asm_counts)
    # FP64 peak from the unit counts: 2 FP64 lanes per clock per SM (the issue rate ncu
    # reports for DFMA) x 2 FLOP x SMs x the maximum SM clock
    sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
    peak64 = 2 * 2 * sms * 2.032e9 / 1e12
    # cuBLAS DGEMM rate on this GPU (1.05 TFLOP/s when last measured); off by default so
    # that the run's launch list holds only the library's own kernels
    peak64_meas = fp64_peak_tflops(torch) if args.measure_fp64_peak else 1.05

    # FP32 apply pair rate (hot loop of the inner solver)
    x32 = torch.randn((N, R), dtype=torch.complex64, device="cuda")
    y32 = torch.empty_like(x32)
    ctx.apply(x32, y32, q.PREC_FP32)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(5):
        ctx.apply(x32, y32, q.PREC_FP32)
    e1.record()
    torch.cuda.synchronize()
    apply_ms = e0.elapsed_time(e1) / 5

    # the other hot kernels alone, each against its own roofline
    kernels = kernel_rooflines(torch, q, ctx, sc, N, R, pairs, local_rank)

    # e2e: through the C ABI from host descriptors to host results
    e2e_steps = max(1, min(args.steps, 3))
    mu_h = torch.empty((N, R), dtype=torch.complex128, pin_memory=True)
    u_h = torch.empty((M, R), dtype=torch.complex128, pin_memory=True)
    torch.cuda.synchronize()
    t_start = time.perf_counter()
    e2e_pairs = 0
    for _ in range(e2e_steps):
        c2 = q.Context(local_rank)
        c2.set_bodies(sc.bodies)
        c2.set_wavenumber(sc.k, sc.eta)
        c2.assemble()
        bb = torch.zeros((N, R), dtype=torch.complex128, device="cuda")
        c2.incident_plane(sc.directions, bb)
        mm = torch.zeros_like(bb)
        st = c2.solve(bb, mm, q.PREC_FP32, tol=args.tol)
        uu = torch.zeros((M, R), dtype=torch.complex128, device="cuda")
        c2.farfield(mm, xh, uu)
        mu_h.copy_(mm, non_blocking=True)
        u_h.copy_(uu, non_blocking=True)
        torch.cuda.synchronize()
        c2.close()
        e2e_pairs += (st["applies_fp32"] + st["applies_fp64"]) * pairs * R
    e2e_t = time.perf_counter() - t_start
    h2d = sum(8 * (9 + 3 + 6 + len(bd.mode_cos) + len(bd.mode_sin)) for bd in sc.bodies) + 8 * 3 * R + 8 * 3 * M
    d2h = 16 * N * R + 16 * M * R

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    ms = elapsed / args.steps * 1e3
    lat = sorted(step_ms)

    def pct(p):
        return lat[min(len(lat) - 1, int(math.ceil(p / 100 * len(lat))) - 1)]

    achieved = flops / asm_alone / 1e12
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64",
        "precision_note": ("f32 inner operator; f64 and float-float (pairs of f32) in the assembly, "
                           "refinement residual and far field; f64 Krylov basis"),
        "data": "synthetic (seeded quasi-axisymmetric bodies)",
        "config": {"workload": sc.name, "n_bodies": len(sc.bodies), "N": N, "R": R, "k": sc.k, "eta": sc.eta,
                   "tol": args.tol, "far_field_dirs": M, "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (self blocks %.2f GB resident)" % (
                       sum(bd.n_nodes ** 2 for bd in sc.bodies) * 24 / 1e9)},
        "solves_per_s": args.steps * world / elapsed,
        "latency_ms": {"p50": pct(50), "p99": pct(99)},
        "breakdown_ms": {"assembly": statistics.mean(asm_ms), "solve": statistics.mean(solve_ms),
                         "far_field": statistics.mean(ff_ms)},
        "solver": {"applies_per_solve": statistics.mean(applies), "iterations": recs[-1][1]["iterations"],
                   "refinements": recs[-1][1]["refinements"], "rel_residual": recs[-1][1]["rel_residual"],
                   "rel_err_vs_fp64_gpu": rel_err},
        "fp32_apply": {"ms": apply_ms, "pairs_per_s": pairs / (apply_ms / 1e3),
                       "pair_rhs_per_s": pairs * R / (apply_ms / 1e3)},
        "assembly_outer_nodes": {"modal": asm_counts[0], "far": asm_counts[1]},
        "roofline": {"kernel": "selfblock_kernel (FP64 self-block assembly)", "bound": "alu",
                     "achieved": achieved, "peak": peak64, "unit": "TFLOP/s", "frac": achieved / peak64,
                     "traffic": None,
                     "peak_note": ("derived: 2 FP64 lanes/clk/SM x 2 FLOP x %d SMs x 2.032 GHz (nominal 1.25); "
                                   "cuBLAS DGEMM %.3f TFLOP/s on this GPU%s"
                                   % (sms, peak64_meas, "" if args.measure_fp64_peak else " (earlier measurement)"))},
        "e2e": {"value": e2e_pairs / e2e_t, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
        "kernels": kernels,
    }
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(sc, args.cpu_seconds)
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def cpu_baseline(sc, seconds: float):
    """The FP64 oracle as it stands, on this host's cores: its explicit pair sum
    over a bounded sample of target rows of the same scene, in pair-interactions/s."""
    import numpy as np

    from oracle import operator as op
    from oracle.geometry import body_nodes
    import scenes

    nodes = [body_nodes(b) for b in sc.bodies]
    N = sum(n.count for n in nodes)
    sigma = scenes.rhs_seeded(N, sc.n_rhs, 1)
    rng = np.random.default_rng(0)
    done_pairs, t0 = 0, time.perf_counter()
    off = op.body_offsets(nodes)
    rows_done = 0
    while time.perf_counter() - t0 < seconds:
        rows = rng.integers(0, N, 16)
        op.pair_sum(nodes, sigma, sc.k, sc.eta, targets=rows)
        for g in rows:
            b = int(np.searchsorted(off, g, side="right") - 1)
            done_pairs += N - nodes[b].count
        rows_done += 16
    t = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": done_pairs / t, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{rows_done} random target rows x all other-body sources of the same scene "
                      f"(explicit FP64 pair sum, numpy), {t:.1f} s"}


def run_reference(args, rank, world):
    """The oracle (the reference arm for this build) on the host cores."""
    if rank != 0:
        return
    import scenes
    sc = scenes.config(args.config)
    for _ in range(args.warmup):
        cpu_baseline(sc, 1.0)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(sc, args.cpu_seconds / max(1, args.steps)))
    elapsed = time.perf_counter() - t0
    v = statistics.mean(x["value"] for x in vals)
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded quasi-axisymmetric bodies)",
           "config": {"workload": sc.name, "N": sc.n_nodes, "R": sc.n_rhs, "k": sc.k},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": vals[0]["cores"], "kind": "oracle",
                            "sample": vals[0]["sample"]},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_serve(args):
    """Serving stream: seeded requests with 10..max_bodies bodies, {16x32, 24x48}
    nodes, k ~ U[1, 15], 1..16 RHS, each a full mixed solve to 1e-11 plus 400
    far-field directions.  A burst (all requests at once) measures the
    saturated rate; Poisson arrivals at 0.8 of it give the latency distribution."""
    import numpy as np

    import paper_2606_31380_b300 as q
    import scenes

    reqs = [scenes.serving_request(i, max_bodies=args.serve_max_bodies) for i in range(args.serve_requests)]
    far = scenes.fibonacci_directions(400)
    srv = q.Server(0, 0, slots=args.serve_slots)
    srv.wait(srv.submit(reqs[0], far))  # warm-up
    t0 = time.perf_counter()
    tickets = [srv.submit(r, far) for r in reqs]
    burst = [srv.wait(t) for t in tickets]
    t_burst = time.perf_counter() - t0
    sat = len(reqs) / t_burst
    rng = np.random.default_rng(31380)
    lam = 0.8 * sat
    arrivals = np.cumsum(rng.exponential(1.0 / lam, size=len(reqs)))
    t0 = time.perf_counter()
    tickets = []
    for r, at in zip(reqs, arrivals):
        dt = at - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        tickets.append(srv.submit(r, far))
    res = [srv.wait(t) for t in tickets]
    t_stream = time.perf_counter() - t0
    srv.close()
    lat = np.array([r["latency_ms"] for r in res])
    ok = all(r["status"] == 0 for r in res + burst)
    failed = [{"request": i % len(reqs), "phase": "burst" if i < len(burst) else "stream", "status": r["status"],
               "iterations": r["iterations"], "refinements": r["refinements"], "rel_residual": r["rel_residual"],
               "k": reqs[i % len(reqs)].k, "n_nodes": r["n_nodes"]}
              for i, r in enumerate(burst + res) if r["status"] != 0]
    out = {"metric": "serving solves/s and p50/p99 solve latency", "value": len(reqs) / t_stream,
           "unit": "solves/s", "higher_is_better": True, "n_gpus": 1, "data": "synthetic (seeded requests)",
           "config": {"workload": f"{len(reqs)} requests, 10..{args.serve_max_bodies} bodies, "
                                  "{16x32, 24x48} nodes, k ~ U[1,15], 1..16 RHS, tol 1e-11",
                      "slots": args.serve_slots, "arrival_rate_per_s": lam},
           "saturated_solves_per_s": sat, "latency_ms": {"p50": float(np.percentile(lat, 50)),
                                                         "p99": float(np.percentile(lat, 99))},
           "mean_nodes": float(np.mean([r["n_nodes"] for r in res])), "all_ok": ok, "failed": failed}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, default=1, help="workload index (1 = 16 bodies x 2048 nodes, k = 5)")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--measure-fp64-peak", action="store_true", help="time a cuBLAS DGEMM for the FP64 peak note")
    ap.add_argument("--bodies", type=int, default=0, help="use only the first B bodies (small profiling case)")
    ap.add_argument("--tol", type=float, default=1e-10,
                    help="relative FP64 residual target of the mixed solve (the metric asks 1e-8 relative error)")
    ap.add_argument("--serve", action="store_true", help="serving stream instead of the single-solve step")
    ap.add_argument("--serve-requests", type=int, default=24)
    ap.add_argument("--serve-max-bodies", type=int, default=40)
    ap.add_argument("--serve-slots", type=int, default=4)
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus if args.gpus == 1 else 1)))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.serve:
        if rank == 0:
            run_serve(args)
    elif args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
