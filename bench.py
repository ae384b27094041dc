#!/usr/bin/env python
"""Benchmark of the multi-body Nystrom solve on B300.

One step = one full mixed-precision solve of a seeded scene: self-block
assembly for the wavenumber, incident right-hand sides, the block-Jacobi
preconditioner, GMRES with the FP32 operator inside FP64 iterative
refinement to ||b - A mu|| <= 1e-10 ||b|| (the metric asks for 1e-8
relative error), and the far field on 200 x 200 directions.  The default
workload is the largest configuration of the metric: 1000 bodies x 512
nodes (N = 512,000), k = 3, 4 incident directions.  The 16- and 100-body
workloads are measured in the same run (a few solves each) and reported
under "other_workloads".  Per result the accuracy is given as the
FP64-accurate residual of the returned densities and their distance to a
solve refined to 1e-13 (and, where it is affordable, to the plain FP64
GPU solve).  Geometry (qams_set_bodies) is resident before the timed
region; the e2e figure repeats the step through the C ABI starting from
host descriptors and ending with the densities and far field copied back
to host memory.

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


def pair_roofline(sms: int, f_hz: float, R: int) -> float:
    """Pair-interactions/s ceiling of the FP32 pair sum at R right-hand sides:
    min over the FP32 pipe (128 lanes/clk/SM, 30 + 4R operations per pair) and
    MUFU (16/clk/SM, 4 per pair: rsqrt, rcp, sin, cos)."""
    return min(128 * sms * f_hz / (30 + 4 * R), 16 * sms * f_hz / 4)


def pair_roofline_tc(sms: int, f_hz: float, R: int) -> float:
    """Ceiling of the pair sum whose multiply-adds run on the tensor cores:
    the FP32 pipe evaluates K (30 operations per pair) and MUFU its 4
    transcendental steps; the tensor pipe has ample room for the 4R MACs."""
    return min(128 * sms * f_hz / 30, 16 * sms * f_hz / 4)


def solve_step(q, ctx, sc, b, mu, u, xh, tol, record=None):
    """One full mixed-precision solve: assembly for k, right-hand sides, GMRES
    with iterative refinement, far field."""
    import torch
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record()
    ctx.assemble()
    ev[1].record()
    ctx.incident_plane(sc.directions, b)
    st = ctx.solve(b, mu, q.PREC_FP32, tol=tol)
    ev[2].record()
    ctx.farfield(mu, xh, u)
    ev[3].record()
    if record is not None:
        record.append((ev, st))
    return st


def accuracy(q, torch, ctx, sc, b, mu, fp64_solve: bool):
    """Per-result accuracy of the mixed solve: its FP64-accurate residual
    (float-float apply) and its distance to a solve refined to 1e-13; on
    small workloads also to the plain FP64 GPU solve."""
    R = sc.n_rhs
    y = torch.empty_like(mu)
    ctx.apply(mu, y, q.PREC_FF)
    res = torch.linalg.norm(b - y, dim=0) / torch.linalg.norm(b, dim=0)
    ref = torch.zeros_like(mu)
    ctx.solve(b, ref, q.PREC_FP32, tol=1e-13)
    out = {"rel_residual_fp64_accurate": float(res.max()),
           "rel_err_vs_1e-13_solve": float(torch.linalg.norm(mu - ref) / torch.linalg.norm(ref))}
    if fp64_solve:
        m64 = torch.zeros_like(mu)
        ctx.solve(b, m64, q.PREC_FP64, tol=1e-12)
        out["rel_err_vs_fp64_gpu"] = float(torch.linalg.norm(mu - m64) / torch.linalg.norm(m64))
    return out


def run_workload(q, torch, cfg, steps, warmup, tol, local_rank, dist=None, rank=0, profile=False, clocks=None,
                 bodies=0):
    """Warm-up, then exactly ``steps`` timed solves between barriers and device
    synchronisation; returns the context and the per-step records."""
    import scenes
    sc = scenes.config(cfg, request_id=rank)  # replicas: an independent request per rank
    if bodies:  # the first bodies only: a small case of the same workload (profiling captures)
        sc = scenes.Scene(sc.name + f" (first {bodies} bodies)", sc.bodies[:bodies], sc.k, sc.eta, sc.directions)
    R = sc.n_rhs
    xh = far_directions()
    ctx = q.Context(local_rank)
    ctx.set_bodies(sc.bodies)
    ctx.set_wavenumber(sc.k, sc.eta)
    N = ctx.N
    b = torch.zeros((N, R), dtype=torch.complex128, device="cuda")
    mu = torch.zeros_like(b)
    u = torch.zeros((xh.shape[0], R), dtype=torch.complex128, device="cuda")
    ctx.assemble()
    tuning = ctx.autotune(R)  # launch shapes for this body set and R (outside the timed region)
    for _ in range(warmup):
        solve_step(q, ctx, sc, b, mu, u, xh, tol)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    if clocks:
        clocks.start()
    if profile:
        ctx.profile(True)
    launches0 = q.kernel_launches()
    recs = []
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record()
    for _ in range(steps):
        solve_step(q, ctx, sc, b, mu, u, xh, tol, recs)
    t1.record()
    torch.cuda.synchronize()
    launches = q.kernel_launches() - launches0
    clk = clocks.stop() if clocks else None
    elapsed = t0.elapsed_time(t1) / 1e3
    if dist:
        elapsed = max_over_ranks(elapsed, dist, "cuda")
        dist.barrier()
    prof = {}
    if profile:
        for name, slot in (("pairsum_f32_kernel", q.PROF_PAIRSUM_FP32), ("pairsum_tc_kernel", q.PROF_PAIRSUM_TC),
                           ("tc_block_kernel", q.PROF_BLOCK_TC), ("pairsum_ff_kernel", q.PROF_PAIRSUM_FF),
                           ("block_apply_kernel<float2>", q.PROF_BLOCK_FP32),
                           ("block_apply_kernel<double2>", q.PROF_BLOCK_FP64),
                           ("selfblock_kernel", q.PROF_ASSEMBLY)):
            prof[name] = ctx.profile_read(slot)
        ctx.profile(False)
    applies = [r[1]["applies_fp32"] + r[1]["applies_fp64"] for r in recs]
    pairs = sc.pair_count()
    return dict(sc=sc, ctx=ctx, b=b, mu=mu, xh=xh, recs=recs, elapsed=elapsed, launches=launches, clocks=clk,
                prof=prof, applies=applies, pair_evals=sum(a * pairs * R for a in applies), pairs=pairs,
                tuning=tuning)


def run_lattice(q, torch, sc, steps, warmup, tol, local_rank):
    """Solves of a regular array (Sec. 4; Table tab:multibody_cubic) with the
    pair sum through the circulant embedding: per step assembly (one self
    block, the transformed displacement blocks), right-hand sides, mixed
    solve, far field.  The rate counts the same N^2 - sum n_b^2 pair
    interactions per apply as the direct workloads.  Accuracy: the residual
    of the result under the direct float-float operator (every node pair
    evaluated)."""
    R = sc.n_rhs
    xh = far_directions()
    ctx = q.Context(local_rank)
    ctx.set_lattice(sc.body, sc.dims, sc.basis)
    ctx.set_wavenumber(sc.k, sc.eta)
    N = ctx.N
    b = torch.zeros((N, R), dtype=torch.complex128, device="cuda")
    mu = torch.zeros_like(b)
    u = torch.zeros((xh.shape[0], R), dtype=torch.complex128, device="cuda")
    for _ in range(warmup):
        solve_step(q, ctx, sc, b, mu, u, xh, tol)
    torch.cuda.synchronize()
    ctx.profile(True)
    recs = []
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(steps):
        solve_step(q, ctx, sc, b, mu, u, xh, tol, recs)
    t1.record()
    torch.cuda.synchronize()
    elapsed = t0.elapsed_time(t1) / 1e3
    nlat, ms_lat = ctx.profile_read(q.PROF_PAIRSUM_LATTICE)
    np32, ms32 = ctx.profile_read(q.PROF_LATTICE_PRODUCT32)
    np64, ms64 = ctx.profile_read(q.PROF_LATTICE_PRODUCT64)
    ctx.profile(False)
    applies = [r[1]["applies_fp32"] + r[1]["applies_fp64"] for r in recs]
    pairs = sc.pair_count()
    w = dict(recs=recs, elapsed=elapsed, applies=applies, pair_evals=sum(a * pairs * R for a in applies))
    out = summary(w, steps, 1)
    out["workload"] = sc.name
    out["value_note"] = ("equivalent rate: the N^2 - sum n_b^2 pair interactions of each apply, applied through "
                         "the circulant embedding of the displacement blocks")
    out["lattice_pairsum_ms_per_apply"] = ms_lat / max(nlat, 1)
    # the per-frequency products stream the transformed blocks: (2P-1)(2Q-1)(2R-1) n^2 entries
    F = 1
    for p_ in sc.dims:
        F *= 2 * p_ - 1
    n = sc.body.n_nodes
    hbm = measured_peaks()[0]["hbm_gbs"]
    prods = {}
    for name, cnt, ms, eb in (("complex64", np32, ms32, 8), ("complex128", np64, ms64, 16)):
        if cnt:
            gbs = F * n * n * eb / (ms / cnt / 1e3) / 1e9
            prods[name] = {"launches": cnt, "ms_per_launch": ms / cnt, "algorithmic_bytes": F * n * n * eb,
                           "achieved_gbs": gbs, "peak_gbs": hbm, "frac": gbs / hbm, "bound": "hbm"}
    out["freq_product_kernel"] = prods
    # independent check: the residual under the direct float-float operator
    ctx.set_option(q.OPT_LATTICE, 0)
    y = torch.empty_like(mu)
    ctx.apply(mu, y, q.PREC_FF)
    ctx.set_option(q.OPT_LATTICE, 1)
    res = torch.linalg.norm(b - y, dim=0) / torch.linalg.norm(b, dim=0)
    out["rel_residual_direct_ff"] = float(res.max())
    ctx.close()
    return out


def summary(w, steps, world):
    recs = w["recs"]
    step_ms = [r[0][0].elapsed_time(r[0][3]) for r in recs]
    lat = sorted(step_ms)

    def pct(p):
        return lat[min(len(lat) - 1, int(math.ceil(p / 100 * len(lat))) - 1)]

    st = recs[-1][1]
    return {
        "ms_per_step": w["elapsed"] / steps * 1e3,
        "value": job_value(w["pair_evals"], world, w["elapsed"]),
        "solves_per_s": steps * world / w["elapsed"],
        "latency_ms": {"p50": pct(50), "p99": pct(99)},
        "breakdown_ms": {"assembly": statistics.mean(r[0][0].elapsed_time(r[0][1]) for r in recs),
                         "solve": statistics.mean(r[0][1].elapsed_time(r[0][2]) for r in recs),
                         "far_field": statistics.mean(r[0][2].elapsed_time(r[0][3]) for r in recs)},
        "solver": {"applies_per_solve": statistics.mean(w["applies"]), "iterations": st["iterations"],
                   "refinements": st["refinements"], "fp64_accurate_applies": st["applies_fp64"],
                   "rel_residual": st["rel_residual"]},
    }


def run_ours(args, rank, world, local_rank):
    import torch

    import paper_2606_31380_b300 as q

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
    clocks = ClockSampler(local_rank)
    w = run_workload(q, torch, args.config, args.steps, args.warmup, args.tol, local_rank, dist, rank,
                     profile=True, clocks=clocks, bodies=args.bodies)
    sc, ctx, R, N = w["sc"], w["ctx"], w["sc"].n_rhs, w["ctx"].N
    head = summary(w, args.steps, world)
    acc = accuracy(q, torch, ctx, sc, w["b"], w["mu"], fp64_solve=N <= 40000) if not args.no_accuracy else None
    clk = w["clocks"]
    f_hz = (clk.get("sm_mhz") or 2032.0) * 1e6

    # every profiled kernel of the timed region: launches, device time, share
    prof = w["prof"]
    t_all = w["elapsed"] * 1e3
    kernels = {name: {"launches": n, "ms_total": ms, "ms_per_launch": ms / n if n else None,
                      "share_of_step": ms / t_all} for name, (n, ms) in prof.items()}
    pairs = w["pairs"]
    # FP32 pair sum: CUDA-core kernel (one launch per group of up to 16 right-hand
    # sides) or tensor-core kernel (one launch for all); whichever the autotuner chose
    groups = 1 if R in (1, 2, 4, 8, 16) else len(range(0, R, 16))
    for name, per_launch, peak_fn, bound in (
            ("pairsum_f32_kernel", groups, pair_roofline, "alu (FP32 pipe + MUFU)"),
            ("pairsum_tc_kernel", 1, pair_roofline_tc, "alu (MUFU; products on the tensor pipe)")):
        n_l, ms_l = prof[name]
        if n_l:
            ach = n_l * pairs / per_launch / (ms_l / 1e3)
            pk = peak_fn(sms, f_hz, R)
            kernels[name].update({"bound": bound, "pairs_per_s": ach, "peak_pairs_per_s": pk, "frac": ach / pk})
    nff, msff = prof["pairsum_ff_kernel"]
    if nff:
        aff = nff * pairs / (msff / 1e3)
        pff = 128 * sms * f_hz / (FF_OPS_PER_PAIR + 72 * (R - 1))
        kernels["pairsum_ff_kernel"].update({"bound": "alu (FP32 pipe)", "pairs_per_s": aff,
                                             "peak_pairs_per_s": pff, "frac": aff / pff})
    entries = sum(bd.n_nodes ** 2 for bd in sc.bodies)
    hbm = measured_peaks()[0]["hbm_gbs"]
    nb32, msb32 = prof["block_apply_kernel<float2>"]
    if nb32:
        gbs = nb32 * entries * 8 * ((R + 15) // 16) / (msb32 / 1e3) / 1e9
        kernels["block_apply_kernel<float2>"].update({"bound": "hbm", "achieved_gbs": gbs, "peak_gbs": hbm,
                                                      "frac": gbs / hbm})
    ntc, mstc = prof["tc_block_kernel"]
    if ntc:
        # one launch per equal-size group streams every block once: 8 bytes (FP16 hi + lo) per complex entry
        groups_b = len({bd.n_nodes for bd in sc.bodies})
        gbs = ntc / groups_b * entries * 8 / (mstc / 1e3) / 1e9
        kernels["tc_block_kernel"].update({"bound": "hbm", "achieved_gbs": gbs, "peak_gbs": hbm, "frac": gbs / hbm})
    na, msa = prof["selfblock_kernel"]
    asm_counts = ctx.assembly_counts()
    flops = assembly_flops(sc, asm_counts)
    peak64 = 2 * 2 * sms * f_hz / 1e12
    peak64_meas = fp64_peak_tflops(torch) if not args.no_fp64_probe else None
    if na:
        a_tf = flops / (msa / 1e3 / args.steps) / 1e12  # one assembly per step
        kernels["selfblock_kernel"].update({"bound": "alu (FP64 pipe)", "achieved_tflops": a_tf,
                                            "peak_tflops": peak64, "frac": a_tf / peak64})
    dominant = max(prof, key=lambda k: prof[k][1])
    k_dom = kernels[dominant]
    if dominant in ("pairsum_f32_kernel", "pairsum_tc_kernel"):
        tag = "<%d>" % min(R, 16) if dominant == "pairsum_f32_kernel" else "<NH=%d>" % (16 if 2 * R <= 16 else 32)
        note = ("min(128 FP32 lanes/clk/SM / (30+4R) ops, 16 MUFU/clk/SM / 4)" if dominant == "pairsum_f32_kernel"
                else "min(128 FP32 lanes/clk/SM / 30 ops, 16 MUFU/clk/SM / 4): the 4R multiply-adds run on the "
                     "tensor pipe")
        roof = {"kernel": f"{dominant}{tag} (FP32 inter-body pair sum)", "bound": "alu",
                "achieved": k_dom["pairs_per_s"], "peak": k_dom["peak_pairs_per_s"], "unit": "pair-interactions/s",
                "frac": k_dom["frac"], "traffic": None,
                "peak_note": "derived: %s pairs x %d SMs x %.0f MHz (median sampled SM clock)" % (note, sms, f_hz / 1e6)}
    else:
        roof = {"kernel": dominant, "bound": k_dom.get("bound"),
                "achieved": k_dom.get("pairs_per_s") or k_dom.get("achieved_tflops") or k_dom.get("achieved_gbs"),
                "peak": k_dom.get("peak_pairs_per_s") or k_dom.get("peak_tflops") or k_dom.get("peak_gbs"),
                "frac": k_dom.get("frac"), "traffic": None,
                "unit": "pair-interactions/s" if "pairs_per_s" in k_dom else "TFLOP/s" if "achieved_tflops" in k_dom
                else "GB/s"}
    kernels["note"] = ("device time of every launch in the timed region (CUDA events around each launch on its "
                       "stream); peaks at the median sampled SM clock; HBM peak of %s" % measured_peaks()[1])

    # the same workload through the C ABI from host descriptors to host results
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    M = w["xh"].shape[0]
    mu_h = torch.empty((N, R), dtype=torch.complex128, pin_memory=True)
    u_h = torch.empty((M, R), dtype=torch.complex128, pin_memory=True)
    torch.cuda.synchronize()
    t_start = time.perf_counter()
    e2e_pairs = 0
    for _ in range(e2e_steps):
        c2 = q.Context(local_rank)
        c2.set_bodies(sc.bodies)
        c2.set_wavenumber(sc.k, sc.eta)
        c2.autotune(R)  # the process-wide cache holds this shape's choice: no timing
        bb = torch.zeros((N, R), dtype=torch.complex128, device="cuda")
        mm = torch.zeros_like(bb)
        uu = torch.zeros((M, R), dtype=torch.complex128, device="cuda")
        st = solve_step(q, c2, sc, bb, mm, uu, w["xh"], args.tol)
        mu_h.copy_(mm, non_blocking=True)
        u_h.copy_(uu, non_blocking=True)
        torch.cuda.synchronize()
        c2.close()
        e2e_pairs += (st["applies_fp32"] + st["applies_fp64"]) * pairs * R
    e2e_t = time.perf_counter() - t_start
    h2d = sum(8 * (9 + 3 + 6 + len(bd.mode_cos) + len(bd.mode_sin)) for bd in sc.bodies) + 8 * 3 * R + 8 * 3 * M
    d2h = 16 * N * R + 16 * M * R

    # the other workloads of the metric, a few solves each
    extra = {}
    if not args.no_extra:
        for cfg, st_, wu in ((1, 5, 2), (2, 3, 1)):
            if cfg == args.config:
                continue
            wx = run_workload(q, torch, cfg, st_, wu, args.tol, local_rank, dist, rank)
            sx = summary(wx, st_, world)
            sx["workload"] = wx["sc"].name
            sx.update(accuracy(q, torch, wx["ctx"], wx["sc"], wx["b"], wx["mu"], fp64_solve=wx["ctx"].N <= 40000))
            extra[f"config{cfg}"] = sx
            wx["ctx"].close()
            del wx
            torch.cuda.empty_cache()

        import scenes as scn
        for name, lsc in (("lattice_1000", scn.lattice_of_workload(3)),
                          ("paper_cubic_1000_k5", scn.paper_cubic(10, 5.0))):
            extra[name] = run_lattice(q, torch, lsc, 3, 2, args.tol, local_rank)
            torch.cuda.empty_cache()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    out = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64",
        "precision_note": ("f32 inner operator; f64 and float-float (pairs of f32) in the assembly, "
                           "refinement residual and far field; f64 Krylov basis"),
        "data": "synthetic (seeded quasi-axisymmetric bodies)",
        "config": {"workload": sc.name, "n_bodies": len(sc.bodies), "N": N, "R": R, "k": sc.k, "eta": sc.eta,
                   "tol": args.tol, "far_field_dirs": M, "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (self blocks %.2f GB resident)" % (entries * 24 / 1e9)},
        "solves_per_s": head["solves_per_s"], "latency_ms": head["latency_ms"],
        "breakdown_ms": head["breakdown_ms"], "solver": head["solver"], "accuracy": acc,
        "assembly_outer_nodes": {"modal": asm_counts[0], "far": asm_counts[1]},
        "roofline": roof,
        "tuning": w["tuning"],
        "fp64_peak": {"dgemm_tflops_measured": peak64_meas, "derived_tflops": peak64,
                      "note": "cuBLAS DGEMM 8192^3 best of 5 in this run; derived = 2 lanes/clk/SM x 2 x SMs x clock"},
        "e2e": {"value": e2e_pairs / e2e_t, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e2e_steps},
        "gpu_launches": w["launches"],
        "clocks": clk,
        "kernels": kernels,
        "other_workloads": extra,
    }
    if args.serve_sample:
        # a bounded sample of the serving stream (10..500 bodies), reported beside the step
        ctx.close()
        torch.cuda.empty_cache()
        import scenes as scn
        sreqs = [scn.serving_request(i) for i in range(args.serve_sample)]
        sv = serve_stream(q, sreqs, args.serve_slots, (0.8,))
        sv["latency_ms"] = sv["streams"][0]["latency_ms"]
        sv["solves_per_s"] = sv["streams"][0]["solves_per_s"]
        sv["workload"] = (f"{len(sreqs)} requests of the serving distribution (10..500 bodies, "
                          "{16x32, 24x48} nodes, k ~ U[1,15], 1..16 RHS, tol 1e-11)")
        out["serving"] = sv
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(sc, args.cpu_seconds)
    print(json.dumps(out), flush=True)
    ctx.close()
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


def serve_stream(q, reqs, slots, lam_fracs=(0.8,), seed=31380):
    """A burst of all requests (the saturated rate), then for each fraction
    the same requests with Poisson arrivals at that fraction of the rate:
    solves/s and p50/p99 latency per rate."""
    import numpy as np

    import scenes
    far = scenes.fibonacci_directions(400)
    srv = q.Server(0, 0, slots=slots)
    srv.wait(srv.submit(reqs[0], far))  # warm-up
    t0 = time.perf_counter()
    tickets = [srv.submit(r, far) for r in reqs]
    burst = [srv.wait(t) for t in tickets]
    t_burst = time.perf_counter() - t0
    sat = len(reqs) / t_burst
    streams = []
    failed = [{"request": i, "phase": "burst", "status": r["status"], "rel_residual": r["rel_residual"]}
              for i, r in enumerate(burst) if r["status"] != 0]
    for frac in lam_fracs:
        rng = np.random.default_rng(seed)
        lam = frac * sat
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
        lat = np.array([r["latency_ms"] for r in res])
        failed += [{"request": i, "phase": f"stream {frac}", "status": r["status"], "rel_residual": r["rel_residual"]}
                   for i, r in enumerate(res) if r["status"] != 0]
        streams.append({"rate_fraction": frac, "arrival_rate_per_s": lam, "solves_per_s": len(reqs) / t_stream,
                        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))}})
    srv.close()
    return {"saturated_solves_per_s": sat, "streams": streams,
            "mean_nodes": float(np.mean([r["n_nodes"] for r in burst])), "slots": slots,
            "all_ok": not failed, "failed": failed}


def run_serve(args):
    """Serving stream: seeded requests with 10..max_bodies bodies, {16x32, 24x48}
    nodes, k ~ U[1, 15], 1..16 RHS, each a full mixed solve to 1e-11 plus 400
    far-field directions; a burst measures the saturated rate, Poisson
    arrivals at 0.8 of it (or --serve-rates) give the latency distribution."""
    import paper_2606_31380_b300 as q
    import scenes

    reqs = [scenes.serving_request(i, max_bodies=args.serve_max_bodies) for i in range(args.serve_requests)]
    r = serve_stream(q, reqs, args.serve_slots, tuple(args.serve_rates))
    mid = min(r["streams"], key=lambda x: abs(x["rate_fraction"] - 0.8))
    out = {"metric": "serving solves/s and p50/p99 solve latency", "value": mid["solves_per_s"],
           "unit": "solves/s", "higher_is_better": True, "n_gpus": 1, "data": "synthetic (seeded requests)",
           "config": {"workload": f"{len(reqs)} requests, 10..{args.serve_max_bodies} bodies, "
                                  "{16x32, 24x48} nodes, k ~ U[1,15], 1..16 RHS, tol 1e-11",
                      "slots": args.serve_slots, "arrival_rate_fraction": mid["rate_fraction"]},
           "latency_ms": mid["latency_ms"]}
    out.update(r)
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, default=3,
                    help="workload index (3 = 1000 bodies x 512 nodes, k = 3, 4 RHS; 1 = 16 x 2048, 2 = 100 x 1152)")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-probe", action="store_true", help="skip the cuBLAS DGEMM that measures the FP64 peak")
    ap.add_argument("--no-extra", action="store_true", help="measure the headline workload only")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the accuracy solves after the timed region (profiling runs)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--bodies", type=int, default=0, help="use only the first B bodies (small profiling case)")
    ap.add_argument("--tol", type=float, default=1e-10,
                    help="relative FP64 residual target of the mixed solve (the metric asks 1e-8 relative error)")
    ap.add_argument("--serve", action="store_true", help="serving stream instead of the single-solve step")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-max-bodies", type=int, default=500)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[0.5, 0.8, 1.0],
                    help="Poisson arrival rates as fractions of the saturated rate")
    ap.add_argument("--serve-sample", type=int, default=8,
                    help="requests of the serving distribution measured in the default run (0: none)")
    ap.add_argument("--lattice", choices=["workload", "paper"], default=None,
                    help="time solves of a regular array instead (10^3 copies of the 1000-body workload's body, "
                         "or the paper's 10^3 quasi-ellipsoids at k = 5) and print one JSON line")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus if args.gpus == 1 else 1)))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.serve:
        if rank == 0:
            run_serve(args)
    elif args.lattice and args.impl == "ours":
        if rank == 0:
            import torch

            import paper_2606_31380_b300 as q
            import scenes
            sc = scenes.lattice_of_workload(3) if args.lattice == "workload" else scenes.paper_cubic(10, 5.0)
            out = run_lattice(q, torch, sc, args.steps, args.warmup, args.tol, local_rank)
            out.update({"metric": METRIC, "unit": UNIT, "steps": args.steps, "warmup": args.warmup,
                        "n_gpus": 1, "higher_is_better": True, "data": "synthetic (regular array)"})
            print(json.dumps(out), flush=True)
    elif args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
