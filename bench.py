"""Benchmark: converged short-characteristics + Jacobi-ALI solves of the 256^3
stratified turbulent atmosphere.

Workload (the largest single-GPU case): a 256^3 grid whose opacity is the
stratified profile (vertical optical depth log-spaced from 1e-4 at the top to
1e3 at the bottom) times a log-normal turbulent density (k^-11/3 Gaussian random
field, seed 1), photon destruction probability eps = 1e-3, B = T^4 (log-normal
T, seed 2), periodic x/y, I = B below and vacuum above, 48 rays (LQ6), float32
sweeps with the FP64 ALI update, solved to max|dS|/S <= 1e-6; outputs J, the
Eddington tensor K/J and the heating rate.  Synthetic inputs, generated here.

One step = the whole hot path on resident device inputs: set the medium
(validation, sweep-precision copies, Lambda*, ghosts), the ALI solve to
convergence (formal solutions + updates), and the outputs (J, H, K, K/J, Q).
Metric: cell*ray*frequency updates per second (updates = cells * rays *
frequencies * formal solutions).  The L2 cache is flushed (256 MB written)
before every timed step (the step's inputs, 400 MB, exceed it anyway).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank solves its own copy (independent solves, no data-path
collective: weak scaling); rank 0 prints one JSON line with the whole-job rate.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell*ray*nu updates/s"
UNIT = "updates/s"
N_BOX = 256
N_MU = 6
TOL = 1e-6
# algorithmic FP32 operations of one cell*ray update (Eq. 20 with linear
# interpolation): three bilinear interpolants (chi-, S-, I-: 4 multiplies + 3 adds
# each, 21), dtau = (chi- + chi0) s/2 (add, multiply), e0 = 1 - E, e1 = dtau - e0,
# Psi0 = e1 / dtau, Psi- = e0 - Psi0 (4), I0 = I- E + Psi- S- + Psi0 S0 (3 multiplies
# + 2 adds), the J accumulation (multiply, add); the exponential is counted apart
FLOPS_PER_UPDATE = 34
# special-function results per update: the exponential and the reciprocal of dtau
MUFU_PER_UPDATE = 2
# CTAs per cluster of every grid in the request server's shared-launch mode
SHARED_CLUSTER = 4

# DRAM read + write bytes per launch of the sweep kernel from an ncu capture of
# the same workload and plan (None when none was taken for the plan in use, or
# the kernel has changed since); keyed by workload, plan, shared-memory size and groups
PROFILED_TRAFFIC = {
    # one launch of the 256^3 x 48-ray solve's sweep (dram__bytes_read.sum +
    # dram__bytes_write.sum, one ncu pass)
    ("stratified_turbulent_256^3_lq6", 3, 2, 16, 512, 197312, 27): 1235145216 + 1810619648,
}


def profiled_traffic(plan, p):
    key = (p.name, plan["variant"], plan["rays_per_group"], plan["cluster"], plan["threads"], plan["smem"],
           plan["groups"])
    return PROFILED_TRAFFIC.get(key)


# sweep kernel of each planner variant (simple, tiled, pipelined)
SWEEP_KERNEL_NAMES = {1: "sc_sweep_kernel<float>", 2: "sc_sweep_tiled_kernel<float>",
                      3: "sc_sweep_pipe_kernel<float>"}


def workload():
    from paper_1201_2222_gb300 import workloads as W
    return W.large_stratified_turbulent(N_BOX, n_mu=N_MU, tol=TOL)


def config_dict(p, flush):
    return {"workload": f"stratified_turbulent_{p.nx}^3_LQ{p.n_mu}_{p.n_angles}rays_grey_eps1e-3_tol{TOL:g}",
            "cells": p.cells, "rays": p.n_angles, "frequencies": p.nf,
            "precision": "float32 sweeps, FP64 ALI", "l2": flush}


# --------------------------------------------------------------- multi-rank glue

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def shard(n_units: int, rank: int, world: int) -> list:
    """Units (independent solves) owned by this rank: a contiguous balanced slice."""
    base, extra = divmod(n_units, world)
    lo = rank * base + min(rank, extra)
    return list(range(lo, lo + base + (1 if rank < extra else 0)))


def reduce_max_sum(t_local: float, u_local: float, dist) -> tuple:
    """(max over ranks of the timed seconds, sum over ranks of the updates)."""
    if dist is None:
        return t_local, u_local
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([t_local], dtype=torch.float64, device=dev)
    u = torch.tensor([u_local], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# --------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # raw samples go to RT_BENCH_CLOCKS_DIR (default: the system temporary directory)
        out_dir = os.environ.get("RT_BENCH_CLOCKS_DIR", tempfile.gettempdir())
        self.path = os.path.join(out_dir, f"clocks_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv",
                                          "-lms", "200", "-i", str(self.gpu)],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9 or not parts[1].split()[0].isdigit():
                continue
            sm.append(float(parts[1].split()[0]))
            mx.append(float(parts[2].split()[0]))
            for name, val in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                  "sw_power_cap"), parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# -------------------------------------------------------------- CPU baseline

def oracle_rate(p, min_seconds=10.0, max_runs=40):
    """The FP64 CPU oracle's formal-solution rate on this workload (all host cores)."""
    from oracle import oracle as O
    og = O.Grid.from_problem(p)
    nt = O.max_threads()
    S = p.B[0]
    runs, t_total = 0, 0.0
    while runs < max_runs and (runs == 0 or t_total < min_seconds):
        t = time.perf_counter()
        O.formal_solution(og, p.chi[0], S, p.B[0], nthreads=nt)
        t_total += time.perf_counter() - t
        runs += 1
    upd = runs * og.cells * og.na * p.nf
    return {"value": upd / t_total, "unit": UNIT, "cores": nt, "kind": "oracle",
            "sample": f"{runs} FP64 formal solution(s) of the full {p.nx}^3 x {og.na}-ray box "
                      f"({og.cells * og.na:,} updates each), {t_total:.1f} s"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    p = workload()
    from oracle import oracle as O
    og = O.Grid.from_problem(p)
    nt = O.max_threads()
    times = []
    for i in range(args.warmup + args.steps):
        t = time.perf_counter()
        O.formal_solution(og, p.chi[0], p.B[0], p.B[0], nthreads=nt)
        if i >= args.warmup:
            times.append(time.perf_counter() - t)
    upd = og.cells * og.na * p.nf
    value = upd * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(p, "n/a (CPU)"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nt, "kind": "oracle",
                             "sample": f"each step one FP64 formal solution of the full box "
                                       f"({upd:,} updates)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm

def sweep_roofline(stats_list, p, rates):
    """Roofline of the formal-solution kernel from the sweep launches timed inside
    the solves (CUDA events on the launching stream)."""
    sweep_ms = sum(s["sweep_ms"] for s in stats_list)
    sweep_n = sum(s["sweep_launches"] for s in stats_list)
    per_launch_upd = p.cells * p.n_angles * p.nf
    avg_s = (sweep_ms / sweep_n) / 1e3 if sweep_n else float("nan")
    achieved = FLOPS_PER_UPDATE * per_launch_upd / avg_s / 1e12
    peak = max(rates["fp32_fma_flops"], rates["fp32x2_fma_flops"]) / 1e12
    mufu_peak = min(rates["mufu_ex2_per_s"], rates["mufu_rcp_per_s"])
    return {"avg_launch_ms": avg_s * 1e3, "launches": sweep_n, "achieved": achieved, "peak": peak,
            "frac": achieved / peak, "updates_per_s": per_launch_upd / avg_s,
            "mufu_frac": MUFU_PER_UPDATE * per_launch_upd / avg_s / mufu_peak}


def solve_rate(rt, p, prec, dev, n=2, tol=None, autotune=True):
    """Time n converged solves (after one untimed) of problem p; CUDA-event sweep
    statistics of the last one."""
    import torch
    tol = p.tol if tol is None else tol
    chi, eps, B, fw = (torch.from_numpy(x).to(dev) for x in (p.chi, p.eps, p.B, p.freq_w))
    g = rt.Grid.from_problem(p, prec=prec)
    g.set_opacity_source(chi, eps, B, fw)
    if autotune:
        g.autotune()
    g.ali_solve(tol=tol, max_iter=20000)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(n):
        it, _, _ = g.ali_solve(tol=tol, max_iter=20000)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t) / n
    g.enable_timing(True)
    g.ali_solve(tol=tol, max_iter=20000)
    st = g.stats()
    plan = g.sweep_plan()
    g.close()
    return {"workload": p.name, "iters": it, "ms_per_solve": 1e3 * dt, "solves_per_s": 1.0 / dt,
            "updates_per_s": p.cells * p.n_angles * p.nf * it / dt, "plan": plan, "stats": st}


def run_gpu(args):
    import torch
    ws, rank, local = dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
        dist = tdist
    else:
        torch.cuda.set_device(0)
    from paper_1201_2222_gb300 import build, rt, workloads as W
    build.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    rates = rt.measure_rates()          # measured arithmetic peaks of this GPU
    p = workload()
    chi = torch.from_numpy(p.chi).to(dev)
    eps = torch.from_numpy(p.eps).to(dev)
    B = torch.from_numpy(p.B).to(dev)
    fw = torch.from_numpy(p.freq_w).to(dev)
    g = rt.Grid.from_problem(p, prec=rt.MIXED)
    g.set_opacity_source(chi, eps, B, fw)
    if args.plan:                 # a given sweep plan (e.g. to list one run's launches)
        v, apg, c, th = (int(x) for x in (args.plan + ",0").split(",")[:4])
        g.set_sweep_config(apg, c, th, v)
    else:                         # set-up: pick the sweep launch plan once per problem shape
        g.autotune()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(out):
        g.set_opacity_source(chi, eps, B, fw)
        iters, resid, st = g.ali_solve(tol=TOL, max_iter=20000)
        m = g.moments(on_device=True, want=("J", "f", "Q"))
        out.append((iters, resid, g.stats()))
        return m

    for _ in range(args.warmup):
        step([])
    torch.cuda.synchronize()
    rec = []
    ev = []
    g.enable_timing(True)
    launches0 = g.stats()["kernel_launches"]
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step(rec)
        b.record(stream)
        ev.append((a, b))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    wall1 = time.perf_counter()
    clk = clocks.stop()
    g.enable_timing(False)
    launches = g.stats()["kernel_launches"] - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_local = sum(step_ms) / 1e3
    upd_local = float(sum(s["updates"] for _, _, s in rec))
    t_max, upd_all = reduce_max_sum(t_local, upd_local, dist)
    iters = [i for i, _, _ in rec]
    roof = sweep_roofline([s for _, _, s in rec], p, rates)

    # end to end through the C ABI with host buffers (copies inside the timed region)
    e2e_t = []
    e2e_upd = 0
    N = p.chi.size
    h2d = 3 * N * 8 + p.nf * 8
    d2h = (N + p.cells) * 8
    # the step's inputs and its results (J, Q) in pinned host memory
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).pin_memory()
    chi_h, eps_h, B_h, fw_h = pin(p.chi), pin(p.eps), pin(p.B), pin(p.freq_w)
    J_h = torch.empty(p.chi.shape, dtype=torch.float64).pin_memory()
    Q_h = torch.empty(p.chi.shape[1:], dtype=torch.float64).pin_memory()
    for i in range(1 + max(2, args.steps // 2)):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t = time.perf_counter()
        g.set_opacity_source(chi_h, eps_h, B_h, fw_h)
        it, _, _ = g.ali_solve(tol=TOL, max_iter=20000)
        m = g.moments(on_device=False, want=("J", "Q"), out={"J": J_h, "Q": Q_h})
        _ = float(m["Q"].sum())
        dt = time.perf_counter() - t
        if i > 0:
            e2e_t.append(dt)
            e2e_upd += p.cells * p.n_angles * p.nf * it
    e2e_tmax, e2e_updall = reduce_max_sum(sum(e2e_t), float(e2e_upd), dist)
    e2e = {"value": e2e_updall / e2e_tmax, "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h}
    plan = g.sweep_plan()
    g.close()

    extras = {}
    if not args.skip_extras:
        # the 128^3 periodic turbulent box (80 rays): mixed, and the plain FP64 path
        pb = W.turbulent_box(128, n_mu=8, tol=TOL)
        box = solve_rate(rt, pb, rt.MIXED, dev)
        box["roofline"] = sweep_roofline([box.pop("stats")], pb, rates)
        extras["turbulent_box_128"] = box
        b64 = solve_rate(rt, pb, rt.FP64, dev, n=1)
        b64.pop("stats")
        extras["turbulent_box_128_fp64_path"] = b64
        extras["mixed_over_fp64_solves_per_s"] = box["solves_per_s"] / b64["solves_per_s"]
    if not args.skip_extras and not args.skip_multifreq:
        # the 64^3 atmosphere with 64 frequency bins (all bins in one launch)
        pm = W.multifrequency_atmosphere(64, nf=64)
        mf = solve_rate(rt, pm, rt.MIXED, dev, n=1)
        mf["roofline"] = sweep_roofline([mf.pop("stats")], pm, rates)
        extras["multifrequency_64_64bins"] = mf
    if not args.skip_extras and not args.skip_gs:
        # the Gauss-Seidel scheme against Jacobi on the stratified scattering
        # atmosphere (32^3, LQ4, eps 1e-2, FP64, tol 1e-6): iterations and solve time
        pa = W.stratified_atmosphere(32)
        gs = {"workload": f"{pa.name} (FP64, tol {pa.tol:g})"}
        for scheme in ("jacobi", "gauss_seidel"):
            ga = rt.Grid.from_problem(pa, prec=rt.FP64)
            ga.set_iteration(scheme)
            ga.set_opacity_source(pa.chi, pa.eps, pa.B, pa.freq_w)
            ga.ali_solve(tol=pa.tol, max_iter=5000)
            best = math.inf
            for _ in range(3):
                torch.cuda.synchronize()
                t = time.perf_counter()
                ita, _, _ = ga.ali_solve(tol=pa.tol, max_iter=5000)
                best = min(best, time.perf_counter() - t)
            gs[scheme] = {"iters": ita, "ms_per_solve": 1e3 * best, "ms_per_iter": 1e3 * best / ita}
            ga.close()
        gs["iteration_ratio"] = gs["jacobi"]["iters"] / gs["gauss_seidel"]["iters"]
        gs["time_ratio"] = gs["jacobi"]["ms_per_solve"] / gs["gauss_seidel"]["ms_per_solve"]
        extras["gauss_seidel"] = gs
    if not args.skip_extras and not args.skip_quad:
        # the second-order option (quadratic face interpolation): formal-solution
        # rate on the 128^3 box, mixed precision, its own tuned plan
        pb = W.turbulent_box(128, n_mu=8, tol=TOL)
        gq = rt.Grid.from_problem(pb, prec=rt.MIXED)
        gq.set_interpolation(rt.INTERP_QUADRATIC)
        gq.set_opacity_source(pb.chi, pb.eps, pb.B, pb.freq_w)
        gq.autotune()
        gq.enable_timing(True)
        gq.formal_solve(None)
        qms = []
        for _ in range(5):
            gq.formal_solve(None)
            qms.append(gq.stats()["sweep_ms"])
        qms.sort()
        extras["quadratic_path"] = {"workload": pb.name, "kernel": "sc_sweep_quad_kernel<float>",
                                    "sweep_ms_median": qms[len(qms) // 2],
                                    "updates_per_s": pb.cells * pb.n_angles * pb.nf / (qms[len(qms) // 2] / 1e3),
                                    "plan": gq.sweep_plan()}
        gq.close()

    if not args.skip_extras and not args.skip_serve:
        # the request stream (first 16 requests, 4 arrivals/s, the full eps range)
        # through the server: each solve on its worker, then the shared-launch mode
        extras["serving_16_requests"] = {
            "per_worker_solves": serve_sample(rt, W, 16, 4.0, 4, 0),
            "shared_launches": serve_sample(rt, W, 16, 4.0, 4, SHARED_CLUSTER)}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    cpu = oracle_rate(p) if ws == 1 and not args.skip_cpu else None
    lat = sorted(step_ms)
    line = {
        "metric": METRIC, "value": upd_all / t_max, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": config_dict(p, "flushed (256 MB written) before every timed step; inputs 400 MB"),
        "solves_per_s": ws * args.steps / t_max,
        "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)]},
        "ali_iterations": iters[0] if len(set(iters)) == 1 else iters,
        "sweep_plan": plan,
        "roofline": {"bound": "alu", "kernel": SWEEP_KERNEL_NAMES[plan["variant"]],
                     "achieved": roof["achieved"], "peak": roof["peak"], "unit": "TFLOP/s",
                     "frac": roof["frac"], "traffic": profiled_traffic(plan, p),
                     "peak_source": "measured on this GPU by rt_measure_rates: the larger of its scalar "
                                    "and packed-pair FP32 FMA rates (of measured)",
                     "flops_per_update": FLOPS_PER_UPDATE, "avg_launch_ms": roof["avg_launch_ms"],
                     "launches": roof["launches"], "sweep_updates_per_s": roof["updates_per_s"],
                     "mufu_frac": roof["mufu_frac"]},
        "measured_peaks": dict(rates, sm_count=sm_count),
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "wall_s": wall1 - wall0,
    }
    line.update(extras)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_profile(args):
    """Short run for profilers: set the medium and do a few ALI iterations of the
    same workload (no warm-up loop, no baselines)."""
    import torch
    torch.cuda.set_device(0)
    from paper_1201_2222_gb300 import build, rt, workloads as W
    build.build()
    p = W.turbulent_box(128, n_mu=8, tol=TOL) if args.box128 else workload()
    g = rt.Grid.from_problem(p, prec=rt.FP64 if args.fp64 else rt.MIXED)
    if args.quadratic:
        g.set_interpolation(rt.INTERP_QUADRATIC)
    if args.gauss_seidel:
        g.set_iteration(rt.ITER_GAUSS_SEIDEL)
    g.set_opacity_source(p.chi, p.eps, p.B, p.freq_w)
    if args.plan:
        v, apg, c, th = (int(x) for x in (args.plan + ",0").split(",")[:4])
        g.set_sweep_config(apg, c, th, v)
    elif not args.no_autotune:
        g.autotune()
    it, resid, st = g.ali_solve(tol=TOL, max_iter=args.profile_iters, raise_on_fail=False)
    torch.cuda.synchronize()
    print(json.dumps({"profile_run": p.name, "iters": it, "resid": resid, "plan": g.sweep_plan()}), flush=True)
    return 0


def serve_sample(rt, W, n, rate, workers, shared_cluster=0, log=None):
    """The first ``n`` requests of the mixed-size request stream (arrival seed 7,
    Poisson arrivals at ``rate``/s, eps log-uniform in [1e-4, 1]) through the
    request server; returns p50/p99 latency (arrival to result), aggregate
    updates/s and solves/s."""
    import torch
    stream = W.serving_stream(n, seed=7, rate=rate)
    probs = [W.build_request(d) for d in stream]
    srv = rt.Server(workers=workers, shared_cluster=shared_cluster)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ids = []
    for d, p in zip(stream, probs):
        wait = d["t_arrival"] - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        ids.append((srv.submit(p, prec=rt.MIXED, max_iter=20000), time.perf_counter() - t0, p))
    lat, upd, iters, bad = [], 0, [], 0
    for rid, t_sub, p in ids:
        info = srv.wait(rid, timeout=3600)
        srv.fetch(rid, raise_on_fail=False)
        if log:
            print(f"request {rid}: {p.name} iters {info['iters']} status {info['status']} "
                  f"queue {info['queue_ms']:.0f} ms solve {info['solve_ms']:.0f} ms", file=log, flush=True)
        bad += info["status"] != rt.RT_OK
        lat.append(info["queue_ms"] + info["solve_ms"])
        upd += p.cells * p.n_angles * p.nf * info["iters"]
        iters.append(info["iters"])
    wall = time.perf_counter() - t0
    shared = srv.shared_launches()
    srv.close()
    lat = np.array(lat)
    return {"requests": len(ids), "workers": workers, "shared_cluster": shared_cluster,
            "rate_per_s": rate, "value": upd / wall, "unit": UNIT, "solves_per_s": len(ids) / wall,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "failed": int(bad), "iters_median": float(np.median(iters)), "wall_s": wall,
            "shared_launches": shared}


def run_serve(args):
    """A sample of the mixed-size request stream through the request server:
    Poisson arrivals at ``--rate`` requests/s, ``--workers`` worker threads
    (``--shared C``: the shared-launch mode with C CTAs per cluster); prints one
    JSON line with p50/p99 latency (arrival to result) and throughput."""
    import torch
    torch.cuda.set_device(0)
    from paper_1201_2222_gb300 import build, rt, workloads as W
    build.build()
    res = serve_sample(rt, W, args.serve, args.rate, args.workers, args.shared, log=sys.stderr)
    line = {"mode": "serve", "metric": METRIC, **res, "data": "synthetic", "dtype": "f32+f64",
            "config": {"workload": f"serving stream sample: the first {res['requests']} requests (arrival "
                                   "seed 7) of sizes 32^3..128^3 and 512x512 2D, 1/4/16 frequencies, "
                                   "24/48/80 rays, eps log-uniform in [1e-4, 1]"}}
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--skip-cpu", action="store_true", help="omit the CPU oracle baseline")
    ap.add_argument("--skip-fp64", action="store_true", help="omit the FP64 GPU comparison solves")
    ap.add_argument("--skip-quad", action="store_true", help="omit the second-order formal-solution rate")
    ap.add_argument("--skip-multifreq", action="store_true", help="omit the 64-bin atmosphere solve")
    ap.add_argument("--skip-extras", action="store_true", help="omit every comparison beyond the headline")
    ap.add_argument("--skip-gs", action="store_true", help="omit the Gauss-Seidel against Jacobi comparison")
    ap.add_argument("--profile", action="store_true", help="one short solve for profilers")
    ap.add_argument("--profile-iters", type=int, default=3)
    ap.add_argument("--fp64", action="store_true", help="with --profile: the FP64 path")
    ap.add_argument("--quadratic", action="store_true", help="with --profile: the second-order sweep")
    ap.add_argument("--gauss-seidel", action="store_true", help="with --profile: the Gauss-Seidel iteration")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default sweep plan")
    ap.add_argument("--box128", action="store_true", help="with --profile: the 128^3 periodic box (80 rays)")
    ap.add_argument("--plan", default="", help="sweep plan variant,rays_per_group,cluster[,threads] instead of autotuning")
    ap.add_argument("--serve", type=int, default=0, help="run N requests of the serving stream instead")
    ap.add_argument("--rate", type=float, default=2.0, help="with --serve: arrivals per second")
    ap.add_argument("--workers", type=int, default=4, help="with --serve: worker threads")
    ap.add_argument("--shared", type=int, default=0,
                    help="with --serve: shared-launch mode with this many CTAs per cluster (0: off)")
    ap.add_argument("--skip-serve", action="store_true", help="omit the request-stream sample")
    args = ap.parse_args(argv)
    if args.serve:
        return run_serve(args)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.profile:
        return run_profile(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
