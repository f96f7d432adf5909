#!/usr/bin/env python
"""Benchmark: level-scheduled ILU-FGMRES on the 3D 7-point log-normal finite-volume matrix, 128^3.

One step = one pass of the whole hot path over the workload: level analysis of L and U (Eq. 2, 3),
HEC packing of L, U and A (Sec. 2.1, Alg. 1), solve plans, and an ILU(0)-preconditioned FGMRES(30)
solve of A x = b to a 1e-8 relative residual (FP32 factor values, FP64 outer loop), whose every
inner iteration runs the lower and upper sweeps (Alg. 2), SpMV and the Gram-Schmidt kernels.  The
sweeps run partitioned by default (`--sweep part`: 256 x-pencils of the grid, one 512-thread block
each, same results up to summation order); `--sweep global` times the global level-ordered kernel.  The
ILU(0) factors are computed once on the GPU before timing.  Inputs are seeded and synthetic
(ln k ~ N(0, 2^2), b = A x_true with x_true ~ U[-1, 1]); the working set (~1 GB) is larger than L2.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle instead: whole steps of the
same workload (analysis, packing, ILU(0)-FGMRES(30) to 1e-8) on one host core, at most
--ref-max-steps of them (the paper ships no code to run).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "L+U sweep GB/s vs HBM peak; ILU-FGMRES time to 1e-8, FP64 vs mixed/learned"
RESTART = 30
RTOL = 1e-8


def workload_name(m):
    return ("3D 7-point FV %d^3 (n=%d), ln k ~ N(0,2^2), harmonic faces; GPU ILU(0); FP32 L/U values; "
            "FGMRES(%d) FP64 to %.0e" % (m, m ** 3, RESTART, RTOL))


def workload_config(m, nnz_a, nnz_l, nnz_u, world):
    """The `config` object of the JSON line; both arms run the same workload and print the same
    object (the factors' patterns are the same on both sides: ILU(0) of the same matrix)."""
    return {"workload": workload_name(m), "n": m ** 3, "nnz_A": int(nnz_a), "nnz_L": int(nnz_l),
            "nnz_U": int(nnz_u), "parallelism": "replicas" if world > 1 else "single",
            "l2": "inputs larger than L2 (about 1 GB working set)"}


def make_problem(m, seed=0):
    from paper_1606_00541_gb300 import synth
    A = synth.fv7_lognormal(m, sigma=2.0, seed=seed)
    xt = synth.uniform_vector(m ** 3, seed + 1)
    return A, xt


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


SWEEP_PROFILES = {"global": os.path.join(ROOT, "profiles", "k_sweep_fv7_128cubed_ilu0_f32.md"),
                  "part": os.path.join(ROOT, "profiles", "k_sweep_part_fv7_128cubed_pencils_f32.md")}
SWEEP_SOURCES = ("paper_1606_00541_gb300/csrc/sweep.cu", "paper_1606_00541_gb300/csrc/sync.cuh",
                 "paper_1606_00541_gb300/csrc/internal.cuh")


def sweep_source_digest():
    """First 16 hex digits of the SHA-256 of the sweep kernel's sources."""
    h = hashlib.sha256()
    for p in SWEEP_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(schedule):
    """DRAM bytes (read + write) per sweep launch from the committed ncu capture of this workload
    and sweep schedule, or None when the sweep's sources have changed since that capture."""
    try:
        with open(SWEEP_PROFILES[schedule]) as f:
            text = f.read()
    except (OSError, KeyError):
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*(\d+)\s+source_digest:\s*([0-9a-f]+)", text)
    if not m or m.group(2) != sweep_source_digest():
        return None
    return int(m.group(1))


def sweep_bytes(nnz, n, k, sv):
    """Algorithmic bytes of one triangular sweep: values + column indices, tail row pointers, the
    right-hand side read and the solution write (FP64), and the gather / scatter index reads."""
    return nnz * (sv + 4) + 4 * (n + 1) + 2 * n * k * 8 + 2 * 4 * n


# --- clocks ------------------------------------------------------------------------------------

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None
        self.out = None

    def start(self):
        try:
            self.out = open(os.devnull, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            txt, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            txt = ""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in txt.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm), "reasons": sorted(reasons)}


# --- reference arm: the CPU oracle ---------------------------------------------------------------

def oracle_factors(A):
    """The oracle's ILU(0) factors (computed once, before any timing, as the GPU arm's are)."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    L, U = oracle.ilu0(A)
    return L, U, time.perf_counter() - t0


def oracle_step(A, b, L, U, max_iters=5000):
    """One step of the workload on the oracle (serial C, one host core), as the GPU step does it:
    level analysis and HEC packing (FP32 values) of both factors, then ILU(0)-FGMRES(30) from x0 = 0
    to a 1e-8 relative residual.  Returns (seconds, setup seconds, iterations, converged)."""
    import oracle
    t0 = time.perf_counter()
    for T, up in ((L, 0), (U, 1)):
        an = oracle.analyze(T, up)
        oracle.hec_pack(T, 1, up, an["perm"], an["iperm"], vdt="f32")
    t1 = time.perf_counter()
    out = oracle.fgmres(A, b, ("ilu", L, U), m=RESTART, rtol=RTOL, max_iters=max_iters)
    t2 = time.perf_counter()
    return t2 - t0, t1 - t0, out["iters"], bool(out["converged"])


def oracle_warm(A, b, L, U):
    """An untimed warm-up of the oracle: the setup and two FGMRES iterations."""
    import oracle
    an = oracle.analyze(L, 0)
    oracle.hec_pack(L, 1, 0, an["perm"], an["iperm"], vdt="f32")
    oracle.fgmres(A, b, ("ilu", L, U), m=RESTART, rtol=1e-300, max_iters=2)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    m = args.size
    A, xt = make_problem(m)
    import scipy.sparse as sp
    b = sp.csr_matrix((A[2], A[1], A[0])) @ xt
    L, U, fac_s = oracle_factors(A)
    # every step is a whole solve to 1e-8 (several seconds on one core), so the count of timed
    # steps is capped to keep the run within a few minutes; the line reports the count run
    steps = max(1, min(args.steps, args.ref_max_steps))
    warm = max(1, args.warmup)  # each warm-up is short: set-up and two iterations
    for _ in range(warm):
        oracle_warm(A, b, L, U)
    times, its, conv, setups = [], [], [], []
    for _ in range(steps):
        t, ts, it, c = oracle_step(A, b, L, U)
        times.append(t)
        setups.append(ts)
        its.append(it)
        conv.append(c)
    total = sum(times)
    v = steps / total
    line = {"metric": METRIC, "value": v, "unit": "solves/s", "impl": "reference", "n_gpus": args.gpus,
            "steps": steps, "warmup": warm, "ms_per_step": 1000.0 * total / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(m, A[0][-1], len(L[1]), len(U[1]), args.gpus),
            "fgmres_iterations": its[-1], "converged": all(conv),
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": "serial C oracle, one host core: %d whole steps, each level analysis + HEC "
                                       "packing of L and U (%.2f s) and ILU(0)-FGMRES(30) from x0 = 0 to 1e-8 (%d "
                                       "iterations); oracle ILU(0) %.2f s before timing, not counted; %d warm-up "
                                       "steps of setup + 2 iterations"
                                       % (steps, statistics.median(setups), its[-1], fac_s, warm)},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --- replicas (one process per GPU, no collective on the data path) ----------------------------

def max_over_ranks(x, device):
    """The slowest rank's time: the job's time.  A no-op on one process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world, steps, elapsed_max):
    """Solves per second over all replicas: each rank solves `steps` independent systems."""
    return world * steps / elapsed_max


# --- our arm --------------------------------------------------------------------------------------

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=128)
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cfg4", action="store_true", help="also run the 200^3 learned-stage comparison")
    ap.add_argument("--ref-max-steps", type=int, default=20,
                    help="at most this many timed oracle steps (each a whole solve, about 11 s on one Grace "
                         "core) in the reference arm")
    ap.add_argument("--sweep", default="part", choices=["part", "global"],
                    help="single-RHS sweep schedule of the timed step: x-pencil partitioned (default) or global")
    ap.add_argument("--apply-only", choices=["ilu0_16rhs", "ras64_16rhs", "ras_pencils_1rhs", "stage"], default=None,
                    help="only time the L+U apply of this preconditioner (16 right-hand sides, or one for RAS on "
                         "x-pencil subdomains with partitioned sweeps), or one learned-stage application (a "
                         "short run, e.g. to profile a sweep or the convolution)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.apply_only:
        return run_apply_only(args)

    import torch
    import torch.distributed as dist
    from paper_1606_00541_gb300 import hec

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    devn = torch.device("cuda", local)

    m = args.size
    A, xt = make_problem(m)
    n = m ** 3
    Ad = [torch.as_tensor(a, device=devn) for a in A]
    HA0 = hec.hec_from_csr(*Ad)
    xtd = torch.as_tensor(xt, device=devn)
    bd = hec.spmv(HA0, xtd)  # b = A x_true
    t0 = time.perf_counter()
    Lh, Uh = hec.ilu_factor(*Ad, k=0)
    torch.cuda.synchronize()
    factor_s = time.perf_counter() - t0
    L, U = Lh.tensors(), Uh.tensors()
    nnzL, nnzU = L[1].numel(), U[1].numel()

    sched = Schedule(args.sweep, m, devn, torch)

    def step(vdt="f32", Lf=L, Uf=U, b=bd, A_=Ad):
        s = hec.IluSolver(Lf, Uf, A=A_, vdt=vdt)
        sched.apply(s, vdt)
        x, info = s.solve(b, restart=RESTART, rtol=RTOL, max_iters=5000)
        return x, info, s

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    hec.profile_enable(True, categories=[0])  # event records around the sweep launches only
    hec.profile_read(reset=True)
    l0 = hec.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    infos = []
    for _ in range(args.steps):
        x, info, s = step()
        infos.append(info)
    e1.record()
    torch.cuda.synchronize()
    elapsed = e0.elapsed_time(e1) / 1000.0
    launches = hec.launch_count() - l0
    sweep_ms, sweep_launches = hec.profile_read(reset=True)
    hec.profile_enable(False)
    clk = clocks.stop()
    elapsed = max_over_ranks(elapsed, devn)
    value = whole_job_value(world, args.steps, elapsed)
    its = infos[-1]["iterations"]
    xr = x
    res = bd - hec.spmv(HA0, xr)
    relres = float(torch.linalg.norm(res) / torch.linalg.norm(bd))

    # roofline of the dominant kernel (the sweep) from its live CUDA-event durations
    hbm, src = peaks()
    per_sweep = 0.5 * (sweep_bytes(nnzL, n, 1, 4) + sweep_bytes(nnzU, n, 1, 4))
    # the ILU apply keeps its intermediate y in FP32 with FP32 factor values: the lower sweep
    # writes it and the upper sweep reads it at 4 bytes a row instead of 8 (4 bytes less a sweep)
    per_sweep -= 4 * n
    avg_launch_s = (sweep_ms / 1000.0) / max(sweep_launches, 1)
    achieved = per_sweep / avg_launch_s / 1e9
    step_s = elapsed / args.steps
    kname = sched.kernel()
    roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": hbm,
                "unit": "GB/s", "frac": achieved / hbm, "traffic": recorded_traffic(args.sweep), "traffic_unit": "bytes/launch",
                "peak_source": src,
                "sweep_share_of_step": (sweep_ms / 1000.0) / elapsed,
                "avg_sweep_us": avg_launch_s * 1e6, "bytes_per_sweep": per_sweep}
    if args.sweep == "part":
        # the second bound: the dependency chain at the schedule's own measured hop latencies
        lf = level_floor(hec, torch, devn, s.lvL.nlev, sum(k - 1 for k in sweep_grid(m)), part_threads(m))
        lf["frac"] = lf["floor_us"] / (avg_launch_s * 1e6)
        roofline["latency_floor"] = lf

    # e2e: host buffers through the public API, copies inside the timed region
    host = [a.cpu().pin_memory() for a in (*Ad, *L, *U, bd)]
    dev_bufs = [torch.empty_like(a, device=devn) for a in host]
    xh = torch.empty(n, dtype=torch.float64).pin_memory()
    h2d = sum(a.numel() * a.element_size() for a in host)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0.record()
    for _ in range(args.steps):
        for d_, h_ in zip(dev_bufs, host):
            d_.copy_(h_, non_blocking=True)
        Ae, Le, Ue, be = dev_bufs[0:3], dev_bufs[3:6], dev_bufs[6:9], dev_bufs[9]
        xe, _, _ = step("f32", Le, Ue, be, Ae)
        xh.copy_(xe, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    e2e_s = e0.elapsed_time(e1) / 1000.0
    e2e_s = max_over_ranks(e2e_s, devn)

    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * step_s, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": workload_config(m, A[0][-1], nnzL, nnzU, world),
            "fgmres_iterations": its, "true_rel_residual": relres, "factor_s": factor_s,
            "sweep_schedule": sched.describe(),
            "roofline": roofline,
            "e2e": {"value": world * args.steps / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": n * 8},
            "gpu_launches": launches, "clocks": clk}

    if args.sweep in SWEEP_PROFILES:
        tr = recorded_traffic(args.sweep)
        roofline["traffic_source"] = (
            "committed ncu capture %s (dram read + write per launch), sweep source digest %s"
            % (os.path.relpath(SWEEP_PROFILES[args.sweep], ROOT), sweep_source_digest()) if tr is not None
            else "none: the sweep sources changed since the committed capture")
    if rank == 0:
        # where one solve's device time goes, by kernel class (an untimed solve with every launch
        # bracketed by events)
        torch.cuda.synchronize()
        hec.profile_enable(True)
        hec.profile_read(reset=True)
        step()
        torch.cuda.synchronize()
        br = hec.profile_breakdown()
        hec.profile_read(reset=True)
        hec.profile_enable(False)
        line["breakdown_ms"] = {k: round(v[0], 3) for k, v in br.items()}
    if rank == 0:
        # the metric's comparison, short enough to stay in view: FP64 against mixed-precision
        # factors, time to 1e-8 with the bench's schedule
        pt = precision_times(hec, torch, Ad, L, U, bd, sched)
        head = {}
        for k, v in line.items():
            head[k] = v
            if k == "ms_per_step":
                head["time_to_1e-8_s"] = {k2: v2["time_to_1e-8_s"] for k2, v2 in pt.items()}
                head["iterations_to_1e-8"] = {k2: v2["iterations"] for k2, v2 in pt.items()}
                if "latency_floor" in roofline:
                    head["latency_floor_us"] = roofline["latency_floor"]["floor_us"]
                    head["sweep_us"] = roofline["avg_sweep_us"]
                head["breakdown_ms"] = line.get("breakdown_ms")
                head["gram_schmidt"] = gram_schmidt_times(hec, torch, Ad, L, U, bd, sched)
                head["ras_pencils"] = ras_pencil_times(hec, torch, Ad, bd, m, hbm)
        line = head
    if rank == 0 and not args.no_variants:
        line["variants"] = variants(hec, torch, Ad, L, U, bd, HA0, n, nnzL, nnzU, hbm, Schedule("part", m, devn, torch))
        line["variants"]["learned_%d" % m] = learned_variant(hec, torch, m)
        if args.cfg4:
            line["variants"]["learned_200"] = learned_variant(hec, torch, 200)
    if rank == 0 and world == 1 and not args.no_cpu:
        try:
            bh = bd.cpu().numpy()
            Lo, Uo, fac = oracle_factors(A)
            t, ts, it, conv = oracle_step(A, bh, Lo, Uo)
            line["cpu_baseline"] = {"value": 1.0 / t, "unit": "solves/s", "cores": 1, "kind": "oracle",
                                    "sample": "serial C oracle on one host core, one whole step: level analysis + "
                                              "HEC packing of L and U (%.2f s) and ILU(0)-FGMRES(30) to 1e-8 "
                                              "(%d iterations, converged %s); oracle ILU(0) %.2f s not counted"
                                              % (ts, it, conv, fac)}
        except Exception as e:  # the baseline is reported, not required
            line["cpu_baseline"] = {"value": None, "unit": "solves/s", "cores": 1, "kind": "oracle",
                                    "sample": "failed: %s" % e}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def precision_times(hec, torch, Ad, L, U, bd, sched):
    """Time to a 1e-8 relative residual (solve only, after one warm solve) with FP64, FP32 and BF16
    factor values, on the given single-RHS schedule."""
    out = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for vdt in ("f64", "f32", "bf16"):
        s = hec.IluSolver(L, U, A=Ad, vdt=vdt)
        sched.apply(s, vdt)
        s.solve(bd, restart=RESTART, rtol=RTOL, max_iters=5000)
        torch.cuda.synchronize()
        e0.record()
        _, info = s.solve(bd, restart=RESTART, rtol=RTOL, max_iters=5000)
        e1.record()
        torch.cuda.synchronize()
        out[vdt] = {"time_to_1e-8_s": e0.elapsed_time(e1) / 1000.0, "iterations": info["iterations"],
                    "converged": info["converged"], "reorthogonalized": info["reorthogonalized"]}
    return out


def gram_schmidt_times(hec, torch, Ad, L, U, bd, sched):
    """Time to 1e-8 with FP32 factor values under each Gram-Schmidt variant of the Arnoldi step
    (classical with selective reorthogonalization, the library default, and modified), and the
    device time of the Gram-Schmidt kernel in each solve."""
    out = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    default = hec.get_gram_schmidt()
    try:
        for mode in ("classical", "modified"):
            hec.set_gram_schmidt(mode)
            s = hec.IluSolver(L, U, A=Ad, vdt="f32")
            sched.apply(s, "f32")
            s.solve(bd, restart=RESTART, rtol=RTOL, max_iters=5000)
            torch.cuda.synchronize()
            e0.record()
            _, info = s.solve(bd, restart=RESTART, rtol=RTOL, max_iters=5000)
            e1.record()
            torch.cuda.synchronize()
            hec.profile_enable(True, categories=[2])
            hec.profile_read(reset=True)
            s.solve(bd, restart=RESTART, rtol=RTOL, max_iters=5000)
            torch.cuda.synchronize()
            gs_ms = hec.profile_breakdown()["gram_schmidt"][0]
            hec.profile_read(reset=True)
            hec.profile_enable(False)
            out[mode] = {"time_to_1e-8_s": e0.elapsed_time(e1) / 1000.0, "iterations": info["iterations"],
                         "reorthogonalized": info["reorthogonalized"], "gram_schmidt_ms": round(gs_ms, 3)}
    finally:
        hec.set_gram_schmidt(default)
    return out


def variants(hec, torch, Ad, L, U, bd, HA0, n, nnzL, nnzU, hbm, part):
    """Time-to-1e-8 of the plain FP64 form next to the mixed forms, and L+U sweep bandwidth, with
    the global and the x-pencil partitioned single-RHS sweep schedules."""
    out = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed_solve(s):
        s.solve(bd, restart=RESTART, rtol=RTOL, max_iters=5000)
        torch.cuda.synchronize()
        e0.record()
        x, info = s.solve(bd, restart=RESTART, rtol=RTOL, max_iters=5000)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1000.0, info

    def timed_apply(s, r, reps=10):
        for _ in range(3):
            s.apply(r)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            s.apply(r)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1000.0 / reps

    for vdt in ["f64", "f32", "bf16"]:
        s = hec.IluSolver(L, U, A=Ad, vdt=vdt, max_nrhs=16)
        t, info = timed_solve(s)
        sv = {"f64": 8, "f32": 4, "bf16": 2}[vdt]
        gbs = {}
        for k in (1, 16):
            r = torch.randn(n, k, dtype=torch.float64, device=bd.device) if k > 1 else bd
            ta = timed_apply(s, r)
            B = sweep_bytes(nnzL, n, k, sv) + sweep_bytes(nnzU, n, k, sv)
            gbs["nrhs%d" % k] = {"lu_us": ta * 1e6, "lu_gbs": B / ta / 1e9, "frac_hbm": B / ta / 1e9 / hbm,
                                 "rows_per_s": n * k / ta}
        out[vdt] = {"time_to_1e-8_s": t, "iterations": info["iterations"], "converged": info["converged"],
                    "true_rel_residual": info["rel_residual"]}
        # the same factors with the partitioned single-RHS schedule
        for key, sch in (("partitioned", part),):
            sch.apply(s, vdt)
            tp, infop = timed_solve(s)
            ta = timed_apply(s, bd)
            B = sweep_bytes(nnzL, n, 1, sv) + sweep_bytes(nnzU, n, 1, sv)
            gbs["nrhs1_" + key] = {"lu_us": ta * 1e6, "lu_gbs": B / ta / 1e9, "frac_hbm": B / ta / 1e9 / hbm,
                                   "rows_per_s": n / ta}
            out[vdt][key] = {"time_to_1e-8_s": tp, "iterations": infop["iterations"],
                             "converged": infop["converged"], "true_rel_residual": infop["rel_residual"]}
        out[vdt].update({"sweeps": gbs, "levels_L": s.lvL.nlev, "levels_U": s.lvU.nlev})
    out.update(batched_variants(hec, torch, Ad, L, U, n, hbm))
    out["stencil27_ilu0_100"] = long_row_variant(hec, torch, hbm, Ad[0].device)
    out["stencil27_ilut_100"] = long_row_variant(hec, torch, hbm, Ad[0].device, ilut=(10, 1e-3))
    return out


def learned_variant(hec, torch, m, seed=0, crop=32, crops=125, epochs=8, log=None):
    """ILU(0)-FGMRES(30) with and without the learned correction stage on the m^3 log-normal
    7-point problem (FP32 factor values).  The network is trained from scratch on 2000 (residual,
    error) pairs (125 crops of crop^3 from the same permeability field x 16 seeded right-hand
    sides) generated by the FP64 solver; data generation and training times are reported apart."""
    from paper_1606_00541_gb300 import learn, synth
    lnk = np.log(synth.lognormal_perm(m, 2.0, seed))
    A = synth.fv7_lognormal(m, perm=np.exp(lnk))
    net, tinfo = learn.train_stage(lnk, m, crop=crop, crops=crops, rhs_per_crop=16, epochs=epochs, batch=8, lr=2e-3,
                                   seed=seed + 1, log=log)
    Ad = [torch.as_tensor(a, device="cuda") for a in A]
    Lh, Uh = hec.ilu_factor(*Ad, k=0)
    s = hec.IluSolver(Lh.tensors(), Uh.tensors(), A=Ad, vdt="f32")
    b = hec.spmv(s.A, torch.as_tensor(synth.uniform_vector(m ** 3, seed + 1), device="cuda"))
    # the single-RHS schedule for both forms: the library's autotuner keeps the x-pencil partition
    # or the global sweep, whichever is faster on these factors
    sched = Schedule("part", m, b.device, torch)
    sched.apply(s)
    tuned = s.autotune(1)
    schedule = ("x-pencil partitioned, %d parts" % sched.nparts if all(t["partitioned"] for t in tuned)
                else "global") + " (sptrsv_autotune: %s)" % (list(tuned),)
    stage = hec.Stage(net, s.A, (m, m, m), torch.as_tensor(lnk, device="cuda"), rho=0.99)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {"train": tinfo, "sweep_schedule": schedule}
    for name, st in (("plain", None), ("learned", stage)):
        hec.fgmres_solve(s.A, s.M, b, stage=st, restart=RESTART, rtol=RTOL, max_iters=5000)  # warm
        if st is not None:
            st.stats(reset=True)
        torch.cuda.synchronize()
        e0.record()
        x, info = hec.fgmres_solve(s.A, s.M, b, stage=st, restart=RESTART, rtol=RTOL, max_iters=5000)
        e1.record()
        torch.cuda.synchronize()
        rel = float(torch.linalg.norm(b - hec.spmv(s.A, x)) / torch.linalg.norm(b))
        res[name] = {"time_to_1e-8_s": e0.elapsed_time(e1) / 1000.0, "iterations": info["iterations"],
                     "converged": info["converged"], "true_rel_residual": rel}
        if st is not None:
            res[name]["stage"] = st.stats()
    res["n"] = m ** 3
    return res




class Schedule:
    """The single-RHS sweep schedule a solver is given: "global" (the level-ordered kernel over the
    whole factor) or "part" (x-pencil parts, one resident block each, sptrsv_plan_partition)."""

    def __init__(self, kind, m, device, torch):
        from paper_1606_00541_gb300 import synth
        self.kind, self.m = kind, m
        if kind == "part":
            part, self.nparts = synth.grid_boxes(m, sweep_grid(m))
            self.part = torch.as_tensor(part, device=device)

    def apply(self, s, vdt="f32"):
        if self.kind == "part":
            s.partition(self.part, self.nparts, threads=part_threads(self.m))

    def kernel(self):
        return {"global": "k_sweep<float,float,1,4>", "part": "k_sweep_part<float,float,4>"}[self.kind]

    def describe(self):
        if self.kind == "part":
            return "x-pencil partitioned: %d parts, %d threads per part" % (self.nparts, part_threads(self.m))
        return "global level-ordered"


def chain_csr(n):
    """CSR of the lower bidiagonal chain used by level_floor: row 0 holds only
    its diagonal, row i > 0 holds (i-1, i); so row i is at level i and every level has one row
    with one dependency."""
    import numpy as np
    col = np.empty(2 * n - 1, np.int32)
    col[0] = 0
    col[1::2] = np.arange(0, n - 1)
    col[2::2] = np.arange(1, n)
    val = np.empty(2 * n - 1)
    val[0] = 1.0
    val[1::2] = -0.5
    val[2::2] = 1.0
    rp = np.concatenate([[0], np.arange(1, 2 * n, 2)]).astype(np.int32)
    return rp, col, val


def level_floor(hec, torch, device, levels, crossings, threads, vdt="f32", n=4096, reps=10):
    """The level-latency bound of the partitioned sweep, measured with its own synchronisation (an
    empty-level micro-benchmark): a bidiagonal lower factor of n rows (one row and one dependency
    per level) swept as one part gives the in-part hop t_local; with its rows alternating between
    two parts every dependency crosses, which gives the cross-part hop t_cross.  A sweep of
    `levels` levels whose chain crosses `crossings` part boundaries cannot finish in less than
    (levels - crossings) t_local + crossings t_cross.  Kernel-only times (library event profile)."""
    rp_d, ci_d, v_d = (torch.as_tensor(a, device=device) for a in chain_csr(n))
    lv = hec.sptrsv_analyze(rp_d, ci_d, 0)
    plan = hec.sptrsv_plan_create(hec.hec_from_csr(rp_d, ci_d, v_d, levels=lv, vdt=vdt), lv)
    b = torch.ones(n, dtype=torch.float64, device=device)
    x = torch.empty_like(b)
    hop = {}
    for name, part, nparts in (("t_local_us", torch.zeros(n, dtype=torch.int32, device=device), 1),
                               ("t_cross_us", (torch.arange(n, device=device) % 2).to(torch.int32), 2)):
        hec.sptrsv_plan_partition(plan, part, nparts, threads)
        for _ in range(3):
            hec.sptrsv_lower(plan, b, x)
        torch.cuda.synchronize()
        hec.profile_enable(True)
        hec.profile_read(reset=True)
        for _ in range(reps):
            hec.sptrsv_lower(plan, b, x)
        torch.cuda.synchronize()
        ms, nl = hec.profile_read(reset=True)
        hec.profile_enable(False)
        hop[name] = ms * 1000.0 / max(nl, 1) / n
    floor = (levels - crossings) * hop["t_local_us"] + crossings * hop["t_cross_us"]
    return {"levels": levels, "crossings": crossings, **hop, "floor_us": floor,
            "method": "bidiagonal chain of %d rows, one part / two alternating parts, %d threads" % (n, threads)}


def sweep_grid(m):
    """Boxes per axis of the x-pencil partition used on an m^3 grid: the y-z plane cut into 16 x 16
    boxes (256 parts, two resident 512-thread blocks an SM), so a dependency chain crosses a part
    boundary at most 30 times and every other step stays in one SM's shared memory.  Measured at
    128^3, FP32 ILU(0) apply: 403 us against 432-436 us for 12 x 12 pencils of 1024 threads, 417 us
    for 8 x 19, 432 us for 8 x 38 and 445 us for 16 x 16 with 256 threads.  Grids above 160^3
    take 8 x 19 pencils (152 parts, one 1024-thread block each) so that a part's FP32 solution
    still fits in shared memory."""
    return (1, 16, 16) if m <= 160 else (1, 8, 19)


def part_threads(m):
    """Threads of a part's block for the partition of sweep_grid(m)."""
    return 512 if m <= 160 else 1024


def ras_cuts(m):
    """Per-axis box cuts: [25, 39, 25, 39] on 128 (64 boxes of 25^3 .. 39^3 owned rows)."""
    a, b = m * 25 // 128, m * 39 // 128
    return [a, b, a, m - 2 * a - b]


def long_row_variant(hec, torch, hbm, device, m=100, ilut=None):
    """Long rows: the 27-point jittered stencil on 100^3 (a_ii = 1.05 sum |a_ij|, +-30 % jitter)
    with its GPU ILU(0) (13 strictly lower entries per interior row) or GPU ILUT(p, tol);
    single-RHS L+U apply with one lane per row against the autotuned plans (launch shape and lanes
    per row of each factor), 16-RHS L+U, and FGMRES(30) to 1e-8 with FP32 and FP64 factor values."""
    from paper_1606_00541_gb300 import synth
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    A = [torch.as_tensor(a, device=device) for a in synth.stencil27_jitter(m, seed=0)]
    n = m ** 3
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Lh, Uh = hec.ilut_factor(*A, p=ilut[0], tol=ilut[1]) if ilut else hec.ilu_factor(*A, k=0)
    torch.cuda.synchronize()
    factor_s = time.perf_counter() - t0
    L, U = Lh.tensors(), Uh.tensors()
    nnzL, nnzU = L[1].numel(), U[1].numel()
    b = hec.spmv(hec.hec_from_csr(*A), torch.as_tensor(synth.uniform_vector(n, 600), device=device))
    out = {"factorization": "ILUT(%d, %g)" % ilut if ilut else "ILU(0)", "factor_s": factor_s, "n": n,
           "nnz_A": int(A[1].numel()), "nnz_L": nnzL, "nnz_U": nnzU}
    for vdt, sv in (("f64", 8), ("f32", 4)):
        res = {}
        for lpr in (1, 0):
            s = hec.IluSolver(L, U, A=A, vdt=vdt, lanes_per_row=lpr)
            tuned = s.autotune(1) if lpr == 0 else None  # launch shape and lanes per row by the autotuner
            for _ in range(3):
                s.apply(b)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(10):
                s.apply(b)
            e1.record()
            torch.cuda.synchronize()
            ta = e0.elapsed_time(e1) / 1000.0 / 10
            B = sweep_bytes(nnzL, n, 1, sv) + sweep_bytes(nnzU, n, 1, sv)
            key = "one_lane" if lpr == 1 else "autotuned_lanes_%d_%d" % (tuned[0]["lanes_per_row"],
                                                                           tuned[1]["lanes_per_row"])
            res[key] = {"lu_us": ta * 1e6, "lu_gbs": B / ta / 1e9, "frac_hbm": B / ta / 1e9 / hbm}
            if lpr == 0:
                s.solve(b, restart=RESTART, rtol=RTOL, max_iters=5000)
                torch.cuda.synchronize()
                e0.record()
                _, info = s.solve(b, restart=RESTART, rtol=RTOL, max_iters=5000)
                e1.record()
                torch.cuda.synchronize()
                res["time_to_1e-8_s"] = e0.elapsed_time(e1) / 1000.0
                res["iterations"] = info["iterations"]
                res["converged"] = info["converged"]
                res["levels_L"], res["levels_U"] = s.lvL.nlev, s.lvU.nlev
        s16 = hec.IluSolver(L, U, vdt=vdt, max_nrhs=16)
        r16 = torch.randn(n, 16, dtype=torch.float64, device=device)
        for _ in range(3):
            s16.apply(r16)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(5):
            s16.apply(r16)
        e1.record()
        torch.cuda.synchronize()
        t16 = e0.elapsed_time(e1) / 1000.0 / 5
        B16 = sweep_bytes(nnzL, n, 16, sv) + sweep_bytes(nnzU, n, 16, sv)
        res["nrhs16"] = {"lu_us": t16 * 1e6, "lu_gbs": B16 / t16 / 1e9, "frac_hbm": B16 / t16 / 1e9 / hbm}
        out[vdt] = res
    return out


def run_stage_only(args):
    """One learned-stage application (z1 -> z: the residual's SpMV, the 4-layer network on the m^3
    field, the correction's SpMV and the gated step) on the log-normal 7-point problem with ILU(0)
    FP32 factors and an untrained network, W untimed and K timed applications per engine (tcgen05,
    then mma.sync); prints one JSON line with the application times."""
    import torch
    from paper_1606_00541_gb300 import hec, learn, synth
    m = args.size
    n = m ** 3
    lnk = np.log(synth.lognormal_perm(m, 2.0, 0))
    A = synth.fv7_lognormal(m, perm=np.exp(lnk))
    Ad = [torch.as_tensor(a, device="cuda") for a in A]
    Lh, Uh = hec.ilu_factor(*Ad, k=0)
    s = hec.IluSolver(Lh.tensors(), Uh.tensors(), A=Ad, vdt="f32")
    net = hec.Net(learn.init_params(1))
    stage = hec.Stage(net, s.A, (m, m, m), torch.as_tensor(lnk, device="cuda"))
    v = torch.as_tensor(synth.uniform_vector(n, 7), device="cuda")
    z1 = s.apply(v)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"apply": "stage", "n": n}
    for engine, tc in (("tcgen05", True), ("mma_sync", False)):
        net.set_engine(tc)
        for _ in range(args.warmup):
            stage.apply(v, z1)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            stage.apply(v, z1)
        e1.record()
        torch.cuda.synchronize()
        net.sync_status()
        out["stage_apply_us_" + engine] = e0.elapsed_time(e1) * 1000.0 / args.steps
    net.set_engine(True)
    print(json.dumps(out), flush=True)


def run_apply_only(args):
    """The 16-right-hand-side L+U apply of one preconditioner (GPU ILU(0) of the whole matrix, or
    RAS with 64 box subdomains), FP32 factor values, autotuned launch shape, or the single-RHS
    apply of RAS on box subdomains (ras_pencil_grid) with one partitioned part per subdomain: W untimed
    and K timed applies; prints one JSON line with the apply time and its algorithmic GB/s."""
    import torch
    from paper_1606_00541_gb300 import hec, synth
    if args.apply_only == "stage":
        return run_stage_only(args)
    m = args.size
    n = m ** 3
    A, _ = make_problem(m)
    Ad = [torch.as_tensor(a, device="cuda") for a in A]
    k = 1 if args.apply_only == "ras_pencils_1rhs" else 16
    B = torch.as_tensor(synth.uniform_vector(n, 500, nrhs=k), device="cuda")
    if args.apply_only == "ras_pencils_1rhs":
        nb, threads = ras_pencil_grid(m)
        part, ns = synth.grid_boxes(m, nb)
        s = hec.RasSolver(Ad, torch.as_tensor(part, device="cuda"), ns, vdt="f32")
        sp, nsp = subdomain_parts(s.ext_ptr.cpu().numpy())
        s.partition(torch.as_tensor(sp, device="cuda"), nsp, threads=threads)
        nnzl, nnzu = int(s.L[1].numel()), int(s.U[1].numel())
    elif args.apply_only == "ras64_16rhs":
        part, ns = synth.box_partition(m, ras_cuts(m))
        s = hec.RasSolver(Ad, torch.as_tensor(part, device="cuda"), ns, vdt="f32", max_nrhs=16)
        nnzl, nnzu = int(s.L[1].numel()), int(s.U[1].numel())
    else:
        Lh, Uh = hec.ilu_factor(*Ad, k=0)
        L, U = Lh.tensors(), Uh.tensors()
        s = hec.IluSolver(L, U, vdt="f32", max_nrhs=16)
        nnzl, nnzu = int(L[1].numel()), int(U[1].numel())
    shapes = s.autotune(16) if k == 16 else "%s box subdomains, %d threads a part" % ras_pencil_grid(m)
    for _ in range(args.warmup):
        s.apply(B)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        s.apply(B)
    e1.record()
    torch.cuda.synchronize()
    ta = e0.elapsed_time(e1) / 1000.0 / args.steps
    nl = s.HL.info().n
    Bytes = sweep_bytes(nnzl, nl, k, 4) + sweep_bytes(nnzu, nl, k, 4)
    hbm, src = peaks()
    print(json.dumps({"apply": args.apply_only, "rows": nl, "levels_L": s.lvL.nlev, "levels_U": s.lvU.nlev,
                      "lu_apply_us": ta * 1e6, "bytes": Bytes, "lu_gbs": Bytes / ta / 1e9,
                      "frac_hbm": Bytes / ta / 1e9 / hbm, "launch_shape": shapes}), flush=True)


def ras_pencil_grid(m):
    """Subdomain boxes per axis and threads a part of the RAS form with one partitioned part per
    subdomain, or None where the extended solution cannot stay in the SMs' shared memory.  On
    128^3, 4 x 12 x 12 boxes of 32 x 10..11 x 10..11 cells (576 subdomains, 54 levels a factor,
    four 256-thread parts an SM).  Measured there, FP32 values, FGMRES(30) to 1e-8 (iterations,
    levels a factor): 4 x 12 x 12 / 256 threads 51.0 ms (148, 54); 2 x 8 x 19 / 512 52.5 ms
    (149, 87); 2 x 12 x 12 / 512 52.6 ms (147, 86); 3 x 12 x 12 / 256 52.9 ms (148, 65);
    2 x 16 x 16 / 256 56.8 ms (157, 80); 1 x 12 x 12 / 1024 58.3 ms (148, 150); 1 x 16 x 16 / 512
    61.0 ms (155, 144); 1 x 20 x 20 / 256 63.4 ms (149, 142); 1 x 16 x 16 without overlap (block
    ILU) 83.7 ms (225, 142)."""
    return ((4, 12, 12), 256) if m <= 160 else None


def subdomain_parts(ext_ptr):
    """Part vector over the extended rows of a RAS system that makes every subdomain one part of
    the partitioned sweep (the block-diagonal factors have no dependency between subdomains, so
    no chain crosses a part)."""
    sizes = np.diff(np.asarray(ext_ptr, dtype=np.int64))
    return np.repeat(np.arange(len(sizes), dtype=np.int32), sizes), len(sizes)


def ras_pencil_times(hec, torch, Ad, bd, m, hbm, vdts=("f64", "f32")):
    """RAS (Sec. 3, Eq. 4) with the m^3 grid cut into box subdomains (ras_pencil_grid, overlap 1),
    one resident part per subdomain, single right-hand side b of the main workload: set-up
    (GPU extension, ILU(0) of every block, analysis, packing, partitioned layout) and
    FGMRES(30) to 1e-8 with plain FP64 and mixed FP32 factor values, and the L+U apply."""
    from paper_1606_00541_gb300 import synth
    grid = ras_pencil_grid(m)
    if grid is None:
        return {"skipped": "the extended solution of %d^3 does not fit in the SMs' shared memory" % m}
    nb, threads = grid
    dev = Ad[0].device
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    part, ns = synth.grid_boxes(m, nb)
    out = {"subdomains": ns, "boxes": list(nb), "overlap": 1, "threads_per_part": threads}
    for vdt in vdts:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = hec.RasSolver(Ad, torch.as_tensor(part, device=dev), ns, vdt=vdt)
        sp, nsp = subdomain_parts(s.ext_ptr.cpu().numpy())
        s.partition(torch.as_tensor(sp, device=dev), nsp, threads=threads)
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        s.solve(bd, restart=RESTART, rtol=RTOL, max_iters=5000)
        torch.cuda.synchronize()
        e0.record()
        _, info = s.solve(bd, restart=RESTART, rtol=RTOL, max_iters=5000)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1000.0
        r = torch.zeros(bd.shape[0], dtype=torch.float64, device=dev)
        r.copy_(bd)
        for _ in range(3):
            s.apply(r)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(10):
            s.apply(r)
        e1.record()
        torch.cuda.synchronize()
        ta = e0.elapsed_time(e1) / 1000.0 / 10
        sv = {"f64": 8, "f32": 4, "bf16": 2}[vdt]
        nl, nu = s.HL.info(), s.HU.info()
        B = sweep_bytes(int(s.L[1].numel()), nl.n, 1, sv) + sweep_bytes(int(s.U[1].numel()), nu.n, 1, sv)
        out[vdt] = {"time_to_1e-8_s": t, "iterations": info["iterations"], "converged": info["converged"],
                    "true_rel_residual": info["rel_residual"], "setup_s": setup_s, "rows": nl.n,
                    "levels_L": s.lvL.nlev, "levels_U": s.lvU.nlev, "lu_apply_us": ta * 1e6,
                    "lu_gbs": B / ta / 1e9, "frac_hbm": B / ta / 1e9 / hbm}
        del s
    return out


def batched_variants(hec, torch, Ad, L, U, n, hbm):
    """16 right-hand sides: global ILU(0) and batched RAS (64 box subdomains, overlap 1, one pair of
    sweeps for all subdomains), FP32 factor values, autotuned launch shapes, FGMRES(30) to 1e-8."""
    from paper_1606_00541_gb300 import synth
    out = {}
    m = round(n ** (1.0 / 3.0))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    Xt = torch.as_tensor(synth.uniform_vector(n, 500, nrhs=16), device=Ad[0].device)
    HA = hec.hec_from_csr(*Ad)
    B = hec.spmv(HA, Xt)
    part, ns = synth.box_partition(m, ras_cuts(m))
    t0 = time.perf_counter()
    ras = hec.RasSolver(Ad, torch.as_tensor(part, device=Ad[0].device), ns, vdt="f32", max_nrhs=16)
    torch.cuda.synchronize()
    ras_setup_s = time.perf_counter() - t0
    ilu = hec.IluSolver(L, U, A=Ad, vdt="f32", max_nrhs=16)
    for name, s in (("ilu0_f32_16rhs", ilu), ("ras64_f32_16rhs", ras)):
        shapes = s.autotune(16)
        s.solve(B, restart=RESTART, rtol=RTOL, max_iters=5000)
        torch.cuda.synchronize()
        e0.record()
        X, info = s.solve(B, restart=RESTART, rtol=RTOL, max_iters=5000)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1000.0
        # L+U bandwidth of one 16-column apply
        for _ in range(3):
            s.apply(B)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(5):
            s.apply(B)
        e1.record()
        torch.cuda.synchronize()
        ta = e0.elapsed_time(e1) / 1000.0 / 5
        nl, nu = s.HL.info(), s.HU.info()
        nnzl = int(s.L[1].numel()) if hasattr(s, "L") else int(L[1].numel())
        nnzu = int(s.U[1].numel()) if hasattr(s, "U") else int(U[1].numel())
        Bytes = sweep_bytes(nnzl, nl.n, 16, 4) + sweep_bytes(nnzu, nu.n, 16, 4)
        out[name] = {"time_to_1e-8_s": t, "iterations": info["iterations"], "converged": info["converged"],
                     "true_rel_residual": info["rel_residual"], "rows": nl.n, "levels_L": s.lvL.nlev,
                     "levels_U": s.lvU.nlev, "lu_apply_us": ta * 1e6, "lu_gbs": Bytes / ta / 1e9,
                     "frac_hbm": Bytes / ta / 1e9 / hbm, "launch_shape": shapes}
    out["ras64_f32_16rhs"]["subdomains"] = ns
    out["ras64_f32_16rhs"]["setup_s"] = ras_setup_s
    return out


if __name__ == "__main__":
    main()
