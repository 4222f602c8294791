#!/usr/bin/env python
"""ORAS-GMRES time-to-1e-8 on one GB300: solves/s of the mixed-precision path vs FP64.

Workload (default "sphere_h0025"): unit sphere, h = 0.025, tricubic CPM band (N_A =
140,270), c = 1, f = (c+12) xyz at the closest points, 64 subdomains by coordinate
bisection, overlap 3, ORAS with alpha = 4 and alpha_x = 40 near cross points,
right-preconditioned FGMRES(50) to a 1e-8 relative residual.  Factors are set up once
(setup timed separately); one step = one complete FGMRES solve with the factors resident.
The mixed path keeps the local LU factors in FP32 (FP64 Krylov and operator); the FP64
path keeps them in FP64; BF16 factors are reported as a third form.

Multi-GPU: `torchrun --nproc-per-node N bench.py --gpus N` runs N independent replicas
(one per GPU, no collective on the data path); value = all ranks' solves / max time.
`--impl reference` times the CPU FP64 oracle on the same workload (bounded sample).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ORAS-GMRES time-to-1e-8 residual, mixed vs FP64 (solves/s, HBM GB/s); p50/p99"
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "trsv_fp32_sphere_h0025.md")


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def replica_rate(total_ms: float, steps: int, device=None):
    """Replicas (one independent solver per GPU, no collective on the data path): the job's
    timed region is the slowest rank's, the rate counts every rank's solves.  Returns
    (max total ms over ranks, whole-job solves/s)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, world * steps / (total_ms / 1e3)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _file_sha(path):
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def _profiled_traffic():
    """DRAM bytes per launch from the committed ncu summary, if it still matches the kernel."""
    src = os.path.join(ROOT, "paper_1909_08734_gb300", "csrc", "cuda", "trsv.cu")
    if not os.path.exists(PROFILE_SUMMARY):
        return None
    fields = {}
    for line in open(PROFILE_SUMMARY):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            fields[k.strip()] = v.strip()
    if fields.get("source_sha256_16") != _file_sha(src):
        return None
    try:
        return float(fields["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def run_kernel_only(args):
    """Set up one preconditioner and launch only the batched solve (for profiler captures)."""
    import torch
    import paper_1909_08734_gb300 as G
    from workloads import WORKLOADS, leaf_weights
    wl = WORKLOADS[args.workload]
    band = G.cpm_build_band(wl.surface, wl.R, wl.r, wl.h, wl.p)
    part = G.cpm_partition(band, wl.n_sub, leaf_weights(wl.n_sub, wl.weight_seed), wl.n_overlap)
    pc = G.oras_setup(band, part, wl.c, wl.method, wl.alpha, wl.alpha_x, args.precision)
    schedule = G.oras_autotune(pc)                 # the schedule the timed solves use
    r = torch.randn(pc.n_active, dtype=torch.float64, device="cuda")
    z = torch.empty_like(r)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("kernel_only")
    for _ in range(args.kernel_only):
        G.oras_apply(pc, r, z)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    G.oras_check_status(pc)
    print(json.dumps({"workload": wl.name, "precision": args.precision, "launches": args.kernel_only,
                      "schedule": schedule,
                      **{k: v for k, v in pc.info().items()
                         if k in ("factor_bytes", "sum_n2", "n_sub", "tile_rows", "solve_offdiag_tiles")}}))


def run_native(args):
    import torch
    import paper_1909_08734_gb300 as G
    from workloads import WORKLOADS, rhs

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    wl = WORKLOADS[args.workload]
    dev = torch.device("cuda", local)

    t0 = time.time()
    band = G.cpm_build_band(wl.surface, wl.R, wl.r, wl.h, wl.p)
    from workloads import leaf_weights
    part = G.cpm_partition(band, wl.n_sub, leaf_weights(wl.n_sub, wl.weight_seed), wl.n_overlap)
    host_setup_s = time.time() - t0
    cp = band.info()["cp"]
    pcs = {}
    setup_s = {}
    schedules = {}
    for prec in ["fp32", "bf16", "fp64"] if not args.no_fp64 else ["fp32", "bf16"]:
        torch.cuda.synchronize()
        t = time.time()
        pcs[prec] = G.oras_setup(band, part, wl.c, wl.method, wl.alpha, wl.alpha_x, prec)
        torch.cuda.synchronize()
        setup_s[prec] = time.time() - t
        t = time.time()
        schedules[prec] = G.oras_autotune(pcs[prec])
        setup_s[prec + "_autotune"] = time.time() - t
    pc = pcs["fp32"]
    n = pc.n_active
    f_host = rhs(wl, cp[:n])
    f = torch.tensor(f_host, dtype=torch.float64, device=dev)
    u = torch.zeros_like(f)
    stream = torch.cuda.current_stream(dev)

    def solve(p, ff, uu):
        return G.cpm_gmres_solve(p, ff, uu, restart=wl.restart, tol=wl.tol, max_it=wl.max_it,
                                 stream=stream)

    def timed_solves(p, k, w):
        for _ in range(w):
            solve(p, f, u)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(k + 1)]
        res = []
        ev[0].record(stream)
        for i in range(k):
            res.append(solve(p, f, u))
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
        per = [ev[i].elapsed_time(ev[i + 1]) for i in range(k)]
        return per, res

    # ---- headline: mixed (FP32 factors) ----
    for _ in range(args.warmup):
        solve(pc, f, u)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = pc.info()["kernel_launches"]
    sampler = ClockSampler(local)
    sampler.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    results = []
    torch.cuda.nvtx.range_push("timed_solves")
    ev[0].record(stream)
    for i in range(args.steps):
        results.append(solve(pc, f, u))
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    clocks = sampler.stop()
    if world > 1:
        torch.distributed.barrier()
    per_step = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    total_ms, value = replica_rate(sum(per_step), args.steps, dev)
    launches = pc.info()["kernel_launches"] - launches0
    iters = results[-1][0]["iterations"]
    relres = results[-1][0]["relres"]

    # ---- solution error of the mixed path against the FP64 path ----
    extra = {}
    if "fp64" in pcs:
        u64 = torch.zeros_like(f)
        per64, res64 = timed_solves(pcs["fp64"], max(3, args.steps // 2), 1)
        solve(pcs["fp64"], f, u64)
        solve(pc, f, u)
        torch.cuda.synchronize()
        diff = (torch.linalg.norm(u - u64) / torch.linalg.norm(u64)).item()
        extra["fp64"] = {"solves_per_s": 1e3 / statistics.mean(per64),
                         "ms_p50": statistics.median(per64), "iterations": res64[-1][0]["iterations"],
                         "relres": res64[-1][0]["relres"], "setup_s": setup_s["fp64"],
                         "setup_ms_factor": pcs["fp64"].info()["setup_ms_factor"]}
        extra["mixed_vs_fp64_solution_rel_diff"] = diff
        extra["mixed_speedup_vs_fp64_solve"] = extra["fp64"]["ms_p50"] / statistics.median(per_step)
        extra["mixed_speedup_vs_fp64_setup_plus_solve"] = (
            (setup_s["fp64"] + extra["fp64"]["ms_p50"] / 1e3) /
            (setup_s["fp32"] + statistics.median(per_step) / 1e3))
        # the metric reported twice: solve with factors resident (value) and set-up + solve
        extra["setup_plus_solve_s"] = {
            "fp32": round(host_setup_s + setup_s["fp32"] + statistics.median(per_step) / 1e3, 4),
            "fp64": round(host_setup_s + setup_s["fp64"] + extra["fp64"]["ms_p50"] / 1e3, 4)}
    per16, res16 = timed_solves(pcs["bf16"], max(3, args.steps // 2), 1)
    extra["bf16"] = {"solves_per_s": 1e3 / statistics.mean(per16), "ms_p50": statistics.median(per16),
                     "iterations": res16[-1][0]["iterations"], "relres": res16[-1][0]["relres"],
                     "setup_s": setup_s["bf16"]}

    # ---- roofline of the dominant kernel: the batched restrict / LU solve / prolong ----
    info = pc.info()
    r = torch.randn(n, dtype=torch.float64, device=dev)
    z = torch.empty_like(r)

    def apply_time(p, nl=20):
        for _ in range(3):
            G.oras_apply(p, r, z, stream=stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(nl):
            G.oras_apply(p, r, z, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        G.oras_check_status(p)
        return e0.elapsed_time(e1) / nl

    apply_ms = apply_time(pc)
    # bytes one application must stream: the off-diagonal factor tiles inside the tile
    # envelope (storage precision), two inverted diagonal blocks per tile row (compute
    # precision), the restricted residual reads and the prolonged writes
    tiles_off, tiles_inv = info["solve_offdiag_tiles"] * 4096, 2 * info["tile_rows"] * 4096
    vec_bytes = 8 * info["sum_sigma"] + 8 * n
    alg_bytes = 4 * tiles_off + 4 * tiles_inv + vec_bytes
    peak, peak_kind = _peaks()
    ms16 = apply_time(pcs["bf16"])
    b16 = 2 * tiles_off + 4 * tiles_inv + vec_bytes
    extra["bf16"]["solve_kernel"] = {"launch_ms": round(ms16, 4), "achieved_gbs": round(b16 / ms16 / 1e6, 1),
                                     "frac": round(b16 / ms16 / 1e6 / peak, 4)}
    if "fp64" in pcs:
        ms64 = apply_time(pcs["fp64"], 5)
        b64 = 8 * tiles_off + 8 * tiles_inv + vec_bytes
        extra["fp64"]["solve_kernel"] = {
            "launch_ms": round(ms64, 4), "achieved_gbs": round(b64 / ms64 / 1e6, 1),
            "fp64_tflops": round(2 * (tiles_off + tiles_inv) / ms64 / 1e9, 3), "bound": "fp64 alu"}
    achieved = alg_bytes / (apply_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": _profiled_traffic(),
                "kernel": "trsv_kernel<float,float>", "launch_ms": round(apply_ms, 4),
                "algorithmic_bytes": alg_bytes, "peak_source": peak_kind}

    # ---- end to end through the C ABI with host buffers ----
    f_pin = torch.tensor(f_host, dtype=torch.float64).pin_memory()
    u_pin = torch.empty(n, dtype=torch.float64).pin_memory()
    fd = torch.empty_like(f)
    ud = torch.empty_like(f)
    ke = max(3, args.steps // 2)
    for _ in range(2):
        fd.copy_(f_pin, non_blocking=True)
        solve(pc, fd, ud)
        u_pin.copy_(ud, non_blocking=True)
    torch.cuda.synchronize()
    ee0 = torch.cuda.Event(enable_timing=True)
    ee1 = torch.cuda.Event(enable_timing=True)
    ee0.record(stream)
    for _ in range(ke):
        fd.copy_(f_pin, non_blocking=True)
        solve(pc, fd, ud)
        u_pin.copy_(ud, non_blocking=True)
    ee1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = ee0.elapsed_time(ee1) / ke
    e2e = {"value": round(world * 1e3 / e2e_ms, 3), "unit": "solves/s",
           "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n}

    # ---- several right-hand sides per streamed factor tile (after every single-rhs timing:
    # the first multi-rhs launch grows the solve's tagged-word buffers) ----
    r8 = torch.randn(8 * n, dtype=torch.float64, device="cuda")
    z8 = torch.empty_like(r8)
    for _ in range(3):
        G.oras_apply(pc, r8, z8, nrhs=8, stream=stream)
    m0 = torch.cuda.Event(enable_timing=True)
    m1 = torch.cuda.Event(enable_timing=True)
    m0.record(stream)
    for _ in range(10):
        G.oras_apply(pc, r8, z8, nrhs=8, stream=stream)
    m1.record(stream)
    torch.cuda.synchronize()
    G.oras_check_status(pc)
    ms8 = m0.elapsed_time(m1) / 10
    extra["multi_rhs_apply"] = {"nrhs": 8, "launch_ms": round(ms8, 4), "ms_per_rhs": round(ms8 / 8, 4),
                                "speedup_per_rhs_vs_single": round(8 * apply_ms / ms8, 2)}

    # ---- CPU baseline: the oracle, rank 0 at N = 1 only ----
    cpu_baseline = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_baseline = oracle_solve_rate(wl, sample_iterations=None)

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(total_ms / args.steps, 3),
        "ms_p50": round(statistics.median(per_step), 3),
        "ms_p99": round(float(np.percentile(per_step, 99)), 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 local factors and solves + f64 Krylov/operator",
        "data": "synthetic (seeded workloads module; unit sphere, f=(c+12)xyz at closest points)",
        "config": {"workload": wl.name, "surface": "unit sphere", "h": wl.h, "p": wl.p, "c": wl.c,
                   "N_A": n, "n_sub": wl.n_sub, "overlap": wl.n_overlap, "method": "ORAS",
                   "alpha": wl.alpha, "alpha_x": wl.alpha_x, "krylov": f"FGMRES({wl.restart})",
                   "tol": wl.tol, "factor_precision": "fp32",
                   "factor_bytes": info["factor_bytes"],
                   "l2": "inputs larger than L2: every iteration streams %.2f GB of factor tiles"
                         % ((alg_bytes - vec_bytes) / 1e9),
                   "parallelism": f"replicas x{world}"},
        "iterations": iters, "relres": relres,
        "setup_s": {"host_band_partition": round(host_setup_s, 3),
                    **{k: round(v, 3) for k, v in setup_s.items()},
                    "fp32_factor_ms": round(info["setup_ms_factor"], 2)},
        "solve_schedule": schedules,
        "roofline": roofline, "clocks": clocks, "e2e": e2e, "gpu_launches": launches,
        "cpu_baseline": cpu_baseline, **extra,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def oracle_solve_rate(wl, sample_iterations=None):
    """Time the CPU oracle (FP64, single-threaded SciPy SuperLU + sparse matvec)."""
    from oracle import problems
    t = time.time()
    P = problems.setup_workload(wl)
    setup = time.time() - t
    t = time.time()
    if sample_iterations is None:
        res = problems.solve(P, P.f, wl.tol, wl.restart, wl.max_it)
        dt = time.time() - t
        return {"value": round(1.0 / dt, 5), "unit": "solves/s", "cores": 1, "kind": "oracle",
                "sample": f"one full FGMRES({wl.restart}) solve to {wl.tol:g} of {wl.name} "
                          f"({res.iterations} iterations, oracle set-up of {setup:.1f} s excluded)",
                "iterations": res.iterations, "setup_s": round(setup, 2)}
    raise ValueError


def run_reference(args):
    """The reference arm: the CPU FP64 oracle, timed on the host cores."""
    from oracle import problems
    from workloads import WORKLOADS
    world, rank, local = _dist()
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    t = time.time()
    P = problems.setup_workload(wl)
    setup = time.time() - t
    full = problems.solve(P, P.f, wl.tol, wl.restart, wl.max_it)    # iteration count, untimed
    its = full.iterations
    sample = 10
    times = []
    for i in range(args.warmup + args.steps):
        t = time.time()
        problems.solve(P, P.f, wl.tol, wl.restart, wl.max_it, stop_after=sample)
        dt = time.time() - t
        if i >= args.warmup:
            times.append(dt * its / sample)       # scaled to one full solve
    ms = statistics.mean(times) * 1e3
    value = 1e3 / ms
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "solves/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl.name},
            "cpu_baseline": {"value": round(value, 5), "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": f"{sample} FGMRES iterations per step scaled to the "
                                       f"{its}-iteration solve; oracle set-up {setup:.1f} s excluded"},
            "e2e": {"value": round(value, 5), "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_serving(args):
    """Serving stream (no JSON bench line of the main metric): capacity of the seeded request
    mix served back to back, then the same mix with Poisson arrivals at a fraction of that
    capacity; p50/p99 latency (arrival to result), queue / service split; mixed (FP32
    factors) against FP64 factors."""
    import torch
    from paper_1909_08734_gb300.serving import Request, Server, summarize
    from workloads import (WORKLOADS, poisson_arrivals, serving_stream, smooth_rhs,
                           surface_mesh)
    V, T = surface_mesh(WORKLOADS["mesh_h001"])
    specs = serving_stream(args.serving_requests, seed=5)
    out = {"mode": "serving", "requests": len(specs), "stream_seed": 5,
           "mix": "surface in {sphere, torus(1,0.4), 81,920-triangle mesh}, h in {0.05, 0.025, "
                  "0.0125} w.p. {0.5, 0.35, 0.15}, c log-uniform [0.1, 100], 1-32 rhs, 25% "
                  "backward-Euler chains, 30% operator reuse"}

    def make_server(prec):
        srv = Server(precision=prec)
        srv.register_surface("sphere", "sphere", 1.0, 0.0)
        srv.register_surface("torus", "torus", 1.0, 0.4)
        srv.register_surface("mesh", "trimesh", verts=V, tris=T)
        return srv

    host = make_server("fp32")        # bands and right-hand sides, built once outside timing
    rhs = {}
    for sp in specs:
        cp = host.band(sp.surface, sp.h)[2]
        rhs[sp.rid] = smooth_rhs(cp, sp.rhs_seed, sp.nrhs)

    def requests(arrivals):
        return [Request(sp.rid, float(a), sp.surface, sp.h, sp.c, rhs[sp.rid], sp.chain_steps)
                for sp, a in zip(specs, arrivals)]

    for prec in args.serving_precisions.split(","):
        srv = make_server(prec)
        srv._bands = host._bands                  # share host-side bands and partitions
        cap = summarize(srv.serve(requests(np.zeros(len(specs))), realtime=False))
        srv.close()
        res = {"capacity": cap}
        for frac in [float(x) for x in args.serving_load.split(",")]:
            rate = frac * cap["requests_per_s"]
            srv = make_server(prec)
            srv._bands = host._bands
            st = summarize(srv.serve(requests(poisson_arrivals(len(specs), rate, seed=5))))
            st["offered_rate_per_s"] = rate
            st["counters"] = dict(srv.counters)
            srv.close()
            res[f"load_{frac:g}"] = st
        out[prec] = res
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)


# Sec. 6.5, subdomain-count table: iterations to a 10^6 residual reduction, unit sphere,
# p = 2, h = 1/100 (N_A = 654,630), N_O = 4, alpha = 4, alpha_x = 40
PAPER_SUBDOMAIN_TABLE = {32: (500, 245, 53, 33), 64: (704, 278, 57, 46), 96: (818, 405, 59, 49)}


def run_subdomain_table(args):
    """Iteration counts of RAS / ORAS as solver and preconditioner against the paper's table
    (no bench line).  Factors in FP32 (the iteration counts match FP64 factors to within
    one iteration on the bench workload)."""
    import torch
    import paper_1909_08734_gb300 as G
    h, p = 0.01, 2
    band = G.cpm_build_band("sphere", 1.0, 0.0, h, p)
    n = band.info()["n_active"]
    cp = band.info()["cp"][:n]
    f = torch.tensor((1.0 + 12.0) * cp[:, 0] * cp[:, 1] * cp[:, 2], dtype=torch.float64, device="cuda")
    out = {"mode": "subdomain_table", "surface": "unit sphere", "h": h, "p": p, "N_A": n, "overlap": 4,
           "tol": 1e-6, "factors": args.precision, "rows": []}
    for ns in [int(x) for x in args.table_subdomains.split(",")]:
        part = G.cpm_partition(band, ns, None, 4, align_passes=args.table_align)
        row = {"n_sub": ns, "align_passes": args.table_align, "paper_ras_solver_ras_prec_oras_solver_oras_prec":
               [PAPER_SUBDOMAIN_TABLE.get(ns, (None,) * 4)[i] for i in (0, 2, 1, 3)]}
        for method in ("ras", "oras"):
            t0 = time.time()
            pc = G.oras_setup(band, part, 1.0, method, 4.0, 40.0, args.precision)
            setup_s = time.time() - t0
            u = torch.zeros_like(f)
            st = G.oras_stationary_solve(pc, f, u, tol=1e-6, max_it=3000, raise_on_failure=False)[0]
            gm = G.cpm_gmres_solve(pc, f, u, tol=1e-6, max_it=2000, raise_on_failure=False)[0]
            row[method] = {"solver": st["iterations"], "solver_status": st["status"],
                           "preconditioner": gm["iterations"], "setup_s": round(setup_s, 2),
                           "factor_gb": round(pc.info()["factor_bytes"] / 1e9, 2)}
            del pc
            torch.cuda.empty_cache()
        out["rows"].append(row)
        print(json.dumps(row), flush=True)
    print(json.dumps(out), flush=True)


def run_peaks(args):
    """FP64 FMA peak and dependent-FMA latency of this GPU (the FP64-ALU roofline denominator):
    a sweep of block counts, block sizes and independent chains per thread."""
    import torch
    import paper_1909_08734_gb300 as G
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    rows = []
    for threads in (128, 256, 512, 1024):
        for per_sm in (1, 2, 4, 8):
            if threads * per_sm > 2048:
                continue
            for chains in (1, 2, 4, 8):
                tf, _ = G.cpm_probe_fp64(sms * per_sm, threads, chains, 4096, latency=False)
                rows.append({"threads": threads, "blocks_per_sm": per_sm, "chains": chains,
                             "tflop_s": round(tf, 4)})
    _, lat = G.cpm_probe_fp64(1, 1, 1, 1 << 16, latency=True)
    best = max(rows, key=lambda r: r["tflop_s"])
    print(json.dumps({"fp64_fma_peak_tflop_s": best["tflop_s"], "best": best,
                      "dependent_fma_cycles": round(lat, 2), "sms": sms, "sweep": rows}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="sphere_h0025")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--kernel-only", type=int, default=0,
                    help="profiling aid: only N launches of the batched solve, no JSON bench line")
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "bf16"])
    ap.add_argument("--serving", action="store_true",
                    help="serve the seeded request stream instead of the bench line")
    ap.add_argument("--serving-requests", type=int, default=40)
    ap.add_argument("--serving-load", default="0.7", help="offered load(s), fractions of capacity")
    ap.add_argument("--serving-precisions", default="fp32,fp64")
    ap.add_argument("--peaks", action="store_true",
                    help="FP64 FMA peak / latency probe sweep (the FP64 roofline denominator)")
    ap.add_argument("--subdomain-table", action="store_true",
                    help="iteration counts against the paper's subdomain-count table")
    ap.add_argument("--table-subdomains", default="32,64,96")
    ap.add_argument("--table-align", type=int, default=3,
                    help="interface alignment passes (the paper uses p + 1 = 3)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "native":
        args.warmup = 3
    if args.peaks:
        run_peaks(args)
    elif args.kernel_only:
        run_kernel_only(args)
    elif args.serving:
        run_serving(args)
    elif args.subdomain_table:
        run_subdomain_table(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
