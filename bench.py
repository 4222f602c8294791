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
# ncu summaries of the solve kernel's DRAM traffic at full size, per (workload, factor precision)
PROFILE_SUMMARIES = {("sphere_h0025", "fp32"): os.path.join(ROOT, "profiles", "trsv_fp32_sphere_h0025.md"),
                     ("torus_h00125", "bf16"): os.path.join(ROOT, "profiles", "trsv_bf16_torus_h00125.md")}


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


def _profiled_traffic(workload, precision):
    """DRAM bytes per launch from the committed ncu summary of this workload and precision, if
    there is one and it still matches the kernel source."""
    src = os.path.join(ROOT, "paper_1909_08734_gb300", "csrc", "cuda", "trsv.cu")
    summary = PROFILE_SUMMARIES.get((workload, precision))
    if summary is None or not os.path.exists(summary):
        return None
    fields = {}
    for line in open(summary):
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


# ---- the oracle with its local solves on all host cores (cpu_baseline and reference arm) ----
def _oracle_worker(conn, r_name, z_name, n, lps):
    """One process of the pool: factors its share of the oracle's local matrices with the
    oracle's own SciPy SuperLU, then answers apply requests (r and z in shared memory; each
    worker writes only the disjoint sets of its subdomains)."""
    from multiprocessing import shared_memory
    import scipy.sparse.linalg as spla
    rs = shared_memory.SharedMemory(name=r_name)
    zs = shared_memory.SharedMemory(name=z_name)
    r = np.ndarray((n,), dtype=np.float64, buffer=rs.buf)
    z = np.ndarray((n,), dtype=np.float64, buffer=zs.buf)
    facs = [spla.splu(lp.A.tocsc()) for lp in lps]
    conn.send("ready")
    while conn.recv() is not None:
        for lp, fac in zip(lps, facs):
            e = fac.solve(lp.rhs(r))
            z[lp.own_global] = e[lp.own_local]
        conn.send(1)
    del r, z
    rs.close()
    zs.close()


class OraclePool:
    """The oracle's Schwarz preconditioner (oracle.schwarz.Schwarz.apply) with its local
    solves spread over `workers` spawned processes; the Krylov iteration stays the oracle's."""

    def __init__(self, prob, workers: int):
        import multiprocessing as mp
        from multiprocessing import shared_memory
        n = prob.band.n_active
        self.n = n
        self.rs = shared_memory.SharedMemory(create=True, size=8 * n)
        self.zs = shared_memory.SharedMemory(create=True, size=8 * n)
        self.r = np.ndarray((n,), dtype=np.float64, buffer=self.rs.buf)
        self.z = np.ndarray((n,), dtype=np.float64, buffer=self.zs.buf)
        # largest subdomains first, each to the least loaded worker (cost ~ n_j^1.5)
        loads, shares = [0.0] * workers, [[] for _ in range(workers)]
        for j in sorted(range(len(prob.lps)), key=lambda j: -prob.lps[j].n):
            w = int(np.argmin(loads))
            shares[w].append(prob.lps[j])
            loads[w] += prob.lps[j].n ** 1.5
        ctx = mp.get_context("spawn")
        self.conns, self.procs = [], []
        for share in shares:
            a, b = ctx.Pipe()
            pr = ctx.Process(target=_oracle_worker, args=(b, self.rs.name, self.zs.name, n, share), daemon=True)
            pr.start()
            self.conns.append(a)
            self.procs.append(pr)
        for c in self.conns:
            c.recv()

    def apply(self, r):
        self.r[:] = r
        for c in self.conns:
            c.send(1)
        for c in self.conns:
            c.recv()
        return self.z.copy()

    def close(self):
        for c in self.conns:
            c.send(None)
        for pr in self.procs:
            pr.join(timeout=10)
        del self.r, self.z
        self.rs.close()
        self.rs.unlink()
        self.zs.close()
        self.zs.unlink()


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_baseline(wl, full_solves: int = 1, one_core: bool = True):
    """The CPU FP64 oracle on this host: full FGMRES solves with the local solves on all cores
    (spawned process pool), and one full single-process solve.  Returns (summary, x)."""
    from oracle import krylov, problems
    t = time.time()
    P = problems.setup_workload(wl)
    setup = time.time() - t
    cores = _host_cores()
    out = {"kind": "oracle", "unit": "solves/s", "oracle_setup_s": round(setup, 2)}
    x = None
    if one_core:
        t = time.time()
        res = problems.solve(P, P.f, wl.tol, wl.restart, wl.max_it)
        dt = time.time() - t
        x = res.x
        out["one_core"] = {"value": round(1.0 / dt, 5), "cores": 1, "iterations": res.iterations,
                           "sample": f"one full FGMRES({wl.restart}) solve to {wl.tol:g}"}
    pool = OraclePool(P, cores)
    try:
        times = []
        for _ in range(full_solves):
            t = time.time()
            res = krylov.fgmres(lambda v: P.A @ v, pool.apply, P.f, wl.tol, wl.restart, wl.max_it)
            times.append(time.time() - t)
        x = res.x if x is None else x
    finally:
        pool.close()
    out.update({"value": round(1.0 / statistics.mean(times), 5), "cores": cores, "iterations": res.iterations,
                "sample": f"{full_solves} full FGMRES({wl.restart}) solve(s) to {wl.tol:g} of {wl.name}, "
                          f"local SuperLU solves on {cores} processes (spawn), Krylov and operator in the "
                          f"parent; oracle set-up of {setup:.1f} s excluded",
                "times_s": [round(v, 3) for v in times]})
    return out, x, P


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


SURFACE_LABEL = {"sphere": "unit sphere", "torus": "torus", "trimesh": "perturbed icosphere (triangles)"}
RHS_LABEL = {"xyz": "f=(c+12)xyz at closest points", "torus_modes": "16 seeded trig modes in the torus angles",
             "ambient_modes": "8 seeded ambient cosine modes"}
DTYPE = {"fp32": "f32 local factors and solves + f64 Krylov/operator",
         "bf16": "bf16 local factors (f32 solves) + f64 Krylov/operator",
         "fp64": "f64 local factors, solves, Krylov and operator"}


def _build_band(G, wl, on_device=False):
    from workloads import surface_mesh
    mesh = surface_mesh(wl)
    if mesh is None:
        return G.cpm_build_band(wl.surface, wl.R, wl.r, wl.h, wl.p, on_device=on_device)
    return G.cpm_build_band(wl.surface, wl.R, wl.r, wl.h, wl.p, verts=mesh[0], tris=mesh[1], on_device=on_device)


def _workload_config(wl, info, n, world, alg_bytes, vec_bytes):
    cfg = {"workload": wl.name, "surface": SURFACE_LABEL.get(wl.surface, wl.surface), "h": wl.h, "p": wl.p,
           "c": wl.c, "N_A": n, "n_sub": wl.n_sub, "overlap": wl.n_overlap, "method": wl.method.upper(),
           "krylov": f"FGMRES({wl.restart})", "tol": wl.tol, "factor_precision": wl.precision,
           "factor_bytes": info["factor_bytes"],
           "l2": "inputs larger than L2: every iteration streams %.2f GB of factor tiles"
                 % ((alg_bytes - vec_bytes) / 1e9),
           "parallelism": f"replicas x{world}"}
    if wl.method == "oras":
        cfg.update({"alpha": wl.alpha, "alpha_x": wl.alpha_x})
    if wl.surface == "torus":
        cfg.update({"R": wl.R, "r": wl.r})
    if wl.surface == "trimesh":
        cfg.update({"triangles": 20 * 4 ** wl.mesh_level, "radial_noise": wl.mesh_amp})
    if wl.weight_seed is not None:
        cfg["leaf_weights"] = f"seeded uniform [256, 1024] (seed {wl.weight_seed})"
    return cfg


def run_native(args):
    import torch
    import paper_1909_08734_gb300 as G
    from workloads import WORKLOADS, leaf_weights, rhs

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    wl = WORKLOADS[args.workload]
    dev = torch.device("cuda", local)
    head = wl.precision                         # the workload's factor precision is the headline
    precs = [head] + [p for p in ("fp32", "bf16", "fp64") if p != head and not (args.no_fp64 and p == "fp64")]

    _build_band(G, wl, on_device=True)          # first device build: module and context warm-up
    torch.cuda.synchronize()
    t0 = time.time()
    band = _build_band(G, wl, on_device=True)  # band on the device (bit-exact with the host build)
    torch.cuda.synchronize()
    t1 = time.time()
    part = G.cpm_partition(band, wl.n_sub, leaf_weights(wl.n_sub, wl.weight_seed), wl.n_overlap)
    t2 = time.time()
    band_s, partition_s = t1 - t0, t2 - t1
    band_partition_s = band_s + partition_s
    cp = band.info()["cp"]
    pcs, setup_s, schedules = {}, {}, {}
    for prec in precs:
        torch.cuda.synchronize()
        t = time.time()
        pcs[prec] = G.oras_setup(band, part, wl.c, wl.method, wl.alpha, wl.alpha_x, prec)
        torch.cuda.synchronize()
        setup_s[prec] = time.time() - t
        t = time.time()
        schedules[prec] = G.oras_autotune(pcs[prec])
        setup_s[prec + "_autotune"] = time.time() - t
    pc = pcs[head]
    n = pc.n_active
    f_host = rhs(wl, cp[:n])
    f = torch.tensor(f_host, dtype=torch.float64, device=dev)
    u = torch.zeros_like(f)
    stream = torch.cuda.current_stream(dev)

    def solve(p, ff, uu, nrhs=1):
        return G.cpm_gmres_solve(p, ff, uu, nrhs=nrhs, restart=wl.restart, tol=wl.tol, max_it=wl.max_it,
                                 stream=stream)

    def timed_solves(p, k, w, ff=f, uu=u, nrhs=1):
        for _ in range(w):
            solve(p, ff, uu, nrhs)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(k + 1)]
        res = []
        ev[0].record(stream)
        for i in range(k):
            res.append(solve(p, ff, uu, nrhs))
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
        return [ev[i].elapsed_time(ev[i + 1]) for i in range(k)], res

    # ---- headline: the workload's factor precision, factors resident ----
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
    u_head = u.clone()
    head_ms = statistics.median(per_step)

    # ---- the other factor precisions on the same operators ----
    extra, sols = {}, {head: u_head}
    for prec in precs[1:]:
        uu = torch.zeros_like(f)
        per, res = timed_solves(pcs[prec], max(3, args.steps // 2), 1, f, uu)
        sols[prec] = uu.clone()
        extra[prec] = {"solves_per_s": 1e3 / statistics.mean(per), "ms_p50": statistics.median(per),
                       "iterations": res[-1][0]["iterations"], "relres": res[-1][0]["relres"],
                       "setup_s": setup_s[prec], "setup_ms_factor": pcs[prec].info()["setup_ms_factor"]}
    if "fp64" in pcs and head != "fp64":
        u64 = sols["fp64"]
        extra["mixed_vs_fp64_solution_rel_diff"] = (torch.linalg.norm(u_head - u64) / torch.linalg.norm(u64)).item()
        extra["mixed_speedup_vs_fp64_solve"] = extra["fp64"]["ms_p50"] / head_ms
        extra["mixed_speedup_vs_fp64_setup_plus_solve"] = (
            (setup_s["fp64"] + extra["fp64"]["ms_p50"] / 1e3) / (setup_s[head] + head_ms / 1e3))
        # the metric reported twice: solve with factors resident (value) and set-up + solve
        extra["setup_plus_solve_s"] = {
            head: round(band_partition_s + setup_s[head] + head_ms / 1e3, 4),
            "fp64": round(band_partition_s + setup_s["fp64"] + extra["fp64"]["ms_p50"] / 1e3, 4)}


    # ---- rooflines: the batched solve (dominant), the operator apply, the Arnoldi kernels ----
    info = pc.info()
    r = torch.randn(n, dtype=torch.float64, device=dev)
    z = torch.empty_like(r)

    def event_ms(fn, nl):
        for _ in range(3):
            fn()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(nl):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / nl

    def apply_time(p, nl=20):
        ms = event_ms(lambda: G.oras_apply(p, r, z, stream=stream), nl)
        G.oras_check_status(p)
        return ms

    fp64_peak, fp64_dep_cycles = G.cpm_probe_fp64(2 * torch.cuda.get_device_properties(dev).multi_processor_count,
                                                  1024, 8, 4096, latency=True)
    peak, peak_kind = _peaks()
    # bytes one application must stream: the off-diagonal factor tiles inside the tile
    # envelope (storage precision), the two inverted diagonal blocks of every tile row, each
    # stored as its triangle of 64 * 65 / 2 entries (compute precision), the restricted residual
    # reads and the prolonged writes
    tiles_off, tiles_inv = info["solve_offdiag_tiles"] * 4096, 2 * info["tile_rows"] * 2080
    vec_bytes = 8 * info["sum_sigma"] + 8 * n
    store = {"fp32": 4, "bf16": 2, "fp64": 8}
    comp = {"fp32": 4, "bf16": 4, "fp64": 8}
    solve_ms = {}
    for prec in precs:
        ms = apply_time(pcs[prec], 20 if prec != "fp64" else 5)
        solve_ms[prec] = ms
        b = store[prec] * tiles_off + comp[prec] * tiles_inv + vec_bytes
        k = {"launch_ms": round(ms, 4), "achieved_gbs": round(b / ms / 1e6, 1), "frac_hbm": round(b / ms / 1e6 / peak, 4),
             "algorithmic_bytes": b}
        if prec == "fp64":
            k.update({"fp64_tflops": round(2 * (tiles_off + tiles_inv) / ms / 1e9, 3), "bound": "fp64 alu",
                      "frac_fp64": round(2 * (tiles_off + tiles_inv) / ms / 1e9 / fp64_peak, 4)})
        if prec == head:
            head_bytes = b
        else:
            extra[prec]["solve_kernel"] = k
    apply_ms = solve_ms[head]
    if head == "fp64":
        fl = 2 * (tiles_off + tiles_inv)
        achieved = fl / (apply_ms / 1e3) / 1e12
        roofline = {"bound": "alu", "achieved": round(achieved, 4), "peak": round(fp64_peak, 4), "unit": "TFLOP/s",
                    "frac": round(achieved / fp64_peak, 4), "traffic": None, "kernel": "trsv_kernel<double,double>",
                    "launch_ms": round(apply_ms, 4), "algorithmic_flops": fl,
                    "peak_source": "measured FP64 FMA probe (cpm_probe_fp64), this run"}
    else:
        achieved = head_bytes / (apply_ms / 1e3) / 1e9
        roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(achieved / peak, 4),
                    "traffic": _profiled_traffic(wl.name, head),
                    "kernel": "trsv_kernel<%s>" % ("float,float" if head == "fp32" else "bf16,float"),
                    "launch_ms": round(apply_ms, 4), "algorithmic_bytes": head_bytes, "peak_source": peak_kind}
    # operator apply y = A x (FP64, matrix-free): extension values at every band node, then the
    # 7-point sums; algorithmic work per the scope table: 2 (p+1)^3 (N_A + N_G) + 8 N_A flops and
    # 8 N_A (x) + 8 N_A (y) + 24 (N_A + N_G) + 4 (p+1)^2 (N_A + N_G) + 24 N_A bytes
    NN = info["n_nodes"]
    P3, P2 = (wl.p + 1) ** 3, (wl.p + 1) ** 2
    y = torch.empty_like(r)
    op_ms = event_ms(lambda: G.cpm_op_apply(pc, r, y, stream=stream), 20)
    op_flops = 2 * P3 * NN + 8 * n
    op_bytes = 8 * n + 8 * n + 24 * NN + 4 * P2 * NN + 24 * n
    impl_fma = (P3 + wl.p + 1) * NN + 8 * n            # FP64 operations the kernels issue
    iter_ms = head_ms / max(1, iters)
    arn_ms = iter_ms - apply_ms - op_ms
    kbar = (iters - 1) / 2.0 if iters < wl.restart else (wl.restart - 1) / 2.0
    arn_flops = 8 * (kbar + 1) * n + 10 * n                # CGS2 at the mean step + w and the norm
    extra["operator_apply"] = {
        "launch_ms": round(op_ms, 4), "bound": "alu",
        "fp64_tflops_algorithmic": round(op_flops / op_ms / 1e9, 4),
        "fp64_tflops_issued": round(2 * impl_fma / op_ms / 1e9, 4),
        "frac_fp64_issued": round(2 * impl_fma / op_ms / 1e9 / fp64_peak, 4),
        "achieved_gbs_algorithmic": round(op_bytes / op_ms / 1e6, 1),
        "frac_hbm_algorithmic": round(op_bytes / op_ms / 1e6 / peak, 4)}
    extra["iteration_breakdown_ms"] = {
        "iteration": round(iter_ms, 4), "solve_kernel": round(apply_ms, 4), "operator_apply": round(op_ms, 4),
        "arnoldi_cgs2_givens_and_per_solve": round(arn_ms, 4),
        "arnoldi_fp64_tflops": round(arn_flops / (arn_ms / 1e3) / 1e12, 4) if arn_ms > 0 else None,
        "arnoldi_frac_fp64": round(arn_flops / (arn_ms / 1e3) / 1e12 / fp64_peak, 4) if arn_ms > 0 else None}
    extra["fp64_peak"] = {"fma_tflop_s": round(fp64_peak, 4), "dependent_fma_cycles": round(fp64_dep_cycles, 1),
                          "source": "cpm_probe_fp64 in this run (bench.py --peaks sweeps it)"}

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

    # ---- several right-hand sides: one solve launch for 8 per iteration, and FGMRES over 8
    # right-hand sides in lock step (after every single-rhs timing: the first multi-rhs launch
    # grows the solve's tagged-word buffers) ----
    r8 = torch.randn(8 * n, dtype=torch.float64, device=dev)
    z8 = torch.empty_like(r8)
    ms8 = event_ms(lambda: G.oras_apply(pc, r8, z8, nrhs=8, stream=stream), 10)
    G.oras_check_status(pc)
    extra["multi_rhs_apply"] = {"nrhs": 8, "launch_ms": round(ms8, 4), "ms_per_rhs": round(ms8 / 8, 4),
                                "speedup_per_rhs_vs_single": round(8 * apply_ms / ms8, 2)}
    from workloads import smooth_rhs
    F8 = torch.tensor(smooth_rhs(cp[:n], 77, 8).T.copy(), dtype=torch.float64, device=dev).reshape(-1)
    U8 = torch.zeros_like(F8)
    lock = {}
    for prec in [head] + (["fp64"] if "fp64" in pcs and head != "fp64" else []):
        per8, res8 = timed_solves(pcs[prec], 3, 1, F8, U8, nrhs=8)
        lock[prec] = {"ms_per_batch_p50": round(statistics.median(per8), 3),
                      "solves_per_s": round(8e3 / statistics.median(per8), 3),
                      "iterations": [q["iterations"] for q in res8[-1]],
                      "max_relres": max(q["relres"] for q in res8[-1])}
    if len(lock) == 2:
        lock["mixed_speedup_vs_fp64"] = round(lock[head]["solves_per_s"] / lock["fp64"]["solves_per_s"], 3)
    extra["lock_step_8_rhs"] = lock

    # ---- CPU baseline: the oracle, rank 0 at N = 1 only; and the solution errors against it ----
    cpu_baseline = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_baseline, x_or, _ = oracle_baseline(wl, full_solves=1, one_core=True)
        xo = torch.tensor(x_or, dtype=torch.float64, device=dev)
        extra["solution_rel_err_vs_oracle"] = {
            prec: (torch.linalg.norm(sols[prec] - xo) / torch.linalg.norm(xo)).item() for prec in sols}
        extra["solution_rel_err_vs_oracle"]["note"] = f"both sides solved to {wl.tol:g} relative residual"

    info = pc.info()
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(total_ms / args.steps, 3),
        "ms_p50": round(head_ms, 3),
        "ms_p99": round(float(np.percentile(per_step, 99)), 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[head],
        "data": "synthetic (seeded workloads module; %s, %s)" % (SURFACE_LABEL.get(wl.surface, wl.surface),
                                                              RHS_LABEL.get(wl.rhs, wl.rhs)),
        "config": _workload_config(wl, info, n, world, head_bytes, vec_bytes),
        "iterations": iters, "relres": relres,
        "setup_s": {"band_device": round(band_s, 4), "partition_host": round(partition_s, 3),
                    **{k: round(v, 3) for k, v in setup_s.items()},
                    head + "_factor_ms": round(info["setup_ms_factor"], 2)},
        "solve_schedule": schedules,
        "roofline": roofline, "clocks": clocks, "e2e": e2e, "gpu_launches": launches,
        "cpu_baseline": cpu_baseline, **extra,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()

def run_reference(args):
    """The reference arm: the CPU FP64 oracle on the host cores.  Each step is one full FGMRES
    solve of the workload with the oracle's local solves spread over all cores (spawned
    process pool); one single-process solve is timed once beside it."""
    from oracle import krylov, problems
    from workloads import WORKLOADS
    world, rank, local = _dist()
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    t = time.time()
    P = problems.setup_workload(wl)
    setup = time.time() - t
    t = time.time()
    one = problems.solve(P, P.f, wl.tol, wl.restart, wl.max_it)
    one_s = time.time() - t
    cores = _host_cores()
    pool = OraclePool(P, cores)
    times = []
    try:
        for i in range(args.warmup + args.steps):
            t = time.time()
            res = krylov.fgmres(lambda v: P.A @ v, pool.apply, P.f, wl.tol, wl.restart, wl.max_it)
            dt = time.time() - t
            if i >= args.warmup:
                times.append(dt)
    finally:
        pool.close()
    ms = statistics.mean(times) * 1e3
    value = 1e3 / ms
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "solves/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 1),
            "ms_p50": round(statistics.median(times) * 1e3, 1),
            "ms_p99": round(float(np.percentile(times, 99)) * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl.name},
            "iterations": res.iterations, "relres": res.relres,
            "cpu_baseline": {"value": round(value, 5), "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": f"one full FGMRES({wl.restart}) solve to {wl.tol:g} per step, local "
                                       f"SuperLU solves on {cores} spawned processes; oracle set-up "
                                       f"{setup:.1f} s excluded",
                             "one_core": {"value": round(1.0 / one_s, 5), "cores": 1,
                                          "sample": "one full single-process solve"}},
            "e2e": {"value": round(value, 5), "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_serving(args):
    """Serving stream (no JSON bench line of the main metric): capacity of the seeded request
    mix served back to back, then the same mix with Poisson arrivals at a fraction of that
    capacity; p50/p99 latency (arrival to result), queue / service split; mixed (FP32
    factors) against FP64 factors."""
    import torch
    from paper_1909_08734_gb300.serving import Request, Server, overlap_seconds, summarize
    from workloads import (WORKLOADS, poisson_arrivals, serving_stream, smooth_rhs,
                           surface_mesh)
    V, T = surface_mesh(WORKLOADS["mesh_h001"])
    specs = serving_stream(args.serving_requests, seed=5)
    out = {"mode": "serving", "requests": len(specs), "stream_seed": 5,
           "mix": "surface in {sphere, torus(1,0.4), 81,920-triangle mesh}, h in {0.05, 0.025, "
                  "0.0125} w.p. {0.5, 0.35, 0.15}, c log-uniform [0.1, 100], 1-32 rhs, 25% "
                  "backward-Euler chains, 30% operator reuse"}

    trace = open(args.serving_trace, "a") if args.serving_trace else None

    def make_server(prec, slots=1):
        srv = Server(precision=prec, slots=slots, trace=trace)
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
        res = {}
        for slots in [int(x) for x in args.serving_slots.split(",")]:
            srv = make_server(prec, slots)
            srv._bands = host._bands                  # share host-side bands and partitions
            cap = summarize(srv.serve(requests(np.zeros(len(specs))), realtime=False))
            cap["device_overlap_s"] = round(overlap_seconds(srv.batches), 3)
            srv.close()
            row = {"capacity": cap}
            for frac in [float(x) for x in args.serving_load.split(",")]:
                rate = frac * cap["requests_per_s"]
                srv = make_server(prec, slots)
                srv._bands = host._bands
                st = summarize(srv.serve(requests(poisson_arrivals(len(specs), rate, seed=5))))
                st["offered_rate_per_s"] = rate
                st["device_overlap_s"] = round(overlap_seconds(srv.batches), 3)
                st["counters"] = dict(srv.counters)
                srv.close()
                row[f"load_{frac:g}"] = st
            res[f"slots_{slots}"] = row
            torch.cuda.empty_cache()
        out[prec] = res
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
        part = G.cpm_partition(band, ns, None, 4, align_passes=args.table_align, split=args.table_split)
        row = {"n_sub": ns, "align_passes": args.table_align, "split": args.table_split, "paper_ras_solver_ras_prec_oras_solver_oras_prec":
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
    ap.add_argument("--serving-trace", default="", help="file for the serving loop's per-batch trace")
    ap.add_argument("--serving-slots", default="1",
                    help="concurrent batches (own stream and host thread each); one run per value")
    ap.add_argument("--peaks", action="store_true",
                    help="FP64 FMA peak / latency probe sweep (the FP64 roofline denominator)")
    ap.add_argument("--subdomain-table", action="store_true",
                    help="iteration counts against the paper's subdomain-count table")
    ap.add_argument("--table-subdomains", default="32,64,96")
    ap.add_argument("--table-split", default="coordinate", choices=["coordinate", "graph"],
                    help="disjoint split of the subdomain table: coordinate or graph bisection")
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
