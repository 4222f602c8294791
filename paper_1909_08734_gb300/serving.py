"""Serving loop: a stream of CPM solve requests on one GPU.  No counterpart in the paper.

A request names an operator -- a registered surface, a grid spacing h and the shift c of
(c - Lap_S) u = f -- and carries right-hand sides evaluated at the band's closest points,
optionally as a backward-Euler chain (c = 1/dt, f_{n+1} = u_n / dt) that reuses one
factorisation.  The server

* keeps bands and partitions on the host (per surface and h) and factorised operators
  resident in HBM (per surface, h, c), least recently used first out;
* admits work by an HBM budget: the library's device plan of an operator (oras_plan: setup
  peak, resident factors + FGMRES workspace) plus the batch's vectors must fit after
  evicting idle operators; a request that cannot fit even alone fails with CPM_ERR_BUDGET;
* batches at dispatch: the oldest queued request picks the operator, and every queued
  plain request for the same operator joins the batch; its right-hand sides go through
  one multi-rhs cpm_gmres_solve.  Requests arriving meanwhile join the next dispatch;
* records per request: arrival, start of its batch, completion, status, iterations and the
  true relative residual of every right-hand side.

Every step on the GPU runs in the library through the C ABI; this module only schedules and
moves vectors.  Results are deterministic: a request gets bit-identical solutions whether it
is served alone or inside a mix, because each right-hand side is solved independently with
the operator's fixed solve schedule (the default schedule unless one is pinned per surface
and h with `pin_schedule`).
"""
from __future__ import annotations

import collections
import dataclasses
import math
import time

import numpy as np

from . import (CpmError, _capi, cpm_build_band, cpm_gmres_solve, cpm_partition, cpm_vec_axpby,
               oras_plan, oras_setup, oras_tune)


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float                  # seconds after the start of the stream
    surface: str
    h: float
    c: float
    f: np.ndarray                   # (nrhs, N_A) FP64 host right-hand sides, band order
    chain_steps: int = 0            # backward-Euler steps after the first solve
    # filled by the server
    status: int = -1
    iterations: list = dataclasses.field(default_factory=list)
    relres: list = dataclasses.field(default_factory=list)
    u: np.ndarray | None = None     # final solutions (nrhs, N_A) if the server keeps them
    t_start: float = math.nan
    t_done: float = math.nan
    factorised: bool = False        # this request's batch set up the operator
    batch_rhs: int = 0              # right-hand sides solved in its batch

    @property
    def nrhs(self) -> int:
        return int(self.f.shape[0])

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival

    @property
    def queue_time(self) -> float:
        return self.t_start - self.arrival


class _Operator:
    def __init__(self, pc, resident: int):
        self.pc = pc
        self.resident = resident


class Server:
    def __init__(self, budget_bytes: int | None = None, precision: str = "fp32", restart: int = 50,
                 tol: float = 1e-8, max_it: int = 1000, method: str = "oras", alpha: float = 4.0,
                 alpha_x: float = 40.0, n_overlap: int = 2, p: int = 3, nodes_per_sub: int = 4000,
                 keep_solutions: bool = False):
        import torch
        self.torch = torch
        if budget_bytes is None:
            free, _ = torch.cuda.mem_get_info()
            budget_bytes = int(0.8 * free)
        self.budget = int(budget_bytes)
        self.precision = precision
        self.restart = restart
        self.tol = tol
        self.max_it = max_it
        self.method = method
        self.alpha = alpha
        self.alpha_x = alpha_x
        self.n_overlap = n_overlap
        self.p = p
        self.nodes_per_sub = nodes_per_sub
        self.keep_solutions = keep_solutions
        self._surfaces = {}
        self._bands = {}
        self._ops: collections.OrderedDict = collections.OrderedDict()
        self._schedules = {}
        self.used = 0
        self.counters = collections.Counter()

    # ---------------------------------------------------------------- registry
    def register_surface(self, name: str, kind: str, R: float = 1.0, r: float = 0.0, verts=None,
                         tris=None):
        self._surfaces[name] = (kind, R, r, verts, tris)

    def band(self, surface: str, h: float):
        """(Band, Partition, closest points of the actives) of a surface at spacing h."""
        key = (surface, float(h))
        if key not in self._bands:
            kind, R, r, V, T = self._surfaces[surface]
            band = cpm_build_band(kind, R, r, h, self.p, verts=V, tris=T)
            inf = band.info()
            n = inf["n_active"]
            n_sub = 2 ** int(round(math.log2(max(1.0, n / self.nodes_per_sub))))
            n_sub = int(min(512, max(2, n_sub)))
            part = cpm_partition(band, n_sub, None, self.n_overlap)
            self._bands[key] = (band, part, inf["cp"][:n].copy())
        return self._bands[key]

    def pin_schedule(self, surface: str, h: float, **knobs):
        """Solve schedule (oras_tune knobs) for every operator of this surface and h."""
        self._schedules[(surface, float(h))] = dict(knobs)

    # ---------------------------------------------------------------- admission
    def _evict_one(self):
        key, op = self._ops.popitem(last=False)
        self.used -= op.resident
        del op.pc
        self.counters["evictions"] += 1

    def _acquire(self, surface: str, h: float, c: float, vec_bytes: int):
        """Resident operator for (surface, h, c); sets it up under the budget if needed."""
        key = (surface, float(h), float(c))
        if key in self._ops:
            self._ops.move_to_end(key)
            self.counters["operator_hits"] += 1
            return self._ops[key].pc, False
        band, part, _ = self.band(surface, h)
        plan = oras_plan(band, part, self.method, self.precision, self.restart, 1)
        need = max(plan["setup_peak_bytes"], plan["resident_bytes"]) + vec_bytes
        if need > self.budget:
            raise CpmError(_capi.CPM_ERR_BUDGET, f"operator {key} needs {need} bytes, budget {self.budget}")
        while self._ops and self.used + need > self.budget:
            self._evict_one()
        if self.used + need > self.budget:
            raise CpmError(_capi.CPM_ERR_BUDGET, f"operator {key} does not fit beside pinned work")
        pc = oras_setup(band, part, c, self.method, self.alpha, self.alpha_x, self.precision)
        for knob, value in self._schedules.get((surface, float(h)), {}).items():
            oras_tune(pc, **{knob: value})
        self._ops[key] = _Operator(pc, plan["resident_bytes"])
        self.used += plan["resident_bytes"]
        self.counters["setups"] += 1
        return pc, True

    # ---------------------------------------------------------------- execution
    def _solve(self, pc, F_dev, U_dev, nrhs):
        res = cpm_gmres_solve(pc, F_dev, U_dev, nrhs=nrhs, restart=self.restart, tol=self.tol,
                              max_it=self.max_it, raise_on_failure=False)
        return res

    def _run_batch(self, batch):
        torch = self.torch
        head = batch[0]
        n = len(self.band(head.surface, head.h)[2])
        nrhs = sum(r.nrhs for r in batch)
        vec_bytes = 2 * 8 * nrhs * n
        try:
            pc, fresh = self._acquire(head.surface, head.h, head.c, vec_bytes)
        except CpmError as e:
            for r in batch:
                r.status = e.status
            self.counters["rejected"] += len(batch)
            return
        for r in batch:
            r.factorised = fresh
            r.batch_rhs = nrhs
        F = np.concatenate([r.f for r in batch], axis=0)
        F_dev = torch.from_numpy(np.ascontiguousarray(F)).pin_memory().to("cuda", non_blocking=True)
        U_dev = torch.empty_like(F_dev)
        chains = [r for r in batch if r.chain_steps > 0]
        res = self._solve(pc, F_dev.view(-1), U_dev.view(-1), nrhs)
        # backward-Euler steps: f_{k+1} = u_k / dt = c u_k, same operator
        row = 0
        rows = {}
        for r in batch:
            rows[r.rid] = (row, row + r.nrhs)
            row += r.nrhs
        for r in chains:
            a, b = rows[r.rid]
            r.iterations = [x["iterations"] for x in res[a:b]]
            r.relres = [x["relres"] for x in res[a:b]]
            for _ in range(r.chain_steps):
                cpm_vec_axpby(r.c, U_dev[a:b].reshape(-1), 0.0, F_dev[a:b].reshape(-1))
                step = self._solve(pc, F_dev[a:b].reshape(-1), U_dev[a:b].reshape(-1), b - a)
                res[a:b] = step
                r.iterations += [x["iterations"] for x in step]
                r.relres += [x["relres"] for x in step]
        U = U_dev.cpu().numpy() if self.keep_solutions else None
        for r in batch:
            a, b = rows[r.rid]
            if r.chain_steps == 0:
                r.iterations = [x["iterations"] for x in res[a:b]]
                r.relres = [x["relres"] for x in res[a:b]]
            sts = [x["status"] for x in res[a:b]]
            r.status = next((s for s in sts if s != 0), 0)
            if U is not None:
                r.u = U[a:b].copy()
        self.counters["batches"] += 1
        self.counters["rhs_solved"] += nrhs + sum(r.chain_steps * r.nrhs for r in chains)

    def serve(self, requests, realtime: bool = True):
        """Serve requests in arrival order (wall clock from the call); returns them, filled."""
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        pending = collections.deque(reqs)
        queue = []
        t0 = time.perf_counter()

        def now():
            return time.perf_counter() - t0

        while pending or queue:
            while pending and (not realtime or pending[0].arrival <= now()):
                queue.append(pending.popleft())
            if not queue:
                time.sleep(max(0.0, min(0.05, pending[0].arrival - now())))
                continue
            head = queue[0]
            key = (head.surface, head.h, head.c)
            if head.chain_steps > 0:
                batch = [head]
            else:
                batch = [r for r in queue if (r.surface, r.h, r.c) == key and r.chain_steps == 0]
            ids = {id(r) for r in batch}
            queue = [r for r in queue if id(r) not in ids]
            t_start = now()
            self._run_batch(batch)
            self.torch.cuda.synchronize()
            t_done = now()
            for r in batch:
                r.t_start = t_start
                r.t_done = t_done
        return reqs

    def close(self):
        while self._ops:
            self._evict_one()


def summarize(reqs) -> dict:
    """Throughput and latency statistics of served requests (seconds)."""
    done = [r for r in reqs if r.status == 0]
    if not done:
        return {"served": 0, "requests": len(reqs)}
    lat = np.array([r.latency for r in done])
    q = np.array([r.queue_time for r in done])
    svc = lat - q
    first = min(r.arrival for r in reqs)
    span = max(r.t_done for r in done) - first
    solves = sum(r.nrhs * (1 + r.chain_steps) for r in done)
    return {
        "requests": len(reqs), "served": len(done),
        "rejected_budget": sum(r.status == _capi.CPM_ERR_BUDGET for r in reqs),
        "failed": sum(r.status not in (0, _capi.CPM_ERR_BUDGET) for r in reqs),
        "makespan_s": span, "requests_per_s": len(done) / span, "solves_per_s": solves / span,
        "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
        "queue_mean_s": float(q.mean()), "service_mean_s": float(svc.mean()),
        "queue_share": float(q.sum() / lat.sum()),
        "max_relres": float(max(max(r.relres) for r in done)),
    }
