"""Serving loop: a stream of CPM solve requests on one GPU.  No counterpart in the paper.

A request names an operator -- a registered surface, a grid spacing h and the shift c of
(c - Lap_S) u = f -- and carries right-hand sides evaluated at the band's closest points,
optionally as a backward-Euler chain (c = 1/dt, f_{n+1} = u_n / dt) that reuses one
factorisation.  The server

* keeps bands and partitions on the host (per surface and h) and factorised operators
  resident in HBM (per surface, h, c), least recently used first out;
* runs `slots` batches at once (default 1): each slot owns a CUDA stream and a host thread,
  and one operator serves one batch at a time, as a handle is not thread-safe.  More than one
  slot lets batches on different operators overlap on the device;
* admits continuously: whenever a slot is free, the oldest queued request whose operator is
  not busy picks the operator, and every queued plain request for the same operator joins its
  batch (one lock-step multi-rhs cpm_gmres_solve); requests arriving meanwhile wait for the
  next free slot, requests for a busy operator for its next batch;
* admits by an HBM budget: a batch reserves its vectors and, for a new operator, the set-up
  peak of the library's device plan (oras_plan); idle operators are evicted to make room,
  operators in use never are; a batch that does not fit now waits for running batches to
  finish, one that cannot fit even alone fails with CPM_ERR_BUDGET;
* records per request: arrival, start of its batch, completion, status, iterations and the
  relative residual of every right-hand side, and per batch CUDA events on its stream.

Every step on the GPU runs in the library through the C ABI; this module only schedules and
moves vectors.  Results are deterministic: a request gets bit-identical solutions whether it
is served alone or inside a mix, because each right-hand side of a batch runs exactly the
operations of a single-rhs solve with the operator's fixed solve schedule (the default
schedule unless one is pinned per surface and h with `pin_schedule`), whatever the other
slots do.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import dataclasses
import math
import threading
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
    slot: int = -1                  # slot that served it

    @property
    def nrhs(self) -> int:
        return int(self.f.shape[0])

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival

    @property
    def queue_time(self) -> float:
        return self.t_start - self.arrival

    @property
    def key(self):
        return (self.surface, float(self.h), float(self.c))


class _Operator:
    def __init__(self, pc, resident: int):
        self.pc = pc
        self.resident = resident


@dataclasses.dataclass
class BatchRecord:
    """One served batch: its requests, slot, and CUDA events recorded on the slot's stream at
    the start of its work and after its last copy (elapsed_time between two records gives the
    device-side interval of the batch)."""
    rids: list
    slot: int
    key: tuple
    start: object
    end: object


class Server:
    def __init__(self, budget_bytes: int | None = None, precision: str = "fp32", restart: int = 50,
                 tol: float = 1e-8, max_it: int = 1000, method: str = "oras", alpha: float = 4.0,
                 alpha_x: float = 40.0, n_overlap: int = 2, p: int = 3, nodes_per_sub: int = 4000,
                 keep_solutions: bool = False, slots: int = 1, trace=None):
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
        self.slots = max(1, int(slots))
        self._streams = [torch.cuda.Stream() for _ in range(self.slots)]
        self._surfaces = {}
        self._bands = {}
        self._ops: collections.OrderedDict = collections.OrderedDict()
        self._schedules = {}
        self._lock = threading.RLock()            # operator table, budget, counters
        self._busy = set()                        # operator keys of batches in flight
        self.used = 0                             # resident operators
        self.reserved = 0                         # vectors and set-up transients in flight
        self.counters = collections.Counter()
        self.batches: list[BatchRecord] = []
        self.trace = trace                         # optional file: one line per batch start / end

    def _log(self, msg: str):
        if self.trace is not None:
            with self._lock:
                self.trace.write(msg + "\n")
                self.trace.flush()

    # ---------------------------------------------------------------- registry
    def register_surface(self, name: str, kind: str, R: float = 1.0, r: float = 0.0, verts=None,
                         tris=None):
        self._surfaces[name] = (kind, R, r, verts, tris)

    def band(self, surface: str, h: float):
        """(Band, Partition, closest points of the actives) of a surface at spacing h."""
        key = (surface, float(h))
        with self._lock:
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
    def _evict_idle(self, need: int, keep=None) -> None:
        """Evict least recently used operators that no batch uses, other than `keep`, until
        `need` more bytes fit."""
        for key in list(self._ops.keys()):
            if self.used + self.reserved + need <= self.budget:
                return
            if key in self._busy or key == keep:
                continue
            op = self._ops.pop(key)
            self.used -= op.resident
            del op.pc
            self.counters["evictions"] += 1

    def _reserve(self, key, nrhs: int):
        """Reserve HBM for a batch of nrhs right-hand sides on operator `key`.  Returns
        (reservation bytes, plan or None), or None when it does not fit now; raises
        CPM_ERR_BUDGET when it can never fit."""
        with self._lock:
            band, part, cp = self.band(key[0], key[1])
            vec_bytes = 2 * 8 * nrhs * len(cp)
            if key in self._ops:
                need, plan = vec_bytes, None
            else:
                plan = oras_plan(band, part, self.method, self.precision, self.restart, min(nrhs, 8))
                need = max(plan["setup_peak_bytes"], plan["resident_bytes"]) + vec_bytes
                if need > self.budget:
                    raise CpmError(_capi.CPM_ERR_BUDGET, f"operator {key} needs {need} bytes, "
                                                         f"budget {self.budget}")
            self._evict_idle(need, keep=key)      # the operator this batch reuses stays
            if self.used + self.reserved + need > self.budget:
                return None
            self.reserved += need
            self._busy.add(key)
            if key in self._ops:
                self._ops.move_to_end(key)
            return need, plan

    def _operator(self, key, plan, stream):
        """The resident operator for `key` (set up on `stream` when new); (pc, fresh)."""
        with self._lock:
            if key in self._ops:
                self.counters["operator_hits"] += 1
                return self._ops[key].pc, False
        band, part, _ = self.band(key[0], key[1])
        pc = oras_setup(band, part, key[2], self.method, self.alpha, self.alpha_x, self.precision,
                        stream=stream)
        for knob, value in self._schedules.get((key[0], key[1]), {}).items():
            oras_tune(pc, **{knob: value})
        with self._lock:
            self._ops[key] = _Operator(pc, plan["resident_bytes"])
            self.used += plan["resident_bytes"]
            self.counters["setups"] += 1
        return pc, True

    def _release(self, key, need: int):
        with self._lock:
            self.reserved -= need
            self._busy.discard(key)

    # ---------------------------------------------------------------- execution
    def _solve(self, pc, F_dev, U_dev, nrhs, stream):
        return cpm_gmres_solve(pc, F_dev, U_dev, nrhs=nrhs, restart=self.restart, tol=self.tol,
                               max_it=self.max_it, raise_on_failure=False, stream=stream)

    def _run_batch(self, batch, slot: int, plan, t0: float):
        """One batch on one slot (its own stream): operator, copies in, the multi-rhs solve,
        backward-Euler chains, copies out.  Runs in the slot's host thread."""
        torch = self.torch
        stream = self._streams[slot]
        key = batch[0].key
        t_start = time.perf_counter() - t0
        self._log(f"start slot={slot} key={key} rids={[r.rid for r in batch]} nrhs={sum(r.nrhs for r in batch)} "
                  f"chains={[r.chain_steps for r in batch]} fresh={key not in self._ops}")
        with torch.cuda.stream(stream):
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            pc, fresh = self._operator(key, plan, stream)
            nrhs = sum(r.nrhs for r in batch)
            F = np.concatenate([r.f for r in batch], axis=0)
            F_dev = torch.from_numpy(np.ascontiguousarray(F)).pin_memory().to("cuda", non_blocking=True)
            U_dev = torch.empty_like(F_dev)
            res = self._solve(pc, F_dev.view(-1), U_dev.view(-1), nrhs, stream)
            rows, row = {}, 0
            for r in batch:
                rows[r.rid] = (row, row + r.nrhs)
                row += r.nrhs
            # backward-Euler steps: f_{k+1} = u_k / dt = c u_k, same operator
            chains = [r for r in batch if r.chain_steps > 0]
            for r in chains:
                a, b = rows[r.rid]
                r.iterations = [x["iterations"] for x in res[a:b]]
                r.relres = [x["relres"] for x in res[a:b]]
                for _ in range(r.chain_steps):
                    cpm_vec_axpby(r.c, U_dev[a:b].reshape(-1), 0.0, F_dev[a:b].reshape(-1), stream=stream)
                    step = self._solve(pc, F_dev[a:b].reshape(-1), U_dev[a:b].reshape(-1), b - a, stream)
                    res[a:b] = step
                    r.iterations += [x["iterations"] for x in step]
                    r.relres += [x["relres"] for x in step]
            U = U_dev.cpu().numpy() if self.keep_solutions else None
            ev1.record(stream)
            stream.synchronize()
        t_done = time.perf_counter() - t0
        self._log(f"done slot={slot} key={key} t={t_done - t_start:.3f}s")
        for r in batch:
            a, b = rows[r.rid]
            if r.chain_steps == 0:
                r.iterations = [x["iterations"] for x in res[a:b]]
                r.relres = [x["relres"] for x in res[a:b]]
            sts = [x["status"] for x in res[a:b]]
            r.status = next((st for st in sts if st != 0), 0)
            if U is not None:
                r.u = U[a:b].copy()
            r.factorised = fresh
            r.batch_rhs = nrhs
            r.slot = slot
            r.t_start = t_start
            r.t_done = t_done
        with self._lock:
            self.batches.append(BatchRecord([r.rid for r in batch], slot, key, ev0, ev1))
            self.counters["batches"] += 1
            self.counters["rhs_solved"] += nrhs + sum(r.chain_steps * r.nrhs for r in chains)

    def _next_batch(self, queue):
        """The oldest queued request whose operator is idle, with the queued plain requests
        of the same operator (a chain runs alone); None if every queued operator is busy."""
        for head in queue:
            if head.key in self._busy:
                continue
            if head.chain_steps > 0:
                return [head]
            return [r for r in queue if r.key == head.key and r.chain_steps == 0]
        return None

    def serve(self, requests, realtime: bool = True):
        """Serve requests in arrival order (wall clock from the call); returns them, filled."""
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        pending = collections.deque(reqs)
        queue = []
        t0 = time.perf_counter()
        free = list(range(self.slots))
        running = {}                              # future -> (slot, key, reservation)

        def now():
            return time.perf_counter() - t0

        with cf.ThreadPoolExecutor(max_workers=self.slots) as pool:
            while pending or queue or running:
                while pending and (not realtime or pending[0].arrival <= now()):
                    queue.append(pending.popleft())
                for fut in [f for f in running if f.done()]:
                    slot, key, need = running.pop(fut)
                    self._release(key, need)
                    free.append(slot)
                    fut.result()                  # a library error ends the stream here
                dispatched = False
                while free and queue:
                    batch = self._next_batch(queue)
                    if batch is None:
                        break
                    key = batch[0].key
                    try:
                        got = self._reserve(key, sum(r.nrhs for r in batch))
                    except CpmError as e:
                        for r in batch:
                            r.status = e.status
                            r.t_start = r.t_done = now()
                        self.counters["rejected"] += len(batch)
                        ids = {id(r) for r in batch}
                        queue = [r for r in queue if id(r) not in ids]
                        continue
                    if got is None:               # waits for running batches to free HBM
                        break
                    need, plan = got
                    ids = {id(r) for r in batch}
                    queue = [r for r in queue if id(r) not in ids]
                    slot = free.pop(0)
                    fut = pool.submit(self._run_batch, batch, slot, plan, t0)
                    running[fut] = (slot, key, need)
                    dispatched = True
                if dispatched:
                    continue
                if running:
                    wait = 0.05 if not pending else max(0.0, min(0.05, pending[0].arrival - now()))
                    cf.wait(list(running), timeout=wait, return_when=cf.FIRST_COMPLETED)
                elif pending:
                    time.sleep(max(0.0, min(0.05, pending[0].arrival - now())))
                elif queue:
                    raise RuntimeError("serving: queued work that can never be dispatched")
        return reqs

    def close(self):
        with self._lock:
            self._busy.clear()
            while self._ops:
                key, op = self._ops.popitem(last=False)
                self.used -= op.resident
                del op.pc
                self.counters["evictions"] += 1


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
        "slots_used": len({r.slot for r in done}),
    }


def overlap_seconds(records) -> float:
    """Total device time during which at least two batches of the records were in flight
    (from their CUDA events; events of different streams are compared through elapsed_time
    against the earliest start)."""
    if len(records) < 2:
        return 0.0
    ref = records[0].start
    iv = sorted((ref.elapsed_time(b.start) / 1e3, ref.elapsed_time(b.end) / 1e3) for b in records)
    total, end = 0.0, iv[0][1]
    for a, b in iv[1:]:
        if a < end:
            total += min(b, end) - a
        end = max(end, b)
    return total
