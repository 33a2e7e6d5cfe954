"""Continuous-batching server for simulation requests (host scheduling on
top of the C ABI; every step of every request runs in the library's
kernels).

A request is one seismic run of Eq. (1.1): a grid, a model Q, a Taylor
power M, a step count and a point source; its answer is the final
wavefield, returned to the host.  Requests arrive over time and are
admitted first come, first served while an active slot is free and their
device footprint (vofl_footprint_bytes) fits the HBM budget.

  * square 2D grids with batched kernels join one shared vofl_batch at the
    next step-quantum boundary and leave it when their steps are done, so
    every quantum advances all admitted 2D requests together
    (continuous batching);
  * other shapes (1D lines, 3D grids) run on their own context and CUDA
    stream, overlapping on the device with the batch and with each other;
  * contexts are kept in a pool per grid shape and reused by later
    requests (freeing device memory synchronises the whole device); idle
    pooled contexts count against the budget and are evicted, least
    recently used first, when an admission needs their memory.

A request's answer does not depend on what else runs: batch members are
bit-identical to the same context stepped alone, and solo contexts run
the same kernels either way.
"""
from __future__ import annotations

import collections
import time

import numpy as np

BATCH_EDGES = (64, 128, 256, 512, 768, 1024)


def batchable(shape):
    return len(shape) == 2 and shape[0] == shape[1] and shape[0] in BATCH_EDGES


class _Lib:
    """The library objects the server drives (replaceable by test fakes)."""

    def __init__(self):
        from . import F32, IMPL_FUSED, Batch, Solver, footprint_bytes
        self.Solver, self.Batch = Solver, Batch
        self.footprint = lambda shape, M: footprint_bytes(shape, F32, IMPL_FUSED, M)


class Request:
    __slots__ = ("spec", "Q", "src_idx", "dt", "ctx", "slot", "left", "state", "admit_t", "done_t", "result", "fp")

    def __init__(self, spec, Q, src_idx, fp):
        self.spec, self.Q, self.src_idx, self.fp = spec, Q, src_idx, fp
        self.dt = self.ctx = self.slot = self.result = None
        self.left = spec["nsteps"]
        self.state = "queued"
        self.admit_t = self.done_t = None


class Server:
    """Serve requests (dicts with id, arrival [s], shape, nsteps, M, c0,
    omega0) whose inputs come from `inputs(spec) -> (Q, src_idx)` and whose
    source samples come from `source(spec, dt) -> samples` (dt is the
    model's suggested step, vofl_suggest_dt with courant 0.25).

    budget_bytes bounds the device footprint of admitted requests plus idle
    pooled contexts; max_active bounds the admitted requests; quantum is the
    largest number of batch steps queued at once.  realtime=False admits
    every request at once (arrival times ignored).  prewarm = {shape:
    count} creates idle contexts before serving starts (device allocation
    is slow and belongs to start-up, not to a request's latency)."""

    def __init__(self, budget_bytes=64 << 30, max_active=48, quantum=50, realtime=True, lib=None, prewarm=None,
                 prewarm_M=16):
        self.budget = int(budget_bytes)
        self.max_active = int(max_active)
        self.quantum = int(quantum)
        self.realtime = realtime
        self.lib = lib or _Lib()
        self.pool = collections.OrderedDict()  # (shape, id) -> (Solver, bytes), least recent first
        self.pooled = 0
        self.batch = None
        self.events = []  # (what, request id) in order, for inspection
        for shape, count in (prewarm or {}).items():
            fp = self.lib.footprint(tuple(shape), prewarm_M)
            for _ in range(count):
                if self.pooled + fp > self.budget:
                    break
                s = self.lib.Solver(tuple(shape))
                self.pool[(tuple(shape), id(s))] = (s, fp)
                self.pooled += fp

    # -- contexts -------------------------------------------------------------
    def _ctx(self, shape, fp, active_bytes):
        for key in self.pool:
            if key[0] == shape:
                s, b = self.pool.pop(key)
                self.pooled -= b
                return s
        # evict idle contexts of other shapes while the new one does not fit
        while self.pool and active_bytes + self.pooled + fp > self.budget:
            _, (s, b) = self.pool.popitem(last=False)
            self.pooled -= b
            s.close()
            self.events.append(("evict", None))
        return self.lib.Solver(shape)

    def _release(self, r):
        self.pool[(r.spec["shape"], id(r.ctx))] = (r.ctx, r.fp)
        self.pooled += r.fp
        r.ctx = None

    def close(self):
        if self.batch is not None:
            self.batch.close()
            self.batch = None
        for s, _ in self.pool.values():
            s.close()
        self.pool.clear()
        self.pooled = 0

    # -- one request ------------------------------------------------------------
    def _start(self, r, source, active_bytes):
        sp = r.spec
        s = self._ctx(sp["shape"], r.fp, active_bytes)
        s.set_q(r.Q, sp["c0"], sp["omega0"])
        s.set_M(sp["M"])
        r.dt = s.suggest_dt(0.25)
        s.set_state(np.zeros(sp["shape"], np.float32))
        s.set_source(r.src_idx, source(sp, r.dt))
        r.ctx = s
        if batchable(sp["shape"]):
            if self.batch is None:
                self.batch = self.lib.Batch()
            r.slot = self.batch.add(s, r.dt)
            r.state = "batched"
        else:
            s.step(sp["nsteps"], r.dt)  # queued on the context's own stream
            r.left = 0
            r.state = "finishing"
        self.events.append(("admit", sp["id"]))

    def run(self, requests, inputs, source):
        """Serve all requests; returns (records, makespan_s).  A record has
        id, shape, nsteps, M, dt, latency_s (arrival to answer on the host),
        queue_s (arrival to admission), point_steps and the result array."""
        reqs = []
        for sp in sorted(requests, key=lambda d: d["arrival"]):
            Q, idx = inputs(sp)
            reqs.append(Request(sp, Q, idx, self.lib.footprint(sp["shape"], sp["M"])))
        if any(r.fp > self.budget for r in reqs):
            raise ValueError("a request does not fit the memory budget on its own")
        pending = collections.deque(reqs)
        queue = collections.deque()
        active = []
        used = 0
        t0 = time.perf_counter()

        def clock():
            return time.perf_counter() - t0

        while pending or queue or active:
            now = clock()
            while pending and (not self.realtime or pending[0].spec["arrival"] <= now):
                queue.append(pending.popleft())
            progressed = False
            # admission: first come, first served, by slots and footprint
            while queue and len(active) < self.max_active and used + queue[0].fp <= self.budget:
                r = queue.popleft()
                r.admit_t = clock()
                self._start(r, source, used)
                used += r.fp
                active.append(r)
                progressed = True
            # one batch quantum once the previous one has finished
            members = [r for r in active if r.state == "batched"]
            if members and self.batch.query():
                q = min(self.quantum, min(r.left for r in members))
                self.batch.step(q)
                for r in members:
                    r.left -= q
                    if r.left == 0:
                        self.batch.remove(r.slot)
                        r.state = "finishing"
                progressed = True
            # completions: the context's stream is idle -> read the answer
            for r in list(active):
                if r.state == "finishing" and r.ctx.query():
                    r.result = r.ctx.get_state()
                    r.done_t = clock()
                    r.state = "done"
                    self._release(r)
                    active.remove(r)
                    used -= r.fp
                    self.events.append(("done", r.spec["id"]))
                    progressed = True
            if not progressed:
                if not active and not queue and pending:
                    time.sleep(max(0.0, min(pending[0].spec["arrival"] - clock(), 0.01)))
                else:
                    time.sleep(5e-5)
        makespan = clock()
        out = []
        for r in reqs:
            arr = r.spec["arrival"] if self.realtime else 0.0
            out.append({"id": r.spec["id"], "shape": r.spec["shape"], "nsteps": r.spec["nsteps"],
                        "M": r.spec["M"], "dt": r.dt, "latency_s": r.done_t - arr, "queue_s": r.admit_t - arr,
                        "point_steps": int(np.prod(r.spec["shape"])) * r.spec["nsteps"], "result": r.result})
        return out, makespan


def solo(spec, Q, src_idx, source):
    """The same request run alone on a fresh context (for equality checks)."""
    from . import Solver
    with Solver(spec["shape"]) as s:
        s.set_q(Q, spec["c0"], spec["omega0"])
        s.set_M(spec["M"])
        dt = s.suggest_dt(0.25)
        s.set_state(np.zeros(spec["shape"], np.float32))
        s.set_source(src_idx, source(spec, dt))
        s.step(spec["nsteps"], dt)
        out = s.get_state()
        s.sync()
        return out


def summarize(records, makespan):
    lat = np.array([r["latency_s"] for r in records])
    ps = sum(r["point_steps"] for r in records)
    return {"requests": len(records), "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
            "queue_p50_s": float(np.percentile([r["queue_s"] for r in records], 50)),
            "makespan_s": makespan, "value": ps / makespan / 1e6, "unit": "Mpoint-steps/s"}
