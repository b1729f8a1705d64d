"""Continuous-batching solve server over the libma C ABI.

Requests (a grid size, f and the Dirichlet data g on the device, a
tolerance) arrive over time.  The server keeps multigrid hierarchies resident
on the device in a per-size pool, admits waiting requests as hierarchies and
HBM budget free up, and drives every admitted solve with the non-blocking
ma_solve_begin / ma_solve_advance calls: each pass over the active set
advances every solve whose last cycle has finished, so the cycles of all
admitted requests overlap on the GPU (each hierarchy has its own stream).  A
request's latency is its completion time minus its arrival time, queueing
included.  A request whose hierarchy alone exceeds the HBM budget can never be
admitted; it is finished at once with status REJECTED_FOOTPRINT.

The scheduling logic only talks to a small backend interface (footprint,
create, begin, advance, result, solution), so it can be exercised on the CPU
with a fake backend; ``LibmaBackend`` is the GPU one.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Any, Callable, Sequence

# Request.status of a request whose hierarchy is larger than the server's
# whole HBM budget (never admitted); the other values are ma_status codes.
REJECTED_FOOTPRINT = -2


@dataclasses.dataclass
class Request:
    rid: int
    n: int
    arrival: float            # seconds after the stream starts
    key: Any                  # which device inputs (f, g) the request uses
    tol: float = 1e-8
    # filled by the server
    admitted: float = float("nan")
    finished: float = float("nan")
    cycles: int = -1
    status: int = -1
    residual: float = float("nan")

    @property
    def latency(self) -> float:
        return self.finished - self.arrival

    @property
    def unknowns(self) -> int:
        return (self.n - 2) ** 3


class LibmaBackend:
    """Hierarchies of libma on one device, one CUDA stream each."""

    def __init__(self, precision: int, inputs: dict, device=None, desc_kw: dict | None = None):
        import torch
        from . import libma as M
        self.M = M
        self.torch = torch
        self.precision = precision
        self.inputs = inputs        # key -> (f_dev, g_dev, length)
        self.device = device or torch.device("cuda")
        self.desc_kw = desc_kw or {}

    def footprint(self, n: int) -> int:
        return self.M.ma_hierarchy_footprint(self.M.make_desc(n, precision=self.precision, **self.desc_kw))

    def create(self, n: int, length: float):
        stream = self.torch.cuda.Stream(device=self.device)
        H = self.M.Hierarchy(self.M.make_desc(n, length=length, precision=self.precision, **self.desc_kw),
                             stream=stream, device=self.device)
        return H

    def begin(self, H, req: Request):
        f, g, _ = self.inputs[req.key]
        # inputs were produced on another stream: order this hierarchy's
        # stream after their producer
        H.stream.wait_stream(self.torch.cuda.current_stream(self.device))
        self.M.ma_set_rhs_bc(H.handle, f, g)
        self.M.ma_solve_begin(H.handle, self.M.ma_solve_opts(req.tol, self.M.MA_NORM_MAX, 1, 60, self.M.MA_INIT_FMG))

    def advance(self, H) -> bool:
        return self.M.ma_solve_advance(H.handle)

    def result(self, H):
        r = self.M.ma_solve_get_result(H.handle, raise_on_error=False)
        return r.cycles, r.status, r.res

    def solution(self, H, out):
        self.M.ma_get_solution(H.handle, out)

    def length_of(self, key) -> float:
        return self.inputs[key][2]


class Server:
    """Continuous batching with admission by HBM footprint.

    hbm_budget: bytes of workspace the resident hierarchies may hold in total.
    max_active: cap on concurrently admitted solves.
    on_complete: callback(req, hierarchy) called at completion (e.g. to copy
    the solution out) before the hierarchy returns to the pool.
    """

    def __init__(self, backend, hbm_budget: int, max_active: int = 32,
                 on_complete: Callable | None = None, clock: Callable[[], float] = time.perf_counter,
                 idle_sleep: float = 20e-6):
        self.b = backend
        self.budget = hbm_budget
        self.max_active = max_active
        self.on_complete = on_complete
        self.clock = clock
        self.idle_sleep = idle_sleep
        # Resident hierarchies are pooled by (n, domain edge length): a
        # hierarchy's mesh width h = length / (n - 1) is fixed when it is
        # created, so one of another length must not serve the request.
        self.free = collections.defaultdict(list)     # (n, length) -> [hierarchy]
        self.held = 0                                  # bytes of all resident hierarchies
        self.live = collections.Counter()              # (n, length) -> resident hierarchies (busy or free)
        self.created = 0
        self.footprints: dict[int, int] = {}

    def _footprint(self, n: int) -> int:
        if n not in self.footprints:
            self.footprints[n] = self.b.footprint(n)
        return self.footprints[n]

    def _acquire(self, n: int, length: float):
        """A resident hierarchy of size n and domain length `length`: a free
        one, else a new one within the budget.  When the budget is full and a
        hierarchy of this kind exists (busy), wait for it rather than evict;
        otherwise evict idle hierarchies of other kinds, largest first, to
        make room."""
        kind = (n, length)
        if self.free[kind]:
            return self.free[kind].pop()
        need = self._footprint(n)
        if self.held + need > self.budget:
            if self.live[kind] > 0:
                return None
            for m in sorted(self.free, key=lambda m: -self._footprint(m[0])):
                while self.free[m] and self.held + need > self.budget:
                    H = self.free[m].pop()
                    self._release_memory(H, m)
            if self.held + need > self.budget:
                return None
        H = self.b.create(n, length)
        self.held += need
        self.live[kind] += 1
        self.created += 1
        return H

    def _release_memory(self, H, kind):
        close = getattr(H, "close", None)
        if close:
            close()
        self.held -= self._footprint(kind[0])
        self.live[kind] -= 1

    def run(self, requests: Sequence[Request]) -> list[Request]:
        """Serve requests (sorted by arrival time) to completion; returns them
        with admission and completion times filled in."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting: collections.deque = collections.deque()
        active: list = []
        done: list[Request] = []
        t0 = self.clock()
        while pending or waiting or active:
            now = self.clock() - t0
            while pending and pending[0].arrival <= now:
                req = pending.popleft()
                if self._footprint(req.n) > self.budget:
                    # can never fit, even with every other hierarchy evicted
                    req.admitted = req.finished = now
                    req.status = REJECTED_FOOTPRINT
                    done.append(req)
                    continue
                waiting.append(req)
            # admission: first come, first served, but a request that does not
            # fit yet does not block smaller ones behind it
            if waiting and len(active) < self.max_active:
                still = collections.deque()
                while waiting:
                    req = waiting.popleft()
                    H = self._acquire(req.n, self.b.length_of(req.key)) if len(active) < self.max_active else None
                    if H is None:
                        still.append(req)
                        continue
                    req.admitted = self.clock() - t0
                    self.b.begin(H, req)
                    active.append((req, H, (req.n, self.b.length_of(req.key))))
                waiting = still
            progressed = False
            still_active = []
            for req, H, kind in active:
                if self.b.advance(H):
                    req.finished = self.clock() - t0
                    req.cycles, req.status, req.residual = self.b.result(H)
                    if self.on_complete:
                        self.on_complete(req, H)
                    self.free[kind].append(H)
                    done.append(req)
                    progressed = True
                else:
                    still_active.append((req, H, kind))
            active = still_active
            if not progressed:
                if active or waiting:
                    time.sleep(self.idle_sleep)
                elif pending and not waiting:
                    time.sleep(max(0.0, min(pending[0].arrival - (self.clock() - t0), 0.01)))
        return done

    def close(self):
        for kind, hs in self.free.items():
            for H in hs:
                self._release_memory(H, kind)
        self.free.clear()


def poisson_stream(count: int, rate: float, sizes: Sequence[int], keys_per_size: int, seed: int,
                   tol: float = 1e-8) -> list[Request]:
    """Seeded Poisson arrivals (exponential inter-arrival times, mean 1/rate)
    with sizes drawn uniformly from `sizes`; each request names one of
    keys_per_size prepared inputs of its size."""
    import numpy as np
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    ns = rng.choice(np.asarray(sizes), size=count)
    ks = rng.integers(0, keys_per_size, size=count)
    return [Request(rid=i, n=int(ns[i]), arrival=float(t[i]), key=(int(ns[i]), int(ks[i])), tol=tol)
            for i in range(count)]


def summarize(done: Sequence[Request], wall: float | None = None) -> dict:
    import numpy as np
    lat = np.array([r.latency for r in done]) * 1e3
    unknowns = sum(r.unknowns for r in done)
    span = wall if wall is not None else (max(r.finished for r in done) - min(r.arrival for r in done))
    return {"requests": len(done), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "throughput_req_s": len(done) / span,
            "unknowns_per_s": unknowns / span, "wall_s": span,
            "converged": int(sum(1 for r in done if r.status == 0)),
            "rejected": int(sum(1 for r in done if r.status == REJECTED_FOOTPRINT))}
