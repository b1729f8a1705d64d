"""Host-side logic of the continuous-batching server, on the CPU with a fake
solver backend (no GPU): admission by footprint, reuse of resident
hierarchies, non-blocking progress of overlapping solves, latency accounting."""
from __future__ import annotations

import pytest

from paper_1411_7018_gb300.serve import REJECTED_FOOTPRINT, Request, Server, poisson_stream, summarize


class FakeClock:
    def __init__(self, dt=1e-3):
        self.t = 0.0
        self.dt = dt

    def __call__(self):
        self.t += self.dt
        return self.t


class FakeHierarchy:
    def __init__(self, n, backend, length=1.0):
        self.n = n
        self.length = length
        self.left = 0
        self.closed = False
        self.solves = 0
        self.backend = backend

    def close(self):
        self.closed = True
        self.backend.live_bytes -= self.n ** 3


class FakeBackend:
    """A solve of size n takes n // 16 advance calls; footprint n^3 bytes."""

    def __init__(self):
        self.created = []
        self.live_bytes = 0
        self.max_live = 0

    def footprint(self, n):
        return n ** 3

    def create(self, n, length):
        H = FakeHierarchy(n, self, length)
        self.created.append(H)
        self.live_bytes += n ** 3
        self.max_live = max(self.max_live, self.live_bytes)
        return H

    def begin(self, H, req):
        assert not H.closed
        assert H.length == self.length_of(req.key), "hierarchy of another domain length"
        H.left = H.n // 16
        H.solves += 1

    def advance(self, H):
        H.left -= 1
        return H.left <= 0

    def result(self, H):
        return H.n // 16, 0, 1e-9

    def length_of(self, key):
        # keys ("L", length) name a domain edge length; every other key the unit cube
        if isinstance(key, tuple) and len(key) == 2 and key[0] == "L":
            return key[1]
        return 1.0


def test_all_requests_complete_and_latency_includes_queueing():
    be = FakeBackend()
    srv = Server(be, hbm_budget=10 ** 9, max_active=4, clock=FakeClock(), idle_sleep=0)
    reqs = [Request(rid=i, n=33, arrival=0.0, key=(33, 0)) for i in range(10)]
    done = srv.run(reqs)
    assert sorted(r.rid for r in done) == list(range(10))
    assert all(r.status == 0 and r.cycles == 2 for r in done)
    # four slots: later requests wait, so their latency is larger
    lat = sorted(r.latency for r in done)
    assert lat[-1] > lat[0]
    assert all(r.admitted >= r.arrival and r.finished > r.admitted for r in done)


def test_admission_respects_the_hbm_budget_and_reuses_hierarchies():
    be = FakeBackend()
    budget = 2 * 65 ** 3 + 33 ** 3
    srv = Server(be, hbm_budget=budget, max_active=16, clock=FakeClock(), idle_sleep=0)
    reqs = [Request(rid=i, n=65 if i % 2 else 33, arrival=0.001 * i, key=None) for i in range(40)]
    done = srv.run(reqs)
    assert len(done) == 40
    assert be.max_live <= budget
    # hierarchies are reused: far fewer created than requests served
    assert len(be.created) < 10
    assert sum(H.solves for H in be.created) == 40


def test_a_request_that_does_not_fit_does_not_block_smaller_ones():
    be = FakeBackend()
    budget = 129 ** 3          # the 129 fits only when nothing else is resident
    srv = Server(be, hbm_budget=budget, max_active=8, clock=FakeClock(), idle_sleep=0)
    reqs = [Request(rid=0, n=65, arrival=0.0, key=None), Request(rid=1, n=129, arrival=0.0005, key=None),
            Request(rid=2, n=33, arrival=0.0006, key=None)]
    done = srv.run(reqs)
    order = [r.rid for r in sorted(done, key=lambda r: r.admitted)]
    assert order.index(2) < order.index(1)
    assert be.max_live <= budget
    # the 129 was admitted after idle hierarchies of other sizes were evicted
    assert any(H.closed for H in be.created)


def test_poisson_stream_is_seeded_and_summary_is_consistent():
    a = poisson_stream(200, rate=200.0, sizes=(65, 129, 257), keys_per_size=3, seed=7)
    b = poisson_stream(200, rate=200.0, sizes=(65, 129, 257), keys_per_size=3, seed=7)
    assert [(r.n, r.arrival, r.key) for r in a] == [(r.n, r.arrival, r.key) for r in b]
    gaps = [y.arrival - x.arrival for x, y in zip(a, a[1:])]
    assert abs(sum(gaps) / len(gaps) - 1 / 200.0) < 0.0015
    assert {r.n for r in a} == {65, 129, 257}
    for i, r in enumerate(a):
        r.finished = r.arrival + 0.01 * (i % 10 + 1)
        r.status = 0
    s = summarize(a)
    assert s["requests"] == 200 and s["converged"] == 200
    assert 10.0 <= s["p50_ms"] <= 60.0 and s["p99_ms"] <= 100.0 + 1e-9


def test_close_releases_resident_hierarchies():
    be = FakeBackend()
    srv = Server(be, hbm_budget=10 ** 9, max_active=2, clock=FakeClock(), idle_sleep=0)
    srv.run([Request(rid=i, n=33, arrival=0.0, key=None) for i in range(3)])
    srv.close()
    assert all(H.closed for H in be.created)
    assert srv.held == 0


def test_a_request_larger_than_the_whole_budget_is_rejected_and_the_server_returns():
    """A hierarchy that alone exceeds the HBM budget can never be admitted:
    the request finishes at once with REJECTED_FOOTPRINT, the others are
    served, and run() returns instead of waiting for it forever."""
    be = FakeBackend()
    srv = Server(be, hbm_budget=65 ** 3, max_active=4, clock=FakeClock(), idle_sleep=0)
    reqs = [Request(rid=0, n=33, arrival=0.0, key=None), Request(rid=1, n=129, arrival=0.0, key=None),
            Request(rid=2, n=65, arrival=0.002, key=None)]
    done = srv.run(reqs)
    by = {r.rid: r for r in done}
    assert sorted(by) == [0, 1, 2]
    assert by[1].status == REJECTED_FOOTPRINT and by[1].cycles == -1
    assert by[0].status == 0 and by[2].status == 0
    assert all(H.n != 129 for H in be.created)
    assert summarize(done)["rejected"] == 1


def test_pool_keeps_hierarchies_of_different_domain_lengths_apart():
    """Two requests of the same grid size on domains of different edge length
    need different mesh widths, so they are never served by one pooled
    hierarchy (the fake backend asserts the length at every begin)."""
    be = FakeBackend()
    srv = Server(be, hbm_budget=10 ** 9, max_active=1, clock=FakeClock(), idle_sleep=0)
    import math
    reqs = [Request(rid=i, n=33, arrival=0.001 * i, key=("L", 1.0 if i % 2 == 0 else math.pi)) for i in range(6)]
    done = srv.run(reqs)
    assert len(done) == 6 and all(r.status == 0 for r in done)
    lengths = sorted(H.length for H in be.created)
    assert lengths == [1.0, math.pi]
