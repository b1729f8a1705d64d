"""GPU tests of batched solves (ma_batch_solve) and of the continuous-batching
server: every result is the same alone and in the mix (bitwise: each
hierarchy's arithmetic is independent of the others), and matches the FP64
oracle at the FP64 bound."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_1411_7018_gb300 import libma as M
from paper_1411_7018_gb300 import problems as P
from paper_1411_7018_gb300.serve import LibmaBackend, Request, Server, summarize

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    M.load()


def solo(pr, precision, tol=1e-10):
    H = M.Hierarchy(M.make_desc(pr.n, length=pr.length, precision=precision))
    H.set_rhs_bc(torch.from_numpy(pr.f).cuda(), torch.from_numpy(pr.initial()).cuda())
    r = H.solve(tol=tol)
    u = torch.empty(pr.f.shape, dtype=torch.float64, device="cuda")
    H.get_solution(u)
    torch.cuda.synchronize()
    H.close()
    return u.cpu().numpy(), r


@pytest.mark.parametrize("precision", [M.MA_MIXED, M.MA_FP64])
def test_batch_solve_equals_solo_solves(precision):
    sizes = [33, 65, 33, 129, 65, 33]
    prs = [P.make("cosine", n, seed=10 + b, eps=(0.005, 0.02)) for b, n in enumerate(sizes)]
    hs, keep = [], []
    for pr in prs:
        H = M.Hierarchy(M.make_desc(pr.n, precision=precision), stream=torch.cuda.Stream())
        f = torch.from_numpy(pr.f).cuda()
        g = torch.from_numpy(pr.initial()).cuda()
        torch.cuda.synchronize()
        H.set_rhs_bc(f, g)
        hs.append(H)
        keep += [f, g]
    res = M.ma_batch_solve([H.handle for H in hs], M.ma_solve_opts(1e-10, M.MA_NORM_MAX, 1, 60, M.MA_INIT_FMG))
    assert all(r.status == 0 and r.res <= 1e-10 for r in res)
    for pr, H in zip(prs, hs):
        u = torch.empty(pr.f.shape, dtype=torch.float64, device="cuda")
        H.get_solution(u)
        torch.cuda.synchronize()
        got = u.cpu().numpy()
        ref, _ = solo(pr, precision)
        assert np.array_equal(got, ref)
        H.close()
    ref = prs[0].initial()
    O.solve(ref, prs[0].f, prs[0].h, tol=1e-10)
    assert np.max(np.abs(solo(prs[0], precision)[0] - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_nonblocking_solve_equals_blocking():
    pr = P.make("exp", 65)
    H = M.Hierarchy(M.make_desc(65, precision=M.MA_MIXED))
    H.set_rhs_bc(torch.from_numpy(pr.f).cuda(), torch.from_numpy(pr.initial()).cuda())
    M.ma_solve_begin(H.handle, M.ma_solve_opts(1e-10, M.MA_NORM_MAX, 1, 60, M.MA_INIT_FMG))
    polls = 0
    while not M.ma_solve_advance(H.handle):
        polls += 1
    r = M.ma_solve_get_result(H.handle)
    u = torch.empty(pr.f.shape, dtype=torch.float64, device="cuda")
    H.get_solution(u)
    torch.cuda.synchronize()
    H.close()
    ref, rr = solo(pr, M.MA_MIXED)
    assert r.cycles == rr.cycles and r.status == 0
    assert np.array_equal(u.cpu().numpy(), ref)


def test_server_results_same_alone_and_in_the_mix():
    sizes = (33, 65)
    inputs, prs = {}, {}
    for n in sizes:
        for k in range(2):
            pr = P.make("cosine", n, seed=100 * n + k, eps=(0.005, 0.02))
            prs[(n, k)] = pr
            inputs[(n, k)] = (torch.from_numpy(pr.f).cuda(), torch.from_numpy(pr.initial()).cuda(), 1.0)
    rng = np.random.default_rng(5)
    reqs = [Request(rid=i, n=int(rng.choice(sizes)), arrival=0.0005 * i, key=None, tol=1e-10) for i in range(16)]
    for r in reqs:
        r.key = (r.n, int(rng.integers(0, 2)))
    sols = {}

    def keep(req, H):
        u = torch.empty((req.n,) * 3, dtype=torch.float64, device="cuda")
        M.ma_get_solution(H.handle, u)
        H.stream.synchronize()
        sols[req.rid] = u.cpu().numpy()

    be = LibmaBackend(M.MA_MIXED, inputs)
    torch.cuda.synchronize()
    srv = Server(be, hbm_budget=4 << 30, max_active=8, on_complete=keep)
    done = srv.run(reqs)
    srv.close()
    assert len(done) == 16 and all(r.status == 0 for r in done)
    # solves overlapped: some request was admitted before an earlier one finished
    assert any(b.admitted < a.finished for a in done for b in done if b.rid > a.rid)
    alone = {key: solo(pr, M.MA_MIXED)[0] for key, pr in prs.items()}
    for r in done:
        assert np.array_equal(sols[r.rid], alone[r.key])
    s = summarize(done)
    assert s["converged"] == 16 and s["p99_ms"] >= s["p50_ms"] > 0
