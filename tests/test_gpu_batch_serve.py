"""Batched and served solves (the table-driven batch driver and the
continuous-batching server) against the FP64 CPU oracle's p*, through the C ABI.

Every grid of a batch and every request of a served mix must reach
||r|| <= 1e-10 ||b|| (re-evaluated with the oracle's operator) and lie within
1e-8 relative L2 of p*, the zero-mean solution of Eq. 10 with the faces of
Eqs. 11-12 (Shin, Chergui & Juric, arXiv 1410.8568, Sec. 2.3); a served
request is also bitwise its solo result.  The server's own bookkeeping shows
that requests were admitted while others were running and that their solves
overlapped.
"""
import time

import numpy as np
import pytest

import oracle
from paper_1410_8568_gb300 import gbmg
from paper_1410_8568_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10
ERR = 1e-8


def cells(shape):
    return (shape[2], shape[1], shape[0])


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=torch.float64)


def sphere_problem(n, ratio, seed):
    """One grid of the batched workload: a sphere of seeded radius (0.05-0.2)
    and centre, the given density ratio, Neumann walls, N(0,1) right-hand side."""
    rng = np.random.default_rng(seed)
    r = rng.uniform(0.05, 0.2)
    h = 1.0 / n
    c = rng.uniform(r + 2 * h, 1.0 - r - 2 * h, size=3)
    shape = (n, n, n)
    rho = I.density_field(shape, None, [(tuple(c), r)], ratio)
    return I.Problem(shape, (I.NEUMANN,) * 3, rho, I.rhs_white(shape, rng),
                     name="sphere_%d_%g_%d" % (n, ratio, seed), ratio=ratio)


_pstar = {}


def pstar_of(P, faces):
    if P.name not in _pstar:
        _pstar[P.name] = oracle.solve_exact(P.shape, P.bc, faces, P.rhs).x
    return _pstar[P.name]


def check_against_oracle(P, faces, x, what):
    bp = P.rhs - P.rhs.mean()
    rel = np.linalg.norm(oracle.residual(P.shape, P.bc, faces, bp, x)) / np.linalg.norm(bp)
    ps = pstar_of(P, faces)
    err = np.linalg.norm(x - ps) / np.linalg.norm(ps)
    print("%s %s rel_res(oracle)=%.2e err=%.2e" % (what, P.name, rel, err))
    assert rel <= 1.05 * TOL, (what, P.name, rel)
    assert err <= ERR, (what, P.name, err)


# a ragged batch: every edge of the batched workload, every density ratio
BATCH = [(32, 10.0), (48, 100.0), (64, 1000.0), (96, 10.0), (128, 100.0), (128, 1000.0), (96, 1000.0),
         (48, 10.0)]


@pytest.mark.parametrize("precision,outer", [(gbmg.MIXED, gbmg.OUTER_FP64), (gbmg.FP64, gbmg.OUTER_FP64),
                                             (gbmg.MIXED, gbmg.OUTER_XP)], ids=["mixed", "fp64", "mixed_xp"])
def test_batch_matches_oracle(precision, outer):
    probs = [sphere_problem(n, ratio, 41 + g) for g, (n, ratio) in enumerate(BATCH)]
    faces = [oracle.faces_from_density(P.shape, P.bc, P.rho) for P in probs]
    solvers = [gbmg.Solver(P.shape, P.bc, faces=[dev(a) for a in f], precision=precision, outer=outer)
               for P, f in zip(probs, faces)]
    B = gbmg.Batch(solvers)
    rhs = [dev(P.rhs) for P in probs]
    ps = [torch.zeros_like(r) for r in rhs]
    sts = B.solve(rhs, ps, tol=TOL)
    torch.cuda.synchronize()
    for P, f, p, st in zip(probs, faces, ps, sts):
        assert st.status == gbmg.OK and st.rel_res <= TOL, (P.name, st.as_dict())
        check_against_oracle(P, f, p.cpu().numpy(), "batch")
    B.close()
    for S in solvers:
        S.close()


def served_mix():
    """Requests of three size lanes (up to 64^3, up to 128^3), drop/film and
    sphere fields, density ratios 10 and 1000."""
    return [I.config2(64), I.config1(32), I.config2(96), I.config1(48), I.config2(128),
            I.config1(32, ratio=10.0), I.config2(48), I.config1(64)]


def poll_all(srv, tickets, limit_s=300):
    results = {}
    deadline = time.time() + limit_s
    while len(results) < len(tickets) and time.time() < deadline:
        for t in tickets:
            if t not in results:
                r = srv.poll(t)
                if r is not None:
                    results[t] = r
        time.sleep(0.0005)
    assert len(results) == len(tickets)
    return results


@pytest.mark.parametrize("outer", [gbmg.OUTER_FP64, gbmg.OUTER_XP], ids=["fp64_outer", "xp_outer"])
def test_server_results_match_oracle_and_alone(outer):
    probs = served_mix()
    faces = [oracle.faces_from_density(P.shape, P.bc, P.rho) for P in probs]
    alone = []
    for P, f in zip(probs, faces):
        with gbmg.Solver(P.shape, P.bc, faces=[dev(a) for a in f], outer=outer) as S:
            p = torch.zeros(cells(P.shape), dtype=torch.float64, device="cuda")
            st = S.solve(dev(P.rhs), p, tol=TOL)
            alone.append((p, st.iters))
    torch.cuda.synchronize()
    srv = gbmg.Server(hbm_budget_bytes=1 << 30, max_slots=4, outer=outer)
    tickets, outs, keep = [], [], []
    for q, (P, f) in enumerate(zip(probs, faces)):
        fd = [dev(a) for a in f]
        b = dev(P.rhs)
        p = torch.zeros_like(b)
        keep.append((fd, b))
        torch.cuda.synchronize()
        tickets.append(srv.submit(P.shape, P.bc, fd, b, p, tol=TOL))
        outs.append(p)
        if q in (2, 5):
            time.sleep(0.005)  # later requests arrive while the first ones run
    results = poll_all(srv, tickets)
    info = srv.info()
    assert info["completed"] == len(tickets)
    assert 2 <= info["max_in_flight"] <= 4
    assert info["peak_bytes"] <= 1 << 30
    sts = []
    for t, (pa, ia), pb, P, f in zip(tickets, alone, outs, probs, faces):
        rc, st = results[t]
        assert rc == gbmg.OK and st.iters == ia, (P.name, rc, st.iters, ia)
        assert torch.equal(pa, pb), P.name
        check_against_oracle(P, f, pb.cpu().numpy(), "served")
        sts.append(st)
    # continuous batching: some request was admitted after another had taken
    # refinement steps and before it finished, so their work overlapped
    overlap = [(a, b) for a in range(len(sts)) for b in range(len(sts))
               if sts[a].admit_tick < sts[b].admit_tick < sts[a].finish_tick]
    assert overlap, [(s.admit_tick, s.finish_tick) for s in sts]
    assert any(s.inflight_at_admit >= 1 for s in sts)
    # requests of different sizes ran in different lanes
    assert len({s.lane for s in sts}) >= 2
    assert srv.close() == gbmg.OK


def test_server_failed_step_releases_handles(monkeypatch):
    """A failing step (injected on the host: the server's second step launch
    reports a CUDA error without launching anything) ends the admitted request
    with that error and destroys its hierarchy (no bytes left held); drain
    returns, and the server then serves the next request normally."""
    P = I.config2(32)
    f = oracle.faces_from_density(P.shape, P.bc, P.rho)
    fd, b = [dev(a) for a in f], dev(P.rhs)
    p = torch.zeros_like(b)
    torch.cuda.synchronize()
    monkeypatch.setenv("MG_SERVER_FAIL_AT_STEP", "2")
    srv = gbmg.Server(hbm_budget_bytes=1 << 30, max_slots=4)
    monkeypatch.delenv("MG_SERVER_FAIL_AT_STEP")
    t = srv.submit(P.shape, P.bc, fd, b, p, tol=TOL)  # a 32^3 solve takes more than 2 steps
    rc, _ = poll_all(srv, [t])[t]
    assert rc == gbmg.ECUDA, gbmg.strerror(rc)
    assert srv.drain() == gbmg.ECUDA  # the loop's error stays reported
    info = srv.info()
    assert info["bytes_in_use"] == 0 and info["completed"] == 1
    # the next request runs
    p.zero_()
    torch.cuda.synchronize()
    t = srv.submit(P.shape, P.bc, fd, b, p, tol=TOL)
    rc, st = poll_all(srv, [t])[t]
    assert rc == gbmg.OK
    check_against_oracle(P, f, p.cpu().numpy(), "served after failure")
    assert srv.info()["bytes_in_use"] == gbmg.memory_estimate(P.shape, P.bc)
    assert srv.close() == gbmg.OK


def test_tail_wait_timeout_reported_then_recovers():
    """The bottom-of-cycle kernel's bounded staging wait: with its limit at 0
    polls it gives up at once and the solve reports ETIMEOUT (the kernel lets
    its copies land before exiting); with the limit restored the same handle
    solves to the oracle's p*."""
    P = I.config2(32)
    f = oracle.faces_from_density(P.shape, P.bc, P.rho)
    fd = [dev(a) for a in f]
    with gbmg.Solver(P.shape, P.bc, faces=fd, precision=gbmg.MIXED) as S:
        assert S.num_levels() >= 3  # 32^3 -> 16^3 ... 2^3: the levels below 32^3 run in the tail kernel
        S.set_wait_limit(0)
        p = torch.zeros(cells(P.shape), dtype=torch.float64, device="cuda")
        st = S.solve(dev(P.rhs), p, tol=TOL, raise_on_error=False)
        assert st.status == gbmg.ETIMEOUT, gbmg.strerror(st.status)
        S.set_wait_limit(1 << 20)
        S.set_faces(*fd)  # clears the reported timeout
        p.zero_()
        st = S.solve(dev(P.rhs), p, tol=TOL)
        assert st.status == gbmg.OK and st.rel_res <= TOL
        check_against_oracle(P, f, p.cpu().numpy(), "after timeout")
