"""Restarted GMRES on the coarsest grid (Sec. 2.3 item 6 of arXiv 1410.8568)
through the C ABI, against the FP64 oracle.

Coarsest grids above 512 cells (sizes with a large odd factor) are solved by
GMRES instead of the dense inverse; MG_COARSE_GMRES forces it on any size.
The single coarse solve is compared with the oracle's exact coarse solve within
the GMRES tolerance, whole solves with the oracle's p*.
"""
import numpy as np
import pytest

import oracle
from paper_1410_8568_gb300 import gbmg
from paper_1410_8568_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL, ERR = 1e-10, 1e-8


def cells(shape):
    return (shape[2], shape[1], shape[0])


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def problem(shape, bc, ratio, seed):
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.25, 0.75, size=3)
    rho = I.density_field(shape, None, [(tuple(c), 0.2)], ratio)
    b = rng.standard_normal(cells(shape))
    b -= b.mean()
    return I.Problem(shape, bc, rho, b, name="gmres_%s_%s_%g" % (shape, bc, ratio), ratio=ratio)


def coarsest(S):
    lvl = S.num_levels() - 1
    return lvl, S.level_shape(lvl)


@pytest.mark.parametrize("shape,bc,forced", [((36, 36, 36), (0, 0, 0), False), ((28, 44, 36), (1, 0, 1), False),
                                             ((32, 32, 32), (1, 1, 0), True), ((9, 9, 9), (1, 1, 1), False)])
def test_gmres_coarse_solve_matches_oracle(shape, bc, forced):
    P = problem(shape, bc, 1000.0, 3)
    f = oracle.faces_from_density(shape, bc, P.rho)
    kw = dict(coarse_solver=gbmg.COARSE_GMRES, coarse_tol=1e-12, coarse_max_iters=3000) if forced else \
        dict(coarse_tol=1e-12, coarse_max_iters=3000)
    with gbmg.Solver(shape, bc, faces=[dev(a) for a in f], precision=gbmg.FP64, **kw) as S:
        lvl, cs = coarsest(S)
        assert forced or np.prod(cs) > gbmg.MAX_COARSE
        fl = f
        sh = shape
        for _ in range(lvl):
            fl = oracle.coarsen_faces(sh, bc, fl)
            sh = oracle.coarse_shape(sh)
        r = np.random.default_rng(9).standard_normal(cells(cs))
        want = oracle.coarse_solve(cs, bc, fl, r) if np.prod(cs) <= 512 else \
            oracle.gmres(cs, bc, fl, r, tol=1e-13, max_it=5000, m=50)[0]
        e = torch.empty(cells(cs), dtype=torch.float64, device="cuda")
        S.coarse_solve(dev(r), e, prec=gbmg.FP64)
        np.testing.assert_allclose(host(e), want, rtol=0, atol=1e-9 * np.abs(want).max())


CASES = [
    ("odd_coarsest_36", lambda: problem((36, 36, 36), (0, 0, 0), 1000.0, 10)),
    ("odd_coarsest_28x44x36", lambda: problem((28, 44, 36), (1, 0, 1), 1000.0, 11)),
    ("single_level_9", lambda: problem((9, 9, 9), (1, 1, 1), 100.0, 12)),
    ("forced_gmres_dropfilm_48", lambda: I.config2(48)),
]


@pytest.mark.parametrize("solver", [gbmg.SOLVER_MG, gbmg.SOLVER_PCG])
@pytest.mark.parametrize("precision", [gbmg.FP64, gbmg.MIXED])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_solve_with_gmres_coarsest_matches_oracle(name, make, precision, solver):
    P = make()
    f = oracle.faces_from_density(P.shape, P.bc, P.rho)
    pstar = oracle.solve_exact(P.shape, P.bc, f, P.rhs).x
    kw = dict(coarse_solver=gbmg.COARSE_GMRES) if name.startswith("forced") else {}
    with gbmg.Solver(P.shape, P.bc, faces=[dev(a) for a in f], precision=precision, solver=solver, **kw) as S:
        p = torch.zeros(cells(P.shape), dtype=torch.float64, device="cuda")
        st = S.solve(dev(P.rhs), p, tol=TOL)
        assert st.status == gbmg.OK and st.rel_res <= TOL
        x = host(p)
        bp = P.rhs - P.rhs.mean()
        rel = np.linalg.norm(oracle.residual(P.shape, P.bc, f, bp, x)) / np.linalg.norm(bp)
        err = np.linalg.norm(x - pstar) / np.linalg.norm(pstar)
        print("%s solver=%d prec=%d iters=%d gamma=%.3f err=%.2e" % (name, solver, precision, st.iters, st.gamma, err))
        assert rel <= 1.05 * TOL and err <= ERR


def test_gmres_batch_with_dense_grids_bitwise():
    """A batch mixing GMRES and dense coarsest grids: each result as alone."""
    probs = [problem((36, 36, 36), (0, 0, 0), 1000.0, 20), I.config2(32)]
    faces = [[dev(a) for a in oracle.faces_from_density(P.shape, P.bc, P.rho)] for P in probs]
    rhs = [dev(P.rhs) for P in probs]
    alone = []
    for P, f, b in zip(probs, faces, rhs):
        with gbmg.Solver(P.shape, P.bc, faces=f, precision=gbmg.MIXED) as S:
            p = torch.zeros_like(b)
            assert S.solve(b, p, tol=TOL).status == gbmg.OK
            torch.cuda.synchronize()
            alone.append(p)
    solvers = [gbmg.Solver(P.shape, P.bc, faces=f, precision=gbmg.MIXED) for P, f in zip(probs, faces)]
    B = gbmg.Batch(solvers)
    ps = [torch.zeros_like(b) for b in rhs]
    sts = B.solve(rhs, ps, tol=TOL)
    torch.cuda.synchronize()
    for st, p, a in zip(sts, ps, alone):
        assert st.status == gbmg.OK and torch.equal(p, a)
    B.close()
    for S in solvers:
        S.close()
