"""Conjugate gradients preconditioned by V-cycles (MG_SOLVER_PCG) through the C
ABI, against the FP64 oracle (oracle.pcg_solve and the converged p*).

The solution does not depend on the iteration, so whole solves are compared
with p* (relative L2 <= 1e-8 at a relative residual <= 1e-10, the residual
re-evaluated by the oracle's operator); iteration counts are compared with the
oracle's own PCG; graph = host loop and batch = alone hold bitwise.
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=torch.float64)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def problem(shape, bc, ratio, seed):
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.25, 0.75, size=3)
    rho = I.density_field(shape, None, [(tuple(c), 0.2)], ratio)
    b = rng.standard_normal(cells(shape))
    b -= b.mean()
    return I.Problem(shape, bc, rho, b, name="pcg_%s_%s_%g" % (shape, bc, ratio), ratio=ratio)


CASES = [
    ("sphere_32", lambda: I.config1(32)),
    ("dropfilm_64", lambda: I.config2(64)),
    ("ragged_64x48x32", lambda: problem((64, 48, 32), (1, 0, 1), 1000.0, 10)),
    ("sphere_24_ratio1e5", lambda: problem((24, 24, 24), (0, 0, 0), 1e5, 12)),
    ("periodic_48_ratio100", lambda: problem((48, 48, 48), (1, 1, 1), 100.0, 14)),
    ("single_level_8x8x2", lambda: problem((8, 8, 2), (0, 0, 0), 1000.0, 17)),
    ("odd_coarsest_6", lambda: problem((6, 6, 6), (1, 1, 1), 100.0, 18)),
]


@pytest.mark.parametrize("precision", [gbmg.FP64, gbmg.MIXED])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_pcg_solve_matches_oracle(name, make, precision):
    P = make()
    f = oracle.faces_from_density(P.shape, P.bc, P.rho)
    pstar = oracle.solve_exact(P.shape, P.bc, f, P.rhs).x
    ref = oracle.pcg_solve(P.shape, P.bc, f, P.rhs, tol=TOL)
    with gbmg.Solver(P.shape, P.bc, faces=[dev(a) for a in f], precision=precision, solver=gbmg.SOLVER_PCG) as S:
        assert S.resolved_params()["inner_cycles"] == 1
        b = dev(P.rhs)
        p = torch.zeros_like(b)
        st = S.solve(b, p, tol=TOL)
        assert st.status == gbmg.OK and st.rel_res <= TOL
        x = host(p)
        bp = P.rhs - P.rhs.mean()
        rel = np.linalg.norm(oracle.residual(P.shape, P.bc, f, bp, x)) / np.linalg.norm(bp)
        err = np.linalg.norm(x - pstar) / np.linalg.norm(pstar)
        print("%s pcg prec=%d iters=%d (oracle %d) gamma=%.3f rel=%.2e err=%.2e" %
              (name, precision, st.iters, ref.cycles, st.gamma, rel, err))
        assert rel <= 1.05 * TOL and err <= ERR
        assert abs(st.iters - ref.cycles) <= (1 if precision == gbmg.FP64 else 3)


def test_pcg_graph_host_loop_and_batch_bitwise():
    probs = [I.config2(48), problem((32, 64, 32), (0, 0, 0), 1000.0, 3), problem((24, 24, 24), (1, 1, 1), 10.0, 4)]
    faces = [[dev(a) for a in oracle.faces_from_density(P.shape, P.bc, P.rho)] for P in probs]
    rhs = [dev(P.rhs) for P in probs]
    alone = []
    for P, f, b in zip(probs, faces, rhs):
        res = []
        for graph in (True, False):
            with gbmg.Solver(P.shape, P.bc, faces=f, precision=gbmg.MIXED, solver=gbmg.SOLVER_PCG,
                             use_graph=graph) as S:
                p = torch.zeros_like(b)
                assert S.solve(b, p, tol=TOL).status == gbmg.OK
                torch.cuda.synchronize()
                res.append(p)
        assert torch.equal(res[0], res[1])
        alone.append(res[0])
    solvers = [gbmg.Solver(P.shape, P.bc, faces=f, precision=gbmg.MIXED, solver=gbmg.SOLVER_PCG)
               for P, f in zip(probs, faces)]
    B = gbmg.Batch(solvers)
    ps = [torch.zeros_like(b) for b in rhs]
    sts = B.solve(rhs, ps, tol=TOL)
    torch.cuda.synchronize()
    for st, p, a in zip(sts, ps, alone):
        assert st.status == gbmg.OK and torch.equal(p, a)
    B.close()
    for S in solvers:
        S.close()


def test_pcg_with_flux_prolongation():
    P = problem((32, 32, 32), (0, 0, 0), 1e5, 21)
    f = oracle.faces_from_density(P.shape, P.bc, P.rho)
    pstar = oracle.solve_exact(P.shape, P.bc, f, P.rhs).x
    with gbmg.Solver(P.shape, P.bc, faces=[dev(a) for a in f], precision=gbmg.MIXED, solver=gbmg.SOLVER_PCG,
                     prolongation=gbmg.PROLONG_FLUX) as S:
        p = torch.zeros(cells(P.shape), dtype=torch.float64, device="cuda")
        st = S.solve(dev(P.rhs), p, tol=TOL)
        assert st.status == gbmg.OK
        err = np.linalg.norm(host(p) - pstar) / np.linalg.norm(pstar)
        assert err <= ERR


def test_pcg_batch_refuses_mixed_solvers():
    P = I.config1(16)
    f = [dev(a) for a in oracle.faces_from_density(P.shape, P.bc, P.rho)]
    A = gbmg.Solver(P.shape, P.bc, faces=f, solver=gbmg.SOLVER_PCG)
    B = gbmg.Solver(P.shape, P.bc, faces=f, solver=gbmg.SOLVER_MG)
    with pytest.raises(gbmg.MGError):
        gbmg.Batch([A, B])
    A.close()
    B.close()
