"""The projection step around the solve (Sec. 2.2 of arXiv 1410.8568: Chorin's
projection on the MAC grid) through the C ABI, against the FP64 oracle.

Divergence and velocity update are compared element by element with
``oracle.divergence`` / ``oracle.project``; the whole step (divergence, solve,
update) is checked against the oracle's projection with p*, and the projected
field's divergence against dt times the solve's tolerance.
"""
import numpy as np
import pytest

import oracle
from paper_1410_8568_gb300 import gbmg
from paper_1410_8568_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def cells(shape):
    return (shape[2], shape[1], shape[0])


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=torch.float64)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 1, 0), (1, 0, 1), (1, 1, 1)])
def test_divergence_and_project_match_oracle(bc):
    shape, length = (40, 24, 12), (1.0, 0.6, 0.3)
    rng = np.random.default_rng(4)
    c = rng.uniform(0.3, 0.7, size=3)
    rho = I.density_field(shape, None, [(tuple(c), 0.2)], 1000.0)
    faces = oracle.faces_from_density(shape, bc, rho, length=length)
    u = [rng.standard_normal(cells(shape)) for _ in range(3)]
    p = rng.standard_normal(cells(shape))
    dt = 0.37
    with gbmg.Solver(shape, bc, faces=[dev(a) for a in faces], length=length, precision=gbmg.MIXED) as S:
        gS = torch.empty(cells(shape), dtype=torch.float64, device="cuda")
        S.divergence([dev(a) for a in u], dt, gS)
        want = oracle.divergence(shape, bc, u, dt=dt, length=length)
        np.testing.assert_allclose(host(gS), want, rtol=0, atol=1e-14 * np.abs(want).max())
        gu = [dev(a) for a in u]
        S.project(dev(p), dt, gu)
        wu = oracle.project(shape, bc, faces, p, u, dt=dt, length=length)
        for d in range(3):
            np.testing.assert_allclose(host(gu[d]), wu[d], rtol=0, atol=1e-13 * np.abs(wu[d]).max())


@pytest.mark.parametrize("precision", [gbmg.MIXED, gbmg.FP64])
@pytest.mark.parametrize("n", [32, 64])
def test_projection_step_matches_oracle(n, precision):
    shape, bc, rho, u, dt = I.projection_problem(n, ratio=1000.0, dt=1e-2)
    faces = oracle.faces_from_density(shape, bc, rho)
    Sw = oracle.divergence(shape, bc, u, dt=dt)
    pstar = oracle.solve_exact(shape, bc, faces, Sw).x
    uw = oracle.project(shape, bc, faces, pstar, u, dt=dt)
    tol = 1e-10
    with gbmg.Solver(shape, bc, rho=dev(rho), precision=precision) as S:
        gu = [dev(a) for a in u]
        gp = torch.zeros(cells(shape), dtype=torch.float64, device="cuda")
        gS = torch.empty_like(gp)
        st = S.projection_step(gu, dt, gp, gS, tol=tol)
        assert st.status == gbmg.OK and st.rel_res <= tol
        np.testing.assert_allclose(host(gS), Sw, rtol=0, atol=1e-13 * np.abs(Sw).max())
        err_p = np.linalg.norm(host(gp) - pstar) / np.linalg.norm(pstar)
        assert err_p <= 1e-8
        un = [host(a) for a in gu]
        # the projected field: divergence = dt x the solve's residual
        div = oracle.divergence(shape, bc, un, dt=1.0)
        assert np.linalg.norm(div) <= 1.05 * tol * np.linalg.norm(dt * (Sw - Sw.mean())) + 1e-12 * np.linalg.norm(dt * Sw)
        corr = np.sqrt(sum(np.sum((a - b) ** 2) for a, b in zip(u, uw)))
        diff = np.sqrt(sum(np.sum((a - b) ** 2) for a, b in zip(un, uw)))
        assert diff <= 1e-7 * corr
        assert np.all(un[2][0] == 0.0)  # Neumann walls keep zero normal velocity
