"""The flux-conserving prolongation (Sec. 2.3 item 4, Eqs. 13-14 of arXiv
1410.8568, MG_PROLONG_FLUX) through the C ABI, against the FP64 oracle.

The cell coefficients and single prolongation steps are compared element by
element with ``oracle.cell_alpha`` and ``oracle.prolong_flux_add``; whole solves
(with the bottom-of-cycle kernel, which prolongs in shared memory) are compared
with the oracle's p*, which does not depend on the prolongation.
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
    return I.Problem(shape, bc, rho, b, name="flux_%s_%s_%g" % (shape, bc, ratio), ratio=ratio)


def level_faces(shape, bc, faces, lvl):
    sh, fl = shape, faces
    for _ in range(lvl):
        fl = oracle.coarsen_faces(sh, bc, fl)
        sh = oracle.coarse_shape(sh)
    return sh, fl


@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 1, 0), (1, 0, 1)])
def test_cell_alpha_matches_oracle(bc):
    shape = (32, 48, 24)
    P = problem(shape, bc, 1000.0, 1)
    f = oracle.faces_from_density(shape, bc, P.rho)
    with gbmg.Solver(shape, bc, faces=[dev(a) for a in f], precision=gbmg.MIXED,
                     prolongation=gbmg.PROLONG_FLUX) as S:
        for lvl in range(S.num_levels()):
            sh, fl = level_faces(shape, bc, f, lvl)
            want = oracle.cell_alpha(sh, bc, fl)
            got = host(S.level_cell_alpha(lvl))
            np.testing.assert_allclose(got, want, rtol=1e-14, atol=0)


@pytest.mark.parametrize("shape", [(32, 48, 64), (40, 24, 12)])
@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 1, 0), (1, 1, 1)])
def test_flux_prolongation_matches_oracle(shape, bc):
    """mg_prolong of a flux handle against oracle.prolong_flux_add, on levels
    with quads (vector path) and with rows of 2 mod 4 cells (scalar path)."""
    P = problem(shape, bc, 1000.0, 6)
    f = oracle.faces_from_density(shape, bc, P.rho)
    rng = np.random.default_rng(7)
    with gbmg.Solver(shape, bc, faces=[dev(a) for a in f], precision=gbmg.MIXED,
                     prolongation=gbmg.PROLONG_FLUX) as S:
        for lvl in range(S.num_levels() - 1):
            sh, fl = level_faces(shape, bc, f, lvl)
            cs, cf = level_faces(sh, bc, fl, 1)
            ac = oracle.cell_alpha(cs, bc, cf)
            e = rng.standard_normal(cells(cs))
            x = rng.standard_normal(cells(sh))
            want = oracle.prolong_flux_add(sh, bc, ac, e, x)
            scale = np.abs(x).max() + np.abs(e).max()
            gx = dev(x)
            S.prolong(lvl, dev(e), gx, prec=gbmg.FP64)
            np.testing.assert_allclose(host(gx), want, rtol=0, atol=1e-14 * scale)
            gx32 = dev(x, torch.float32)
            S.prolong(lvl, dev(e, torch.float32), gx32, prec=gbmg.MIXED)
            np.testing.assert_allclose(host(gx32), want, rtol=0, atol=2e-6 * scale)


CASES = [
    ("sphere_32_ratio1000", lambda: I.config1(32)),
    ("dropfilm_64", lambda: I.config2(64)),
    ("ragged_64x48x32", lambda: problem((64, 48, 32), (1, 0, 1), 1000.0, 10)),
    ("sphere_24_ratio1e5", lambda: problem((24, 24, 24), (0, 0, 0), 1e5, 12)),
    ("periodic_48_ratio100", lambda: problem((48, 48, 48), (1, 1, 1), 100.0, 14)),
]


@pytest.mark.parametrize("precision", [gbmg.FP64, gbmg.MIXED])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_flux_solve_matches_oracle(name, make, precision):
    P = make()
    f = oracle.faces_from_density(P.shape, P.bc, P.rho)
    pstar = oracle.solve_exact(P.shape, P.bc, f, P.rhs).x
    with gbmg.Solver(P.shape, P.bc, faces=[dev(a) for a in f], precision=precision,
                     prolongation=gbmg.PROLONG_FLUX) as S:
        b = dev(P.rhs)
        p = torch.zeros_like(b)
        st = S.solve(b, p, tol=TOL)
        assert st.status == gbmg.OK and st.rel_res <= TOL
        x = host(p)
        bp = P.rhs - P.rhs.mean()
        rel = np.linalg.norm(oracle.residual(P.shape, P.bc, f, bp, x)) / np.linalg.norm(bp)
        err = np.linalg.norm(x - pstar) / np.linalg.norm(pstar)
        print("%s flux prec=%d iters=%d gamma=%.3f err=%.2e" % (name, precision, st.iters, st.gamma, err))
        assert rel <= 1.05 * TOL and err <= ERR


def test_flux_solve_bitwise_equal_across_shapes_and_graph():
    P = I.config2(64)
    f = [dev(a) for a in oracle.faces_from_density(P.shape, P.bc, P.rho)]
    b = dev(P.rhs)
    ref = None
    for tiles, graph in ((gbmg.TILES_AUTO, True), (0, True), (1, False), (4, True), (6, True)):
        with gbmg.Solver(P.shape, P.bc, faces=f, precision=gbmg.MIXED, prolongation=gbmg.PROLONG_FLUX,
                         tiles=tiles, use_graph=graph) as S:
            for lvl in range(S.num_levels()):
                assert S.tile_choice(gbmg.TILE_PROLONG, lvl) == 0  # flux prolongation: row tiles
            p = torch.zeros_like(b)
            st = S.solve(b, p, tol=TOL)
            assert st.status == gbmg.OK
            torch.cuda.synchronize()
            if ref is None:
                ref = p.clone()
            else:
                assert torch.equal(p, ref), tiles
