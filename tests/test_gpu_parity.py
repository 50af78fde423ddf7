"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Single kernels are compared element by element with the oracle function that
computes the same step; whole solves are compared with the oracle's converged
solution p* (relative L2 error <= 1e-8 at a relative residual <= 1e-10, with
the residual re-evaluated by the oracle's own operator).  Sec./Eq. numbers:
Shin, Chergui & Juric, arXiv 1410.8568.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1410_8568_gb300 import gbmg
from paper_1410_8568_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10       # relative residual of every solve
ERR = 1e-8        # relative L2 error against the oracle's p*


def cells(shape):
    return (shape[2], shape[1], shape[0])


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def solver_for(P, faces, precision=gbmg.MIXED, **kw):
    return gbmg.Solver(P.shape, P.bc, faces=[dev(f) for f in faces], length=P.length,
                       precision=precision, **kw)


def random_problem(shape, bc, ratio, seed):
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.25, 0.75, size=3)
    rho = I.density_field(shape, None, [(tuple(c), 0.2)], ratio)
    b = rng.standard_normal(cells(shape))
    b -= b.mean()
    return I.Problem(shape, bc, rho, b, name="random_%s_%s_%g" % (shape, bc, ratio), ratio=ratio)


# ---------------------------------------------------------------------------
# single kernels
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("make", [lambda: I.config1(16), lambda: I.config2(24)])
@pytest.mark.parametrize("mode", [0, 1])
def test_faces_from_density(make, mode):
    P = make()
    want = oracle.faces_from_density(P.shape, P.bc, P.rho, mode=mode)
    out = [torch.empty(cells(P.shape), dtype=torch.float64, device="cuda") for _ in range(3)]
    gbmg.faces_from_density(P.shape, P.bc, dev(P.rho), *out, mode=mode)
    for d in range(3):
        np.testing.assert_allclose(host(out[d]), want[d], rtol=2e-15, atol=0)


@pytest.mark.parametrize("mode", [0, 1])
def test_fp32_faces_are_rounded_fp64_faces(mode):
    """The FP32 faces of every level of a mixed handle (the set-up converts them
    with integer bit operations) equal the FP64 faces rounded to nearest, ties
    to even, bit for bit: faces given by the caller (values over 30 orders of
    magnitude and values exactly halfway between two floats; the scale 1/h^2
    is a power of 2, so the ties survive it, and the coarse faces, means of 4,
    make more), then faces from a density (harmonic or arithmetic mean)."""
    shape, bc = (32, 32, 64), (1, 0, 1)
    rng = np.random.default_rng(7)
    alpha = [10.0 ** rng.uniform(-15, 15, size=cells(shape)) for _ in range(3)]
    for a in alpha:
        a.flat[::7] = 1.0 + 2.0 ** -24        # tie: rounds down to even
        a.flat[3::7] = 1.0 + 3 * 2.0 ** -24   # tie: rounds up to even
        a.flat[5::11] = 2.0 ** -30 * (1.0 + 2.0 ** -24)
    rho = 10.0 ** rng.uniform(-15, 15, size=cells(shape))

    def check(S):
        for lvl in range(S.num_levels()):
            w64, w32 = S.level_faces(lvl), S.level_faces32(lvl)
            for d in range(3):
                assert torch.equal(w32[d], w64[d].float()), (lvl, d)

    with gbmg.Solver(shape, bc, faces=[dev(a) for a in alpha], precision=gbmg.MIXED) as S:
        check(S)
        S.set_density(dev(rho), mode=mode)
        check(S)


@pytest.mark.parametrize("shape,bc", [((32, 32, 32), (0, 0, 0)), ((48, 24, 96), (1, 1, 0)), ((64, 48, 32), (1, 0, 1))])
def test_level_faces_match_oracle_coarsening(shape, bc):
    P = random_problem(shape, bc, 1000.0, 1)
    f = oracle.faces_from_density(shape, bc, P.rho)
    with solver_for(P, f) as S:
        sh, fl = shape, f
        for lvl in range(S.num_levels()):
            assert S.level_shape(lvl) == sh
            got = S.level_faces(lvl)
            for d in range(3):
                h = 1.0 / sh[d]
                want = fl[d] / (h * h)
                if bc[d] == 0:
                    want = want.copy()
                    sl = [slice(None)] * 3
                    sl[2 - d] = 0
                    want[tuple(sl)] = 0.0
                np.testing.assert_allclose(host(got[d]), want, rtol=1e-14, atol=0)
            if lvl + 1 < S.num_levels():
                fl = oracle.coarsen_faces(sh, bc, fl)
                sh = oracle.coarse_shape(sh)


def _level_problem(S, P, faces, lvl):
    sh, fl = P.shape, faces
    for _ in range(lvl):
        fl = oracle.coarsen_faces(sh, P.bc, fl)
        sh = oracle.coarse_shape(sh)
    return sh, fl


@pytest.mark.parametrize("lvl", [0, 1, 2])
@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 1, 0), (1, 1, 1)])
def test_apply_matches_oracle(lvl, bc):
    P = random_problem((32, 48, 64), bc, 1000.0, 2)
    f = oracle.faces_from_density(P.shape, bc, P.rho)
    rng = np.random.default_rng(3)
    with solver_for(P, f, precision=gbmg.MIXED) as S:
        sh, fl = _level_problem(S, P, f, lvl)
        x = rng.standard_normal(cells(sh))
        want = oracle.apply(sh, bc, fl, x)
        scale = np.abs(want).max() + 6 * max(np.abs(a).max() * sh[d] ** 2 for d, a in enumerate(fl)) * np.abs(x).max()
        y = torch.empty(cells(sh), dtype=torch.float64, device="cuda")
        S.apply(lvl, dev(x), y, prec=gbmg.FP64)
        assert np.abs(host(y) - want).max() <= 1e-14 * scale
        y32 = torch.empty(cells(sh), dtype=torch.float32, device="cuda")
        S.apply(lvl, dev(x, torch.float32), y32, prec=gbmg.MIXED)
        assert np.abs(host(y32) - want).max() <= 2e-6 * scale


@pytest.mark.parametrize("shape", [(48, 32, 24), (40, 20, 12)])
@pytest.mark.parametrize("omega", [1.0, 1.3])
@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 1, 0), (1, 0, 1)])
def test_smoother_matches_oracle(shape, omega, bc):
    """Red-black sweeps (fused kernel, tiles ragged in x, y and z) against the oracle's half-sweeps."""
    P = random_problem(shape, bc, 1000.0, 4)
    f = oracle.faces_from_density(P.shape, bc, P.rho)
    rng = np.random.default_rng(5)
    b = rng.standard_normal(cells(P.shape))
    x0 = rng.standard_normal(cells(P.shape))
    with solver_for(P, f, omega=omega) as S:
        for lvl in (0, 1):
            sh, fl = _level_problem(S, P, f, lvl)
            bl = b[: sh[2], : sh[1], : sh[0]].copy()
            xl = x0[: sh[2], : sh[1], : sh[0]].copy()
            want = xl.copy()
            for sw in range(3):
                want = oracle.smooth_colour(sh, bc, fl, bl, want, 0, omega)
                want = oracle.smooth_colour(sh, bc, fl, bl, want, 1, omega)
                got = dev(xl)
                S.smooth(lvl, dev(bl), got, sw + 1, prec=gbmg.FP64)
                scale = np.abs(want).max() + np.abs(xl).max()
                assert np.abs(host(got) - want).max() <= 1e-13 * scale, (lvl, sw)
                got32 = dev(xl, torch.float32)
                S.smooth(lvl, dev(bl, torch.float32), got32, sw + 1, prec=gbmg.MIXED)
                assert np.abs(host(got32) - want).max() <= 1e-5 * scale, (lvl, sw)


@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 1, 0), (1, 1, 1)])
def test_restrict_residual_and_prolong_match_oracle(bc):
    P = random_problem((32, 48, 64), bc, 1000.0, 6)
    f = oracle.faces_from_density(P.shape, bc, P.rho)
    rng = np.random.default_rng(7)
    with solver_for(P, f) as S:
        for lvl in (0, 1):
            sh, fl = _level_problem(S, P, f, lvl)
            cs = oracle.coarse_shape(sh)
            b = rng.standard_normal(cells(sh))
            x = rng.standard_normal(cells(sh))
            r = oracle.residual(sh, bc, fl, b, x)
            want = oracle.restrict(sh, bc, r)
            cb = torch.empty(cells(cs), dtype=torch.float64, device="cuda")
            S.restrict_residual(lvl, dev(b), dev(x), cb, prec=gbmg.FP64)
            scale = np.abs(r).max() + 6 * max(np.abs(a).max() * sh[d] ** 2 for d, a in enumerate(fl)) * np.abs(x).max()
            assert np.abs(host(cb) - want).max() <= 1e-14 * scale
            cb32 = torch.empty(cells(cs), dtype=torch.float32, device="cuda")
            S.restrict_residual(lvl, dev(b, torch.float32), dev(x, torch.float32), cb32, prec=gbmg.MIXED)
            assert np.abs(host(cb32) - want).max() <= 2e-6 * scale
            e = rng.standard_normal(cells(cs))
            want_x = oracle.prolong_add(sh, bc, e, x)
            gx = dev(x)
            S.prolong(lvl, dev(e), gx, prec=gbmg.FP64)
            np.testing.assert_allclose(host(gx), want_x, rtol=0, atol=1e-14 * (np.abs(x).max() + np.abs(e).max()))
            gx32 = dev(x, torch.float32)
            S.prolong(lvl, dev(e, torch.float32), gx32, prec=gbmg.MIXED)
            np.testing.assert_allclose(host(gx32), want_x, rtol=0, atol=1e-6 * (np.abs(x).max() + np.abs(e).max()))


@pytest.mark.parametrize("shape,bc", [((32, 32, 32), (0, 0, 0)), ((48, 48, 48), (1, 1, 0)), ((64, 48, 32), (1, 1, 1)),
                                      ((4, 4, 4), (0, 1, 0)), ((6, 6, 6), (1, 1, 1)), ((40, 40, 40), (0, 0, 0))])
def test_coarse_solve_matches_oracle(shape, bc):
    P = random_problem(shape, bc, 1000.0, 8)
    f = oracle.faces_from_density(shape, bc, P.rho)
    with solver_for(P, f) as S:
        L = S.num_levels()
        sh, fl = _level_problem(S, P, f, L - 1)
        rng = np.random.default_rng(9)
        r = rng.standard_normal(cells(sh))
        want = oracle.coarse_solve(sh, bc, fl, r)  # zero-mean solution of A e = r - mean(r)
        e = torch.empty(cells(sh), dtype=torch.float64, device="cuda")
        S.coarse_solve(dev(r), e, prec=gbmg.FP64)
        got = host(e)
        got -= got.mean()
        assert np.linalg.norm(got - want) <= 1e-11 * np.linalg.norm(want)


# ---------------------------------------------------------------------------
# whole solves against the oracle's p*
# ---------------------------------------------------------------------------

CASES = [
    ("cfg1_sphere_32", lambda: I.config1(32)),
    ("cfg2_dropfilm_48", lambda: I.config2(48)),
    ("ragged_64x48x32_neumann_y", lambda: random_problem((64, 48, 32), (1, 0, 1), 1000.0, 10)),
    ("periodic_32_ratio10", lambda: random_problem((32, 32, 32), (1, 1, 1), 10.0, 11)),
    ("sphere_24_ratio1e5", lambda: random_problem((24, 24, 24), (0, 0, 0), 1e5, 12)),
    ("tiny_4", lambda: random_problem((4, 4, 4), (0, 0, 0), 1000.0, 13)),
    ("single_level_8x8x2", lambda: random_problem((8, 8, 2), (0, 0, 0), 1000.0, 17)),
    ("odd_coarsest_6_periodic", lambda: random_problem((6, 6, 6), (1, 1, 1), 100.0, 14)),
    ("two_cells_periodic", lambda: random_problem((2, 4, 2), (1, 1, 1), 1.0, 15)),
]

_exact_cache = {}


def exact_solution(name, P, faces):
    if name not in _exact_cache:
        _exact_cache[name] = oracle.solve_exact(P.shape, P.bc, faces, P.rhs, length=P.length).x
    return _exact_cache[name]


# (V-cycle precision, outer iteration): FP64 throughout; FP32 cycles in the FP64
# outer iteration; FP32 cycles in the extended-precision outer iteration
MODES = [(gbmg.FP64, gbmg.OUTER_FP64), (gbmg.MIXED, gbmg.OUTER_FP64), (gbmg.MIXED, gbmg.OUTER_XP)]
MODE_IDS = ["fp64", "mixed", "mixed_xp"]


@pytest.mark.parametrize("precision,outer", MODES, ids=MODE_IDS)
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_solve_matches_oracle(name, make, precision, outer):
    P = make()
    f = oracle.faces_from_density(P.shape, P.bc, P.rho)
    pstar = exact_solution(name, P, f)
    with solver_for(P, f, precision=precision, outer=outer) as S:
        b = dev(P.rhs)
        p = torch.zeros_like(b)
        st = S.solve(b, p, tol=TOL)
        assert st.status == gbmg.OK, (st.as_dict(), gbmg.strerror(st.status))
        assert st.rel_res <= TOL
        x = host(p)
        bp = P.rhs - P.rhs.mean()
        rel = np.linalg.norm(oracle.residual(P.shape, P.bc, f, bp, x)) / np.linalg.norm(bp)
        err = np.linalg.norm(x - pstar) / np.linalg.norm(pstar)
        print("%s prec=%d iters=%d gamma=%.3f rel_res=%.2e (oracle %.2e) err=%.2e" %
              (name, precision, st.iters, st.gamma, st.rel_res, rel, err))
        assert rel <= 1.05 * TOL
        assert err <= ERR
        assert abs(x.mean()) <= 1e-13 * np.abs(x).max()


def test_graph_and_host_loop_are_bitwise_equal():
    P = I.config2(48)
    f = oracle.faces_from_density(P.shape, P.bc, P.rho)
    out = []
    for use_graph in (True, False):
        with solver_for(P, f, use_graph=use_graph) as S:
            p = torch.zeros(cells(P.shape), dtype=torch.float64, device="cuda")
            st = S.solve(dev(P.rhs), p, tol=TOL)
            out.append((host(p), st.iters, st.rel_res))
            # a second solve on the same handle repeats bit for bit
            p2 = torch.zeros_like(p)
            st2 = S.solve(dev(P.rhs), p2, tol=TOL)
            assert torch.equal(p, p2) and st2.iters == st.iters
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1] and out[0][2] == out[1][2]


@pytest.mark.parametrize("outer", [gbmg.OUTER_FP64, gbmg.OUTER_XP], ids=["fp64_outer", "xp_outer"])
def test_batch_is_bitwise_equal_to_alone(outer):
    probs = I.config4_batch(6, edges=(32, 48, 64))
    faces = [oracle.faces_from_density(P.shape, P.bc, P.rho) for P in probs]
    alone = []
    for P, f in zip(probs, faces):
        with solver_for(P, f, outer=outer) as S:
            p = torch.zeros(cells(P.shape), dtype=torch.float64, device="cuda")
            st = S.solve(dev(P.rhs), p, tol=TOL)
            assert st.status == gbmg.OK
            alone.append((p, st.iters))
    solvers = [solver_for(P, f, outer=outer) for P, f in zip(probs, faces)]
    B = gbmg.Batch(solvers)
    rhs = [dev(P.rhs) for P in probs]
    ps = [torch.zeros_like(r) for r in rhs]
    sts = B.solve(rhs, ps, tol=TOL)
    for (pa, ia), pb, st in zip(alone, ps, sts):
        assert st.status == gbmg.OK and st.iters == ia
        assert torch.equal(pa, pb)
    B.close()
    for S in solvers:
        S.close()


def test_edge_cases():
    P = I.config1(16)
    f = oracle.faces_from_density(P.shape, P.bc, P.rho)
    with solver_for(P, f, max_iters=50) as S:
        zero = torch.zeros(cells(P.shape), dtype=torch.float64, device="cuda")
        p = torch.full_like(zero, 7.0)
        st = S.solve(zero, p)
        assert st.status == gbmg.OK and st.iters == 0 and torch.count_nonzero(p) == 0
        # a right-hand side with non-zero mean: the mean is removed and reported
        b = dev(P.rhs)
        p1 = torch.zeros_like(b)
        S.solve(b, p1)
        p2 = torch.zeros_like(b)
        st2 = S.solve(b + 3.0, p2)
        assert abs(st2.rhs_mean - 3.0) < 1e-12
        assert torch.allclose(p1, p2, rtol=0, atol=1e-9 * p1.abs().max().item())
        # warm start at the solution: no cycle needed, result kept (mean removed)
        p3 = p1.clone()
        st3 = S.solve(b, p3)
        assert st3.iters == 0 and st3.status == gbmg.OK
        # NaN in the right-hand side: diverged, reported, no exception
        bn = b.clone()
        bn[3, 4, 5] = float("nan")
        st4 = S.solve(bn, torch.zeros_like(b))
        assert st4.status == gbmg.EDIVERGED
        # the handle is still usable afterwards
        p5 = torch.zeros_like(b)
        assert S.solve(b, p5).status == gbmg.OK and torch.equal(p5, p1)
    for max_iters, inner in ((2, 2), (2, 3), (4, 3), (1, 1), (5, 2)):
        with solver_for(P, f, max_iters=max_iters, inner_cycles=inner) as S:
            st = S.solve(dev(P.rhs), torch.zeros(cells(P.shape), dtype=torch.float64, device="cuda"))
            # the last refinement step is cut to the cycles left: exactly max_iters
            assert st.status == gbmg.ENOTCONV and st.iters == max_iters
    # invalid coefficients and sizes are refused
    bad = [a.copy() for a in f]
    bad[0][5, 5, 5] = -1.0
    with pytest.raises(gbmg.MGError) as e:
        solver_for(P, bad)
    assert e.value.code == gbmg.EINVAL
    with pytest.raises(gbmg.MGError):  # coarsest grid above MG_MAX_COARSE_GMRES cells
        gbmg.Solver((2, 2, 16384), (0, 0, 0), faces=[torch.ones(2 * 2 * 16384, dtype=torch.float64, device="cuda")] * 3)


def test_host_entry_points_match_device_path():
    P = I.config2(32)
    f = oracle.faces_from_density(P.shape, P.bc, P.rho)
    with solver_for(P, f) as S:
        p = torch.zeros(cells(P.shape), dtype=torch.float64, device="cuda")
        st = S.solve(dev(P.rhs), p)
        ph = np.zeros(cells(P.shape))
        sth = S.solve_host(np.ascontiguousarray(P.rhs), ph)
        assert sth.iters == st.iters and np.array_equal(ph, host(p))
        # density given on the host: faces built on the device (Eqs. 11-12)
        ps = np.zeros(cells(P.shape))
        sts = S.step_host(np.ascontiguousarray(P.rho), np.ascontiguousarray(P.rhs), ps)
        assert sts.status == gbmg.OK and sts.iters == st.iters
        np.testing.assert_allclose(ps, ph, rtol=0, atol=1e-12 * np.abs(ph).max())


def test_profiling_counts_launches():
    P = I.config1(32)
    f = oracle.faces_from_density(P.shape, P.bc, P.rho)
    with solver_for(P, f) as S:
        S.profile(True)
        p = torch.zeros(cells(P.shape), dtype=torch.float64, device="cuda")
        st = S.solve(dev(P.rhs), p)
        # one launch per colour of each of the nu1 + nu2 sweeps per V-cycle on the finest level
        n, ms = S.profile_read(gbmg.K_SMOOTH, 0)
        assert n == st.iters * 2 * (2 + 2) and ms > 0.0
        # one FP64 residual per refinement step (at most inner_cycles V-cycles
        # each), and the starting one counted apart
        inner = S.resolved_params()["inner_cycles"]
        assert inner == 6  # the mixed-precision default
        n, ms = S.profile_read(gbmg.K_RESIDUAL, 0)
        assert st.steps >= -(-st.iters // inner)
        assert n == st.steps and ms > 0.0
        n, ms = S.profile_read(gbmg.K_RESIDUAL0, 0)
        assert n == 1 and ms > 0.0


# ---------------------------------------------------------------------------
# full sizes: closed-form solutions and the oracle's residual
# ---------------------------------------------------------------------------

def test_full_size_drop_film_128():
    P = I.config2(128)
    f = oracle.faces_from_density(P.shape, P.bc, P.rho)
    pstar = oracle.solve_exact(P.shape, P.bc, f, P.rhs).x
    bp = P.rhs - P.rhs.mean()
    for (precision, outer), mid in zip(MODES, MODE_IDS):
        with solver_for(P, f, precision=precision, outer=outer) as S:
            p = torch.zeros(cells(P.shape), dtype=torch.float64, device="cuda")
            st = S.solve(dev(P.rhs), p, tol=TOL)
            assert st.status == gbmg.OK
            x = host(p)
            rel = np.linalg.norm(oracle.residual(P.shape, P.bc, f, bp, x)) / np.linalg.norm(bp)
            err = np.linalg.norm(x - pstar) / np.linalg.norm(pstar)
            print("128^3 drop/film %s iters=%d gamma=%.3f rel=%.2e err=%.2e" % (mid, st.iters, st.gamma, rel, err))
            assert rel <= 1.05 * TOL and err <= ERR


def test_full_size_drop_film_droplets_512():
    """The 512^3 drop/film field with its seeded droplets (density ratio 1000,
    periodic x and y, walls in z) against the oracle's p* in every mode, at
    the size whose error the benchmark reports; the solver takes the density
    on the device (faces of Eqs. 11-12 built there) and the oracle builds its
    own faces from the same density."""
    P = I.config3(512)
    f = oracle.faces_from_density(P.shape, P.bc, P.rho)
    pstar = oracle.solve_exact(P.shape, P.bc, f, P.rhs).x
    bp = P.rhs - P.rhs.mean()
    rho = dev(P.rho)
    b = dev(P.rhs)
    del f
    for (precision, outer), mid in zip(MODES, MODE_IDS):
        with gbmg.Solver(P.shape, P.bc, rho=rho, precision=precision, outer=outer) as S:
            p = torch.zeros_like(b)
            st = S.solve(b, p, tol=TOL)
            assert st.status == gbmg.OK and st.rel_res <= TOL
            x = host(p)
            del p
        err = np.linalg.norm(x - pstar) / np.linalg.norm(pstar)
        print("512^3 drop/film + droplets %s iters=%d gamma=%.3f rel_res=%.2e err=%.2e" %
              (mid, st.iters, st.gamma, st.rel_res, err))
        assert err <= ERR
        assert abs(x.mean()) <= 1e-13 * np.abs(x).max()


def _mode(n, k, bcv, device):
    i = torch.arange(n, dtype=torch.float64, device=device) + 0.5
    if bcv == 0:
        return torch.cos(math.pi * k * i / n), 4.0 * math.sin(math.pi * k / (2 * n)) ** 2
    return torch.cos(2 * math.pi * k * i / n), 4.0 * math.sin(math.pi * k / n) ** 2


@pytest.mark.parametrize("n,bc", [(512, (1, 1, 0)), (384, (0, 0, 0)), (1024, (1, 1, 0))])
def test_full_size_discrete_eigenvector(n, bc):
    """alpha = 1: b = lambda v has the exact solution v (discrete cosine mode)."""
    shape = (n, n, n)
    ones = torch.ones(cells(shape), dtype=torch.float64, device="cuda")
    vs, lam = [], 0.0
    for d, k in enumerate((3, 1, 2)):
        v, mu = _mode(n, k, bc[d], "cuda")
        vs.append(v)
        lam -= mu * n * n
    v = vs[2][:, None, None] * vs[1][None, :, None] * vs[0][None, None, :]
    b = (lam * v).contiguous()
    with gbmg.Solver(shape, bc, faces=[ones, ones, ones], precision=gbmg.MIXED) as S:
        p = torch.zeros_like(b)
        st = S.solve(b, p, tol=TOL)
        assert st.status == gbmg.OK
        err = (torch.linalg.vector_norm(p - v) / torch.linalg.vector_norm(v)).item()
        print("eigenvector %d^3 bc=%s iters=%d err=%.2e" % (n, bc, st.iters, err))
        assert err <= ERR


def test_full_size_layered_density_512():
    """Film-only density rho(z), 1000:1: one Fourier mode in x, y reduces the
    solve to a tridiagonal system in z (exact solution)."""
    import scipy.linalg
    n = 512
    shape = (n, n, n)
    rho_z = I.density_field((1, 1, n), 0.3, [], 1000.0, length=(1.0, 1.0, 1.0))[:, 0, 0]
    h = 1.0 / n
    kx, ky = 3, 2
    lam_xy = -(4 / h ** 2) * (math.sin(math.pi * kx / n) ** 2 + math.sin(math.pi * ky / n) ** 2)
    az = np.zeros(n + 1)
    az[1:n] = 2.0 / (rho_z[:-1] + rho_z[1:])
    ab = np.zeros((3, n))
    ab[1] = lam_xy / rho_z - (az[:n] + az[1:]) / h ** 2
    ab[0, 1:] = az[1:n] / h ** 2
    ab[2, :-1] = az[1:n] / h ** 2
    g = np.random.default_rng(16).standard_normal(n)
    fz = scipy.linalg.solve_banded((1, 1), ab, g)
    mx = torch.cos(2 * math.pi * kx * (torch.arange(n, dtype=torch.float64, device="cuda") + 0.5) / n)
    my = torch.cos(2 * math.pi * ky * (torch.arange(n, dtype=torch.float64, device="cuda") + 0.5) / n)
    mode = my[:, None] * mx[None, :]
    p_exact = (mode[None] * dev(fz)[:, None, None]).contiguous()
    b = (mode[None] * dev(g)[:, None, None]).contiguous()
    del mode
    rho = dev(rho_z)[:, None, None].expand(n, n, n).contiguous()
    for outer in (gbmg.OUTER_FP64, gbmg.OUTER_XP):
        with gbmg.Solver(shape, I.DROP_FILM_BC, rho=rho, precision=gbmg.MIXED, outer=outer) as S:
            p = torch.zeros_like(b)
            st = S.solve(b, p, tol=TOL)
            assert st.status == gbmg.OK
            err = (torch.linalg.vector_norm(p - p_exact) / torch.linalg.vector_norm(p_exact)).item()
            print("layered 512^3 outer=%d iters=%d gamma=%.3f err=%.2e" % (outer, st.iters, st.gamma, err))
            assert err <= ERR
            del p


@pytest.mark.parametrize("precision", [gbmg.MIXED, gbmg.FP64])
def test_adaptive_cycles_per_step(precision):
    """Adaptive steps stop with fewer or as many V-cycles as fixed ones, at the
    same tolerance, and give the same solution to the oracle's accuracy."""
    P = I.config2(64)
    f = oracle.faces_from_density(P.shape, P.bc, P.rho)
    pstar = exact_solution("cfg2_dropfilm_64", P, f)
    res = {}
    for adaptive in (0, 1):
        with solver_for(P, f, precision=precision, adaptive_cycles=adaptive) as S:
            inner = S.resolved_params()["inner_cycles"]
            p = torch.zeros(cells(P.shape), dtype=torch.float64, device="cuda")
            st = S.solve(dev(P.rhs), p, tol=TOL)
            assert st.status == gbmg.OK and st.rel_res <= TOL
            err = np.linalg.norm(host(p) - pstar) / np.linalg.norm(pstar)
            assert err <= ERR
            res[adaptive] = st
    assert res[0].iters % inner == 0 or res[0].iters == 100
    assert res[1].iters <= res[0].iters
    print("fixed %d cycles / %d steps, adaptive %d cycles / %d steps" %
          (res[0].iters, res[0].steps, res[1].iters, res[1].steps))


@pytest.mark.parametrize("precision,outer", MODES, ids=MODE_IDS)
def test_scaled_rhs_and_offset_iterate(precision, outer):
    """The outer iteration is invariant to the scale of the problem and to a
    constant in the iterate.  A right-hand side scaled by 2^+-100 gives the
    scaled solution bit for bit (the multigrid iteration runs on a copy scaled
    by a power of two taken from the right-hand side, so the FP32 cycles see
    the same numbers); a scale of 1e-30 or 1e30 gives the scaled solution to
    1e-8; a warm start carrying a constant converges to the same zero-mean
    solution: 1e4 times the solution's size for the three-float iterate of the
    extended-precision outer iteration, 10 times for the FP64 iterate (each
    FP64 update rounds at 2^-53 of the constant, which at 1e4 leaves a residual
    near 1e-9 of the right-hand side)."""
    P = I.config2(48)
    f = oracle.faces_from_density(P.shape, P.bc, P.rho)
    pstar = exact_solution("cfg2_dropfilm_48", P, f)
    with solver_for(P, f, precision=precision, outer=outer) as S:
        b = dev(P.rhs)
        p = torch.zeros_like(b)
        st = S.solve(b, p, tol=TOL)
        assert st.status == gbmg.OK
        for m in (-100, 100):
            s = math.ldexp(1.0, m)
            ps = torch.zeros_like(b)
            sts = S.solve(b * s, ps, tol=TOL)
            assert sts.status == gbmg.OK and sts.iters == st.iters
            assert torch.equal(ps, p * s)
        for s in (1e-30, 1e30):
            ps = torch.zeros_like(b)
            sts = S.solve(b * s, ps, tol=TOL)
            assert sts.status == gbmg.OK and sts.rel_res <= TOL
            err = np.linalg.norm(host(ps) / s - pstar) / np.linalg.norm(pstar)
            assert err <= ERR, (s, err)
        c = (1e4 if outer == gbmg.OUTER_XP else 10.0) * np.abs(pstar).max()
        po = torch.full_like(b, c)
        sto = S.solve(b, po, tol=TOL)
        assert sto.status == gbmg.OK
        x = host(po)
        bp = P.rhs - P.rhs.mean()
        rel = np.linalg.norm(oracle.residual(P.shape, P.bc, f, bp, x)) / np.linalg.norm(bp)
        err = np.linalg.norm(x - pstar) / np.linalg.norm(pstar)
        print("offset warm start: iters=%d rel_res=%.2e (oracle %.2e) err=%.2e" % (sto.iters, sto.rel_res, rel, err))
        assert rel <= 1.05 * TOL and err <= ERR


@pytest.mark.parametrize("precision,outer", MODES, ids=MODE_IDS)
def test_zero_start_shortcut(precision, outer):
    """A starting iterate that is zero in every cell gives the starting residual
    b - mean b without evaluating A p (the product is exactly zero there).  An
    iterate of -0.0 everywhere is zero too: the same solve, bit for bit.  One
    nonzero cell takes the full residual: the starting residual norm the solver
    reports is that of b - mean b - A p (oracle operator), not that of
    b - mean b, and the solve still reaches p*."""
    P = I.config2(40)
    f = oracle.faces_from_density(P.shape, P.bc, P.rho)
    pstar = exact_solution("cfg2_dropfilm_40", P, f)
    bp = P.rhs - P.rhs.mean()
    with solver_for(P, f, precision=precision, outer=outer) as S:
        b = dev(P.rhs)
        p = torch.zeros_like(b)
        st = S.solve(b, p, tol=TOL)
        assert st.status == gbmg.OK
        assert st.res0 == pytest.approx(np.linalg.norm(bp), rel=1e-6)
        pm = torch.full_like(b, -0.0)
        stm = S.solve(b, pm, tol=TOL)
        assert stm.iters == st.iters and stm.res0 == st.res0 and torch.equal(pm, p)
        d = np.zeros(cells(P.shape))
        d[17, 5, 23] = 10.0 * np.abs(pstar).max()
        pd = dev(d)
        std = S.solve(b, pd, tol=TOL)
        assert std.status == gbmg.OK and std.rel_res <= TOL
        r0 = np.linalg.norm(oracle.residual(P.shape, P.bc, f, bp, d))
        assert abs(r0 / np.linalg.norm(bp) - 1.0) > 0.1
        assert std.res0 == pytest.approx(r0, rel=1e-6)
        err = np.linalg.norm(host(pd) - pstar) / np.linalg.norm(pstar)
        print("single-cell start: iters=%d res0=%.6e (oracle %.6e) err=%.2e" % (std.iters, std.res0, r0, err))
        assert err <= ERR
