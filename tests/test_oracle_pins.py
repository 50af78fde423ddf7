"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself.  Each test checks one function
of ``oracle/`` against an independent fact: a hand-worked value of Eqs. 11-12,
a closed-form discrete solution, an exact operator identity, a dense direct
solve, or a property that a plausible mistake (dropped term, wrong sign,
shifted index, transposed axis) would break.  Sec./Eq. numbers refer to Shin,
Chergui & Juric, arXiv 1410.8568.
"""
import math
from fractions import Fraction
import os

import numpy as np
import pytest

import oracle
from paper_1410_8568_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
BCS = [(0, 0, 0), (1, 1, 0), (1, 1, 1), (0, 1, 0)]


def cells(shape):
    return (shape[2], shape[1], shape[0])


def ones_faces(shape):
    return [np.ones(cells(shape)) for _ in range(3)]


def coords(shape, length=(1.0, 1.0, 1.0)):
    """Cell-centre coordinates broadcast to (nz, ny, nx)."""
    nx, ny, nz = shape
    x = (np.arange(nx) + 0.5) * length[0] / nx
    y = (np.arange(ny) + 0.5) * length[1] / ny
    z = (np.arange(nz) + 0.5) * length[2] / nz
    return np.meshgrid(z, y, x, indexing="ij")[::-1]  # X, Y, Z


# ---------------------------------------------------------------------------
# Eqs. 11-12: harmonic face coefficient (golden values worked by hand)
# ---------------------------------------------------------------------------

def load_harmonic_golden():
    rows = []
    with open(os.path.join(GOLDEN, "harmonic_faces.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([float(v) for v in line.split()])
    return rows


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("bcv", [0, 1])
def test_faces_from_density_golden(axis, bcv):
    rows = load_harmonic_golden()
    assert len(rows) >= 6
    for rho_l, rho_r, harm, arith in rows:
        shape = [2, 2, 2]
        shape[axis] = 4
        shape = tuple(shape)
        bc = [0, 0, 0]
        bc[axis] = bcv
        X = np.zeros(cells(shape), dtype=int)
        # coordinate along `axis`: cells 0,1 carry rho_l and 2,3 carry rho_r
        idx = np.indices(cells(shape))[2 - axis]
        rho = np.where(idx < 2, rho_l, rho_r).astype(np.float64)
        for mode, want in ((0, harm), (1, arith)):
            f = oracle.faces_from_density(shape, bc, rho, mode=mode)[axis]
            face_between = np.take(f, 2, axis=2 - axis)  # low face of coordinate 2
            assert np.allclose(face_between, want, rtol=2e-16 * 8, atol=0)
            same_l = np.take(f, 1, axis=2 - axis)
            assert np.allclose(same_l, 1.0 / rho_l, rtol=1e-15, atol=0)
            wall = np.take(f, 0, axis=2 - axis)
            if bcv == 0:
                assert np.all(wall == 0.0)
            else:  # periodic wrap face between coordinate 3 (rho_r) and 0 (rho_l)
                assert np.allclose(wall, want, rtol=1e-15, atol=0)
        del X


# ---------------------------------------------------------------------------
# Eq. 10 operator: exact identities and closed forms
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("bc", BCS)
def test_operator_constant_nullspace_and_conservation(bc):
    rng = np.random.default_rng(1)
    shape = (8, 6, 4)
    f = I.random_faces(shape, rng, 1e-3, 1.0)
    A1 = oracle.apply(shape, bc, f, np.ones(cells(shape)))
    assert np.max(np.abs(A1)) == 0.0
    p = rng.standard_normal(cells(shape))
    Ap = oracle.apply(shape, bc, f, p)
    # flux telescoping: every interior face adds +w(p_nb - p_c) to one cell and the negative to the other
    assert abs(Ap.sum()) <= 1e-11 * np.abs(Ap).sum()


def dense_matrix(shape, bc, faces, length=(1.0, 1.0, 1.0)):
    n = int(np.prod(shape))
    A = np.empty((n, n))
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        A[:, c] = oracle.apply(shape, bc, faces, e.reshape(cells(shape)), length).ravel()
    return A


@pytest.mark.parametrize("bc", BCS)
def test_operator_symmetric_negative_semidefinite(bc):
    rng = np.random.default_rng(2)
    shape = (4, 6, 4)
    f = I.random_faces(shape, rng, 1e-5, 1.0)
    A = dense_matrix(shape, bc, f, length=(1.0, 1.5, 0.5))
    assert np.allclose(A, A.T, rtol=0, atol=1e-13 * np.abs(A).max())
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev.max() <= 1e-12 * np.abs(ev).max()
    # the null space is exactly the constants: one zero eigenvalue
    assert np.sum(np.abs(ev) <= 1e-10 * np.abs(ev).max()) == 1


def mode_1d(n, k, bcv):
    i = np.arange(n) + 0.5
    if bcv == 0:  # Neumann: cos(pi k (i+1/2)/n), eigenvalue -(4/h^2) sin^2(pi k / 2n)
        return np.cos(math.pi * k * i / n), 4.0 * math.sin(math.pi * k / (2 * n)) ** 2
    return np.cos(2 * math.pi * k * i / n), 4.0 * math.sin(math.pi * k / n) ** 2


def eigen_mode(shape, bc, kvec, length=(1.0, 1.0, 1.0)):
    vs, lam = [], 0.0
    for d in range(3):
        v, mu = mode_1d(shape[d], kvec[d], bc[d])
        h = length[d] / shape[d]
        vs.append(v)
        lam -= mu / h ** 2
    field = vs[2][:, None, None] * vs[1][None, :, None] * vs[0][None, None, :]
    return field, lam


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("shape,kvec", [((8, 8, 8), (1, 2, 3)), ((16, 8, 12), (3, 1, 2)), ((6, 12, 4), (2, 5, 1))])
def test_operator_discrete_eigenvectors(bc, shape, kvec):
    length = (1.0, 2.0, 0.75)
    v, lam = eigen_mode(shape, bc, kvec, length)
    Av = oracle.apply(shape, bc, ones_faces(shape), v, length)
    assert np.allclose(Av, lam * v, rtol=0, atol=1e-12 * abs(lam))


def flux_solution_nonperiodic(alpha, h, s):
    """Layered coefficients along one Neumann axis, +s on the first plane and -s
    on the last: the flux g_i (p_i - p_{i-1}) = s is the same through every
    interior face, so p_i - p_{i-1} = s h^2 / alpha_i (alpha_i = low face of i)."""
    n = len(alpha)
    p = np.zeros(n)
    for i in range(1, n):
        p[i] = p[i - 1] + s * h * h / alpha[i]
    return p - p.mean()


def flux_solution_periodic(alpha, h, s, m):
    """Ring of n planes, +s on plane 0, -s on plane m: the flux splits over the
    two paths in inverse proportion to their series resistance."""
    n = len(alpha)
    g = alpha / h ** 2
    RA = sum(1.0 / g[i] for i in range(1, m + 1))
    RB = 1.0 / g[0] + sum(1.0 / g[i] for i in range(m + 1, n))
    dP = s / (1.0 / RA + 1.0 / RB)
    FA, FB = dP / RA, dP / RB
    p = np.zeros(n)
    for i in range(1, m + 1):
        p[i] = p[i - 1] + FA / g[i]
    q = 0.0
    prev = 0.0
    for i in [0] + list(range(n - 1, m, -1)):  # walk backwards from plane 0 to plane m+1
        q = prev + FB / g[i]
        tgt = (i - 1) % n
        p[tgt] = q
        prev = q
        if tgt == m + 1:
            break
    assert abs((p[m + 1] + FB / g[m + 1]) - p[m]) < 1e-9 * max(1.0, abs(p[m]))
    return p - p.mean()


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("bcv", [0, 1])
def test_operator_layered_flux_closed_form(axis, bcv):
    rng = np.random.default_rng(10 + axis)
    shape = [4, 4, 4]
    shape[axis] = 12
    shape = tuple(shape)
    length = [1.0, 1.0, 1.0]
    length[axis] = 3.0
    h = length[axis] / shape[axis]
    n = shape[axis]
    alpha = np.exp(rng.uniform(math.log(1e-5), 0.0, size=n))
    faces = [np.full(cells(shape), 0.7) for _ in range(3)]
    sl = [None, None, None]
    sl[2 - axis] = slice(None)
    faces[axis] = np.broadcast_to(alpha[tuple(sl)], cells(shape)).copy()
    bc = [1, 1, 1]
    bc[axis] = bcv
    s = 2.5
    if bcv == 0:
        p1 = flux_solution_nonperiodic(alpha, h, s)
        src = np.zeros(n)
        src[0], src[-1] = s, -s
    else:
        m = 5
        p1 = flux_solution_periodic(alpha, h, s, m)
        src = np.zeros(n)
        src[0], src[m] = s, -s
    p = np.broadcast_to(p1[tuple(sl)], cells(shape)).copy()
    b = np.broadcast_to(src[tuple(sl)], cells(shape)).copy()
    Ap = oracle.apply(shape, bc, faces, p, tuple(length))
    assert np.allclose(Ap, b, rtol=0, atol=1e-9 * s)
    # contrast 1e5 between neighbouring planes: rounding limits the attainable accuracy
    res = oracle.solve_exact(shape, bc, faces, b, length=tuple(length))
    assert res.status in (0, 2)
    assert np.linalg.norm(res.x - p) <= 1e-9 * np.linalg.norm(p)


# ---------------------------------------------------------------------------
# (5) red-black relaxation, (3) restriction, (4) prolongation, coarse faces
# ---------------------------------------------------------------------------

def local_residual(shape, bc, faces, b, p, length=(1.0, 1.0, 1.0)):
    return b - oracle.apply(shape, bc, faces, p, length)


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("omega", [1.0, 1.3])
def test_smoother_zeroes_own_colour_residual(bc, omega):
    rng = np.random.default_rng(3)
    shape = (8, 6, 4)
    length = (1.0, 0.5, 2.0)
    f = I.random_faces(shape, rng, 1e-4, 1.0)
    b = rng.standard_normal(cells(shape))
    p = rng.standard_normal(cells(shape))
    K, J, Ii = np.indices(cells(shape))
    red = ((Ii + J + K) % 2) == 0
    for colour, mask in ((0, red), (1, ~red)):
        r0 = local_residual(shape, bc, f, b, p, length)
        q = oracle.smooth_colour(shape, bc, f, b, p, colour, omega, length)
        r1 = local_residual(shape, bc, f, b, q, length)
        # the other colour is not touched
        assert np.array_equal(q[~mask], p[~mask])
        # Gauss-Seidel zeroes the own-colour residual; SOR scales it by (1 - omega)
        scale = np.abs(b).max() + np.abs(oracle.apply(shape, bc, f, q, length)).max()
        assert np.allclose(r1[mask], (1.0 - omega) * r0[mask], rtol=0, atol=1e-12 * scale)
        p = q


def test_restriction_linear_exact_and_conservative():
    rng = np.random.default_rng(4)
    shape = (8, 12, 16)
    X, Y, Z = coords(shape)
    f = 0.3 + 1.7 * X - 0.4 * Y + 2.2 * Z
    rc = oracle.restrict(shape, (0, 0, 0), f)
    cs = oracle.coarse_shape(shape)
    Xc, Yc, Zc = coords(cs)
    assert np.allclose(rc, 0.3 + 1.7 * Xc - 0.4 * Yc + 2.2 * Zc, rtol=0, atol=1e-14 * 4)
    r = rng.standard_normal(cells(shape))
    assert abs(oracle.restrict(shape, (0, 0, 0), r).sum() - r.sum() / 8.0) < 1e-12


@pytest.mark.parametrize("bc", BCS)
def test_prolongation_constant_and_linear(bc):
    shape = (16, 8, 12)
    cs = oracle.coarse_shape(shape)
    x0 = np.zeros(cells(shape))
    out = oracle.prolong_add(shape, bc, np.full(cells(cs), 3.25), x0)
    assert np.allclose(out, 3.25, rtol=0, atol=1e-14)
    Xc, Yc, Zc = coords(cs)
    X, Y, Z = coords(shape)
    lin_c = 1.0 + 2.0 * Xc - 3.0 * Yc + 0.5 * Zc
    lin = 1.0 + 2.0 * X - 3.0 * Y + 0.5 * Z
    out = oracle.prolong_add(shape, bc, lin_c, x0)
    # exact wherever both bracketing coarse centres exist (not in the first/last fine cell of an axis)
    inner = (slice(1, -1), slice(1, -1), slice(1, -1))
    assert np.allclose(out[inner], lin[inner], rtol=0, atol=1e-13)


def test_prolongation_periodic_translation():
    rng = np.random.default_rng(5)
    shape = (8, 12, 16)
    cs = oracle.coarse_shape(shape)
    e = rng.standard_normal(cells(cs))
    x0 = np.zeros(cells(shape))
    bc = (1, 1, 1)
    base = oracle.prolong_add(shape, bc, e, x0)
    for ax in range(3):
        sh = oracle.prolong_add(shape, bc, np.roll(e, 1, axis=2 - ax), x0)
        assert np.allclose(sh, np.roll(base, 2, axis=2 - ax), rtol=0, atol=1e-14)


@pytest.mark.parametrize("bc", BCS)
def test_coarse_faces_conserve_conductance(bc):
    rng = np.random.default_rng(6)
    shape = (8, 12, 16)
    f = I.random_faces(shape, rng, 1e-3, 1.0)
    cf = oracle.coarsen_faces(shape, bc, f)
    cs = oracle.coarse_shape(shape)
    for d in range(3):
        nax = 2 - d
        for Ic in range(cs[d]):
            fine_plane = np.take(f[d], 2 * Ic, axis=nax)  # faces at even positions coincide with coarse faces
            coarse_plane = np.take(cf[d], Ic, axis=nax)
            # flux through the coarse face: coarse area is 4x a fine face
            assert abs(4.0 * coarse_plane.sum() - fine_plane.sum()) <= 1e-13 * fine_plane.sum()
        # faces inside a coarse cell (odd positions) do not enter the coarse face
        g = [a.copy() for a in f]
        sl = [slice(None)] * 3
        sl[nax] = slice(1, None, 2)
        g[d][tuple(sl)] *= 17.0
        cg = oracle.coarsen_faces(shape, bc, g)
        assert np.array_equal(cg[d], cf[d])
    const = oracle.coarsen_faces(shape, bc, [np.full(cells(shape), 0.37)] * 3)
    for d in range(3):
        assert np.allclose(const[d], 0.37, rtol=1e-15, atol=0)


@pytest.mark.parametrize("bc", BCS)
def test_coarse_operator_is_consistent(bc):
    """Constant alpha: the coarse operator is the fine one at spacing 2h."""
    shape = (16, 8, 12)
    cs = oracle.coarse_shape(shape)
    cf = oracle.coarsen_faces(shape, bc, ones_faces(shape))
    v, lam = eigen_mode(cs, bc, (1, 1, 2))
    Av = oracle.apply(cs, bc, cf, v)  # coarse spacing h = 1/n_c
    assert np.allclose(Av, lam * v, rtol=0, atol=1e-12 * abs(lam))


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("shape", [(4, 4, 4), (3, 3, 3), (2, 3, 4)])
def test_coarse_solve_exact(bc, shape):
    rng = np.random.default_rng(7)
    f = I.random_faces(shape, rng, 1e-5, 1.0)
    r = rng.standard_normal(cells(shape))
    e = oracle.coarse_solve(shape, bc, f, r)
    assert abs(e.mean()) < 1e-13 * np.abs(e).max()
    Ae = oracle.apply(shape, bc, f, e)
    rp = r - r.mean()
    assert np.allclose(Ae, rp, rtol=0, atol=1e-9 * np.abs(rp).max())


# ---------------------------------------------------------------------------
# Whole solve: dense direct solve, eigenvector, separable layered density
# ---------------------------------------------------------------------------

def dense_solution(shape, bc, faces, b, length=(1.0, 1.0, 1.0)):
    A = dense_matrix(shape, bc, faces, length)
    n = A.shape[0]
    c = np.abs(A).max() / n
    bp = b.ravel() - b.mean()
    return np.linalg.solve(A - c * np.ones((n, n)), bp).reshape(b.shape)


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("shape", [(8, 8, 8), (8, 6, 4), (6, 6, 6), (4, 4, 4)])
@pytest.mark.parametrize("ratio", [1.0, 10.0, 1000.0, 1e5])
def test_solve_matches_dense_direct(bc, shape, ratio):
    rng = np.random.default_rng(int(ratio) + shape[0])
    c = rng.uniform(0.3, 0.7, size=3)
    rho = I.density_field(shape, None, [(tuple(c), 0.3)], ratio, eps_cells=1.0)
    faces = oracle.faces_from_density(shape, bc, rho)
    b = rng.standard_normal(cells(shape))
    want = dense_solution(shape, bc, faces, b)
    got = oracle.solve_exact(shape, bc, faces, b, max_cycles=600)
    assert got.status in (0, 2)
    assert np.linalg.norm(got.x - want) <= 1e-12 * np.linalg.norm(want) * max(1.0, math.log10(ratio))


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("shape", [(16, 16, 16), (32, 32, 32), (48, 48, 48), (24, 32, 16)])
def test_solve_eigenvector_closed_form(bc, shape):
    v, lam = eigen_mode(shape, bc, (1, 2, 1))
    res = oracle.solve(shape, bc, ones_faces(shape), lam * v, tol=1e-12)
    assert res.status == 0
    assert np.linalg.norm(res.x - v) <= 1e-10 * np.linalg.norm(v)
    assert res.gamma < 0.3  # (24,32,16) on the unit cube has spacing ratio 2 between axes


def layered_exact(shape, rho_z, kx, ky, g, length=(1.0, 1.0, 1.0)):
    """Film-only density rho(z), periodic x/y, Neumann z.  b = cos-mode(x,y) g(z)
    gives p = cos-mode(x,y) f(z) with f from one tridiagonal system in z:
    a_c(k) lam_xy f_k + (1/hz^2)[az_k (f_{k-1}-f_k) + az_{k+1}(f_{k+1}-f_k)] = g_k."""
    nx, ny, nz = shape
    hx, hy, hz = (length[d] / shape[d] for d in range(3))
    lam_xy = -(4 / hx ** 2) * math.sin(math.pi * kx / nx) ** 2 - (4 / hy ** 2) * math.sin(math.pi * ky / ny) ** 2
    alpha_c = 1.0 / rho_z
    az = np.zeros(nz + 1)
    az[1:nz] = 2.0 / (rho_z[:-1] + rho_z[1:])  # harmonic, Eqs. 11-12; walls 0
    ab = np.zeros((3, nz))
    diag = alpha_c * lam_xy - (az[:nz] + az[1:]) / hz ** 2
    ab[1] = diag
    ab[0, 1:] = az[1:nz] / hz ** 2  # super-diagonal
    ab[2, :-1] = az[1:nz] / hz ** 2  # sub-diagonal
    import scipy.linalg
    f = scipy.linalg.solve_banded((1, 1), ab, g)
    mx = np.cos(2 * math.pi * kx * (np.arange(nx) + 0.5) / nx)
    my = np.cos(2 * math.pi * ky * (np.arange(ny) + 0.5) / ny)
    mode = my[:, None] * mx[None, :]
    return mode[None] * f[:, None, None], mode[None] * g[:, None, None]


@pytest.mark.parametrize("n", [16, 32, 64])
def test_solve_layered_density_separable(n):
    shape = (n, n, n)
    rng = np.random.default_rng(n)
    rho = I.density_field(shape, 0.3, [], 1000.0)
    rho_z = rho[:, 0, 0].copy()
    assert np.all(rho == rho_z[:, None, None])
    faces = oracle.faces_from_density(shape, I.DROP_FILM_BC, rho)
    g = rng.standard_normal(n)
    p_exact, b = layered_exact(shape, rho_z, 2, 1, g)
    res = oracle.solve(shape, I.DROP_FILM_BC, faces, b, tol=1e-12, max_cycles=200)
    assert res.status == 0
    assert np.linalg.norm(res.x - p_exact) <= 1e-9 * np.linalg.norm(p_exact)


@pytest.mark.parametrize("variable", [False, True], ids=["alpha_1", "alpha_1_plus_x_half"])
def test_manufactured_solution_second_order(variable):
    """Eq. 10 against the continuum: p = cos(pi x) cos(pi y) cos(pi z) on the unit
    cube has zero normal derivative on every wall (Neumann), and with alpha = 1
    or alpha = 1 + x/2 (taken at the face centres) S = div(alpha grad p) is
    known in closed form at the cell centres.  The discrete solution (mean
    removed on both sides) approaches p at second order: halving h divides the
    maximum error by 4 (3.6 .. 4.4).  For alpha = 1 the cosine is a discrete
    eigenvector, so the error is also known exactly:
    p_h / p = (pi h / 2)^2 / sin^2(pi h / 2)."""
    errs = []
    for n in (8, 16, 32):
        shape, bc, h = (n, n, n), (0, 0, 0), 1.0 / n
        c = (np.arange(n) + 0.5) * h
        z, y, x = np.meshgrid(c, c, c, indexing="ij")  # cell centres, arrays [k, j, i]
        p = np.cos(np.pi * x) * np.cos(np.pi * y) * np.cos(np.pi * z)
        if variable:
            xf = np.arange(n) * h  # x of the low x face of each cell
            ax = np.broadcast_to(1.0 + 0.5 * xf, cells(shape)).copy()
            a_c = 1.0 + 0.5 * x    # alpha at the centres of y and z faces (same x as the cell)
            faces = [ax, a_c.copy(), a_c.copy()]
            S = -3.0 * np.pi ** 2 * a_c * p - 0.5 * np.pi * np.sin(np.pi * x) * np.cos(np.pi * y) * np.cos(np.pi * z)
        else:
            faces = ones_faces(shape)
            S = -3.0 * np.pi ** 2 * p
        ph = oracle.solve_exact(shape, bc, faces, S).x.reshape(cells(shape))
        ph = ph - ph.mean()
        err = np.abs(ph - (p - p.mean())).max()
        if not variable:
            t = np.pi * h / 2.0
            exact_ratio = t * t / np.sin(t) ** 2
            assert err == pytest.approx((exact_ratio - 1.0) * np.abs(p).max(), rel=1e-6)
        errs.append(err)
    for coarse, fine in zip(errs, errs[1:]):
        assert 3.6 < coarse / fine < 4.4, errs


def test_gamma_eq15_closed_form():
    hist = np.array([2.0, 0.2, 0.02, 0.002])
    assert abs(oracle.gamma(hist) - 0.1) < 1e-15
    assert oracle.gamma(np.array([1.0])) == 0.0


@pytest.mark.parametrize("make", [lambda: I.config1(32), lambda: I.config2(32), lambda: I.config1(48)])
def test_multigrid_health_on_workloads(make):
    """gamma stays below the paper's worst observed value (about 0.5, Sec. 3)."""
    P = make()
    faces = oracle.faces_from_density(P.shape, P.bc, P.rho)
    res = oracle.solve(P.shape, P.bc, faces, P.rhs, tol=1e-10)
    assert res.status == 0
    assert res.gamma < 0.5
    r = oracle.residual(P.shape, P.bc, faces, P.rhs - P.rhs.mean(), res.x)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(P.rhs - P.rhs.mean()) * 1.0000001
    assert abs(res.x.mean()) < 1e-12 * np.abs(res.x).max()


def test_solve_zero_rhs_and_warm_start():
    P = I.config1(16)
    faces = oracle.faces_from_density(P.shape, P.bc, P.rho)
    z = oracle.solve(P.shape, P.bc, faces, np.zeros(cells(P.shape)))
    assert z.status == 0 and np.all(z.x == 0.0)
    ex = oracle.solve_exact(P.shape, P.bc, faces, P.rhs)
    warm = oracle.solve(P.shape, P.bc, faces, P.rhs, tol=1e-10, x0=ex.x + 5.0)
    assert warm.cycles == 0
    assert np.allclose(warm.x, ex.x, rtol=0, atol=1e-12 * np.abs(ex.x).max())


# ---------------------------------------------------------------------------
# Sec. 2.3 item 4, Eqs. 13-14: flux-conserving prolongation
# ---------------------------------------------------------------------------

def load_flux_golden():
    from fractions import Fraction
    rows = {}
    with open(os.path.join(GOLDEN, "flux_prolongation.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            rows[key] = [float(Fraction(v)) for v in vals]
    return rows


def test_trilinear_prolongation_golden():
    """Hand-worked trilinear prolongation at Neumann walls and across periodic
    wraps (tests/golden/trilinear_prolongation.txt): pins the coarse partner of
    the first and last fine cell of every axis."""
    coarse, cases = {}, []
    with open(os.path.join(GOLDEN, "trilinear_prolongation.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            if key.startswith("coarse_"):
                coarse[key] = [float(Fraction(v)) for v in vals]
            elif key == "case":
                cases.append((tuple(int(v) for v in vals), []))
            else:
                i, j, k, v = vals
                cases[-1][1].append((int(i), int(j), int(k), float(Fraction(v))))
    assert len(cases) == 2
    shape = (8, 4, 4)
    a, b, c = (np.array(coarse[k]) for k in ("coarse_a", "coarse_b", "coarse_c"))
    ec = c[:, None, None] + b[None, :, None] + a[None, None, :]  # (K, J, I)
    for bc, cells_ in cases:
        got = oracle.prolong_add(shape, bc, ec, np.zeros(cells(shape)))
        for i, j, k, v in cells_:
            assert got[k, j, i] == v, (bc, (i, j, k), got[k, j, i], v)


def test_flux_prolongation_golden():
    g = load_flux_golden()
    shape, bc = (8, 2, 2), (0, 0, 0)
    ac = np.array(g["coarse_alpha"]).reshape(1, 1, 4)
    ec = np.array(g["coarse_e"]).reshape(1, 1, 4)
    got = oracle.prolong_flux_add(shape, bc, ac, ec, np.zeros(cells(shape)))
    want = np.broadcast_to(np.array(g["fine"]), cells(shape))
    np.testing.assert_allclose(got, want, rtol=2e-16, atol=0)


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("shape", [(8, 8, 8), (12, 8, 6), (6, 4, 10)])
def test_flux_prolongation_constant_alpha_is_trilinear(bc, shape):
    """For a constant coefficient the alpha-weighted corner values are plain
    means, and the mean of an octant's 8 corners is the trilinear 27/9/3/1 rule."""
    rng = np.random.default_rng(sum(shape))
    cs = oracle.coarse_shape(shape)
    e = rng.standard_normal(cells(cs))
    x = rng.standard_normal(cells(shape))
    got = oracle.prolong_flux_add(shape, bc, np.full(cells(cs), 3.7), e, x)
    want = oracle.prolong_add(shape, bc, e, x)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14 * np.abs(want).max())


@pytest.mark.parametrize("bc", BCS)
def test_flux_prolongation_local_maximum_principle(bc):
    """Every corner value is a convex combination (positive weights), so a fine
    value lies between the extremes of the 2 x 2 x 2 coarse cells around it."""
    shape = (8, 6, 10)
    cs = oracle.coarse_shape(shape)
    rng = np.random.default_rng(3)
    ac = 10.0 ** rng.uniform(-3, 3, size=cells(cs))
    e = rng.standard_normal(cells(cs))
    got = oracle.prolong_flux_add(shape, bc, ac, e, np.zeros(cells(shape)))

    def partner(i, nc, periodic):
        I = i // 2
        J = I - 1 if i % 2 == 0 else I + 1
        if 0 <= J < nc:
            return J
        return J % nc if periodic else I

    for k in range(shape[2]):
        for j in range(shape[1]):
            for i in range(shape[0]):
                Is = [i // 2, partner(i, cs[0], bc[0])]
                Js = [j // 2, partner(j, cs[1], bc[1])]
                Ks = [k // 2, partner(k, cs[2], bc[2])]
                vals = [e[K, J, I] for K in Ks for J in Js for I in Is]
                assert min(vals) - 1e-15 <= got[k, j, i] <= max(vals) + 1e-15


def test_flux_prolongation_follows_the_conductive_side():
    """A coarse neighbour with a vanishing coefficient does not pull the face
    value: next to it the fine value is the coarse cell's own (Eq. 13)."""
    shape, bc = (4, 2, 2), (0, 0, 0)
    ac = np.array([1.0, 1e-14]).reshape(1, 1, 2)
    ec = np.array([5.0, -7.0]).reshape(1, 1, 2)
    got = oracle.prolong_flux_add(shape, bc, ac, ec, np.zeros(cells(shape)))
    np.testing.assert_allclose(got[..., 1], 5.0, rtol=1e-12)     # cell 1 of coarse 0, face to coarse 1
    np.testing.assert_allclose(got[..., 2], (-7.0 + 5.0) / 2, rtol=1e-12)  # coarse 1 sees coarse 0's value


def test_cell_alpha_hand_values():
    """Mean of the non-wall face coefficients of each cell."""
    shape, bc = (3, 2, 2), (0, 1, 0)  # walls in x and z, periodic y
    ax = np.zeros(cells(shape))
    ay = np.zeros(cells(shape))
    az = np.zeros(cells(shape))
    ax[...] = np.array([9.0, 2.0, 4.0])      # low x faces: wall (ignored), 2 between i=0|1, 4 between 1|2
    ay[:, 0, :] = 3.0                        # y faces: low face of j=0 (= wrap face) 3, of j=1: 5
    ay[:, 1, :] = 5.0
    az[0] = 7.0                              # low z face of k=0 is a wall
    az[1] = 6.0
    got = oracle.cell_alpha(shape, bc, [ax, ay, az])
    # cell (0,0,0): faces x+ 2, y- 3, y+ 5, z+ 6 (x- and z- are walls)
    assert got[0, 0, 0] == pytest.approx((2 + 3 + 5 + 6) / 4, rel=1e-15)
    # cell (1,1,1): x- 2, x+ 4, y- 5, y+ 3 (wrap), z- 6 (z+ wall)
    assert got[1, 1, 1] == pytest.approx((2 + 4 + 5 + 3 + 6) / 5, rel=1e-15)
    # cell (2,0,1): x- 4 (x+ wall), y- 3, y+ 5, z- 6
    assert got[1, 0, 2] == pytest.approx((4 + 3 + 5 + 6) / 4, rel=1e-15)
    # constant faces give the constant
    np.testing.assert_allclose(oracle.cell_alpha((8, 6, 4), (1, 0, 1), [np.full(cells((8, 6, 4)), 0.3)] * 3),
                               0.3, rtol=1e-15)


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("ratio", [1000.0, 1e5])
def test_flux_prolongation_solve_matches_dense_direct(bc, ratio):
    shape = (8, 8, 8)
    rng = np.random.default_rng(int(ratio) + 11)
    c = rng.uniform(0.3, 0.7, size=3)
    rho = I.density_field(shape, None, [(tuple(c), 0.3)], ratio, eps_cells=1.0)
    faces = oracle.faces_from_density(shape, bc, rho)
    b = rng.standard_normal(cells(shape))
    want = dense_solution(shape, bc, faces, b)
    got = oracle.solve_exact(shape, bc, faces, b, max_cycles=600, prolong=oracle.PROLONG_FLUX)
    assert got.status in (0, 2)
    assert np.linalg.norm(got.x - want) <= 1e-12 * np.linalg.norm(want) * max(1.0, math.log10(ratio))


@pytest.mark.parametrize("ratio", [1000.0, 1e5])
def test_flux_prolongation_converges_on_drop_film(ratio):
    """Multigrid health with the paper's prolongation on a drop/film field."""
    P = I.config2(32)
    rho = I.density_field(P.shape, 0.1, [((0.5, 0.5, 0.3), 0.125)], ratio)
    faces = oracle.faces_from_density(P.shape, P.bc, rho)
    r = oracle.solve(P.shape, P.bc, faces, P.rhs, tol=1e-10, max_cycles=200, prolong=oracle.PROLONG_FLUX)
    assert r.status == 0 and r.gamma < 0.5


# ---------------------------------------------------------------------------
# Projection step around the solve (Sec. 2.2, Chorin's projection on the MAC grid)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("bc", BCS)
def test_divergence_of_projected_gradient_is_the_operator(bc):
    """D(alpha G p) = A p: project a zero field with dt = 1 (u = -alpha G p),
    take its divergence, compare with oracle_apply (Eq. 10)."""
    shape, length = (12, 10, 8), (1.0, 0.7, 1.3)
    rng = np.random.default_rng(21)
    faces = [rng.uniform(0.01, 1.0, size=cells(shape)) for _ in range(3)]
    p = rng.standard_normal(cells(shape))
    zero = [np.zeros(cells(shape)) for _ in range(3)]
    u = oracle.project(shape, bc, faces, p, zero, dt=1.0, length=length)
    div = oracle.divergence(shape, bc, u, dt=1.0, length=length)
    Ap = oracle.apply(shape, bc, faces, p, length=length)
    np.testing.assert_allclose(div, -Ap, rtol=0, atol=1e-13 * np.abs(Ap).max())


@pytest.mark.parametrize("bc", BCS)
def test_divergence_matches_the_rhs_generator(bc):
    """The Fourier velocity field and the RHS generator draw the same field;
    the generator differences it on its own face samples (high faces sampled
    directly), the oracle through the low-face layout and the wrap rule."""
    shape = (16, 12, 20)
    u = I.fourier_velocity(shape, bc, np.random.default_rng(33))
    b = I.rhs_fourier_divergence(shape, bc, np.random.default_rng(33))
    S = oracle.divergence(shape, bc, u, dt=0.25)
    np.testing.assert_allclose(0.25 * S - (0.25 * S).mean(), b, rtol=0, atol=1e-12 * np.abs(b).max())


@pytest.mark.parametrize("bc", BCS)
def test_divergence_sums_to_zero(bc):
    """Discrete divergence theorem: walls carry no flux, periodic faces cancel."""
    shape = (10, 6, 8)
    rng = np.random.default_rng(8)
    u = [rng.standard_normal(cells(shape)) for _ in range(3)]
    S = oracle.divergence(shape, bc, u, dt=1.0)
    assert abs(S.sum()) <= 1e-12 * np.abs(S).sum()


def test_projection_step_removes_the_divergence():
    """S = D u* / dt, p = p*(S), u = u* - dt alpha G p: D u = dt (S - A p)."""
    shape, bc, rho, u, dt = I.projection_problem(32, ratio=1000.0, dt=1e-2)
    faces = oracle.faces_from_density(shape, bc, rho)
    S = oracle.divergence(shape, bc, u, dt=dt)
    p = oracle.solve_exact(shape, bc, faces, S).x
    un = oracle.project(shape, bc, faces, p, u, dt=dt)
    div = oracle.divergence(shape, bc, un, dt=1.0)
    assert np.linalg.norm(div) <= 1e-10 * np.linalg.norm(dt * S)
    # walls keep zero normal velocity
    assert np.all(un[2][0] == 0.0)


# ---------------------------------------------------------------------------
# Conjugate gradients preconditioned by the V-cycle (next rows: MG-PCG)
# ---------------------------------------------------------------------------

def test_cg_finite_termination_on_few_eigenvalues():
    """Plain CG ends in at most as many steps as -A has distinct nonzero
    eigenvalues: 4^3 periodic, alpha = 1: per axis 4 sin^2(pi k / 4) / h^2 is
    0, 2, 4 (x 1/h^2), so the 3-axis sums take 6 distinct nonzero values."""
    shape, bc = (4, 4, 4), (1, 1, 1)
    b = np.random.default_rng(2).standard_normal(cells(shape))
    r = oracle.pcg_solve(shape, bc, ones_faces(shape), b, tol=1e-12, max_it=50, precond=False)
    assert r.status == 0 and r.cycles <= 6


def test_cg_single_eigenvector_one_step():
    """b an eigenvector of A: plain CG is exact after one step."""
    shape, bc = (16, 8, 8), (0, 1, 0)
    X, Y, Z = coords(shape)
    b = np.cos(np.pi * 2 * X) * np.cos(2 * np.pi * Y)  # Neumann mode k=2 in x, periodic mode 1 in y
    r = oracle.pcg_solve(shape, bc, ones_faces(shape), b, tol=1e-12, max_it=5, precond=False)
    assert r.status == 0 and r.cycles == 1


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("ratio", [1.0, 1000.0, 1e5])
def test_pcg_matches_dense_direct(bc, ratio):
    shape = (8, 8, 8)
    rng = np.random.default_rng(int(ratio) + 31)
    c = rng.uniform(0.3, 0.7, size=3)
    rho = I.density_field(shape, None, [(tuple(c), 0.3)], ratio, eps_cells=1.0)
    faces = oracle.faces_from_density(shape, bc, rho)
    b = rng.standard_normal(cells(shape))
    want = dense_solution(shape, bc, faces, b)
    got = oracle.pcg_solve(shape, bc, faces, b, tol=1e-14, max_it=100)
    assert got.status == 0
    assert np.linalg.norm(got.x - want) <= 1e-11 * np.linalg.norm(want) * max(1.0, math.log10(ratio))


@pytest.mark.parametrize("ratio", [1000.0, 1e5])
def test_pcg_converges_on_drop_film(ratio):
    P = I.config2(32)
    rho = I.density_field(P.shape, 0.1, [((0.5, 0.5, 0.3), 0.125)], ratio)
    faces = oracle.faces_from_density(P.shape, P.bc, rho)
    r = oracle.pcg_solve(P.shape, P.bc, faces, P.rhs, tol=1e-10)
    mg = oracle.solve(P.shape, P.bc, faces, P.rhs, tol=1e-10)
    assert r.status == 0 and r.gamma < 0.5 and r.cycles <= mg.cycles


# ---------------------------------------------------------------------------
# Sec. 2.3 item 6: GMRES on the coarsest grid (next rows: coarsest grids above
# the dense solver's 512 cells)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("bc", BCS)
def test_gmres_matches_dense_coarse_solve(bc):
    shape = (9, 7, 5)
    rng = np.random.default_rng(41)
    f = [rng.uniform(0.05, 1.0, size=cells(shape)) for _ in range(3)]
    r = rng.standard_normal(cells(shape))
    e, st, its = oracle.gmres(shape, bc, f, r, tol=1e-13, max_it=2000, m=50)
    want = oracle.coarse_solve(shape, bc, f, r)
    assert st == 0
    np.testing.assert_allclose(e, want, rtol=0, atol=1e-11 * np.abs(want).max())


def test_gmres_finite_termination():
    """Without restarts GMRES is exact after as many steps as the Krylov space
    has dimensions: 2 x 2 x 2 with alpha = 1 has 3 distinct nonzero eigenvalues."""
    shape, bc = (2, 2, 2), (0, 0, 0)
    r = np.random.default_rng(1).standard_normal(cells(shape))
    e, st, its = oracle.gmres(shape, bc, ones_faces(shape), r, tol=1e-13, max_it=20, m=20)
    assert st == 0 and its <= 3
    np.testing.assert_allclose(oracle.apply(shape, bc, ones_faces(shape), e), r - r.mean(), atol=1e-12)


@pytest.mark.parametrize("shape,bc", [((9, 9, 9), (0, 0, 0)), ((18, 18, 14), (1, 0, 1))])
def test_solve_with_gmres_coarsest_matches_dense_direct(shape, bc):
    """Coarsest grids above 512 cells (9^3 single level; 9 x 9 x 7 under
    18 x 18 x 14) take the GMRES coarse solve; the result is still p*."""
    rng = np.random.default_rng(sum(shape))
    c = rng.uniform(0.3, 0.7, size=3)
    rho = I.density_field(shape, None, [(tuple(c), 0.3)], 1000.0, eps_cells=1.0)
    faces = oracle.faces_from_density(shape, bc, rho)
    b = rng.standard_normal(cells(shape))
    want = dense_solution(shape, bc, faces, b)
    got = oracle.solve_exact(shape, bc, faces, b, max_cycles=200)
    assert got.status in (0, 2)
    assert np.linalg.norm(got.x - want) <= 1e-11 * np.linalg.norm(want)
