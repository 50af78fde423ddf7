"""Launch shapes of the V-cycle kernels and their autotuner, through the C ABI.

Every shape runs the same per-cell arithmetic (Sec. 2.3 relaxation,
restriction and prolongation of arXiv 1410.8568), so a shape may change the
speed of a solve but never a bit of its result: the tests compare solves and
single kernels bitwise across all shapes, on level sizes whose quads per row
are not powers of two (the flat shapes divide by them) and on ragged rows
shorter than a warp.
"""
import numpy as np
import pytest

import oracle
from paper_1410_8568_gb300 import gbmg
from paper_1410_8568_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALL = list(range(gbmg.TILE_VARIANTS))


def cells(shape):
    return (shape[2], shape[1], shape[0])


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def problem(shape, bc, seed, ratio=1000.0):
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.3, 0.7, size=3)
    rho = I.density_field(shape, None, [(tuple(c), 0.2)], ratio)
    b = rng.standard_normal(cells(shape))
    b -= b.mean()
    return rho, b


@pytest.mark.parametrize("precision", [gbmg.MIXED, gbmg.FP64])
@pytest.mark.parametrize("shape,bc", [((64, 64, 64), (0, 0, 0)), ((48, 40, 24), (1, 0, 1)),
                                      ((96, 24, 16), (1, 1, 0)), ((40, 20, 12), (0, 1, 0))])
def test_solve_bitwise_equal_across_shapes(shape, bc, precision):
    rho, b = problem(shape, bc, sum(shape) + bc[0])
    f = oracle.faces_from_density(shape, bc, rho)
    faces = [dev(a) for a in f]
    rhs = dev(b)
    ref, ref_it = None, None
    for tiles in [gbmg.TILES_AUTO] + ALL:
        with gbmg.Solver(shape, bc, faces=faces, precision=precision, tiles=tiles) as S:
            for lvl in range(S.num_levels()):
                for kind in (gbmg.TILE_HALF, gbmg.TILE_RESTRICT, gbmg.TILE_PROLONG):
                    v = S.tile_choice(kind, lvl)
                    assert 0 <= v < gbmg.TILE_VARIANTS
                    if tiles >= 0 and v != tiles:
                        # a forced shape is replaced by row tiles only where rows are not quads
                        assert v == 0 and (S.level_shape(lvl)[0] % 4 != 0 or lvl + 1 == S.num_levels())
            p = torch.zeros_like(rhs)
            st = S.solve(rhs, p, tol=1e-10)
            assert st.status == gbmg.OK and st.rel_res <= 1e-10
            torch.cuda.synchronize()
            if ref is None:
                ref, ref_it = p.clone(), st.iters
            else:
                assert st.iters == ref_it, tiles
                assert torch.equal(p, ref), (tiles, (p - ref).abs().max().item())


@pytest.mark.parametrize("shape,bc", [((48, 32, 24), (1, 0, 1)), ((24, 12, 8), (0, 1, 1))])
def test_unit_kernels_bitwise_equal_across_shapes(shape, bc):
    """mg_smooth / mg_restrict_residual / mg_prolong use the handle's shape per level."""
    rho, _ = problem(shape, bc, 11)
    f = oracle.faces_from_density(shape, bc, rho)
    faces = [dev(a) for a in f]
    rng = np.random.default_rng(12)
    outs = {}
    for tiles in ALL:
        with gbmg.Solver(shape, bc, faces=faces, precision=gbmg.MIXED, tiles=tiles) as S:
            res = []
            for lvl in range(S.num_levels() - 1):
                sh, cs = S.level_shape(lvl), S.level_shape(lvl + 1)
                r = np.random.default_rng(100 + lvl)
                b, x, e = r.standard_normal(cells(sh)), r.standard_normal(cells(sh)), r.standard_normal(cells(cs))
                for prec, dt in ((gbmg.FP64, torch.float64), (gbmg.MIXED, torch.float32)):
                    xs = dev(x, dt)
                    S.smooth(lvl, dev(b, dt), xs, 2, prec=prec)
                    cb = torch.empty(cells(cs), dtype=dt, device="cuda")
                    S.restrict_residual(lvl, dev(b, dt), dev(x, dt), cb, prec=prec)
                    xp = dev(x, dt)
                    S.prolong(lvl, dev(e, dt), xp, prec=prec)
                    res += [xs, cb, xp]
            torch.cuda.synchronize()
            outs[tiles] = res
    for tiles in ALL[1:]:
        for a, b in zip(outs[0], outs[tiles]):
            assert torch.equal(a, b), tiles


def test_tune_cache_save_and_load(tmp_path):
    shape, bc = (64, 48, 32), (1, 0, 0)
    rho, _ = problem(shape, bc, 31)
    f = [dev(a) for a in oracle.faces_from_density(shape, bc, rho)]
    gbmg.tune_cache_clear()
    with gbmg.Solver(shape, bc, faces=f, precision=gbmg.FP64) as A:
        ca = [[A.tile_choice(k, l) for l in range(A.num_levels())] for k in range(3)]
    assert gbmg.tune_cache_size() > 0
    path = str(tmp_path / "tune.txt")
    gbmg.tune_cache_save(path)
    n = gbmg.tune_cache_size()
    gbmg.tune_cache_clear()
    assert gbmg.tune_cache_load(path) == n
    with gbmg.Solver(shape, bc, faces=f, precision=gbmg.FP64) as B:
        cb = [[B.tile_choice(k, l) for l in range(B.num_levels())] for k in range(3)]
    assert ca == cb


def test_autotuned_choices_are_cached_and_skip_tail_levels():
    shape, bc = (128, 128, 64), (1, 1, 0)
    rho, _ = problem(shape, bc, 21)
    f = [dev(a) for a in oracle.faces_from_density(shape, bc, rho)]
    gbmg.tune_cache_clear()
    with gbmg.Solver(shape, bc, faces=f, precision=gbmg.MIXED) as A:
        L = A.num_levels()
        ca = [[A.tile_choice(k, l) for l in range(L)] for k in range(3)]
    with gbmg.Solver(shape, bc, faces=f, precision=gbmg.MIXED) as B:
        cb = [[B.tile_choice(k, l) for l in range(L)] for k in range(3)]
    assert ca == cb  # the second handle reuses the first one's timings
    levels = [shape]
    for _ in range(L - 1):
        levels.append(tuple(v // 2 for v in levels[-1]))
    for l, sh in enumerate(levels):
        if l == L - 1 or (l >= 1 and np.prod(sh) <= 4096):
            # coarsest level and levels inside the shared-memory tail: no table launches
            assert all(ca[k][l] == 0 for k in range(3)), (l, sh)
