"""The one-pass red-black sweep (both colours of a sweep in one launch, Sec. 2.3
item 5) through the C ABI: bitwise equal to the red and black half-sweep
launches and to the oracle's red-black sweep within rounding, for every launch
shape that fits (whole-row shapes, and the staged shapes whose tiles of 128
cells are copied into shared memory), on grids whose strips, tiles and plane
chunks are ragged; whole solves with it are bitwise equal to whole solves with
half-sweeps, alone, batched and in the host-driven loop, and reach the
oracle's p*."""
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


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def fits(shape, bc, v, fp32=True):
    threads, _, tile_x = gbmg.sweep_shape(v)
    if (bc[1] and shape[1] % 2) or (bc[2] and shape[2] % 2):
        return False
    if tile_x:
        return fp32 and shape[0] % tile_x == 0
    return shape[0] % 4 == 0 and 3 * (shape[0] // 4) <= threads


def random_faces(shape, bc, seed):
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.3, 0.7, size=3)
    rho = I.density_field(shape, None, [(tuple(c), 0.25)], 1000.0)
    return oracle.faces_from_density(shape, bc, rho)


# rows of 64 cells: a 512-thread block owns 30 rows (32 slots), so 48 rows are
# 2 strips of 24; 40 planes are 3 chunks of 14 / 14 / 12 planes of 16 (or 2 of
# 20 of 32); rows of 160 cells: 40 quads, 12 rows per 512-thread strip
SHAPES = [((64, 48, 40), (1, 1, 0)), ((64, 48, 40), (0, 0, 0)), ((160, 30, 18), (1, 0, 1)),
          ((32, 66, 34), (0, 1, 1)),
          # staged shapes: tiles of 128 cells; 30 rows = 3 strips of 10, 15 rows =
          # strips of 8 / 7; 130 planes in chunks of at most 64: 44 / 44 / 42
          ((128, 30, 18), (1, 1, 0)), ((256, 30, 22), (0, 0, 1)), ((128, 15, 9), (1, 0, 0)),
          ((384, 16, 6), (0, 1, 0)), ((128, 12, 130), (0, 1, 1))]


@pytest.mark.parametrize("shape,bc", SHAPES)
@pytest.mark.parametrize("prec", [gbmg.MIXED, gbmg.FP64])
@pytest.mark.parametrize("omega", [1.0, 1.3])
def test_onepass_equals_half_sweeps_and_oracle(shape, bc, prec, omega):
    f = random_faces(shape, bc, sum(shape))
    dt = torch.float32 if prec == gbmg.MIXED else torch.float64
    rng = np.random.default_rng(3)
    b = rng.standard_normal(cells(shape))
    x0 = rng.standard_normal(cells(shape))
    # the oracle's red-black sweeps (raw faces: the oracle scales by 1/h^2 itself)
    want1 = oracle.smooth_colour(shape, bc, f, b, oracle.smooth_colour(shape, bc, f, b, x0, 0, omega), 1, omega)
    want2 = oracle.smooth_colour(shape, bc, f, b, oracle.smooth_colour(shape, bc, f, b, want1, 0, omega), 1, omega)
    tol = 1e-5 if prec == gbmg.MIXED else 1e-13
    with gbmg.Solver(shape, bc, faces=[dev(a) for a in f], precision=prec, omega=omega) as S:
        ref = dev(x0, dt)
        S.smooth(0, dev(b, dt), ref, 2, prec=prec)
        ref1 = dev(x0, dt)
        S.smooth(0, dev(b, dt), ref1, 1, prec=prec)
        tried = 0
        for v in range(1, gbmg.SWEEP_VARIANTS):
            if not fits(shape, bc, v, prec == gbmg.MIXED):
                continue
            x = dev(x0, dt)
            work = torch.full_like(x, float("nan"))
            S.smooth_onepass(0, dev(b, dt), x, work, 2, prec=prec, variant=v)
            assert torch.equal(x, ref), (v, (x - ref).abs().max().item())
            scale = np.abs(want2).max() + np.abs(x0).max()
            assert np.abs(x.double().cpu().numpy() - want2).max() <= tol * scale, v
            x = dev(x0, dt)
            work = torch.full_like(x, float("nan"))
            S.smooth_onepass(0, dev(b, dt), x, work, 1, prec=prec, variant=v)
            assert torch.equal(work, ref1), (v, (work - ref1).abs().max().item())
            assert np.abs(work.double().cpu().numpy() - want1).max() <= tol * scale, v
            tried += 1
        assert tried >= 3


def test_onepass_refuses_shapes_that_do_not_fit():
    shape, bc = (64, 48, 40), (1, 1, 0)
    f = random_faces(shape, bc, 1)
    with gbmg.Solver(shape, bc, faces=[dev(a) for a in f]) as S:
        x = torch.zeros(cells(shape), dtype=torch.float32, device="cuda")
        for v in (-1, gbmg.SWEEP_VARIANTS):
            with pytest.raises(gbmg.MGError):
                S.smooth_onepass(0, x, x.clone(), x.clone(), 1, prec=gbmg.MIXED, variant=v)
    # an odd periodic y axis: the colours do not alternate across the wrap
    # (a single-level grid, its coarsest solve by GMRES)
    shape, bc = (16, 7, 8), (1, 1, 0)
    f = random_faces(shape, bc, 2)
    with gbmg.Solver(shape, bc, faces=[dev(a) for a in f]) as S:
        x = torch.zeros(cells(shape), dtype=torch.float32, device="cuda")
        with pytest.raises(gbmg.MGError):
            S.smooth_onepass(0, x, x.clone(), x.clone(), 1, prec=gbmg.MIXED, variant=1)
        assert S.tile_choice(gbmg.TILE_SWEEP, 0) == 0
    # staged shapes: FP32 only, and rows of whole 128-cell tiles
    shape, bc = (128, 16, 8), (1, 1, 0)
    f = random_faces(shape, bc, 3)
    staged = [v for v in range(1, gbmg.SWEEP_VARIANTS) if gbmg.sweep_shape(v)[2]]
    assert staged
    with gbmg.Solver(shape, bc, faces=[dev(a) for a in f], precision=gbmg.FP64) as S:
        x = torch.zeros(cells(shape), dtype=torch.float64, device="cuda")
        for v in staged:
            with pytest.raises(gbmg.MGError):
                S.smooth_onepass(0, x, x.clone(), x.clone(), 1, prec=gbmg.FP64, variant=v)
    shape = (64, 16, 8)
    f = random_faces(shape, bc, 4)
    with gbmg.Solver(shape, bc, faces=[dev(a) for a in f]) as S:
        x = torch.zeros(cells(shape), dtype=torch.float32, device="cuda")
        for v in staged:
            with pytest.raises(gbmg.MGError):
                S.smooth_onepass(0, x, x.clone(), x.clone(), 1, prec=gbmg.MIXED, variant=v)


def solve_with(P, f, sweep, precision, outer=gbmg.OUTER_FP64, use_graph=True):
    with gbmg.Solver(P.shape, P.bc, faces=[dev(a) for a in f], precision=precision, outer=outer, sweep=sweep,
                     use_graph=use_graph) as S:
        chosen = S.tile_choice(gbmg.TILE_SWEEP, 0)
        p = torch.zeros(cells(P.shape), dtype=torch.float64, device="cuda")
        st = S.solve(dev(P.rhs), p, tol=TOL)
        assert st.status == gbmg.OK and st.rel_res <= TOL
        return p, st.iters, chosen


@pytest.mark.parametrize("precision,outer", [(gbmg.MIXED, gbmg.OUTER_FP64), (gbmg.FP64, gbmg.OUTER_FP64),
                                             (gbmg.MIXED, gbmg.OUTER_XP)], ids=["mixed", "fp64", "mixed_xp"])
def test_solve_with_onepass_sweeps_is_bitwise_the_half_sweep_solve(precision, outer):
    P = I.config2(64)
    f = oracle.faces_from_density(P.shape, P.bc, P.rho)
    p_half, it_half, chosen = solve_with(P, f, gbmg.SWEEP_HALF, precision, outer)
    assert chosen == 0
    for v in (1, 4, 6, gbmg.SWEEP_AUTO):
        for use_graph in (True, False):
            p, it, chosen = solve_with(P, f, v, precision, outer, use_graph)
            assert v == gbmg.SWEEP_AUTO or chosen == v
            assert it == it_half and torch.equal(p, p_half), (v, use_graph)
    pstar = oracle.solve_exact(P.shape, P.bc, f, P.rhs).x
    err = np.linalg.norm(p_half.cpu().numpy() - pstar) / np.linalg.norm(pstar)
    assert err <= ERR


@pytest.mark.parametrize("outer", [gbmg.OUTER_FP64, gbmg.OUTER_XP], ids=["mixed", "mixed_xp"])
def test_staged_solve_is_bitwise_the_half_sweep_solve(outer):
    """FP32 cycles with the staged one-pass sweep on a 128^3 drop/film grid (one
    128-cell tile per row, 10 strips of up to 13 rows): every staged shape, in the
    graph and in the host-driven loop, bitwise the half-sweep solve."""
    P = I.config2(128)
    f = oracle.faces_from_density(P.shape, P.bc, P.rho)
    p_half, it_half, _ = solve_with(P, f, gbmg.SWEEP_HALF, gbmg.MIXED, outer)
    staged = [v for v in range(1, gbmg.SWEEP_VARIANTS) if gbmg.sweep_shape(v)[2]]
    for v in staged:
        for use_graph in (True, False):
            p, it, chosen = solve_with(P, f, v, gbmg.MIXED, outer, use_graph)
            assert chosen == v
            assert it == it_half and torch.equal(p, p_half), (v, use_graph)


def test_batch_with_onepass_sweeps_matches_alone():
    """A batch of grids of different sizes runs its finest-level sweeps as one
    one-pass launch over all grids (the shape of the largest): each grid's
    result is bitwise its solo result with half-sweeps."""
    probs = [I.config1(32), I.config2(48), I.config2(64), I.config1(64, ratio=10.0)]
    faces = [oracle.faces_from_density(P.shape, P.bc, P.rho) for P in probs]
    alone = [solve_with(P, f, gbmg.SWEEP_HALF, gbmg.MIXED)[:2] for P, f in zip(probs, faces)]
    solvers = [gbmg.Solver(P.shape, P.bc, faces=[dev(a) for a in f], sweep=1) for P, f in zip(probs, faces)]
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


def test_batch_with_staged_sweeps_matches_alone():
    """A batch of grids with rows of whole 128-cell tiles runs its finest-level
    sweeps as one staged launch over all grids (each grid with its own tiles):
    each grid's result is bitwise its solo result with half-sweeps."""
    probs = [I.config2(128), I.config1(128, ratio=10.0), I.config2(256)]
    faces = [oracle.faces_from_density(P.shape, P.bc, P.rho) for P in probs]
    alone = [solve_with(P, f, gbmg.SWEEP_HALF, gbmg.MIXED)[:2] for P, f in zip(probs, faces)]
    staged = [v for v in range(1, gbmg.SWEEP_VARIANTS) if gbmg.sweep_shape(v)[2]]
    solvers = [gbmg.Solver(P.shape, P.bc, faces=[dev(a) for a in f], sweep=staged[1]) for P, f in zip(probs, faces)]
    assert all(S.tile_choice(gbmg.TILE_SWEEP, 0) == staged[1] for S in solvers)
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
