"""The allocation-free small-grid solve (mg_coarse_solve_static) through the C
ABI, against the FP64 CPU oracle's coarsest-grid solve and against the
coarsest-grid solve of a handle (mg_coarse_solve).

mg_coarse_solve_static is for callers that cannot allocate device memory when
they need a solve: a real-time loop whose device memory is budgeted up front,
or a host program whose own allocator has reserved the device memory.  It keeps
its scratch in a static device array of the library.  This file is collected
last so that a failure here leaves every other test already run; it passes
alone in a fresh process as well as after the other tests.
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


def faces_for(shape, bc, seed):
    """alpha = 1/rho of a 1000:1 sphere (Eqs. 11-12 on the device) and the same on the host."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.3, 0.7, size=3)
    rho = I.density_field(shape, None, [(tuple(c), 0.3)], 1000.0, eps_cells=1.0)
    out = [torch.empty(cells(shape), dtype=torch.float64, device="cuda") for _ in range(3)]
    gbmg.faces_from_density(shape, bc, torch.from_numpy(rho).cuda(), *out)
    return out, oracle.faces_from_density(shape, bc, rho)


def trace_minus_a(shape, bc, faces):
    """trace(-A): every face off the walls joins two cells and adds alpha / h^2
    to the diagonal of each (unit box: h_d = 1 / n_d)."""
    t = 0.0
    for d in range(3):
        a = faces[d].copy()
        if not bc[d]:
            idx = [slice(None)] * 3
            idx[2 - d] = 0  # arrays are (z, y, x): axis d is array axis 2 - d
            a[tuple(idx)] = 0.0  # the low wall carries no flux
        elif shape[d] == 1:
            a[...] = 0.0
        t += 2.0 * a.sum() * shape[d] ** 2
    return t


def check_against_oracle(shape, bc, faces_h, r, got):
    """got = oracle's zero-mean solution of A e = r - mean(r) plus -sum(r) / trace(-A)."""
    want = oracle.coarse_solve(shape, bc, faces_h, r)
    offset = -r.sum() / trace_minus_a(shape, bc, faces_h)
    scale = np.abs(want).max()
    np.testing.assert_allclose(got, want + offset, rtol=0, atol=1e-11 * scale)


# grids that are their own coarsest level (no axis can be halved), so a
# handle's mg_coarse_solve acts on the same operator; (2, 16, 16) has exactly
# MG_STATIC_MAX_CELLS cells: the scratch matrix is full and the flag sits just
# past it
@pytest.mark.parametrize("shape,bc", [((8, 8, 2), (1, 1, 0)), ((4, 3, 4), (0, 0, 0)), ((6, 3, 5), (1, 0, 1)),
                                      ((16, 2, 8), (0, 1, 0)), ((2, 16, 16), (0, 1, 0))])
def test_static_solve_matches_oracle_and_handle_twice(shape, bc):
    faces, faces_h = faces_for(shape, bc, sum(shape))
    with gbmg.Solver(shape, bc, faces=faces, precision=gbmg.FP64) as S:
        assert S.num_levels() == 1
        rng = np.random.default_rng(7)
        for call in range(2):  # two calls in a row share the static scratch array
            rh = rng.standard_normal(cells(shape))
            if call == 0:
                rh -= rh.mean()  # a zero-sum right-hand side: zero-mean result
            r = torch.from_numpy(rh).cuda()
            want = torch.empty_like(r)
            S.coarse_solve(r, want, prec=gbmg.FP64)
            got = torch.full_like(r, float("nan"))
            rc = gbmg.coarse_solve_static(shape, bc, faces, r, got)
            assert rc == gbmg.OK, gbmg.strerror(rc)
            torch.cuda.synchronize()
            scale = want.abs().max().item()
            assert torch.allclose(got, want, rtol=0, atol=1e-12 * scale), (call, (got - want).abs().max().item())
            check_against_oracle(shape, bc, faces_h, rh, got.cpu().numpy())


def test_static_solve_largest_grid_matches_oracle():
    """8^3 = MG_STATIC_MAX_CELLS cells with a periodic axis (a handle would
    coarsen this grid, so only the oracle's dense solve compares here)."""
    shape, bc = (8, 8, 8), (1, 0, 1)
    faces, faces_h = faces_for(shape, bc, 5)
    rng = np.random.default_rng(11)
    for call in range(2):
        rh = rng.standard_normal(cells(shape))
        got = torch.full(cells(shape), float("nan"), dtype=torch.float64, device="cuda")
        rc = gbmg.coarse_solve_static(shape, bc, faces, torch.from_numpy(rh).cuda(), got)
        assert rc == gbmg.OK, gbmg.strerror(rc)
        check_against_oracle(shape, bc, faces_h, rh, got.cpu().numpy())


def test_static_solve_limits():
    shape, bc = (16, 16, 4), (0, 0, 0)  # 1024 cells > MG_STATIC_MAX_CELLS
    f = [torch.ones(cells(shape), dtype=torch.float64, device="cuda") for _ in range(3)]
    r = torch.zeros(cells(shape), dtype=torch.float64, device="cuda")
    e = torch.zeros_like(r)
    assert gbmg.coarse_solve_static(shape, bc, f, r, e) == gbmg.ETOOBIG
    # a non-positive coefficient off the walls is refused
    shape = (4, 4, 4)
    f = [torch.ones(cells(shape), dtype=torch.float64, device="cuda") for _ in range(3)]
    f[1][2, 2, 2] = -1.0
    r = torch.zeros(cells(shape), dtype=torch.float64, device="cuda")
    e = torch.zeros_like(r)
    assert gbmg.coarse_solve_static(shape, bc, f, r, e) == gbmg.EINVAL
