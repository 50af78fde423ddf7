"""The allocation-free small-grid solve (mg_coarse_solve_static) against the
coarsest-grid solve of a handle (mg_coarse_solve), through the C ABI.

mg_coarse_solve_static exists for callers that cannot allocate device memory
when they need a solve (during stream capture, in a fixed-budget real-time
loop, or under a host allocator that owns the device memory): it keeps its
scratch in a static device array of the library.  This file is collected last
so that a failure here leaves every other test already run; it passes alone in
a fresh process as well as after the other tests.
"""
import numpy as np
import pytest

from paper_1410_8568_gb300 import gbmg
from paper_1410_8568_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def cells(shape):
    return (shape[2], shape[1], shape[0])


def faces_for(shape, bc, seed):
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.3, 0.7, size=3)
    rho = I.density_field(shape, None, [(tuple(c), 0.3)], 1000.0, eps_cells=1.0)
    out = [torch.empty(cells(shape), dtype=torch.float64, device="cuda") for _ in range(3)]
    gbmg.faces_from_density(shape, bc, torch.from_numpy(rho).cuda(), *out)
    return out


# grids that are their own coarsest level (no axis can be halved), so a
# handle's mg_coarse_solve acts on the same operator
@pytest.mark.parametrize("shape,bc", [((8, 8, 2), (1, 1, 0)), ((4, 3, 4), (0, 0, 0)), ((6, 3, 5), (1, 0, 1)),
                                      ((16, 2, 8), (0, 1, 0))])
def test_static_solve_matches_handle_twice(shape, bc):
    faces = faces_for(shape, bc, sum(shape))
    with gbmg.Solver(shape, bc, faces=faces, precision=gbmg.FP64) as S:
        assert S.num_levels() == 1
        rng = np.random.default_rng(7)
        for call in range(2):  # two calls in a row share the static scratch array
            r = torch.from_numpy(rng.standard_normal(cells(shape))).cuda()
            want = torch.empty_like(r)
            S.coarse_solve(r, want, prec=gbmg.FP64)
            got = torch.full_like(r, float("nan"))
            rc = gbmg.coarse_solve_static(shape, bc, faces, r, got)
            assert rc == gbmg.OK, gbmg.strerror(rc)
            torch.cuda.synchronize()
            scale = want.abs().max().item()
            assert torch.allclose(got, want, rtol=0, atol=1e-12 * scale), (call, (got - want).abs().max().item())


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
