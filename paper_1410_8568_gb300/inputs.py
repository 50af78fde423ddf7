"""Seeded synthetic inputs for the variable-density pressure Poisson problem.

This module builds the *inputs* of the solve and nothing else: cell-centred
density fields rho and right-hand sides S of Eq. 9 (Shin, Chergui & Juric,
arXiv 1410.8568, Sec. 2.3).  It is shared by the CPU oracle (under ``oracle/``)
and the CUDA path, and it contains none of the solver's arithmetic: no face
coefficient (Eqs. 11-12), no operator (Eq. 10), no smoothing or grid transfer.
Each side turns ``rho`` into face coefficients with its own code.

Array convention (the library's documented layout): every cell array has numpy
shape ``(nz, ny, nx)`` in C order, so x is the fastest index and cell (i, j, k)
sits at ``i + nx * (j + ny * k)``.  Boundary codes: 0 = Neumann walls on both
ends of the axis, 1 = periodic.

Workloads (the paper's drop-splash runs, Sec. 3, cannot be reproduced without
the full Navier-Stokes + front-tracking code, so these stand in for them):

* ``config1``: 32^3, Neumann walls, a centred sphere R = 0.2, rho = 1000 inside
  and 1 outside, N(0,1) right-hand side with the mean removed.
* ``config2``: drop-splash field: a liquid film of depth 0.1 at the bottom and a
  drop of radius 0.125 centred at height 0.3, ratio 1000:1, periodic in x and y,
  Neumann in z; S = divergence of a random smooth velocity field made of 8
  Fourier modes, mean removed.
* ``config3``: the config2 geometry at 512^3 / 1024^3 plus 0-4 small droplets.
* ``config4_batch``: 64 independent spheres of uneven sizes.
* ``config5_stream``: a Poisson-arrival stream of drop/film requests.

The material blend rho = rho_G + (rho_L - rho_G) I is Eq. 8 of the paper; the
indicator I is a tanh of the signed distance spread over about 3 cells, which
stands in for the front-tracked distance function of Sec. 2.2.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

NEUMANN = 0
PERIODIC = 1

SEED_BASE = 14108568
ALLOWED_EDGES = (2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024)


def config_seed(config: int, index: int = 0) -> int:
    """Seed of workload ``config`` (1-5), repeat ``index``."""
    return SEED_BASE + 1000 * config + index


@dataclasses.dataclass
class Problem:
    """One solve: grid, boundary codes, cell density and right-hand side."""

    shape: tuple  # (nx, ny, nz)
    bc: tuple  # per axis (x, y, z): NEUMANN or PERIODIC
    rho: np.ndarray  # (nz, ny, nx) float64, cell-centred density
    rhs: np.ndarray  # (nz, ny, nx) float64, S of Eq. 9, zero mean
    length: tuple = (1.0, 1.0, 1.0)
    name: str = ""
    ratio: float = 1.0

    @property
    def h(self):
        return tuple(self.length[a] / self.shape[a] for a in range(3))

    @property
    def cells(self) -> int:
        return int(np.prod(self.shape))


def _centres(n: int, length: float) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) + 0.5) * (length / n)


def indicator(distance: np.ndarray, eps: float) -> np.ndarray:
    """Smoothed Heaviside: 1 in the liquid (distance < 0), 0 in the gas."""
    return 0.5 * (1.0 - np.tanh(distance / eps))


def blend(ind: np.ndarray, rho_liquid: float, rho_gas: float) -> np.ndarray:
    """Eq. 8 of the paper: b = b_1 + (b_2 - b_1) I, here for the density."""
    return rho_gas + (rho_liquid - rho_gas) * ind


def _liquid_distance(shape, length, zslice, film_depth, drops):
    """Signed distance to the liquid (negative inside) on planes ``zslice``."""
    nx, ny, nz = shape
    x = _centres(nx, length[0])[None, None, :]
    y = _centres(ny, length[1])[None, :, None]
    z = _centres(nz, length[2])[zslice][:, None, None]
    d = np.full((z.shape[0], ny, nx), np.inf)
    if film_depth is not None:
        d = np.minimum(d, np.broadcast_to(z - film_depth, d.shape))
    for (cx, cy, cz), r in drops:
        dist = np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) - r
        d = np.minimum(d, dist)
    return d


def density_field(shape, film_depth=None, drops=(), ratio=1000.0, eps_cells=1.5,
                  length=(1.0, 1.0, 1.0), zchunk=64):
    """Density on the cell centres of ``shape`` = (nx, ny, nz).

    Liquid = union of a bottom film of depth ``film_depth`` (None: no film) and
    spheres ``drops`` = [((cx, cy, cz), R), ...]; rho_L = ratio, rho_G = 1.
    """
    nx, ny, nz = shape
    h = min(length[a] / shape[a] for a in range(3))
    eps = eps_cells * h
    rho = np.empty((nz, ny, nx), dtype=np.float64)
    for k0 in range(0, nz, zchunk):
        sl = slice(k0, min(nz, k0 + zchunk))
        d = _liquid_distance(shape, length, sl, film_depth, drops)
        rho[sl] = blend(indicator(d, eps), ratio, 1.0)
    return rho


def rhs_white(shape, rng: np.random.Generator) -> np.ndarray:
    """N(0,1) per cell, mean removed."""
    nx, ny, nz = shape
    b = rng.standard_normal((nz, ny, nx))
    b -= b.mean()
    return b


def rhs_fourier_divergence(shape, bc, rng: np.random.Generator, modes: int = 8,
                           length=(1.0, 1.0, 1.0), zchunk=64) -> np.ndarray:
    """Discrete divergence of a random smooth MAC velocity field, mean removed.

    u_c(x) = sum_m a_{m,c} sin(2 pi k_m . x + phi_m) with integer wave vectors
    k_m in {1..4}^3, amplitudes a ~ N(0,1) and phases phi ~ U[0, 2 pi).  Each
    component is sampled at its own face centres; the normal velocity on a
    Neumann wall is set to zero.  S = sum over axes of (u_high - u_low) / h
    (time step 1), i.e. the source term of the projection method.
    """
    nx, ny, nz = shape
    kvec = rng.integers(1, 5, size=(modes, 3))
    amp = rng.standard_normal((modes, 3))
    phase = rng.uniform(0.0, 2.0 * math.pi, size=modes)
    h = [length[a] / shape[a] for a in range(3)]
    n = (nx, ny, nz)

    def coords(axis, face_axis):
        m = n[axis]
        if axis == face_axis:
            return np.arange(m + 1, dtype=np.float64) * h[axis]
        return (np.arange(m, dtype=np.float64) + 0.5) * h[axis]

    b = np.zeros((nz, ny, nx), dtype=np.float64)
    for comp in range(3):
        cx, cy, cz = coords(0, comp), coords(1, comp), coords(2, comp)
        for k0 in range(0, nz, zchunk):
            k1 = min(nz, k0 + zchunk)
            zs = cz[k0:k1 + 1] if comp == 2 else cz[k0:k1]
            u = np.zeros((zs.shape[0], cy.shape[0], cx.shape[0]))
            for m in range(modes):
                ex = np.exp(2j * math.pi * kvec[m, 0] * cx)[None, None, :]
                ey = np.exp(2j * math.pi * kvec[m, 1] * cy)[None, :, None]
                ez = np.exp(2j * math.pi * kvec[m, 2] * zs)[:, None, None]
                u += amp[m, comp] * np.imag(ex * ey * ez * np.exp(1j * phase[m]))
            if comp == 0:
                if bc[0] == NEUMANN:
                    u[:, :, 0] = 0.0
                    u[:, :, -1] = 0.0
                b[k0:k1] += (u[:, :, 1:] - u[:, :, :-1]) / h[0]
            elif comp == 1:
                if bc[1] == NEUMANN:
                    u[:, 0, :] = 0.0
                    u[:, -1, :] = 0.0
                b[k0:k1] += (u[:, 1:, :] - u[:, :-1, :]) / h[1]
            else:
                if bc[2] == NEUMANN:
                    if k0 == 0:
                        u[0] = 0.0
                    if k1 == nz:
                        u[-1] = 0.0
                b[k0:k1] += (u[1:] - u[:-1]) / h[2]
    b -= b.mean()
    return b


def fourier_velocity(shape, bc, rng: np.random.Generator, modes: int = 8,
                     length=(1.0, 1.0, 1.0), zchunk=64):
    """The random smooth velocity field behind ``rhs_fourier_divergence`` (same
    draws from ``rng``), sampled on the MAC faces in the low-face layout:
    component d of cell c is the normal velocity on c's LOW face along d.  On a
    Neumann axis the low face of the first cell is a wall (set to 0); the high
    wall of the last cell is not stored.  Sampling only: no divergence here.
    """
    nx, ny, nz = shape
    kvec = rng.integers(1, 5, size=(modes, 3))
    amp = rng.standard_normal((modes, 3))
    phase = rng.uniform(0.0, 2.0 * math.pi, size=modes)
    h = [length[a] / shape[a] for a in range(3)]
    n = (nx, ny, nz)

    def coords(axis, face_axis):
        m = n[axis]
        if axis == face_axis:
            return np.arange(m, dtype=np.float64) * h[axis]   # low faces
        return (np.arange(m, dtype=np.float64) + 0.5) * h[axis]

    out = []
    for comp in range(3):
        cx, cy, cz = coords(0, comp), coords(1, comp), coords(2, comp)
        u = np.zeros((nz, ny, nx))
        for k0 in range(0, nz, zchunk):
            k1 = min(nz, k0 + zchunk)
            zs = cz[k0:k1]
            for m in range(modes):
                ex = np.exp(2j * math.pi * kvec[m, 0] * cx)[None, None, :]
                ey = np.exp(2j * math.pi * kvec[m, 1] * cy)[None, :, None]
                ez = np.exp(2j * math.pi * kvec[m, 2] * zs)[:, None, None]
                u[k0:k1] += amp[m, comp] * np.imag(ex * ey * ez * np.exp(1j * phase[m]))
        if bc[comp] == NEUMANN:
            sl = [slice(None)] * 3
            sl[2 - comp] = 0
            u[tuple(sl)] = 0.0
        out.append(u)
    return out


def projection_problem(n: int = 128, ratio: float = 1000.0, dt: float = 1e-3):
    """Drop/film density of config2 with its Fourier velocity field: the
    non-projected velocity u* of one projection step."""
    shape = (n, n, n)
    rho = density_field(shape, 0.1, [((0.5, 0.5, 0.3), 0.125)], ratio)
    rng = np.random.default_rng(config_seed(2, n))
    u = fourier_velocity(shape, DROP_FILM_BC, rng)
    return shape, DROP_FILM_BC, rho, u, dt


def random_faces(shape, rng: np.random.Generator, lo=1e-3, hi=1.0):
    """Three arrays of log-uniform positive face values (operator tests)."""
    nx, ny, nz = shape
    out = []
    for _ in range(3):
        out.append(np.exp(rng.uniform(math.log(lo), math.log(hi), size=(nz, ny, nx))))
    return out


# ----------------------------------------------------------------------------
# The five workloads
# ----------------------------------------------------------------------------

def config1(n: int = 32, ratio: float = 1000.0, index: int = 0) -> Problem:
    """Centred sphere R = 0.2, rho 1000 inside, Neumann walls, N(0,1) RHS."""
    rng = np.random.default_rng(config_seed(1, index))
    shape = (n, n, n)
    rho = density_field(shape, None, [((0.5, 0.5, 0.5), 0.2)], ratio)
    return Problem(shape, (NEUMANN,) * 3, rho, rhs_white(shape, rng),
                   name=f"sphere_{n}^3_neumann_{int(ratio)}to1", ratio=ratio)


DROP_FILM_BC = (PERIODIC, PERIODIC, NEUMANN)


def config2(n: int = 128, ratio: float = 1000.0, index: int = 0) -> Problem:
    """Drop-splash field: film z < 0.1 plus a drop R = 0.125 at (0.5, 0.5, 0.3)."""
    rng = np.random.default_rng(config_seed(2, index))
    shape = (n, n, n)
    rho = density_field(shape, 0.1, [((0.5, 0.5, 0.3), 0.125)], ratio)
    rhs = rhs_fourier_divergence(shape, DROP_FILM_BC, rng)
    return Problem(shape, DROP_FILM_BC, rho, rhs,
                   name=f"drop_film_{n}^3_{int(ratio)}to1", ratio=ratio)


def _gas_droplets(rng, count, film_depth=0.1, drop=((0.5, 0.5, 0.3), 0.125)):
    out = []
    tries = 0
    while len(out) < count and tries < 10000:
        tries += 1
        r = rng.uniform(0.02, 0.05)
        c = rng.uniform(r, 1.0 - r, size=3)
        if c[2] - r < film_depth + 0.02:
            continue
        if np.linalg.norm(c - np.array(drop[0])) < drop[1] + r + 0.02:
            continue
        if any(np.linalg.norm(c - np.array(o[0])) < o[1] + r + 0.02 for o in out):
            continue
        out.append((tuple(float(v) for v in c), float(r)))
    return out


def config3(n: int = 512, ratio: float = 1000.0, index: int = 0) -> Problem:
    """Drop/film geometry of config2 plus 0-4 seeded droplets in the gas."""
    rng = np.random.default_rng(config_seed(3, index))
    extra = _gas_droplets(rng, int(rng.integers(0, 5)))
    shape = (n, n, n)
    rho = density_field(shape, 0.1, [((0.5, 0.5, 0.3), 0.125)] + extra, ratio)
    rhs = rhs_fourier_divergence(shape, DROP_FILM_BC, rng)
    return Problem(shape, DROP_FILM_BC, rho, rhs,
                   name=f"drop_film_{n}^3_{len(extra)}droplets_{int(ratio)}to1", ratio=ratio)


BATCH_EDGES = (32, 48, 64, 96, 128)


def config4_batch(count: int = 64, index: int = 0, edges=BATCH_EDGES):
    """Independent spheres of uneven sizes, Neumann walls, N(0,1) RHS."""
    rng = np.random.default_rng(config_seed(4, index))
    probs = []
    for g in range(count):
        n = int(rng.choice(edges))
        r = rng.uniform(0.05, 0.2)
        hh = 1.0 / n
        c = rng.uniform(r + 2 * hh, 1.0 - r - 2 * hh, size=3)
        ratio = float(rng.choice([10.0, 100.0, 1000.0]))
        shape = (n, n, n)
        rho = density_field(shape, None, [(tuple(c), r)], ratio)
        probs.append(Problem(shape, (NEUMANN,) * 3, rho, rhs_white(shape, rng),
                             name=f"batch{g}_sphere_{n}^3_{int(ratio)}to1", ratio=ratio))
    return probs


STREAM_EDGES = (64, 96, 128, 192, 256, 384, 512)


def stream_edge(rng, edges=STREAM_EDGES) -> int:
    """Edge length log-uniform in [64, 512], rounded (in log space) to an allowed size."""
    u = math.exp(rng.uniform(math.log(edges[0]), math.log(edges[-1])))
    return min(edges, key=lambda e: abs(math.log(e) - math.log(u)))


def config5_stream(count: int = 500, rate: float = 10.0, index: int = 0, edges=STREAM_EDGES):
    """Seeded request stream: list of (arrival_time_s, edge, ratio, seed).

    Arrivals are a Poisson process of ``rate`` requests per second.  The fields
    themselves are built lazily with :func:`stream_problem` so that a long
    stream does not hold every request in host memory.
    """
    rng = np.random.default_rng(config_seed(5, index))
    t = 0.0
    out = []
    for q in range(count):
        t += rng.exponential(1.0 / rate)
        n = stream_edge(rng, edges)
        ratio = math.exp(rng.uniform(math.log(10.0), math.log(1000.0)))
        out.append((t, n, ratio, config_seed(5, index) * 7919 + q))
    return out


def stream_problem(n: int, ratio: float, seed: int) -> Problem:
    """Drop/film request of the served stream (config2 geometry, given ratio)."""
    rng = np.random.default_rng(seed)
    shape = (n, n, n)
    rho = density_field(shape, 0.1, [((0.5, 0.5, 0.3), 0.125)], ratio)
    rhs = rhs_fourier_divergence(shape, DROP_FILM_BC, rng)
    return Problem(shape, DROP_FILM_BC, rho, rhs, name=f"stream_{n}^3_{ratio:.0f}to1", ratio=ratio)
