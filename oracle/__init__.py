"""FP64 CPU oracle for the variable-coefficient pressure multigrid.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the library.  The arithmetic
lives in ``mg_oracle.c`` (plain C, FP64); this module only marshals numpy arrays
through ctypes.  See the header of ``mg_oracle.c`` for what each function
computes and which passage of Shin, Chergui & Juric (arXiv 1410.8568, Sec. 2.3)
it follows.

Arrays are numpy float64 of shape (nz, ny, nx) (x fastest).  Face arrays hold
the coefficient of each cell's LOW face along the axis (Neumann wall entries are
ignored).  ``bc`` is a 3-tuple of 0 (Neumann walls) / 1 (periodic).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


class _Grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("h", ctypes.c_double * 3), ("bc", ctypes.c_int * 3)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER(ctypes.c_double)
        G = ctypes.POINTER(_Grid)
        L.oracle_num_threads.restype = ctypes.c_int
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        L.oracle_set_threads.restype = ctypes.c_int
        L.oracle_faces_from_density.argtypes = [G, P, ctypes.c_int, P, P, P]
        L.oracle_apply.argtypes = [G, P, P, P, P, P]
        L.oracle_residual.argtypes = [G, P, P, P, P, P, P]
        L.oracle_norm2.argtypes = [G, P]
        L.oracle_norm2.restype = ctypes.c_double
        L.oracle_mean.argtypes = [G, P]
        L.oracle_mean.restype = ctypes.c_double
        L.oracle_smooth_colour.argtypes = [G, P, P, P, P, P, ctypes.c_int, ctypes.c_double]
        L.oracle_can_coarsen.argtypes = [G]
        L.oracle_coarsen_faces.argtypes = [G, P, P, P, P, P, P]
        L.oracle_restrict.argtypes = [G, P, P]
        L.oracle_prolong_add.argtypes = [G, P, P]
        L.oracle_cell_alpha.argtypes = [G, P, P, P, P]
        L.oracle_divergence.argtypes = [G, P, P, P, ctypes.c_double, P]
        L.oracle_project.argtypes = [G, P, P, P, P, ctypes.c_double, P, P, P]
        L.oracle_prolong_flux_add.argtypes = [G, P, P, P]
        L.oracle_coarse_solve.argtypes = [G, P, P, P, P, P]
        L.oracle_solve.argtypes = [G, P, P, P, P, P, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, P,
                                   ctypes.POINTER(ctypes.c_int)]
        L.oracle_pcg_solve.argtypes = [G, P, P, P, P, P, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_double, ctypes.c_int, P,
                                       ctypes.POINTER(ctypes.c_int)]
        L.oracle_gmres.argtypes = [G, P, P, P, P, P, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_int)]
        L.oracle_gamma.argtypes = [P, ctypes.c_int]
        L.oracle_gamma.restype = ctypes.c_double
        _lib = L
    return _lib


def num_threads() -> int:
    return lib().oracle_num_threads()


def set_threads(n: int) -> int:
    """Threads of the following oracle calls; returns the number in effect."""
    return lib().oracle_set_threads(int(n))


def grid(shape, bc, length=(1.0, 1.0, 1.0)) -> _Grid:
    g = _Grid()
    for d in range(3):
        g.n[d] = int(shape[d])
        g.h[d] = float(length[d]) / int(shape[d])
        g.bc[d] = int(bc[d])
    return g


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _cells(shape):
    nx, ny, nz = shape
    return (nz, ny, nx)


def _arr(x, shape):
    a = np.ascontiguousarray(x, dtype=np.float64)
    assert a.shape == _cells(shape), (a.shape, shape)
    return a


def faces_from_density(shape, bc, rho, mode=0, length=(1.0, 1.0, 1.0)):
    """Face coefficients from cell density: harmonic (mode 0, Eqs. 11-12) or arithmetic (1)."""
    g = grid(shape, bc, length)
    rho = _arr(rho, shape)
    out = [np.empty(_cells(shape)) for _ in range(3)]
    lib().oracle_faces_from_density(ctypes.byref(g), _ptr(rho), mode, *[_ptr(a) for a in out])
    return out


def apply(shape, bc, faces, p, length=(1.0, 1.0, 1.0)):
    """(A p) of Eq. 10 divided by h^2."""
    g = grid(shape, bc, length)
    f = [_arr(a, shape) for a in faces]
    p = _arr(p, shape)
    out = np.empty(_cells(shape))
    lib().oracle_apply(ctypes.byref(g), *[_ptr(a) for a in f], _ptr(p), _ptr(out))
    return out


def residual(shape, bc, faces, b, p, length=(1.0, 1.0, 1.0)):
    g = grid(shape, bc, length)
    f = [_arr(a, shape) for a in faces]
    b = _arr(b, shape)
    p = _arr(p, shape)
    out = np.empty(_cells(shape))
    lib().oracle_residual(ctypes.byref(g), *[_ptr(a) for a in f], _ptr(b), _ptr(p), _ptr(out))
    return out


def smooth_colour(shape, bc, faces, b, p, colour, omega=1.0, length=(1.0, 1.0, 1.0)):
    """One red (colour 0) or black (1) relaxation half-sweep; returns the new p."""
    g = grid(shape, bc, length)
    f = [_arr(a, shape) for a in faces]
    b = _arr(b, shape)
    p = np.array(_arr(p, shape), copy=True)
    lib().oracle_smooth_colour(ctypes.byref(g), *[_ptr(a) for a in f], _ptr(b), _ptr(p), colour, omega)
    return p


def can_coarsen(shape) -> bool:
    g = grid(shape, (0, 0, 0))
    return bool(lib().oracle_can_coarsen(ctypes.byref(g)))


def coarse_shape(shape):
    return tuple(n // 2 for n in shape)


def coarsen_faces(shape, bc, faces):
    g = grid(shape, bc)
    f = [_arr(a, shape) for a in faces]
    cs = coarse_shape(shape)
    out = [np.empty(_cells(cs)) for _ in range(3)]
    lib().oracle_coarsen_faces(ctypes.byref(g), *[_ptr(a) for a in f], *[_ptr(a) for a in out])
    return out


def restrict(shape, bc, r):
    g = grid(shape, bc)
    r = _arr(r, shape)
    out = np.empty(_cells(coarse_shape(shape)))
    lib().oracle_restrict(ctypes.byref(g), _ptr(r), _ptr(out))
    return out


def prolong_add(shape, bc, e_coarse, x):
    """x + trilinear prolongation of the coarse error (returns a new array)."""
    g = grid(shape, bc)
    e = _arr(e_coarse, coarse_shape(shape))
    x = np.array(_arr(x, shape), copy=True)
    lib().oracle_prolong_add(ctypes.byref(g), _ptr(e), _ptr(x))
    return x


def cell_alpha(shape, bc, faces, length=(1.0, 1.0, 1.0)):
    """Cell coefficient of the flux-conserving prolongation: mean alpha of the
    cell's non-wall faces."""
    g = grid(shape, bc, length)
    f = [_arr(a, shape) for a in faces]
    out = np.empty(_cells(shape))
    lib().oracle_cell_alpha(ctypes.byref(g), *[_ptr(a) for a in f], _ptr(out))
    return out


def prolong_flux_add(shape, bc, alpha_coarse, e_coarse, x):
    """x + flux-conserving prolongation (Eqs. 13-14) of the coarse error, with
    the coarse cell coefficients alpha_coarse (returns a new array)."""
    g = grid(shape, bc)
    cs = coarse_shape(shape)
    a = _arr(alpha_coarse, cs)
    e = _arr(e_coarse, cs)
    x = np.array(_arr(x, shape), copy=True)
    lib().oracle_prolong_flux_add(ctypes.byref(g), _ptr(a), _ptr(e), _ptr(x))
    return x


def divergence(shape, bc, u, dt=1.0, length=(1.0, 1.0, 1.0)):
    """S = D u / dt of face velocities u = (ux, uy, uz) (low-face layout)."""
    g = grid(shape, bc, length)
    uu = [_arr(a, shape) for a in u]
    out = np.empty(_cells(shape))
    lib().oracle_divergence(ctypes.byref(g), *[_ptr(a) for a in uu], float(dt), _ptr(out))
    return out


def project(shape, bc, faces, p, u, dt=1.0, length=(1.0, 1.0, 1.0)):
    """u - dt alpha G p on every non-wall face (returns new arrays)."""
    g = grid(shape, bc, length)
    f = [_arr(a, shape) for a in faces]
    p = _arr(p, shape)
    out = [np.array(_arr(a, shape), copy=True) for a in u]
    lib().oracle_project(ctypes.byref(g), *[_ptr(a) for a in f], _ptr(p), float(dt), *[_ptr(a) for a in out])
    return out


def coarse_solve(shape, bc, faces, r, length=(1.0, 1.0, 1.0)):
    g = grid(shape, bc, length)
    f = [_arr(a, shape) for a in faces]
    r = _arr(r, shape)
    e = np.empty(_cells(shape))
    st = lib().oracle_coarse_solve(ctypes.byref(g), *[_ptr(a) for a in f], _ptr(r), _ptr(e))
    if st != 0:
        raise RuntimeError("oracle coarse solve failed: %d" % st)
    return e


def gmres(shape, bc, faces, r, tol=1e-12, max_it=500, m=30, length=(1.0, 1.0, 1.0)):
    """Restarted GMRES(m) for A e = r - mean(r); returns (e with zero mean,
    status 0 converged / 1 not, Arnoldi steps)."""
    g = grid(shape, bc, length)
    f = [_arr(a, shape) for a in faces]
    r = _arr(r, shape)
    e = np.empty(_cells(shape))
    its = ctypes.c_int(0)
    st = lib().oracle_gmres(ctypes.byref(g), *[_ptr(a) for a in f], _ptr(r), _ptr(e), float(tol), int(max_it),
                            int(m), ctypes.byref(its))
    return e, st, its.value


class SolveResult:
    def __init__(self, x, status, history):
        self.x = x
        self.status = status
        self.history = history
        self.cycles = len(history) - 1

    @property
    def gamma(self) -> float:
        return gamma(self.history)

    @property
    def rel_residual(self) -> float:
        return float(self.history[-1] / self._bnorm) if self._bnorm else 0.0


PROLONG_TRILINEAR, PROLONG_FLUX = 0, 1


def solve(shape, bc, faces, b, tol=1e-10, max_cycles=200, nu1=2, nu2=2, omega=1.0,
          x0=None, stagnate=False, length=(1.0, 1.0, 1.0), prolong=PROLONG_TRILINEAR) -> SolveResult:
    """V(nu1, nu2) multigrid to ||b - A x|| <= tol ||b|| (b projected to zero mean);
    ``prolong`` selects trilinear or flux-conserving (Eqs. 13-14) prolongation.

    With ``stagnate=True`` the iteration continues to rounding level (stops
    when three cycles in a row have not lowered the best residual by 10%): the
    result is then p*.
    """
    g = grid(shape, bc, length)
    f = [_arr(a, shape) for a in faces]
    b = _arr(b, shape)
    x = np.zeros(_cells(shape)) if x0 is None else np.array(_arr(x0, shape), copy=True)
    hist = np.zeros(max_cycles + 1)
    nc = ctypes.c_int(0)
    st = lib().oracle_solve(ctypes.byref(g), *[_ptr(a) for a in f], _ptr(b), _ptr(x), tol,
                            max_cycles, nu1, nu2, omega, 1 if stagnate else 0, int(prolong), _ptr(hist),
                            ctypes.byref(nc))
    if st < 0:
        raise RuntimeError("oracle solve failed: %d" % st)
    res = SolveResult(x, st, hist[: nc.value + 1].copy())
    bp = b - b.mean()
    res._bnorm = float(np.sqrt(np.sum(bp * bp)))
    return res


def pcg_solve(shape, bc, faces, b, tol=1e-10, max_it=200, nu1=2, nu2=2, omega=1.0, precond=True,
              x0=None, length=(1.0, 1.0, 1.0)) -> SolveResult:
    """Conjugate gradients on -A, preconditioned by one V(nu1, nu2) cycle
    (precond=True) or not; b projected to zero mean; history = recursive
    residual norms."""
    g = grid(shape, bc, length)
    f = [_arr(a, shape) for a in faces]
    b = _arr(b, shape)
    x = np.zeros(_cells(shape)) if x0 is None else np.array(_arr(x0, shape), copy=True)
    hist = np.zeros(max_it + 1)
    nit = ctypes.c_int(0)
    st = lib().oracle_pcg_solve(ctypes.byref(g), *[_ptr(a) for a in f], _ptr(b), _ptr(x), tol, max_it,
                                nu1, nu2, omega, 1 if precond else 0, _ptr(hist), ctypes.byref(nit))
    if st < 0:
        raise RuntimeError("oracle PCG failed: %d" % st)
    res = SolveResult(x, st, hist[: nit.value + 1].copy())
    bp = b - b.mean()
    res._bnorm = float(np.sqrt(np.sum(bp * bp)))
    return res


def solve_exact(shape, bc, faces, b, length=(1.0, 1.0, 1.0), max_cycles=400, nu1=2, nu2=2,
                prolong=PROLONG_TRILINEAR):
    """p*: the oracle multigrid iterated until the residual stops falling."""
    return solve(shape, bc, faces, b, tol=0.0, max_cycles=max_cycles, nu1=nu1, nu2=nu2,
                 stagnate=True, length=length, prolong=prolong)


def gamma(history) -> float:
    """Average reduction rate of Eq. 15."""
    h = np.ascontiguousarray(history, dtype=np.float64)
    return float(lib().oracle_gamma(_ptr(h), len(h) - 1))
