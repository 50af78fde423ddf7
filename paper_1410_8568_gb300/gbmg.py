"""ctypes binding of libgbmg.so (C ABI in include/gbmg.h).

Argument marshalling only: every step of the solve runs in the CUDA kernels of
the library.  Device arrays are torch CUDA tensors (float64 unless a call says
otherwise), shape (nz, ny, nx) or flat, contiguous; the binding passes their
data pointers and the current torch stream.  There is no CPU fallback: if the
library is missing or no GPU is present, the calls raise.

Shin, Chergui & Juric, arXiv 1410.8568, Sec. 2.3 (pressure equation Eq. 9,
discretisation Eqs. 10-12, V-cycle multigrid, reduction rate Eq. 15).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libgbmg.so")

OK, EINVAL, ENOMEM, ECUDA, ENOTCONV, EDIVERGED, ETIMEOUT, EBUSY, EAGAIN, EBUDGET, ESINGULAR, ENOTFOUND, ETOOBIG = range(13)
STATIC_MAX_CELLS = 512
NEUMANN, PERIODIC = 0, 1
FP64, MIXED = 0, 1
HARMONIC, ARITHMETIC = 0, 1
K_SMOOTH, K_RESTRICT, K_PROLONG, K_COARSE, K_RESIDUAL, K_OTHER, K_TAIL, K_RESIDUAL0 = range(8)
TILES_AUTO, TILES_ROWS, TILE_VARIANTS = -1, 0, 7
PROLONG_TRILINEAR, PROLONG_FLUX = 0, 1
SOLVER_MG, SOLVER_PCG = 0, 1
COARSE_AUTO, COARSE_GMRES = 0, 1
OUTER_FP64, OUTER_XP = 0, 1
MAX_COARSE, MAX_COARSE_GMRES = 512, 32768
TILE_HALF, TILE_RESTRICT, TILE_PROLONG, TILE_SWEEP = 0, 1, 2, 3
SWEEP_AUTO, SWEEP_HALF, SWEEP_VARIANTS = -1, 0, 11


class MGError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__("%s: %s (status %d, cuda error %d)" % (what, strerror(code), code, last_cuda_error()))


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
                ("bc", ctypes.c_int * 3)]


class Params(ctypes.Structure):
    _fields_ = [("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("omega", ctypes.c_double),
                ("max_iters", ctypes.c_int), ("precision", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("inner_cycles", ctypes.c_int), ("solver", ctypes.c_int), ("prolongation", ctypes.c_int),
                ("tiles", ctypes.c_int), ("coarse_solver", ctypes.c_int), ("coarse_max_iters", ctypes.c_int),
                ("coarse_tol", ctypes.c_double), ("adaptive_cycles", ctypes.c_int), ("outer", ctypes.c_int),
                ("sweep", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int), ("rel_res", ctypes.c_double),
                ("res0", ctypes.c_double), ("res", ctypes.c_double), ("gamma", ctypes.c_double),
                ("bnorm", ctypes.c_double), ("rhs_mean", ctypes.c_double), ("ms", ctypes.c_double),
                ("steps", ctypes.c_int), ("admit_tick", ctypes.c_int64), ("finish_tick", ctypes.c_int64),
                ("inflight_at_admit", ctypes.c_int), ("lane", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None
_V = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_P = ctypes.POINTER


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libgbmg.so is not built (run python -m paper_1410_8568_gb300.build)")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "mg_strerror": (ctypes.c_char_p, [_I]),
            "mg_last_cuda_error": (_I, []),
            "mg_params_default": (_I, [_P(Params)]),
            "mg_faces_from_density": (_I, [_P(Grid), _V, _I, _V, _V, _V, _V]),
            "mg_create": (_I, [_P(Grid), _V, _V, _V, _P(Params), _V, _P(_V)]),
            "mg_set_faces": (_I, [_V, _V, _V, _V]),
            "mg_set_density": (_I, [_V, _V, _I]),
            "mg_solve": (_I, [_V, _V, _V, _D, _P(Stats)]),
            "mg_solve_host": (_I, [_V, _V, _V, _D, _P(Stats)]),
            "mg_step_host": (_I, [_V, _V, _I, _V, _V, _D, _P(Stats)]),
            "mg_destroy": (_I, [_V]),
            "mg_batch_create": (_I, [_P(_V), _I, _P(_V)]),
            "mg_batch_solve": (_I, [_V, _P(_V), _P(_V), _P(_D), _P(Stats)]),
            "mg_batch_destroy": (_I, [_V]),
            "mg_server_create": (_I, [ctypes.c_size_t, _I, _P(Params), _V, _P(_V)]),
            "mg_submit": (_I, [_V, _P(Grid), _V, _V, _V, _V, _V, _D, _P(ctypes.c_int64)]),
            "mg_poll": (_I, [_V, ctypes.c_int64, _P(Stats)]),
            "mg_server_drain": (_I, [_V]),
            "mg_server_info": (_I, [_V, _P(ctypes.c_int64), _P(ctypes.c_size_t), _P(ctypes.c_size_t), _P(_I)]),
            "mg_server_destroy": (_I, [_V]),
            "mg_num_levels": (_I, [_V, _P(_I)]),
            "mg_level_shape": (_I, [_V, _I, _P(_I), _P(_I), _P(_I)]),
            "mg_level_faces": (_I, [_V, _I, _V, _V, _V]),
            "mg_level_faces32": (_I, [_V, _I, _V, _V, _V]),
            "mg_level_cell_alpha": (_I, [_V, _I, _V]),
            "mg_divergence": (_I, [_V, _V, _V, _V, _D, _V]),
            "mg_project": (_I, [_V, _V, _D, _V, _V, _V]),
            "mg_projection_step": (_I, [_V, _V, _V, _V, _D, _V, _V, _D, _P(Stats)]),
            "mg_apply": (_I, [_V, _I, _I, _V, _V]),
            "mg_smooth": (_I, [_V, _I, _I, _V, _V, _I]),
            "mg_restrict_residual": (_I, [_V, _I, _I, _V, _V, _V]),
            "mg_prolong": (_I, [_V, _I, _I, _V, _V]),
            "mg_coarse_solve": (_I, [_V, _I, _V, _V]),
            "mg_profile_enable": (_I, [_V, _I]),
            "mg_profile_read": (_I, [_V, _I, _I, _P(ctypes.c_int64), _P(_D)]),
            "mg_memory_bytes": (_I, [_V, _P(ctypes.c_size_t)]),
            "mg_memory_estimate": (_I, [_P(Grid), _P(Params), _P(ctypes.c_size_t)]),
            "mg_coarse_solve_static": (_I, [_P(Grid), _V, _V, _V, _V, _V, _V]),
            "mg_tile_choice": (_I, [_V, _I, _I, _P(_I)]),
            "mg_tile_shape": (_I, [_I, _P(_I), _P(_I)]),
            "mg_tune_cache_clear": (_I, []),
            "mg_tune_cache_save": (_I, [ctypes.c_char_p]),
            "mg_tune_cache_load": (_I, [ctypes.c_char_p, _P(_I)]),
            "mg_tune_cache_size": (_I, [_P(_I)]),
            "mg_handle_params": (_I, [_V, _P(Params)]),
            "mg_probe_fp64_rate": (_I, [_I, _I, _P(_D), _V]),
            "mg_set_wait_limit": (_I, [_V, ctypes.c_longlong]),
            "mg_sweep_shape": (_I, [_I, _P(_I), _P(_I), _P(_I)]),
            "mg_smooth_onepass": (_I, [_V, _I, _I, _V, _V, _V, _I, _I]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().mg_strerror(code).decode()


def last_cuda_error() -> int:
    return lib().mg_last_cuda_error()


def check(rc: int, what: str = "gbmg") -> int:
    if rc != OK:
        raise MGError(rc, what)
    return rc


def make_grid(shape, bc, length=(1.0, 1.0, 1.0)) -> Grid:
    g = Grid()
    g.nx, g.ny, g.nz = (int(v) for v in shape)
    g.lx, g.ly, g.lz = (float(v) for v in length)
    for d in range(3):
        g.bc[d] = int(bc[d])
    return g


def make_params(precision=MIXED, nu1=2, nu2=2, omega=1.0, max_iters=100, use_graph=True,
                inner_cycles=None, tiles=None, prolongation=None, solver=None, coarse_solver=None,
                coarse_tol=None, coarse_max_iters=None, adaptive_cycles=None, outer=None,
                sweep=None) -> Params:
    p = Params()
    lib().mg_params_default(ctypes.byref(p))
    p.nu1, p.nu2, p.omega = int(nu1), int(nu2), float(omega)
    p.max_iters = int(max_iters)
    p.precision = int(precision)
    p.use_graph = 1 if use_graph else 0
    if inner_cycles is not None:
        p.inner_cycles = int(inner_cycles)
    if tiles is not None:
        p.tiles = int(tiles)
    if prolongation is not None:
        p.prolongation = int(prolongation)
    if solver is not None:
        p.solver = int(solver)
    if coarse_solver is not None:
        p.coarse_solver = int(coarse_solver)
    if coarse_tol is not None:
        p.coarse_tol = float(coarse_tol)
    if coarse_max_iters is not None:
        p.coarse_max_iters = int(coarse_max_iters)
    if adaptive_cycles is not None:
        p.adaptive_cycles = int(adaptive_cycles)
    if outer is not None:
        p.outer = int(outer)
    if sweep is not None:
        p.sweep = int(sweep)
    return p


def sweep_shape(variant):
    """(threads per block, planes per block, tile_x) of one-pass sweep shape
    `variant`; tile_x = 0 for the whole-row shapes, else the cells along x of a
    staged shape's tile (FP32 cycles only)."""
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    check(lib().mg_sweep_shape(int(variant), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
          "mg_sweep_shape")
    return (a.value, b.value, c.value)


def tile_shape(variant):
    """(threads per block, items per thread) of launch shape `variant`."""
    a, b = ctypes.c_int(), ctypes.c_int()
    check(lib().mg_tile_shape(int(variant), ctypes.byref(a), ctypes.byref(b)), "mg_tile_shape")
    return (a.value, b.value)


def probe_fp64_rate(iters=20000, repeats=3, stream=None):
    """Measured FP64 fused multiply-add rate of the current device (FMA/s)."""
    out = ctypes.c_double()
    check(lib().mg_probe_fp64_rate(int(iters), int(repeats), ctypes.byref(out), _stream(stream)),
          "mg_probe_fp64_rate")
    return out.value


def tune_cache_clear():
    """Forget the autotuner's cached launch shapes."""
    check(lib().mg_tune_cache_clear(), "mg_tune_cache_clear")


def tune_cache_save(path):
    check(lib().mg_tune_cache_save(os.fsencode(path)), "mg_tune_cache_save")


def tune_cache_load(path) -> int:
    n = ctypes.c_int()
    check(lib().mg_tune_cache_load(os.fsencode(path), ctypes.byref(n)), "mg_tune_cache_load")
    return n.value


def tune_cache_size() -> int:
    n = ctypes.c_int()
    check(lib().mg_tune_cache_size(ctypes.byref(n)), "mg_tune_cache_size")
    return n.value


def _ptr(t, cells=None, dtype=None):
    """Data pointer of a contiguous CUDA tensor (checked)."""
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError("expected %s, got %s" % (dtype, t.dtype))
    if cells is not None and t.numel() != cells:
        raise ValueError("expected %d elements, got %d" % (cells, t.numel()))
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a: np.ndarray, cells: int):
    if a.dtype != np.float64 or not a.flags.c_contiguous or a.size != cells:
        raise ValueError("host arrays must be contiguous float64 with %d elements" % cells)
    return ctypes.c_void_p(a.ctypes.data)


def _stream(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def faces_from_density(shape, bc, rho, ax, ay, az, mode=HARMONIC, length=(1.0, 1.0, 1.0), stream=None):
    """Face coefficients of Eqs. 11-12 from cell density (device tensors)."""
    import torch

    g = make_grid(shape, bc, length)
    n = int(np.prod(shape))
    d = torch.float64
    check(lib().mg_faces_from_density(ctypes.byref(g), _ptr(rho, n, d), int(mode), _ptr(ax, n, d),
                                      _ptr(ay, n, d), _ptr(az, n, d), _stream(stream)),
          "mg_faces_from_density")


class Solver:
    """One grid's hierarchy (mg_create ... mg_destroy)."""

    def __init__(self, shape, bc, faces=None, rho=None, face_mode=HARMONIC, length=(1.0, 1.0, 1.0),
                 precision=MIXED, nu1=2, nu2=2, omega=1.0, max_iters=100, use_graph=True, stream=None,
                 inner_cycles=None, tiles=None, prolongation=None, solver=None, coarse_solver=None,
                 coarse_tol=None, coarse_max_iters=None, adaptive_cycles=None, outer=None, sweep=None):
        import torch

        self.shape = tuple(int(v) for v in shape)
        self.bc = tuple(int(v) for v in bc)
        self.length = tuple(float(v) for v in length)
        self.cells = int(np.prod(self.shape))
        self.precision = precision
        self.grid = make_grid(self.shape, self.bc, self.length)
        self.params = make_params(precision, nu1, nu2, omega, max_iters, use_graph, inner_cycles, tiles,
                                  prolongation, solver, coarse_solver, coarse_tol, coarse_max_iters,
                                  adaptive_cycles, outer, sweep)
        self._h = ctypes.c_void_p()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        if faces is None:
            if rho is None:
                raise ValueError("give face coefficients or a density")
            nz, ny, nx = self.shape[2], self.shape[1], self.shape[0]
            faces = [torch.empty((nz, ny, nx), dtype=torch.float64, device=rho.device) for _ in range(3)]
            faces_from_density(self.shape, self.bc, rho, *faces, mode=face_mode, length=self.length,
                               stream=self.stream)
        ax, ay, az = (_ptr(f, self.cells, torch.float64) for f in faces)
        check(lib().mg_create(ctypes.byref(self.grid), ax, ay, az, ctypes.byref(self.params),
                              ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self._h)), "mg_create")

    # -- life cycle --------------------------------------------------------
    def close(self):
        if self._h:
            lib().mg_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    # -- coefficients ------------------------------------------------------
    def set_faces(self, ax, ay, az):
        import torch

        d = torch.float64
        check(lib().mg_set_faces(self._h, _ptr(ax, self.cells, d), _ptr(ay, self.cells, d),
                                 _ptr(az, self.cells, d)), "mg_set_faces")

    def set_density(self, rho, mode=HARMONIC):
        import torch

        check(lib().mg_set_density(self._h, _ptr(rho, self.cells, torch.float64), int(mode)), "mg_set_density")

    # -- solves -----------------------------------------------------------
    def solve(self, rhs, p, tol=1e-10, raise_on_error=True) -> Stats:
        """Solve in place into p (warm start).  Returns the statistics."""
        import torch

        st = Stats()
        rc = lib().mg_solve(self._h, _ptr(rhs, self.cells, torch.float64), _ptr(p, self.cells, torch.float64),
                            float(tol), ctypes.byref(st))
        if raise_on_error and rc not in (OK, ENOTCONV, EDIVERGED):
            check(rc, "mg_solve")
        st.status = rc if rc not in (OK, ENOTCONV, EDIVERGED) else st.status
        return st

    # -- projection step around the solve (MAC face velocities, low-face layout)
    def divergence(self, u, dt, S):
        """S = D u / dt for face velocities u = (ux, uy, uz)."""
        import torch

        d = torch.float64
        check(lib().mg_divergence(self._h, *[_ptr(a, self.cells, d) for a in u], float(dt),
                                  _ptr(S, self.cells, d)), "mg_divergence")

    def project(self, p, dt, u):
        """u -= dt alpha G p in place."""
        import torch

        d = torch.float64
        check(lib().mg_project(self._h, _ptr(p, self.cells, d), float(dt), *[_ptr(a, self.cells, d) for a in u]),
              "mg_project")

    def projection_step(self, u, dt, p, S, tol=1e-10) -> Stats:
        """S = D u / dt, solve A p = S (p warm start), u -= dt alpha G p."""
        import torch

        d = torch.float64
        st = Stats()
        rc = lib().mg_projection_step(self._h, *[_ptr(a, self.cells, d) for a in u], float(dt),
                                      _ptr(p, self.cells, d), _ptr(S, self.cells, d), float(tol), ctypes.byref(st))
        if rc not in (OK, ENOTCONV):
            check(rc, "mg_projection_step")
        st.status = rc
        return st

    def solve_host(self, rhs: np.ndarray, p: np.ndarray, tol=1e-10) -> Stats:
        st = Stats()
        rc = lib().mg_solve_host(self._h, _hptr(rhs, self.cells), _hptr(p, self.cells), float(tol),
                                 ctypes.byref(st))
        if rc not in (OK, ENOTCONV, EDIVERGED):
            check(rc, "mg_solve_host")
        return st

    def step_host(self, rho: np.ndarray, rhs: np.ndarray, p: np.ndarray, tol=1e-10, mode=HARMONIC) -> Stats:
        st = Stats()
        rc = lib().mg_step_host(self._h, _hptr(rho, self.cells), int(mode), _hptr(rhs, self.cells),
                                _hptr(p, self.cells), float(tol), ctypes.byref(st))
        if rc not in (OK, ENOTCONV, EDIVERGED):
            check(rc, "mg_step_host")
        return st

    def resolved_params(self) -> dict:
        """The handle's parameters with defaults resolved (e.g. inner_cycles)."""
        p = Params()
        check(lib().mg_handle_params(self._h, ctypes.byref(p)), "mg_handle_params")
        return {f: getattr(p, f) for f, _ in Params._fields_}

    def set_wait_limit(self, polls):
        """Polls of the bottom-of-cycle kernel's staging wait before it gives up
        (0: at once; the solve then reports ETIMEOUT).  A test aid."""
        check(lib().mg_set_wait_limit(self._h, int(polls)), "mg_set_wait_limit")

    def tile_choice(self, kind, level) -> int:
        """Launch shape used for kernel `kind` (TILE_*) on `level`."""
        v = ctypes.c_int()
        check(lib().mg_tile_choice(self._h, int(kind), int(level), ctypes.byref(v)), "mg_tile_choice")
        return v.value

    # -- single steps (unit checks) ----------------------------------------
    def num_levels(self) -> int:
        v = ctypes.c_int()
        check(lib().mg_num_levels(self._h, ctypes.byref(v)))
        return v.value

    def level_shape(self, level):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(lib().mg_level_shape(self._h, int(level), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return (a.value, b.value, c.value)

    def level_faces(self, level):
        import torch

        nx, ny, nz = self.level_shape(level)
        out = [torch.empty((nz, ny, nx), dtype=torch.float64, device="cuda") for _ in range(3)]
        check(lib().mg_level_faces(self._h, int(level), *[_ptr(o) for o in out]), "mg_level_faces")
        return out

    def level_faces32(self, level):
        """FP32 copies of the level's scaled faces (mixed-precision handles)."""
        import torch

        nx, ny, nz = self.level_shape(level)
        out = [torch.empty((nz, ny, nx), dtype=torch.float32, device="cuda") for _ in range(3)]
        check(lib().mg_level_faces32(self._h, int(level), *[_ptr(o) for o in out]), "mg_level_faces32")
        return out

    def level_cell_alpha(self, level):
        """Cell coefficients of the flux-conserving prolongation on `level` (FP64)."""
        import torch

        nx, ny, nz = self.level_shape(level)
        out = torch.empty((nz, ny, nx), dtype=torch.float64, device="cuda")
        check(lib().mg_level_cell_alpha(self._h, int(level), _ptr(out)), "mg_level_cell_alpha")
        return out

    def apply(self, level, x, y, prec=FP64):
        check(lib().mg_apply(self._h, int(level), int(prec), _ptr(x), _ptr(y)), "mg_apply")

    def smooth(self, level, b, x, sweeps, prec=FP64):
        check(lib().mg_smooth(self._h, int(level), int(prec), _ptr(b), _ptr(x), int(sweeps)), "mg_smooth")

    def smooth_onepass(self, level, b, x, work, sweeps, prec=FP64, variant=0):
        """`sweeps` one-pass red-black sweeps alternating between x and work
        (the result is in x after an even number, in work after an odd one)."""
        check(lib().mg_smooth_onepass(self._h, int(level), int(prec), _ptr(b), _ptr(x), _ptr(work), int(sweeps),
                                      int(variant)), "mg_smooth_onepass")

    def restrict_residual(self, level, b, x, coarse_b, prec=FP64):
        check(lib().mg_restrict_residual(self._h, int(level), int(prec), _ptr(b), _ptr(x), _ptr(coarse_b)),
              "mg_restrict_residual")

    def prolong(self, level, coarse_e, x, prec=FP64):
        check(lib().mg_prolong(self._h, int(level), int(prec), _ptr(coarse_e), _ptr(x)), "mg_prolong")

    def coarse_solve(self, r, e, prec=FP64):
        check(lib().mg_coarse_solve(self._h, int(prec), _ptr(r), _ptr(e)), "mg_coarse_solve")

    # -- profiling / memory --------------------------------------------------
    def profile(self, enable=True):
        check(lib().mg_profile_enable(self._h, 1 if enable else 0))

    def profile_read(self, kind, level):
        n = ctypes.c_int64()
        ms = ctypes.c_double()
        check(lib().mg_profile_read(self._h, int(kind), int(level), ctypes.byref(n), ctypes.byref(ms)))
        return n.value, ms.value

    def memory_bytes(self) -> int:
        v = ctypes.c_size_t()
        check(lib().mg_memory_bytes(self._h, ctypes.byref(v)))
        return v.value


def coarse_solve_static(shape, bc, faces, r, e, length=(1.0, 1.0, 1.0), stream=None) -> int:
    """Exact FP64 solve of a grid of at most STATIC_MAX_CELLS cells without any
    device allocation (mg_coarse_solve_static).  Returns the status code."""
    import torch

    g = make_grid(shape, bc, length)
    n = int(np.prod(shape))
    d = torch.float64
    return lib().mg_coarse_solve_static(ctypes.byref(g), *[_ptr(f, n, d) for f in faces], _ptr(r, n, d),
                                        _ptr(e, n, d), _stream(stream))


def memory_estimate(shape, bc, precision=MIXED, length=(1.0, 1.0, 1.0), outer=None) -> int:
    g = make_grid(shape, bc, length)
    p = make_params(precision, outer=outer)
    v = ctypes.c_size_t()
    check(lib().mg_memory_estimate(ctypes.byref(g), ctypes.byref(p), ctypes.byref(v)), "mg_memory_estimate")
    return v.value


class Batch:
    """Several solvers advanced together (mg_batch_*)."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        arr = (ctypes.c_void_p * len(self.solvers))(*[s.handle.value for s in self.solvers])
        self._b = ctypes.c_void_p()
        check(lib().mg_batch_create(arr, len(self.solvers), ctypes.byref(self._b)), "mg_batch_create")

    def solve(self, rhs_list, p_list, tol=1e-10):
        import torch

        G = len(self.solvers)
        tols = list(tol) if hasattr(tol, "__len__") else [tol] * G
        r = (ctypes.c_void_p * G)(*[_ptr(t, s.cells, torch.float64).value for t, s in zip(rhs_list, self.solvers)])
        p = (ctypes.c_void_p * G)(*[_ptr(t, s.cells, torch.float64).value for t, s in zip(p_list, self.solvers)])
        tl = (ctypes.c_double * G)(*[float(v) for v in tols])
        st = (Stats * G)()
        rc = lib().mg_batch_solve(self._b, r, p, tl, st)
        if rc not in (OK, ENOTCONV, EDIVERGED):
            check(rc, "mg_batch_solve")
        return list(st)

    def close(self):
        if self._b:
            lib().mg_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop (mg_server_*)."""

    def __init__(self, hbm_budget_bytes, max_slots=16, precision=MIXED, max_iters=100, stream=None,
                 solver=None, prolongation=None, outer=None):
        self.params = make_params(precision, max_iters=max_iters, solver=solver, prolongation=prolongation,
                                  outer=outer)
        self._s = ctypes.c_void_p()
        st = ctypes.c_void_p(stream.cuda_stream) if stream is not None else ctypes.c_void_p()
        check(lib().mg_server_create(int(hbm_budget_bytes), int(max_slots), ctypes.byref(self.params), st,
                                     ctypes.byref(self._s)), "mg_server_create")
        self._keep = {}

    def submit(self, shape, bc, faces, rhs, p, tol=1e-10, length=(1.0, 1.0, 1.0)) -> int:
        g = make_grid(shape, bc, length)
        t = ctypes.c_int64()
        check(lib().mg_submit(self._s, ctypes.byref(g), *[_ptr(f) for f in faces], _ptr(rhs), _ptr(p),
                              float(tol), ctypes.byref(t)), "mg_submit")
        self._keep[t.value] = (faces, rhs, p)
        return t.value

    def poll(self, ticket):
        """None while pending, else (status, Stats)."""
        st = Stats()
        rc = lib().mg_poll(self._s, int(ticket), ctypes.byref(st))
        if rc == EAGAIN:
            return None
        if rc == ENOTFOUND:
            raise MGError(rc, "mg_poll")
        self._keep.pop(int(ticket), None)
        return rc, st

    def drain(self):
        return lib().mg_server_drain(self._s)

    def info(self):
        c, b, pk, m = ctypes.c_int64(), ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_int()
        check(lib().mg_server_info(self._s, ctypes.byref(c), ctypes.byref(b), ctypes.byref(pk), ctypes.byref(m)))
        return {"completed": c.value, "bytes_in_use": b.value, "peak_bytes": pk.value, "max_in_flight": m.value}

    def close(self):
        if self._s:
            rc = lib().mg_server_destroy(self._s)
            if rc == OK:
                self._s = ctypes.c_void_p()
            return rc
        return OK

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
