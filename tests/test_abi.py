"""The C-ABI library builds, loads and exports every entry point of include/gbmg.h.

No compute call is made here (no GPU in the build container)."""
import ctypes
import os
import re

import pytest

from paper_1410_8568_gb300 import build as B
from paper_1410_8568_gb300 import gbmg

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gbmg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w \*]*?\b(mg_\w+)\s*\(", text, flags=re.M)))


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    assert os.path.exists(path)
    L = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 30, names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    gbmg.lib()
    import inspect
    src = inspect.getsource(gbmg)
    missing = [n for n in declared_functions() if '"%s"' % n not in src]
    assert not missing, missing


def test_host_only_calls():
    """Calls that need no device: messages, defaults, size rules, estimates."""
    L = gbmg.lib()
    assert gbmg.strerror(gbmg.ENOTCONV).startswith("not converged")
    p = gbmg.Params()
    assert L.mg_params_default(ctypes.byref(p)) == 0
    assert (p.nu1, p.nu2, p.omega, p.precision, p.use_graph) == (2, 2, 1.0, gbmg.MIXED, 1)
    # mixed precision, multigrid iteration: about 58 B per finest cell for the
    # levels and the FP64 outer iteration ...
    est = gbmg.memory_estimate((64, 64, 64), (1, 1, 0))
    assert 64 ** 3 * 52 < est < 64 ** 3 * 70
    # ... plus 32 B for the extended-precision outer iteration (three-float
    # iterate, float-pair b, low parts of the finest faces)
    est_xp = gbmg.memory_estimate((64, 64, 64), (1, 1, 0), outer=gbmg.OUTER_XP)
    assert est_xp - est == 64 ** 3 * 32
    with pytest.raises(gbmg.MGError) as e:
        gbmg.memory_estimate((64, 64, 64), (1, 1, 0), outer=2)
    assert e.value.code == gbmg.EINVAL
    # FP64 cycles keep the FP64 outer iteration only, and the inverse
    # diagonals of the relaxed levels (8 B per cell of every level but the coarsest)
    est64 = gbmg.memory_estimate((64, 64, 64), (1, 1, 0), precision=gbmg.FP64)
    assert 64 ** 3 * 60 < est64 < 64 ** 3 * 76
    # a coarsest grid above 512 cells takes GMRES (2 x 2 x 256 cannot be coarsened) ...
    assert gbmg.memory_estimate((2, 2, 256), (0, 0, 0)) > 0
    # ... up to 32768 cells
    with pytest.raises(gbmg.MGError) as e:
        gbmg.memory_estimate((2, 2, 16384), (0, 0, 0))
    assert e.value.code == gbmg.EINVAL
    with pytest.raises(gbmg.MGError):
        gbmg.memory_estimate((1, 8, 8), (0, 0, 0))
    # level read-back without a handle is refused before any device call
    buf = (ctypes.c_double * 8)()
    fbuf = (ctypes.c_float * 8)()
    assert L.mg_level_faces(None, 0, buf, buf, buf) == gbmg.EINVAL
    assert L.mg_level_faces32(None, 0, fbuf, fbuf, fbuf) == gbmg.EINVAL


def test_tile_shapes_and_params():
    """Launch-shape table and the tiles parameter (host only)."""
    L = gbmg.lib()
    p = gbmg.Params()
    assert L.mg_params_default(ctypes.byref(p)) == 0
    assert p.tiles == gbmg.TILES_AUTO
    shapes = [gbmg.tile_shape(v) for v in range(gbmg.TILE_VARIANTS)]
    assert shapes[0] == (256, 1)  # row tiling: 8 rows of one warp
    assert len(set(shapes[1:])) == gbmg.TILE_VARIANTS - 1
    for threads, q in shapes:
        assert threads % 32 == 0 and 32 <= threads <= 1024 and q >= 1
    with pytest.raises(gbmg.MGError):
        gbmg.tile_shape(gbmg.TILE_VARIANTS)
    g = gbmg.make_grid((32, 32, 32), (0, 0, 0))
    size = ctypes.c_size_t()
    for tiles in (gbmg.TILES_AUTO, gbmg.TILES_ROWS, gbmg.TILE_VARIANTS - 1):
        p.tiles = tiles
        assert L.mg_memory_estimate(ctypes.byref(g), ctypes.byref(p), ctypes.byref(size)) == gbmg.OK
    for tiles in (-2, gbmg.TILE_VARIANTS):
        p.tiles = tiles
        assert L.mg_memory_estimate(ctypes.byref(g), ctypes.byref(p), ctypes.byref(size)) == gbmg.EINVAL
    assert gbmg.lib().mg_tune_cache_clear() == gbmg.OK


def test_sweep_shapes_and_param():
    """One-pass sweep shapes and the sweep parameter (host only)."""
    L = gbmg.lib()
    p = gbmg.Params()
    assert L.mg_params_default(ctypes.byref(p)) == 0
    assert p.sweep == gbmg.SWEEP_AUTO
    assert gbmg.sweep_shape(0) == (0, 0, 0)
    shapes = [gbmg.sweep_shape(v) for v in range(1, gbmg.SWEEP_VARIANTS)]
    assert len(set(shapes)) == gbmg.SWEEP_VARIANTS - 1
    for threads, planes, tile_x in shapes:
        # whole-row shapes, or staged tiles of 128 cells (16 row warps, a halo-quad warp)
        assert (threads in (512, 1024) and tile_x == 0) or (threads == 544 and tile_x == 128)
        assert planes >= 8
    assert any(s[2] for s in shapes) and any(not s[2] for s in shapes)
    with pytest.raises(gbmg.MGError):
        gbmg.sweep_shape(gbmg.SWEEP_VARIANTS)
    g = gbmg.make_grid((64, 64, 64), (1, 1, 0))
    size = ctypes.c_size_t()
    est = {}
    for sweep in (gbmg.SWEEP_AUTO, gbmg.SWEEP_HALF, 1, gbmg.SWEEP_VARIANTS - 1):
        p.sweep = sweep
        assert L.mg_memory_estimate(ctypes.byref(g), ctypes.byref(p), ctypes.byref(size)) == gbmg.OK
        est[sweep] = size.value
    # the one-pass sweep's second FP32 iterate buffer on the finest level
    assert est[gbmg.SWEEP_AUTO] - est[gbmg.SWEEP_HALF] == 64 ** 3 * 4
    for sweep in (-2, gbmg.SWEEP_VARIANTS):
        p.sweep = sweep
        assert L.mg_memory_estimate(ctypes.byref(g), ctypes.byref(p), ctypes.byref(size)) == gbmg.EINVAL
    # odd nu: the sweeps must end in the first buffer, so no second buffer
    p.sweep, p.nu1 = gbmg.SWEEP_AUTO, 1
    assert L.mg_memory_estimate(ctypes.byref(g), ctypes.byref(p), ctypes.byref(size)) == gbmg.OK
    assert size.value == est[gbmg.SWEEP_HALF]


def test_tune_cache_file_roundtrip(tmp_path):
    """Saved launch-shape choices load back; bad lines are skipped (host only)."""
    src = tmp_path / "tune.txt"
    src.write_text("0 1 3 128 128 128 1\n"      # half-sweep, FP32, periodic x y
                   "1 0 0 64 48 32 5\n"         # restriction, FP64
                   "garbage line\n"
                   "0 1 0 30 16 16 2\n"         # rows of 30 cells: flat shapes do not fit
                   "2 1 0 64 64 64 9\n"         # no such shape
                   "3 1 3 128 128 128 2\n"      # one-pass sweep, FP32, periodic x y
                   "3 1 3 128 127 128 2\n"      # odd periodic y: the one-pass sweep does not fit
                   "3 1 3 256 256 256 8\n"      # staged one-pass sweep, FP32
                   "3 0 3 256 256 128 8\n"      # staged shapes are FP32 only
                   "3 1 0 96 64 64 7\n")        # rows of 96 cells: no whole 128-cell tiles
    gbmg.tune_cache_clear()
    assert gbmg.tune_cache_size() == 0
    assert gbmg.tune_cache_load(str(src)) == 4
    assert gbmg.tune_cache_size() == 4
    out = tmp_path / "out.txt"
    gbmg.tune_cache_save(str(out))
    assert sorted(out.read_text().split("\n")[:-1]) == ["0 1 3 128 128 128 1", "1 0 0 64 48 32 5",
                                                        "3 1 3 128 128 128 2", "3 1 3 256 256 256 8"]
    with pytest.raises(gbmg.MGError) as e:
        gbmg.tune_cache_load(str(tmp_path / "missing.txt"))
    assert e.value.code == gbmg.ENOTFOUND
    gbmg.tune_cache_clear()
    assert gbmg.tune_cache_size() == 0


def test_no_gpu_fails_loudly():
    """Without a usable GPU the product path raises instead of computing on the host."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(Exception):
        gbmg.Solver((8, 8, 8), (0, 0, 0), faces=[torch.ones(512, dtype=torch.float64)] * 3)


# kernels launched with a plain <<< >>> launch, outside any dependent-launch
# scope (the allocation-free solve and the FP64 rate probe): they need no wait
PLAIN_LAUNCH = {"k_coarse_static", "k_fp64_fma"}


def test_every_launched_kernel_waits_for_its_predecessor_first():
    """A launch with programmatic stream serialization (launch_k inside a
    dependent-launch scope) may be scheduled while the previous kernel runs, so
    every kernel defined anywhere in csrc (.cu and .cuh) must begin with
    dep_entry() (griddepcontrol.wait, then the release of the next grid) or
    dep_wait() (the wait alone, with dep_release() later in the kernel) before
    any other statement, except the plain-launched ones, which must never be
    launched through launch_k."""
    import glob

    csrc = os.path.join(os.path.dirname(gbmg.__file__), "csrc")
    files = sorted(glob.glob(os.path.join(csrc, "*.cu")) + glob.glob(os.path.join(csrc, "*.cuh")))
    sources = {os.path.basename(p): open(p).read() for p in files}
    checked, plain = 0, set()
    for name, src in sources.items():
        for m in re.finditer(r"__global__[^;{]*\{", src):
            head = src[m.start():m.end()]
            kernel = re.search(r"\b(k_\w+)\s*\(", head).group(1)
            lines = [ln.strip() for ln in src[m.end():].split("\n")]
            body = [ln for ln in lines if ln and not ln.startswith("//")]
            first = body[0]
            if kernel in PLAIN_LAUNCH:
                plain.add(kernel)
                assert "<<<" in src, (name, kernel)
                continue
            assert first in ("dep_entry();", "dep_wait();"), (name, head[:90])
            if first == "dep_wait();":
                depth, i = 1, m.end()
                while depth:
                    depth += {"{": 1, "}": -1}.get(src[i], 0)
                    i += 1
                assert "dep_release();" in src[m.end():i], (name, kernel)
            checked += 1
    assert checked >= 30
    assert plain == PLAIN_LAUNCH
    for kernel in PLAIN_LAUNCH:
        for name, src in sources.items():
            assert not re.search(r"launch_k\(\s*%s\b" % kernel, src), (name, kernel)
