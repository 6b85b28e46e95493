"""CPU oracle for the TileGS forward path (test infrastructure).

Only tests/, ``__graft_entry__.smoke()`` and the cpu_baseline / reference leg
of ``bench.py`` may import this package.  The CUDA library never calls it and
shares no code with it.

The arithmetic lives in ``tilegs_oracle.c`` (plain C, float32 in a fixed
operation order, built with ``-ffp-contract=off``; an fp64 twin for pins).
This module compiles it with gcc on first use and wraps it with ctypes/numpy.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tilegs_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_LOCK = threading.Lock()
_lib = None

_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile liboracle.so next to the source (gcc, -O2, no fp contraction)."""
    with _LOCK:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-fopenmp", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        L.orc_expf.restype = C.c_float
        L.orc_expf.argtypes = [C.c_float]
        L.orc_logf.restype = C.c_float
        L.orc_logf.argtypes = [C.c_float]
        L.orc_sh_basis.restype = None
        L.orc_sh_basis.argtypes = [C.c_float, C.c_float, C.c_float, _f32p]
        L.orc_project.restype = None
        L.orc_project.argtypes = [C.c_int64, _f32p, _f32p, _f32p, _f32p, _f32p, C.c_int, _f32p,
                                  C.c_float, C.c_float, C.c_float, C.c_float, C.c_int, C.c_int,
                                  C.c_float, C.c_float, C.c_int,
                                  _f32p, _f32p, _f32p, _i32p, _i32p, _f32p, _u8p]
        L.orc_count_entries.restype = C.c_int64
        L.orc_count_entries.argtypes = [C.c_int64, _i32p]
        L.orc_emit.restype = None
        L.orc_emit.argtypes = [C.c_int64, _i32p, _f32p, C.c_int, _u32p, _u32p, _u32p]
        L.orc_sort_tiles.restype = None
        L.orc_sort_tiles.argtypes = [C.c_int64, _u32p, _u32p, _u32p, C.c_int32, _i32p, _u64p]
        L.orc_composite.restype = None
        L.orc_composite.argtypes = [_f32p, _f32p, _f32p, _f32p, _i32p, C.c_int, _u64p,
                                    C.c_int, C.c_int, C.c_int, _f32p, C.c_void_p, C.c_int64,
                                    _f32p, _f32p, _i32p, C.c_void_p]
        L.orc_zkey.restype = C.c_float
        L.orc_zkey.argtypes = [C.c_float, _f32p, C.c_float, C.c_float]
        L.orc_depth_range.restype = C.c_int64
        L.orc_depth_range.argtypes = [C.c_int64, _u32p, _f32p, _f32p, C.c_float, C.c_float,
                                      C.c_int, C.c_int, C.c_float, C.c_float, C.c_float,
                                      C.c_float, C.c_float, C.c_float, _f32p]
        L.orc_bin_params.restype = None
        L.orc_bin_params.argtypes = [C.c_float, C.c_float, C.c_int, C.c_float,
                                     C.POINTER(C.c_float), C.POINTER(C.c_float), _f32p]
        L.orc_bin_log.restype = C.c_int
        L.orc_bin_log.argtypes = [C.c_float, C.c_float, C.c_float, C.c_int, C.c_float]
        L.orc_bin_split.restype = C.c_int
        L.orc_bin_split.argtypes = [C.c_float, _f32p, C.c_int]
        L.orc_bin_build.restype = None
        L.orc_bin_build.argtypes = [C.c_int64, _u32p, _u32p, _u32p, C.c_void_p, C.c_int,
                                    C.c_float, C.c_float, C.c_void_p, C.c_float, C.c_int32,
                                    C.c_int, _i32p, _u64p]
        L.orc_repair_select.restype = C.c_int64
        L.orc_repair_select.argtypes = [C.c_int32, C.c_int, _i32p, C.c_int64, C.c_double, _u8p]
        L.orc_sort_segments.restype = None
        L.orc_sort_segments.argtypes = [C.c_int64, _i32p, C.c_void_p, _u64p]
        L.orc64_project.restype = None
        L.orc64_project.argtypes = [C.c_int64, _f32p, _f32p, _f32p, _f32p, C.c_int, _f32p,
                                    C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int,
                                    _f64p, _f64p, _f64p, _f64p, _f64p, _u8p]
        L.orc64_composite_pixel.restype = C.c_double
        L.orc64_composite_pixel.argtypes = [C.c_double, C.c_double, _f64p, _f64p, _f32p, _f64p,
                                            _u32p, C.c_int64, _f64p]
        _i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
        L.orc_composite_grad.restype = None
        L.orc_composite_grad.argtypes = [_f32p, _f32p, _f32p, _f32p, _i32p, C.c_int, _u64p, C.c_int, C.c_int,
                                         C.c_int, _f32p, _f32p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int,
                                         _f64p, _f64p, _f64p, _f64p, C.c_void_p]
        L.orc64_composite_frozen.restype = None
        L.orc64_composite_frozen.argtypes = [_f64p, _f64p, _f64p, _f64p, _i64p, _i32p, C.c_int, C.c_int, _f64p,
                                             _f64p, _f64p]
        L.orc_applied_lists.restype = C.c_int64
        L.orc_applied_lists.argtypes = [_f32p, _f32p, _f32p, _i32p, C.c_int, _u64p, C.c_int, C.c_int, C.c_int,
                                        _i64p, _i32p, C.c_int64]
        _lib = L
    return _lib


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def tiles_xy(width, height, tile=16):
    return (width + tile - 1) // tile, (height + tile - 1) // tile


def project(scene, cam, tile=16):
    """Oracle projection.  Returns a dict of per-Gaussian arrays."""
    n = scene.n
    out = dict(mean2d=np.zeros((n, 2), np.float32), conic=np.zeros((n, 3), np.float32),
               depth=np.zeros(n, np.float32), radius=np.zeros(n, np.int32),
               rect=np.zeros((n, 4), np.int32), rgb=np.zeros((n, 3), np.float32),
               visible=np.zeros(n, np.uint8))
    lib().orc_project(n, _c(scene.means, np.float32), _c(scene.scales, np.float32),
                      _c(scene.quats, np.float32), _c(scene.opacities, np.float32),
                      _c(scene.sh, np.float32), scene.sh_degree,
                      _c(cam.viewmat, np.float32).reshape(-1),
                      cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height,
                      cam.near, cam.far, tile,
                      out["mean2d"], out["conic"], out["depth"], out["radius"],
                      out["rect"], out["rgb"], out["visible"])
    out["opacity"] = _c(scene.opacities, np.float32)
    return out


def emit(proj, width, height, tile=16):
    """Entries (tile, zbits, gid) in emission order."""
    tx, _ = tiles_xy(width, height, tile)
    L = lib()
    m = L.orc_count_entries(proj["rect"].shape[0], proj["rect"])
    tile_a = np.zeros(m, np.uint32)
    z_a = np.zeros(m, np.uint32)
    g_a = np.zeros(m, np.uint32)
    L.orc_emit(proj["rect"].shape[0], proj["rect"], proj["depth"], tx, tile_a, z_a, g_a)
    return tile_a, z_a, g_a


def sort_tiles(entries, n_tiles):
    """Baseline tile lists: offsets [T+1] and stream words (zbits<<32 | gid)."""
    tile_a, z_a, g_a = entries
    off = np.zeros(n_tiles + 1, np.int32)
    stream = np.zeros(tile_a.shape[0], np.uint64)
    lib().orc_sort_tiles(tile_a.shape[0], tile_a, z_a, g_a, n_tiles, off, stream)
    return off, stream


def composite(proj, offsets, stream, width, height, tile=16, bg=(0.0, 0.0, 0.0), K=1,
              tiles=None, ntests=False):
    rgb = np.zeros((height, width, 3), np.float32)
    alpha = np.zeros((height, width), np.float32)
    last = np.full((height, width), -1, np.int32)
    nt = np.zeros((height, width), np.int32) if ntests else None
    bgv = np.asarray(bg, np.float32)
    sel = None if tiles is None else _c(tiles, np.int32)
    lib().orc_composite(_c(proj["mean2d"], np.float32), _c(proj["conic"], np.float32),
                        _c(proj["opacity"], np.float32), _c(proj["rgb"], np.float32),
                        _c(offsets, np.int32), K, _c(stream, np.uint64),
                        width, height, tile, bgv,
                        None if sel is None else sel.ctypes.data, 0 if sel is None else sel.shape[0],
                        rgb, alpha, last, None if nt is None else nt.ctypes.data)
    if ntests:
        return rgb, alpha, last, nt
    return rgb, alpha, last


def render(scene, cam, tile=16, bg=(0.0, 0.0, 0.0), tiles=None, ntests=False):
    """Full oracle frame: project, baseline tile lists, composite."""
    proj = project(scene, cam, tile)
    tx, ty = tiles_xy(cam.width, cam.height, tile)
    ent = emit(proj, cam.width, cam.height, tile)
    off, stream = sort_tiles(ent, tx * ty)
    res = composite(proj, off, stream, cam.width, cam.height, tile, bg, 1, tiles, ntests)
    return proj, ent, (off, stream), res


def expf(x: float) -> float:
    return lib().orc_expf(x)


def logf(x: float) -> float:
    return lib().orc_logf(x)


def sh_basis(x, y, z):
    Y = np.zeros(16, np.float32)
    lib().orc_sh_basis(x, y, z, Y)
    return Y


def zkeys(depth, scales, near_alpha=1.0, near_gamma=0.25):
    L = lib()
    sc = _c(scales, np.float32)
    out = np.zeros(depth.shape[0], np.float32)
    for i in range(depth.shape[0]):
        out[i] = L.orc_zkey(float(depth[i]), sc[i], near_alpha, near_gamma)
    return out


def depth_range(entry_gid, depth, scales, near=0.01, far=1e10, S=8192, near_shift=True,
                near_alpha=1.0, near_gamma=0.25, p_lo=1.0, p_hi=99.0, pad=0.05, eps=1e-4):
    zr = np.zeros(2, np.float32)
    kept = lib().orc_depth_range(entry_gid.shape[0], _c(entry_gid, np.uint32), _c(depth, np.float32),
                                 _c(scales, np.float32), near, far, S, int(near_shift),
                                 near_alpha, near_gamma, p_lo, p_hi, pad, eps, zr)
    return zr, kept


def bin_params(zmin, zmax, K, eps=1e-4):
    lmin = C.c_float()
    lmax = C.c_float()
    splits = np.zeros(max(K - 1, 1), np.float32)
    lib().orc_bin_params(zmin, zmax, K, eps, C.byref(lmin), C.byref(lmax), splits)
    return lmin.value, lmax.value, splits[: K - 1]


def bin_log(z, lmin, lmax, K, eps=1e-4):
    return lib().orc_bin_log(z, lmin, lmax, K, eps)


def bin_split(z, splits, K):
    return lib().orc_bin_split(z, _c(splits if K > 1 else np.zeros(1), np.float32), K)


def bin_build(entries, n_tiles, K, map_mode, zrange, zkey=None, eps=1e-4):
    """Tile-local bin construction; map_mode 0 = monotone splits on depth,
    1 = the paper's log map on the per-Gaussian near-shifted key."""
    tile_a, z_a, g_a = entries
    lmin, lmax, splits = bin_params(float(zrange[0]), float(zrange[1]), K, eps)
    sp = _c(splits if K > 1 else np.zeros(1, np.float32), np.float32)
    zk = None if zkey is None else _c(zkey, np.float32)
    off = np.zeros(n_tiles * K + 1, np.int32)
    stream = np.zeros(tile_a.shape[0], np.uint64)
    lib().orc_bin_build(tile_a.shape[0], tile_a, z_a, g_a, None if zk is None else zk.ctypes.data,
                        map_mode, lmin, lmax, sp.ctypes.data, eps, n_tiles, K, off, stream)
    return off, stream


def repair_select(bin_offsets, n_tiles, K, m, budget_frac=0.25):
    sel = np.zeros(n_tiles * K, np.uint8)
    used = lib().orc_repair_select(n_tiles, K, _c(bin_offsets, np.int32), m, budget_frac, sel)
    return sel, used


def sort_segments(bin_offsets, stream, selected=None):
    s = np.array(stream, np.uint64, copy=True)
    sel = None if selected is None else _c(selected, np.uint8)
    lib().orc_sort_segments(bin_offsets.shape[0] - 1, _c(bin_offsets, np.int32),
                            None if sel is None else sel.ctypes.data, s)
    return s


def project64(scene, cam):
    n = scene.n
    out = dict(mean2d=np.zeros((n, 2)), conic=np.zeros((n, 3)), depth=np.zeros(n),
               radius=np.zeros(n), rgb=np.zeros((n, 3)), ok=np.zeros(n, np.uint8))
    lib().orc64_project(n, _c(scene.means, np.float32), _c(scene.scales, np.float32),
                        _c(scene.quats, np.float32), _c(scene.sh, np.float32), scene.sh_degree,
                        _c(cam.viewmat, np.float32).reshape(-1), cam.fx, cam.fy, cam.cx, cam.cy,
                        cam.width, cam.height, out["mean2d"], out["conic"], out["depth"],
                        out["radius"], out["rgb"], out["ok"])
    return out


def composite_pixel64(px, py, proj64, opacity, gids):
    Cout = np.zeros(3)
    T = lib().orc64_composite_pixel(px, py, _c(proj64["mean2d"], np.float64),
                                    _c(proj64["conic"], np.float64), _c(opacity, np.float32),
                                    _c(proj64["rgb"], np.float64), _c(gids, np.uint32),
                                    len(gids), Cout)
    return Cout, T


def set_threads(n: int) -> None:
    """Threads used by the oracle's compositing loop (OpenMP over tiles)."""
    lib().orc_set_threads.argtypes = [C.c_int]
    lib().orc_set_threads(int(n))


def composite_grad(proj, offsets, stream, width, height, dl_drgb, dl_dalpha=None, tile=16, bg=(0.0, 0.0, 0.0),
                   K=1, with_abs=False, tiles=None, at_f32=False):
    """Gradient of the compositing (float32 decisions, double arithmetic):
    dict of mean2d [n,2], conic [n,3], opacity [n], rgb [n,3] (float64), and
    with_abs: "abs" [n,9], the sums of the absolute per-pixel terms.
    tiles: optional list of tile ids whose pixels contribute (the others are
    as if their incoming gradient were zero).
    at_f32: evaluate at the float32 forward's own exp, alpha and
    transmittances instead of recomputing them in double."""
    n = proj["mean2d"].shape[0]
    g = dict(mean2d=np.zeros((n, 2)), conic=np.zeros((n, 3)), opacity=np.zeros(n), rgb=np.zeros((n, 3)))
    if with_abs:
        g["abs"] = np.zeros((n, 9))
    da = None if dl_dalpha is None else _c(dl_dalpha, np.float32)
    sel = None if tiles is None else _c(np.unique(np.asarray(tiles)), np.int32)
    lib().orc_composite_grad(_c(proj["mean2d"], np.float32), _c(proj["conic"], np.float32),
                             _c(proj["opacity"], np.float32), _c(proj["rgb"], np.float32), _c(offsets, np.int32), K,
                             _c(stream, np.uint64), width, height, tile, np.asarray(bg, np.float32),
                             _c(dl_drgb, np.float32), None if da is None else da.ctypes.data,
                             None if sel is None else sel.ctypes.data, 0 if sel is None else sel.shape[0],
                             1 if at_f32 else 0, g["mean2d"], g["conic"], g["opacity"], g["rgb"],
                             g["abs"].ctypes.data if with_abs else None)
    return g


def applied_lists(proj, offsets, stream, width, height, tile=16, K=1):
    P = width * height
    off = np.zeros(P + 1, np.int64)
    L = lib()
    args = (_c(proj["mean2d"], np.float32), _c(proj["conic"], np.float32), _c(proj["opacity"], np.float32),
            _c(offsets, np.int32), K, _c(stream, np.uint64), width, height, tile)
    na = L.orc_applied_lists(*args, off, np.zeros(1, np.int32), 0)
    ap = np.zeros(max(na, 1), np.int32)
    L.orc_applied_lists(*args, off, ap, na)
    return off, ap[:na]


def composite_frozen64(mean2d, conic, opacity, rgb, applied_off, applied, width, height, bg=(0.0, 0.0, 0.0)):
    out_rgb = np.zeros((height, width, 3))
    out_a = np.zeros((height, width))
    lib().orc64_composite_frozen(_c(mean2d, np.float64), _c(conic, np.float64), _c(opacity, np.float64),
                                 _c(rgb, np.float64), _c(applied_off, np.int64), _c(applied, np.int32), width, height,
                                 np.asarray(bg, np.float64), out_rgb, out_a)
    return out_rgb, out_a
