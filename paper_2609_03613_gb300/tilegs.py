"""Thin ctypes binding of libtilegs.so (include/tilegs.h).

Argument marshalling only: every step of the frame runs in the library's
CUDA kernels.  Tensors are torch CUDA tensors (torch supplies device memory
and the current stream).  Importing works without a GPU; any call that needs
the library raises when libtilegs.so is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtilegs.so")

GS_OK = 0
ERRORS = {1: "invalid argument", 2: "entry capacity exceeded", 3: "CUDA runtime error",
          4: "bounded device wait timed out", 5: "out of device memory", 6: "non-finite input"}

MODE_GLOBAL_SORT, MODE_BINNED_EXACT, MODE_BINNED_PAPER, MODE_BINNED_NOREPAIR = 0, 1, 2, 3
MODES = {"global": 0, "exact": 1, "paper": 2, "norepair": 3}
STAGES = ["project", "intersect", "depth_range", "bin", "repair", "sort", "raster", "complete"]
MAX_K = 128
MAX_VIEWS = 32
PLAN_FEATURES, PLAN_HIDDEN, PLAN_CLASSES = 8, 64, 6
PLAN_PARAMS = PLAN_HIDDEN * PLAN_FEATURES + PLAN_HIDDEN + PLAN_HIDDEN * PLAN_HIDDEN + PLAN_HIDDEN + \
    PLAN_CLASSES * PLAN_HIDDEN + PLAN_CLASSES
RENDER_HOST_INPUTS, RENDER_HOST_OUTPUTS, RENDER_NO_SYNC, RENDER_GRAPH, RENDER_SAVE = 1, 2, 4, 8, 16
RENDER_PIPELINE = 32
P_XY_AB, P_C_O_Z, P_RGB, P_RECT, P_RADIUS = range(5)

# Every symbol include/tilegs.h declares (checked by the CPU export test).
EXPORTS = [
    "gs_status_string", "gs_config_default", "gs_create", "gs_destroy", "gs_set_config",
    "gs_get_config", "gs_reserve", "gs_get_error", "gs_clear_error", "gs_enable_timing",
    "gs_get_stage_times", "gs_projected_bytes", "gs_projected_offset", "gs_isect_bytes",
    "gs_isect_offset", "gs_num_tiles", "gs_project", "gs_tile_intersect", "gs_sort_or_bin",
    "gs_depth_range", "gs_bin_build", "gs_repair", "gs_rasterize_fwd", "gs_render",
    "gs_last_entry_count", "gs_launch_count", "gs_last_raster_ops", "gs_depth_range_noalloc",
    "gs_grad2d_bytes", "gs_grad2d_offset", "gs_rasterize_bwd", "gs_render_bwd",
    "gs_render_batch", "gs_batch_set_view_config", "gs_batch_get_view_config", "gs_batch_last_entry_count",
    "gs_batch_autotune", "gs_rasterize_fwd_plan", "gs_tile_features", "gs_planner_set_weights", "gs_plan_tiles",
    "gs_mlp_forward", "gs_mlp_loss_grad", "gs_mlp_backward", "gs_adam_step", "gs_spatial_order",
    "gs_gather_rows", "gs_last_flagged_tiles", "gs_reciprocal", "gs_render_wait",
]


class TileGSError(RuntimeError):
    pass


class GsCamera(C.Structure):
    _fields_ = [("viewmat", C.c_float * 16), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("near_plane", C.c_float), ("far_plane", C.c_float)]


class GsConfig(C.Structure):
    _fields_ = [("mode", C.c_int32), ("tile_size", C.c_int32), ("K", C.c_int32),
                ("sample_count", C.c_int32), ("p_lo", C.c_float), ("p_hi", C.c_float),
                ("pad", C.c_float), ("near_alpha", C.c_float), ("near_gamma", C.c_float),
                ("eps", C.c_float), ("repair_budget_frac", C.c_float), ("near_shift", C.c_int32),
                ("tile_cull", C.c_int32), ("persistent", C.c_int32), ("repair_in_raster", C.c_int32),
                ("chunk_cap", C.c_int32), ("planner", C.c_int32), ("wait_polls", C.c_int32),
                ("planner_quantile", C.c_float), ("pdl", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class GsScene(C.Structure):
    _fields_ = [("means", C.c_void_p), ("scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacities", C.c_void_p), ("sh", C.c_void_p), ("sh_degree", C.c_int32),
                ("n", C.c_int64)]


_lib = None


def lib_available() -> bool:
    return os.path.exists(LIB_PATH)


def lib():
    """Load libtilegs.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise TileGSError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                          "(nvcc, sm_103a); there is no CPU fallback")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t
    sig = {
        "gs_status_string": (C.c_char_p, [C.c_int]),
        "gs_config_default": (None, [C.POINTER(GsConfig), i32]),
        "gs_create": (C.c_int, [C.POINTER(vp), C.POINTER(GsConfig)]),
        "gs_destroy": (C.c_int, [vp]),
        "gs_set_config": (C.c_int, [vp, C.POINTER(GsConfig)]),
        "gs_get_config": (C.c_int, [vp, C.POINTER(GsConfig)]),
        "gs_reserve": (C.c_int, [vp, i64, i64, i32, i32]),
        "gs_get_error": (C.c_int, [vp, vp]),
        "gs_clear_error": (C.c_int, [vp, vp]),
        "gs_enable_timing": (C.c_int, [vp, i32]),
        "gs_get_stage_times": (C.c_int, [vp, C.POINTER(C.c_float)]),
        "gs_projected_bytes": (sz, [i64]),
        "gs_projected_offset": (sz, [i64, i32]),
        "gs_isect_bytes": (sz, [i64]),
        "gs_isect_offset": (sz, [i64, i32]),
        "gs_num_tiles": (i32, [i32, i32, i32]),
        "gs_project": (C.c_int, [vp, vp, vp, vp, vp, vp, i32, i64, C.POINTER(GsCamera), vp, vp]),
        "gs_tile_intersect": (C.c_int, [vp, vp, i64, C.POINTER(GsCamera), vp, i64, vp,
                                        C.POINTER(i64), vp]),
        "gs_sort_or_bin": (C.c_int, [vp, vp, vp, i64, C.POINTER(GsCamera), vp, i64, vp, vp, vp,
                                     vp, vp]),
        "gs_depth_range": (C.c_int, [vp, vp, vp, i64, C.POINTER(GsCamera), vp, i64, vp, vp, vp]),
        "gs_bin_build": (C.c_int, [vp, vp, vp, i64, C.POINTER(GsCamera), vp, i64, vp, vp, vp, vp,
                                   vp]),
        "gs_repair": (C.c_int, [vp, C.POINTER(GsCamera), vp, vp, vp, vp, vp]),
        "gs_rasterize_fwd": (C.c_int, [vp, vp, i64, C.POINTER(GsCamera), vp, vp, i32,
                                       C.POINTER(C.c_float), vp, vp, vp, vp, vp, vp, vp]),
        "gs_render": (C.c_int, [vp, C.POINTER(GsScene), C.POINTER(GsCamera),
                                C.POINTER(C.c_float), vp, vp, vp, i32, vp]),
        "gs_last_entry_count": (i64, [vp]),
        "gs_launch_count": (i64, [vp]),
        "gs_last_raster_ops": (i64, [vp, vp]),
        "gs_last_flagged_tiles": (i32, [vp, vp]),
        "gs_depth_range_noalloc": (C.c_int, [C.POINTER(GsConfig), vp, vp, i64, C.POINTER(GsCamera), vp, i64,
                                             vp, vp, vp]),
        "gs_grad2d_bytes": (sz, [i64]),
        "gs_render_bwd": (C.c_int, [vp, vp, vp, vp, vp]),
        "gs_render_wait": (C.c_int, [vp]),
        "gs_render_batch": (C.c_int, [vp, C.POINTER(GsScene), C.POINTER(GsCamera), i32, C.POINTER(C.c_float),
                                      C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), i32, vp]),
        "gs_batch_set_view_config": (C.c_int, [vp, i32, C.POINTER(GsConfig)]),
        "gs_batch_get_view_config": (C.c_int, [vp, i32, C.POINTER(GsConfig)]),
        "gs_batch_last_entry_count": (i64, [vp, i32]),
        "gs_rasterize_fwd_plan": (C.c_int, [vp, vp, i64, C.POINTER(GsCamera), vp, vp, i32, C.POINTER(C.c_float),
                                            vp, vp, vp, vp, vp, vp, vp]),
        "gs_tile_features": (C.c_int, [vp, C.POINTER(GsCamera), vp, i32, vp, vp]),
        "gs_planner_set_weights": (C.c_int, [vp, vp, vp]),
        "gs_plan_tiles": (C.c_int, [vp, C.POINTER(GsCamera), vp, i32, vp, vp, vp]),
        "gs_mlp_forward": (C.c_int, [vp, vp, i32, vp, vp, vp]),
        "gs_mlp_loss_grad": (C.c_int, [vp, vp, i32, vp, vp, vp]),
        "gs_mlp_backward": (C.c_int, [vp, vp, vp, vp, i32, vp, vp, vp]),
        "gs_adam_step": (C.c_int, [vp, vp, vp, vp, i32, C.c_float, C.c_float, C.c_float, C.c_float, i32, vp]),
        "gs_batch_autotune": (C.c_int, [vp, C.POINTER(GsScene), C.POINTER(GsCamera), i32, i32, i32,
                                        C.POINTER(C.c_float), vp]),
        "gs_grad2d_offset": (sz, [i64, i32]),
        "gs_spatial_order": (C.c_int, [vp, vp, i64, vp, vp]),
        "gs_gather_rows": (C.c_int, [vp, vp, i64, vp, i32, vp, vp]),
        "gs_reciprocal": (C.c_int, [vp, vp, i64, vp]),
        "gs_rasterize_bwd": (C.c_int, [vp, vp, i64, C.POINTER(GsCamera), vp, vp, i32, C.POINTER(C.c_float), vp, vp,
                                       vp, vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def check(status: int, what: str = "") -> None:
    if status != GS_OK:
        raise TileGSError(f"{what}: {ERRORS.get(status, status)}")


def default_config(mode="exact", **kw) -> GsConfig:
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    cfg = GsConfig()
    lib().gs_config_default(C.byref(cfg), m)
    for k, v in kw.items():
        setattr(cfg, k, v)
    return cfg


def gs_camera(cam) -> GsCamera:
    """Marshal a scenes.Camera (or anything with the same fields)."""
    c = GsCamera()
    vm = np.ascontiguousarray(cam.viewmat, np.float32).reshape(-1)
    for k in range(16):
        c.viewmat[k] = float(vm[k])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    c.near_plane, c.far_plane = float(cam.near), float(cam.far)
    return c


def _ptr(t) -> int | None:
    return None if t is None else int(t.data_ptr())


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


@dataclasses.dataclass
class DeviceScene:
    means: "torch.Tensor"
    scales: "torch.Tensor"
    quats: "torch.Tensor"
    opacities: "torch.Tensor"
    sh: "torch.Tensor"
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @staticmethod
    def from_numpy(scene, device="cuda"):
        import torch
        f = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(device)
        return DeviceScene(f(scene.means), f(scene.scales), f(scene.quats), f(scene.opacities),
                           f(scene.sh), int(scene.sh_degree))


def n_tiles(width, height, tile=16) -> int:
    return int(lib().gs_num_tiles(width, height, tile))


@dataclasses.dataclass
class Saved:
    """What rasterize_fwd(save=True) keeps for the backward."""
    last: object
    final_T: object
    tile_end: object
    bg: tuple


class Context:
    """Owns a gs_ctx (scratch, error word, timing events)."""

    def __init__(self, mode="exact", **cfg_overrides):
        self.cfg = default_config(mode, **cfg_overrides)
        h = C.c_void_p()
        check(lib().gs_create(C.byref(h), C.byref(self.cfg)), "gs_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().gs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------- config
    def set_config(self, **kw):
        for k, v in kw.items():
            if k == "mode" and isinstance(v, str):
                v = MODES[v]
            setattr(self.cfg, k, v)
        check(lib().gs_set_config(self.h, C.byref(self.cfg)), "gs_set_config")

    @property
    def mode(self) -> int:
        return int(self.cfg.mode)

    @property
    def stride(self) -> int:
        return 1 if self.cfg.mode == MODE_GLOBAL_SORT else int(self.cfg.K)

    def reserve(self, n, m_cap, width, height):
        check(lib().gs_reserve(self.h, int(n), int(m_cap), int(width), int(height)), "gs_reserve")

    def error(self) -> int:
        return int(lib().gs_get_error(self.h, _stream()))

    def clear_error(self):
        check(lib().gs_clear_error(self.h, _stream()), "gs_clear_error")

    def enable_timing(self, on=True):
        check(lib().gs_enable_timing(self.h, 1 if on else 0), "gs_enable_timing")

    def stage_times(self) -> dict:
        ms = (C.c_float * len(STAGES))()
        check(lib().gs_get_stage_times(self.h, ms), "gs_get_stage_times")
        return {s: float(ms[i]) for i, s in enumerate(STAGES)}

    # ------------------------------------------------------------- stages
    def project(self, sc: DeviceScene, cam, out=None):
        import torch
        n = sc.n
        nbytes = int(lib().gs_projected_bytes(n))
        if out is None:
            out = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=sc.means.device)
        c = gs_camera(cam)
        check(lib().gs_project(self.h, _ptr(sc.means), _ptr(sc.scales), _ptr(sc.quats),
                               _ptr(sc.opacities), _ptr(sc.sh), sc.sh_degree, n, C.byref(c),
                               _ptr(out), _stream()), "gs_project")
        return out

    def tile_intersect(self, projected, n, cam, m_cap=None, isect=None, m_dev=None):
        """Returns (isect buffer, m_cap, m_dev tensor, M).  Grows once if needed
        (one host read of M)."""
        import torch
        dev = projected.device
        c = gs_camera(cam)
        if m_dev is None:
            m_dev = torch.zeros(1, dtype=torch.int64, device=dev)
        if m_cap is None:
            m_cap = max(1024, 4 * n)
        while True:
            if isect is None or isect.numel() < int(lib().gs_isect_bytes(m_cap)):
                isect = torch.empty(int(lib().gs_isect_bytes(m_cap)), dtype=torch.uint8, device=dev)
            m_host = C.c_int64(0)
            st = lib().gs_tile_intersect(self.h, _ptr(projected), n, C.byref(c), _ptr(isect), m_cap,
                                         _ptr(m_dev), C.byref(m_host), _stream())
            if st == 2 and m_host.value > m_cap:  # capacity: grow and redo
                self.clear_error()
                m_cap = int(m_host.value)
                isect = None
                continue
            check(st, "gs_tile_intersect")
            return isect, m_cap, m_dev, int(m_host.value)

    def isect_arrays(self, isect, m_cap, m):
        """(tile, zbits, gid) int32 views of the first m entries."""
        out = []
        for f in range(3):
            o = int(lib().gs_isect_offset(m_cap, f))
            out.append(isect[o:o + 4 * m].view(dtype=__import__("torch").int32))
        return out

    def sort_or_bin(self, projected, scales, n, cam, isect, m_cap, m_dev, m=None):
        import torch
        dev = projected.device
        T = n_tiles(cam.width, cam.height, int(self.cfg.tile_size))
        words = torch.empty(max(m_cap, 1), dtype=torch.int64, device=dev)
        offsets = torch.empty(T * self.stride + 1, dtype=torch.int32, device=dev)
        zr = torch.zeros(2, dtype=torch.float32, device=dev)
        c = gs_camera(cam)
        check(lib().gs_sort_or_bin(self.h, _ptr(projected), _ptr(scales), n, C.byref(c), _ptr(isect),
                                   m_cap, _ptr(m_dev), _ptr(words), _ptr(offsets), _ptr(zr), _stream()),
              "gs_sort_or_bin")
        return words, offsets, zr

    def depth_range(self, projected, scales, n, cam, isect, m_cap, m_dev):
        import torch
        zr = torch.zeros(2, dtype=torch.float32, device=projected.device)
        c = gs_camera(cam)
        check(lib().gs_depth_range(self.h, _ptr(projected), _ptr(scales), n, C.byref(c), _ptr(isect),
                                   m_cap, _ptr(m_dev), _ptr(zr), _stream()), "gs_depth_range")
        return zr

    def bin_build(self, projected, scales, n, cam, isect, m_cap, m_dev, zrange):
        import torch
        dev = projected.device
        T = n_tiles(cam.width, cam.height, int(self.cfg.tile_size))
        words = torch.empty(max(m_cap, 1), dtype=torch.int64, device=dev)
        offsets = torch.empty(T * int(self.cfg.K) + 1, dtype=torch.int32, device=dev)
        c = gs_camera(cam)
        check(lib().gs_bin_build(self.h, _ptr(projected), _ptr(scales), n, C.byref(c), _ptr(isect),
                                 m_cap, _ptr(m_dev), _ptr(zrange), _ptr(words), _ptr(offsets),
                                 _stream()), "gs_bin_build")
        return words, offsets

    def repair(self, cam, m_dev, words, offsets, want_selected=True):
        import torch
        sel = None
        if want_selected:
            sel = torch.zeros(offsets.numel() - 1, dtype=torch.uint8, device=words.device)
        c = gs_camera(cam)
        check(lib().gs_repair(self.h, C.byref(c), _ptr(m_dev), _ptr(words), _ptr(offsets), _ptr(sel),
                              _stream()), "gs_repair")
        return sel

    def rasterize_fwd(self, projected, n, cam, words, offsets, stride=None, bg=(0.0, 0.0, 0.0),
                      count_tests=False, save=False):
        """(rgb, alpha, last[, ntests]); with save=True also a Saved record
        (final_T, tile_end, bg) for rasterize_bwd, appended last."""
        import torch
        dev = projected.device
        H, W = int(cam.height), int(cam.width)
        rgb = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
        alpha = torch.empty((H, W), dtype=torch.float32, device=dev)
        last = torch.empty((H, W), dtype=torch.int32, device=dev)
        nt = torch.empty((H, W), dtype=torch.int32, device=dev) if count_tests else None
        fT = torch.empty((H, W), dtype=torch.float32, device=dev) if save else None
        te = (torch.empty(n_tiles(W, H, self.cfg.tile_size), dtype=torch.int32, device=dev)
              if save else None)
        bgv = (C.c_float * 3)(*[float(x) for x in bg])
        c = gs_camera(cam)
        check(lib().gs_rasterize_fwd(self.h, _ptr(projected), n, C.byref(c), _ptr(words), _ptr(offsets),
                                     self.stride if stride is None else int(stride), bgv, _ptr(rgb),
                                     _ptr(alpha), _ptr(last), _ptr(nt), _ptr(fT), _ptr(te), _stream()),
              "gs_rasterize_fwd")
        out = (rgb, alpha, last) + ((nt,) if count_tests else ())
        if save:
            out = out + (Saved(last, fT, te, tuple(float(x) for x in bg)),)
        return out

    def rasterize_bwd(self, projected, n, cam, words, offsets, saved, dl_drgb, dl_dalpha=None,
                      stride=None, grad=None):
        """Backward of rasterize_fwd(..., save=True) (saved = its Saved
        record): returns the gradient buffer (uint8, gs_grad2d_bytes(n));
        grad_fields() gives its [n,4] float views."""
        import torch
        if grad is None:
            grad = torch.empty(int(lib().gs_grad2d_bytes(n)), dtype=torch.uint8, device=projected.device)
        for t, shape in ((dl_drgb, (cam.height, cam.width, 3)), (dl_dalpha, (cam.height, cam.width))):
            if t is not None and (t.dtype != torch.float32 or not t.is_contiguous() or tuple(t.shape) != shape):
                raise TileGSError(f"gs_rasterize_bwd: expected a contiguous float32 tensor of shape {shape}")
        bgv = (C.c_float * 3)(*saved.bg)
        c = gs_camera(cam)
        check(lib().gs_rasterize_bwd(self.h, _ptr(projected), n, C.byref(c), _ptr(words), _ptr(offsets),
                                     self.stride if stride is None else int(stride), bgv, _ptr(saved.last),
                                     _ptr(saved.final_T), _ptr(saved.tile_end), _ptr(dl_drgb), _ptr(dl_dalpha),
                                     _ptr(grad), _stream()), "gs_rasterize_bwd")
        return grad

    def render(self, sc: DeviceScene, cam, bg=(0.0, 0.0, 0.0), out=None, flags=0):
        """One frame through gs_render (all intermediates in context scratch).
        With RENDER_PIPELINE (and both host flags) the call returns before its
        outputs land; render_wait() waits for them."""
        import torch
        H, W = int(cam.height), int(cam.width)
        if out is None:
            dev = sc.means.device
            out = (torch.empty((H, W, 3), dtype=torch.float32, device=dev),
                   torch.empty((H, W), dtype=torch.float32, device=dev),
                   torch.empty((H, W), dtype=torch.int32, device=dev))
        rgb, alpha, last = out
        s = GsScene(_ptr(sc.means), _ptr(sc.scales), _ptr(sc.quats), _ptr(sc.opacities), _ptr(sc.sh),
                    sc.sh_degree, sc.n)
        bgv = (C.c_float * 3)(*[float(x) for x in bg])
        c = gs_camera(cam)
        check(lib().gs_render(self.h, C.byref(s), C.byref(c), bgv, _ptr(rgb), _ptr(alpha), _ptr(last),
                              int(flags), _stream()), "gs_render")
        self._saved_n = int(sc.n) if flags & RENDER_SAVE else None
        return rgb, alpha, last

    def render_wait(self):
        """Wait for every render(..., flags=RENDER_PIPELINE | RENDER_HOST_INPUTS
        | RENDER_HOST_OUTPUTS) made so far: their outputs are in host memory."""
        check(lib().gs_render_wait(self.h), "gs_render_wait")

    def render_bwd(self, dl_drgb, dl_dalpha=None, grad=None):
        """Backward of the last render(..., flags=RENDER_SAVE): the gradient
        buffer (grad_fields() gives its [n,4] views)."""
        import torch
        n = getattr(self, "_saved_n", None)
        if n is None:
            raise TileGSError("gs_render_bwd: invalid argument (no render with RENDER_SAVE on this context)")
        if grad is None:
            grad = torch.empty(int(lib().gs_grad2d_bytes(n)), dtype=torch.uint8, device=dl_drgb.device)
        check(lib().gs_render_bwd(self.h, _ptr(dl_drgb), _ptr(dl_dalpha), _ptr(grad), _stream()), "gs_render_bwd")
        return grad

    # ------------------------------------------------------------- bin planner
    def rasterize_fwd_plan(self, projected, n, cam, words, offsets, plan=None, flags=False, needed=False,
                           stride=None, bg=(0.0, 0.0, 0.0)):
        """One pass of a planned frame: (rgb, alpha, last, flags or None,
        bins_needed or None).  plan: uint8 [T] bins walked per tile (None:
        all); flags: also return the tiles left for a completing pass;
        needed: also return each tile's bins needed (requires plan=None)."""
        import torch
        dev = projected.device
        H, W = int(cam.height), int(cam.width)
        T = n_tiles(W, H, self.cfg.tile_size)
        rgb = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
        alpha = torch.empty((H, W), dtype=torch.float32, device=dev)
        last = torch.empty((H, W), dtype=torch.int32, device=dev)
        fl = torch.empty(T, dtype=torch.uint8, device=dev) if flags else None
        nd = torch.empty(T, dtype=torch.int32, device=dev) if needed else None
        bgv = (C.c_float * 3)(*[float(x) for x in bg])
        c = gs_camera(cam)
        check(lib().gs_rasterize_fwd_plan(self.h, _ptr(projected), n, C.byref(c), _ptr(words), _ptr(offsets),
                                          self.stride if stride is None else int(stride), bgv, _ptr(rgb),
                                          _ptr(alpha), _ptr(last), _ptr(plan), _ptr(fl), _ptr(nd), _stream()),
              "gs_rasterize_fwd_plan")
        return rgb, alpha, last, fl, nd

    def tile_features(self, cam, offsets, stride=None):
        import torch
        T = n_tiles(cam.width, cam.height, self.cfg.tile_size)
        f = torch.empty((T, PLAN_FEATURES), dtype=torch.float32, device=offsets.device)
        c = gs_camera(cam)
        check(lib().gs_tile_features(self.h, C.byref(c), _ptr(offsets), self.stride if stride is None else int(stride),
                                     _ptr(f), _stream()), "gs_tile_features")
        return f

    def set_planner_weights(self, params):
        """params: float32 tensor of PLAN_PARAMS values (device or CPU), or None."""
        import torch
        if params is None:
            check(lib().gs_planner_set_weights(self.h, None, _stream()), "gs_planner_set_weights")
            return
        p = torch.as_tensor(params, dtype=torch.float32).contiguous()
        if p.numel() != PLAN_PARAMS:
            raise TileGSError(f"gs_planner_set_weights: invalid argument (expected {PLAN_PARAMS} floats)")
        self._planner_params = p  # kept alive until the copy has run
        check(lib().gs_planner_set_weights(self.h, _ptr(p), _stream()), "gs_planner_set_weights")

    def plan_tiles(self, cam, offsets, stride=None):
        """(plan, classes): each tile's first-pass bins and planner class
        (uint8 [T] each) from a binned stream's offsets."""
        import torch
        T = n_tiles(cam.width, cam.height, self.cfg.tile_size)
        plan = torch.empty(T, dtype=torch.uint8, device=offsets.device)
        cls = torch.empty(T, dtype=torch.uint8, device=offsets.device)
        c = gs_camera(cam)
        check(lib().gs_plan_tiles(self.h, C.byref(c), _ptr(offsets), self.stride if stride is None else int(stride),
                                  _ptr(plan), _ptr(cls), _stream()), "gs_plan_tiles")
        return plan, cls

    # ------------------------------------------------------------- scene order
    def spatial_order(self, means):
        """perm [n] int32 (device): the Morton order of the means (gs_spatial_order)."""
        import torch
        n = int(means.shape[0])
        perm = torch.empty(n, dtype=torch.int32, device=means.device)
        check(lib().gs_spatial_order(self.h, _ptr(means.contiguous()), n, _ptr(perm), _stream()),
              "gs_spatial_order")
        return perm

    def gather_rows(self, perm, src):
        """dst[i] = src[perm[i]] for a float32 tensor of n rows (gs_gather_rows)."""
        import torch
        src = src.contiguous()
        n = int(src.shape[0])
        if int(perm.shape[0]) != n:
            raise TileGSError("gs_gather_rows: invalid argument (perm and src lengths differ)")
        width = int(src.numel() // n) if n else 1
        dst = torch.empty_like(src)
        check(lib().gs_gather_rows(self.h, _ptr(perm), n, _ptr(src), width, _ptr(dst), _stream()),
              "gs_gather_rows")
        return dst

    def reorder_scene(self, sc: DeviceScene):
        """(the scene in raster-order-aware storage, perm): every per-Gaussian
        array gathered in the Morton order of the means."""
        perm = self.spatial_order(sc.means)
        g = lambda a: self.gather_rows(perm, a)
        return DeviceScene(g(sc.means), g(sc.scales), g(sc.quats), g(sc.opacities), g(sc.sh), sc.sh_degree), perm

    # ------------------------------------------------------------- batches
    def render_batch(self, sc: DeviceScene, cams, bg=(0.0, 0.0, 0.0), outs=None, flags=0):
        """All views of cams in one gs_render_batch call.  outs: list of
        (rgb, alpha, last) per view (allocated when None).  Returns outs."""
        import torch
        dev = sc.means.device
        if outs is None:
            outs = [(torch.empty((c.height, c.width, 3), dtype=torch.float32, device=dev),
                     torch.empty((c.height, c.width), dtype=torch.float32, device=dev),
                     torch.empty((c.height, c.width), dtype=torch.int32, device=dev)) for c in cams]
        nv = len(cams)
        carr = (GsCamera * nv)(*[gs_camera(c) for c in cams])
        P = C.c_void_p * nv
        rgb = P(*[_ptr(o[0]) for o in outs])
        alpha = P(*[_ptr(o[1]) for o in outs])
        last = P(*[_ptr(o[2]) if len(o) > 2 else None for o in outs])
        s = GsScene(_ptr(sc.means), _ptr(sc.scales), _ptr(sc.quats), _ptr(sc.opacities), _ptr(sc.sh),
                    sc.sh_degree, sc.n)
        bgv = (C.c_float * 3)(*[float(x) for x in bg])
        check(lib().gs_render_batch(self.h, C.byref(s), carr, nv, bgv, rgb, alpha, last, int(flags), _stream()),
              "gs_render_batch")
        return outs

    def batch_view_config(self, view) -> GsConfig:
        cfg = GsConfig()
        check(lib().gs_batch_get_view_config(self.h, int(view), C.byref(cfg)), "gs_batch_get_view_config")
        return cfg

    def set_batch_view_config(self, view, cfg=None, **kw):
        if cfg is None and kw:
            cfg = GsConfig.from_buffer_copy(self.cfg)
            for k, v in kw.items():
                setattr(cfg, k, MODES[v] if k == "mode" and isinstance(v, str) else v)
        check(lib().gs_batch_set_view_config(self.h, int(view), None if cfg is None else C.byref(cfg)),
              "gs_batch_set_view_config")

    def batch_entry_count(self, view) -> int:
        return int(lib().gs_batch_last_entry_count(self.h, int(view)))

    def batch_autotune(self, sc: DeviceScene, cams, tune_tile=True, iters=3):
        """Times the candidates per view and sets each view's config; returns the
        chosen configs' frame times (ms)."""
        nv = len(cams)
        carr = (GsCamera * nv)(*[gs_camera(c) for c in cams])
        s = GsScene(_ptr(sc.means), _ptr(sc.scales), _ptr(sc.quats), _ptr(sc.opacities), _ptr(sc.sh),
                    sc.sh_degree, sc.n)
        best = (C.c_float * nv)()
        check(lib().gs_batch_autotune(self.h, C.byref(s), carr, nv, 1 if tune_tile else 0, int(iters), best,
                                      _stream()), "gs_batch_autotune")
        return list(best)

    def last_entry_count(self) -> int:
        return int(lib().gs_last_entry_count(self.h))

    def launch_count(self) -> int:
        return int(lib().gs_launch_count(self.h))

    def flagged_tiles(self) -> int:
        """Tiles the last planned render left to its second pass."""
        return int(lib().gs_last_flagged_tiles(self.h, _stream()))

    def last_raster_ops(self) -> int:
        return int(lib().gs_last_raster_ops(self.h, _stream()))


def projected_fields(projected, n):
    """Views of the projected buffer's fields (float32 / int32 tensors)."""
    import torch
    L = lib()
    o = [int(L.gs_projected_offset(n, f)) for f in range(5)]
    xy_ab = projected[o[0]:o[0] + 16 * n].view(torch.float32).view(n, 4)
    c_o_z = projected[o[1]:o[1] + 16 * n].view(torch.float32).view(n, 4)
    rgb = projected[o[2]:o[2] + 16 * n].view(torch.float32).view(n, 4)
    rect = projected[o[3]:o[3] + 8 * n].view(torch.int32).view(n, 2)
    radius = projected[o[4]:o[4] + 4 * n].view(torch.int32)
    return dict(xy_ab=xy_ab, c_o_z=c_o_z, rgb=rgb, rect=rect, radius=radius)


def reciprocal(x):
    """1/x (device float32) by the reciprocal the raster backward uses to
    recover transmittances (within one rounding of the exact value)."""
    import torch
    out = torch.empty_like(x)
    check(lib().gs_reciprocal(_ptr(x), _ptr(out), int(x.numel()), _stream()), "gs_reciprocal")
    return out


def mlp_forward(params, X):
    """Planner network on X [B][8] (device float32): (acts [B][128], logits [B][6])."""
    import torch
    B = int(X.shape[0])
    acts = torch.empty((B, 2 * PLAN_HIDDEN), dtype=torch.float32, device=X.device)
    logits = torch.empty((B, PLAN_CLASSES), dtype=torch.float32, device=X.device)
    check(lib().gs_mlp_forward(_ptr(params), _ptr(X), B, _ptr(acts), _ptr(logits), _stream()), "gs_mlp_forward")
    return acts, logits


def mlp_loss_grad(logits, labels):
    """(loss [1], dlogits [B][6]) of the mean softmax cross entropy."""
    import torch
    B = int(logits.shape[0])
    d = torch.empty_like(logits)
    loss = torch.empty(1, dtype=torch.float32, device=logits.device)
    check(lib().gs_mlp_loss_grad(_ptr(logits), _ptr(labels), B, _ptr(d), _ptr(loss), _stream()), "gs_mlp_loss_grad")
    return loss, d


def mlp_backward(params, X, acts, dlogits, grads=None, deltas=None):
    import torch
    B = int(X.shape[0])
    if deltas is None:
        deltas = torch.empty((B, 2 * PLAN_HIDDEN), dtype=torch.float32, device=X.device)
    if grads is None:
        grads = torch.empty(PLAN_PARAMS, dtype=torch.float32, device=X.device)
    check(lib().gs_mlp_backward(_ptr(params), _ptr(X), _ptr(acts), _ptr(dlogits), B, _ptr(deltas), _ptr(grads),
                                _stream()), "gs_mlp_backward")
    return grads


def adam_step(params, grads, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    check(lib().gs_adam_step(_ptr(params), _ptr(grads), _ptr(m), _ptr(v), int(params.numel()), float(lr),
                             float(beta1), float(beta2), float(eps), int(step), _stream()), "gs_adam_step")


def grad_fields(grad, n):
    """[n,4] float32 views of a gs_rasterize_bwd gradient buffer, keyed like
    the projected fields they differentiate: xy_ab {dmx, dmy, da, db},
    c_o_z {dc, dopacity, 0, 0}, rgb {dr, dg, db, 0}."""
    import torch
    L = lib()
    o = [int(L.gs_grad2d_offset(n, f)) for f in range(3)]
    return {k: grad[o[f]:o[f] + 16 * n].view(torch.float32).view(n, 4)
            for f, k in enumerate(("xy_ab", "c_o_z", "rgb"))}


def depth_range_noalloc(cfg: GsConfig, projected, scales, n, cam, isect, m_cap, m_dev, zrange):
    """gs_depth_range_noalloc: the depth range with no context and no device
    allocation (all buffers, zrange included, come from the caller)."""
    c = gs_camera(cam)
    check(lib().gs_depth_range_noalloc(C.byref(cfg), _ptr(projected), _ptr(scales), int(n), C.byref(c),
                                       _ptr(isect), int(m_cap), _ptr(m_dev), _ptr(zrange), _stream()),
          "gs_depth_range_noalloc")
    return zrange
