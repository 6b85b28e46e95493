"""Seeded synthetic scenes and cameras.

This module only draws inputs: Gaussian parameters (means, linear scales,
unit quaternions, opacities in [0, 1], SH coefficients) and pinhole cameras.
It holds none of the renderer's arithmetic, so both the CUDA path and the CPU
oracle consume the same float32 bits from here.

The workloads stand in for the trained captured scenes the paper measures on
(Mip-NeRF 360, Tanks and Temples, Deep Blending; Sec. 4.2), which are not
available; their shapes follow the paper's problem statement (resident 3D
Gaussians with SH colour, one pinhole view, Sec. 3.1) and the configurations
listed below.

All draws use numpy's PCG64 generator in float64 and are rounded to float32
once, at the end.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Camera:
    """Pinhole camera, OpenCV axes (x right, y down, z forward).

    viewmat is the row-major 4x4 world-to-camera transform.
    """

    viewmat: np.ndarray  # (4, 4) float32
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near: float = 0.01
    far: float = 1e10


@dataclasses.dataclass
class Scene:
    means: np.ndarray      # (N, 3) float32
    scales: np.ndarray     # (N, 3) float32, linear (already activated)
    quats: np.ndarray      # (N, 4) float32, (w, x, y, z)
    opacities: np.ndarray  # (N,) float32 in [0, 1]
    sh: np.ndarray         # (N, (deg+1)^2, 3) float32
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])


def look_at(position, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0)) -> np.ndarray:
    """World-to-camera matrix for a camera at `position` looking at `target`.

    OpenCV convention: camera x = right, y = down, z = forward.  Built in
    float64, returned as float32.
    """
    p = np.asarray(position, np.float64)
    f = np.asarray(target, np.float64) - p
    f /= np.linalg.norm(f)
    right = np.cross(f, np.asarray(up, np.float64))
    nr = np.linalg.norm(right)
    if nr < 1e-9:  # looking along the up axis: pick another up
        right = np.cross(f, np.array([1.0, 0.0, 0.0]))
        nr = np.linalg.norm(right)
    right /= nr
    down = np.cross(f, right)
    R = np.stack([right, down, f])
    t = -R @ p
    m = np.eye(4)
    m[:3, :3] = R
    m[:3, 3] = t
    return m.astype(np.float32)


def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


# Half-width of the uniform draw for a degree-0 SH coefficient that makes the
# degree-0 colour uniform on [0, 1]: sqrt(pi) = 0.5 / Y_00.
_DC_HALF_RANGE = math.sqrt(math.pi)


def tiny_scene(n: int = 10_000, seed: int = 0) -> Scene:
    """10k plain Gaussians: means U[-1,1]^3, log-scales N(-4, 0.5) per axis,
    uniform unit quaternions, opacity sigmoid(N(0,1)), degree-0 colour U[0,1]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    means = rng.uniform(-1.0, 1.0, (n, 3))
    scales = np.exp(rng.normal(-4.0, 0.5, (n, 3)))
    quats = _unit_quats(rng, n)
    opac = _sigmoid(rng.normal(0.0, 1.0, n))
    dc = rng.uniform(-_DC_HALF_RANGE, _DC_HALF_RANGE, (n, 1, 3))
    return Scene(means.astype(np.float32), scales.astype(np.float32),
                 quats.astype(np.float32), opac.astype(np.float32),
                 dc.astype(np.float32), 0)


def mixture_scene(n: int = 1_000_000, seed: int = 1, sh_degree: int = 3,
                  n_components: int = 64, shell_fraction: float = 0.10) -> Scene:
    """Captured-scene-like distribution.

    90 % of the means come from a 64-component anisotropic Gaussian mixture
    (centres U[-1,1]^3, per-axis std U(0.05, 0.3), random orientation, equal
    weights); 10 % lie on a background shell of radius U[8, 10] with uniform
    direction.  Log-scales N(-5, 1) per axis (heavy tail), SH coefficients
    N(0, 0.3), opacity sigmoid(N(0, 1.5)).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n_shell = int(round(n * shell_fraction))
    n_mix = n - n_shell
    centres = rng.uniform(-1.0, 1.0, (n_components, 3))
    sig = rng.uniform(0.05, 0.3, (n_components, 3))
    rots = []
    for _ in range(n_components):  # Haar-random orthogonal matrix via QR
        qm, rm = np.linalg.qr(rng.standard_normal((3, 3)))
        rots.append(qm * np.sign(np.diag(rm)))
    rots = np.stack(rots)
    comp = rng.integers(0, n_components, n_mix)
    local = rng.standard_normal((n_mix, 3)) * sig[comp]
    mix = centres[comp] + np.einsum("nij,nj->ni", rots[comp], local)
    d = rng.standard_normal((n_shell, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    shell = d * rng.uniform(8.0, 10.0, (n_shell, 1))
    means = np.concatenate([mix, shell])
    perm = rng.permutation(n)  # interleave so gid order is not spatial order
    means = means[perm]
    scales = np.exp(rng.normal(-5.0, 1.0, (n, 3)))
    quats = _unit_quats(rng, n)
    opac = _sigmoid(rng.normal(0.0, 1.5, n))
    nc = (sh_degree + 1) ** 2
    sh = rng.normal(0.0, 0.3, (n, nc, 3))
    return Scene(means.astype(np.float32), scales.astype(np.float32),
                 quats.astype(np.float32), opac.astype(np.float32),
                 sh.astype(np.float32), sh_degree)


def mixture_centres(seed: int, n_components: int = 64) -> np.ndarray:
    """The mixture centres drawn by `mixture_scene(seed=seed)` (same stream)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-1.0, 1.0, (n_components, 3))


def tiny_camera() -> Camera:
    """(0,0,3) looking at the origin, 256x256, fx=fy=256, black background."""
    return Camera(look_at((0.0, 0.0, 3.0)), 256.0, 256.0, 128.0, 128.0, 256, 256)


def hd_camera(position=(0.0, 0.0, 3.0), width=1920, height=1080, f=1100.0) -> Camera:
    return Camera(look_at(position), f, f, width / 2.0, height / 2.0, width, height)


def heavy_camera(scene_seed: int, cam_seed: int, width=1920, height=1080, f=1100.0) -> Camera:
    """Camera inside a dense cluster: a mixture centre plus a 0.05*N(0,1)^3
    offset, looking at the origin (deep per-tile ranges)."""
    c = mixture_centres(scene_seed)
    rng = np.random.Generator(np.random.PCG64(cam_seed))
    k = int(rng.integers(0, c.shape[0]))
    pos = c[k] + 0.05 * rng.standard_normal(3)
    if np.linalg.norm(pos) < 0.2:  # keep the look-at direction well defined
        pos = pos + np.array([0.0, 0.0, 0.5])
    return Camera(look_at(pos), f, f, width / 2.0, height / 2.0, width, height)


BATCH_RESOLUTIONS = [(512, 512), (768, 768), (1024, 768), (1280, 720), (1600, 900), (1920, 1080)]


def batch_cameras(n_views: int = 16, seed0: int = 100) -> list[Camera]:
    """Cameras on spheres of radius U[2.5, 4] looking at the origin, with
    resolutions drawn from 512^2 .. 1920x1080 (focal scaled with width)."""
    cams = []
    for i in range(n_views):
        rng = np.random.Generator(np.random.PCG64(seed0 + i))
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        r = rng.uniform(2.5, 4.0)
        w, h = BATCH_RESOLUTIONS[int(rng.integers(0, len(BATCH_RESOLUTIONS)))]
        f = w * (1100.0 / 1920.0)
        cams.append(Camera(look_at(d * r), f, f, w / 2.0, h / 2.0, w, h))
    return cams


def random_target(height: int, width: int, seed: int = 5) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(0.0, 1.0, (height, width, 3)).astype(np.float32)


def grad_check_scene(n: int = 64, seed: int = 6) -> tuple[Scene, Camera]:
    """64 Gaussians in front of a 32x32, fx=32 camera, for gradient checks."""
    rng = np.random.Generator(np.random.PCG64(seed))
    means = rng.uniform(-0.6, 0.6, (n, 3))
    scales = np.exp(rng.normal(-2.3, 0.3, (n, 3)))
    quats = _unit_quats(rng, n)
    opac = rng.uniform(0.05, 0.6, n)
    dc = rng.uniform(-_DC_HALF_RANGE, _DC_HALF_RANGE, (n, 1, 3))
    scene = Scene(means.astype(np.float32), scales.astype(np.float32),
                  quats.astype(np.float32), opac.astype(np.float32), dc.astype(np.float32), 0)
    cam = Camera(look_at((0.0, 0.0, 3.0)), 32.0, 32.0, 16.0, 16.0, 32, 32)
    return scene, cam


def incoming_grads(height: int, width: int, seed: int = 5):
    """Seeded upstream gradients dL/drgb [H,W,3] and dL/dalpha [H,W] (N(0,1), float32)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dC = rng.normal(0.0, 1.0, (height, width, 3)).astype(np.float32)
    dA = rng.normal(0.0, 1.0, (height, width)).astype(np.float32)
    return dC, dA


def plant_nonfinite(scene: Scene, seed: int = 9, count: int = 48):
    """A copy of `scene` with non-finite values written into `count` seeded
    Gaussians, one kind per Gaussian in turn: NaN / +inf / -inf in a mean,
    scale or quaternion component or in the opacity, a NaN or inf SH
    coefficient, and (degree >= 2) three finite SH coefficients of 3.3e38
    whose weighted sum overflows for a camera on the +z axis beyond the scene
    (the default cameras).  Returns (scene, gids, kinds)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gids = np.sort(rng.choice(scene.n, size=count, replace=False))
    sc = Scene(scene.means.copy(), scene.scales.copy(), scene.quats.copy(), scene.opacities.copy(),
               scene.sh.copy(), scene.sh_degree)
    kinds = ["mean_nan", "mean_inf", "scale_ninf", "scale_nan", "quat_nan", "quat_inf", "opacity_nan",
             "opacity_inf", "sh_nan", "sh_inf"]
    if scene.sh_degree >= 2:
        kinds.append("sh_overflow")
    used = []
    for j, g in enumerate(gids):
        k = kinds[j % len(kinds)]
        a = int(rng.integers(0, 3))
        if k == "mean_nan":
            sc.means[g, a] = np.nan
        elif k == "mean_inf":
            sc.means[g, a] = np.inf
        elif k == "scale_ninf":
            sc.scales[g, a] = -np.inf
        elif k == "scale_nan":
            sc.scales[g, a] = np.nan
        elif k == "quat_nan":
            sc.quats[g, a] = np.nan
        elif k == "quat_inf":
            sc.quats[g, a + 1] = np.inf
        elif k == "opacity_nan":
            sc.opacities[g] = np.nan
        elif k == "opacity_inf":
            sc.opacities[g] = np.inf
        elif k == "sh_nan":
            sc.sh[g, 0, a] = np.nan
        elif k == "sh_inf":
            sc.sh[g, 0, a] = np.inf
        else:
            # Y_0, Y_2 (signed as the view direction's z) and Y_6 (positive
            # along the axis) all weigh their coefficient positively
            sc.sh[g, 0, a] = 3.3e38
            sc.sh[g, 2, a] = -3.3e38 if sc.means[g, 2] < 3.0 else 3.3e38
            sc.sh[g, 6, a] = 3.3e38
        used.append(k)
    return sc, gids, used


def workload(name: str):
    """Named workloads: returns (scene, camera or list of cameras)."""
    if name == "tiny":
        return tiny_scene(), tiny_camera()
    if name == "mid":
        return mixture_scene(1_000_000, 1), hd_camera()
    if name == "heavy3m":
        return mixture_scene(3_000_000, 2), heavy_camera(2, 200)
    if name == "heavy6m_4k":
        return mixture_scene(6_000_000, 3), heavy_camera(3, 300, 3840, 2160, 2200.0)
    if name == "batch16":
        return mixture_scene(2_000_000, 4), batch_cameras()
    raise KeyError(name)
