"""Pins for the CPU oracle against facts fixed outside it: closed forms,
library routines, brute force, invariants of alpha compositing, and the
paper's printed defaults and selection rules.

None of these runs the CUDA path.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2609_03613_gb300 import scenes

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- elementary

def test_expf_matches_libm_within_3ulp():
    xs = np.concatenate([np.linspace(-87.0, 88.0, 40001), np.linspace(-6.0, 0.0, 20001),
                         -np.logspace(-8, 0, 2001)]).astype(np.float32)
    worst = 0.0
    for x in xs:
        got = O.expf(float(x))
        ref = math.exp(float(x))
        worst = max(worst, abs(got - ref) / ref)
    assert worst < 3.0 * 2.0 ** -23, worst
    assert O.expf(0.0) == 1.0


def test_expf_below_alpha_threshold_past_cut():
    # The raster may skip exp for q > 5.6: exp(-q) < 1/255 there, so
    # alpha = min(0.99, o*exp(-q)) <= exp(-q) < 1/255 for every o <= 1.
    qs = np.linspace(5.6, 100.0, 20001).astype(np.float32)
    thr = np.float32(1.0) / np.float32(255.0)
    assert all(O.expf(-float(q)) < thr for q in qs)


def test_logf_matches_libm():
    xs = np.concatenate([np.logspace(-4, 10, 30001), np.linspace(0.5, 2.0, 10001)]).astype(np.float32)
    for x in xs:
        got = O.logf(float(x))
        ref = math.log(float(x))
        assert abs(got - ref) <= 1.5e-7 + 2.5e-7 * abs(ref), (x, got, ref)
    assert O.logf(1.0) == 0.0


def test_sh_basis_unsold_and_orthonormal():
    # Unsold's theorem: sum_m Y_lm(d)^2 = (2l+1)/(4 pi) for every direction d.
    rng = np.random.default_rng(0)
    d = rng.standard_normal((200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    bands = [(0, 1), (1, 4), (4, 9), (9, 16)]
    for v in d.astype(np.float32):
        Y = O.sh_basis(*map(float, v)).astype(np.float64)
        for l, (a, b) in enumerate(bands):
            assert abs(np.sum(Y[a:b] ** 2) - (2 * l + 1) / (4 * math.pi)) < 2e-6
    # Orthonormality by Gauss-Legendre (cos theta) x uniform (phi) quadrature.
    ct, wt = np.polynomial.legendre.leggauss(16)
    phis = np.arange(32) * (2 * math.pi / 32)
    G = np.zeros((16, 16))
    for c, w in zip(ct, wt):
        s = math.sqrt(1 - c * c)
        for p in phis:
            Y = O.sh_basis(float(s * math.cos(p)), float(s * math.sin(p)), float(c)).astype(np.float64)
            G += np.outer(Y, Y) * w * (2 * math.pi / 32)
    assert np.abs(G - np.eye(16)).max() < 2e-6


# ---------------------------------------------------------------- projection

def _one(mean, scale, quat, opac=0.5, sh=None):
    sh = np.zeros((1, 1, 3), np.float32) if sh is None else sh
    return scenes.Scene(np.array([mean], np.float32), np.array([scale], np.float32),
                        np.array([quat], np.float32), np.array([opac], np.float32),
                        sh.astype(np.float32), int(round(math.sqrt(sh.shape[1]))) - 1)


def test_project_on_axis_closed_form():
    cam = scenes.hd_camera()
    z = 3.0
    sx, sy, sz = 0.02, 0.05, 0.01
    P = O.project(_one((0, 0, 0), (sx, sy, sz), (1, 0, 0, 0)), cam)
    a = (1100.0 * sx / z) ** 2 + 0.3
    c = (1100.0 * sy / z) ** 2 + 0.3
    assert P["visible"][0] == 1
    np.testing.assert_allclose(P["conic"][0], [1 / a, 0.0, 1 / c], rtol=2e-6, atol=1e-12)
    np.testing.assert_allclose(P["mean2d"][0], [960.0, 540.0], rtol=0, atol=1e-4)
    assert P["depth"][0] == np.float32(3.0)
    lam = max(a, c)  # |a - c| / 2 > 0.1 here, so lambda_max = max(a, c)
    assert P["radius"][0] == math.ceil(3 * math.sqrt(lam))


def test_project_rotation_about_optical_axis_closed_form():
    # A world rotation by theta about z shows as a rotation by -theta in the
    # image (the camera flips y): Sigma' = (f/z)^2 Rot(-th) diag(sx^2, sy^2) Rot(-th)^T + 0.3 I.
    cam = scenes.hd_camera()
    th = 0.7
    quat = (math.cos(th / 2), 0.0, 0.0, math.sin(th / 2))
    sx, sy = 0.04, 0.01
    P = O.project(_one((0, 0, 0), (sx, sy, 0.02), quat), cam)
    R = np.array([[math.cos(-th), -math.sin(-th)], [math.sin(-th), math.cos(-th)]])
    S2 = (1100.0 / 3.0) ** 2 * R @ np.diag([sx * sx, sy * sy]) @ R.T + 0.3 * np.eye(2)
    inv = np.linalg.inv(S2)
    np.testing.assert_allclose(P["conic"][0], [inv[0, 0], inv[0, 1], inv[1, 1]], rtol=5e-5,
                               atol=1e-7)


def test_project_matches_ewa_with_finite_difference_jacobian():
    """Sigma' - 0.3 I = J R Sigma R^T J^T with J = d(pinhole)/d(p_cam) by
    central differences and the 3D rotation from scipy (not the oracle)."""
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    rng = np.random.default_rng(3)
    cam = scenes.hd_camera(position=(0.3, -0.2, 3.0))
    n = 60
    means = rng.uniform(-0.6, 0.6, (n, 3))
    scales = np.exp(rng.normal(-4, 0.5, (n, 3)))
    quats = rng.standard_normal((n, 4))
    quats /= np.linalg.norm(quats, axis=1, keepdims=True)
    sc = scenes.Scene(means.astype(np.float32), scales.astype(np.float32), quats.astype(np.float32),
                      np.full(n, 0.5, np.float32), np.zeros((n, 1, 3), np.float32), 0)
    P = O.project(sc, cam)
    P64 = O.project64(sc, cam)
    W = cam.viewmat.astype(np.float64)

    def pin(pc):
        return np.array([cam.fx * pc[0] / pc[2] + cam.cx, cam.fy * pc[1] / pc[2] + cam.cy])

    for i in range(n):
        m = sc.means[i].astype(np.float64)
        pc = W[:3, :3] @ m + W[:3, 3]
        J = np.zeros((2, 3))
        for k in range(3):
            h = np.zeros(3)
            h[k] = 1e-6 * pc[2]
            J[:, k] = (pin(pc + h) - pin(pc - h)) / (2 * h[k])
        q = sc.quats[i].astype(np.float64)
        Rq = Rot.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        Sig = Rq @ np.diag(sc.scales[i].astype(np.float64) ** 2) @ Rq.T
        S2 = J @ W[:3, :3] @ Sig @ W[:3, :3].T @ J.T + 0.3 * np.eye(2)
        inv = np.linalg.inv(S2)
        ref = np.array([inv[0, 0], inv[0, 1], inv[1, 1]])
        np.testing.assert_allclose(P64["conic"][i], ref, rtol=1e-6, atol=1e-9 * np.abs(ref).max())
        np.testing.assert_allclose(P["conic"][i], ref, rtol=2e-3, atol=2e-4 * np.abs(ref).max())
        np.testing.assert_allclose(P["mean2d"][i], pin(pc), rtol=0, atol=2e-3)
        assert abs(P["depth"][i] - pc[2]) < 1e-5


def test_project_rigid_motion_invariance():
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    sc = scenes.tiny_scene(500, 11)
    cam = scenes.tiny_camera()
    P0 = O.project(sc, cam)
    R = Rot.from_euler("xyz", [0.3, -0.5, 1.1]).as_matrix()
    t = np.array([0.4, -1.2, 2.0])
    means2 = (sc.means.astype(np.float64) @ R.T + t).astype(np.float32)
    # rotate the Gaussians' frames too: q2 = q_R * q
    qR = Rot.from_matrix(R)
    q_xyzw = np.concatenate([sc.quats[:, 1:], sc.quats[:, :1]], axis=1).astype(np.float64)
    q2 = (qR * Rot.from_quat(q_xyzw)).as_quat()
    quats2 = np.concatenate([q2[:, 3:], q2[:, :3]], axis=1).astype(np.float32)
    sc2 = scenes.Scene(means2, sc.scales, quats2, sc.opacities, sc.sh, 0)
    Winv = np.eye(4)
    Winv[:3, :3] = R.T
    Winv[:3, 3] = -R.T @ t
    cam2 = scenes.Camera((cam.viewmat.astype(np.float64) @ Winv).astype(np.float32), cam.fx, cam.fy,
                         cam.cx, cam.cy, cam.width, cam.height)
    P1 = O.project(sc2, cam2)
    vis = (P0["visible"] == 1) & (P1["visible"] == 1)
    assert vis.sum() > 300
    np.testing.assert_allclose(P1["mean2d"][vis], P0["mean2d"][vis], atol=2e-3)
    np.testing.assert_allclose(P1["conic"][vis], P0["conic"][vis], rtol=2e-3,
                               atol=2e-4 * np.abs(P0["conic"][vis]).max())
    np.testing.assert_allclose(P1["rgb"][vis], P0["rgb"][vis], atol=1e-5)


def test_project_sh_colour_closed_forms():
    cam = scenes.hd_camera()
    # degree 0: rgb = 0.5 + Y00 * dc with Y00 = 1 / (2 sqrt(pi)); dc = sqrt(pi) gives 1.
    sh = np.zeros((1, 1, 3), np.float32)
    sh[0, 0] = [math.sqrt(math.pi), 0.0, -math.sqrt(math.pi)]
    P = O.project(_one((0.1, 0.1, 0), (0.01, 0.01, 0.01), (1, 0, 0, 0), sh=sh), cam)
    np.testing.assert_allclose(P["rgb"][0], [1.0, 0.5, 0.0], atol=1e-6)
    # band 1 alone is odd in the view direction: rgb(d) + rgb(-d) = 1 (no clamp)
    sh = np.zeros((1, 4, 3), np.float32)
    sh[0, 1:] = np.array([[0.2, -0.1, 0.3], [0.1, 0.2, -0.2], [-0.3, 0.1, 0.1]])
    camA = scenes.hd_camera(position=(0.0, 0.0, 3.0))
    camB = scenes.hd_camera(position=(0.0, 0.0, -3.0))
    g = _one((0, 0, 0), (0.01, 0.01, 0.01), (1, 0, 0, 0), sh=sh)
    a, b = O.project(g, camA)["rgb"][0], O.project(g, camB)["rgb"][0]
    np.testing.assert_allclose(a + b, [1.0, 1.0, 1.0], atol=1e-6)


def test_tile_rect_brute_force():
    sc = scenes.tiny_scene()
    cam = scenes.tiny_camera()
    P = O.project(sc, cam)
    tx, ty = O.tiles_xy(cam.width, cam.height)
    vis = P["visible"] == 1
    assert vis.sum() > 5000
    mx = P["mean2d"][:, 0]
    my = P["mean2d"][:, 1]
    r = P["radius"].astype(np.float32)
    hx = (mx + r).astype(np.float64)  # the same float32 sums the rect uses
    lx = (mx - r).astype(np.float64)
    hy = (my + r).astype(np.float64)
    ly = (my - r).astype(np.float64)
    for i in np.nonzero(vis)[0][:3000]:
        inx = [(16.0 * t < hx[i]) and (16.0 * (t + 1) > lx[i]) for t in range(tx)]
        iny = [(16.0 * t < hy[i]) and (16.0 * (t + 1) > ly[i]) for t in range(ty)]
        xs = [t for t in range(tx) if inx[t]]
        ys = [t for t in range(ty) if iny[t]]
        assert P["rect"][i, 0] == xs[0] and P["rect"][i, 2] == xs[-1] + 1
        assert P["rect"][i, 1] == ys[0] and P["rect"][i, 3] == ys[-1] + 1
    # invisible ones have an empty rect and radius 0
    assert np.all(P["radius"][~vis] == 0)


def test_tile_lists_match_lexsort():
    sc = scenes.tiny_scene()
    cam = scenes.tiny_camera()
    P = O.project(sc, cam)
    ent = O.emit(P, cam.width, cam.height)
    tile_a, z_a, g_a = ent
    assert tile_a.shape[0] == int(((P["rect"][:, 2] - P["rect"][:, 0]) * (P["rect"][:, 3] - P["rect"][:, 1])).sum())
    off, stream = O.sort_tiles(ent, 256)
    order = np.lexsort((g_a, z_a, tile_a))
    np.testing.assert_array_equal(stream & np.uint64(0xFFFFFFFF), g_a[order].astype(np.uint64))
    np.testing.assert_array_equal(stream >> np.uint64(32), z_a[order].astype(np.uint64))
    np.testing.assert_array_equal(np.diff(off), np.bincount(tile_a, minlength=256))
    # z bits order is numeric order for positive depths
    zs = z_a.view(np.float32)
    assert np.all(zs > 0)


# ---------------------------------------------------------------- compositing

def _manual_proj(mean2d, conic, opac, rgb):
    return dict(mean2d=np.asarray(mean2d, np.float32).reshape(-1, 2),
                conic=np.asarray(conic, np.float32).reshape(-1, 3),
                opacity=np.asarray(opac, np.float32).reshape(-1),
                rgb=np.asarray(rgb, np.float32).reshape(-1, 3))


def _stream_for(gids, depth=None):
    g = np.asarray(gids, np.uint64)
    z = np.zeros_like(g) if depth is None else np.asarray(depth, np.float32).view(np.uint32).astype(np.uint64)
    return (z << np.uint64(32)) | g


def test_composite_single_gaussian_closed_form():
    conic = (0.05, 0.01, 0.08)
    proj = _manual_proj([[8.3, 7.1]], [conic], [0.8], [[0.2, 0.5, 0.9]])
    off = np.array([0, 1], np.int32)
    rgb, alpha, last = O.composite(proj, off, _stream_for([0]), 16, 16)
    for j in range(16):
        for i in range(16):
            dx, dy = 8.3 - (i + 0.5), 7.1 - (j + 0.5)
            q = 0.5 * (conic[0] * dx * dx + conic[2] * dy * dy) + conic[1] * dx * dy
            a = min(0.99, 0.8 * math.exp(-q))
            if a < 1 / 255:
                a = 0.0
            assert abs(alpha[j, i] - a) < 2e-6
            np.testing.assert_allclose(rgb[j, i], a * np.array([0.2, 0.5, 0.9]), atol=2e-6)
            assert last[j, i] == (0 if a > 0 else -1)


def test_composite_two_layer_order():
    proj = _manual_proj([[4, 4], [4, 4]], [(0.001, 0, 0.001)] * 2, [0.6, 0.7],
                        [[1, 0, 0], [0, 0, 1]])
    off = np.array([0, 2], np.int32)
    bg = (0.1, 0.2, 0.3)
    for order in ([0, 1], [1, 0]):
        rgb, alpha, last = O.composite(proj, off, _stream_for(order), 16, 16, bg=bg)
        a = [min(0.99, [0.6, 0.7][g] * math.exp(-0.5 * 0.001 * 0.0)) for g in order]
        # pixel (4,4) has centre (4.5, 4.5): recompute exactly in fp64
        dx = dy = 4 - 4.5
        q = 0.5 * (0.001 * dx * dx + 0.001 * dy * dy)
        a = [min(0.99, [0.6, 0.7][g] * math.exp(-q)) for g in order]
        cols = [np.array([[1, 0, 0], [0, 0, 1]][g], float) for g in order]
        C = a[0] * cols[0] + a[1] * (1 - a[0]) * cols[1]
        T = (1 - a[0]) * (1 - a[1])
        np.testing.assert_allclose(rgb[4, 4], C + T * np.array(bg), atol=2e-6)
        assert abs(alpha[4, 4] - (1 - T)) < 2e-6
        assert last[4, 4] == order[1]  # the id of the last applied Gaussian


def _scene_all(sc, cam, tile=16):
    proj, ent, (off, stream), res = O.render(sc, cam, tile)
    return proj, off, stream, res


def test_composite_telescoping_and_background_linearity():
    sc = scenes.tiny_scene(3000, 5)
    cam = scenes.tiny_camera()
    proj, off, stream, _ = _scene_all(sc, cam)
    ones = dict(proj)
    ones["rgb"] = np.ones_like(proj["rgb"])
    rgb, alpha, _ = O.composite(ones, off, stream, cam.width, cam.height)
    T = 1.0 - alpha.astype(np.float64)
    # sum_i alpha_i T_i + T_final = 1 for unit colours and black background
    assert np.abs(rgb[..., 0].astype(np.float64) + T - 1.0).max() < 2e-6
    rgb0, a0, _ = O.composite(proj, off, stream, cam.width, cam.height, bg=(0, 0, 0))
    bg = (0.25, 0.5, 1.0)
    rgb1, a1, _ = O.composite(proj, off, stream, cam.width, cam.height, bg=bg)
    np.testing.assert_array_equal(a0, a1)
    diff = rgb1.astype(np.float64) - rgb0
    np.testing.assert_allclose(diff, (1.0 - a0.astype(np.float64))[..., None] * np.array(bg), atol=3e-7)


def test_transmittance_non_increasing_along_list():
    sc = scenes.tiny_scene(2000, 7)
    cam = scenes.tiny_camera()
    proj, off, stream, _ = _scene_all(sc, cam)
    prev = None
    for k in [0, 1, 2, 4, 8, 16, 32, 64, 128, 100000]:
        # keep the first k entries of every tile
        lens = np.minimum(np.diff(off), k)
        noff = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
        nstream = np.concatenate([stream[off[t]:off[t] + lens[t]] for t in range(256)])
        _, alpha, _ = O.composite(proj, noff, nstream, cam.width, cam.height)
        if prev is not None:
            assert np.all(alpha >= prev)
        prev = alpha


def test_nonfinite_inputs_are_culled():
    """Reading of the paper's silence on non-finite parameters: a Gaussian
    with a non-finite mean, scale, quaternion or opacity, or a non-finite SH
    sum, is culled.  Pinned against the opacity cull (opacity 0 < 1/255, a
    different rule): the frame with the planted values equals, bit for bit,
    the frame with those Gaussians' opacities set to zero, and every other
    Gaussian projects as before."""
    cam = scenes.hd_camera(width=480, height=270, f=275.0)
    for sc0 in (scenes.tiny_scene(4000, 3), scenes.mixture_scene(30000, 11)):
        bad, gids, kinds = scenes.plant_nonfinite(sc0)
        ref = scenes.Scene(sc0.means.copy(), sc0.scales.copy(), sc0.quats.copy(), sc0.opacities.copy(),
                           sc0.sh.copy(), sc0.sh_degree)
        ref.opacities[gids] = 0.0
        c = cam if sc0.sh_degree else scenes.tiny_camera()
        pb, _, _, (rgb_b, a_b, l_b) = O.render(bad, c)
        pr, _, _, (rgb_r, a_r, l_r) = O.render(ref, c)
        assert not pb["visible"][gids].any()
        for k in ("mean2d", "conic", "depth", "radius", "rect", "rgb", "visible"):
            np.testing.assert_array_equal(pb[k], pr[k])
        np.testing.assert_array_equal(rgb_b.view(np.uint32), rgb_r.view(np.uint32))
        np.testing.assert_array_equal(a_b, a_r)
        np.testing.assert_array_equal(l_b, l_r)
        assert np.isfinite(rgb_b).all()
        # the planted Gaussians would be drawn if their values were finite
        p0 = O.project(sc0, c)
        assert p0["visible"][gids].sum() >= 4
    assert "sh_overflow" in kinds


def test_composite_brute_force_all_gaussians_low_opacity():
    """With every opacity <= 0.3, a Gaussian outside its tile rectangle has
    alpha < 1/255 everywhere, so per-pixel compositing over ALL Gaussians in
    (depth, gid) order (fp64, no tiling) equals the tiled oracle."""
    rng = np.random.default_rng(9)
    n = 120
    sc = scenes.Scene(rng.uniform(-0.5, 0.5, (n, 3)).astype(np.float32),
                      np.exp(rng.normal(-2.6, 0.4, (n, 3))).astype(np.float32),
                      (lambda q: q / np.linalg.norm(q, axis=1, keepdims=True))(rng.standard_normal((n, 4))).astype(np.float32),
                      rng.uniform(0.05, 0.3, n).astype(np.float32),
                      rng.uniform(-1.7, 1.7, (n, 1, 3)).astype(np.float32), 0)
    cam = scenes.Camera(scenes.look_at((0, 0, 3.0)), 40.0, 40.0, 16.0, 16.0, 32, 32)
    proj, off, stream, (rgb, alpha, last) = _scene_all(sc, cam, tile=8)
    vis = np.nonzero(proj["visible"])[0]
    order = vis[np.lexsort((vis, proj["depth"][vis]))]
    checked = 0
    for j in range(32):
        for i in range(32):
            px, py = i + 0.5, j + 0.5
            T, C, near = 1.0, np.zeros(3), False
            for g in order:
                dx, dy = proj["mean2d"][g, 0] - px, proj["mean2d"][g, 1] - py
                c = proj["conic"][g].astype(np.float64)
                q = 0.5 * (c[0] * dx * dx + c[2] * dy * dy) + c[1] * dx * dy
                a = min(0.99, float(proj["opacity"][g]) * math.exp(-q))
                if abs(a - 1 / 255) < 1e-5:
                    near = True
                if a < 1 / 255:
                    continue
                if abs(T * (1 - a) - 1e-4) < 1e-7:
                    near = True
                if T * (1 - a) < 1e-4:
                    break
                C += proj["rgb"][g] * a * T
                T *= 1 - a
            if near:
                continue
            checked += 1
            np.testing.assert_allclose(rgb[j, i], C, atol=2e-5)
            assert abs(alpha[j, i] - (1 - T)) < 2e-5
    assert checked > 900


def test_fp32_oracle_close_to_fp64_twin():
    sc = scenes.tiny_scene(4000, 13)
    cam = scenes.tiny_camera()
    proj, off, stream, (rgb, alpha, _) = _scene_all(sc, cam)
    p64 = O.project64(sc, cam)
    rng = np.random.default_rng(1)
    bad = 0
    for _ in range(400):
        i, j = int(rng.integers(0, 256)), int(rng.integers(0, 256))
        t = (j // 16) * 16 + i // 16
        gids = (stream[off[t]:off[t + 1]] & np.uint64(0xFFFFFFFF)).astype(np.uint32)
        C, T = O.composite_pixel64(i + 0.5, j + 0.5, p64, sc.opacities, gids)
        if np.abs(rgb[j, i] - C).max() > 1e-5 or abs(alpha[j, i] - (1 - T)) > 1e-5:
            bad += 1
    assert bad <= 2  # threshold flips between precisions are rare


# ---------------------------------------------------------------- depth range / bins

def test_depth_range_order_statistics_all_sampled():
    rng = np.random.default_rng(2)
    n = 3000
    depth = rng.lognormal(1.0, 0.6, n).astype(np.float32)
    scales = rng.uniform(0.0, 0.1, (n, 3)).astype(np.float32)
    gid = rng.integers(0, n, 5000).astype(np.uint32)  # M = 5000 <= S: every entry sampled
    zr, kept = O.depth_range(gid, depth, scales, near_shift=False)
    v = depth[gid]
    assert kept == 5000
    k_lo, k_hi = math.ceil(0.01 * 5000), math.ceil(0.99 * 5000)
    zlo = np.partition(v, k_lo - 1)[k_lo - 1]
    zhi = np.partition(v, k_hi - 1)[k_hi - 1]
    span = np.float32(zhi - zlo)
    assert zr[0] == np.float32(max(np.float32(0.01), np.float32(zlo - np.float32(0.05) * span)))
    assert zr[1] == np.float32(zhi + np.float32(0.05) * span)


def test_depth_range_degenerate_and_shift():
    depth = np.full(10, 2.0, np.float32)
    scales = np.full((10, 3), 0.1, np.float32)
    gid = np.arange(10, dtype=np.uint32)
    zr, _ = O.depth_range(gid, depth, scales, near_shift=False)
    assert zr[0] <= 2.0 <= zr[1] and zr[1] - zr[0] < 1e-6
    # near shift: z - min(alpha * s_max, gamma * z) = 2 - min(0.1, 0.5) = 1.9
    zr, _ = O.depth_range(gid, depth, scales, near_shift=True)
    assert abs(zr[0] - 1.9) < 1e-6 and abs(zr[1] - 1.9) < 1e-6
    # gamma caps the shift for large Gaussians: 2 - min(10, 0.5) = 1.5
    zr, _ = O.depth_range(gid, depth, np.full((10, 3), 10.0, np.float32), near_shift=True)
    assert abs(zr[0] - 1.5) < 1e-6
    # no entries: fallback range
    zr, kept = O.depth_range(np.zeros(0, np.uint32), depth, scales)
    assert kept == 0 and zr[0] == np.float32(0.01) and zr[1] == np.float32(1e10)


def test_depth_range_samples_capped():
    n = 100000
    depth = np.linspace(1.0, 10.0, n).astype(np.float32)
    scales = np.zeros((n, 3), np.float32)
    zr, kept = O.depth_range(np.arange(n, dtype=np.uint32), depth, scales, S=8192)
    assert kept == 8192
    # uniform depths: 1st / 99th percentiles near 1.09 / 9.91, padded by 5 % of the span
    assert abs(zr[0] - (1.09 - 0.05 * 8.82)) < 0.01 and abs(zr[1] - (9.91 + 0.05 * 8.82)) < 0.01


def test_log_bin_map_closed_form():
    zmin, zmax, K = 0.7, 23.0, 64
    lmin, lmax, splits = O.bin_params(zmin, zmax, K)
    for k in range(K):
        zc = zmin * (zmax / zmin) ** ((k + 0.5) / K)  # log-space centre of bin k
        assert O.bin_log(np.float32(zc), lmin, lmax, K) == k
        assert O.bin_split(np.float32(zc), splits, K) == k
    assert O.bin_log(zmin, lmin, lmax, K) == 0
    assert O.bin_log(zmax, lmin, lmax, K) == K - 1
    assert O.bin_log(0.01, lmin, lmax, K) == 0 and O.bin_log(1e6, lmin, lmax, K) == K - 1
    ref = zmin * (zmax / zmin) ** (np.arange(1, K) / K)
    np.testing.assert_allclose(splits, ref, rtol=3e-6)
    # geometric midpoint lands at K/2
    assert O.bin_log(np.float32(math.sqrt(zmin * zmax) * 1.0001), lmin, lmax, K) == K // 2


def test_split_map_monotone():
    lmin, lmax, splits = O.bin_params(0.5, 40.0, 64)
    zs = np.sort(np.random.default_rng(4).uniform(0.01, 100.0, 5000).astype(np.float32))
    bins = [O.bin_split(float(z), splits, 64) for z in zs]
    assert all(b1 <= b2 for b1, b2 in zip(bins, bins[1:]))
    assert bins[0] == 0 and bins[-1] == 63


def _tiny_entries():
    sc = scenes.tiny_scene()
    cam = scenes.tiny_camera()
    proj = O.project(sc, cam)
    ent = O.emit(proj, cam.width, cam.height)
    return sc, proj, ent


@pytest.mark.parametrize("map_mode", [0, 1])
def test_bin_build_preserves_tile_spans_and_multisets(map_mode):
    sc, proj, ent = _tiny_entries()
    off_g, stream_g = O.sort_tiles(ent, 256)
    zk = O.zkeys(proj["depth"], sc.scales) if map_mode == 1 else None
    zr, _ = O.depth_range(ent[2], proj["depth"], sc.scales, near_shift=(map_mode == 1))
    K = 16
    off_b, stream_b = O.bin_build(ent, 256, K, map_mode, zr, zkey=zk)
    np.testing.assert_array_equal(off_b[::K], off_g)  # tile spans unchanged
    for t in range(256):
        a = np.sort(stream_b[off_g[t]:off_g[t + 1]])
        b = np.sort(stream_g[off_g[t]:off_g[t + 1]])
        np.testing.assert_array_equal(a, b)


def test_monotone_bins_fully_sorted_equal_global_order():
    sc, proj, ent = _tiny_entries()
    off_g, stream_g = O.sort_tiles(ent, 256)
    zr, _ = O.depth_range(ent[2], proj["depth"], sc.scales, near_shift=False)
    for K in (1, 4, 64):
        off_b, stream_b = O.bin_build(ent, 256, K, 0, zr)
        np.testing.assert_array_equal(O.sort_segments(off_b, stream_b), stream_g)


def test_repair_selection_golden_cases():
    cases = json.load(open(os.path.join(GOLD, "repair_rules_cases.json")))["cases"]
    for case in cases:
        K = case["K"]
        lens = np.array(case["tiles"], np.int64).reshape(-1)
        off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
        sel, used = O.repair_select(off, len(case["tiles"]), K, case["M"])
        np.testing.assert_array_equal(sel.reshape(-1, K), np.array(case["expect"], np.uint8),
                                      err_msg=case["name"])
        assert used == case["used"], case["name"]


def test_selected_segments_sorted_others_untouched():
    sc, proj, ent = _tiny_entries()
    zk = O.zkeys(proj["depth"], sc.scales)
    zr, _ = O.depth_range(ent[2], proj["depth"], sc.scales, near_shift=True)
    K = 8
    off_b, stream_b = O.bin_build(ent, 256, K, 1, zr, zkey=zk)
    sel, used = O.repair_select(off_b, 256, K, ent[0].shape[0])
    rep = O.sort_segments(off_b, stream_b, sel)
    for q in range(256 * K):
        seg = rep[off_b[q]:off_b[q + 1]]
        if sel[q]:
            assert np.all(seg[:-1] <= seg[1:])
        else:
            np.testing.assert_array_equal(seg, stream_b[off_b[q]:off_b[q + 1]])
    assert used <= ent[0].shape[0] // 4
