"""Pins for the oracle's compositing gradient (the backward of the raster).

The analytic gradient (float32 decisions, double arithmetic) is checked
against closed forms for one and two layers, a telescoping identity of the
colour weights, the clamp rule, and central finite differences of a
double-precision forward whose per-pixel lists are frozen at the float32
forward's decisions (so the differenced function is smooth).

None of these runs the CUDA path.
"""
import math

import numpy as np

import oracle as O
from paper_2609_03613_gb300 import scenes


def _one_tile_stream(order, depths=None):
    """A 1-tile stream listing the given gids in order (one 16x16 tile)."""
    n = len(order)
    z = np.arange(1, n + 1, dtype=np.float32) if depths is None else np.asarray(depths, np.float32)
    words = np.array([(int(z[k].view(np.uint32)) << 32) | int(g) for k, g in enumerate(order)], np.uint64)
    return np.array([0, n], np.int32), words


def _proj(mean2d, conic, opac, rgb):
    return dict(mean2d=np.asarray(mean2d, np.float32).reshape(-1, 2),
                conic=np.asarray(conic, np.float32).reshape(-1, 3),
                opacity=np.asarray(opac, np.float32).reshape(-1),
                rgb=np.asarray(rgb, np.float32).reshape(-1, 3))


def test_grad_single_gaussian_closed_form():
    # one Gaussian, one 1x1 image: out = c a + (1 - a) bg, alpha_out = a,
    # a = o exp(-q), q = 1/2 (A dx^2 + 2 B dx dy + C dy^2), d = mean - (0.5, 0.5)
    A, B, Cc, o = 0.8, 0.15, 0.5, 0.7
    mx, my = 0.5 + 0.4, 0.5 - 0.7
    col = np.array([0.9, 0.2, 0.6])
    # the oracle takes bg and the incoming gradients as float32
    bg = np.float32([0.1, 0.3, 0.05]).astype(np.float64)
    dC = np.float32([0.7, -1.3, 0.4]).astype(np.float64)
    dA = float(np.float32(-0.6))
    P = _proj([mx, my], [A, B, Cc], [o], col)
    off, words = _one_tile_stream([0])
    g = O.composite_grad(P, off, words, 1, 1, dC.reshape(1, 1, 3), np.float32([[dA]]), bg=tuple(bg))
    # closed form from the float32-rounded parameters
    mx, my = float(P["mean2d"][0, 0]), float(P["mean2d"][0, 1])
    A, B, Cc = (float(v) for v in P["conic"][0])
    o = float(P["opacity"][0])
    col = P["rgb"][0].astype(np.float64)
    dx, dy = mx - 0.5, my - 0.5
    q = 0.5 * (A * dx * dx + 2.0 * B * dx * dy + Cc * dy * dy)
    G = math.exp(-q)
    a = o * G
    dL_da = float(dC @ (col - bg)) + dA
    dL_dq = -dL_da * a
    np.testing.assert_allclose(g["rgb"][0], dC * a, rtol=1e-12)
    np.testing.assert_allclose(g["opacity"][0], dL_da * G, rtol=1e-12)
    np.testing.assert_allclose(g["mean2d"][0], [dL_dq * (A * dx + B * dy), dL_dq * (B * dx + Cc * dy)], rtol=1e-12)
    np.testing.assert_allclose(g["conic"][0], [dL_dq * 0.5 * dx * dx, dL_dq * dx * dy, dL_dq * 0.5 * dy * dy],
                               rtol=1e-12)


def test_grad_two_layers_closed_form_and_order():
    # two Gaussians centred on the pixel (q = 0): a_k = o_k,
    # out = c1 a1 + c2 a2 (1 - a1) + bg (1 - a1)(1 - a2)
    o1, o2 = 0.6, 0.3
    c1, c2 = np.array([1.0, 0.2, 0.4]), np.array([0.1, 0.9, 0.5])
    bg = np.float32([0.25, 0.5, 0.75]).astype(np.float64)
    dC = np.float32([1.0, 2.0, -0.5]).astype(np.float64)
    dA = float(np.float32(0.3))
    P = _proj([0.5, 0.5, 0.5, 0.5], [1.0, 0.0, 1.0, 1.0, 0.0, 1.0], [o1, o2], np.stack([c1, c2]))
    o1, o2 = (float(v) for v in P["opacity"])
    c1, c2 = P["rgb"].astype(np.float64)
    for order in ([0, 1], [1, 0]):
        off, words = _one_tile_stream(order)
        g = O.composite_grad(P, off, words, 1, 1, dC.reshape(1, 1, 3), np.float32([[dA]]), bg=tuple(bg))
        f, b = order
        of, ob = (o1, o2) if f == 0 else (o2, o1)
        cf, cb = (c1, c2) if f == 0 else (c2, c1)
        # d/da_front = cf - cb ab - bg (1 - ab); d/da_back = (cb - bg)(1 - af); alpha_out = 1 - (1-af)(1-ab)
        dfront = float(dC @ (cf - cb * ob - bg * (1 - ob))) + dA * (1 - ob)
        dback = float(dC @ ((cb - bg) * (1 - of))) + dA * (1 - of)
        np.testing.assert_allclose(g["opacity"][f], dfront, rtol=1e-12)
        np.testing.assert_allclose(g["opacity"][b], dback, rtol=1e-12)
        np.testing.assert_allclose(g["rgb"][f], dC * of, rtol=1e-12)
        np.testing.assert_allclose(g["rgb"][b], dC * ob * (1 - of), rtol=1e-12)
        # centred: q has zero gradient w.r.t. the mean and the conic
        assert np.all(g["mean2d"] == 0.0) and np.all(g["conic"] == 0.0)


def test_grad_clamped_alpha_passes_no_gradient_to_opacity_or_shape():
    # o exp(-q) > 0.99 at the pixel: alpha = 0.99 is flat in o, mean and conic
    P = _proj([0.6, 0.45], [0.5, 0.1, 0.5], [1.0], [0.3, 0.6, 0.9])
    off, words = _one_tile_stream([0])
    g = O.composite_grad(P, off, words, 1, 1, np.ones((1, 1, 3), np.float32), np.ones((1, 1), np.float32))
    assert g["opacity"][0] == 0.0 and np.all(g["mean2d"] == 0.0) and np.all(g["conic"] == 0.0)
    np.testing.assert_allclose(g["rgb"][0], 0.99, rtol=1e-12)


def _grad_case(seed=6, bg=(0.2, 0.1, 0.3)):
    sc, cam = scenes.grad_check_scene(seed=seed)
    proj, ent, (off, words), (rgb, alpha, last) = O.render(sc, cam, bg=bg)
    rng = np.random.Generator(np.random.PCG64(1000 + seed))
    dC = rng.normal(0.0, 1.0, (cam.height, cam.width, 3)).astype(np.float32)
    dA = rng.normal(0.0, 1.0, (cam.height, cam.width)).astype(np.float32)
    return sc, cam, proj, off, words, rgb, alpha, dC, dA


def test_frozen_forward_matches_float32_composite():
    sc, cam, proj, off, words, rgb, alpha, dC, dA = _grad_case()
    aoff, ap = O.applied_lists(proj, off, words, cam.width, cam.height)
    assert ap.shape[0] > 2000  # several layers per pixel on average
    r64, a64 = O.composite_frozen64(proj["mean2d"], proj["conic"], proj["opacity"], proj["rgb"], aoff, ap,
                                    cam.width, cam.height, bg=(0.2, 0.1, 0.3))
    assert np.max(np.abs(r64 - rgb)) < 1e-5 and np.max(np.abs(a64 - alpha)) < 1e-5


def test_grad_matches_central_finite_differences():
    bg = (0.2, 0.1, 0.3)
    sc, cam, proj, off, words, rgb, alpha, dC, dA = _grad_case(bg=bg)
    W, H = cam.width, cam.height
    g = O.composite_grad(proj, off, words, W, H, dC, dA, bg=bg)
    aoff, ap = O.applied_lists(proj, off, words, W, H)
    # every o exp(-q) <= o < 0.99 - 1e-3: no applied entry is near the alpha
    # clamp, so the frozen map is smooth within the differencing steps
    assert float(np.max(proj["opacity"])) < 0.989
    base = {k: proj[k].astype(np.float64) for k in ("mean2d", "conic", "opacity", "rgb")}
    dC64, dA64 = dC.astype(np.float64), dA.astype(np.float64)

    def loss(p):
        r, a = O.composite_frozen64(p["mean2d"], p["conic"], p["opacity"], p["rgb"], aoff, ap, W, H, bg=bg)
        return float(np.sum(r * dC64) + np.sum(a * dA64))

    checked = 0
    for key in ("mean2d", "conic", "opacity", "rgb"):
        flat = base[key].reshape(-1)
        an = g[key].reshape(-1)
        fd = np.zeros_like(an)
        for i in range(flat.shape[0]):
            h = 1e-6 * max(1.0, abs(flat[i]))
            p = {k: v.copy() for k, v in base.items()}
            p[key].reshape(-1)[i] = flat[i] + h
            lp = loss(p)
            p[key].reshape(-1)[i] = flat[i] - h
            lm = loss(p)
            fd[i] = (lp - lm) / (2.0 * h)
        scale = np.max(np.abs(an))
        assert scale > 0.0, key
        err = np.abs(fd - an)
        assert np.all(err <= 1e-6 * scale + 1e-6 * np.abs(an)), (key, float(np.max(err / scale)))
        checked += int(np.count_nonzero(an))
    assert checked > 300  # most of the 64 x 9 parameters receive gradient


def test_grad_colour_weights_telescope_to_alpha():
    # with bg = 0 and dL/d out_rgb = 1 on one channel: sum_g dL/d c_g = sum_p sum_i a_i T_i = sum_p (1 - T_N)
    sc, cam, proj, off, words, rgb, alpha, dC, dA = _grad_case(bg=(0.0, 0.0, 0.0))
    ones = np.zeros((cam.height, cam.width, 3), np.float32)
    ones[..., 1] = 1.0
    g = O.composite_grad(proj, off, words, cam.width, cam.height, ones)
    np.testing.assert_allclose(np.sum(g["rgb"][:, 1]), np.sum(alpha.astype(np.float64)), rtol=1e-6)
    assert np.all(g["rgb"][:, 0] == 0.0) and np.all(g["rgb"][:, 2] == 0.0)
    assert np.all(g["rgb"][:, 1] >= 0.0)


def test_grad_abs_sums_bound_the_gradient():
    sc, cam, proj, off, words, rgb, alpha, dC, dA = _grad_case()
    g = O.composite_grad(proj, off, words, cam.width, cam.height, dC, dA, bg=(0.2, 0.1, 0.3), with_abs=True)
    flat = np.concatenate([g["mean2d"], g["conic"], g["opacity"][:, None], g["rgb"]], axis=1)
    assert np.all(np.abs(flat) <= g["abs"] * (1 + 1e-12))


def test_grad_tile_subsets_partition_the_frame():
    # per-pixel terms only: the gradients of complementary tile subsets add up to the whole frame's
    sc, cam, proj, off, words, rgb, alpha, dC, dA = _grad_case()
    W, H = cam.width, cam.height
    full = O.composite_grad(proj, off, words, W, H, dC, dA, bg=(0.2, 0.1, 0.3))
    a = O.composite_grad(proj, off, words, W, H, dC, dA, bg=(0.2, 0.1, 0.3), tiles=[0, 3])
    b = O.composite_grad(proj, off, words, W, H, dC, dA, bg=(0.2, 0.1, 0.3), tiles=[1, 2])
    for k in full:
        np.testing.assert_allclose(a[k] + b[k], full[k], rtol=1e-12, atol=1e-14)
        assert np.any(a[k] != full[k])


def test_grad_at_float32_state_matches_exact_on_shallow_lists():
    # at the float32 forward's own alphas and transmittances the gradient moves
    # only by the forward's rounding (shallow lists: a few ulp per layer)
    sc, cam, proj, off, words, rgb, alpha, dC, dA = _grad_case()
    W, H = cam.width, cam.height
    ex = O.composite_grad(proj, off, words, W, H, dC, dA, bg=(0.2, 0.1, 0.3))
    f32 = O.composite_grad(proj, off, words, W, H, dC, dA, bg=(0.2, 0.1, 0.3), at_f32=True)
    for k in ex:
        rel = np.linalg.norm(f32[k] - ex[k]) / np.linalg.norm(ex[k])
        assert 0.0 < rel < 2e-6, (k, rel)


def test_grad_at_float32_state_closed_form_single_gaussian():
    # one Gaussian centred on the pixel: q = 0, exp(-q) = 1 and alpha = o
    # exactly in float32, so dL/dc = G o and dL/do = G.(c - bg) + dA
    P = _proj([0.5, 0.5], [0.8, 0.15, 0.5], [0.7], [0.9, 0.2, 0.6])
    bg = np.float32([0.1, 0.3, 0.05]).astype(np.float64)
    dC = np.float32([0.7, -1.3, 0.4]).astype(np.float64)
    dA = float(np.float32(-0.6))
    off, words = _one_tile_stream([0])
    g = O.composite_grad(P, off, words, 1, 1, dC.reshape(1, 1, 3), np.float32([[dA]]), bg=tuple(bg), at_f32=True)
    o = float(P["opacity"][0])
    col = P["rgb"][0].astype(np.float64)
    np.testing.assert_allclose(g["rgb"][0], dC * o, rtol=1e-15)
    np.testing.assert_allclose(g["opacity"][0], float(dC @ (col - bg)) + dA, rtol=1e-14)
    assert np.all(g["mean2d"] == 0.0) and np.all(g["conic"] == 0.0)
