"""GPU parity of the bin planner (K23) against the planner oracle, and the
guarantee that a plan changes speed only: any per-tile chunk plan gives the
oracle's image bit for bit.  The last test measures what the trained network
gains over the fixed chunk size on held-out renders.
"""
import os

import numpy as np
import pytest

import oracle as O
from oracle import planner as PL
from paper_2609_03613_gb300 import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2609_03613_gb300 import tilegs as G  # noqa: E402
from paper_2609_03613_gb300 import planner_train as PT  # noqa: E402


def exact_frame(sc, cam, K=64):
    ctx = G.Context("exact", K=K)
    ds = G.DeviceScene.from_numpy(sc)
    proj, words, offsets = PT.frame(ctx, ds, cam)
    torch.cuda.synchronize()
    return ctx, ds, proj, words, offsets


@pytest.mark.parametrize("K", [64, 128, 16])
def test_tile_features_match_oracle(K):
    sc = scenes.mixture_scene(200_000, 51)
    cam = scenes.hd_camera(width=640, height=360, f=370.0)
    ctx, ds, proj, words, offsets = exact_frame(sc, cam, K)
    f = ctx.tile_features(cam, offsets).cpu().numpy()
    T = G.n_tiles(cam.width, cam.height)
    ref = PL.tile_features(offsets.cpu().numpy(), K, T)
    np.testing.assert_allclose(f, ref, rtol=5e-7, atol=1e-6)
    assert np.count_nonzero(ref[:, 0]) > T // 2


def _random_batch(seed, B):
    rng = np.random.Generator(np.random.PCG64(seed))
    X = rng.normal(0.0, 1.5, (B, G.PLAN_FEATURES)).astype(np.float32)
    y = rng.integers(0, G.PLAN_CLASSES, B).astype(np.int32)
    P = rng.normal(0.0, 0.25, G.PLAN_PARAMS).astype(np.float32)
    return X, y, P


def test_mlp_forward_loss_backward_match_oracle():
    X, y, P = _random_batch(5, 1000)
    Xd, yd, Pd = (torch.from_numpy(a).cuda() for a in (X, y, P))
    acts, logits = G.mlp_forward(Pd, Xd)
    loss, dz = G.mlp_loss_grad(logits, yd)
    grads = G.mlp_backward(Pd, Xd, acts, dz)
    torch.cuda.synchronize()
    h1, h2, z = PL.forward(P.astype(np.float64), X.astype(np.float64))
    np.testing.assert_allclose(logits.cpu().numpy(), z, rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(acts.cpu().numpy(), np.concatenate([h1, h2], axis=1), rtol=1e-5, atol=1e-5)
    l_ref, dz_ref = PL.xent(z, y)
    assert abs(float(loss.item()) - l_ref) <= 1e-5 * abs(l_ref)
    np.testing.assert_allclose(dz.cpu().numpy(), dz_ref, rtol=1e-4, atol=1e-8)
    g_ref = PL.backward(P.astype(np.float64), X.astype(np.float64), h1, h2, dz_ref)
    g = grads.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    assert rel <= 1e-4, rel


def test_adam_step_matches_oracle():
    rng = np.random.Generator(np.random.PCG64(9))
    p, g, m, v = (rng.normal(0, 1, G.PLAN_PARAMS).astype(np.float32) for _ in range(4))
    v = np.abs(v)
    pd, gd, md, vd = (torch.from_numpy(a.copy()).cuda() for a in (p, g, m, v))
    G.adam_step(pd, gd, md, vd, 7, 1e-3)
    torch.cuda.synchronize()
    p2, m2, v2 = PL.adam(p.astype(np.float64), g.astype(np.float64), m, v, 7, lr=1e-3)
    np.testing.assert_allclose(pd.cpu().numpy(), p2, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(md.cpu().numpy(), m2, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(vd.cpu().numpy(), v2, rtol=1e-5, atol=1e-7)


def test_plan_tiles_is_oracle_argmax():
    X, _, P = _random_batch(6, 5000)
    ctx = G.Context("exact")
    ctx.set_planner_weights(torch.from_numpy(P))
    plan = ctx.plan_tiles(torch.from_numpy(X).cuda()).cpu().numpy()
    z = PL.forward(P.astype(np.float64), X.astype(np.float64))[2]
    top2 = np.sort(z, axis=1)[:, -2:]
    clear = (top2[:, 1] - top2[:, 0]) > 1e-3  # float32 vs float64 can swap near-ties only
    np.testing.assert_array_equal(plan[clear], np.argmax(z, axis=1)[clear])
    assert clear.mean() > 0.99


def test_any_plan_gives_the_oracle_image():
    sc = scenes.mixture_scene(250_000, 52)
    cam = scenes.hd_camera(width=517, height=301, f=320.0)
    bg = (0.1, 0.0, 0.2)
    ctx, ds, proj, words, offsets = exact_frame(sc, cam)
    _, _, _, (rgb_o, alpha_o, last_o) = O.render(sc, cam, bg=bg)
    T = G.n_tiles(cam.width, cam.height)
    rng = np.random.Generator(np.random.PCG64(8))
    for plan in (None, np.zeros(T), np.full(T, 5), rng.integers(0, G.PLAN_CLASSES, T)):
        p = None if plan is None else torch.from_numpy(plan.astype(np.uint8)).cuda()
        rgb, alpha, last, cyc = ctx.rasterize_fwd_plan(proj, ds.n, cam, words, offsets, plan=p, cycles=True, bg=bg)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(rgb.cpu().numpy().view(np.uint32), rgb_o.view(np.uint32))
        np.testing.assert_array_equal(last.cpu().numpy(), last_o)
        assert np.all(cyc.cpu().numpy() > 0)
    assert ctx.error() == 0


def _trained():
    if not os.path.exists(PT.WEIGHTS):
        pytest.skip("no trained planner weights in the package")
    return np.load(PT.WEIGHTS).astype(np.float32)


def test_planner_render_matches_oracle_and_fixed():
    P = _trained()
    sc, cam = scenes.mixture_scene(300_000, 53), scenes.hd_camera(width=800, height=450, f=460.0)
    ctx = G.Context("exact", planner=1)
    ctx.set_planner_weights(torch.from_numpy(P))
    ds = G.DeviceScene.from_numpy(sc)
    rgb, alpha, last = ctx.render(ds, cam)
    torch.cuda.synchronize()
    assert ctx.error() == 0
    _, _, _, (rgb_o, alpha_o, last_o) = O.render(sc, cam)
    np.testing.assert_array_equal(rgb.cpu().numpy().view(np.uint32), rgb_o.view(np.uint32))
    np.testing.assert_array_equal(last.cpu().numpy(), last_o)
    # without weights the planner-on context refuses to render
    ctx2 = G.Context("exact", planner=1)
    with pytest.raises(G.TileGSError, match="invalid argument"):
        ctx2.render(ds, cam)


def test_trained_planner_gain_on_held_out_renders():
    """What the trained network gains over the fixed chunk size: raster time
    summed over held-out renders (scenes and cameras not seen in training),
    images bit-identical (checked inside evaluate)."""
    P = _trained()
    res = PT.evaluate(P, PT.training_renders(2, 4, 9100, 31000), iters=15)
    fixed = sum(a for a, _ in res)
    planned = sum(b for _, b in res)
    gain = 1.0 - planned / fixed
    print(f"planner gain on held-out renders: {gain:+.3%} (fixed {fixed:.3f} ms, planned {planned:.3f} ms)")
    assert gain > 0.0, (fixed, planned)
