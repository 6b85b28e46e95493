"""GPU parity of the bin planner (K23) against the planner oracle, and the
guarantee that a plan changes speed only: whatever bins a plan gives each
tile's first pass, the two-pass frame is the oracle's image bit for bit.
The labels the raster logs (each tile's bins needed) equal the oracle's, and
the last test checks what the trained network saves on held-out renders in
work (entries left out of the first pass, tiles sent to the second), not in
time; the bench reports the time.
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


def _bias_only(cls):
    """Zero weights and an output bias that puts all probability on `cls`."""
    b3 = np.full(G.PLAN_CLASSES, -40.0)
    b3[cls] = 0.0
    P = np.zeros(G.PLAN_PARAMS, np.float32)
    P[-G.PLAN_CLASSES:] = b3
    return P


def test_plan_tiles_match_oracle():
    sc = scenes.mixture_scene(200_000, 61)
    cam = scenes.hd_camera(width=640, height=360, f=370.0)
    ctx, ds, proj, words, offsets = exact_frame(sc, cam)
    T = G.n_tiles(cam.width, cam.height)
    off = offsets.cpu().numpy()
    X = PL.tile_features(off, 64, T)
    seen = set()
    for seed, q in ((6, 0.9), (7, 0.5), (8, 0.99)):
        P = np.random.Generator(np.random.PCG64(seed)).normal(0.0, 0.06, G.PLAN_PARAMS).astype(np.float32)
        ctx.set_config(planner_quantile=q)
        ctx.set_planner_weights(torch.from_numpy(P))
        bins, cls = (t.cpu().numpy().astype(np.int64) for t in ctx.plan_tiles(cam, offsets))
        cls_o, bins_o = PL.plan(P.astype(np.float64), X, off, 64, T, q=q)
        # float32 against float64: only decisions near the quantile may differ
        z = PL.forward(P.astype(np.float64), X)[2]
        e = np.exp(z - z.max(axis=1, keepdims=True))
        cum = np.cumsum(e, axis=1) / e.sum(axis=1, keepdims=True)
        clear = np.abs(cum[:, :-1] - q).min(axis=1) > 1e-4
        np.testing.assert_array_equal(cls[clear], cls_o[clear])
        np.testing.assert_array_equal(bins[clear], bins_o[clear])
        np.testing.assert_array_equal(bins, PL.class_bins(off, 64, T, cls))  # bins of the GPU's own classes
        assert clear.mean() > 0.99
        seen |= set(cls.tolist())
    assert len(seen) >= 2, seen


def test_bins_needed_match_oracle():
    """The raster's logged label: the bins each tile needs, against the
    oracle's compositing of the same culled stream (segments sorted)."""
    sc = scenes.mixture_scene(150_000, 62)
    cam = scenes.hd_camera(width=480, height=270, f=280.0)
    ctx, ds, proj, words, offsets = exact_frame(sc, cam)
    T = G.n_tiles(cam.width, cam.height)
    needed = ctx.rasterize_fwd_plan(proj, ds.n, cam, words, offsets, needed=True)[4].cpu().numpy()
    m = int(offsets[-1].item())
    off = offsets.cpu().numpy()
    stream = O.sort_segments(off, words[:m].cpu().numpy().view(np.uint64))
    P = O.project(sc, cam)
    _, _, _, nt = O.composite(P, off, stream, cam.width, cam.height, K=64, ntests=True)
    ref = PL.bins_needed(off, 64, T, PL.tile_end_from_visits(off, 64, 16, cam.width, cam.height, nt))
    np.testing.assert_array_equal(needed, ref)
    lens = off[64:T * 64 + 1:64] - off[0:T * 64:64]
    assert (ref < 64).sum() > T // 10 and (ref[lens > 0] > 0).all()


def test_pass_flags_are_plan_below_needed():
    """One planned raster pass: a tile is flagged exactly when its plan gives
    it fewer bins than it needs, and every tile it does not flag is final
    (the oracle's pixels)."""
    sc = scenes.mixture_scene(250_000, 52)
    cam = scenes.hd_camera(width=517, height=301, f=320.0)
    bg = (0.1, 0.0, 0.2)
    ctx, ds, proj, words, offsets = exact_frame(sc, cam)
    _, _, _, (rgb_o, alpha_o, last_o) = O.render(sc, cam, bg=bg)
    T = G.n_tiles(cam.width, cam.height)
    needed = ctx.rasterize_fwd_plan(proj, ds.n, cam, words, offsets, needed=True)[4].cpu().numpy()
    off = offsets.cpu().numpy().astype(np.int64)
    lens = off[64:T * 64 + 1:64] - off[0:T * 64:64]
    tx = (cam.width + 15) // 16
    rng = np.random.Generator(np.random.PCG64(8))
    for plan in (np.zeros(T), np.full(T, 64), np.full(T, 200), rng.integers(0, 65, T), needed, needed - 1):
        plan = np.clip(plan, 0, 255).astype(np.uint8)
        rgb, alpha, last, flags, _ = ctx.rasterize_fwd_plan(proj, ds.n, cam, words, offsets,
                                                            plan=torch.from_numpy(plan).cuda(), flags=True, bg=bg)
        torch.cuda.synchronize()
        flags = flags.cpu().numpy()
        # flagged iff a pixel still composites when the plan's bins end and
        # later bins hold entries: exactly plan < needed
        want = (np.minimum(plan, 64) < needed)
        np.testing.assert_array_equal(flags.astype(bool), want)
        rgb, last = rgb.cpu().numpy(), last.cpu().numpy()
        for t in np.nonzero(~want)[0][:400]:
            y0, x0 = (t // tx) * 16, (t % tx) * 16
            sl = (slice(y0, y0 + 16), slice(x0, x0 + 16))
            np.testing.assert_array_equal(rgb[sl].view(np.uint32), rgb_o[sl].view(np.uint32))
            np.testing.assert_array_equal(last[sl], last_o[sl])
    assert ((needed > 0) & (needed < 64)).sum() > 0 and (lens > 0).sum() > T // 2
    assert ctx.error() == 0


@pytest.mark.parametrize("deep", [False, True])
def test_planned_frames_are_the_oracle_image(deep):
    """Whole two-pass frames (gs_render) under planners that put every tile
    in one class (0 sends most tiles to the second pass, 5 none), a random
    network, and the trained one: bit for bit the oracle's image, launched
    and graph-replayed.  deep: capacity reserved so that the bin scatter
    groups the row records (the deep-frame path)."""
    sc = scenes.mixture_scene(250_000, 54)
    cam = scenes.hd_camera(width=517, height=301, f=320.0)
    bg = (0.0, 0.3, 0.1)
    _, _, _, (rgb_o, alpha_o, last_o) = O.render(sc, cam, bg=bg)
    ds = G.DeviceScene.from_numpy(sc)
    planners = [("class%d" % c, _bias_only(c)) for c in range(G.PLAN_CLASSES)]
    planners.append(("random", np.random.Generator(np.random.PCG64(3)).normal(0, 0.3, G.PLAN_PARAMS)
                     .astype(np.float32)))
    if os.path.exists(PT.WEIGHTS):
        planners.append(("trained", np.load(PT.WEIGHTS).astype(np.float32)))
    side = torch.cuda.Stream()
    T = G.n_tiles(cam.width, cam.height)
    flagged = {}
    for name, P in planners:
        ctx = G.Context("exact", planner=1)
        ctx.set_planner_weights(torch.from_numpy(P))
        with torch.cuda.stream(side):
            out = ctx.render(ds, cam, bg)
            if deep:
                ctx.reserve(ds.n, 8192 * T, cam.width, cam.height)
                out = ctx.render(ds, cam, bg)
        torch.cuda.synchronize()
        flagged[name] = ctx.flagged_tiles()
        for k in range(2):
            np.testing.assert_array_equal(out[0].cpu().numpy().view(np.uint32), rgb_o.view(np.uint32), err_msg=name)
            np.testing.assert_array_equal(out[2].cpu().numpy(), last_o, err_msg=name)
            if k == 0:  # again as a replayed graph, outputs cleared first
                for t in out:
                    t.zero_()
                with torch.cuda.stream(side):
                    ctx.render(ds, cam, bg, out, flags=G.RENDER_GRAPH)
                    ctx.render(ds, cam, bg, out, flags=G.RENDER_GRAPH)
                torch.cuda.synchronize()
        assert ctx.error() == 0, name
    assert flagged["class0"] > T // 10 and flagged["class5"] == 0, flagged


def test_planner_render_requires_weights():
    sc, cam = scenes.mixture_scene(30_000, 53), scenes.hd_camera(width=320, height=180, f=184.0)
    ctx = G.Context("exact", planner=1)
    with pytest.raises(G.TileGSError, match="invalid argument"):
        ctx.render(G.DeviceScene.from_numpy(sc), cam)


def _trained():
    if not os.path.exists(PT.WEIGHTS):
        pytest.skip("no trained planner weights in the package")
    return np.load(PT.WEIGHTS).astype(np.float32)


def test_trained_planner_saves_work_on_held_out_renders():
    """What the trained network gains over building every bin, in work: on
    held-out renders (scenes and cameras not seen in training) its first pass
    scatters at most half of the entries while sending at most a tenth of
    the tiles to the second pass.  (Time is the bench's to report.)"""
    P = _trained()
    ctx = G.Context("exact")
    ctx.set_planner_weights(torch.from_numpy(P))
    kept = total = flagged = tiles = 0
    last_sc, ds = None, None
    for sc, cam in PT.training_renders(2, 4, 9100, 31000):
        if sc is not last_sc:
            ds, last_sc = G.DeviceScene.from_numpy(sc), sc
        proj, words, offsets = PT.frame(ctx, ds, cam)
        bins, _ = ctx.plan_tiles(cam, offsets)
        needed = ctx.rasterize_fwd_plan(proj, ds.n, cam, words, offsets, needed=True)[4]
        torch.cuda.synchronize()
        off = offsets.cpu().numpy().astype(np.int64)
        T = len(bins)
        b = bins.cpu().numpy().astype(np.int64)
        kept += int((off[np.arange(T) * 64 + b] - off[np.arange(T) * 64]).sum())
        total += int(off[T * 64] - off[0])
        flagged += int((b < needed.cpu().numpy()).sum())
        tiles += T
    print(f"trained planner, held out: first pass {kept / total:.1%} of entries, "
          f"{flagged / tiles:.1%} of tiles to the second pass")
    assert kept <= 0.5 * total and flagged <= 0.1 * tiles, (kept, total, flagged, tiles)
