"""GPU parity of the batched multi-view render (gs_render_batch) and the
per-view autotuner: every view's image and last ids are bit-identical to the
oracle's frame for that camera at the view's tile size (and to a single-view
gs_render with the view's configuration), plain, graph-replayed and after
autotuning.
"""
import numpy as np
import pytest

import oracle as O
from paper_2609_03613_gb300 import scenes
from sampling import sampled_stream, tile_counts

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2609_03613_gb300 import tilegs as G  # noqa: E402


def small_batch():
    sc = scenes.mixture_scene(60_000, 41)
    cams = [scenes.hd_camera(width=320, height=200, f=220.0),
            scenes.hd_camera(position=(0.4, 0.3, 2.6), width=257, height=129, f=180.0),
            scenes.hd_camera(position=(-0.5, 0.2, 3.2), width=128, height=128, f=120.0),
            scenes.hd_camera(position=(0.0, -0.6, 2.8), width=400, height=224, f=260.0)]
    return sc, cams


def oracle_view(sc, cam, tile, bg):
    _, _, _, (rgb, alpha, last) = O.render(sc, cam, tile=tile, bg=bg)
    return rgb, alpha, last


def assert_view_equal(out, ref):
    rgb, alpha, last = (t.cpu().numpy() for t in out)
    np.testing.assert_array_equal(rgb.view(np.uint32), ref[0].view(np.uint32))
    np.testing.assert_array_equal(alpha.view(np.uint32), ref[1].view(np.uint32))
    np.testing.assert_array_equal(last, ref[2])


@pytest.mark.parametrize("mode", ["exact", "global"])
def test_batch_views_match_oracle_with_per_view_configs(mode):
    sc, cams = small_batch()
    bg = (0.05, 0.1, 0.2)
    ctx = G.Context(mode)
    tiles = [16, 8, 32, 16]
    for v, t in enumerate(tiles):
        ctx.set_batch_view_config(v, tile_size=t, K=[64, 32, 128, 16][v])
    ds = G.DeviceScene.from_numpy(sc)
    l0 = ctx.launch_count()
    outs = ctx.render_batch(ds, cams, bg)
    torch.cuda.synchronize()
    assert ctx.error() == 0
    assert ctx.launch_count() > l0
    for v, cam in enumerate(cams):
        assert ctx.batch_view_config(v).tile_size == tiles[v]
        assert_view_equal(outs[v], oracle_view(sc, cam, tiles[v], bg))
        assert ctx.batch_entry_count(v) > 0


def test_batch_graph_replay_matches_single_view_renders():
    sc, cams = small_batch()
    bg = (0.0, 0.0, 0.0)
    ctx = G.Context("exact")
    ds = G.DeviceScene.from_numpy(sc)
    outs = ctx.render_batch(ds, cams, bg)  # sizes every view
    torch.cuda.synchronize()
    ref = [tuple(t.clone() for t in o) for o in outs]
    for o in outs:
        for t in o:
            t.zero_()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        for _ in range(3):
            ctx.render_batch(ds, cams, bg, outs, flags=G.RENDER_NO_SYNC | G.RENDER_GRAPH)
    torch.cuda.synchronize()
    assert ctx.error() == 0
    for o, r in zip(outs, ref):
        for a, b in zip(o, r):
            assert torch.equal(a, b)
    # each view equals a single-view gs_render of that camera
    single = G.Context("exact")
    for cam, o in zip(cams, outs):
        s = single.render(ds, cam, bg)
        torch.cuda.synchronize()
        for a, b in zip(o, s):
            assert torch.equal(a, b)


def test_batch_autotune_picks_candidates_and_keeps_images():
    sc, cams = small_batch()
    cams = cams[:2]
    ctx = G.Context("exact")
    ds = G.DeviceScene.from_numpy(sc)
    best = ctx.batch_autotune(ds, cams, tune_tile=True, iters=2)
    assert len(best) == 2 and all(t > 0.0 for t in best)
    for v, cam in enumerate(cams):
        cfg = ctx.batch_view_config(v)
        assert cfg.tile_size in (8, 16, 32) and cfg.K in (32, 64, 128)
    outs = ctx.render_batch(ds, cams)
    torch.cuda.synchronize()
    assert ctx.error() == 0
    for v, cam in enumerate(cams):
        assert_view_equal(outs[v], oracle_view(sc, cam, ctx.batch_view_config(v).tile_size, (0.0, 0.0, 0.0)))


def test_batch_rejects_bad_arguments():
    sc, cams = small_batch()
    ctx = G.Context("exact")
    ds = G.DeviceScene.from_numpy(sc)
    with pytest.raises(G.TileGSError, match="invalid argument"):
        ctx.render_batch(ds, cams[:1] * (G.MAX_VIEWS + 1))
    with pytest.raises(G.TileGSError, match="invalid argument"):
        ctx.render_batch(ds, cams, flags=G.RENDER_HOST_OUTPUTS)
    with pytest.raises(G.TileGSError, match="invalid argument"):
        ctx.set_batch_view_config(G.MAX_VIEWS, tile_size=16)
    torch.cuda.synchronize()
    assert ctx.error() == 0


def test_batch16_fullsize_autotuned_sampled_tiles():
    """The 16-view workload as bench.py runs it (2M Gaussians, resolutions
    512x512 .. 1920x1080, autotuned tile size and K per view, the batch as
    one graph): on seeded tiles of every view (plus its deepest) bit-exact
    against the oracle's compositing at that view's tile size."""
    import os
    sc, cams = scenes.workload("batch16")
    O.set_threads(max(1, len(os.sched_getaffinity(0))))
    ctx = G.Context("exact")
    ds = G.DeviceScene.from_numpy(sc)
    ctx.batch_autotune(ds, cams, tune_tile=True, iters=2)
    outs = ctx.render_batch(ds, cams)  # sizes the views
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        for _ in range(2):
            ctx.render_batch(ds, cams, (0.0, 0.0, 0.0), outs, flags=G.RENDER_NO_SYNC | G.RENDER_GRAPH)
    torch.cuda.synchronize()
    assert ctx.error() == 0
    rng = np.random.default_rng(16)
    for v, cam in enumerate(cams):
        tile = ctx.batch_view_config(v).tile_size
        P = O.project(sc, cam, tile)
        tx, ty = O.tiles_xy(cam.width, cam.height, tile)
        cnt = tile_counts(P, tx, ty)
        tiles = np.unique(np.concatenate([rng.choice(tx * ty, 5, replace=False), np.argsort(cnt)[-1:]]))
        off, stream = sampled_stream(P, tiles, tx, ty)
        rgb_o, a_o, l_o = O.composite(P, off, stream, cam.width, cam.height, tile, tiles=tiles.astype(np.int32))
        rgb, alpha, last = (t.cpu().numpy() for t in outs[v])
        for t in tiles:
            y, x = divmod(int(t), tx)
            ys = slice(y * tile, min(y * tile + tile, cam.height))
            xs = slice(x * tile, min(x * tile + tile, cam.width))
            np.testing.assert_array_equal(rgb[ys, xs].view(np.uint32), rgb_o[ys, xs].view(np.uint32))
            np.testing.assert_array_equal(alpha[ys, xs].view(np.uint32), a_o[ys, xs].view(np.uint32))
            np.testing.assert_array_equal(last[ys, xs], l_o[ys, xs])
