"""GPU parity on the heavy depth-complexity workloads (3M Gaussians at
1920x1080 and 6M at 3840x2160, cameras inside dense clusters: per-tile
ranges of ~18k-70k Gaussians): the frame as bench.py runs it (gs_render,
reserved scratch, no host read of the entry count) for the binned EXACT
path, the same path with the trained bin planner and the global-sort
baseline, checked bit for bit on seeded tiles (plus the deepest) composited
by the oracle from their brute-force lists, and the three images against each
other in full."""
import os

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
from paper_2609_03613_gb300 import planner_train as PT  # noqa: E402


def bits(a):
    return np.ascontiguousarray(a).view(np.uint32)


@pytest.mark.parametrize("name", ["heavy3m", "heavy6m_4k"])
def test_heavy_sampled_tiles_exact_planner_global(name):
    sc, cam = scenes.workload(name)
    O.set_threads(max(1, len(os.sched_getaffinity(0))))
    P = O.project(sc, cam)
    tx, ty = O.tiles_xy(cam.width, cam.height)
    cnt = tile_counts(P, tx, ty)
    M = int(cnt.sum())
    assert np.percentile(cnt, 50) > 10_000  # deep per-tile ranges, as the workload asks
    rng = np.random.default_rng(7 + len(name))
    tiles = np.unique(np.concatenate([rng.choice(tx * ty, 24, replace=False), np.argsort(cnt)[-4:]]))
    off, stream = sampled_stream(P, tiles, tx, ty)
    assert np.array_equal(np.diff(off)[tiles], cnt[tiles])
    rgb_o, a_o, l_o = O.composite(P, off, stream, cam.width, cam.height, tiles=tiles.astype(np.int32))

    ds = G.DeviceScene.from_numpy(sc)
    H, W = cam.height, cam.width
    weights = np.load(PT.WEIGHTS).astype(np.float32) if os.path.exists(PT.WEIGHTS) else None
    images = {}
    for label, mode, kw in (("exact", "exact", {}), ("planner", "exact", {"planner": 1}), ("global", "global", {})):
        if label == "planner" and weights is None:
            continue
        ctx = G.Context(mode, **kw)
        if label == "planner":
            ctx.set_planner_weights(torch.from_numpy(weights))
        ctx.reserve(sc.n, int(M * 1.05) + 1024, W, H)
        out = (torch.empty((H, W, 3), device="cuda"), torch.empty((H, W), device="cuda"),
               torch.empty((H, W), dtype=torch.int32, device="cuda"))
        ctx.render(ds, cam, out=out, flags=G.RENDER_NO_SYNC)
        torch.cuda.synchronize()
        assert ctx.error() == 0, label
        rgb, alpha, last = [t.cpu().numpy() for t in out]
        ctx.close()
        del out
        torch.cuda.empty_cache()
        images[label] = (rgb, last)
        for t in tiles:
            y, x = divmod(int(t), tx)
            ys, xs = slice(y * 16, min(y * 16 + 16, H)), slice(x * 16, min(x * 16 + 16, W))
            np.testing.assert_array_equal(bits(rgb[ys, xs]), bits(rgb_o[ys, xs]))
            np.testing.assert_array_equal(bits(alpha[ys, xs]), bits(a_o[ys, xs]))
            np.testing.assert_array_equal(last[ys, xs], l_o[ys, xs])
    for label in images:
        np.testing.assert_array_equal(bits(images[label][0]), bits(images["exact"][0]))
        np.testing.assert_array_equal(images[label][1], images["exact"][1])
