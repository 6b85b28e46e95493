"""gs_depth_range_noalloc against gs_depth_range.

Callers that cannot allocate device memory -- their device memory belongs to
their own allocator or budget, or a cudaMalloc would synchronise the device
under work in flight -- use the entry point that needs no context and keeps its
scratch in a static device array.  It must give the same depth range as the
context-based entry point, call after call, whatever the previous call left in
the shared scratch.
"""
import numpy as np
import pytest

from paper_2609_03613_gb300 import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2609_03613_gb300 import tilegs as G  # noqa: E402


def _inputs(mode, seed):
    sc = scenes.mixture_scene(150000, seed)
    cam = scenes.hd_camera()
    ctx = G.Context(mode)
    ds = G.DeviceScene.from_numpy(sc)
    proj = ctx.project(ds, cam)
    isect, m_cap, m_dev, m = ctx.tile_intersect(proj, sc.n, cam)
    ref = ctx.depth_range(proj, ds.scales, sc.n, cam, isect, m_cap, m_dev)
    torch.cuda.synchronize()
    return sc, cam, ds, proj, isect, m_cap, m_dev, ref.cpu().numpy()


@pytest.mark.parametrize("mode", ["exact", "paper"])
def test_noalloc_depth_range_matches_context_entry_point(mode):
    cfg = G.default_config(mode)
    # two different inputs, each called twice in a row: the shared scratch
    # carries the previous call's record into the next call
    for seed in (71, 72):
        sc, cam, ds, proj, isect, m_cap, m_dev, ref = _inputs(mode, seed)
        for _ in range(2):
            zr = torch.full((2,), -1.0, dtype=torch.float32, device="cuda")
            G.depth_range_noalloc(cfg, proj, ds.scales, sc.n, cam, isect, m_cap, m_dev, zr)
            torch.cuda.synchronize()
            got = zr.cpu().numpy()
            np.testing.assert_array_equal(got.view(np.uint32), ref.view(np.uint32))
            assert 0.0 < got[0] < got[1]


def test_noalloc_rejects_sizes_beyond_its_scratch():
    sc, cam, ds, proj, isect, m_cap, m_dev, ref = _inputs("exact", 73)
    zr = torch.zeros(2, dtype=torch.float32, device="cuda")
    for field, value in (("K", G.MAX_K + 1), ("sample_count", 8193)):
        cfg = G.default_config("exact")
        setattr(cfg, field, value)
        with pytest.raises(G.TileGSError, match="invalid argument"):
            G.depth_range_noalloc(cfg, proj, ds.scales, sc.n, cam, isect, m_cap, m_dev, zr)
    torch.cuda.synchronize()
    assert np.all(zr.cpu().numpy() == 0.0)  # nothing was enqueued
