"""GPU parity of the raster-order-aware scene storage (gs_spatial_order,
gs_gather_rows) against the spatial-order oracle: the permutation bit for
bit (ragged sizes, duplicates, a flat axis, the 1M-Gaussian scene), the
gathers exactly, and the reordered scene's frame bit-exact against the
oracle's render of the same permuted scene."""
import numpy as np
import pytest

import oracle as O
from oracle import order as OR
from paper_2609_03613_gb300 import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2609_03613_gb300 import tilegs as G  # noqa: E402


@pytest.mark.parametrize("n", [1, 7, 2048, 2049, 100_003])
def test_spatial_order_matches_oracle_ragged(n):
    rng = np.random.Generator(np.random.PCG64(n))
    pts = (rng.normal(0.0, 2.0, (n, 3)) * np.array([1.0, 0.3, 3.0])).astype(np.float32)
    ctx = G.Context("exact")
    perm = ctx.spatial_order(torch.from_numpy(pts).cuda()).cpu().numpy()
    np.testing.assert_array_equal(perm, OR.spatial_order(pts))
    assert ctx.error() == 0


def test_spatial_order_duplicates_and_flat_axis():
    rng = np.random.Generator(np.random.PCG64(5))
    base = rng.random((300, 3)).astype(np.float32)
    pts = np.concatenate([base, base[::-1], base[:50]])  # every point two or three times
    pts[:, 1] = 0.25  # one axis with zero extent: its cells are all 0
    ctx = G.Context("exact")
    perm = ctx.spatial_order(torch.from_numpy(pts).cuda()).cpu().numpy()
    np.testing.assert_array_equal(perm, OR.spatial_order(pts))
    assert ctx.spatial_order(torch.zeros((0, 3), device="cuda")).shape == (0,)


def test_gather_rows_exact_and_bad_index_reported():
    rng = np.random.Generator(np.random.PCG64(6))
    n = 5003
    perm = rng.permutation(n).astype(np.int32)
    ctx = G.Context("exact")
    for width in (1, 3, 48):
        src = rng.normal(0, 1, (n, width)).astype(np.float32)
        got = ctx.gather_rows(torch.from_numpy(perm).cuda(), torch.from_numpy(src).cuda()).cpu().numpy()
        np.testing.assert_array_equal(got, src[perm])
    assert ctx.error() == 0
    bad = perm.copy()
    bad[17] = n  # out of range: the kernel skips the row and records the error
    ctx.gather_rows(torch.from_numpy(bad).cuda(), torch.zeros((n, 3), device="cuda"))
    torch.cuda.synchronize()
    assert ctx.error() == 1  # GS_ERR_INVALID_ARG
    ctx.clear_error()


def test_reordered_scene_frame_matches_oracle():
    sc = scenes.mixture_scene(200_000, 61)
    cam = scenes.hd_camera(width=640, height=360, f=370.0)
    ctx = G.Context("exact")
    ds = G.DeviceScene.from_numpy(sc)
    rs, perm = ctx.reorder_scene(ds)
    perm_o = OR.spatial_order(sc.means)
    np.testing.assert_array_equal(perm.cpu().numpy(), perm_o)
    psc = OR.permute_scene(sc, perm_o)
    for name in ("means", "scales", "quats", "opacities", "sh"):
        np.testing.assert_array_equal(getattr(rs, name).cpu().numpy(), getattr(psc, name))
    rgb, alpha, last = ctx.render(rs, cam)
    torch.cuda.synchronize()
    assert ctx.error() == 0
    _, _, (off_o, stream_o), (rgb_o, alpha_o, last_o) = O.render(psc, cam)
    np.testing.assert_array_equal(rgb.cpu().numpy().view(np.uint32), rgb_o.view(np.uint32))
    np.testing.assert_array_equal(last.cpu().numpy(), last_o)
    # against the original storage: the same picture except in tiles where two
    # Gaussians share a depth bit for bit (their tie order follows the gids)
    rgb0, _, _ = ctx.render(ds, cam)
    torch.cuda.synchronize()
    differ = np.any(rgb0.cpu().numpy() != rgb.cpu().numpy(), axis=2)
    zb = (stream_o >> np.uint64(32)).astype(np.int64)
    tie = np.zeros(len(off_o) - 1, bool)
    same = np.nonzero(zb[1:] == zb[:-1])[0]  # pairs of neighbours in the sorted stream
    tile_of = np.searchsorted(off_o, same, side="right") - 1
    tie[tile_of[np.searchsorted(off_o, same + 1, side="right") - 1 == tile_of]] = True
    ys, xs = np.nonzero(differ)
    tx = (cam.width + 15) // 16
    assert np.all(tie[(ys // 16) * tx + xs // 16]), "pixels differ outside tiles with depth ties"
    assert differ.mean() < 1e-3


def test_spatial_order_fullsize_mid():
    sc, _ = scenes.workload("mid")
    ctx = G.Context("exact")
    perm = ctx.spatial_order(torch.from_numpy(sc.means).cuda()).cpu().numpy()
    np.testing.assert_array_equal(perm, OR.spatial_order(sc.means))
