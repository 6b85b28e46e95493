"""Failure detection on the device, in forms that fault and hang nothing.

* A bounded device wait that runs out: the projection's wait on its TMA copy
  of SH coefficients is given zero polls, so it gives up at once and raises
  GS_ERR_TIMEOUT in the context's sticky error word; the copy is still drained
  by the second bounded wait, so the frame is still the oracle's, and the
  context stays usable (the error clears, the next frame reports none).
* Non-finite inputs: NaN / +-inf planted in means, scales, quaternions,
  opacities and SH coefficients.  The defined behaviour is a cull plus
  GS_ERR_NUMERIC: the projection equals the oracle's bit for bit (which culls
  the same Gaussians), and so does the image, single-view and batched.
"""
import numpy as np
import pytest

import oracle as O
from paper_2609_03613_gb300 import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2609_03613_gb300 import tilegs as G  # noqa: E402

GS_ERR_TIMEOUT, GS_ERR_NUMERIC = 4, 6


def bits(a):
    return np.ascontiguousarray(a).view(np.uint32)


@pytest.mark.parametrize("mode", ["exact", "global"])
def test_projection_wait_that_runs_out_reports_timeout(mode):
    sc, cam = scenes.mixture_scene(20000, 12), scenes.hd_camera(width=480, height=270, f=275.0)
    _, _, _, (rgb_o, _, last_o) = O.render(sc, cam)
    ds = G.DeviceScene.from_numpy(sc)
    ctx = G.Context(mode, wait_polls=0)
    rgb, _, last = ctx.render(ds, cam)
    torch.cuda.synchronize()
    assert ctx.error() == GS_ERR_TIMEOUT
    # the drained copy still fed the projection: the frame is the oracle's
    np.testing.assert_array_equal(bits(rgb.cpu().numpy()), bits(rgb_o))
    np.testing.assert_array_equal(last.cpu().numpy(), last_o)
    # the context stays usable: with the default limit the next frame is clean
    ctx.clear_error()
    ctx.set_config(wait_polls=1 << 22)
    rgb2, _, _ = ctx.render(ds, cam)
    torch.cuda.synchronize()
    assert ctx.error() == 0
    np.testing.assert_array_equal(bits(rgb2.cpu().numpy()), bits(rgb_o))


def test_default_wait_limit_and_negative_limit_rejected():
    assert G.default_config("exact").wait_polls == 1 << 22
    with pytest.raises(G.TileGSError):
        G.Context("exact", wait_polls=-1)


@pytest.mark.parametrize("mode", ["exact", "global", "paper"])
def test_nonfinite_inputs_culled_with_numeric_error(mode):
    cam = scenes.hd_camera(width=480, height=270, f=275.0)
    sc, gids, kinds = scenes.plant_nonfinite(scenes.mixture_scene(30000, 11))
    assert "sh_overflow" in kinds
    P, _, _, (rgb_o, a_o, last_o) = O.render(sc, cam)
    ds = G.DeviceScene.from_numpy(sc)
    ctx = G.Context(mode)
    proj = ctx.project(ds, cam)
    torch.cuda.synchronize()
    assert ctx.error() == GS_ERR_NUMERIC
    f = {k: v.cpu().numpy() for k, v in G.projected_fields(proj, sc.n).items()}
    assert np.all(f["radius"][gids] == 0) and not P["visible"][gids].any()
    np.testing.assert_array_equal(f["radius"], P["radius"])
    vis = P["visible"] == 1
    np.testing.assert_array_equal(bits(f["xy_ab"][:, 0:2][vis]), bits(P["mean2d"][vis]))
    np.testing.assert_array_equal(bits(f["rgb"][:, 0:3][vis]), bits(P["rgb"][vis]))
    ctx.clear_error()
    rgb, alpha, last = ctx.render(ds, cam)
    torch.cuda.synchronize()
    assert ctx.error() == GS_ERR_NUMERIC
    if mode == "paper":  # approximate by design: finite and close, not equal
        assert np.isfinite(rgb.cpu().numpy()).all()
    else:
        np.testing.assert_array_equal(bits(rgb.cpu().numpy()), bits(rgb_o))
        np.testing.assert_array_equal(last.cpu().numpy(), last_o)
    # the same scene without the planted values reports nothing
    ctx.clear_error()
    ctx.render(G.DeviceScene.from_numpy(scenes.mixture_scene(30000, 11)), cam)
    torch.cuda.synchronize()
    assert ctx.error() == 0


def test_nonfinite_inputs_in_a_batch():
    sc, gids, _ = scenes.plant_nonfinite(scenes.mixture_scene(30000, 11))
    cams = [scenes.hd_camera(width=480, height=270, f=275.0),
            scenes.hd_camera(position=(0.5, 0.2, 3.2), width=320, height=240, f=200.0)]
    ds = G.DeviceScene.from_numpy(sc)
    ctx = G.Context("exact")
    outs = ctx.render_batch(ds, cams)
    torch.cuda.synchronize()
    assert ctx.error() == GS_ERR_NUMERIC
    for cam, (rgb, _, last) in zip(cams, outs):
        _, _, _, (rgb_o, _, last_o) = O.render(sc, cam)
        np.testing.assert_array_equal(bits(rgb.cpu().numpy()), bits(rgb_o))
        np.testing.assert_array_equal(last.cpu().numpy(), last_o)
