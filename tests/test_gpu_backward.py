"""GPU parity of the raster backward (gs_rasterize_bwd) against the oracle's
analytic gradient (float32 decisions, fp64 arithmetic; pinned in
test_oracle_grad.py by closed forms and central finite differences).

Both sides start from their own projection and tile stream (bit-identical, as
the forward parity tests establish) and the same seeded upstream gradients.
The kernel works in float32 and sums per-pixel terms with float atomics, so
the bar is a tolerance, checked against two references:
  * the oracle gradient at the float32 forward's own state (its exp(-q),
    alphas and transmittances): what the kernel computes, up to its own
    rounding -- per tensor ||g - g_ref|| <= 1e-5 ||g_ref||, per element
    |g - g_ref| <= 2e-5 A + 1e-7 max|g_ref|;
  * the exact-arithmetic gradient: per tensor rel-err <= 1e-4 (the stated
    bar) and per element |g - g_ref| <= 1e-4 A + 1e-6 max|g_ref|.  On the
    1080p workload the float32 forward's own transmittance drifts from fp64
    by up to ~1e-4 relative deep in the ~100-layer pixel lists (rounding of q
    and alpha amplified by 1/(1 - a)), and the gradient inherits it; there
    the exact check is a sanity bound of 5e-4.
A is the oracle's error scale of the element: the sum over pixels of each
term's magnitude with dL/da_i = (G.c_i) T_i - (G.S_i - dA T_N)/(1 - a_i)
replaced by the sum of its two parts' magnitudes (a float32 evaluation of the
difference errs relative to those, not to the difference).
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
from paper_2609_03613_gb300 import autograd as GA  # noqa: E402

# oracle abs-term columns (mx, my, a, b, c, o, r, g, b) of each grad field slot
_SLOTS = {"xy_ab": [0, 1, 2, 3], "c_o_z": [4, 5], "rgb": [6, 7, 8]}


def gpu_frame(mode, sc, cam, tile=16, K=64, bg=(0.0, 0.0, 0.0)):
    ctx = G.Context(mode, K=K, tile_size=tile)
    ds = G.DeviceScene.from_numpy(sc)
    proj = ctx.project(ds, cam)
    isect, m_cap, m_dev, m = ctx.tile_intersect(proj, sc.n, cam)
    words, offsets, _ = ctx.sort_or_bin(proj, ds.scales, sc.n, cam, isect, m_cap, m_dev)
    rgb, alpha, _, saved = ctx.rasterize_fwd(proj, sc.n, cam, words, offsets, bg=bg, save=True)
    return ctx, ds, proj, words, offsets, rgb, alpha, saved


def gpu_grad(mode, sc, cam, dC, dA, tile=16, K=64, bg=(0.0, 0.0, 0.0)):
    ctx, ds, proj, words, offsets, rgb, alpha, saved = gpu_frame(mode, sc, cam, tile, K, bg)
    dCd = torch.from_numpy(dC).cuda()
    dAd = None if dA is None else torch.from_numpy(dA).cuda()
    grad = ctx.rasterize_bwd(proj, sc.n, cam, words, offsets, saved, dCd, dAd)
    torch.cuda.synchronize()
    assert ctx.error() == 0
    return {k: v.cpu().numpy() for k, v in G.grad_fields(grad, sc.n).items()}


def oracle_grad(sc, cam, dC, dA, tile=16, bg=(0.0, 0.0, 0.0), tiles=None, at_f32=False):
    proj = O.project(sc, cam, tile)
    tx, ty = O.tiles_xy(cam.width, cam.height, tile)
    off, words = O.sort_tiles(O.emit(proj, cam.width, cam.height, tile), tx * ty)
    return O.composite_grad(proj, off, words, cam.width, cam.height, dC, dA, tile=tile, bg=bg,
                            with_abs=True, tiles=tiles, at_f32=at_f32)


def oracle_grads(sc, cam, dC, dA, **kw):
    return oracle_grad(sc, cam, dC, dA, **kw), oracle_grad(sc, cam, dC, dA, at_f32=True, **kw)


def as_slots(g):
    """Oracle gradient in the kernel's [n,4] field layout."""
    n = g["opacity"].shape[0]
    xy = np.zeros((n, 4))
    xy[:, 0:2] = g["mean2d"]
    xy[:, 2:4] = g["conic"][:, 0:2]
    coz = np.zeros((n, 4))
    coz[:, 0] = g["conic"][:, 2]
    coz[:, 1] = g["opacity"]
    rgb = np.zeros((n, 4))
    rgb[:, 0:3] = g["rgb"]
    return {"xy_ab": xy, "c_o_z": coz, "rgb": rgb}


def assert_grad_close(got, ref, rel_tol=1e-4, tau=1e-4, atol_frac=1e-6):
    want = as_slots(ref)
    for field, cols in _SLOTS.items():
        g = got[field][:, :len(cols)].astype(np.float64)
        r = want[field][:, :len(cols)]
        A = ref["abs"][:, cols]
        assert np.all(got[field][:, len(cols):] == 0.0), field
        rel = np.linalg.norm(g - r) / max(np.linalg.norm(r), 1e-300)
        assert rel <= rel_tol, (field, rel)
        err = np.abs(g - r)
        bound = tau * A + atol_frac * np.max(np.abs(r))
        worst = np.unravel_index(np.argmax(err - bound), err.shape)
        assert np.all(err <= bound), (field, worst, float(g[worst]), float(r[worst]), float(A[worst]))


def assert_both(got, exact, f32, exact_rel=1e-4):
    assert_grad_close(got, f32, rel_tol=1e-5, tau=2e-5, atol_frac=1e-7)
    assert_grad_close(got, exact, rel_tol=exact_rel)


@pytest.mark.parametrize("mode", ["global", "exact"])
def test_bwd_grad_check_scene(mode):
    sc, cam = scenes.grad_check_scene()
    bg = (0.2, 0.1, 0.3)
    dC, dA = scenes.incoming_grads(cam.height, cam.width, seed=11)
    got = gpu_grad(mode, sc, cam, dC, dA, bg=bg)
    assert_both(got, *oracle_grads(sc, cam, dC, dA, bg=bg))


@pytest.mark.parametrize("mode,tile", [("exact", 16), ("global", 16), ("exact", 8), ("exact", 32)])
def test_bwd_mixture_ragged_frame(mode, tile):
    # several hundred tiles with ragged right and bottom edges, long spans
    # (EXACT: chunks of in-raster sorted segments), no dL/dalpha
    sc = scenes.mixture_scene(120_000, 31)
    cam = scenes.hd_camera(width=500, height=284, f=300.0)
    dC, _ = scenes.incoming_grads(cam.height, cam.width, seed=12)
    got = gpu_grad(mode, sc, cam, dC, None, tile=tile)
    assert_both(got, *oracle_grads(sc, cam, dC, None, tile=tile))


def test_bwd_mid_workload_sampled_tiles():
    # the 1080p / 1M-Gaussian workload, with the upstream gradient nonzero on
    # 24 seeded tiles only: the gradient is then the sum over those tiles, which
    # the oracle computes tile by tile
    sc, cam = scenes.workload("mid")
    T = G.n_tiles(cam.width, cam.height)
    rng = np.random.Generator(np.random.PCG64(77))
    tiles = np.sort(rng.choice(T, 24, replace=False))
    dC, dA = scenes.incoming_grads(cam.height, cam.width, seed=13)
    mask = np.zeros((cam.height, cam.width), bool)
    tx = (cam.width + 15) // 16
    for t in tiles:
        y0, x0 = (t // tx) * 16, (t % tx) * 16
        mask[y0:y0 + 16, x0:x0 + 16] = True
    dC[~mask] = 0.0
    dA[~mask] = 0.0
    got = gpu_grad("exact", sc, cam, dC, dA)
    exact, f32 = oracle_grads(sc, cam, dC, dA, tiles=tiles)
    assert_grad_close(got, f32, rel_tol=1e-5, tau=2e-5, atol_frac=1e-7)
    assert_grad_close(got, exact, rel_tol=5e-4, tau=5e-4)


def test_bwd_zero_upstream_gives_zero_and_empty_scene():
    sc, cam = scenes.grad_check_scene()
    z = np.zeros((cam.height, cam.width, 3), np.float32)
    got = gpu_grad("exact", sc, cam, z, None)
    assert all(np.all(v == 0.0) for v in got.values())
    # a scene entirely behind the camera: no entries, all-zero gradient
    sc2 = scenes.Scene(sc.means + np.float32([0, 0, 10]), sc.scales, sc.quats, sc.opacities, sc.sh, 0)
    got2 = gpu_grad("exact", sc2, cam, np.ones_like(z), None)
    assert all(np.all(v == 0.0) for v in got2.values())


def test_bwd_rejects_bad_arguments():
    sc, cam = scenes.grad_check_scene()
    ctx, ds, proj, words, offsets, rgb, alpha, saved = gpu_frame("exact", sc, cam)
    dC = torch.zeros_like(rgb)
    grad = torch.empty(int(G.lib().gs_grad2d_bytes(sc.n)) + 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(G.TileGSError, match="invalid argument"):
        ctx.rasterize_bwd(proj, sc.n, cam, words, offsets, saved, dC, grad=grad[16:])  # misaligned
    with pytest.raises(G.TileGSError, match="invalid argument"):
        ctx.rasterize_bwd(proj, sc.n, cam, words, offsets, saved, dC, stride=G.MAX_K + 1)
    with pytest.raises(G.TileGSError, match="invalid argument"):
        ctx.rasterize_bwd(proj, sc.n, cam, words, offsets, G.Saved(saved.last, None, saved.tile_end, saved.bg), dC)
    torch.cuda.synchronize()
    assert ctx.error() == 0


def test_autograd_l1_step_matches_direct_backward():
    sc, cam = scenes.grad_check_scene()
    ctx, ds, proj, words, offsets, rgb0, alpha0, saved = gpu_frame("exact", sc, cam)
    f = G.projected_fields(proj, sc.n)
    xy, coz, col = (f[k].requires_grad_() for k in ("xy_ab", "c_o_z", "rgb"))
    frame = GA.Frame(ctx, proj, sc.n, cam, words, offsets, ctx.stride)
    target = torch.from_numpy(scenes.random_target(cam.height, cam.width, seed=5)).cuda()
    img, alpha = GA.rasterize(xy, coz, col, frame)
    assert torch.equal(img, rgb0) and torch.equal(alpha, alpha0)
    loss = (img - target).abs().mean()
    loss.backward()
    dl = (torch.sign(img.detach() - target) / img.numel()).contiguous()
    grad = ctx.rasterize_bwd(proj, sc.n, cam, words, offsets, saved, dl)
    ref = G.grad_fields(grad, sc.n)
    for k, t in (("xy_ab", xy), ("c_o_z", coz), ("rgb", col)):
        np.testing.assert_allclose(t.grad.cpu().numpy(), ref[k].cpu().numpy(), rtol=1e-5,
                                   atol=1e-6 * float(ref[k].abs().max()))
    # and the same against the oracle
    dln = dl.cpu().numpy()
    assert_both({k: v.grad.cpu().numpy() for k, v in (("xy_ab", xy), ("c_o_z", coz), ("rgb", col))},
                *oracle_grads(sc, cam, dln, None))


def test_render_save_then_render_bwd_whole_frame_and_graph_replay():
    sc = scenes.mixture_scene(120_000, 32)
    cam = scenes.hd_camera(width=500, height=284, f=300.0)
    bg = (0.1, 0.2, 0.3)
    dC, dA = scenes.incoming_grads(cam.height, cam.width, seed=14)
    dCd, dAd = torch.from_numpy(dC).cuda(), torch.from_numpy(dA).cuda()
    ctx = G.Context("exact")
    ds = G.DeviceScene.from_numpy(sc)
    ctx.render(ds, cam, bg, flags=G.RENDER_SAVE)
    got = {k: v.cpu().numpy() for k, v in G.grad_fields(ctx.render_bwd(dCd, dAd), sc.n).items()}
    torch.cuda.synchronize()
    assert ctx.error() == 0
    assert_both(got, *oracle_grads(sc, cam, dC, dA, bg=bg))
    # the same frame replayed from a CUDA graph, backward after each replay
    side = torch.cuda.Stream()
    out = tuple(torch.empty(s, dtype=d, device="cuda") for s, d in (((cam.height, cam.width, 3), torch.float32),
                                                                    ((cam.height, cam.width), torch.float32),
                                                                    ((cam.height, cam.width), torch.int32)))
    grad = torch.empty(int(G.lib().gs_grad2d_bytes(sc.n)), dtype=torch.uint8, device="cuda")
    with torch.cuda.stream(side):
        for _ in range(3):
            ctx.render(ds, cam, bg, out, flags=G.RENDER_NO_SYNC | G.RENDER_GRAPH | G.RENDER_SAVE)
            ctx.render_bwd(dCd, dAd, grad=grad)
    torch.cuda.synchronize()
    assert ctx.error() == 0
    rep = {k: v.cpu().numpy() for k, v in G.grad_fields(grad, sc.n).items()}
    for k in got:
        np.testing.assert_allclose(rep[k], got[k], rtol=1e-5, atol=1e-6 * float(np.abs(got[k]).max()))
    # a frame rendered without RENDER_SAVE leaves nothing to differentiate
    ctx.render(ds, cam, bg)
    with pytest.raises(G.TileGSError, match="invalid argument"):
        ctx.render_bwd(dCd, dAd)


def test_reciprocal_within_one_rounding():
    """The backward's reciprocal (hardware approximation + one Newton-Raphson
    step) against the correctly rounded 1/x, for every float32 x in
    [0.01, 1] (the backward takes 1/(1 - a) with a in [1/255, 0.99]): at most
    one unit in the last place away, and equal for nearly all."""
    lo = int(np.float32(0.01).view(np.int32))
    hi = int(np.float32(1.0).view(np.int32))
    bits_x = torch.arange(lo, hi + 1, dtype=torch.int32, device="cuda")
    x = bits_x.view(torch.float32)
    got = G.reciprocal(x)
    ref = (1.0 / x.double()).float()  # the exact quotient rounded once more
    ulp = (got.view(torch.int32).long() - ref.view(torch.int32).long()).abs()
    assert int(ulp.max().item()) <= 1
    assert float((ulp == 0).double().mean().item()) > 0.99
    with pytest.raises(G.TileGSError):
        G.check(G.lib().gs_reciprocal(None, None, -1, None))
