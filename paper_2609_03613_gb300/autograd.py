"""torch.autograd binding of the raster forward and backward.

The differentiable inputs are the projected record's own 2D fields
(``projected_fields(buf, n)``: xy_ab = {mean_x, mean_y, conic_a, conic_b},
c_o_z = {conic_c, opacity, depth, cull_tau}, rgb = {r, g, b, cull_margin});
gradients come back in the same [n,4] layout (zero in the depth and cull
slots).  Every step runs in libtilegs.so: gs_rasterize_fwd (saving the
final transmittance and each tile's end position) for the forward and
gs_rasterize_bwd, which walks the tiles in the forward's order reversed, for
the backward.
"""
from __future__ import annotations

import dataclasses

import torch

from . import tilegs as G


@dataclasses.dataclass
class Frame:
    """What the raster needs besides the differentiable fields: the context
    (its configuration fixes the mode and tile size), the projected buffer the
    fields live in, the tile-major stream and its offsets."""
    ctx: G.Context
    projected: torch.Tensor
    n: int
    cam: object
    words: torch.Tensor
    offsets: torch.Tensor
    stride: int
    bg: tuple = (0.0, 0.0, 0.0)


class RasterizeFunction(torch.autograd.Function):
    @staticmethod
    def forward(fctx, xy_ab, c_o_z, rgb, frame: Frame):
        fields = G.projected_fields(frame.projected, frame.n)
        for name, t in (("xy_ab", xy_ab), ("c_o_z", c_o_z), ("rgb", rgb)):
            if t.data_ptr() != fields[name].data_ptr() or t.shape != fields[name].shape:
                raise G.TileGSError(f"rasterize: {name} must be the projected buffer's own field view")
        img, alpha, _, saved = frame.ctx.rasterize_fwd(frame.projected, frame.n, frame.cam, frame.words,
                                                      frame.offsets, frame.stride, frame.bg, save=True)
        fctx.saved = saved
        fctx.frame = frame
        return img, alpha

    @staticmethod
    def backward(fctx, g_img, g_alpha):
        fr = fctx.frame
        H, W = int(fr.cam.height), int(fr.cam.width)
        g_img = (torch.zeros((H, W, 3), dtype=torch.float32, device=fr.projected.device) if g_img is None
                 else g_img.contiguous().float())
        g_alpha = None if g_alpha is None else g_alpha.contiguous().float()
        grad = fr.ctx.rasterize_bwd(fr.projected, fr.n, fr.cam, fr.words, fr.offsets, fctx.saved, g_img, g_alpha,
                                    stride=fr.stride)
        gf = G.grad_fields(grad, fr.n)
        return gf["xy_ab"], gf["c_o_z"], gf["rgb"], None


def rasterize(xy_ab, c_o_z, rgb, frame: Frame):
    """Differentiable (rgb [H,W,3], alpha [H,W]) of the frame's stream."""
    return RasterizeFunction.apply(xy_ab, c_o_z, rgb, frame)
