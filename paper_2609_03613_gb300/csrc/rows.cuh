// rows.cuh -- the per-(Gaussian, tile row) span geometry of EXACT bin
// construction with the tile cull (tiles.cu, and its multi-view form in
// batch_bins.cu): which tiles of a row of the Gaussian's rect can hold a pixel
// with alpha >= 1/255, and the row record that carries the span.
#pragma once
#include "internal.cuh"

namespace gs {

// ------------------------------------------------------------------ row spans (tile cull)
struct CullArgs {
    const float4* xy_ab;
    const float4* c_o_z;
    const float4* rgb;
    int tile;
};

// Tiles [*a, *b) of row ty (inside [tx0, tx1)) whose pixel-centre boxes can
// hold a pixel with alpha >= 1/255.  A contributing pixel p has
// Q(m - p) <= tau / margin (the tile cull's bound), so it lies in that
// ellipse; the ellipse meets the row's band of pixel centres in a convex set
// whose x-projection is one interval, found from the band ends and the
// ellipse's leftmost/rightmost points.  Every box is widened (5e-3 relative +
// 0.05 px) to cover float32 rounding; margin 0 (ill-conditioned conic) keeps
// the whole row.  The per-Gaussian part (RowGeom) is computed once by the
// lane that owns the Gaussian; the widening also covers the reciprocals it
// multiplies by in place of divisions.
struct RowGeom {
    float my, hb, inv2ha, a4tp, D, dymax, ext, dyl;  // dymax < 0: keep the whole row
};

__device__ __forceinline__ RowGeom row_geom(float ha, float hb, float hc, float tau, float margin, float my)
{
    RowGeom g;
    g.my = my;
    g.hb = hb;
    g.inv2ha = 0.0f;
    g.a4tp = g.D = g.ext = g.dyl = 0.0f;
    g.dymax = -1.0f;
    if (!(margin > 0.0f)) return g;
    const float tp = tau / margin;
    const float D = 4.0f * ha * hc - hb * hb;
    if (!(D > 0.0f) || !(tp > 0.0f)) return g;
    g.D = D;
    g.a4tp = 4.0f * ha * tp;
    g.dymax = sqrtf(g.a4tp / D) * (1.0f + 5e-3f) + 0.05f;
    g.ext = sqrtf(4.0f * hc * tp / D);
    g.dyl = hb * g.ext / (2.0f * hc);  // dy of the leftmost point (dx = -ext)
    g.inv2ha = 1.0f / (2.0f * ha);
    return g;
}

__device__ __forceinline__ void row_span(float mx, const RowGeom& g, int ty, int tile, float inv_tile, int tx0,
                                         int tx1, int* a, int* b)
{
    *a = tx0;
    *b = tx1;
    if (g.dymax < 0.0f) return;
    const float y0 = (float)(ty * tile);
    float yl = g.my - (y0 + (float)tile - 0.5f), yh = g.my - (y0 + 0.5f);
    yl = yl - (0.05f + 5e-3f * fabsf(yl));
    yh = yh + (0.05f + 5e-3f * fabsf(yh));
    const float ya = fmaxf(yl, -g.dymax), yb = fminf(yh, g.dymax);
    if (ya > yb) {
        *b = *a;  // the band misses the ellipse
        return;
    }
    // the hardware's approximate square root (relative error below 2^-22):
    // the widening below is 5e-3 relative + 0.05 px
    float s_a, s_b;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(s_a) : "f"(fmaxf(0.0f, g.a4tp - g.D * ya * ya)));
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(s_b) : "f"(fmaxf(0.0f, g.a4tp - g.D * yb * yb)));
    const float La = (-g.hb * ya - s_a) * g.inv2ha, Lb = (-g.hb * yb - s_b) * g.inv2ha;
    const float Ra = (-g.hb * ya + s_a) * g.inv2ha, Rb = (-g.hb * yb + s_b) * g.inv2ha;
    float dxmin = (g.dyl >= ya && g.dyl <= yb) ? -g.ext : fminf(La, Lb);
    float dxmax = (-g.dyl >= ya && -g.dyl <= yb) ? g.ext : fmaxf(Ra, Rb);
    dxmin = dxmin - (0.05f + 5e-3f * fabsf(dxmin));
    dxmax = dxmax + (0.05f + 5e-3f * fabsf(dxmax));
    const float ft = (float)tile;
    float fa = ceilf((mx - dxmax - (ft - 0.5f)) * inv_tile), fb = floorf((mx - dxmin - 0.5f) * inv_tile) + 1.0f;
    fa = fminf(fmaxf(fa, (float)tx0), (float)tx1);
    fb = fminf(fmaxf(fb, (float)tx0), (float)tx1);
    *a = (int)fa;
    *b = fb > fa ? (int)fb : (int)fa;
}

// Row record word: tile row (12 bits) | first tile of the span (12 bits) |
// bin (8 bits); exact_bins checks tiles_x, tiles_y <= 4096 (K <= 128 < 256).
__device__ __forceinline__ uint32_t row_record(int ty, int a, uint32_t bin)
{
    return (uint32_t)ty | ((uint32_t)a << 12) | (bin << 24);
}

}  // namespace gs
