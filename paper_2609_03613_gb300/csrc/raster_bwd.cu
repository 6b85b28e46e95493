// raster_bwd.cu -- K22: backward of the tile compositing.  The paper leaves
// the backward pass to future work and requires it to follow the forward's
// compositing order (Sec. 7); this kernel walks every tile's span in that
// order, back to front, from the position where the forward's tile ended
// (raster_common.cuh: same staging and culls; an EXACT forward that saved its
// state wrote its in-raster sorts back, so the composited prefix is already
// in order and nothing is sorted here).  One CTA per tile, one thread per
// pixel.
//
// Each pixel starts from the forward's saved final transmittance T_N and the
// id of its last applied Gaussian, becomes active when the walk reaches that
// entry, and then, entry by entry towards the front, repeats the forward's
// float32 skip test (q, exp, alpha >= 1/255; the same bits as the forward)
// and recovers T_i = T_{i+1} / (1 - a_i).  With G = dL/drgb, dA = dL/dalpha
// and S_i the colour behind entry i (background included), accumulated from
// the back so that it stays accurate deep in the list:
//   dL/da_i = (G.c_i) T_i - (G.S_i - dA T_N) / (1 - a_i),
//   dL/dc_i = G a_i T_i;  and, unless the clamp a_i = 0.99 is active,
//   with v_i = dL/da_i exp(-q_i):  dL/do_i = v_i,  dL/dq_i = -o_i v_i,
//   q = 1/2 (a dx^2 + 2 b dx dy + c dy^2), d = mean - pixel centre.
// Per entry the warp sums nine per-pixel terms (v, v dx, v dy, v dx^2,
// v dx dy, v dy^2, G a T), the per-Gaussian factors (o, conic) are applied
// once per tile and batch, and the sums go to global memory with one vector
// atomic per gradient field per entry.
#include "raster_common.cuh"

namespace gs {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kTerms = 9;

struct GradState {
    float T;           // transmittance behind the current entry (starts at the forward's final T)
    float GS;          // G.S - dA T_N, S = colour behind the current entry, background included
    float G0, G1, G2;  // dL/drgb
    uint32_t last;     // id of the last Gaussian the forward applied (0xffffffff: none)
    bool active;       // the walk has reached that entry
};

// Sums over the warp of eight per-lane values by a transposing butterfly
// (12 shuffles instead of 40): returns in every lane the warp total of value
// (lane >> 2) & 7.
__device__ __forceinline__ float warp_sum8(const float (&v)[8], int lane)
{
    const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
    float w[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const float send = h16 ? v[s] : v[4 + s];
        const float keep = h16 ? v[4 + s] : v[s];
        w[s] = keep + __shfl_xor_sync(kFull, send, 16);
    }
    float x[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const float send = h8 ? w[s] : w[2 + s];
        const float keep = h8 ? w[2 + s] : w[s];
        x[s] = keep + __shfl_xor_sync(kFull, send, 8);
    }
    float y = (h4 ? x[1] : x[0]) + __shfl_xor_sync(kFull, h4 ? x[0] : x[1], 4);
    y += __shfl_xor_sync(kFull, y, 2);
    y += __shfl_xor_sync(kFull, y, 1);
    return y;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

template <int TILE>
struct BwdSpan {
    using SH = RasterShared<TILE, false>;
    static constexpr int BS = SH::BS, BATCH = SH::BATCH;
    SH& sh;
    float* acc;  // [BATCH][kTerms] shared
    const float4* __restrict__ xy_ab;
    const float4* __restrict__ c_o_z;
    const float4* __restrict__ rgbv;
    float4* __restrict__ g_xy_ab;
    float4* __restrict__ g_c_o_z;
    float4* __restrict__ g_rgb;
    int cullmode, tx, ty;
    float pxc, pyc;
    GradState& st;

    __device__ __forceinline__ void operator()(const uint64_t* src, int32_t n_entries)
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int32_t b0 = n_entries > 0 ? ((n_entries - 1) / BATCH) * BATCH : -1; b0 >= 0; b0 -= BATCH) {
            __syncthreads();  // the previous batch's staging and sums are consumed
            const int cnt = stage_batch<TILE, false>(src, b0, n_entries, sh, xy_ab, c_o_z, rgbv, cullmode, tx, ty);
            __syncthreads();
            // the entries this warp's strip mask admits, walked back to front
            const int nk = warp_strip_list<TILE>(sh, cnt);
            for (int i = nk - 1; i >= 0; --i) {
                const int k = sh.list[warp][i];
                const float4 gb = sh.b[k];
                if (!st.active) st.active = __float_as_uint(gb.w) == st.last;
                float v = 0.0f, wgt = 0.0f, dx = 0.0f, dy = 0.0f;
                bool contrib = false;
                if (st.active) {
                    const float4 ga = sh.a[k];
                    dx = ga.x - pxc;
                    dy = ga.y - pyc;
                    const float q = fmaf(dx, fmaf(ga.z, dx, ga.w * dy), (gb.x * dy) * dy);
                    if (__float_as_uint(q) <= __float_as_uint(gb.z)) {
                        const float e = spec_exp_core(-q);
                        const float oe = gb.y * e;
                        const float alpha = fminf(0.99f, oe);
                        if (alpha >= 1.0f / 255.0f) {
                            // correctly rounded: an approximate reciprocal's bias
                            // compounds along the chain of recovered T_i
                            const float r = __frcp_rn(1.0f - alpha);
                            const float Ti = st.T * r;
                            const float4 col = sh.c[k];
                            wgt = alpha * Ti;
                            const float gc = fmaf(st.G2, col.z, fmaf(st.G1, col.y, st.G0 * col.x));
                            const float dl_da = fmaf(gc, Ti, -st.GS * r);
                            v = oe <= 0.99f ? dl_da * e : 0.0f;
                            st.GS = fmaf(gc, wgt, st.GS);
                            st.T = Ti;
                            contrib = true;
                        }
                    }
                }
                if (__ballot_sync(kFull, contrib) == 0u) continue;
                const float vx = v * dx, vy = v * dy;
                const float t8[8] = {v, vx, vy, vx * dx, vx * dy, vy * dy, wgt * st.G0, wgt * st.G1};
                const float s8 = warp_sum8(t8, lane);
                const float s9 = warp_sum(wgt * st.G2);
                if ((lane & 3) == 0) atomicAdd(acc + k * kTerms + ((lane >> 2) & 7), s8);
                else if (lane == 1) atomicAdd(acc + k * kTerms + 8, s9);
            }
            __syncthreads();
            // the tile's sums of this batch -> per-Gaussian gradients
            if ((int)threadIdx.x < cnt) {
                float s[kTerms];
                bool any = false;
#pragma unroll
                for (int j = 0; j < kTerms; ++j) {
                    s[j] = acc[threadIdx.x * kTerms + j];
                    acc[threadIdx.x * kTerms + j] = 0.0f;
                    any = any || s[j] != 0.0f;
                }
                if (any) {
                    const float4 A = sh.a[threadIdx.x], B = sh.b[threadIdx.x];
                    const uint32_t g = __float_as_uint(B.w);
                    const float o = B.y, ca = 2.0f * A.z, cb = A.w, cc = 2.0f * B.x;
                    atomicAdd(g_xy_ab + g, make_float4(-o * fmaf(ca, s[1], cb * s[2]), -o * fmaf(cb, s[1], cc * s[2]),
                                                       -0.5f * o * s[3], -o * s[4]));
                    atomicAdd(reinterpret_cast<float2*>(g_c_o_z + g), make_float2(-0.5f * o * s[5], s[0]));
                    atomicAdd(g_rgb + g, make_float4(s[6], s[7], s[8], 0.0f));
                }
            }
        }
    }
};

template <int TILE>
__global__ void __launch_bounds__(TILE * TILE, TILE == 16 ? 5 : 1)
k_raster_bwd(const float4* __restrict__ xy_ab, const float4* __restrict__ c_o_z, const float4* __restrict__ rgbv,
             const uint64_t* __restrict__ words, const int32_t* __restrict__ off, RasterArgs a, int cullmode,
             const int32_t* __restrict__ last, const float* __restrict__ final_T,
             const int32_t* __restrict__ tile_end, const float* __restrict__ dl_drgb,
             const float* __restrict__ dl_dalpha, float4* __restrict__ g_xy_ab, float4* __restrict__ g_c_o_z,
             float4* __restrict__ g_rgb)
{
    using SH = RasterShared<TILE, false>;
    __shared__ SH sh;
    __shared__ float acc[SH::BATCH * kTerms];

    const int t = blockIdx.x;
    const int tx = t % a.tiles_x, ty = t / a.tiles_x;
    const int lx = WarpBlocks<TILE>::lx(), ly = WarpBlocks<TILE>::ly();
    const int px = tx * TILE + lx, py = ty * TILE + ly;
    const bool inside = px < a.width && py < a.height;

    for (int i = threadIdx.x; i < SH::BATCH * kTerms; i += SH::BS) acc[i] = 0.0f;

    GradState st;
    st.T = 1.0f;
    st.GS = 0.0f;
    st.G0 = st.G1 = st.G2 = 0.0f;
    st.last = 0xffffffffu;
    st.active = false;
    if (inside) {
        const int64_t p = (int64_t)py * a.width + px;
        st.G0 = dl_drgb[3 * p];
        st.G1 = dl_drgb[3 * p + 1];
        st.G2 = dl_drgb[3 * p + 2];
        const float dA = dl_dalpha ? dl_dalpha[p] : 0.0f;
        st.T = final_T[p];
        st.GS = st.T * (fmaf(st.G2, a.bg2, fmaf(st.G1, a.bg1, st.G0 * a.bg0)) - dA);
        st.last = (uint32_t)last[p];
    }

    BwdSpan<TILE> span{sh, acc, xy_ab, c_o_z, rgbv, g_xy_ab, g_c_o_z, g_rgb, cullmode, tx, ty,
                       (float)px + 0.5f, (float)py + 0.5f, st};
    walk_tile_rev(words, off, t, a.stride, tile_end[t], span);
}

template <int TILE>
void launch_bwd(unsigned grid, cudaStream_t st, const ProjView& pv, const uint64_t* words, const int32_t* off,
                const RasterArgs& a, int cull, const int32_t* last, const float* final_T, const int32_t* tile_end,
                const float* dl_drgb, const float* dl_dalpha, const GradView& gv)
{
    k_raster_bwd<TILE><<<grid, TILE * TILE, 0, st>>>(pv.xy_ab, pv.c_o_z, pv.rgb, words, off, a, cull, last, final_T,
                                                    tile_end, dl_drgb, dl_dalpha, gv.xy_ab, gv.c_o_z, gv.rgb);
}

}  // namespace

int raster_bwd(gs_ctx* ctx, const ProjView& pv, const gs_camera* cam, const uint64_t* words, const int32_t* offsets,
               int32_t stride, const float* bg, const int32_t* last, const float* final_T,
               const int32_t* tile_end, const float* dl_drgb, const float* dl_dalpha, const GradView& gv,
               cudaStream_t st)
{
    const int tile = ctx->cfg.tile_size;
    RasterArgs a;
    a.width = cam->width;
    a.height = cam->height;
    a.tiles_x = (cam->width + tile - 1) / tile;
    a.n_tiles = gs_num_tiles(cam->width, cam->height, tile);
    a.stride = stride;
    a.bg0 = bg[0];
    a.bg1 = bg[1];
    a.bg2 = bg[2];
    // the staging culls are conservative, so they change no decision: EXACT
    // streams were culled when built (strip mask only), the others are culled
    // here as in the binned forward
    const int cull = !ctx->cfg.tile_cull ? 0 : (ctx->cfg.mode == GS_MODE_BINNED_EXACT ? 2 : 3);
    const unsigned grid = (unsigned)a.n_tiles;
    if (grid == 0) return GS_OK;
    switch (tile) {
        case 8: launch_bwd<8>(grid, st, pv, words, offsets, a, cull, last, final_T, tile_end, dl_drgb, dl_dalpha, gv); break;
        case 32: launch_bwd<32>(grid, st, pv, words, offsets, a, cull, last, final_T, tile_end, dl_drgb, dl_dalpha, gv); break;
        default: launch_bwd<16>(grid, st, pv, words, offsets, a, cull, last, final_T, tile_end, dl_drgb, dl_dalpha, gv); break;
    }
    ctx->launches += 1;
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

}  // namespace gs
