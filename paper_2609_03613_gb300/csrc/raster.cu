// raster.cu -- K6 / K16: front-to-back compositing over each tile's span of
// the tile-major stream (Sec. 3.4; supplement "Binned raster traversal after
// repair").  One CTA per tile, one thread per pixel, the span consumed in
// batches of one entry per thread staged through shared memory, and a
// block-wide vote ends the tile once every pixel has terminated.
//
// Per pixel centre (x + 0.5, y + 0.5) and entry in stream order, in this exact
// float32 order (the same as the compositing definition of the library):
//   dx = mx - px; dy = my - py;
//   q  = fmaf(dx, fmaf(a/2, dx, b*dy), ((c/2)*dy)*dy)
//   skip unless q >= 0;  e = exp(-q) (Cody-Waite/Taylor, internal.cuh)
//   alpha = min(0.99, o*e); skip if alpha < 1/255
//   Tn = T*(1 - alpha); stop before applying if Tn < 1e-4
//   C = fmaf(col, alpha*T, C); T = Tn; last = gid
//
// Two kernels, identical images:
//   baseline -- the plain kernel of the global-sort path: stages
//               (mean, conic, opacity) per batch, evaluates exp for every
//               test, reads colours from global memory when applied;
//   binned   -- the paper's default raster additions: a conservative
//               tile-level alpha cull at staging (entries that cannot reach
//               alpha >= 1/255 anywhere in the tile are dropped, order kept),
//               colour staging, and a per-entry early-out q > tau with
//               tau >= ln(255 o), past which alpha < 1/255 is certain.
#include "device.cuh"

namespace gs {

struct RasterArgs {
    int width, height, tiles_x, n_tiles, stride;
    float bg0, bg1, bg2;
};

// Per-thread compositing state.
struct PixelState {
    float T, C0, C1, C2;
    int32_t last, ntests;
    unsigned long long ops;
    bool done;
};

template <int TILE, bool BASELINE>
struct RasterShared {
    static constexpr int BS = TILE * TILE;
    static constexpr int BATCH = BS < 256 ? BS : 256;  // entries staged per batch
    static constexpr int NW = BATCH / 32;              // warps that load a batch
    float4 a[BATCH];                       // {mx, my, a/2, b}
    float4 b[BATCH];                       // {c/2, o, tau, gid bits}
    float4 c[BASELINE ? 1 : BATCH];        // colour (binned)
    uint32_t g[BASELINE ? BATCH : 1];      // gid (baseline colour lookup)
    int wc[NW];
};

// Composite n_entries stream words from src (global or shared memory) into
// every pixel of the tile, in batches.
// Returns true (uniformly) once every pixel of the tile has terminated.
// Rows of the tile a warp owns: the strip mask bit w is set when the
// entry's alpha >= 1/255 ellipse (the tile cull's bound tau / margin, widened
// as there) can reach rows [y0 + w*RPW, y0 + (w+1)*RPW) of the tile.
template <int TILE>
__device__ __forceinline__ uint32_t strip_mask(float my, float ha, float hb, float hc, float tau, float margin,
                                               float y0)
{
    constexpr int RPW = 32 / TILE > 0 ? 32 / TILE : 1;  // pixel rows per warp
    constexpr int NWT = TILE * TILE / 32;               // warps per tile
    const uint32_t all = NWT >= 32 ? 0xffffffffu : ((1u << NWT) - 1u);
    if (!(margin > 0.0f)) return all;
    const float D = 4.0f * ha * hc - hb * hb;
    const float tp = tau / margin;
    if (!(D > 0.0f) || !(tp > 0.0f)) return all;
    const float dymax = sqrtf(4.0f * ha * tp / D) * (1.0f + 5e-3f) + 0.05f;
    // pixel rows (centres y0 + row + 0.5) with |my - py| <= dymax
    const float rlo = fmaxf(ceilf(my - dymax - y0 - 0.5f), 0.0f);
    const float rhi = fminf(floorf(my + dymax - y0 - 0.5f), (float)(TILE - 1));
    if (rlo > rhi) return 0u;
    const int wlo = (int)rlo / RPW, whi = (int)rhi / RPW;
    const uint32_t upto = whi >= 31 ? 0xffffffffu : ((2u << whi) - 1u);
    return upto & ~((1u << wlo) - 1u) & all;
}

// cullmode bit 1: tile-alpha cull at staging; bit 2: per-warp strip mask.
template <int TILE, bool BASELINE, bool COUNT>
__device__ __forceinline__ bool raster_span(const uint64_t* src, int32_t n_entries,
                                            RasterShared<TILE, BASELINE>& sh, const float4* __restrict__ xy_ab,
                                            const float4* __restrict__ c_o_z, const float4* __restrict__ rgbv,
                                            int cullmode, int tx, int ty, float pxc, float pyc, PixelState& st)
{
    using SH = RasterShared<TILE, BASELINE>;
    constexpr int BS = SH::BS, BATCH = SH::BATCH, NW = SH::NW;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int32_t b0 = 0; b0 < n_entries; b0 += BATCH) {
        if (__syncthreads_count(st.done) == BS) return true;
        const int32_t idx = b0 + threadIdx.x;
        const bool valid = threadIdx.x < BATCH && idx < n_entries;
        float4 A = make_float4(0.f, 0.f, 0.f, 0.f), B = A, Cc = A;
        uint32_t g = 0;
        bool keep = valid;
        if (valid) {
            g = (uint32_t)(src[idx] & 0xffffffffull);
            const float4 p = __ldg(xy_ab + g);
            const float4 q = __ldg(c_o_z + g);
            A = make_float4(p.x, p.y, 0.5f * p.z, p.w);
            B = make_float4(0.5f * q.x, q.y, q.w, __uint_as_float(g));
            if (!BASELINE) {
                Cc = __ldg(rgbv + g);
                if (cullmode & 1)
                    keep = !tile_culled(A.x, A.y, A.z, A.w, B.x, q.w, Cc.w, (float)(tx * TILE),
                                        (float)(ty * TILE), (float)TILE);
                const uint32_t m = (cullmode & 2) ? strip_mask<TILE>(A.y, A.z, A.w, B.x, q.w, Cc.w, (float)(ty * TILE))
                                                  : 0xffffffffu;
                keep = keep && m != 0u;
                Cc.w = __uint_as_float(m);  // the colour record carries the mask
            }
        }
        int cnt, pos;
        if (BASELINE) {
            pos = threadIdx.x;
            cnt = min(BATCH, n_entries - b0);
        } else {
            // order-preserving compaction of the kept entries
            const unsigned ball = __ballot_sync(0xffffffffu, keep);
            if (lane == 0 && warp < NW) sh.wc[warp] = __popc(ball);
            __syncthreads();
            int wp = 0;
            cnt = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                const int c = sh.wc[w];
                wp += (w < warp) ? c : 0;
                cnt += c;
            }
            pos = wp + __popc(ball & ((1u << lane) - 1u));
        }
        if (keep) {
            sh.a[pos] = A;
            sh.b[pos] = B;
            if (BASELINE) sh.g[pos] = g;
            else sh.c[pos] = Cc;
        }
        __syncthreads();
        if (!st.done) {
            for (int k = 0; k < cnt; ++k) {
                if (!BASELINE && !((__float_as_uint(sh.c[k].w) >> warp) & 1u)) continue;  // warp-uniform
                const float4 ga = sh.a[k];
                const float4 gb = sh.b[k];
                if (COUNT) {
                    ++st.ntests;
                    st.ops += 8;
                }
                const float dx = ga.x - pxc, dy = ga.y - pyc;
                const float q = fmaf(dx, fmaf(ga.z, dx, ga.w * dy), (gb.x * dy) * dy);
                if (BASELINE) {
                    if (!(q >= 0.0f)) continue;
                } else {
                    // 0 <= q <= tau as one unsigned compare of the float bits
                    // (negative q and NaN compare above any positive tau)
                    if (__float_as_uint(q) > __float_as_uint(gb.z)) continue;
                }
                // the binned path reaches exp only for q <= tau (< 6), inside the
                // core's range; the baseline evaluates every q >= 0 and needs the
                // clamped form (exp(-q) for q > 87 would leave the 2^n range)
                const float e = BASELINE ? spec_exp(-q) : spec_exp_core(-q);
                const float alpha = fminf(0.99f, gb.y * e);
                if (COUNT) st.ops += 17;
                if (alpha < 1.0f / 255.0f) continue;
                const float Tn = st.T * (1.0f - alpha);
                if (COUNT) st.ops += 3;
                if (Tn < 1e-4f) {
                    st.done = true;
                    break;
                }
                if (COUNT) st.ops += 4;
                const float w = alpha * st.T;
                float4 col;
                if (BASELINE) col = __ldg(rgbv + sh.g[k]);
                else col = sh.c[k];
                st.C0 = fmaf(col.x, w, st.C0);
                st.C1 = fmaf(col.y, w, st.C1);
                st.C2 = fmaf(col.z, w, st.C2);
                st.T = Tn;
                st.last = __float_as_int(gb.w);
            }
        }
    }
    return false;
}

// LAZY (EXACT mode with the repair in the raster): the tile's segments are
// walked front to back; each segment of 2..kRasterSortCap entries is loaded
// into shared memory and sorted by (depth bits, gid) right before it is
// composited (longer ones were sorted eagerly), so segments after every
// pixel's termination are never sorted.
template <int TILE, bool BASELINE, bool COUNT, bool LAZY>
__global__ void __launch_bounds__(TILE * TILE, TILE == 16 ? 5 : 1)
k_raster(const float4* __restrict__ xy_ab, const float4* __restrict__ c_o_z, const float4* __restrict__ rgbv,
         const uint64_t* __restrict__ words, const int32_t* __restrict__ off, RasterArgs a, int cullmode,
         float* __restrict__ out_rgb, float* __restrict__ out_alpha, int32_t* __restrict__ out_last,
         int32_t* __restrict__ out_ntests, unsigned long long* __restrict__ ops_total)
{
    constexpr int BS = TILE * TILE;
    __shared__ RasterShared<TILE, BASELINE> sh;
    __shared__ uint64_t s_sort[LAZY ? kRasterSortCap : 1];
    __shared__ int32_t s_off[LAZY ? GS_MAX_K + 1 : 1];

    const int t = blockIdx.x;
    const int tx = t % a.tiles_x, ty = t / a.tiles_x;
    const int lx = threadIdx.x % TILE, ly = threadIdx.x / TILE;
    const int px = tx * TILE + lx, py = ty * TILE + ly;
    const bool inside = px < a.width && py < a.height;
    const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;

    // float32 operations of the compositing definition each pixel executes
    // (COUNT builds): 8 per visit (offsets, q, sign test), 17 more when exp is
    // evaluated (exp, o*e, clamp, threshold), 3 when alpha passes (1-alpha,
    // T*, stop test), 4 when applied (alpha*T and three colour fmas)
    PixelState st;
    st.T = 1.0f;
    st.C0 = st.C1 = st.C2 = 0.0f;
    st.last = -1;
    st.ntests = 0;
    st.ops = 0;
    st.done = !inside;

    if (!LAZY) {
        const int32_t s0 = off[(int64_t)t * a.stride], s1 = off[(int64_t)(t + 1) * a.stride];
        raster_span<TILE, BASELINE, COUNT>(words + s0, s1 - s0, sh, xy_ab, c_o_z, rgbv, cullmode, tx, ty, pxc, pyc,
                                           st);
    } else {
        // chunks of consecutive segments (at most kRasterSortCap entries) are
        // loaded into shared memory, every segment of the chunk is sorted
        // (small ones by one warp each, long ones by the whole block), and the
        // chunk is streamed in full batches across segment boundaries
        constexpr int NWB = BS / 32;
        __shared__ int s_big[GS_MAX_K];
        __shared__ int s_nbig;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int K = a.stride;
        for (int b = threadIdx.x; b <= K; b += BS) s_off[b] = off[(int64_t)t * K + b];
        __syncthreads();
        int b = 0;
        while (b < K) {
            const int32_t c0 = s_off[b];
            if (s_off[b + 1] - c0 > kRasterSortCap) {  // sorted before the raster
                if (raster_span<TILE, BASELINE, COUNT>(words + c0, s_off[b + 1] - c0, sh, xy_ab, c_o_z, rgbv,
                                                       cullmode, tx, ty, pxc, pyc, st))
                    break;
                ++b;
                continue;
            }
            int e = b + 1;
            while (e < K && s_off[e + 1] - c0 <= kRasterSortCap) ++e;
            const int32_t len = s_off[e] - c0;
            const int bfirst = b;
            b = e;
            if (len == 0) continue;
            if (__syncthreads_count(st.done) == BS) break;
            for (int i = threadIdx.x; i < len; i += BS) s_sort[i] = words[c0 + i];
            if (threadIdx.x == 0) s_nbig = 0;
            __syncthreads();
            for (int j = bfirst + warp; j < e; j += NWB) {
                const int l = s_off[j + 1] - s_off[j];
                uint64_t* seg = s_sort + (s_off[j] - c0);
                if (l < 2) continue;
                if (l <= 32) {
                    uint64_t v = lane < l ? seg[lane] : ~0ull;
                    v = warp_bitonic32(v);
                    if (lane < l) seg[lane] = v;
                } else if (l <= 256) {
                    bitonic_mem(seg, l, lane, 32, SyncWarp{});
                } else if (lane == 0) {
                    s_big[atomicAdd(&s_nbig, 1)] = j;
                }
            }
            __syncthreads();
            const int nbig = s_nbig;
            for (int k = 0; k < nbig; ++k) {
                const int j = s_big[k];
                bitonic_mem(s_sort + (s_off[j] - c0), s_off[j + 1] - s_off[j], threadIdx.x, BS, SyncBlock{});
            }
            if (raster_span<TILE, BASELINE, COUNT>(s_sort, len, sh, xy_ab, c_o_z, rgbv, cullmode, tx, ty, pxc, pyc,
                                                   st))
                break;
        }
    }
    if (inside) {
        const int64_t p = (int64_t)py * a.width + px;
        out_rgb[3 * p] = fmaf(st.T, a.bg0, st.C0);
        out_rgb[3 * p + 1] = fmaf(st.T, a.bg1, st.C1);
        out_rgb[3 * p + 2] = fmaf(st.T, a.bg2, st.C2);
        out_alpha[p] = 1.0f - st.T;
        out_last[p] = st.last;
        if (COUNT) out_ntests[p] = st.ntests;
    }
    if (COUNT) {
        // block reduction of the op count, one atomic per block
        __shared__ unsigned long long s_ops;
        if (threadIdx.x == 0) s_ops = 0;
        __syncthreads();
        atomicAdd(&s_ops, st.ops);
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(ops_total, s_ops);
    }
}

template <int TILE>
static void launch_tile(bool baseline, bool count, bool lazy, unsigned grid, cudaStream_t st, const ProjView& pv,
                        const uint64_t* words, const int32_t* off, const RasterArgs& a, int cull, float* rgb,
                        float* alpha, int32_t* last, int32_t* ntests, unsigned long long* ops)
{
    constexpr int BS = TILE * TILE;
#define GS_RASTER_LAUNCH(B, CNT, LZ)                                                                        \
    k_raster<TILE, B, CNT, LZ><<<grid, BS, 0, st>>>(pv.xy_ab, pv.c_o_z, pv.rgb, words, off, a, (B) ? 0 : cull, \
                                                   rgb, alpha, last, ntests, ops)
    if (baseline) {
        if (count) GS_RASTER_LAUNCH(true, true, false);
        else GS_RASTER_LAUNCH(true, false, false);
    } else if (lazy) {
        if (count) GS_RASTER_LAUNCH(false, true, true);
        else GS_RASTER_LAUNCH(false, false, true);
    } else {
        if (count) GS_RASTER_LAUNCH(false, true, false);
        else GS_RASTER_LAUNCH(false, false, false);
    }
#undef GS_RASTER_LAUNCH
}

int raster_fwd(gs_ctx* ctx, const ProjView& pv, const gs_camera* cam, const uint64_t* words,
               const int32_t* offsets, int32_t stride, const float* bg, float* rgb, float* alpha,
               int32_t* last, int32_t* ntests, bool baseline, cudaStream_t st)
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
    const int cull = ctx->cfg.tile_cull ? 1 : 0;
    const bool count = ntests != nullptr;
    const bool lazy = !baseline && ctx->cfg.mode == GS_MODE_BINNED_EXACT && ctx->cfg.repair_in_raster;
    // EXACT streams are culled when they are built: no second tile test at
    // staging, only the per-warp strip mask
    const int cull_here = !cull ? 0 : (ctx->cfg.mode == GS_MODE_BINNED_EXACT ? 2 : 3);
    const unsigned grid = (unsigned)a.n_tiles;
    if (grid == 0) return GS_OK;
    unsigned long long* ops = reinterpret_cast<unsigned long long*>(ctx->d_ops);
    if (count) GS_CUDA_TRY(cudaMemsetAsync(ops, 0, sizeof(unsigned long long), st));
    switch (tile) {
        case 8: launch_tile<8>(baseline, count, lazy, grid, st, pv, words, offsets, a, cull_here, rgb, alpha, last, ntests, ops); break;
        case 32: launch_tile<32>(baseline, count, lazy, grid, st, pv, words, offsets, a, cull_here, rgb, alpha, last, ntests, ops); break;
        default: launch_tile<16>(baseline, count, lazy, grid, st, pv, words, offsets, a, cull_here, rgb, alpha, last, ntests, ops); break;
    }
    ctx->launches += 1;
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

}  // namespace gs
