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
//   C = fmaf(col, alpha*T, C); T = Tn; last = stream index
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
#include "internal.cuh"

namespace gs {

struct RasterArgs {
    int width, height, tiles_x, n_tiles, stride;
    float bg0, bg1, bg2;
};

// True when no pixel centre of the tile can give alpha >= 1/255 (nor a
// q < 0 skip would change anything).  Minimum of the quadratic
// Q = ha dx^2 + hb dx dy + hc dy^2 over the tile's (slightly widened) box of
// pixel offsets; the unconstrained minimum (0) outside the box puts the
// constrained one on an edge.  margin < 1 covers float32 cancellation in the
// per-pixel q (it shrinks with the conditioning of the conic; 0 = never cull).
__device__ __forceinline__ bool tile_culled(float mx, float my, float ha, float hb, float hc, float tau,
                                            float margin, float x0, float y0, float span)
{
    if (!(margin > 0.0f)) return false;
    float xl = mx - (x0 + span - 0.5f), xh = mx - (x0 + 0.5f);
    float yl = my - (y0 + span - 0.5f), yh = my - (y0 + 0.5f);
    xl = xl - 1e-3f * (1.0f + fabsf(xl));
    xh = xh + 1e-3f * (1.0f + fabsf(xh));
    yl = yl - 1e-3f * (1.0f + fabsf(yl));
    yh = yh + 1e-3f * (1.0f + fabsf(yh));
    if (xl <= 0.0f && xh >= 0.0f && yl <= 0.0f && yh >= 0.0f) return false;
    const float ry = -hb / (2.0f * hc), rx = -hb / (2.0f * ha);
    float qmin = 3.0e38f;
    {
        const float X = xl, Yc = fminf(fmaxf(ry * X, yl), yh);
        qmin = fminf(qmin, ha * X * X + hb * X * Yc + hc * Yc * Yc);
    }
    {
        const float X = xh, Yc = fminf(fmaxf(ry * X, yl), yh);
        qmin = fminf(qmin, ha * X * X + hb * X * Yc + hc * Yc * Yc);
    }
    {
        const float Y = yl, Xc = fminf(fmaxf(rx * Y, xl), xh);
        qmin = fminf(qmin, ha * Xc * Xc + hb * Xc * Y + hc * Y * Y);
    }
    {
        const float Y = yh, Xc = fminf(fmaxf(rx * Y, xl), xh);
        qmin = fminf(qmin, ha * Xc * Xc + hb * Xc * Y + hc * Y * Y);
    }
    return qmin * margin > tau;
}

template <int TILE, bool BASELINE, bool COUNT>
__global__ void __launch_bounds__(TILE * TILE)
k_raster(const float4* __restrict__ xy_ab, const float4* __restrict__ c_o_z, const float4* __restrict__ rgbv,
         const uint64_t* __restrict__ words, const int32_t* __restrict__ off, RasterArgs a, int cull,
         float* __restrict__ out_rgb, float* __restrict__ out_alpha, int32_t* __restrict__ out_last,
         int32_t* __restrict__ out_ntests, unsigned long long* __restrict__ ops_total)
{
    constexpr int BS = TILE * TILE;
    constexpr int BATCH = BS < 256 ? BS : 256;  // entries staged per batch
    constexpr int NW = BATCH / 32;              // warps that load a batch
    __shared__ float4 s_a[BATCH];  // {mx, my, a/2, b}
    __shared__ float4 s_b[BATCH];  // {c/2, o, tau, stream index bits}
    __shared__ float4 s_c[BASELINE ? 1 : BATCH];  // colour (binned)
    __shared__ uint32_t s_g[BASELINE ? BATCH : 1];  // gid (baseline colour lookup)
    __shared__ int s_wc[NW];

    const int t = blockIdx.x;
    const int tx = t % a.tiles_x, ty = t / a.tiles_x;
    const int lx = threadIdx.x % TILE, ly = threadIdx.x / TILE;
    const int px = tx * TILE + lx, py = ty * TILE + ly;
    const bool inside = px < a.width && py < a.height;
    const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    const int32_t s0 = off[(int64_t)t * a.stride], s1 = off[(int64_t)(t + 1) * a.stride];
    float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
    int32_t last = -1, ntests = 0;
    // float32 operations of the compositing definition this pixel executed:
    // 8 per visit (offsets, q, sign test), 17 more when exp is evaluated
    // (exp, o*e, clamp, threshold), 3 when alpha passes (1-alpha, T*, stop
    // test), 4 when applied (alpha*T and three colour fmas)
    unsigned long long ops = 0;
    bool done = !inside;

    for (int32_t b0 = s0; b0 < s1; b0 += BATCH) {
        if (__syncthreads_count(done) == BS) break;
        const int32_t idx = b0 + threadIdx.x;
        const bool valid = threadIdx.x < BATCH && idx < s1;
        float4 A = make_float4(0.f, 0.f, 0.f, 0.f), B = A, Cc = A;
        uint32_t g = 0;
        bool keep = valid;
        if (valid) {
            g = (uint32_t)(words[idx] & 0xffffffffull);
            const float4 p = __ldg(xy_ab + g);
            const float4 q = __ldg(c_o_z + g);
            A = make_float4(p.x, p.y, 0.5f * p.z, p.w);
            B = make_float4(0.5f * q.x, q.y, q.w, __int_as_float(idx));
            if (!BASELINE) {
                Cc = __ldg(rgbv + g);
                if (cull)
                    keep = !tile_culled(A.x, A.y, A.z, A.w, B.x, q.w, Cc.w, (float)(tx * TILE),
                                        (float)(ty * TILE), (float)TILE);
            }
        }
        int cnt, pos;
        if (BASELINE) {
            pos = threadIdx.x;
            cnt = min(BATCH, s1 - b0);
        } else {
            // order-preserving compaction of the kept entries
            const unsigned ball = __ballot_sync(0xffffffffu, keep);
            if (lane == 0 && warp < NW) s_wc[warp] = __popc(ball);
            __syncthreads();
            int wp = 0;
            cnt = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                const int c = s_wc[w];
                wp += (w < warp) ? c : 0;
                cnt += c;
            }
            pos = wp + __popc(ball & ((1u << lane) - 1u));
        }
        if (keep) {
            s_a[pos] = A;
            s_b[pos] = B;
            if (BASELINE) s_g[pos] = g;
            else s_c[pos] = Cc;
        }
        __syncthreads();
        if (!done) {
            for (int k = 0; k < cnt; ++k) {
                const float4 ga = s_a[k];
                const float4 gb = s_b[k];
                if (COUNT) {
                    ++ntests;
                    ops += 8;
                }
                const float dx = ga.x - pxc, dy = ga.y - pyc;
                const float q = fmaf(dx, fmaf(ga.z, dx, ga.w * dy), (gb.x * dy) * dy);
                if (BASELINE) {
                    if (!(q >= 0.0f)) continue;
                } else {
                    if (!(q >= 0.0f) || q > gb.z) continue;
                }
                // the binned path reaches exp only for q <= tau (< 6), inside the
                // core's range; the baseline evaluates every q >= 0 and needs the
                // clamped form (exp(-q) for q > 87 would leave the 2^n range)
                const float e = BASELINE ? spec_exp(-q) : spec_exp_core(-q);
                const float alpha = fminf(0.99f, gb.y * e);
                if (COUNT) ops += 17;
                if (alpha < 1.0f / 255.0f) continue;
                const float Tn = T * (1.0f - alpha);
                if (COUNT) ops += 3;
                if (Tn < 1e-4f) {
                    done = true;
                    break;
                }
                if (COUNT) ops += 4;
                const float w = alpha * T;
                float4 col;
                if (BASELINE) col = __ldg(rgbv + s_g[k]);
                else col = s_c[k];
                C0 = fmaf(col.x, w, C0);
                C1 = fmaf(col.y, w, C1);
                C2 = fmaf(col.z, w, C2);
                T = Tn;
                last = __float_as_int(gb.w);
            }
        }
    }
    if (inside) {
        const int64_t p = (int64_t)py * a.width + px;
        out_rgb[3 * p] = fmaf(T, a.bg0, C0);
        out_rgb[3 * p + 1] = fmaf(T, a.bg1, C1);
        out_rgb[3 * p + 2] = fmaf(T, a.bg2, C2);
        out_alpha[p] = 1.0f - T;
        out_last[p] = last;
        if (COUNT) out_ntests[p] = ntests;
    }
    if (COUNT) {
        // block reduction of the op count, one atomic per block
        __shared__ unsigned long long s_ops;
        if (threadIdx.x == 0) s_ops = 0;
        __syncthreads();
        atomicAdd(&s_ops, ops);
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(ops_total, s_ops);
    }
}

template <int TILE>
static void launch_tile(bool baseline, bool count, unsigned grid, cudaStream_t st, const ProjView& pv,
                        const uint64_t* words, const int32_t* off, const RasterArgs& a, int cull, float* rgb,
                        float* alpha, int32_t* last, int32_t* ntests, unsigned long long* ops)
{
    constexpr int BS = TILE * TILE;
    if (baseline) {
        if (count)
            k_raster<TILE, true, true><<<grid, BS, 0, st>>>(pv.xy_ab, pv.c_o_z, pv.rgb, words, off, a, 0, rgb, alpha, last, ntests, ops);
        else
            k_raster<TILE, true, false><<<grid, BS, 0, st>>>(pv.xy_ab, pv.c_o_z, pv.rgb, words, off, a, 0, rgb, alpha, last, ntests, ops);
    } else {
        if (count)
            k_raster<TILE, false, true><<<grid, BS, 0, st>>>(pv.xy_ab, pv.c_o_z, pv.rgb, words, off, a, cull, rgb, alpha, last, ntests, ops);
        else
            k_raster<TILE, false, false><<<grid, BS, 0, st>>>(pv.xy_ab, pv.c_o_z, pv.rgb, words, off, a, cull, rgb, alpha, last, ntests, ops);
    }
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
    const unsigned grid = (unsigned)a.n_tiles;
    if (grid == 0) return GS_OK;
    unsigned long long* ops = reinterpret_cast<unsigned long long*>(ctx->d_ops);
    if (count) GS_CUDA_TRY(cudaMemsetAsync(ops, 0, sizeof(unsigned long long), st));
    switch (tile) {
        case 8: launch_tile<8>(baseline, count, grid, st, pv, words, offsets, a, cull, rgb, alpha, last, ntests, ops); break;
        case 32: launch_tile<32>(baseline, count, grid, st, pv, words, offsets, a, cull, rgb, alpha, last, ntests, ops); break;
        default: launch_tile<16>(baseline, count, grid, st, pv, words, offsets, a, cull, rgb, alpha, last, ntests, ops); break;
    }
    ctx->launches += 1;
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

}  // namespace gs
