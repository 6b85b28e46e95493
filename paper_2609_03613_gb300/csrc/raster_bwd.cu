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
// and recovers T_i = T_{i+1} / (1 - a_i) (a reciprocal within one rounding,
// then a product).  With G = dL/drgb, dA = dL/dalpha
// and S_i the colour behind entry i (background included), accumulated from
// the back so that it stays accurate deep in the list:
//   dL/da_i = (G.c_i) T_i - (G.S_i - dA T_N) / (1 - a_i),
//   dL/dc_i = G a_i T_i;  and, unless the clamp a_i = 0.99 is active,
//   with v_i = dL/da_i exp(-q_i):  dL/do_i = v_i,  dL/dq_i = -o_i v_i,
//   q = 1/2 (a dx^2 + 2 b dx dy + c dy^2), d = mean - pixel centre.
// Per entry nine sums over the pixels are needed (v, v dx, v dy, v dx^2,
// v dx dy, v dy^2, G a T).  A warp does not reduce them entry by entry:
// each lane stores its pixel's v and a T of every entry that contributes
// anywhere in the warp's 8 x 4 block into a per-warp shared buffer of 8
// rows, and when the buffer is full (and at the end of each batch) the rows
// are summed entry by lane group instead of pixel by lane -- four lanes a
// row, one pixel row of 8 each, from the row and the pixel positions and
// upstream gradients, which are fixed for the tile -- and the four partial
// sums meet in two shuffle steps.  That replaces a 17-shuffle butterfly per
// (entry, warp).  The row's first lane applies the per-Gaussian factors
// (o, conic) and adds the warp's sums to global memory, one vector atomic
// per gradient field: no shared accumulator, no per-batch flush, and a
// smaller footprint (five blocks an SM).
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

// A warp's buffer of per-pixel terms: SLOTS entries x 32 pixels of v and of
// a T.  Row s holds its 32 floats as eight 16-byte chunks, chunk c stored at
// c ^ (s & 7): a row written by the warp (one pixel a lane) and rows read in
// chunks by one lane each hit distinct banks.
template <int SLOTS>
struct PixelRows {
    float v[SLOTS][32];
    float w[SLOTS][32];
};

__device__ __forceinline__ int row_pos(int slot, int pixel)
{
    return ((((pixel >> 2) ^ slot) & 7) << 2) | (pixel & 3);
}

template <int TILE, int SLOTS>
struct BwdSpan {
    using SH = RasterShared<TILE, false>;
    static constexpr int BS = SH::BS, BATCH = SH::BATCH;
    static constexpr int P = 32 / SLOTS;  // lanes that share one row when it is summed
    static constexpr int R = 4 / P;       // pixel rows (of 8) each of them takes
    static_assert(SLOTS == 8 || SLOTS == 16 || SLOTS == 32, "a row is split over 1, 2 or 4 lanes");
    SH& sh;
    PixelRows<SLOTS>& rows;   // this warp's buffer
    const float4* gpix;       // this warp's upstream gradients, pixel (x, y) at y * 8 + (x ^ y)
    const float4* __restrict__ xy_ab;
    const float4* __restrict__ c_o_z;
    const float4* __restrict__ rgbv;
    float4* __restrict__ g_xy_ab;
    float4* __restrict__ g_c_o_z;
    float4* __restrict__ g_rgb;
    int cullmode, tx, ty;
    float pxc, pyc;  // this lane's pixel centre
    float bxc, byc;  // centre of the warp block's first pixel
    GradState& st;
    int32_t wend;    // span-relative: the warp has nothing to do at or beyond it

    // The first n rows of the buffer -> the nine sums of each row's entry ->
    // its gradients (row s: the entry's batch slot in lane s's `kslot`).
    __device__ __forceinline__ void drain(int n, int kslot)
    {
        const int lane = threadIdx.x & 31;
        const int s = lane % SLOTS, p = lane / SLOTS;
        const int k = __shfl_sync(kFull, kslot, s);
        float S[kTerms];
#pragma unroll
        for (int j = 0; j < kTerms; ++j) S[j] = 0.0f;
        if (s < n) {
            const float4 ga = sh.a[k];
            float dx[8];
#pragma unroll
            for (int x = 0; x < 8; ++x) dx[x] = ga.x - (bxc + (float)x);  // the lanes' own dx, bit for bit
            const float4* vr = reinterpret_cast<const float4*>(rows.v[s]);
            const float4* wr = reinterpret_cast<const float4*>(rows.w[s]);
#pragma unroll 1
            for (int r = 0; r < R; ++r) {
                const int y = p * R + r;
                const float dy = ga.y - (byc + (float)y);
                const float4 v0 = vr[(2 * y) ^ (s & 7)], v1 = vr[(2 * y + 1) ^ (s & 7)];
                const float4 w0 = wr[(2 * y) ^ (s & 7)], w1 = wr[(2 * y + 1) ^ (s & 7)];
                const float v[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
                const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
                float sv = 0.0f, svx = 0.0f, svxx = 0.0f;
#pragma unroll
                for (int x = 0; x < 8; ++x) {
                    const float vx = v[x] * dx[x];
                    sv += v[x];
                    svx += vx;
                    svxx = fmaf(vx, dx[x], svxx);
                    const float4 g = gpix[y * 8 + (x ^ y)];
                    S[6] = fmaf(w[x], g.x, S[6]);
                    S[7] = fmaf(w[x], g.y, S[7]);
                    S[8] = fmaf(w[x], g.z, S[8]);
                }
                // dy is one value along the pixel row
                S[0] += sv;
                S[1] += svx;
                S[2] = fmaf(sv, dy, S[2]);
                S[3] += svxx;
                S[4] = fmaf(svx, dy, S[4]);
                S[5] = fmaf(sv * dy, dy, S[5]);
            }
        }
#pragma unroll
        for (int o = 16; o >= SLOTS; o >>= 1)
#pragma unroll
            for (int j = 0; j < kTerms; ++j) S[j] += __shfl_xor_sync(kFull, S[j], o);
        if (p == 0 && s < n) {
            const float4 A = sh.a[k], B = sh.b[k];
            const uint32_t g = __float_as_uint(B.w);
            const float o = B.y, ca = 2.0f * A.z, cb = A.w, cc = 2.0f * B.x;
            atomicAdd(g_xy_ab + g, make_float4(-o * fmaf(ca, S[1], cb * S[2]), -o * fmaf(cb, S[1], cc * S[2]),
                                               -0.5f * o * S[3], -o * S[4]));
            atomicAdd(reinterpret_cast<float2*>(g_c_o_z + g), make_float2(-0.5f * o * S[5], S[0]));
            atomicAdd(g_rgb + g, make_float4(S[6], S[7], S[8], 0.0f));
        }
    }

    __device__ __forceinline__ void operator()(const uint64_t* src, int32_t n_entries)
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int32_t b0 = n_entries > 0 ? ((n_entries - 1) / BATCH) * BATCH : -1; b0 >= 0; b0 -= BATCH) {
            __syncthreads();  // the previous batch's staging and sums are consumed
            const int cnt = stage_batch<TILE, false>(src, b0, n_entries, sh, xy_ab, c_o_z, rgbv, cullmode, tx, ty);
            __syncthreads();
            // the entries before the warp's end that its strip mask admits,
            // walked back to front (the list is built over that prefix of
            // the batch only: stepping back over the entries past the end,
            // one shared load at a time, took 12.6 % of the backward's warp
            // time at 1080p, measured with clock counters)
            const int nk = b0 < wend ? warp_strip_list<TILE>(sh, min(cnt, wend - b0)) : 0;
            int nrow = 0, kslot = 0;
            for (int i = nk - 1; i >= 0; --i) {
                const int k = sh.list[warp][i];
                const float4 gb = sh.b[k];
                if (!st.active) st.active = __float_as_uint(gb.w) == st.last;
                float v = 0.0f, wgt = 0.0f;
                bool contrib = false;
                // exp(-q) for every q (used only when 0 <= q <= tau) and one
                // condition for the step: backward 0.585 -> 0.570 ms at 1080p
                // against branching past the exp
                const float4 ga = sh.a[k];
                const float dx = ga.x - pxc, dy = ga.y - pyc;
                const float q = fmaf(dx, fmaf(ga.z, dx, ga.w * dy), (gb.x * dy) * dy);
                const float e = spec_exp_core(-q);
                const float oe = gb.y * e;
                const float alpha = fminf(0.99f, oe);
                if (st.active && __float_as_uint(q) <= __float_as_uint(gb.z) && alpha >= 1.0f / 255.0f) {
                    // within one rounding of 1/(1 - a): an approximate
                    // reciprocal's bias would compound along the chain of
                    // recovered T_i (the IEEE-rounded intrinsic measured
                    // 0.754 ms for this kernel at 1080p, this 0.652 ms)
                    const float r = rcp_newton(1.0f - alpha);
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
                if (__ballot_sync(kFull, contrib) == 0u) continue;
                const int pos = row_pos(nrow, lane);
                rows.v[nrow][pos] = v;
                rows.w[nrow][pos] = wgt;
                if (lane == nrow) kslot = k;
                if (++nrow == SLOTS) {
                    __syncwarp();
                    drain(SLOTS, kslot);
                    __syncwarp();  // the rows are read before they are rewritten
                    nrow = 0;
                }
            }
            if (nrow > 0) {
                __syncwarp();
                drain(nrow, kslot);
                __syncwarp();
            }
        }
    }
};

// Rows buffered per warp.  Measured on the 1080p backward (1M Gaussians):
// 8 rows at five blocks an SM 0.754 ms; 16 rows (two lanes a row, 80
// registers, three blocks) 0.807 ms; 32 rows (two blocks) 0.989 ms.
constexpr int kBwdSlots = 8;

template <int TILE>
constexpr size_t bwd_dyn_smem()
{
    constexpr int NWT = TILE * TILE / 32;
    return (size_t)NWT * (sizeof(PixelRows<kBwdSlots>) + 32 * sizeof(float4));
}

template <int TILE>
__global__ void __launch_bounds__(TILE * TILE, TILE == 16 ? 5 : 1)
k_raster_bwd(const float4* __restrict__ xy_ab, const float4* __restrict__ c_o_z, const float4* __restrict__ rgbv,
             const uint64_t* __restrict__ words, const int32_t* __restrict__ off, RasterArgs a, int cullmode,
             const int32_t* __restrict__ last, const float* __restrict__ final_T,
             const int32_t* __restrict__ tile_end, const float* __restrict__ dl_drgb,
             const float* __restrict__ dl_dalpha, float4* __restrict__ g_xy_ab, float4* __restrict__ g_c_o_z,
             float4* __restrict__ g_rgb, const int32_t* __restrict__ warp_end)
{
    using SH = RasterShared<TILE, false>;
    using WB = WarpBlocks<TILE>;
    constexpr int SLOTS = kBwdSlots;
    constexpr int NWT = TILE * TILE / 32;
    __shared__ SH sh;
    extern __shared__ float4 bwd_dyn[];
    PixelRows<SLOTS>* rows = reinterpret_cast<PixelRows<SLOTS>*>(bwd_dyn);
    float4* gpix = reinterpret_cast<float4*>(rows + NWT);

    const int t = blockIdx.x;
    const int tx = t % a.tiles_x, ty = t / a.tiles_x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int lx = WB::lx(), ly = WB::ly();
    const int px = tx * TILE + lx, py = ty * TILE + ly;
    const bool inside = px < a.width && py < a.height;


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
    {
        const int x = lane & 7, y = lane >> 3;  // lanes row-major in the warp's 8 x 4 block
        gpix[warp * 32 + y * 8 + (x ^ y)] = make_float4(st.G0, st.G1, st.G2, 0.0f);
    }
    // pixel centres: integer + 0.5, exact in float32, so the drain's
    // block origin + offset reproduces each lane's own centre
    const float bxc = (float)(px - (lane & 7)) + 0.5f, byc = (float)(py - (lane >> 3)) + 0.5f;
    __syncwarp();

    // the walk ends where the forward's tile ended, or (per-warp ends saved)
    // where the last of its warps ended; each warp skips what lies past its
    // own end (every one of its pixels had stopped before)
    const int32_t s0 = off[(int64_t)t * a.stride];
    int32_t end = tile_end[t], wend = end;
    if (warp_end) {
        __shared__ int32_t s_end;
        wend = min(warp_end[(int64_t)t * NWT + warp], end);
        if (threadIdx.x == 0) s_end = s0;
        __syncthreads();
        if (lane == 0) atomicMax(&s_end, wend);
        __syncthreads();
        end = s_end;
    }
    BwdSpan<TILE, SLOTS> span{sh, rows[warp], gpix + warp * 32, xy_ab, c_o_z, rgbv, g_xy_ab, g_c_o_z, g_rgb,
                              cullmode, tx, ty, (float)px + 0.5f, (float)py + 0.5f, bxc, byc, st, wend - s0};
    walk_tile_rev(words, off, t, a.stride, end, span);
}

template <int TILE>
int launch_bwd(unsigned grid, cudaStream_t st, const ProjView& pv, const uint64_t* words, const int32_t* off,
               const RasterArgs& a, int cull, const int32_t* last, const float* final_T, const int32_t* tile_end,
               const float* dl_drgb, const float* dl_dalpha, const GradView& gv, const int32_t* warp_end)
{
    constexpr size_t dyn = bwd_dyn_smem<TILE>();
    k_raster_bwd<TILE><<<grid, TILE * TILE, dyn, st>>>(pv.xy_ab, pv.c_o_z, pv.rgb, words, off, a, cull, last,
                                                      final_T, tile_end, dl_drgb, dl_dalpha, gv.xy_ab, gv.c_o_z,
                                                      gv.rgb, warp_end);
    return GS_OK;
}

}  // namespace

// The backward's row buffers are dynamic shared memory above the 48 KB a
// kernel may take without opting in: set once per context, on its device.
int raster_bwd_prepare()
{
    GS_CUDA_TRY(cudaFuncSetAttribute(k_raster_bwd<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)bwd_dyn_smem<8>()));
    GS_CUDA_TRY(cudaFuncSetAttribute(k_raster_bwd<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)bwd_dyn_smem<16>()));
    GS_CUDA_TRY(cudaFuncSetAttribute(k_raster_bwd<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)bwd_dyn_smem<32>()));
    return GS_OK;
}

int raster_bwd(gs_ctx* ctx, const ProjView& pv, const gs_camera* cam, const uint64_t* words, const int32_t* offsets,
               int32_t stride, const float* bg, const int32_t* last, const float* final_T,
               const int32_t* tile_end, const float* dl_drgb, const float* dl_dalpha, const GradView& gv,
               cudaStream_t st, const int32_t* warp_end)
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
    int r;
    switch (tile) {
        case 8: r = launch_bwd<8>(grid, st, pv, words, offsets, a, cull, last, final_T, tile_end, dl_drgb, dl_dalpha, gv, warp_end); break;
        case 32: r = launch_bwd<32>(grid, st, pv, words, offsets, a, cull, last, final_T, tile_end, dl_drgb, dl_dalpha, gv, warp_end); break;
        default: r = launch_bwd<16>(grid, st, pv, words, offsets, a, cull, last, final_T, tile_end, dl_drgb, dl_dalpha, gv, warp_end); break;
    }
    if (r != GS_OK) return r;
    ctx->launches += 1;
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

}  // namespace gs

namespace gs {
namespace {
__global__ void k_reciprocal(const float* __restrict__ x, float* __restrict__ out, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = rcp_newton(x[i]);
}
}  // namespace
}  // namespace gs

extern "C" int gs_reciprocal(const float* x, float* out, int64_t n, void* stream)
{
    if (n < 0 || (n > 0 && (!x || !out))) return GS_ERR_INVALID_ARG;
    if (n == 0) return GS_OK;
    const int64_t blocks = (n + 255) / 256;
    gs::k_reciprocal<<<(unsigned)(blocks < 65536 ? blocks : 65536), 256, 0, (cudaStream_t)stream>>>(x, out, n);
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}
