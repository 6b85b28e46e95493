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
#include <string.h>

#include "raster_common.cuh"

namespace gs {

// Per-thread compositing state.
struct PixelState {
    float T, C0, C1, C2;
    int32_t last, ntests;
    int32_t stop;  // stream position of the entry that stopped the pixel
    unsigned long long ops;
    bool done;
};

// The binned step at one pixel once q and exp(-q) are known.  exp(-q) is
// evaluated for every q -- its value is used only when 0 <= q <= tau, where
// it lies inside the core's range -- and the step has no early exit but the
// stop, so a warp issues the tests of two entries without diverging around
// each one (raster 0.296 -> 0.274 ms at 1080p against the form that
// branched past the exp and the colour update).  Returns true when the pixel
// stops (the entry is not applied).
template <bool COUNT>
__device__ __forceinline__ bool composite_binned(float q, float e, const float4& gb, const float4& col,
                                                 PixelState& st)
{
    // 0 <= q <= tau as one unsigned compare of the float bits
    // (negative q and NaN compare above any positive tau)
    const bool inq = __float_as_uint(q) <= __float_as_uint(gb.z);
    const float alpha = fminf(0.99f, gb.y * e);
    const bool pass = inq && alpha >= 1.0f / 255.0f;
    const float Tn = st.T * (1.0f - alpha);
    if (COUNT) {
        ++st.ntests;
        st.ops += 8 + (inq ? 17 : 0) + (pass ? 3 : 0);
    }
    if (pass && Tn < 1e-4f) {
        st.done = true;
        return true;
    }
    if (pass) {
        if (COUNT) st.ops += 4;
        const float w = alpha * st.T;
        st.C0 = fmaf(col.x, w, st.C0);
        st.C1 = fmaf(col.y, w, st.C1);
        st.C2 = fmaf(col.z, w, st.C2);
        st.T = Tn;
        st.last = __float_as_int(gb.w);
    }
    return false;
}

// One entry at one pixel, q given: the compositing definition's steps.
// Returns true when the pixel stops (the entry is not applied).
template <bool BASELINE, bool COUNT, class SH>
__device__ __forceinline__ bool composite_entry(float q, const float4& ga, const float4& gb, const SH& sh, int k,
                                                const float4* __restrict__ rgbv, PixelState& st)
{
    if constexpr (!BASELINE) {
        return composite_binned<COUNT>(q, spec_exp_core(-q), gb, sh.c[k], st);
    } else {
        if (COUNT) {
            ++st.ntests;
            st.ops += 8;
        }
        if (!(q >= 0.0f)) return false;
        // every q >= 0 reaches exp here: the clamped form (exp(-q) for
        // q > 87 would leave the 2^n range)
        const float e = spec_exp(-q);
        const float alpha = fminf(0.99f, gb.y * e);
        if (COUNT) st.ops += 17;
        if (alpha < 1.0f / 255.0f) return false;
        const float Tn = st.T * (1.0f - alpha);
        if (COUNT) st.ops += 3;
        if (Tn < 1e-4f) {
            st.done = true;
            return true;
        }
        if (COUNT) st.ops += 4;
        const float w = alpha * st.T;
        const float4 col = __ldg(rgbv + sh.g[k]);
        st.C0 = fmaf(col.x, w, st.C0);
        st.C1 = fmaf(col.y, w, st.C1);
        st.C2 = fmaf(col.z, w, st.C2);
        st.T = Tn;
        st.last = __float_as_int(gb.w);
        return false;
    }
}

// Composite the cnt staged entries of a batch into the calling thread's
// pixel (slot k is stream position base + k).  Binned: the warp composites
// only the entries its warp mask admits.
template <int TILE, bool BASELINE, bool COUNT>
__device__ __forceinline__ void composite_batch(int cnt, RasterShared<TILE, BASELINE>& sh,
                                                const float4* __restrict__ rgbv, float pxc, float pyc, PixelState& st,
                                                int32_t base)
{
    const int warp = threadIdx.x >> 5;
    int nk = cnt;
    if constexpr (!BASELINE) nk = __all_sync(0xffffffffu, st.done) ? 0 : warp_strip_list<TILE>(sh, cnt);
    if (st.done) return;
    if constexpr (BASELINE) {
        for (int k = 0; k < nk; ++k) {
            const float4 ga = sh.a[k];
            const float4 gb = sh.b[k];
            const float dx = ga.x - pxc, dy = ga.y - pyc;
            const float q = fmaf(dx, fmaf(ga.z, dx, ga.w * dy), (gb.x * dy) * dy);
            if (composite_entry<BASELINE, COUNT>(q, ga, gb, sh, k, rgbv, st)) {
                st.stop = base + k;
                break;
            }
        }
    } else {
        // two entries a round: both q and exp(-q) first (independent), then
        // the two compositing steps in stream order
        int i = 0;
        for (; i + 1 < nk; i += 2) {
            const int k0 = sh.list[warp][i], k1 = sh.list[warp][i + 1];
            const float4 ga0 = sh.a[k0], gb0 = sh.b[k0];
            const float4 ga1 = sh.a[k1], gb1 = sh.b[k1];
            const float dx0 = ga0.x - pxc, dy0 = ga0.y - pyc;
            const float dx1 = ga1.x - pxc, dy1 = ga1.y - pyc;
            const float q0 = fmaf(dx0, fmaf(ga0.z, dx0, ga0.w * dy0), (gb0.x * dy0) * dy0);
            const float q1 = fmaf(dx1, fmaf(ga1.z, dx1, ga1.w * dy1), (gb1.x * dy1) * dy1);
            const float e0 = spec_exp_core(-q0), e1 = spec_exp_core(-q1);
            if (composite_binned<COUNT>(q0, e0, gb0, sh.c[k0], st)) {
                st.stop = base + k0;
                break;
            }
            if (composite_binned<COUNT>(q1, e1, gb1, sh.c[k1], st)) {
                st.stop = base + k1;
                break;
            }
        }
        if (!st.done && i < nk) {
            const int k = sh.list[warp][i];
            const float4 ga = sh.a[k], gb = sh.b[k];
            const float dx = ga.x - pxc, dy = ga.y - pyc;
            const float q = fmaf(dx, fmaf(ga.z, dx, ga.w * dy), (gb.x * dy) * dy);
            if (composite_entry<BASELINE, COUNT>(q, ga, gb, sh, k, rgbv, st)) st.stop = base + k;
        }
    }
}

// Composite n_entries stream words from src (global or shared memory) into
// every pixel of the tile, in batches.  Returns -1 after the last entry, or,
// block-uniformly, the offset of the first batch left unprocessed once every
// pixel of the tile has terminated.
// cullmode bit 1: tile-alpha cull at staging; bit 2: per-warp strip mask.
template <int TILE, bool BASELINE, bool COUNT>
__device__ __forceinline__ int32_t raster_span(const uint64_t* src, int32_t n_entries,
                                            RasterShared<TILE, BASELINE>& sh, const float4* __restrict__ xy_ab,
                                            const float4* __restrict__ c_o_z, const float4* __restrict__ rgbv,
                                            int cullmode, int tx, int ty, float pxc, float pyc, PixelState& st,
                                            bool checked, int32_t base)
{
    using SH = RasterShared<TILE, BASELINE>;
    constexpr int BS = SH::BS, BATCH = SH::BATCH;
    for (int32_t b0 = 0; b0 < n_entries; b0 += BATCH) {
        // checked: the caller has just counted the terminated pixels (block
        // barrier included) with nothing composited since
        if (!(checked && b0 == 0) && __syncthreads_count(st.done) == BS) return b0;
        const int cnt = stage_batch<TILE, BASELINE>(src, b0, n_entries, sh, xy_ab, c_o_z, rgbv, cullmode, tx, ty);
        __syncthreads();
        composite_batch<TILE, BASELINE, COUNT>(cnt, sh, rgbv, pxc, pyc, st, base + b0);
    }
    return -1;
}

template <int TILE, bool BASELINE, bool COUNT>
struct FwdSpan {
    RasterShared<TILE, BASELINE>& sh;
    const float4* __restrict__ xy_ab;
    const float4* __restrict__ c_o_z;
    const float4* __restrict__ rgbv;
    int cullmode, tx, ty;
    float pxc, pyc;
    PixelState& st;
    __device__ __forceinline__ int32_t operator()(const uint64_t* src, int32_t n, bool checked, int32_t base)
    {
        return raster_span<TILE, BASELINE, COUNT>(src, n, sh, xy_ab, c_o_z, rgbv, cullmode, tx, ty, pxc, pyc, st,
                                                  checked, base);
    }
    __device__ __forceinline__ bool done() const { return st.done; }
    // binned: a chunk of one batch is staged slot by slot by the walk
    static constexpr bool kStageAtRank = !BASELINE;
    static constexpr int kBatch = RasterShared<TILE, BASELINE>::BATCH;
    __device__ __forceinline__ void stage_at(int slot, uint32_t g)
    {
        if constexpr (!BASELINE) {
            float4 A, B, C;
            stage_record<TILE>(g, __ldg(xy_ab + g), __ldg(c_o_z + g), __ldg(rgbv + g), cullmode, tx, ty, A, B, C);
            sh.a[slot] = A;
            sh.b[slot] = B;
            sh.c[slot] = C;
        }
    }
    __device__ __forceinline__ void composite_staged(int cnt, int32_t base)
    {
        composite_batch<TILE, BASELINE, COUNT>(cnt, sh, rgbv, pxc, pyc, st, base);
    }
};

// LAZY (EXACT mode with the repair in the raster): the tile's segments are
// walked front to back; each segment of 2..kRasterSortCap entries is loaded
// into shared memory and sorted by (depth bits, gid) right before it is
// composited (longer ones were sorted eagerly), so segments after every
// pixel's termination are never sorted.
// One tile t by the whole block (the body of both raster kernels below).
template <int TILE, bool BASELINE, bool COUNT, bool LAZY>
__device__ __forceinline__ void raster_tile(
    int t, RasterShared<TILE, BASELINE>& sh, WalkShared<LAZY>& ws, const float4* __restrict__ xy_ab,
    const float4* __restrict__ c_o_z, const float4* __restrict__ rgbv, uint64_t* words,
    const int32_t* __restrict__ off, const RasterArgs& a, int cullmode, float* __restrict__ out_rgb,
    float* __restrict__ out_alpha, int32_t* __restrict__ out_last, int32_t* __restrict__ out_ntests,
    unsigned long long* __restrict__ ops_total, float* __restrict__ out_T, int32_t* __restrict__ out_end,
    const PlanView& pl, int cap, int32_t* __restrict__ out_wend = nullptr)
{
    const int tx = t % a.tiles_x, ty = t / a.tiles_x;
    const int lx = WarpBlocks<TILE>::lx(), ly = WarpBlocks<TILE>::ly();
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
    st.stop = -1;
    st.ops = 0;
    st.done = !inside;

    const int K = a.stride;
    int kbegin = 0, kend = K;
    if (pl.bins) {
        const int B = min((int)pl.bins[t], K);
        if (pl.resume) kbegin = B;
        else kend = B;
    }
    if (pl.resume && inside) {
        const int64_t p = (int64_t)py * a.width + px;
        // the first pass's state: C in rgb, T in alpha (negative once the
        // pixel stopped), last
        const float Ts = out_alpha[p];
        st.T = fabsf(Ts);
        st.done = signbit(Ts);
        st.C0 = out_rgb[3 * p];
        st.C1 = out_rgb[3 * p + 1];
        st.C2 = out_rgb[3 * p + 2];
        st.last = out_last[p];
    }
    FwdSpan<TILE, BASELINE, COUNT> span{sh, xy_ab, c_o_z, rgbv, cullmode, tx, ty, pxc, pyc, st};
    // saving for the backward: the sorted chunks go back into the stream
    const int32_t end =
        walk_tile<TILE, LAZY>(words, off, t, K, kbegin, kend, cap, ws, span, out_end ? words : nullptr);
    if (out_end && threadIdx.x == 0) out_end[t] = end;
    if (out_wend) {
        // per warp, the stream position past the entry that stopped its last
        // pixel (the tile's end when one of its pixels never stopped): the
        // backward has nothing to do for the warp at or beyond it
        const int32_t wv = !inside ? INT32_MIN : (st.done ? st.stop + 1 : end);
        const int32_t m = __reduce_max_sync(0xffffffffu, wv);
        if ((threadIdx.x & 31) == 0)
            out_wend[(int64_t)t * (TILE * TILE / 32) + (threadIdx.x >> 5)] = m == INT32_MIN ? 0 : min(m, end);
    }
    // the pixel's index formed again after the walk: kept live across it,
    // it cost the kernel a spill at its register budget (raster 0.274 ->
    // 0.264 ms at 1080p)
    const int64_t p = (int64_t)(ty * TILE + WarpBlocks<TILE>::ly()) * a.width + (tx * TILE + WarpBlocks<TILE>::lx());
    bool unfinished = false;
    if (pl.flag && kend < K) {
        // a planned first pass: a tile with a pixel still compositing when its
        // bins ran out, and entries in later bins, is left to the completing
        // pass with its pixels' state in the outputs
        const bool all_done = __syncthreads_count(st.done) == TILE * TILE;
        unfinished = !all_done && off[(int64_t)t * K + K] > off[(int64_t)t * K + kend];
        if (unfinished && threadIdx.x == 0) {
            pl.flag[t] = 1;
            pl.flag[a.n_tiles + ty] = 1;
            pl.list[1 + atomicAdd(&pl.list[0], 1)] = t;
        }
    }
    if (COUNT && pl.needed) {
        // the bins the tile needs: through the one holding the last entry any
        // pixel visits (a pixel that never stops visits the whole span)
        __shared__ int32_t s_end;
        const int32_t s0 = off[(int64_t)t * K], s1 = off[(int64_t)t * K + K];
        if (threadIdx.x == 0) s_end = s0;
        __syncthreads();
        if (inside) atomicMax(&s_end, st.done ? st.stop + 1 : s1);
        __syncthreads();
        if (threadIdx.x == 0) {
            int need = 0;
            if (s_end > s0) {
                int lo = 0, hi = K - 1;  // the last bin starting at or before s_end - 1
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (off[(int64_t)t * K + mid] <= s_end - 1) lo = mid;
                    else hi = mid - 1;
                }
                need = lo + 1;
            }
            pl.needed[t] = need;
        }
    }
    if (inside && unfinished) {
        out_rgb[3 * p] = st.C0;
        out_rgb[3 * p + 1] = st.C1;
        out_rgb[3 * p + 2] = st.C2;
        out_alpha[p] = st.done ? -st.T : st.T;
        out_last[p] = st.last;
    } else if (inside) {
        // the image is not read again on the device: streaming stores
        __stcs(out_rgb + 3 * p, fmaf(st.T, a.bg0, st.C0));
        __stcs(out_rgb + 3 * p + 1, fmaf(st.T, a.bg1, st.C1));
        __stcs(out_rgb + 3 * p + 2, fmaf(st.T, a.bg2, st.C2));
        __stcs(out_alpha + p, 1.0f - st.T);
        __stcs(out_last + p, st.last >= 0 ? st.last - a.gid_base : st.last);
        if (out_T) out_T[p] = st.T;
        if (COUNT && out_ntests) out_ntests[p] = st.ntests;
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


template <int TILE, bool BASELINE, bool COUNT, bool LAZY>
__global__ void __launch_bounds__(TILE * TILE, TILE == 16 ? 5 : 1)
k_raster(const float4* __restrict__ xy_ab, const float4* __restrict__ c_o_z, const float4* __restrict__ rgbv,
         uint64_t* words, const int32_t* __restrict__ off, RasterArgs a, int cullmode,
         float* __restrict__ out_rgb, float* __restrict__ out_alpha, int32_t* __restrict__ out_last,
         int32_t* __restrict__ out_ntests, unsigned long long* __restrict__ ops_total, float* __restrict__ out_T,
         int32_t* __restrict__ out_end, const PlanView pl, int cap, int32_t* __restrict__ out_wend)
{
    grid_dependency_sync();
    __shared__ RasterShared<TILE, BASELINE> sh;
    __shared__ WalkShared<LAZY> ws;
    raster_tile<TILE, BASELINE, COUNT, LAZY>(blockIdx.x, sh, ws, xy_ab, c_o_z, rgbv, words, off, a, cullmode, out_rgb,
                                             out_alpha, out_last, out_ntests, ops_total, out_T, out_end, pl, cap,
                                             out_wend);
}

// The completing pass of a planned frame: persistent blocks take the listed
// tiles ({count, tiles...}) one at a time and composite each on from the bin
// where its first pass stopped, from the pixel state that pass left.
template <int TILE>
__global__ void __launch_bounds__(TILE * TILE, TILE == 16 ? 5 : 1)
k_raster_listed(const float4* __restrict__ xy_ab, const float4* __restrict__ c_o_z, const float4* __restrict__ rgbv,
                uint64_t* words, const int32_t* __restrict__ off, RasterArgs a, int cullmode,
                float* __restrict__ out_rgb, float* __restrict__ out_alpha, int32_t* __restrict__ out_last,
                float* __restrict__ out_T, int32_t* __restrict__ out_end, const uint8_t* __restrict__ plan,
                const int32_t* __restrict__ list, int cap)
{
    grid_dependency_sync();
    __shared__ RasterShared<TILE, false> sh;
    __shared__ WalkShared<true> ws;
    PlanView pl;
    pl.bins = plan;
    pl.resume = 1;
    const int32_t nl = list[0];
    for (int32_t k = blockIdx.x; k < nl; k += gridDim.x) {
        const int t = list[1 + k];
        raster_tile<TILE, false, false, true>(t, sh, ws, xy_ab, c_o_z, rgbv, words, off, a, cullmode, out_rgb,
                                              out_alpha, out_last, nullptr, nullptr, out_T, out_end, pl, cap);
        __syncthreads();  // the next tile reuses the shared memory
    }
}

// Several views in one persistent launch: blocks take (view, tile) work items
// from a counter, in view order, until all views' tiles are composited.
struct ViewRasterSet {
    struct View {
        const float4* xy_ab;
        const float4* c_o_z;
        const float4* rgbv;
        uint64_t* words;
        const int32_t* off;
        RasterArgs a;
        int cullmode, cap;
        float* rgb;
        float* alpha;
        int32_t* last;
        int32_t item0;  // first work item of the view
    } v[kMaxBatchViews];
    int nviews;
    int32_t total;
};

__device__ __forceinline__ int view_of(const ViewRasterSet& vs, int32_t item)
{
    int v = 0;
    while (v + 1 < vs.nviews && vs.v[v + 1].item0 <= item) ++v;
    return v;
}

// Longest tiles first: work items bucketed by floor(log2(span + 1)), buckets
// handed out from the longest (so the last items of the persistent launch are
// the short ones).  sched: [0..32) bucket counts, [32..64) cursors.
__global__ void k_view_buckets(const __grid_constant__ ViewRasterSet vs, int32_t* __restrict__ sched)
{
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < vs.total; i += gridDim.x * blockDim.x) {
        const ViewRasterSet::View& V = vs.v[view_of(vs, i)];
        const int64_t t = i - V.item0;
        const int32_t len = V.off[(t + 1) * V.a.stride] - V.off[t * V.a.stride];
        atomicAdd(&sched[31 - __clz(len + 1)], 1);
    }
}

__global__ void k_view_bucket_starts(int32_t* __restrict__ sched)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int32_t run = 0;
    for (int b = 31; b >= 0; --b) {
        sched[32 + b] = run;
        run += sched[b];
    }
}

__global__ void k_view_order(const __grid_constant__ ViewRasterSet vs, int32_t* __restrict__ sched,
                             int32_t* __restrict__ order)
{
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < vs.total; i += gridDim.x * blockDim.x) {
        const ViewRasterSet::View& V = vs.v[view_of(vs, i)];
        const int64_t t = i - V.item0;
        const int32_t len = V.off[(t + 1) * V.a.stride] - V.off[t * V.a.stride];
        order[atomicAdd(&sched[32 + 31 - __clz(len + 1)], 1)] = i;
    }
}

template <int TILE, bool LAZY>
__global__ void __launch_bounds__(TILE * TILE, TILE == 16 ? 5 : 1)
k_raster_views(const __grid_constant__ ViewRasterSet vs, const int32_t* __restrict__ order,
               int32_t* __restrict__ counter)
{
    __shared__ RasterShared<TILE, false> sh;
    __shared__ WalkShared<LAZY> ws;
    __shared__ int32_t s_item;
    for (;;) {
        if (threadIdx.x == 0) {
            const int32_t k = atomicAdd(counter, 1);
            s_item = k < vs.total ? order[k] : vs.total;
        }
        __syncthreads();  // also: every thread is done with the previous tile's shared memory
        const int32_t item = s_item;
        __syncthreads();
        if (item >= vs.total) break;
        const ViewRasterSet::View& V = vs.v[view_of(vs, item)];
        raster_tile<TILE, false, false, LAZY>(item - V.item0, sh, ws, V.xy_ab, V.c_o_z, V.rgbv, V.words, V.off, V.a,
                                              V.cullmode, V.rgb, V.alpha, V.last, nullptr, nullptr, nullptr, nullptr,
                                              PlanView(), V.cap);
    }
}

template <int TILE>
static cudaError_t launch_tile(const gs_ctx* ctx, bool baseline, bool count, bool lazy, unsigned grid,
                               cudaStream_t st, const ProjView& pv, uint64_t* words, const int32_t* off,
                               const RasterArgs& a, int cull, float* rgb, float* alpha, int32_t* last,
                               int32_t* ntests, unsigned long long* ops, float* final_T, int32_t* tile_end,
                               const PlanView& pl, int cap, int32_t* warp_end)
{
    constexpr int BS = TILE * TILE;
#define GS_RASTER_LAUNCH(B, CNT, LZ)                                                                          \
    return launch_k(ctx, k_raster<TILE, B, CNT, LZ>, grid, BS, 0, st, pv.xy_ab, pv.c_o_z, pv.rgb, words, off, a, \
                    (B) ? 0 : cull, rgb, alpha, last, ntests, ops, final_T, tile_end, pl, cap, warp_end)
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

int raster_fwd(gs_ctx* ctx, const ProjView& pv, const gs_camera* cam, uint64_t* words,
               const int32_t* offsets, int32_t stride, const float* bg, float* rgb, float* alpha,
               int32_t* last, int32_t* ntests, bool baseline, cudaStream_t st, float* final_T, int32_t* tile_end,
               const PlanView& pl, int32_t* warp_end)
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
    const bool count = ntests != nullptr || pl.needed != nullptr;
    const bool lazy = !baseline && ctx->cfg.mode == GS_MODE_BINNED_EXACT && ctx->cfg.repair_in_raster;
    // EXACT streams are culled when they are built: no second tile test at
    // staging, only the per-warp strip mask
    const int cull_here = !cull ? 0 : (ctx->cfg.mode == GS_MODE_BINNED_EXACT ? 2 : 3);
    const int cap = chunk_cap(ctx->cfg);
    const unsigned grid = (unsigned)a.n_tiles;
    if (grid == 0) return GS_OK;
    unsigned long long* ops = reinterpret_cast<unsigned long long*>(ctx->d_ops);
    if (count) GS_CUDA_TRY(cudaMemsetAsync(ops, 0, sizeof(unsigned long long), st));
    cudaError_t e;
    switch (tile) {
        case 8: e = launch_tile<8>(ctx, baseline, count, lazy, grid, st, pv, words, offsets, a, cull_here, rgb, alpha, last, ntests, ops, final_T, tile_end, pl, cap, warp_end); break;
        case 32: e = launch_tile<32>(ctx, baseline, count, lazy, grid, st, pv, words, offsets, a, cull_here, rgb, alpha, last, ntests, ops, final_T, tile_end, pl, cap, warp_end); break;
        default: e = launch_tile<16>(ctx, baseline, count, lazy, grid, st, pv, words, offsets, a, cull_here, rgb, alpha, last, ntests, ops, final_T, tile_end, pl, cap, warp_end); break;
    }
    GS_CUDA_TRY(e);
    ctx->launches += 1;
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

int raster_listed(gs_ctx* ctx, const ProjView& pv, const gs_camera* cam, uint64_t* words, const int32_t* offsets,
                  int32_t stride, const float* bg, float* rgb, float* alpha, int32_t* last, const uint8_t* plan,
                  const int32_t* list, cudaStream_t st, float* final_T, int32_t* tile_end)
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
    if (a.n_tiles == 0) return GS_OK;
    // EXACT streams are culled when built: the strip mask only
    const int cull = ctx->cfg.tile_cull ? 2 : 0;
    const int cap = chunk_cap(ctx->cfg);
    switch (tile) {
        case 8: GS_CUDA_TRY(launch_k(ctx, k_raster_listed<8>, (unsigned)ctx->num_sms, 64, 0, st, pv.xy_ab, pv.c_o_z, pv.rgb, words, offsets, a, cull, rgb, alpha, last, final_T, tile_end, plan, list, cap)); break;
        case 32: GS_CUDA_TRY(launch_k(ctx, k_raster_listed<32>, (unsigned)ctx->num_sms, 1024, 0, st, pv.xy_ab, pv.c_o_z, pv.rgb, words, offsets, a, cull, rgb, alpha, last, final_T, tile_end, plan, list, cap)); break;
        default: GS_CUDA_TRY(launch_k(ctx, k_raster_listed<16>, (unsigned)ctx->num_sms * 5, 256, 0, st, pv.xy_ab, pv.c_o_z, pv.rgb, words, offsets, a, cull, rgb, alpha, last, final_T, tile_end, plan, list, cap)); break;
    }
    ctx->launches += 1;
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

int raster_views(gs_ctx* ctx, const RasterView* views, int nv, int32_t* sched, int32_t* order, cudaStream_t st)
{
    if (nv < 1 || nv > kMaxBatchViews) return GS_ERR_INVALID_ARG;
    ViewRasterSet vs;
    memset(&vs, 0, sizeof(vs));
    int32_t total = 0;
    for (int i = 0; i < nv; ++i) {
        const RasterView& r = views[i];
        ViewRasterSet::View& V = vs.v[i];
        const int tile = 16;
        V.xy_ab = r.pv.xy_ab;
        V.c_o_z = r.pv.c_o_z;
        V.rgbv = r.pv.rgb;
        V.words = r.words;
        V.off = r.offsets;
        V.a.width = r.cam.width;
        V.a.height = r.cam.height;
        V.a.tiles_x = (r.cam.width + tile - 1) / tile;
        V.a.n_tiles = gs_num_tiles(r.cam.width, r.cam.height, tile);
        V.a.stride = r.stride;
        V.a.bg0 = r.bg[0];
        V.a.bg1 = r.bg[1];
        V.a.bg2 = r.bg[2];
        V.cullmode = r.cull ? 2 : 0;
        V.cap = r.cap;
        V.rgb = r.rgb;
        V.alpha = r.alpha;
        V.last = r.last;
        V.a.gid_base = r.gid_base;
        V.item0 = total;
        total += V.a.n_tiles;
    }
    vs.nviews = nv;
    vs.total = total;
    if (total == 0) return GS_OK;
    // sched: [0..32) bucket counts, [32..64) bucket cursors, [64] work counter
    GS_CUDA_TRY(cudaMemsetAsync(sched, 0, 65 * sizeof(int32_t), st));
    const unsigned gi = (unsigned)((total + 255) / 256 < ctx->num_sms * 4 ? (total + 255) / 256 : ctx->num_sms * 4);
    k_view_buckets<<<gi, 256, 0, st>>>(vs, sched);
    k_view_bucket_starts<<<1, 32, 0, st>>>(sched);
    k_view_order<<<gi, 256, 0, st>>>(vs, sched, order);
    const unsigned grid = (unsigned)(ctx->num_sms * 5 < total ? ctx->num_sms * 5 : total);
    k_raster_views<16, true><<<grid, 256, 0, st>>>(vs, order, sched + 64);
    ctx->launches += 4;
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

}  // namespace gs
