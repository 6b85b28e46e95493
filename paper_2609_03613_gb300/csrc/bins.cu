// bins.cu -- the TileGS ordering path:
//   K7  robust depth range      (supplement, "Robust depth-range estimation")
//   K8  depth-to-bin maps       (supplement, the log-depth-bin formula; and the
//                                monotone split map of EXACT mode)
//   K9-K11 count / scan / scatter into the tile-bin-major stream
//                               (Sec. 3.3; supplement "Tile-local bin construction")
//   K13 repair selection        (Sec. 3.5 rule table; supplement "Selective
//                                repair selection and local exact sorting")
//   K14 segment sorts by the baseline key (depth bits, gid)
#include "depth_range.cuh"

namespace gs {

// ------------------------------------------------------------------ depth range: depth_range.cuh

// Sample j of the emission order -> gid, from the materialised entries ...
struct GidFromIsect {
    static constexpr bool kKeys = false;
    const uint32_t* gid;
    __device__ uint32_t operator()(int64_t, int64_t j) const { return gid[j]; }
};
// Sample i of S' = min(S, M) is entry j = floor(i M / S') of the emission
// order.  Gaussian g owns entries [goff[g], goff[g+1]), so its samples are the
// i with goff[g] <= floor(i M / S') < goff[g+1], i.e.
// i in [ceil(goff[g] S' / M), ceil(goff[g+1] S' / M)) -- exact in integers.
// One thread per Gaussian (coalesced reads of goff; empty Gaussians own none),
// which writes its samples' key (depth or near-shifted key, float bits).
__global__ void __launch_bounds__(256)
k_sample_keys(const int32_t* __restrict__ goff, int64_t n, const int64_t* __restrict__ m_dev, int64_t m_cap, int S,
              uint32_t* __restrict__ out, FrameZero fz, const float4* __restrict__ c_o_z,
              const float* __restrict__ scales, DrArgs dr)
{
    grid_dependency_sync();
    frame_zero(fz);  // the frame's bin-stage counts, later scan flags, repair counter
    const int64_t M = live_count(m_dev, m_cap);
    if (M <= 0) return;
    const uint64_t ns = (uint64_t)(M < (int64_t)S ? M : (int64_t)S);
    const uint64_t uM = (uint64_t)M;
    // ceil(x / M) by a multiply with inv = floor((2^64 - 1) / M): for
    // x < 2^63 the product's high word is floor(x / M) or one less, and one
    // comparison corrects it (x = goff * ns + M - 1 < 2^31 * 2^13 + 2^31)
    const uint64_t inv = ~0ull / uM;
    auto ceil_div = [&](uint64_t a) {
        const uint64_t x = a * ns + uM - 1;
        uint64_t q = __umul64hi(x, inv);
        if ((q + 1) * uM <= x) ++q;
        return q;
    };
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = goff[g], b = goff[g + 1];
        if (b <= a) continue;
        const uint64_t i0 = ceil_div((uint64_t)a), i1 = ceil_div((uint64_t)b);
        if (i0 >= i1 || i0 >= ns) continue;
        // the samples' key, gathered here by many blocks rather than by the
        // one block that selects
        const uint32_t key = __float_as_uint(sample_key(c_o_z, scales, (uint32_t)g, dr));
        for (uint64_t i = i0; i < i1 && i < ns; ++i) out[i] = key;
    }
}

template <class GidOf>
__global__ void __launch_bounds__(kDrThreads)
k_depth_range(const float4* __restrict__ c_o_z, const float* __restrict__ scales, GidOf gid_of,
              const int64_t* __restrict__ m_dev, int64_t m_cap, DrArgs a, BinParams* bp)
{
    grid_dependency_sync();
    depth_range_block(c_o_z, scales, gid_of, live_count(m_dev, m_cap), a, bp);
}

__global__ void k_bin_params_from(const float* __restrict__ zrange, int K, float eps, BinParams* bp)
{
    write_bin_params(bp, zrange[0], zrange[1], K, eps, -1);
}

int depth_range(gs_ctx* ctx, const ProjView& pv, const float* scales, const IsectView& is, int64_t m_cap,
                const int64_t* m_dev, const gs_camera* cam, cudaStream_t st)
{
    const gs_config& c = ctx->cfg;
    DrArgs a;
    a.near_plane = cam->near_plane;
    a.far_plane = cam->far_plane;
    a.S = c.sample_count;
    a.near_shift = c.near_shift;
    a.near_alpha = c.near_alpha;
    a.near_gamma = c.near_gamma;
    a.p_lo = c.p_lo;
    a.p_hi = c.p_hi;
    a.pad = c.pad;
    a.eps = c.eps;
    a.K = c.K;
    GS_CUDA_TRY(launch_k(ctx, k_depth_range<GidFromIsect>, 1, kDrThreads, 0, st, pv.c_o_z, scales, GidFromIsect{is.gid}, m_dev, m_cap, a, ctx->d_bp));
    ctx->launches += 1;
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

// The same launch with the bin-parameter record placed by the caller (used by
// the entry point that allocates nothing).
int launch_depth_range_into(const gs_config& c, const ProjView& pv, const float* scales, const IsectView& is,
                            int64_t m_cap, const int64_t* m_dev, const gs_camera* cam, BinParams* bp,
                            cudaStream_t st)
{
    DrArgs a;
    a.near_plane = cam->near_plane;
    a.far_plane = cam->far_plane;
    a.S = c.sample_count;
    a.near_shift = c.near_shift;
    a.near_alpha = c.near_alpha;
    a.near_gamma = c.near_gamma;
    a.p_lo = c.p_lo;
    a.p_hi = c.p_hi;
    a.pad = c.pad;
    a.eps = c.eps;
    a.K = c.K;
    k_depth_range<<<1, kDrThreads, 0, st>>>(pv.c_o_z, scales, GidFromIsect{is.gid}, m_dev, m_cap, a, bp);
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

int samples_reserve(gs_ctx* ctx)
{
    void* p = ctx->d_samples;
    int r = ensure(&p, &ctx->samples_cap, (size_t)kDrMaxS * 4);
    ctx->d_samples = (uint32_t*)p;
    return r;
}

int depth_range_goff(gs_ctx* ctx, const ProjView& pv, const float* scales, int64_t n, int64_t m_cap,
                     const int64_t* m_dev, const gs_camera* cam, cudaStream_t st)
{
    const gs_config& c = ctx->cfg;
    DrArgs a;
    a.near_plane = cam->near_plane;
    a.far_plane = cam->far_plane;
    a.S = c.sample_count;
    a.near_shift = c.near_shift;
    a.near_alpha = c.near_alpha;
    a.near_gamma = c.near_gamma;
    a.p_lo = c.p_lo;
    a.p_hi = c.p_hi;
    a.pad = c.pad;
    a.eps = c.eps;
    a.K = c.K;
    int r = samples_reserve(ctx);
    if (r != GS_OK) return r;
    if (n > 0) {
        FrameZero late;
        for (int k = 0; k < 3; ++k) {
            late.p[k] = ctx->late_p[k];
            late.n[k] = ctx->late_n[k];
            ctx->late_p[k] = nullptr;
        }
        GS_CUDA_TRY(launch_k(ctx, k_sample_keys, (unsigned)ctx->num_sms * 4, 256, 0, st, ctx->d_goff, n, m_dev,
                             m_cap, a.S, ctx->d_samples, late, pv.c_o_z, scales, a));
    }
    GS_CUDA_TRY(launch_k(ctx, k_depth_range<KeyFromSamples>, 1, kDrThreads, 0, st, pv.c_o_z, scales,
                         KeyFromSamples{ctx->d_samples}, m_dev, m_cap, a, ctx->d_bp));
    ctx->launches += 2;
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

int set_zrange(gs_ctx* ctx, const float* zrange, cudaStream_t st)
{
    k_bin_params_from<<<1, 128, 0, st>>>(zrange, ctx->cfg.K, ctx->cfg.eps, ctx->d_bp);
    ctx->launches += 1;
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

// The paper's clamped log map.
__device__ __forceinline__ int bin_log(float z, float lmin, float lmax, int K, float eps)
{
    float u = (spec_log(fmaxf(z, eps)) - lmin) / (lmax - lmin);
    u = fminf(fmaxf(u, 0.0f), 1.0f - 1e-6f);
    int b = (int)floorf((float)K * u);
    b = b < 0 ? 0 : b;
    b = b > K - 1 ? K - 1 : b;
    return b;
}

struct BinArgs {
    int K;
    int map_log;  // 1: paper log map on the near-shifted key
    int near_shift;
    float near_alpha, near_gamma, eps;
};

__global__ void __launch_bounds__(256)
k_bin_count(IsectView is, const float4* __restrict__ c_o_z, const float* __restrict__ scales,
            const int64_t* __restrict__ m_dev, int64_t m_cap, const BinParams* __restrict__ bp, BinArgs a,
            int32_t* __restrict__ count, uint8_t* __restrict__ bin_of)
{
    __shared__ float s_split[GS_MAX_K];
    for (int k = threadIdx.x; k < a.K - 1; k += blockDim.x) s_split[k] = bp->splits[k];
    __syncthreads();
    const float lmin = bp->lmin, lmax = bp->lmax;
    const int64_t M = live_count(m_dev, m_cap);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < M; e += stride) {
        const uint32_t t = is.tile[e];
        int b;
        if (a.map_log) {
            const uint32_t g = is.gid[e];
            float z = __uint_as_float(is.zbits[e]);
            if (a.near_shift) z = zkey_of(z, scales, g, a.near_alpha, a.near_gamma);
            b = bin_log(z, lmin, lmax, a.K, a.eps);
        } else {
            b = bin_split(__uint_as_float(is.zbits[e]), s_split, a.K);
        }
        bin_of[e] = (uint8_t)b;
        atomicAdd(&count[(int64_t)t * a.K + b], 1);
    }
}

// Fill each (tile, bin) segment from its end: the counter returns to zero.
__global__ void __launch_bounds__(256)
k_bin_scatter(IsectView is, const int64_t* __restrict__ m_dev, int64_t m_cap, int K,
              const uint8_t* __restrict__ bin_of, const int32_t* __restrict__ offsets,
              int32_t* __restrict__ count, uint64_t* __restrict__ words)
{
    const int64_t M = live_count(m_dev, m_cap);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < M; e += stride) {
        const int64_t seg = (int64_t)is.tile[e] * K + bin_of[e];
        const int32_t p = offsets[seg] + atomicSub(&count[seg], 1) - 1;
        words[p] = ((uint64_t)is.zbits[e] << 32) | is.gid[e];
    }
}

constexpr int32_t kTailCap = 1 << 16;
// long-segment list capacity: every segment may be long on deep frames
static int32_t tail_capacity(int64_t nseg) { return nseg > kTailCap ? (int32_t)nseg : kTailCap; }

int bins_reserve(gs_ctx* ctx, int64_t m_cap, int64_t nseg)
{
    int r;
    void* p = ctx->d_count;
    if ((r = ensure(&p, &ctx->count_cap, (size_t)(nseg + 1) * 4)) != GS_OK) return r;
    ctx->d_count = (int32_t*)p;
    p = ctx->d_bin;
    if ((r = ensure(&p, &ctx->bin_cap, (size_t)(m_cap > 0 ? m_cap : 1))) != GS_OK) return r;
    ctx->d_bin = (uint8_t*)p;
    p = ctx->d_sel;
    if ((r = ensure(&p, &ctx->sel_cap, align256((size_t)nseg) + (size_t)(nseg + 1) * 8 + 256)) != GS_OK) return r;
    ctx->d_sel = (uint8_t*)p;
    p = ctx->d_tail;
    if ((r = ensure(&p, &ctx->tail_cap, (size_t)(tail_capacity(nseg) + 1) * 4)) != GS_OK) return r;
    ctx->d_tail = (int32_t*)p;
    return GS_OK;
}

int bin_build(gs_ctx* ctx, const ProjView& pv, const float* scales, const IsectView& is, int64_t m_cap,
              const int64_t* m_dev, int32_t n_tiles, uint64_t* stream_words, int32_t* offsets,
              cudaStream_t st)
{
    const gs_config& c = ctx->cfg;
    const int64_t nseg = (int64_t)n_tiles * c.K;
    int r;
    if ((r = bins_reserve(ctx, m_cap, nseg)) != GS_OK) return r;
    GS_CUDA_TRY(cudaMemsetAsync(ctx->d_count, 0, (size_t)nseg * 4, st));
    BinArgs a;
    a.K = c.K;
    a.map_log = (c.mode == GS_MODE_BINNED_EXACT) ? 0 : 1;
    a.near_shift = c.near_shift;
    a.near_alpha = c.near_alpha;
    a.near_gamma = c.near_gamma;
    a.eps = c.eps;
    const unsigned grid = (unsigned)ctx->num_sms * 8;
    k_bin_count<<<grid, 256, 0, st>>>(is, pv.c_o_z, scales, m_dev, m_cap, ctx->d_bp, a, ctx->d_count, ctx->d_bin);
    ctx->launches += 1;
    GS_CUDA_TRY(cudaGetLastError());
    if ((r = exclusive_scan_i32(ctx, ctx->d_count, nseg, offsets, nullptr, st)) != GS_OK) return r;
    k_bin_scatter<<<grid, 256, 0, st>>>(is, m_dev, m_cap, c.K, ctx->d_bin, offsets, ctx->d_count, stream_words);
    ctx->launches += 1;
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

// ------------------------------------------------------------------ repair selection
// The rules of the paper's selection table in exact integer form.
__device__ __forceinline__ int keep_len(int64_t l, int64_t ltile, int b)
{
    if (l <= 1) return 0;
    bool keep = false;
    if (l >= 320) keep = true;
    if (l > 512) keep = true;
    if (100 * l >= 45 * ltile) keep = true;
    if (l >= 129 && l <= 256 && 100 * l >= 10 * ltile) keep = true;
    if (b < 2 && l >= 16) keep = true;
    return keep ? (int)l : 0;
}

__global__ void k_keep_lengths(const int32_t* __restrict__ off, int64_t nseg, int K, int32_t* __restrict__ klen)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nseg; q += stride) {
        const int64_t t = q / K;
        const int b = (int)(q - t * K);
        const int64_t l = (int64_t)off[q + 1] - off[q];
        const int64_t ltile = (int64_t)off[(t + 1) * K] - off[t * K];
        klen[q] = keep_len(l, ltile, b);
    }
}

// Budget B = floor(frac * M).  Segments whose inclusive prefix of kept lengths
// stays within B are selected (the greedy accepts all of them); the first one
// that overflows and everything after it go to the one-block greedy below.
__global__ void k_select_prefix(const int32_t* __restrict__ klen, const int32_t* __restrict__ pre, int64_t nseg,
                                const int64_t* __restrict__ m_dev, double frac, uint8_t* __restrict__ sel)
{
    const int64_t B = (int64_t)floor(frac * (double)(*m_dev));
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nseg; q += stride)
        sel[q] = (klen[q] > 0 && (int64_t)pre[q] + klen[q] <= B) ? 1 : 0;
}

// Exact sequential greedy from the first overflow: keep if used + l <= B.
// Chunks of 1024 segments; inside a chunk, candidates longer than the room
// left are rejected at once (used only grows), the rest accepted up to the
// first that overflows, which is rejected; repeat.
__global__ void __launch_bounds__(1024)
k_select_greedy(const int32_t* __restrict__ klen, const int32_t* __restrict__ pre, int64_t nseg,
                const int64_t* __restrict__ m_dev, double frac, uint8_t* __restrict__ sel)
{
    __shared__ int64_t s_warp[32];
    __shared__ int64_t s_used;
    __shared__ int64_t s_first;
    const int64_t B = (int64_t)floor(frac * (double)(*m_dev));
    // first q whose inclusive prefix exceeds B (pre is non-decreasing)
    if (threadIdx.x == 0) {
        int64_t lo = 0, hi = nseg;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)pre[mid] + klen[mid] > B) hi = mid;
            else lo = mid + 1;
        }
        s_first = lo;
        s_used = lo < nseg ? (int64_t)pre[lo] : 0;
    }
    __syncthreads();
    const int64_t q0 = s_first;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t c0 = q0; c0 < nseg; c0 += blockDim.x) {
        const int64_t q = c0 + threadIdx.x;
        int64_t len = q < nseg ? klen[q] : 0;
        bool undecided = len > 0;
        bool accept = false;
        while (true) {
            const int64_t room = B - s_used;
            if (undecided && len > room) undecided = false;  // can never fit
            const int64_t v = undecided ? len : 0;
            // inclusive block prefix of v
            int64_t incl = v;
            for (int d = 1; d < 32; d <<= 1) {
                const int64_t t = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += t;
            }
            if (lane == 31) s_warp[warp] = incl;
            __syncthreads();
            int64_t wp = 0;
            for (int w = 0; w < warp; ++w) wp += s_warp[w];
            incl += wp;
            // candidates whose prefix overflows: the earliest is rejected
            const bool over = undecided && incl > room;
            const unsigned ball = __ballot_sync(0xffffffffu, over);
            __shared__ int s_firstover;
            if (threadIdx.x == 0) s_firstover = 1 << 30;
            __syncthreads();
            if (ball && lane == __ffs(ball) - 1) atomicMin(&s_firstover, (int)threadIdx.x);
            __syncthreads();
            const int fo = s_firstover;
            if (fo == (1 << 30)) {
                if (undecided) accept = true;
                __syncthreads();
                if (threadIdx.x == blockDim.x - 1) s_used += incl;
                __syncthreads();
                break;
            }
            if (undecided && (int)threadIdx.x < fo) {
                accept = true;
                undecided = false;
            }
            if ((int)threadIdx.x == fo) undecided = false;
            // used grows by the accepted prefix before fo
            __syncthreads();
            if ((int)threadIdx.x == fo) s_used += incl - v;
            __syncthreads();
        }
        if (q < nseg) sel[q] = accept ? 1 : 0;
        __syncthreads();
    }
}

constexpr int kRpThreads = 256;
constexpr int kRpWarps = kRpThreads / 32;
constexpr int kRpWarpCap = 512;                     // per-warp shared sort
constexpr int kRpCtaCap = kRpWarps * kRpWarpCap;    // whole-CTA shared sort (4096)

// One block per tile: sort the tile's selected segments (sel == nullptr:
// every segment with length >= 2).  Longer than kRpCtaCap: queued as a tail.
__global__ void __launch_bounds__(kRpThreads)
k_repair_tiles(const int32_t* __restrict__ off, int K, const uint8_t* __restrict__ sel, uint64_t* __restrict__ words,
               int32_t* __restrict__ tail, int32_t tail_cap, int* err, int min_len)
{
    __shared__ uint64_t s_buf[kRpCtaCap];
    __shared__ int32_t s_off[GS_MAX_K + 1];
    __shared__ int s_big[GS_MAX_K];
    __shared__ int s_nbig;
    const int64_t t = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int b = threadIdx.x; b <= K; b += blockDim.x) s_off[b] = off[t * K + b];
    if (threadIdx.x == 0) s_nbig = 0;
    __syncthreads();
    if (s_off[K] - s_off[0] < min_len) return;
    uint64_t* wbuf = s_buf + warp * kRpWarpCap;
    for (int b = warp; b < K; b += kRpWarps) {
        const int l = s_off[b + 1] - s_off[b];
        if (l < 2 || l < min_len) continue;
        if (sel && !sel[t * K + b]) continue;
        uint64_t* seg = words + s_off[b];
        if (l <= 32) {
            uint64_t v = lane < l ? seg[lane] : ~0ull;
            v = warp_bitonic32(v);
            if (lane < l) seg[lane] = v;
        } else if (l <= kRpWarpCap) {
            for (int i = lane; i < l; i += 32) wbuf[i] = seg[i];
            __syncwarp();
            bitonic_mem(wbuf, l, lane, 32, SyncWarp{});
            for (int i = lane; i < l; i += 32) seg[i] = wbuf[i];
            __syncwarp();
        } else if (lane == 0) {
            s_big[atomicAdd(&s_nbig, 1)] = b;
        }
    }
    __syncthreads();
    const int nbig = s_nbig;
    for (int k = 0; k < nbig; ++k) {
        const int b = s_big[k];
        const int l = s_off[b + 1] - s_off[b];
        uint64_t* seg = words + s_off[b];
        if (l <= kRpCtaCap) {
            for (int i = threadIdx.x; i < l; i += blockDim.x) s_buf[i] = seg[i];
            __syncthreads();
            bitonic_mem(s_buf, l, threadIdx.x, blockDim.x, SyncBlock{});
            for (int i = threadIdx.x; i < l; i += blockDim.x) seg[i] = s_buf[i];
            __syncthreads();
        } else if (threadIdx.x == 0) {
            const int slot = atomicAdd(&tail[0], 1);
            if (slot < tail_cap) tail[1 + slot] = (int32_t)(t * K + b);
            else raise_error(err, GS_ERR_CAPACITY);
        }
    }
}

// One block per queued long segment: bitonic sort in global memory.
__global__ void __launch_bounds__(1024)
k_repair_tail(const int32_t* __restrict__ off, const int32_t* __restrict__ tail, int32_t tail_cap,
              uint64_t* __restrict__ words)
{
    const int ntail = min(tail[0], tail_cap);
    for (int k = blockIdx.x; k < ntail; k += gridDim.x) {
        const int32_t q = tail[1 + k];
        const int l = off[q + 1] - off[q];
        bitonic_mem(words + off[q], l, threadIdx.x, blockDim.x, SyncBlock{});
        __syncthreads();
    }
}

// EXACT with the repair in the raster: only segments of at least min_len
// entries are sorted here.  A flat pass over the offsets lists them (one
// thread per segment; most frames have none), then one block per listed
// segment sorts it -- in shared memory when it fits, else in place.
__global__ void k_list_long(const int32_t* __restrict__ off, int64_t nseg, int min_len, int32_t* __restrict__ list,
                            int32_t cap, int* err, const ScatterPass sp, int K, const int32_t* __restrict__ flagged)
{
    grid_dependency_sync();
    if (sp.pass == 2 && flagged[0] == 0) return;  // no tile to complete
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nseg; q += (int64_t)gridDim.x * blockDim.x) {
        if (off[q + 1] - off[q] < min_len) continue;
        if (!sp.keep(q / K, (int)(q % K))) continue;
        const int slot = atomicAdd(&list[0], 1);
        if (slot < cap) list[1 + slot] = (int32_t)q;
        else raise_error(err, GS_ERR_CAPACITY);
    }
}

__global__ void __launch_bounds__(1024)
k_sort_listed(const int32_t* __restrict__ off, const int32_t* __restrict__ list, int32_t cap,
              uint64_t* __restrict__ words)
{
    grid_dependency_sync();
    __shared__ uint64_t s_buf[kRpCtaCap];
    const int nl = min(list[0], cap);
    for (int k = blockIdx.x; k < nl; k += gridDim.x) {
        const int32_t q = list[1 + k];
        const int l = off[q + 1] - off[q];
        uint64_t* seg = words + off[q];
        if (l <= kRpCtaCap) {
            for (int i = threadIdx.x; i < l; i += blockDim.x) s_buf[i] = seg[i];
            __syncthreads();
            bitonic_mem(s_buf, l, threadIdx.x, blockDim.x, SyncBlock{});
            for (int i = threadIdx.x; i < l; i += blockDim.x) seg[i] = s_buf[i];
        } else {
            bitonic_mem(seg, l, threadIdx.x, blockDim.x, SyncBlock{});
        }
        __syncthreads();
    }
}

__global__ void k_fill_selected(const int32_t* __restrict__ off, int64_t nseg, const uint8_t* __restrict__ sel,
                                int mode, int min_len, uint8_t* __restrict__ out)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nseg; q += stride) {
        const int l = off[q + 1] - off[q];
        uint8_t v = 0;
        if (mode == GS_MODE_BINNED_EXACT) v = l >= min_len;
        else if (mode == GS_MODE_BINNED_PAPER) v = sel[q] && l >= 2;
        out[q] = v;
    }
}

int sort_long_segments(gs_ctx* ctx, int64_t nseg, const int32_t* offsets, uint64_t* words, int32_t min_len,
                       cudaStream_t st)
{
    if (nseg <= 0) return GS_OK;
    int r;
    const int32_t tail_cap = tail_capacity(nseg);
    if ((r = bins_reserve(ctx, 1, nseg)) != GS_OK) return r;
    GS_CUDA_TRY(cudaMemsetAsync(ctx->d_tail, 0, 4, st));
    const int64_t want = (nseg + 255) / 256, grid = (int64_t)ctx->num_sms * 8;
    GS_CUDA_TRY(launch_k(ctx, k_list_long, (unsigned)(want < grid ? want : grid), 256, 0, st, offsets, nseg, min_len, ctx->d_tail, tail_cap,
                                                                        ctx->d_err, ScatterPass(), 1, nullptr));
    GS_CUDA_TRY(launch_k(ctx, k_sort_listed, (unsigned)ctx->num_sms, 1024, 0, st, offsets, ctx->d_tail, tail_cap, words));
    ctx->launches += 2;
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

int repair(gs_ctx* ctx, int32_t n_tiles, const int64_t* m_dev, uint64_t* words, const int32_t* offsets,
           uint8_t* selected_out, cudaStream_t st)
{
    return repair_min(ctx, n_tiles, m_dev, words, offsets, selected_out, 2, st);
}

int repair_min(gs_ctx* ctx, int32_t n_tiles, const int64_t* m_dev, uint64_t* words, const int32_t* offsets,
               uint8_t* selected_out, int32_t min_len, cudaStream_t st, int pass)
{
    const gs_config& c = ctx->cfg;
    const int64_t nseg = (int64_t)n_tiles * c.K;
    int r;
    const unsigned grid = (unsigned)ctx->num_sms * 8;
    if (c.mode == GS_MODE_BINNED_NOREPAIR) {
        if (selected_out) GS_CUDA_TRY(cudaMemsetAsync(selected_out, 0, (size_t)nseg, st));
        return GS_OK;
    }
    const uint8_t* sel = nullptr;
    if (c.mode == GS_MODE_BINNED_PAPER) {
        // kept lengths -> exclusive prefix -> prefix-fitting selection -> exact greedy tail
        if ((r = bins_reserve(ctx, 1, nseg)) != GS_OK) return r;
        uint8_t* s = ctx->d_sel;
        int32_t* klen = reinterpret_cast<int32_t*>(s + align256((size_t)nseg));
        int32_t* pre = klen + (nseg + 1);
        k_keep_lengths<<<grid, 256, 0, st>>>(offsets, nseg, c.K, klen);
        if ((r = exclusive_scan_i32(ctx, klen, nseg, pre, nullptr, st)) != GS_OK) return r;
        k_select_prefix<<<grid, 256, 0, st>>>(klen, pre, nseg, m_dev, (double)c.repair_budget_frac, s);
        k_select_greedy<<<1, 1024, 0, st>>>(klen, pre, nseg, m_dev, (double)c.repair_budget_frac, s);
        ctx->launches += 3;
        GS_CUDA_TRY(cudaGetLastError());
        sel = s;
    }
    const int32_t tail_cap = tail_capacity(nseg);
    if ((r = bins_reserve(ctx, 1, nseg)) != GS_OK) return r;
    if (!(ctx->zeroed_tail == ctx->d_tail && ctx->zeroed_tail_bytes == ctx->tail_cap))
        GS_CUDA_TRY(cudaMemsetAsync(ctx->d_tail, 0, 4, st));
    ctx->zeroed_tail = nullptr;  // zeroed by the frame's first kernel once, for this call
    if (c.mode == GS_MODE_BINNED_EXACT && min_len > kRpWarpCap) {
        if (nseg > 0) {
            const int64_t want = (nseg + 255) / 256;
            const unsigned g = (unsigned)(want < (int64_t)grid ? want : (int64_t)grid);
            ScatterPass sp;
            if (pass) {
                sp.plan = ctx->d_plan;
                sp.T = n_tiles;
                sp.pass = pass;
            }
            GS_CUDA_TRY(launch_k(ctx, k_list_long, g, 256, 0, st, offsets, nseg, min_len, ctx->d_tail, tail_cap, ctx->d_err, sp, c.K,
                                           pass ? ctx->d_plist : nullptr));
            GS_CUDA_TRY(launch_k(ctx, k_sort_listed, (unsigned)ctx->num_sms, 1024, 0, st, offsets, ctx->d_tail, tail_cap, words));
            ctx->launches += 2;
        }
    } else if (n_tiles > 0)
        k_repair_tiles<<<(unsigned)n_tiles, kRpThreads, 0, st>>>(offsets, c.K, sel, words, ctx->d_tail, tail_cap,
                                                                 ctx->d_err, min_len);
    if (!(c.mode == GS_MODE_BINNED_EXACT && min_len > kRpWarpCap)) {
        k_repair_tail<<<(unsigned)ctx->num_sms, 1024, 0, st>>>(offsets, ctx->d_tail, tail_cap, words);
        ctx->launches += (n_tiles > 0 ? 2 : 1);
    }
    GS_CUDA_TRY(cudaGetLastError());
    if (selected_out) {
        k_fill_selected<<<grid, 256, 0, st>>>(offsets, nseg, sel, c.mode, min_len < 2 ? 2 : min_len, selected_out);
        ctx->launches += 1;
        GS_CUDA_TRY(cudaGetLastError());
    }
    return GS_OK;
}

}  // namespace gs
