// intersect.cu -- K3 tile intersection (Sec. 3.1: one record per covered
// tile) and the device-wide exclusive scans it and the binning use.
//
// Scan: three kernels without inter-block waits (reduce per block ->
// one-block scan of the block sums -> per-block rescan with the prefix), all
// in int64 so an overflowing total is detected instead of wrapping.
#include "internal.cuh"

namespace gs {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;  // per thread per block tile
constexpr int kScanTile = kScanThreads * kScanItems;

// Exclusive block scan of one value per thread (256 threads).  Returns the
// exclusive prefix; *total receives the block total.
__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t* s_warp, int64_t* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < (kScanThreads / 32) ? s_warp[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t t = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += t;
        }
        if (lane < (kScanThreads / 32)) s_warp[lane] = w;  // inclusive warp totals
    }
    __syncthreads();
    const int64_t warp_prefix = warp > 0 ? s_warp[warp - 1] : 0;
    *total = s_warp[kScanThreads / 32 - 1];
    __syncthreads();  // s_warp is reused by the next call
    return warp_prefix + incl - v;
}

struct LoadI32 {
    const int32_t* p;
    __device__ int64_t operator()(int64_t i) const { return p[i]; }
};

struct LoadRectCount {
    const uint2* rect;
    __device__ int64_t operator()(int64_t i) const
    {
        const uint2 r = rect[i];
        const int64_t w = (int64_t)(r.y & 0xffffu) - (int64_t)(r.x & 0xffffu);
        const int64_t h = (int64_t)(r.y >> 16) - (int64_t)(r.x >> 16);
        return w * h;
    }
};

template <class Load>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(Load ld, int64_t n, int64_t* sums)
{
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t acc = 0;
#pragma unroll 4
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < n) acc += ld(i);
    }
    __shared__ int64_t s_warp[kScanThreads / 32];
    int64_t total;
    block_exclusive_scan(acc, s_warp, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// One block: exclusive scan of sums[0..nb) in place; sums[nb] = grand total.
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(int64_t* sums, int64_t nb)
{
    __shared__ int64_t s_warp[kScanThreads / 32];
    int64_t carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += kScanThreads) {
        const int64_t i = b0 + threadIdx.x;
        const int64_t v = i < nb ? sums[i] : 0;
        int64_t total;
        const int64_t ex = block_exclusive_scan(v, s_warp, &total);
        if (i < nb) sums[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) sums[nb] = carry;
}

// Per-block rescan.  out[i] (int32) = exclusive prefix; out[n] = total.  The
// int64 total goes to total64.  A total >= 2^31 raises GS_ERR_CAPACITY and
// leaves out[] unwritten.
template <class Load>
__global__ void __launch_bounds__(kScanThreads)
k_scan_down(Load ld, int64_t n, const int64_t* sums, int64_t nb, int32_t* out, int64_t* total64, int* err)
{
    __shared__ int64_t s_warp[kScanThreads / 32];
    const int64_t grand = sums[nb];
    if (grand > (int64_t)INT32_MAX - 1) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            raise_error(err, GS_ERR_CAPACITY);
            if (total64) *total64 = grand;
        }
        return;
    }
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t carry = sums[blockIdx.x];
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        const int64_t v = i < n ? ld(i) : 0;
        int64_t total;
        const int64_t ex = block_exclusive_scan(v, s_warp, &total);
        if (i < n) out[i] = (int32_t)(carry + ex);
        carry += total;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        out[n] = (int32_t)grand;
        if (total64) *total64 = grand;
    }
}

int scan_reserve(gs_ctx* ctx, int64_t n)
{
    const int64_t nb = n > 0 ? (n + kScanTile - 1) / kScanTile : 1;
    return ensure(&ctx->d_scan, &ctx->scan_bytes, (size_t)(nb + 1) * sizeof(int64_t));
}

int goff_reserve(gs_ctx* ctx, int64_t n)
{
    size_t cap = ctx->goff_cap;
    void* p = ctx->d_goff;
    int r = ensure(&p, &cap, (size_t)(n + 1) * sizeof(int32_t));
    ctx->d_goff = static_cast<int32_t*>(p);
    ctx->goff_cap = cap;
    return r;
}

template <class Load>
static int scan_impl(gs_ctx* ctx, Load ld, int64_t n, int32_t* out, int64_t* total64, cudaStream_t st)
{
    const int64_t nb = n > 0 ? (n + kScanTile - 1) / kScanTile : 1;
    int r = ensure(&ctx->d_scan, &ctx->scan_bytes, (size_t)(nb + 1) * sizeof(int64_t));
    if (r != GS_OK) return r;
    int64_t* sums = static_cast<int64_t*>(ctx->d_scan);
    k_scan_reduce<Load><<<(unsigned)nb, kScanThreads, 0, st>>>(ld, n, sums);
    k_scan_sums<<<1, kScanThreads, 0, st>>>(sums, nb);
    k_scan_down<Load><<<(unsigned)nb, kScanThreads, 0, st>>>(ld, n, sums, nb, out, total64, ctx->d_err);
    ctx->launches += 3;
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

int exclusive_scan_i32(gs_ctx* ctx, const int32_t* counts, int64_t n, int32_t* out, int64_t* total64,
                       cudaStream_t st)
{
    return scan_impl(ctx, LoadI32{counts}, n, out, total64, st);
}

int scan_tile_counts(gs_ctx* ctx, const uint2* rect, int64_t n, int32_t* out, int64_t* total64,
                     cudaStream_t st)
{
    return scan_impl(ctx, LoadRectCount{rect}, n, out, total64, st);
}

// ------------------------------------------------------------------ emission
// One thread per Gaussian writes its tiles (row-major inside its rect) at its
// scanned offset: tile id, depth bits, gid.  Nothing is written when the
// total exceeds the capacity.
__global__ void __launch_bounds__(256)
k_emit(const uint2* __restrict__ rect, const float4* __restrict__ c_o_z, const int32_t* __restrict__ goff,
       int64_t n, int tiles_x, const int64_t* __restrict__ m_dev, int64_t m_cap, IsectView is, int* err)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t M = *m_dev;
    if (M > m_cap) {
        if (i == 0) raise_error(err, GS_ERR_CAPACITY);
        return;
    }
    if (i >= n) return;
    const uint2 r = rect[i];
    const uint32_t tx0 = r.x & 0xffffu, ty0 = r.x >> 16, tx1 = r.y & 0xffffu, ty1 = r.y >> 16;
    if (tx0 >= tx1 || ty0 >= ty1) return;
    const uint32_t zb = __float_as_uint(c_o_z[i].z);
    int64_t k = goff[i];
    for (uint32_t ty = ty0; ty < ty1; ++ty)
        for (uint32_t tx = tx0; tx < tx1; ++tx, ++k) {
            is.tile[k] = ty * (uint32_t)tiles_x + tx;
            is.zbits[k] = zb;
            is.gid[k] = (uint32_t)i;
        }
}

int count_scan(gs_ctx* ctx, const ProjView& pv, int64_t n, int64_t* m_dev, cudaStream_t st)
{
    int r = goff_reserve(ctx, n);
    if (r != GS_OK) return r;
    if (n == 0) {
        GS_CUDA_TRY(cudaMemsetAsync(m_dev, 0, sizeof(int64_t), st));
        return GS_OK;
    }
    return scan_tile_counts(ctx, pv.rect, n, ctx->d_goff, m_dev, st);
}

int emit_only(gs_ctx* ctx, const ProjView& pv, int64_t n, const gs_camera* cam, const IsectView& is,
              int64_t m_cap, const int64_t* m_dev, cudaStream_t st)
{
    if (n == 0) return GS_OK;
    const int tile = ctx->cfg.tile_size;
    const int tiles_x = (cam->width + tile - 1) / tile;
    k_emit<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pv.rect, pv.c_o_z, ctx->d_goff, n, tiles_x, m_dev,
                                                          m_cap, is, ctx->d_err);
    ctx->launches += 1;
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

int launch_emit(gs_ctx* ctx, const ProjView& pv, int64_t n, const gs_camera* cam, const IsectView& is,
                int64_t m_cap, int64_t* m_dev, cudaStream_t st)
{
    int r = count_scan(ctx, pv, n, m_dev, st);
    if (r != GS_OK) return r;
    return emit_only(ctx, pv, n, cam, is, m_cap, m_dev, st);
}

}  // namespace gs

namespace gs {
int sort_reserve(gs_ctx* ctx, int64_t m_cap);
int bins_reserve(gs_ctx* ctx, int64_t m_cap, int64_t nseg);

int reserve_internal(gs_ctx* ctx, int64_t n, int64_t m_cap, int32_t n_tiles)
{
    int r;
    const int64_t nseg = (int64_t)n_tiles * GS_MAX_K;
    if ((r = scan_reserve(ctx, n > nseg ? n : nseg)) != GS_OK) return r;
    if ((r = goff_reserve(ctx, n)) != GS_OK) return r;
    if (ctx->cfg.mode == GS_MODE_GLOBAL_SORT) return sort_reserve(ctx, m_cap);
    return bins_reserve(ctx, m_cap, (int64_t)n_tiles * ctx->cfg.K);
}
}  // namespace gs
