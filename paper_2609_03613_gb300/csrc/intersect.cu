// intersect.cu -- K3 tile intersection (Sec. 3.1: one record per covered
// tile) and the device-wide exclusive scans it and the binning use.
//
// Scan (scan.cuh): one pass with decoupled look-back and bounded waits,
// totals in int64 so an overflowing total is detected instead of wrapping.
#include "device.cuh"
#include "scan.cuh"

namespace gs {

int scan_reserve(gs_ctx* ctx, int64_t n)
{
    // two scans' block sums (scan2_impl)
    const int64_t nb = n > 0 ? (n + kScanTile - 1) / kScanTile : 1;
    return ensure(&ctx->d_scan, &ctx->scan_bytes, (size_t)2 * (nb + 1) * sizeof(int64_t));
}

// ctx->d_goff holds the per-Gaussian entry offsets [n+1], then the
// per-Gaussian row-record offsets [n+1] and the row-record total (int64)
static size_t goff_bytes(int64_t n) { return align256((size_t)(n + 1) * sizeof(int32_t)); }
int32_t* rows_offsets(gs_ctx* ctx, int64_t n) { return (int32_t*)((char*)ctx->d_goff + goff_bytes(n)); }
int64_t* rows_total(gs_ctx* ctx, int64_t n) { return (int64_t*)((char*)ctx->d_goff + 2 * goff_bytes(n)); }

int goff_reserve(gs_ctx* ctx, int64_t n)
{
    size_t cap = ctx->goff_cap;
    void* p = ctx->d_goff;
    int r = ensure(&p, &cap, 2 * goff_bytes(n) + sizeof(int64_t));
    ctx->d_goff = static_cast<int32_t*>(p);
    ctx->goff_cap = cap;
    return r;
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
// Warp-cooperative expansion (device.cuh): writes are coalesced and the work
// per lane is balanced whatever the rect sizes.  Nothing is written when the
// total exceeds the capacity.
__global__ void __launch_bounds__(256)
k_emit(const uint2* __restrict__ rect, const float4* __restrict__ c_o_z, const int32_t* __restrict__ goff,
       int64_t n, int tiles_x, const int64_t* __restrict__ m_dev, int64_t m_cap, IsectView is, int* err)
{
    const int64_t M = *m_dev;
    if (M > m_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) raise_error(err, GS_ERR_CAPACITY);
        return;
    }
    const int64_t g0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32;
    if (g0 >= n) return;
    const WarpExpand wx(rect, c_o_z, goff, n, g0);
    const int lane = threadIdx.x & 31;
    for (int32_t e0 = wx.base; e0 < wx.end; e0 += 32) {
        const int32_t e = e0 + lane;
        uint32_t g, t, z;
        wx.entry(e, tiles_x, &g, &t, &z);
        if (e < wx.end) {
            is.tile[e] = t;
            is.zbits[e] = z;
            is.gid[e] = g;
        }
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

// count_scan and, in the same pass, the row-record offsets of the EXACT
// bin construction (rows_offsets / rows_total)
int count_rows_scan(gs_ctx* ctx, const ProjView& pv, int64_t n, int64_t* m_dev, cudaStream_t st)
{
    int r = goff_reserve(ctx, n);
    if (r != GS_OK) return r;
    if (n == 0) {
        GS_CUDA_TRY(cudaMemsetAsync(m_dev, 0, sizeof(int64_t), st));
        GS_CUDA_TRY(cudaMemsetAsync(rows_offsets(ctx, 0), 0, sizeof(int32_t), st));
        GS_CUDA_TRY(cudaMemsetAsync(rows_total(ctx, 0), 0, sizeof(int64_t), st));
        return GS_OK;
    }
    return scan2_impl(ctx, LoadRectCountRows{pv.rect}, n, ctx->d_goff, m_dev, rows_offsets(ctx, n),
                      rows_total(ctx, n), st);
}

int emit_only(gs_ctx* ctx, const ProjView& pv, int64_t n, const gs_camera* cam, const IsectView& is,
              int64_t m_cap, const int64_t* m_dev, cudaStream_t st)
{
    if (n == 0) return GS_OK;
    const int tile = ctx->cfg.tile_size;
    const int tiles_x = (cam->width + tile - 1) / tile;
    const int64_t warps = (n + 31) / 32;
    k_emit<<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(pv.rect, pv.c_o_z, ctx->d_goff, n, tiles_x, m_dev,
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

int exact_bins_reserve(gs_ctx* ctx, int64_t n, int64_t m_cap, int32_t tiles_x, int32_t tiles_y, int K);
int samples_reserve(gs_ctx* ctx);

// Every stage's scratch for (n, m_cap, image), so that a later frame (or a
// stream capture of one) allocates nothing.
int reserve_internal(gs_ctx* ctx, int64_t n, int64_t m_cap, int32_t width, int32_t height)
{
    int r;
    const int tile = ctx->cfg.tile_size;
    const int32_t tiles_x = (width + tile - 1) / tile, tiles_y = (height + tile - 1) / tile;
    const int64_t nseg = (int64_t)tiles_x * tiles_y * GS_MAX_K;
    int64_t nscan = n > nseg ? n : nseg;
    const int64_t ngroup = group_scan_items(ctx, tiles_y, GS_MAX_K);
    if (ngroup > nscan) nscan = ngroup;
    // a frame's scan-flag arena (the row-count scan's two channels, the
    // offsets scan, the grouped scatter's scan) and, past it, the flags of
    // any one further scan
    auto blocks = [](int64_t items) { return items > 0 ? (items + kScanTile - 1) / kScanTile : 1; };
    const int64_t words = 2 * blocks(n) + blocks(nseg) + tiles_y + blocks(ngroup) + 2 * blocks(nscan) + 4;
    if ((r = ensure(&ctx->d_scan, &ctx->scan_bytes, (size_t)words * sizeof(uint64_t))) != GS_OK) return r;
    if ((r = goff_reserve(ctx, n)) != GS_OK) return r;
    if ((r = samples_reserve(ctx)) != GS_OK) return r;
    if (ctx->cfg.mode == GS_MODE_GLOBAL_SORT) return sort_reserve(ctx, m_cap);
    if ((r = bins_reserve(ctx, m_cap, (int64_t)tiles_x * tiles_y * ctx->cfg.K)) != GS_OK) return r;
    if (ctx->cfg.mode == GS_MODE_BINNED_EXACT)
        return exact_bins_reserve(ctx, n, m_cap, tiles_x, tiles_y, ctx->cfg.K);
    return GS_OK;
}
}  // namespace gs
