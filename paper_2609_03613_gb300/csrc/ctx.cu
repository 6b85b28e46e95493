// ctx.cu -- context, configuration, layouts, error word, stage timing and the
// C-ABI entry points that sequence the kernels of the other translation units.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "internal.cuh"

int gs_cuda_fail(cudaError_t e, const char* what)
{
    if (getenv("TILEGS_DEBUG")) fprintf(stderr, "tilegs: %s failed: %s\n", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? GS_ERR_NO_MEMORY : GS_ERR_CUDA;
}

extern "C" const char* gs_status_string(int status)
{
    switch (status) {
        case GS_OK: return "ok";
        case GS_ERR_INVALID_ARG: return "invalid argument";
        case GS_ERR_CAPACITY: return "entry capacity exceeded";
        case GS_ERR_CUDA: return "CUDA runtime error";
        case GS_ERR_TIMEOUT: return "bounded device wait timed out";
        case GS_ERR_NO_MEMORY: return "out of device memory";
        case GS_ERR_NUMERIC: return "non-finite input";
        default: return "unknown status";
    }
}

// Defaults: the paper's supplement tables (default No-GW configuration and
// default selective-repair thresholds) and Sec. 4.4 (K = 64).
extern "C" void gs_config_default(gs_config* cfg, int32_t mode)
{
    memset(cfg, 0, sizeof(*cfg));
    cfg->mode = mode;
    cfg->tile_size = 16;
    cfg->K = 64;
    cfg->sample_count = 8192;
    cfg->p_lo = 1.0f;
    cfg->p_hi = 99.0f;
    cfg->pad = 0.05f;
    cfg->near_alpha = 1.0f;
    cfg->near_gamma = 0.25f;
    cfg->eps = 1e-4f;
    cfg->repair_budget_frac = 0.25f;
    cfg->near_shift = (mode == GS_MODE_BINNED_PAPER || mode == GS_MODE_BINNED_NOREPAIR) ? 1 : 0;
    // GLOBAL: the plain baseline raster; 1 there rasters the global stream
    // with the binned kernel's culls (an ablation of the raster's additions)
    cfg->tile_cull = (mode == GS_MODE_GLOBAL_SORT) ? 0 : 1;
    cfg->persistent = 1;
    cfg->repair_in_raster = (mode == GS_MODE_BINNED_EXACT) ? 1 : 0;
    cfg->chunk_cap = 256;
    cfg->planner = 0;
    cfg->wait_polls = 1 << 22;
    cfg->planner_quantile = 0.9f;
    cfg->pdl = 1;
}

namespace gs {

int check_config(const gs_config* c)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (c->mode < GS_MODE_GLOBAL_SORT || c->mode > GS_MODE_BINNED_NOREPAIR) return GS_ERR_INVALID_ARG;
    if (c->tile_size != 8 && c->tile_size != 16 && c->tile_size != 32) return GS_ERR_INVALID_ARG;
    if (c->K < 1 || c->K > GS_MAX_K) return GS_ERR_INVALID_ARG;
    if (c->sample_count < 1 || c->sample_count > 8192) return GS_ERR_INVALID_ARG;
    if (!(c->p_lo >= 0.0f && c->p_lo <= 100.0f && c->p_hi >= c->p_lo && c->p_hi <= 100.0f))
        return GS_ERR_INVALID_ARG;
    if (!(c->pad >= 0.0f) || !(c->eps > 0.0f) || !(c->repair_budget_frac >= 0.0f))
        return GS_ERR_INVALID_ARG;
    if (c->mode == GS_MODE_BINNED_EXACT && c->near_shift) return GS_ERR_INVALID_ARG;
    if (c->chunk_cap != 0 && (c->chunk_cap < 32 || c->chunk_cap > 2048)) return GS_ERR_INVALID_ARG;
    if (c->planner != 0 && c->planner != 1) return GS_ERR_INVALID_ARG;
    if (c->wait_polls < 0) return GS_ERR_INVALID_ARG;
    if (!(c->planner_quantile > 0.0f && c->planner_quantile <= 1.0f)) return GS_ERR_INVALID_ARG;
    if (c->pdl != 0 && c->pdl != 1) return GS_ERR_INVALID_ARG;
    return GS_OK;
}

int ensure(void** p, size_t* cap, size_t bytes)
{
    if (bytes == 0) bytes = 256;
    if (*p && *cap >= bytes) return GS_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    size_t want = align256(bytes + bytes / 8);
    cudaError_t e = cudaMalloc(p, want);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return GS_ERR_NO_MEMORY;
    }
    *cap = want;
    return GS_OK;
}

// Inside a stream capture the records become external event-record nodes,
// so the graph's replays still time every stage.
static void record(gs_ctx* ctx, cudaEvent_t ev, cudaStream_t st)
{
    if (ctx->capturing) cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
    else cudaEventRecord(ev, st);
}

void stage_begin(gs_ctx* ctx, int stage, cudaStream_t st)
{
    if (ctx->timing && ctx->ev_ok) {
        record(ctx, ctx->ev_b[stage], st);
        ctx->stage_used[stage] = 1;
    }
}

void stage_end(gs_ctx* ctx, int stage, cudaStream_t st)
{
    if (ctx->timing && ctx->ev_ok) record(ctx, ctx->ev_e[stage], st);
}

}  // namespace gs

using namespace gs;

extern "C" int gs_create(gs_ctx** out, const gs_config* cfg)
{
    if (!out || check_config(cfg) != GS_OK) return GS_ERR_INVALID_ARG;
    gs_ctx* c = new gs_ctx();
    c->cfg = *cfg;
    cudaGetDevice(&c->device);
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (cudaMalloc(&c->d_err, sizeof(int)) != cudaSuccess) { delete c; return GS_ERR_NO_MEMORY; }
    cudaMemset(c->d_err, 0, sizeof(int));
    if (cudaMalloc(&c->d_bp, sizeof(BinParams)) != cudaSuccess) { gs_destroy(c); return GS_ERR_NO_MEMORY; }
    if (cudaMalloc(&c->d_tile_counter, 64 * sizeof(int32_t)) != cudaSuccess) { gs_destroy(c); return GS_ERR_NO_MEMORY; }
    if (cudaMalloc(&c->r_m, 2 * sizeof(int64_t)) != cudaSuccess) { gs_destroy(c); return GS_ERR_NO_MEMORY; }
    if (cudaMalloc(&c->d_ops, sizeof(int64_t)) != cudaSuccess) { gs_destroy(c); return GS_ERR_NO_MEMORY; }
    if (cudaMalloc(&c->d_scan_done, sizeof(unsigned int)) != cudaSuccess) { gs_destroy(c); return GS_ERR_NO_MEMORY; }
    cudaMemset(c->d_scan_done, 0, sizeof(unsigned int));
    if (raster_bwd_prepare() != GS_OK || bin_offsets_prepare() != GS_OK) { gs_destroy(c); return GS_ERR_CUDA; }
    if (cudaMallocHost(&c->h_m, 2 * sizeof(int64_t)) != cudaSuccess) { gs_destroy(c); return GS_ERR_NO_MEMORY; }
    c->ev_ok = 1;
    for (int s = 0; s < GS_STAGE_COUNT; ++s) {
        if (cudaEventCreate(&c->ev_b[s]) != cudaSuccess || cudaEventCreate(&c->ev_e[s]) != cudaSuccess)
            c->ev_ok = 0;
        c->stage_used[s] = 0;
        c->stage_ms[s] = 0.0f;
    }
    *out = c;
    return GS_OK;
}

extern "C" int gs_destroy(gs_ctx* c)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (c->pipe_down) {
        // pipelined frames still in flight finish before their buffers go
        cudaStreamSynchronize(c->pipe_up);
        cudaStreamSynchronize(c->pipe_down);
        cudaStreamDestroy(c->pipe_up);
        cudaStreamDestroy(c->pipe_down);
    }
    for (auto& P : c->pipe) {
        if (P.scene) cudaFree(P.scene);
        if (P.out) cudaFree(P.out);
        for (cudaEvent_t e : {P.uploaded, P.rendered, P.downloaded})
            if (e) cudaEventDestroy(e);
    }
    void* ptrs[] = {c->d_err, c->d_scan, c->d_goff, c->d_keys[0], c->d_keys[1], c->d_vals[0],
                    c->d_vals[1], c->d_hist, c->d_count, c->d_bin, c->d_bp, c->d_sel, c->d_tail,
                    c->d_tiles_order, c->d_tile_counter, c->r_proj, c->r_isect, c->r_stream,
                    c->r_off, c->r_m, c->r_scene, c->r_out, c->d_ops, c->d_tiles, c->d_samples,
                    c->r_T, c->r_tend, c->r_wend, c->d_planner, c->d_feat, c->d_plan, c->d_plist,
                    c->d_order_ws, c->d_scan_done};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->h_m) cudaFreeHost(c->h_m);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    batch_destroy(c);
    if (c->ev_ok)
        for (int s = 0; s < GS_STAGE_COUNT; ++s) {
            cudaEventDestroy(c->ev_b[s]);
            cudaEventDestroy(c->ev_e[s]);
        }
    delete c;
    return GS_OK;
}

extern "C" int gs_set_config(gs_ctx* c, const gs_config* cfg)
{
    if (!c || check_config(cfg) != GS_OK) return GS_ERR_INVALID_ARG;
    c->cfg = *cfg;
    return GS_OK;
}

extern "C" int gs_get_config(const gs_ctx* c, gs_config* cfg)
{
    if (!c || !cfg) return GS_ERR_INVALID_ARG;
    *cfg = c->cfg;
    return GS_OK;
}

extern "C" int gs_get_error(gs_ctx* c, void* stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    int h = 0;
    GS_CUDA_TRY(cudaMemcpyAsync(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    GS_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    if (h == 0) h = batch_error(c, (cudaStream_t)stream);
    return h;
}

extern "C" int gs_clear_error(gs_ctx* c, void* stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    GS_CUDA_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(int), (cudaStream_t)stream));
    return batch_clear_error(c, (cudaStream_t)stream);
}

extern "C" int gs_enable_timing(gs_ctx* c, int32_t on)
{
    if (!c) return GS_ERR_INVALID_ARG;
    c->timing = on ? 1 : 0;
    return GS_OK;
}

extern "C" int gs_get_stage_times(gs_ctx* c, float* ms)
{
    if (!c || !ms) return GS_ERR_INVALID_ARG;
    for (int s = 0; s < GS_STAGE_COUNT; ++s) {
        ms[s] = 0.0f;
        if (c->timing && c->ev_ok && c->stage_used[s]) {
            GS_CUDA_TRY(cudaEventSynchronize(c->ev_e[s]));
            float v = 0.0f;
            if (cudaEventElapsedTime(&v, c->ev_b[s], c->ev_e[s]) == cudaSuccess) ms[s] = v;
            else cudaGetLastError();
        }
        c->stage_used[s] = 0;
    }
    return GS_OK;
}

// ------------------------------------------------------------------ layouts
extern "C" size_t gs_projected_offset(int64_t n, int32_t field)
{
    const size_t sizes[GS_P_NFIELDS] = {16, 16, 16, 8, 4};
    size_t off = 0;
    for (int f = 0; f < field && f < GS_P_NFIELDS; ++f) off += align256(sizes[f] * (size_t)n);
    return off;
}

extern "C" size_t gs_projected_bytes(int64_t n) { return gs_projected_offset(n, GS_P_NFIELDS); }

extern "C" size_t gs_grad2d_offset(int64_t n, int32_t field)
{
    return (size_t)(field < 0 ? 0 : field > 3 ? 3 : field) * align256((size_t)n * 16);
}

extern "C" size_t gs_grad2d_bytes(int64_t n) { return gs_grad2d_offset(n, 3); }

extern "C" size_t gs_isect_offset(int64_t m_cap, int32_t field)
{
    return (size_t)field * align256((size_t)m_cap * 4);
}

extern "C" size_t gs_isect_bytes(int64_t m_cap) { return gs_isect_offset(m_cap, 3); }

extern "C" int32_t gs_num_tiles(int32_t width, int32_t height, int32_t tile)
{
    if (tile <= 0 || width <= 0 || height <= 0) return 0;
    return ((width + tile - 1) / tile) * ((height + tile - 1) / tile);
}

bool gs::camera_ok(const gs_camera* cam)
{
    if (!cam) return false;
    if (cam->width <= 0 || cam->height <= 0 || cam->width > 65535 * 8 || cam->height > 65535 * 8)
        return false;
    if (!(cam->fx > 0.0f) || !(cam->fy > 0.0f)) return false;
    if (!(cam->near_plane >= 0.0f) || !(cam->far_plane > cam->near_plane)) return false;
    return true;
}

static bool cam_ok(const gs_camera* cam) { return camera_ok(cam); }

// ------------------------------------------------------------------ entry points
namespace gs {
int launch_project(gs_ctx* ctx, const float* means, const float* scales, const float* quats,
                   const float* opac, const float* sh, int32_t sh_degree, int64_t n,
                   const gs_camera* cam, const ProjView& pv, cudaStream_t st, const FrameZero& fz = FrameZero());
int launch_emit(gs_ctx* ctx, const ProjView& pv, int64_t n, const gs_camera* cam,
                const IsectView& is, int64_t m_cap, int64_t* m_dev, cudaStream_t st);
}  // namespace gs

extern "C" int gs_project(gs_ctx* ctx, const float* means, const float* scales, const float* quats,
                          const float* opacities, const float* sh, int32_t sh_degree, int64_t n,
                          const gs_camera* cam, void* projected, void* stream)
{
    if (!ctx || !cam_ok(cam) || n < 0 || n > INT32_MAX - 1 || sh_degree < 0 || sh_degree > 3)
        return GS_ERR_INVALID_ARG;
    if (n > 0 && (!means || !scales || !quats || !opacities || !sh || !projected))
        return GS_ERR_INVALID_ARG;
    if (n == 0) return GS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    stage_begin(ctx, GS_STAGE_PROJECT, st);
    int r = launch_project(ctx, means, scales, quats, opacities, sh, sh_degree, n, cam,
                           proj_view(projected, n), st);
    stage_end(ctx, GS_STAGE_PROJECT, st);
    return r;
}

extern "C" int gs_tile_intersect(gs_ctx* ctx, const void* projected, int64_t n, const gs_camera* cam,
                                 void* isect, int64_t m_cap, int64_t* m_dev, int64_t* m_host,
                                 void* stream)
{
    if (!ctx || !cam_ok(cam) || n < 0 || n > INT32_MAX - 1 || m_cap < 0 || m_cap > INT32_MAX - 1 || !m_dev)
        return GS_ERR_INVALID_ARG;
    if ((n > 0 && !projected) || (m_cap > 0 && !isect)) return GS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    stage_begin(ctx, GS_STAGE_INTERSECT, st);
    int r = launch_emit(ctx, proj_view(const_cast<void*>(projected), n), n, cam,
                        isect_view(isect, m_cap), m_cap, m_dev, st);
    stage_end(ctx, GS_STAGE_INTERSECT, st);
    if (r != GS_OK) return r;
    if (m_host) {
        GS_CUDA_TRY(cudaMemcpyAsync(ctx->h_m, m_dev, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        GS_CUDA_TRY(cudaStreamSynchronize(st));
        *m_host = ctx->h_m[0];
        if (ctx->h_m[0] > m_cap) return GS_ERR_CAPACITY;
    }
    return GS_OK;
}

static int sort_args_ok(gs_ctx* ctx, const gs_camera* cam, int64_t n, int64_t m_cap, const int64_t* m_dev)
{
    if (!ctx || !cam_ok(cam) || n < 0 || m_cap < 0 || m_cap > INT32_MAX - 1 || !m_dev) return 0;
    return 1;
}

extern "C" int gs_depth_range(gs_ctx* ctx, const void* projected, const float* scales, int64_t n,
                              const gs_camera* cam, const void* isect, int64_t m_cap,
                              const int64_t* m_dev, float* zrange, void* stream)
{
    if (!sort_args_ok(ctx, cam, n, m_cap, m_dev) || !zrange) return GS_ERR_INVALID_ARG;
    if (ctx->cfg.near_shift && !scales) return GS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int r = depth_range(ctx, proj_view(const_cast<void*>(projected), n), scales,
                        isect_view(const_cast<void*>(isect), m_cap), m_cap, m_dev, cam, st);
    if (r != GS_OK) return r;
    GS_CUDA_TRY(cudaMemcpyAsync(zrange, ctx->d_bp, 2 * sizeof(float), cudaMemcpyDeviceToDevice, st));
    return GS_OK;
}

extern "C" int gs_bin_build(gs_ctx* ctx, const void* projected, const float* scales, int64_t n,
                            const gs_camera* cam, const void* isect, int64_t m_cap,
                            const int64_t* m_dev, const float* zrange, uint64_t* stream_words,
                            int32_t* offsets, void* stream)
{
    if (!sort_args_ok(ctx, cam, n, m_cap, m_dev) || !zrange || !stream_words || !offsets)
        return GS_ERR_INVALID_ARG;
    if (ctx->cfg.mode == GS_MODE_GLOBAL_SORT) return GS_ERR_INVALID_ARG;
    if (ctx->cfg.near_shift && !scales) return GS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int r = set_zrange(ctx, zrange, st);
    if (r != GS_OK) return r;
    const int32_t T = gs_num_tiles(cam->width, cam->height, ctx->cfg.tile_size);
    return bin_build(ctx, proj_view(const_cast<void*>(projected), n), scales,
                     isect_view(const_cast<void*>(isect), m_cap), m_cap, m_dev, T, stream_words,
                     offsets, st);
}

extern "C" int gs_repair(gs_ctx* ctx, const gs_camera* cam, const int64_t* m_dev, uint64_t* stream_words,
                         const int32_t* offsets, uint8_t* selected_out, void* stream)
{
    if (!ctx || !cam_ok(cam) || !m_dev || !stream_words || !offsets) return GS_ERR_INVALID_ARG;
    if (ctx->cfg.mode == GS_MODE_GLOBAL_SORT) return GS_ERR_INVALID_ARG;
    const int32_t T = gs_num_tiles(cam->width, cam->height, ctx->cfg.tile_size);
    return repair(ctx, T, m_dev, stream_words, offsets, selected_out, (cudaStream_t)stream);
}

extern "C" int gs_sort_or_bin(gs_ctx* ctx, const void* projected, const float* scales, int64_t n,
                              const gs_camera* cam, const void* isect, int64_t m_cap,
                              const int64_t* m_dev, uint64_t* stream_words, int32_t* offsets,
                              float* zrange_out, void* stream)
{
    if (!sort_args_ok(ctx, cam, n, m_cap, m_dev) || !stream_words || !offsets) return GS_ERR_INVALID_ARG;
    if (m_cap > 0 && !isect) return GS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int32_t T = gs_num_tiles(cam->width, cam->height, ctx->cfg.tile_size);
    IsectView is = isect_view(const_cast<void*>(isect), m_cap);
    if (ctx->cfg.mode == GS_MODE_GLOBAL_SORT) {
        stage_begin(ctx, GS_STAGE_SORT, st);
        int r = global_sort(ctx, is, m_cap, m_dev, T, stream_words, offsets, st);
        stage_end(ctx, GS_STAGE_SORT, st);
        return r;
    }
    if (ctx->cfg.near_shift && !scales) return GS_ERR_INVALID_ARG;
    ProjView pv = proj_view(const_cast<void*>(projected), n);
    stage_begin(ctx, GS_STAGE_DEPTH_RANGE, st);
    int r = depth_range(ctx, pv, scales, is, m_cap, m_dev, cam, st);
    stage_end(ctx, GS_STAGE_DEPTH_RANGE, st);
    if (r != GS_OK) return r;
    if (zrange_out)
        GS_CUDA_TRY(cudaMemcpyAsync(zrange_out, ctx->d_bp, 2 * sizeof(float), cudaMemcpyDeviceToDevice, st));
    if (ctx->cfg.mode == GS_MODE_BINNED_EXACT) {
        stage_begin(ctx, GS_STAGE_BIN, st);
        r = exact_bins(ctx, pv, n, cam, false, m_cap, m_dev, stream_words, offsets, st);
        stage_end(ctx, GS_STAGE_BIN, st);
        if (r != GS_OK) return r;
        stage_begin(ctx, GS_STAGE_REPAIR, st);
        r = repair_min(ctx, T, m_dev, stream_words, offsets, nullptr,
                       ctx->cfg.repair_in_raster ? kRasterSortCap + 1 : 2, st);
        stage_end(ctx, GS_STAGE_REPAIR, st);
        return r;
    }
    stage_begin(ctx, GS_STAGE_BIN, st);
    r = bin_build(ctx, pv, scales, is, m_cap, m_dev, T, stream_words, offsets, st);
    stage_end(ctx, GS_STAGE_BIN, st);
    if (r != GS_OK) return r;
    stage_begin(ctx, GS_STAGE_REPAIR, st);
    r = repair(ctx, T, m_dev, stream_words, offsets, nullptr, st);
    stage_end(ctx, GS_STAGE_REPAIR, st);
    return r;
}

extern "C" int gs_rasterize_fwd(gs_ctx* ctx, const void* projected, int64_t n, const gs_camera* cam,
                                uint64_t* stream_words, const int32_t* offsets,
                                int32_t offsets_stride, const float* bg, float* rgb, float* alpha,
                                int32_t* last, int32_t* ntests, float* final_T, int32_t* tile_end, void* stream)
{
    if (!ctx || !cam_ok(cam) || n < 0 || !offsets || !bg || !rgb || !alpha || !last)
        return GS_ERR_INVALID_ARG;
    if (n > 0 && (!projected || !stream_words)) return GS_ERR_INVALID_ARG;
    if (offsets_stride < 1 || offsets_stride > GS_MAX_K) return GS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const bool baseline = baseline_raster(ctx->cfg);
    stage_begin(ctx, GS_STAGE_RASTER, st);
    int r = raster_fwd(ctx, proj_view(const_cast<void*>(projected), n), cam, stream_words, offsets,
                       offsets_stride, bg, rgb, alpha, last, ntests, baseline, st, final_T, tile_end);
    stage_end(ctx, GS_STAGE_RASTER, st);
    return r;
}

extern "C" int gs_rasterize_fwd_plan(gs_ctx* ctx, const void* projected, int64_t n, const gs_camera* cam,
                                     uint64_t* stream_words, const int32_t* offsets, int32_t offsets_stride,
                                     const float* bg, float* rgb, float* alpha, int32_t* last, const uint8_t* plan,
                                     uint8_t* flags, int32_t* bins_needed, void* stream)
{
    if (!ctx || !cam_ok(cam) || n < 0 || !offsets || !bg || !rgb || !alpha || !last)
        return GS_ERR_INVALID_ARG;
    if (n > 0 && (!projected || !stream_words)) return GS_ERR_INVALID_ARG;
    if (offsets_stride < 1 || offsets_stride > GS_MAX_K) return GS_ERR_INVALID_ARG;
    if (bins_needed && plan) return GS_ERR_INVALID_ARG;
    if (ctx->cfg.mode != GS_MODE_BINNED_EXACT || !ctx->cfg.repair_in_raster) return GS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int32_t T = gs_num_tiles(cam->width, cam->height, ctx->cfg.tile_size);
    PlanView pl;
    pl.bins = plan;
    pl.needed = bins_needed;
    int r;
    if (flags) {
        // the context's flag region (tile flags, then row flags), copied out
        if ((r = planner_buffers(ctx, T)) != GS_OK) return r;
        GS_CUDA_TRY(cudaMemsetAsync(ctx->d_plan + T, 0, 2 * (size_t)T, st));
        GS_CUDA_TRY(cudaMemsetAsync(ctx->d_plist, 0, sizeof(int32_t), st));
        pl.flag = ctx->d_plan + T;
        pl.list = ctx->d_plist;
    }
    stage_begin(ctx, GS_STAGE_RASTER, st);
    r = raster_fwd(ctx, proj_view(const_cast<void*>(projected), n), cam, stream_words, offsets, offsets_stride, bg,
                   rgb, alpha, last, nullptr, false, st, nullptr, nullptr, pl);
    stage_end(ctx, GS_STAGE_RASTER, st);
    if (r == GS_OK && flags)
        GS_CUDA_TRY(cudaMemcpyAsync(flags, ctx->d_plan + T, (size_t)T, cudaMemcpyDeviceToDevice, st));
    return r;
}

extern "C" int gs_rasterize_bwd(gs_ctx* ctx, const void* projected, int64_t n, const gs_camera* cam,
                                const uint64_t* stream_words, const int32_t* offsets, int32_t offsets_stride,
                                const float* bg, const int32_t* last, const float* final_T,
                                const int32_t* tile_end, const float* dl_drgb, const float* dl_dalpha, void* grad,
                                void* stream)
{
    if (!ctx || !cam_ok(cam) || n < 0 || !offsets || !bg || !last || !final_T || !tile_end || !dl_drgb || !grad)
        return GS_ERR_INVALID_ARG;
    if (n > 0 && (!projected || !stream_words)) return GS_ERR_INVALID_ARG;
    if (offsets_stride < 1 || offsets_stride > GS_MAX_K) return GS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(grad) & 255u) != 0) return GS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    GS_CUDA_TRY(cudaMemsetAsync(grad, 0, gs_grad2d_bytes(n), st));
    if (n == 0) return GS_OK;
    return raster_bwd(ctx, proj_view(const_cast<void*>(projected), n), cam, stream_words, offsets, offsets_stride,
                      bg, last, final_T, tile_end, dl_drgb, dl_dalpha, grad_view(grad, n), st);
}

// ------------------------------------------------------------------ whole frame
int gs::render_buffers(gs_ctx* c, int64_t n, int64_t m_cap, int32_t T)
{
    int r;
    if ((r = ensure(&c->r_proj, &c->r_proj_cap, gs_projected_bytes(n))) != GS_OK) return r;
    if (m_cap > c->r_m_cap) {
        size_t cap_bytes = 0;
        if (c->r_isect) cudaFree(c->r_isect);
        if (c->r_stream) cudaFree(c->r_stream);
        c->r_isect = nullptr;
        c->r_stream = nullptr;
        c->r_m_cap = 0;
        if ((r = ensure(&c->r_isect, &cap_bytes, gs_isect_bytes(m_cap))) != GS_OK) return r;
        size_t sb = 0;
        void* sp = nullptr;
        if ((r = ensure(&sp, &sb, (size_t)m_cap * 8)) != GS_OK) return r;
        c->r_stream = (uint64_t*)sp;
        c->r_m_cap = m_cap;
    }
    const int32_t kmax = c->cfg.mode == GS_MODE_GLOBAL_SORT ? 1 : c->cfg.K;
    void* op = c->r_off;
    if ((r = ensure(&op, &c->r_off_cap, ((size_t)T * kmax + 1) * 4)) != GS_OK) return r;
    c->r_off = (int32_t*)op;
    return GS_OK;
}

extern "C" int gs_reserve(gs_ctx* c, int64_t n, int64_t m_cap, int32_t width, int32_t height)
{
    if (!c || n < 0 || m_cap < 0 || m_cap > INT32_MAX - 1 || width <= 0 || height <= 0)
        return GS_ERR_INVALID_ARG;
    const int32_t T = gs_num_tiles(width, height, c->cfg.tile_size);
    int r = render_buffers(c, n, m_cap, T);
    if (r != GS_OK) return r;
    // grow the internal scratch of every stage once, outside any capture
    return gs::reserve_internal(c, n, m_cap, width, height);
}

extern "C" int64_t gs_last_entry_count(gs_ctx* c) { return c ? c->last_m : -1; }

extern "C" int64_t gs_launch_count(const gs_ctx* c) { return c ? c->launches + batch_launch_count(c) : -1; }

extern "C" int32_t gs_last_flagged_tiles(gs_ctx* c, void* stream)
{
    if (!c) return -1;
    if (!c->d_plist) return 0;
    int32_t h = 0;
    if (cudaMemcpyAsync(&h, c->d_plist, sizeof(int32_t), cudaMemcpyDeviceToHost, (cudaStream_t)stream) != cudaSuccess ||
        cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
        return -1;
    return h;
}

extern "C" int64_t gs_last_raster_ops(gs_ctx* c, void* stream)
{
    if (!c) return -1;
    int64_t h = 0;
    if (cudaMemcpyAsync(&h, c->d_ops, sizeof(int64_t), cudaMemcpyDeviceToHost, (cudaStream_t)stream) != cudaSuccess ||
        cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
        return -1;
    return h;
}

// per-frame planner features and plan
int gs::planner_buffers(gs_ctx* c, int32_t T)
{
    int r;
    void* p = c->d_feat;
    if ((r = ensure(&p, &c->feat_cap, (size_t)T * GS_PLAN_FEATURES * 4 + 16)) != GS_OK) return r;
    c->d_feat = (float*)p;
    p = c->d_plan;
    if ((r = ensure(&p, &c->plan_cap_bytes, 3 * (size_t)T + 16)) != GS_OK) return r;
    c->d_plan = (uint8_t*)p;
    p = c->d_plist;
    if ((r = ensure(&p, &c->plist_cap, ((size_t)T + 1) * 4)) != GS_OK) return r;
    c->d_plist = (int32_t*)p;
    return GS_OK;
}

// buffers of the state GS_RENDER_SAVE keeps for gs_render_bwd
int gs::render_save_buffers(gs_ctx* c, int32_t W, int32_t H, int32_t T)
{
    int r;
    void* p = c->r_T;
    if ((r = ensure(&p, &c->r_T_cap, (size_t)W * H * 4)) != GS_OK) return r;
    c->r_T = (float*)p;
    p = c->r_tend;
    if ((r = ensure(&p, &c->r_tend_cap, (size_t)T * 4 + 4)) != GS_OK) return r;
    c->r_tend = (int32_t*)p;
    p = c->r_wend;
    const int ts = c->cfg.tile_size;
    if ((r = ensure(&p, &c->r_wend_cap, (size_t)T * (ts * ts / 32) * 4 + 4)) != GS_OK) return r;
    c->r_wend = (int32_t*)p;
    return GS_OK;
}

// Everything of a frame after the projection (the record is in c->r_proj):
// intersect, sort or bin, repair, raster (and the saved state).  Device
// outputs.  Without GS_RENDER_NO_SYNC the entry count is read back once to
// grow the entry buffers.
int gs::render_binning(gs_ctx* c, int64_t n, const float* scales, const gs_camera* cam, int32_t flags,
                       cudaStream_t st)
{
    const int32_t W = cam->width, H = cam->height;
    const int32_t T = gs_num_tiles(W, H, c->cfg.tile_size);
    ProjView pv = proj_view(c->r_proj, n);
    int r;
    stage_begin(c, GS_STAGE_INTERSECT, st);
    // EXACT with the tile cull: the row-record offsets in the same pass
    const bool rows = c->cfg.mode == GS_MODE_BINNED_EXACT && c->cfg.tile_cull;
    r = rows ? count_rows_scan(c, pv, n, c->r_m, st) : count_scan(c, pv, n, c->r_m, st);
    if (r != GS_OK) return r;
    if (!(flags & GS_RENDER_NO_SYNC)) {
        // size the entry buffers: read M once, grow if needed
        GS_CUDA_TRY(cudaMemcpyAsync(c->h_m, c->r_m, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        GS_CUDA_TRY(cudaStreamSynchronize(st));
        if (c->h_m[0] > c->r_m_cap) {
            if ((r = render_buffers(c, n, c->h_m[0], T)) != GS_OK) return r;
        }
    }
    if (c->cfg.mode == GS_MODE_BINNED_EXACT) {
        // the emission is fused with the bucketing by tile: no emission-order
        // entries are written; depth samples map to gids through the offsets
        stage_end(c, GS_STAGE_INTERSECT, st);
        stage_begin(c, GS_STAGE_DEPTH_RANGE, st);
        r = depth_range_goff(c, pv, scales, n, c->r_m_cap, c->r_m, cam, st);
        stage_end(c, GS_STAGE_DEPTH_RANGE, st);
        if (r != GS_OK) return r;
        const bool planned = frame_planned(c);
        if (planned) {
            if (!c->planner_ready) return GS_ERR_INVALID_ARG;  // gs_planner_set_weights first
            if ((r = planner_buffers(c, T)) != GS_OK) return r;
        }
        stage_begin(c, GS_STAGE_BIN, st);
        r = exact_bins(c, pv, n, cam, true, c->r_m_cap, c->r_m, c->r_stream, c->r_off, st, rows, planned);
        stage_end(c, GS_STAGE_BIN, st);
        if (r != GS_OK) return r;
        stage_begin(c, GS_STAGE_REPAIR, st);
        r = repair_min(c, T, c->r_m, c->r_stream, c->r_off, nullptr,
                       c->cfg.repair_in_raster ? kRasterSortCap + 1 : 2, st, planned ? 1 : 0);
        stage_end(c, GS_STAGE_REPAIR, st);
    } else {
        r = emit_only(c, pv, n, cam, isect_view(c->r_isect, c->r_m_cap), c->r_m_cap, c->r_m, st);
        stage_end(c, GS_STAGE_INTERSECT, st);
        if (r != GS_OK) return r;
        r = gs_sort_or_bin(c, c->r_proj, scales, n, cam, c->r_isect, c->r_m_cap, c->r_m, c->r_stream,
                           c->r_off, nullptr, st);
    }
    return r;
}

int gs::render_after_project(gs_ctx* c, int64_t n, const float* scales, const gs_camera* cam, const float* bg,
                             float* d_rgb, float* d_alpha, int32_t* d_last, int32_t flags, cudaStream_t st)
{
    const int32_t W = cam->width, H = cam->height;
    const int32_t T = gs_num_tiles(W, H, c->cfg.tile_size);
    const int32_t stride = c->cfg.mode == GS_MODE_GLOBAL_SORT ? 1 : c->cfg.K;
    ProjView pv = proj_view(c->r_proj, n);
    int r = render_binning(c, n, scales, cam, flags, st);
    if (r != GS_OK) return r;
    const bool save = (flags & GS_RENDER_SAVE) != 0;
    if (save && (r = render_save_buffers(c, W, H, T)) != GS_OK) return r;
    c->r_saved = 0;
    stage_begin(c, GS_STAGE_RASTER, st);
    const bool planned = c->cfg.mode == GS_MODE_BINNED_EXACT && frame_planned(c);
    PlanView pl;
    if (planned) {
        pl.bins = c->d_plan;
        pl.flag = c->d_plan + T;
        pl.list = c->d_plist;
    }
    // per-warp ends for the backward (a planned frame's completing pass
    // resumes pixels whose stops it does not know: tile ends only)
    int32_t* wend = save && !planned ? c->r_wend : nullptr;
    r = raster_fwd(c, pv, cam, c->r_stream, c->r_off, stride, bg, d_rgb, d_alpha, d_last, nullptr,
                   baseline_raster(c->cfg), st, save ? c->r_T : nullptr, save ? c->r_tend : nullptr, pl, wend);
    stage_end(c, GS_STAGE_RASTER, st);
    if (r != GS_OK) return r;
    if (planned) {
        // the completing pass: the other bins of the flagged tiles, their long
        // segments sorted, the tiles composited on from where they stopped
        stage_begin(c, GS_STAGE_COMPLETE, st);
        r = exact_scatter_rest(c, n, cam, c->r_m_cap, c->r_m, c->r_stream, c->r_off, st);
        if (r == GS_OK) r = repair_min(c, T, c->r_m, c->r_stream, c->r_off, nullptr, kRasterSortCap + 1, st, 2);
        if (r == GS_OK)
            r = raster_listed(c, pv, cam, c->r_stream, c->r_off, stride, bg, d_rgb, d_alpha, d_last, c->d_plan,
                              c->d_plist, st, save ? c->r_T : nullptr, save ? c->r_tend : nullptr);
        stage_end(c, GS_STAGE_COMPLETE, st);
        if (r != GS_OK) return r;
    }
    if (save) {
        c->r_saved = 1;
        c->r_wend_valid = wend != nullptr;
        c->r_last = d_last;
        c->r_n = n;
        c->r_cam = *cam;
        for (int k = 0; k < 3; ++k) c->r_bg[k] = bg[k];
    }
    return GS_OK;
}

static int render_impl(gs_ctx* c, const gs_scene* sc, const gs_camera* cam, const float* bg, float* rgb,
                       float* alpha, int32_t* last, int32_t flags, void* stream)
{
    if (!c || !sc || !cam_ok(cam) || !bg || !rgb || !alpha) return GS_ERR_INVALID_ARG;
    if (sc->n < 0 || sc->n > INT32_MAX - 1 || sc->sh_degree < 0 || sc->sh_degree > 3) return GS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = sc->n;
    const int32_t W = cam->width, H = cam->height;
    const int32_t T = gs_num_tiles(W, H, c->cfg.tile_size);
    const int ncoef = (sc->sh_degree + 1) * (sc->sh_degree + 1);
    int r;
    const float *means = sc->means, *scales = sc->scales, *quats = sc->quats, *opac = sc->opacities,
                *sh = sc->sh;
    if (flags & GS_RENDER_HOST_INPUTS) {
        // one device copy of the scene, refreshed every call
        const size_t fl = (size_t)n * (3 + 3 + 4 + 1 + 3 * ncoef);
        void* p = c->r_scene;
        if ((r = ensure(&p, &c->r_scene_cap, fl * 4 + 5 * 256)) != GS_OK) return r;
        c->r_scene = (float*)p;
        char* b = (char*)p;
        const float* src[5] = {means, scales, quats, opac, sh};
        const size_t cnt[5] = {(size_t)n * 3, (size_t)n * 3, (size_t)n * 4, (size_t)n, (size_t)n * 3 * ncoef};
        const float* dst[5];
        for (int k = 0; k < 5; ++k) {
            dst[k] = (const float*)b;
            if (cnt[k]) GS_CUDA_TRY(cudaMemcpyAsync(b, src[k], cnt[k] * 4, cudaMemcpyHostToDevice, st));
            b += align256(cnt[k] * 4);
        }
        means = dst[0]; scales = dst[1]; quats = dst[2]; opac = dst[3]; sh = dst[4];
    }
    float *d_rgb = rgb, *d_alpha = alpha;
    int32_t* d_last = last;
    if ((flags & GS_RENDER_HOST_OUTPUTS) || !last) {
        const size_t px = (size_t)W * H;
        void* p = c->r_out;
        if ((r = ensure(&p, &c->r_out_cap, px * 5 * 4 + 3 * 256)) != GS_OK) return r;
        c->r_out = (float*)p;
        char* b = (char*)p;
        float* o_rgb = (float*)b; b += align256(px * 12);
        float* o_alpha = (float*)b; b += align256(px * 4);
        int32_t* o_last = (int32_t*)b;
        if (flags & GS_RENDER_HOST_OUTPUTS) { d_rgb = o_rgb; d_alpha = o_alpha; d_last = o_last; }
        else d_last = o_last;
    }
    if ((r = render_buffers(c, n, c->r_m_cap > 0 ? c->r_m_cap : 1, T)) != GS_OK) return r;
    ProjView pv = proj_view(c->r_proj, n);
    frame_zero_reset(c);
    if (n > 0) {
        // the projection and the depth-range sampling also zero what the
        // frame's later kernels count into (EXACT with the tile cull), so no
        // memset sits between kernels
        FrameZero fz;
        if (c->cfg.mode == GS_MODE_BINNED_EXACT && c->cfg.tile_cull &&
            (r = exact_frame_zero(c, n, cam, c->r_m_cap, &fz)) != GS_OK)
            return r;
        stage_begin(c, GS_STAGE_PROJECT, st);
        r = launch_project(c, means, scales, quats, opac, sh, sc->sh_degree, n, cam, pv, st, fz);
        stage_end(c, GS_STAGE_PROJECT, st);
        if (r != GS_OK) {
            frame_zero_reset(c);
            return r;
        }
    }
    r = render_after_project(c, n, scales, cam, bg, d_rgb, d_alpha, d_last, flags, st);
    frame_zero_reset(c);
    if (r != GS_OK) return r;
    if (flags & GS_RENDER_HOST_OUTPUTS) {
        const size_t px = (size_t)W * H;
        GS_CUDA_TRY(cudaMemcpyAsync(rgb, d_rgb, px * 12, cudaMemcpyDeviceToHost, st));
        GS_CUDA_TRY(cudaMemcpyAsync(alpha, d_alpha, px * 4, cudaMemcpyDeviceToHost, st));
        if (last) GS_CUDA_TRY(cudaMemcpyAsync(last, d_last, px * 4, cudaMemcpyDeviceToHost, st));
    }
    GS_CUDA_TRY(cudaMemcpyAsync(c->h_m + 1, c->r_m, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    if (flags & (GS_RENDER_HOST_INPUTS | GS_RENDER_HOST_OUTPUTS)) {
        GS_CUDA_TRY(cudaStreamSynchronize(st));
        c->last_m = c->h_m[1];
        if (c->last_m > c->r_m_cap) return GS_ERR_CAPACITY;
    } else {
        c->last_m = c->h_m[0];
    }
    return GS_OK;
}

// ------------------------------------------------------------------ pipelined host-buffer frames
static int pipe_init(gs_ctx* c)
{
    if (c->pipe_down) return GS_OK;
    cudaStream_t up = nullptr, down = nullptr;
    if (cudaStreamCreateWithFlags(&up, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&down, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        if (up) cudaStreamDestroy(up);
        return GS_ERR_CUDA;
    }
    for (auto& P : c->pipe)
        for (cudaEvent_t* e : {&P.uploaded, &P.rendered, &P.downloaded})
            if (!*e && cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                *e = nullptr;
                cudaStreamDestroy(up);
                cudaStreamDestroy(down);
                return GS_ERR_CUDA;
            }
    c->pipe_up = up;
    c->pipe_down = down;
    return GS_OK;
}

// One pipelined frame in the next slot: the scene up on the upload stream,
// the frame on `st`, the outputs down on the download stream, each step
// ordered by the slot's events after the slot's previous use.
static int render_pipelined(gs_ctx* c, const gs_scene* sc, const gs_camera* cam, const float* bg, float* rgb,
                            float* alpha, int32_t* last, int32_t flags, cudaStream_t st)
{
    const int32_t host = GS_RENDER_HOST_INPUTS | GS_RENDER_HOST_OUTPUTS;
    if (!c || !sc || !cam_ok(cam) || !bg || !rgb || !alpha) return GS_ERR_INVALID_ARG;
    if ((flags & host) != host || (flags & (GS_RENDER_SAVE | GS_RENDER_GRAPH))) return GS_ERR_INVALID_ARG;
    if (sc->n < 0 || sc->n > INT32_MAX - 1 || sc->sh_degree < 0 || sc->sh_degree > 3) return GS_ERR_INVALID_ARG;
    if (c->r_m_cap <= 1) return GS_ERR_INVALID_ARG;  // capacity must be reserved first
    int r;
    if ((r = pipe_init(c)) != GS_OK) return r;
    gs_ctx::PipeSlot& P = c->pipe[c->pipe_next];
    const int64_t n = sc->n;
    const int ncoef = (sc->sh_degree + 1) * (sc->sh_degree + 1);
    const size_t px = (size_t)cam->width * cam->height;
    const float* src[5] = {sc->means, sc->scales, sc->quats, sc->opacities, sc->sh};
    const size_t cnt[5] = {(size_t)n * 3, (size_t)n * 3, (size_t)n * 4, (size_t)n, (size_t)n * 3 * ncoef};
    size_t scene_bytes = 0;
    for (size_t k : cnt) scene_bytes += align256(k * 4);
    // a buffer that grows is freed first, and cudaFree waits for the device
    void* ps = P.scene;
    if ((r = ensure(&ps, &P.scene_cap, scene_bytes)) != GS_OK) return r;
    P.scene = (float*)ps;
    void* po = P.out;
    if ((r = ensure(&po, &P.out_cap, align256(px * 12) + align256(px * 4) + px * 4)) != GS_OK) return r;
    P.out = (float*)po;
    // up: after the frame that last read this slot's scene
    if (P.used) GS_CUDA_TRY(cudaStreamWaitEvent(c->pipe_up, P.rendered, 0));
    const float* dst[5];
    char* b = (char*)P.scene;
    for (int k = 0; k < 5; ++k) {
        dst[k] = (const float*)b;
        if (cnt[k]) GS_CUDA_TRY(cudaMemcpyAsync(b, src[k], cnt[k] * 4, cudaMemcpyHostToDevice, c->pipe_up));
        b += align256(cnt[k] * 4);
    }
    GS_CUDA_TRY(cudaEventRecord(P.uploaded, c->pipe_up));
    // the frame: after the upload, and after the download that last read
    // this slot's outputs
    GS_CUDA_TRY(cudaStreamWaitEvent(st, P.uploaded, 0));
    if (P.used) GS_CUDA_TRY(cudaStreamWaitEvent(st, P.downloaded, 0));
    P.used = true;
    c->pipe_next ^= 1;
    const gs_scene dsc = {dst[0], dst[1], dst[2], dst[3], dst[4], sc->sh_degree, n};
    char* o = (char*)P.out;
    float* d_rgb = (float*)o;
    o += align256(px * 12);
    float* d_alpha = (float*)o;
    o += align256(px * 4);
    int32_t* d_last = (int32_t*)o;
    r = render_impl(c, &dsc, cam, bg, d_rgb, d_alpha, d_last,
                    (flags & ~(host | GS_RENDER_PIPELINE)) | GS_RENDER_NO_SYNC, st);
    // recorded whatever the frame did, so the slot's next use never waits on
    // an event that was not recorded after this one's
    GS_CUDA_TRY(cudaEventRecord(P.rendered, st));
    if (r != GS_OK) {
        GS_CUDA_TRY(cudaEventRecord(P.downloaded, c->pipe_down));
        return r;
    }
    // down: after the frame
    GS_CUDA_TRY(cudaStreamWaitEvent(c->pipe_down, P.rendered, 0));
    GS_CUDA_TRY(cudaMemcpyAsync(rgb, d_rgb, px * 12, cudaMemcpyDeviceToHost, c->pipe_down));
    GS_CUDA_TRY(cudaMemcpyAsync(alpha, d_alpha, px * 4, cudaMemcpyDeviceToHost, c->pipe_down));
    if (last) GS_CUDA_TRY(cudaMemcpyAsync(last, d_last, px * 4, cudaMemcpyDeviceToHost, c->pipe_down));
    GS_CUDA_TRY(cudaEventRecord(P.downloaded, c->pipe_down));
    return GS_OK;
}

extern "C" int gs_render_wait(gs_ctx* c)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (!c->pipe_down) return GS_OK;
    const cudaError_t a = cudaStreamSynchronize(c->pipe_up);
    const cudaError_t d = cudaStreamSynchronize(c->pipe_down);
    if (a != cudaSuccess || d != cudaSuccess) {
        cudaGetLastError();
        return GS_ERR_CUDA;
    }
    return GS_OK;
}

// The frame as a CUDA graph: captured on first use (and whenever any pointer,
// size, camera, background or configuration value changes), replayed after.
extern "C" int gs_render(gs_ctx* c, const gs_scene* sc, const gs_camera* cam, const float* bg, float* rgb,
                         float* alpha, int32_t* last, int32_t flags, void* stream)
{
    if (flags & GS_RENDER_PIPELINE)
        return render_pipelined(c, sc, cam, bg, rgb, alpha, last, flags, (cudaStream_t)stream);
    if (!(flags & GS_RENDER_GRAPH)) return render_impl(c, sc, cam, bg, rgb, alpha, last, flags, stream);
    if (!c || !sc || !cam || !bg || !rgb || !alpha) return GS_ERR_INVALID_ARG;
    if (flags & (GS_RENDER_HOST_INPUTS | GS_RENDER_HOST_OUTPUTS)) return GS_ERR_INVALID_ARG;
    if (c->r_m_cap <= 1) return GS_ERR_INVALID_ARG;  // capacity must be reserved first
    if (!stream) return GS_ERR_INVALID_ARG;          // the legacy stream cannot be captured
    cudaStream_t st = (cudaStream_t)stream;
    struct Key {
        gs_scene sc;
        gs_camera cam;
        float bg[3];
        void *rgb, *alpha, *last, *proj, *isect, *stream, *off, *scene_copy, *out, *saved_T, *saved_end, *saved_wend;
        int64_t m_cap;
        gs_config cfg;
        int timing, device, flags;
        // the internal scratch the captured kernels address (a grown buffer
        // is a new allocation: the graph is captured again)
        const void* scratch[14];
        size_t scratch_bytes[10];
    } key;
    if (flags & GS_RENDER_SAVE) {
        // allocate outside the capture
        int rs = render_save_buffers(c, cam->width, cam->height, gs_num_tiles(cam->width, cam->height,
                                                                              c->cfg.tile_size));
        if (rs != GS_OK) return rs;
    }
    memset(&key, 0, sizeof(key));
    key.sc = *sc;
    key.cam = *cam;
    for (int k = 0; k < 3; ++k) key.bg[k] = bg[k];
    key.rgb = rgb;
    key.alpha = alpha;
    key.last = last;
    key.proj = c->r_proj;
    key.isect = c->r_isect;
    key.stream = c->r_stream;
    key.off = c->r_off;
    key.scene_copy = c->r_scene;
    key.out = c->r_out;
    key.m_cap = c->r_m_cap;
    key.cfg = c->cfg;
    key.timing = c->timing;
    key.device = c->device;
    key.flags = flags;
    key.saved_T = c->r_T;
    key.saved_end = c->r_tend;
    key.saved_wend = c->r_wend;
    const void* scratch[] = {c->d_scan, c->d_goff, c->d_keys[0], c->d_keys[1], c->d_vals[0], c->d_vals[1],
                             c->d_hist, c->d_count, c->d_bin, c->d_sel, c->d_tail, c->d_tiles, c->d_samples,
                             c->d_plan};
    const size_t scratch_bytes[] = {c->scan_bytes, c->goff_cap, c->sort_cap, c->hist_cap, c->count_cap,
                                    c->bin_cap, c->sel_cap, c->tail_cap, c->tiles_cap, c->samples_cap};
    static_assert(sizeof(scratch) == sizeof(key.scratch) && sizeof(scratch_bytes) == sizeof(key.scratch_bytes),
                  "graph key scratch");
    memcpy(key.scratch, scratch, sizeof(scratch));
    memcpy(key.scratch_bytes, scratch_bytes, sizeof(scratch_bytes));
    static_assert(sizeof(Key) <= sizeof(c->gkey), "graph key");
    if (!(c->gexec && c->gkey_len == sizeof(Key) && memcmp(c->gkey, &key, sizeof(Key)) == 0)) {
        if (c->gexec) {
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
        }
        const int64_t l0 = c->launches;
        cudaGraph_t graph = nullptr;
        GS_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        c->capturing = 1;
        int r = render_impl(c, sc, cam, bg, rgb, alpha, last, flags | GS_RENDER_NO_SYNC, stream);
        c->capturing = 0;
        cudaError_t e = cudaStreamEndCapture(st, &graph);
        if (r != GS_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return r != GS_OK ? r : gs_cuda_fail(e, "cudaStreamEndCapture");
        }
        e = cudaGraphInstantiate(&c->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            c->gexec = nullptr;
            return gs_cuda_fail(e, "cudaGraphInstantiate");
        }
        c->glaunches = c->launches - l0;
        c->launches = l0;
        c->g_last = c->r_last;  // the last-id buffer the captured frame writes
        c->g_wend_valid = c->r_wend_valid;
        memcpy(c->gkey, &key, sizeof(Key));
        c->gkey_len = sizeof(Key);
    }
    GS_CUDA_TRY(cudaGraphLaunch(c->gexec, st));
    c->launches += c->glaunches;
    c->r_saved = 0;
    if (flags & GS_RENDER_SAVE) {
        // the replayed frame is the captured one: its saved state is current
        c->r_saved = 1;
        c->r_wend_valid = c->g_wend_valid;
        c->r_last = c->g_last;
        c->r_n = sc->n;
        c->r_cam = *cam;
        for (int k = 0; k < 3; ++k) c->r_bg[k] = bg[k];
    }
    return GS_OK;
}

extern "C" int gs_render_bwd(gs_ctx* c, const float* dl_drgb, const float* dl_dalpha, void* grad, void* stream)
{
    if (!c || !dl_drgb || !grad) return GS_ERR_INVALID_ARG;
    if (!c->r_saved || !c->r_last) return GS_ERR_INVALID_ARG;  // no saved gs_render on this context
    if ((reinterpret_cast<uintptr_t>(grad) & 255u) != 0) return GS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = c->r_n;
    GS_CUDA_TRY(cudaMemsetAsync(grad, 0, gs_grad2d_bytes(n), st));
    if (n == 0) return GS_OK;
    const int32_t stride = c->cfg.mode == GS_MODE_GLOBAL_SORT ? 1 : c->cfg.K;
    return raster_bwd(c, proj_view(c->r_proj, n), &c->r_cam, c->r_stream, c->r_off, stride, c->r_bg, c->r_last,
                      c->r_T, c->r_tend, dl_drgb, dl_dalpha, grad_view(grad, n), st,
                      c->r_wend_valid ? c->r_wend : nullptr);
}
