// batch.cu -- K24: several views of one scene in one call.  The paper renders
// single views only; a training or serving system renders many.  GB300 design:
//   * one projection launch for all views: each Gaussian's parameters and SH
//     coefficients are read from HBM once and projected for every view
//     (k_project_batch);
//   * the views that are EXACT with the repair in the raster, 16x16 tiles, the
//     tile cull and no planner form one group binned as a single frame of
//     V n items (batch_bins.cu): one launch per stage for all of them, on the
//     caller's stream, then one persistent raster launch composites all their
//     tiles (blocks take (view, tile) items from a counter, longest first);
//   * every other view runs the whole-frame pipeline on its own stream,
//     forked from and joined back into the caller's stream;
//   * with GS_RENDER_GRAPH the whole batch (fork, V pipelines, join) is one
//     CUDA graph, replayed while the arguments stay the same;
//   * per-view tile size and bin count come from gs_batch_autotune, which
//     times the candidates on the view itself.
// Every view has its own sub-context (scratch, stream, error word), created
// on first use with the parent's configuration or the one set for the view.
#include <string.h>

#include <vector>

#include "internal.cuh"

namespace gs {

struct BatchState {
    gs_ctx* views[kMaxBatchViews] = {};
    cudaStream_t streams[kMaxBatchViews] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kMaxBatchViews] = {};
    gs_config vcfg[kMaxBatchViews];
    int has_cfg[kMaxBatchViews] = {};
    cudaGraphExec_t gexec = nullptr;
    std::vector<unsigned char> gkey;
    int64_t glaunches = 0;
    int32_t* d_counter = nullptr;  // schedule of the persistent multi-view raster (65 int32)
    int32_t* d_order = nullptr;    // its work items, longest tiles first
    size_t order_cap = 0;
    // the group of views binned together (batch_bins.cu)
    gs_ctx* group = nullptr;                  // its scratch, stream and offsets, error word
    GroupViews* gview = nullptr;              // its view table
    int64_t* h_group_m = nullptr;             // pinned: per-view entry counts of the last batch
    int group_pos[kMaxBatchViews];            // position of view v in the group, -1: not in it
    int ngroup = 0;
};

void batch_destroy(gs_ctx* c)
{
    BatchState* b = c->batch;
    if (!b) return;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    for (int v = 0; v < kMaxBatchViews; ++v) {
        if (b->views[v]) gs_destroy(b->views[v]);
        if (b->streams[v]) cudaStreamDestroy(b->streams[v]);
        if (b->join[v]) cudaEventDestroy(b->join[v]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->d_counter) cudaFree(b->d_counter);
    if (b->d_order) cudaFree(b->d_order);
    if (b->group) gs_destroy(b->group);
    if (b->gview) group_views_free(b->gview);
    if (b->h_group_m) cudaFreeHost(b->h_group_m);
    delete b;
    c->batch = nullptr;
}

int batch_error(gs_ctx* c, cudaStream_t st)
{
    if (!c->batch) return GS_OK;
    if (c->batch->group) {
        const int e = gs_get_error(c->batch->group, st);
        if (e != GS_OK) return e;
    }
    for (int v = 0; v < kMaxBatchViews; ++v)
        if (c->batch->views[v]) {
            const int e = gs_get_error(c->batch->views[v], st);
            if (e != GS_OK) return e;
        }
    return GS_OK;
}

int batch_clear_error(gs_ctx* c, cudaStream_t st)
{
    if (!c->batch) return GS_OK;
    if (c->batch->group) {
        const int e = gs_clear_error(c->batch->group, st);
        if (e != GS_OK) return e;
    }
    for (int v = 0; v < kMaxBatchViews; ++v)
        if (c->batch->views[v]) {
            const int e = gs_clear_error(c->batch->views[v], st);
            if (e != GS_OK) return e;
        }
    return GS_OK;
}

static BatchState* batch_state(gs_ctx* c)
{
    if (!c->batch) {
        BatchState* b = new BatchState();
        if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaMalloc(&b->d_counter, 65 * sizeof(int32_t)) != cudaSuccess ||
            cudaMallocHost(&b->h_group_m, kMaxBatchViews * sizeof(int64_t)) != cudaSuccess ||
            !(b->gview = group_views_new())) {
            if (b->fork) cudaEventDestroy(b->fork);
            if (b->d_counter) cudaFree(b->d_counter);
            if (b->h_group_m) cudaFreeHost(b->h_group_m);
            delete b;
            return nullptr;
        }
        for (int v = 0; v < kMaxBatchViews; ++v) b->group_pos[v] = -1;
        c->batch = b;
    }
    return c->batch;
}

// The view's configuration: the one set for it, else the parent's.
static const gs_config& view_config(gs_ctx* c, int v)
{
    BatchState* b = c->batch;
    return b->has_cfg[v] ? b->vcfg[v] : c->cfg;
}

// Sub-context, stream and join event of view v, with the view's configuration.
static int view_ctx(gs_ctx* c, int v, gs_ctx** out)
{
    BatchState* b = batch_state(c);
    if (!b) return GS_ERR_NO_MEMORY;
    const gs_config& cfg = view_config(c, v);
    if (!b->views[v]) {
        int r = gs_create(&b->views[v], &cfg);
        if (r != GS_OK) return r;
        if (cudaStreamCreateWithFlags(&b->streams[v], cudaStreamNonBlocking) != cudaSuccess) return GS_ERR_CUDA;
        if (cudaEventCreateWithFlags(&b->join[v], cudaEventDisableTiming) != cudaSuccess) return GS_ERR_CUDA;
    } else if (memcmp(&b->views[v]->cfg, &cfg, sizeof(gs_config)) != 0) {
        int r = gs_set_config(b->views[v], &cfg);
        if (r != GS_OK) return r;
    }
    *out = b->views[v];
    return GS_OK;
}

int64_t batch_launch_count(const gs_ctx* c)
{
    int64_t s = 0;
    if (c->batch) {
        for (int v = 0; v < kMaxBatchViews; ++v)
            if (c->batch->views[v]) s += c->batch->views[v]->launches;
        if (c->batch->group) s += c->batch->group->launches;
    }
    return s;
}

// Whether two view configurations may share a group: every field but the
// bin count.
static bool same_but_k(gs_config a, gs_config b)
{
    a.K = b.K = 0;
    return memcmp(&a, &b, sizeof(gs_config)) == 0;
}

static bool groupable(const gs_config& cfg)
{
    return cfg.mode == GS_MODE_BINNED_EXACT && cfg.repair_in_raster && cfg.tile_size == 16 && cfg.tile_cull &&
           !cfg.planner;
}

// The group: the groupable views whose configuration equals (but for K) the
// first groupable view's; its context carries that configuration.
static int batch_group(gs_ctx* c, const gs_scene* sc, const gs_camera* cams, int nv)
{
    BatchState* b = c->batch;
    gs_camera gcams[kMaxBatchViews];
    int32_t gk[kMaxBatchViews];
    int first = -1;
    b->ngroup = 0;
    for (int v = 0; v < kMaxBatchViews; ++v) b->group_pos[v] = -1;
    for (int v = 0; v < nv; ++v) {
        const gs_config& cfg = view_config(c, v);
        if (!groupable(cfg)) continue;
        if (first < 0) first = v;
        else if (!same_but_k(cfg, view_config(c, first))) continue;
        b->group_pos[v] = b->ngroup;
        gcams[b->ngroup] = cams[v];
        gk[b->ngroup] = cfg.K;
        ++b->ngroup;
    }
    if (b->ngroup == 0) return GS_OK;
    const gs_config& gcfg = view_config(c, first);
    int r;
    if (!b->group) {
        if ((r = gs_create(&b->group, &gcfg)) != GS_OK) return r;
    } else if (memcmp(&b->group->cfg, &gcfg, sizeof(gs_config)) != 0 && (r = gs_set_config(b->group, &gcfg)) != GS_OK) {
        return r;
    }
    group_views_set(b->gview, sc->n, b->ngroup, gcams, gk);
    return group_reserve(b->group, b->gview, b->group->r_m_cap > 0 ? b->group->r_m_cap : 1);
}

// Device buffers of every view, allocated outside any capture.
static int batch_buffers(gs_ctx* c, const gs_scene* sc, const gs_camera* cams, int nv, int32_t* const* last,
                         int32_t flags)
{
    {
        BatchState* b = batch_state(c);
        if (!b) return GS_ERR_NO_MEMORY;
        size_t tiles = 0;
        for (int v = 0; v < nv; ++v) tiles += (size_t)gs_num_tiles(cams[v].width, cams[v].height, 16);
        void* p = b->d_order;
        const int r = ensure(&p, &b->order_cap, tiles * sizeof(int32_t) + 256);
        if (r != GS_OK) return r;
        b->d_order = (int32_t*)p;
    }
    for (int v = 0; v < nv; ++v) {
        gs_ctx* vc;
        int r = view_ctx(c, v, &vc);
        if (r != GS_OK) return r;
    }
    {
        const int r = batch_group(c, sc, cams, nv);
        if (r != GS_OK) return r;
    }
    for (int v = 0; v < nv; ++v) {
        gs_ctx* vc = c->batch->views[v];
        int r;
        const int32_t T = gs_num_tiles(cams[v].width, cams[v].height, vc->cfg.tile_size);
        if (c->batch->group_pos[v] < 0 && (r = render_buffers(vc, sc->n, vc->r_m_cap > 0 ? vc->r_m_cap : 1, T)) != GS_OK)
            return r;
        if (!last || !last[v]) {
            const size_t px = (size_t)cams[v].width * cams[v].height;
            void* p = vc->r_out;
            if ((r = ensure(&p, &vc->r_out_cap, px * 4 + 256)) != GS_OK) return r;
            vc->r_out = (float*)p;
        }
        if ((flags & GS_RENDER_SAVE) &&
            (r = render_save_buffers(vc, cams[v].width, cams[v].height, T)) != GS_OK)
            return r;
    }
    return GS_OK;
}

static int batch_impl(gs_ctx* c, const gs_scene* sc, const gs_camera* cams, int nv, const float* bg,
                      float* const* rgb, float* const* alpha, int32_t* const* last, int32_t flags, cudaStream_t st)
{
    BatchState* b = c->batch;
    const int64_t n = sc->n;
    int r;
    gs_ctx* gc = b->group;
    const ProjView big = b->ngroup > 0 ? proj_view(gc->r_proj, n * b->ngroup) : ProjView();
    // one projection launch for all views, on the caller's stream: a group
    // view's records at items [p n, (p+1) n) of the group's buffer
    {
        ProjView pvs[kMaxBatchViews];
        int tiles[kMaxBatchViews];
        for (int v = 0; v < nv; ++v) {
            const int p = b->group_pos[v];
            if (p >= 0) {
                ProjView x = big;
                x.xy_ab += p * n;
                x.c_o_z += p * n;
                x.rgb += p * n;
                x.rect += p * n;
                x.radius += p * n;
                pvs[v] = x;
            } else {
                pvs[v] = proj_view(b->views[v]->r_proj, n);
            }
            tiles[v] = b->views[v]->cfg.tile_size;
        }
        r = launch_project_batch(c, sc->means, sc->scales, sc->quats, sc->opacities, sc->sh, sc->sh_degree, n, nv,
                                 cams, tiles, pvs, st);
        if (r != GS_OK) return r;
    }
    // the views outside the group: the whole-frame pipeline on their streams
    GS_CUDA_TRY(cudaEventRecord(b->fork, st));
    bool forked[kMaxBatchViews] = {};
    for (int v = 0; v < nv; ++v) {
        if (b->group_pos[v] >= 0) continue;
        gs_ctx* vc = b->views[v];
        cudaStream_t vs = b->streams[v];
        GS_CUDA_TRY(cudaStreamWaitEvent(vs, b->fork, 0));
        vc->capturing = c->capturing;
        int32_t* d_last = (last && last[v]) ? last[v] : reinterpret_cast<int32_t*>(vc->r_out);
        r = render_after_project(vc, n, sc->scales, cams + v, bg, rgb[v], alpha[v], d_last, flags, vs);
        vc->capturing = 0;
        if (r != GS_OK) return r;
        GS_CUDA_TRY(cudaMemcpyAsync(vc->h_m + 1, vc->r_m, sizeof(int64_t), cudaMemcpyDeviceToHost, vs));
        GS_CUDA_TRY(cudaEventRecord(b->join[v], vs));
        forked[v] = true;
    }
    // the group: its binning as one frame on the caller's stream, then one
    // persistent raster launch over all its views' tiles
    if (b->ngroup > 0) {
        gc->capturing = c->capturing;
        r = group_binning(gc, b->gview, flags, b->h_group_m, st);
        gc->capturing = 0;
        if (r != GS_OK) return r;
        RasterView rv[kMaxBatchViews];
        int k = 0;
        for (int v = 0; v < nv; ++v) {
            const int p = b->group_pos[v];
            if (p < 0) continue;
            RasterView& x = rv[k++];
            x.pv = big;
            x.cam = cams[v];
            x.words = gc->r_stream;
            x.offsets = gc->r_off + group_seg_base(b->gview, p);
            x.stride = b->views[v]->cfg.K;
            for (int q = 0; q < 3; ++q) x.bg[q] = bg[q];
            x.cull = gc->cfg.tile_cull;
            x.cap = chunk_cap(gc->cfg);
            x.rgb = rgb[v];
            x.alpha = alpha[v];
            x.last = (last && last[v]) ? last[v] : reinterpret_cast<int32_t*>(b->views[v]->r_out);
            x.gid_base = (int32_t)(p * n);
        }
        if ((r = raster_views(c, rv, k, b->d_counter, b->d_order, st)) != GS_OK) return r;
    }
    for (int v = 0; v < nv; ++v)
        if (forked[v]) GS_CUDA_TRY(cudaStreamWaitEvent(st, b->join[v], 0));
    return GS_OK;
}

static int batch_args_ok(gs_ctx* c, const gs_scene* sc, const gs_camera* cams, int32_t nv, const float* bg,
                         float* const* rgb, float* const* alpha)
{
    if (!c || !sc || !cams || !bg || !rgb || !alpha || nv < 1 || nv > kMaxBatchViews) return 0;
    if (sc->n < 0 || sc->n > INT32_MAX - 1 || sc->sh_degree < 0 || sc->sh_degree > 3) return 0;
    if (sc->n > 0 && (!sc->means || !sc->scales || !sc->quats || !sc->opacities || !sc->sh)) return 0;
    for (int v = 0; v < nv; ++v)
        if (!camera_ok(cams + v) || !rgb[v] || !alpha[v]) return 0;
    return 1;
}

}  // namespace gs

using namespace gs;

extern "C" int gs_batch_set_view_config(gs_ctx* c, int32_t view, const gs_config* cfg)
{
    if (!c || view < 0 || view >= kMaxBatchViews) return GS_ERR_INVALID_ARG;
    BatchState* b = batch_state(c);
    if (!b) return GS_ERR_NO_MEMORY;
    if (!cfg) {
        b->has_cfg[view] = 0;
        return GS_OK;
    }
    if (check_config(cfg) != GS_OK) return GS_ERR_INVALID_ARG;
    b->vcfg[view] = *cfg;
    b->has_cfg[view] = 1;
    return GS_OK;
}

extern "C" int gs_batch_get_view_config(gs_ctx* c, int32_t view, gs_config* cfg)
{
    if (!c || !cfg || view < 0 || view >= kMaxBatchViews) return GS_ERR_INVALID_ARG;
    *cfg = (c->batch && c->batch->has_cfg[view]) ? c->batch->vcfg[view] : c->cfg;
    return GS_OK;
}

extern "C" int64_t gs_batch_last_entry_count(gs_ctx* c, int32_t view)
{
    if (!c || !c->batch || view < 0 || view >= kMaxBatchViews || !c->batch->views[view]) return -1;
    if (c->batch->group_pos[view] >= 0) return c->batch->h_group_m[c->batch->group_pos[view]];
    return c->batch->views[view]->h_m[1];
}

extern "C" int gs_render_batch(gs_ctx* c, const gs_scene* sc, const gs_camera* cams, int32_t n_cams,
                               const float* bg, float* const* rgb, float* const* alpha, int32_t* const* last,
                               int32_t flags, void* stream)
{
    if (!batch_args_ok(c, sc, cams, n_cams, bg, rgb, alpha)) return GS_ERR_INVALID_ARG;
    if (flags & (GS_RENDER_HOST_INPUTS | GS_RENDER_HOST_OUTPUTS | GS_RENDER_SAVE | GS_RENDER_PIPELINE))
        return GS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int r = batch_buffers(c, sc, cams, n_cams, last, flags);
    if (r != GS_OK) return r;
    BatchState* b = c->batch;
    const int64_t l0 = c->launches + batch_launch_count(c);
    if (!(flags & GS_RENDER_GRAPH)) {
        r = batch_impl(c, sc, cams, n_cams, bg, rgb, alpha, last, flags, st);
        if (r != GS_OK) return r;
        if (!(flags & GS_RENDER_NO_SYNC)) GS_CUDA_TRY(cudaStreamSynchronize(st));
        return GS_OK;
    }
    // graph: capacity must have been sized by an earlier call without NO_SYNC
    if (!stream) return GS_ERR_INVALID_ARG;
    for (int v = 0; v < n_cams; ++v)
        if (b->group_pos[v] < 0 && b->views[v]->r_m_cap <= 1) return GS_ERR_INVALID_ARG;
    if (b->ngroup > 0 && b->group->r_m_cap <= 1) return GS_ERR_INVALID_ARG;
    std::vector<unsigned char> key;
    auto put = [&key](const void* p, size_t nbytes) {
        const unsigned char* q = static_cast<const unsigned char*>(p);
        key.insert(key.end(), q, q + nbytes);
    };
    put(sc, sizeof(gs_scene));
    put(&n_cams, sizeof(n_cams));
    put(cams, sizeof(gs_camera) * (size_t)n_cams);
    put(bg, 3 * sizeof(float));
    put(rgb, sizeof(float*) * (size_t)n_cams);
    put(alpha, sizeof(float*) * (size_t)n_cams);
    for (int v = 0; v < n_cams; ++v) {
        const void* lp = (last && last[v]) ? (const void*)last[v] : (const void*)b->views[v]->r_out;
        gs_ctx* vc = b->views[v];
        const void* ptrs[] = {lp, vc->r_proj, vc->r_isect, vc->r_stream, vc->r_off};
        put(ptrs, sizeof(ptrs));
        put(&vc->r_m_cap, sizeof(vc->r_m_cap));
        put(&vc->cfg, sizeof(gs_config));
    }
    if (b->group) {
        const gs_ctx* gc = b->group;
        const void* gptr[] = {gc->r_proj, gc->r_stream, gc->r_off, gc->d_tiles, gc->d_goff, gc->d_scan, gc->d_tail};
        put(gptr, sizeof(gptr));
        put(&gc->r_m_cap, sizeof(gc->r_m_cap));
        put(b->group_pos, sizeof(b->group_pos));
    }
    put(&flags, sizeof(flags));
    put(&c->device, sizeof(c->device));
    put(&b->d_order, sizeof(b->d_order));
    if (!(b->gexec && b->gkey == key)) {
        if (b->gexec) {
            cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        GS_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        c->capturing = 1;
        r = batch_impl(c, sc, cams, n_cams, bg, rgb, alpha, last, flags | GS_RENDER_NO_SYNC, st);
        c->capturing = 0;
        cudaError_t e = cudaStreamEndCapture(st, &graph);
        if (r != GS_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return r != GS_OK ? r : gs_cuda_fail(e, "cudaStreamEndCapture");
        }
        e = cudaGraphInstantiate(&b->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->gexec = nullptr;
            return gs_cuda_fail(e, "cudaGraphInstantiate");
        }
        b->glaunches = c->launches + batch_launch_count(c) - l0;
        b->gkey = key;
    } else {
        c->launches += b->glaunches;
    }
    GS_CUDA_TRY(cudaGraphLaunch(b->gexec, st));
    return GS_OK;
}

// Mean time of `iters` batches of the views with configurations cfgs (after
// one sizing batch and one warm batch), for the autotuner; outputs go to
// temporary buffers.
static int time_batch(gs_ctx* c, const gs_scene* sc, const gs_camera* cams, int nv, const gs_config* cfgs, int iters,
                      cudaEvent_t e0, cudaEvent_t e1, cudaStream_t st, float* ms_out)
{
    const float zero_bg[3] = {0.0f, 0.0f, 0.0f};
    float* rgb[kMaxBatchViews] = {};
    float* alpha[kMaxBatchViews] = {};
    int status = GS_OK;
    for (int v = 0; v < nv && status == GS_OK; ++v) {
        const size_t px = (size_t)cams[v].width * cams[v].height;
        if (cudaMalloc(&rgb[v], px * 12) != cudaSuccess || cudaMalloc(&alpha[v], px * 4) != cudaSuccess)
            status = GS_ERR_NO_MEMORY;
        if (status == GS_OK) status = gs_batch_set_view_config(c, v, &cfgs[v]);
    }
    if (status == GS_OK) status = gs_render_batch(c, sc, cams, nv, zero_bg, rgb, alpha, nullptr, 0, st);
    if (status == GS_OK)
        status = gs_render_batch(c, sc, cams, nv, zero_bg, rgb, alpha, nullptr, GS_RENDER_NO_SYNC, st);
    if (status == GS_OK && cudaEventRecord(e0, st) != cudaSuccess) status = GS_ERR_CUDA;
    for (int i = 0; i < iters && status == GS_OK; ++i)
        status = gs_render_batch(c, sc, cams, nv, zero_bg, rgb, alpha, nullptr, GS_RENDER_NO_SYNC, st);
    float ms = 0.0f;
    if (status == GS_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        status = GS_ERR_CUDA;
    if (status == GS_OK && gs_get_error(c, st) != GS_OK) status = GS_ERR_CAPACITY;
    for (int v = 0; v < nv; ++v) {
        if (rgb[v]) cudaFree(rgb[v]);
        if (alpha[v]) cudaFree(alpha[v]);
    }
    *ms_out = ms / (float)iters;
    return status;
}

extern "C" int gs_batch_autotune(gs_ctx* c, const gs_scene* sc, const gs_camera* cams, int32_t n_cams,
                                 int32_t tune_tile, int32_t iters, float* best_ms, void* stream)
{
    if (!c || !sc || !cams || n_cams < 1 || n_cams > kMaxBatchViews || iters < 1) return GS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const float zero_bg[3] = {0.0f, 0.0f, 0.0f};
    static const int tiles_all[3] = {16, 8, 32};
    static const int ks[3] = {64, 32, 128};
    const int ntile = tune_tile ? 3 : 1;
    const int nk = c->cfg.mode == GS_MODE_GLOBAL_SORT ? 1 : 3;
    gs_config choice[kMaxBatchViews], choice16[kMaxBatchViews];
    float t16[kMaxBatchViews];
    cudaEvent_t e0, e1;
    GS_CUDA_TRY(cudaEventCreate(&e0));
    GS_CUDA_TRY(cudaEventCreate(&e1));
    int status = GS_OK;
    for (int v = 0; v < n_cams && status == GS_OK; ++v) {
        const size_t px = (size_t)cams[v].width * cams[v].height;
        float *d_rgb = nullptr, *d_alpha = nullptr;
        int32_t* d_last = nullptr;
        if (cudaMalloc(&d_rgb, px * 12) != cudaSuccess || cudaMalloc(&d_alpha, px * 4) != cudaSuccess ||
            cudaMalloc(&d_last, px * 4) != cudaSuccess) {
            status = GS_ERR_NO_MEMORY;
        }
        gs_config best = c->cfg;
        float best_t = 3.4e38f;
        const gs_config base = (c->batch && c->batch->has_cfg[v]) ? c->batch->vcfg[v] : c->cfg;
        // the best candidate that keeps 16 x 16 tiles (the views binned as one group)
        gs_config best16 = base;
        float best16_t = 3.4e38f;
        for (int it = 0; it < ntile && status == GS_OK; ++it)
            for (int ik = 0; ik < nk && status == GS_OK; ++ik) {
                gs_config cfg = base;
                if (tune_tile) cfg.tile_size = tiles_all[it];
                if (nk > 1) cfg.K = ks[ik];
                gs_ctx* t = nullptr;
                if ((status = gs_create(&t, &cfg)) != GS_OK) break;
                // one sizing frame, one warm frame, then the timed ones
                status = gs_render(t, sc, cams + v, zero_bg, d_rgb, d_alpha, d_last, 0, st);
                if (status == GS_OK)
                    status = gs_render(t, sc, cams + v, zero_bg, d_rgb, d_alpha, d_last,
                                       GS_RENDER_NO_SYNC, st);
                if (status == GS_OK && cudaEventRecord(e0, st) != cudaSuccess) status = GS_ERR_CUDA;
                for (int i = 0; i < iters && status == GS_OK; ++i)
                    status = gs_render(t, sc, cams + v, zero_bg, d_rgb, d_alpha, d_last,
                                       GS_RENDER_NO_SYNC, st);
                float ms = 0.0f;
                if (status == GS_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                                        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                    status = GS_ERR_CUDA;
                if (status == GS_OK && gs_get_error(t, st) != GS_OK) status = GS_ERR_CAPACITY;
                gs_destroy(t);
                if (status == GS_OK && ms / iters < best_t) {
                    best_t = ms / iters;
                    best = cfg;
                }
                if (status == GS_OK && cfg.tile_size == 16 && ms / iters < best16_t) {
                    best16_t = ms / iters;
                    best16 = cfg;
                }
            }
        if (d_rgb) cudaFree(d_rgb);
        if (d_alpha) cudaFree(d_alpha);
        if (d_last) cudaFree(d_last);
        if (status == GS_OK) {
            status = gs_batch_set_view_config(c, v, &best);
            if (best_ms) best_ms[v] = best_t;
            choice[v] = best;
            choice16[v] = best16.tile_size == 16 && best16_t < 3.4e38f ? best16 : best;
            t16[v] = best16_t < 3.4e38f ? best16_t : best_t;
        }
    }
    // a view whose fastest tile size is not 16 leaves the group of views
    // binned and rasterised together; whether that pays is a property of the
    // batch, so the two assignments are timed as whole batches
    bool differ = false;
    for (int v = 0; v < n_cams && status == GS_OK; ++v)
        differ = differ || memcmp(&choice[v], &choice16[v], sizeof(gs_config)) != 0;
    if (status == GS_OK && tune_tile && differ) {
        float ms_a = 0.0f, ms_b = 0.0f;
        status = time_batch(c, sc, cams, n_cams, choice, iters, e0, e1, st, &ms_a);
        if (status == GS_OK) status = time_batch(c, sc, cams, n_cams, choice16, iters, e0, e1, st, &ms_b);
        if (status == GS_OK && ms_b < ms_a)
            for (int v = 0; v < n_cams && status == GS_OK; ++v) {
                status = gs_batch_set_view_config(c, v, &choice16[v]);
                if (best_ms) best_ms[v] = t16[v];
            }
        else if (status == GS_OK)
            for (int v = 0; v < n_cams && status == GS_OK; ++v) status = gs_batch_set_view_config(c, v, &choice[v]);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return status;
}
