// batch_bins.cu -- the EXACT binning of several views of one scene in one
// launch per stage (the batched render of gs_render_batch; the paper renders
// single views only).
//
// The views that can share it (EXACT, repair in the raster, 16x16 tiles, the
// tile cull, no planner) form one group: their projected records sit side by
// side in one buffer, so Gaussian g of view v is item G = v n + g of a single
// frame of V n items, and their tiles and (tile, bin) segments are
// concatenated.  Every stage then runs once over all views:
//   counts and row counts of every item, one scan     (as a single frame)
//   per-view entry counts, samples and depth range    (Alg. 2, a block a view)
//   row spans, per-row difference counts per view     (Alg. 3's histogram)
//   per-view layer prefixes, transposition, one scan  (bin offsets)
//   the scatter of every view's row records           (one cursor per segment)
//   the eager sort of segments over 2048 entries
// and the persistent multi-view raster composites every view's tiles from
// the group's stream, view v's offsets starting at its first segment.  Stream
// words carry G, so the raster gathers from the shared records; the last-id
// output subtracts the view's first item (v n).
#include <string.h>

#include "depth_range.cuh"
#include "rows.cuh"
#include "scan.cuh"

namespace gs {

// Per-view geometry of a group (a kernel parameter).
struct GroupViews {
    int nv;
    int64_t n;                                  // Gaussians per view
    int32_t K[kMaxBatchViews];                  // bins per tile
    int32_t tiles_x[kMaxBatchViews], tiles_y[kMaxBatchViews];
    int32_t tile_base[kMaxBatchViews + 1];      // first tile of view v in the group
    int64_t seg_base[kMaxBatchViews + 1];       // first (tile, bin) segment of view v
    int32_t row_base[kMaxBatchViews + 1];       // first tile row of view v
    int32_t layer_base[kMaxBatchViews + 1];     // first bin layer of view v
    int64_t d_base[kMaxBatchViews + 1];         // first difference count of view v (K layers of ty x (tx + 1))
    float near_plane[kMaxBatchViews], far_plane[kMaxBatchViews];
    __device__ __forceinline__ int view_of(int64_t G) const { return (int)((uint32_t)G / (uint32_t)n); }
};

// Entries of each view: view v owns the entries [base, base + M) of the
// group, and takes S' = min(S, M) depth samples of them.
struct ViewCount {
    int64_t base, M, ns;
};

__global__ void k_group_counts(const int32_t* __restrict__ goff, int64_t n, int nv, int S,
                               ViewCount* __restrict__ vc, int64_t* __restrict__ m_out)
{
    const int v = threadIdx.x;
    if (v >= nv) return;
    const int64_t b = goff[(int64_t)v * n], e = goff[(int64_t)(v + 1) * n];
    ViewCount c;
    c.base = b;
    c.M = e - b;
    c.ns = c.M < (int64_t)S ? c.M : (int64_t)S;
    vc[v] = c;
    m_out[v] = c.M;
}

// Sample i of view v's S' is its entry j = floor(i M / S') (Alg. 2's
// sampling, as for a single frame); its item is the G of the view with
// goff[G] - base <= j < goff[G + 1] - base, found by binary search over the
// view's items (one thread per sample, grid.y = the view).
__global__ void __launch_bounds__(256)
k_group_sample_gids(const int32_t* __restrict__ goff, const GroupViews gv, const ViewCount* __restrict__ vc, int S,
                    uint32_t* __restrict__ out)
{
    const int v = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const ViewCount c = vc[v];
    if (i >= c.ns) return;
    const int64_t j = c.base + ((int64_t)i * c.M) / c.ns;
    // the last item G in [v n, (v+1) n) with goff[G] <= j
    int64_t lo = (int64_t)v * gv.n, hi = lo + gv.n - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (goff[mid] <= j) lo = mid;
        else hi = mid - 1;
    }
    out[(int64_t)v * S + i] = (uint32_t)lo;
}

// One block per view: Alg. 2 over the view's samples, its bin parameters.
__global__ void __launch_bounds__(kDrThreads)
k_group_depth_range(const float4* __restrict__ c_o_z, const GroupViews gv, const ViewCount* __restrict__ vc,
                    const uint32_t* __restrict__ samples, DrArgs a, BinParams* __restrict__ bp)
{
    const int v = blockIdx.x;
    a.near_plane = gv.near_plane[v];
    a.far_plane = gv.far_plane[v];
    a.K = gv.K[v];
    depth_range_block(c_o_z, nullptr, GidFromSamples{samples + (int64_t)v * a.S}, vc[v].M, a, bp + v);
}

// The row spans of k_row_spans (tiles.cu) for the group's items: each lane's
// item and each record's owner look up their view (tile grid, bin splits,
// difference counts); records carry the item G.
__global__ void __launch_bounds__(256)
k_group_row_spans(const uint2* __restrict__ rect, const int32_t* __restrict__ roff, CullArgs ca, const GroupViews gv,
                  const BinParams* __restrict__ bp, const int64_t* __restrict__ m_dev, int64_t m_cap,
                  int32_t* __restrict__ D, uint32_t* __restrict__ rs_g, uint32_t* __restrict__ rs_ya,
                  uint32_t* __restrict__ rs_w, uint32_t* __restrict__ rs_z)
{
    if (*m_dev > m_cap) return;
    const int64_t n = gv.n * gv.nv;
    const int64_t g0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32;
    if (g0 >= n) return;
    const int lane = threadIdx.x & 31;
    const int64_t gl = g0 + lane;
    const bool ok = gl < n;
    const int32_t my_off = roff[ok ? gl : n];
    const int32_t base = __shfl_sync(0xffffffffu, my_off, 0);
    const int32_t end = roff[(g0 + 32) < n ? (g0 + 32) : n];
    uint2 r = make_uint2(0u, 0u);
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f), q = p;
    float margin = 0.0f;
    uint32_t bin = 0u;
    const int view = ok ? gv.view_of(gl) : 0;
    if (ok) {
        r = rect[gl];
        if ((r.x & 0xffffu) < (r.y & 0xffffu) && (r.x >> 16) < (r.y >> 16)) {
            p = __ldg(ca.xy_ab + gl);
            q = __ldg(ca.c_o_z + gl);
            margin = __ldg(&ca.rgb[gl].w);
            bin = (uint32_t)bin_split(q.z, bp[view].splits, gv.K[view]);
        }
    }
    const RowGeom mine = row_geom(0.5f * p.z, p.w, 0.5f * q.x, q.w, margin, p.y);
    const float inv_tile = 1.0f / (float)ca.tile;
    for (int32_t e0 = base; e0 < end; e0 += 32) {
        const int32_t e = e0 + lane;
        int k = 0;
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) {
            const int32_t v = __shfl_sync(0xffffffffu, my_off, (k + s) & 31);
            if (k + s < 32 && v <= e) k += s;
        }
        const uint32_t ra = __shfl_sync(0xffffffffu, r.x, k), rb = __shfl_sync(0xffffffffu, r.y, k);
        const float mx = __shfl_sync(0xffffffffu, p.x, k);
        RowGeom g;
        g.my = __shfl_sync(0xffffffffu, mine.my, k);
        g.hb = __shfl_sync(0xffffffffu, mine.hb, k);
        g.inv2ha = __shfl_sync(0xffffffffu, mine.inv2ha, k);
        g.a4tp = __shfl_sync(0xffffffffu, mine.a4tp, k);
        g.D = __shfl_sync(0xffffffffu, mine.D, k);
        g.dymax = __shfl_sync(0xffffffffu, mine.dymax, k);
        g.ext = __shfl_sync(0xffffffffu, mine.ext, k);
        g.dyl = __shfl_sync(0xffffffffu, mine.dyl, k);
        const uint32_t zb = __shfl_sync(0xffffffffu, __float_as_uint(q.z), k);
        const uint32_t b = __shfl_sync(0xffffffffu, bin, k);
        const int32_t o = __shfl_sync(0xffffffffu, my_off, k);
        const int vk = __shfl_sync(0xffffffffu, view, k);
        if (e < end) {
            const int tx0 = ra & 0xffff, ty0 = ra >> 16, tx1 = rb & 0xffff;
            const int ty = ty0 + (e - o);
            int a, x1;
            row_span(mx, g, ty, ca.tile, inv_tile, tx0, tx1, &a, &x1);
            rs_g[e] = (uint32_t)(g0 + k);
            rs_ya[e] = row_record(ty, a, b);
            rs_w[e] = (uint32_t)(x1 - a);
            rs_z[e] = zb;
            if (x1 > a) {
                const int W1 = gv.tiles_x[vk] + 1;
                int32_t* L = D + gv.d_base[vk] + (int64_t)b * gv.tiles_y[vk] * W1;
                atomicAdd(&L[ty * W1 + a], 1);
                atomicAdd(&L[ty * W1 + x1], -1);
            }
        }
    }
}

// One block per (view, bin layer): inclusive prefix along each tile row.
__global__ void __launch_bounds__(1024) k_group_layer_prefix(int32_t* __restrict__ D, const GroupViews gv)
{
    int v = 0;
    while (v + 1 < gv.nv && gv.layer_base[v + 1] <= (int)blockIdx.x) ++v;
    const int b = (int)blockIdx.x - gv.layer_base[v];
    const int tiles_x = gv.tiles_x[v], tiles_y = gv.tiles_y[v], W1 = tiles_x + 1;
    int32_t* L = D + gv.d_base[v] + (int64_t)b * tiles_y * W1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int y = warp; y < tiles_y; y += blockDim.x / 32) {
        int32_t carry = 0;
        for (int x0 = 0; x0 < tiles_x; x0 += 32) {
            const int x = x0 + lane;
            int32_t val = x < tiles_x ? L[y * W1 + x] : 0;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int32_t u = __shfl_up_sync(0xffffffffu, val, d);
                if (lane >= d) val += u;
            }
            if (x < tiles_x) L[y * W1 + x] = carry + val;
            carry += __shfl_sync(0xffffffffu, val, 31);
        }
    }
}

// count[t, b] of every view into the group's segment order (view v's tile t,
// bin b at seg_base[v] + t K_v + b), through 32 x 32 shared-memory blocks;
// blockIdx.z is the group's tile row.
__global__ void __launch_bounds__(256)
k_group_transpose(const int32_t* __restrict__ D, const GroupViews gv, int32_t* __restrict__ C)
{
    __shared__ int32_t s[32][33];
    int v = 0;
    while (v + 1 < gv.nv && gv.row_base[v + 1] <= (int)blockIdx.z) ++v;
    const int y = (int)blockIdx.z - gv.row_base[v];
    const int tiles_x = gv.tiles_x[v], K = gv.K[v], W1 = tiles_x + 1;
    const int x0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
    if (x0 >= tiles_x || b0 >= K) return;  // block-uniform
    const int64_t layer = (int64_t)gv.tiles_y[v] * W1;
    const int32_t* Dv = D + gv.d_base[v];
    const int lx = threadIdx.x & 31;
    for (int r = threadIdx.x >> 5; r < 32; r += blockDim.x >> 5) {
        const int b = b0 + r, x = x0 + lx;
        s[r][lx] = (b < K && x < tiles_x) ? Dv[b * layer + (int64_t)y * W1 + x] : 0;
    }
    __syncthreads();
    int32_t* Cv = C + gv.seg_base[v];
    for (int r = threadIdx.x >> 5; r < 32; r += blockDim.x >> 5) {
        const int x = x0 + r, b = b0 + lx;
        if (x < tiles_x && b < K) Cv[((int64_t)y * tiles_x + x) * K + b] = s[lx][r];
    }
}

// The scatter of k_bin_scatter_rows (tiles.cu) for the group: a record's
// item gives its view, whose tile grid, bin count and first segment place the
// entry; four entries a lane in flight.
__global__ void __launch_bounds__(256)
k_group_scatter(const uint32_t* __restrict__ rs_g, const uint32_t* __restrict__ rs_ya, const uint32_t* __restrict__ rs_w,
                const uint32_t* __restrict__ rs_z, const int32_t* __restrict__ roff, const GroupViews gv,
                const int64_t* __restrict__ m_dev, int64_t m_cap, int32_t* __restrict__ cur,
                uint64_t* __restrict__ words)
{
    if (*m_dev > m_cap) return;
    const int64_t R = roff[gv.n * gv.nv];
    const int lane = threadIdx.x & 31;
    const int64_t nchunks = (R + 31) / 32;
    const int64_t wstride = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < nchunks; c += wstride) {
        const int64_t k = c * 32 + lane;
        uint32_t w = 0, g = 0, ya = 0, z = 0;
        int view = 0;
        if (k < R) {  // read once: streamed past L2
            w = __ldcs(rs_w + k);
            g = __ldcs(rs_g + k);
            ya = __ldcs(rs_ya + k);
            z = __ldcs(rs_z + k);
            view = gv.view_of(g);
        }
        uint32_t incl = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += u;
        }
        const uint32_t excl = incl - w;
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        for (uint32_t e0 = 0; e0 < total; e0 += 32 * 4) {
            int32_t pos[4];
            uint64_t word[4];
            bool live[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t e = e0 + 32 * u + lane;
                int o = 0;
#pragma unroll
                for (int s = 16; s > 0; s >>= 1) {
                    const uint32_t vv = __shfl_sync(0xffffffffu, excl, (o + s) & 31);
                    if (o + s < 32 && vv <= e) o += s;
                }
                const uint32_t oex = __shfl_sync(0xffffffffu, excl, o);
                const uint32_t og = __shfl_sync(0xffffffffu, g, o), oya = __shfl_sync(0xffffffffu, ya, o);
                const uint32_t oz = __shfl_sync(0xffffffffu, z, o);
                const int ov = __shfl_sync(0xffffffffu, view, o);
                live[u] = e < total;
                if (live[u]) {
                    const int ty = (int)(oya & 0xfffu), tx = (int)((oya >> 12) & 0xfffu) + (int)(e - oex);
                    const int64_t q = gv.seg_base[ov] + ((int64_t)ty * gv.tiles_x[ov] + tx) * gv.K[ov] + (oya >> 24);
                    pos[u] = atomicAdd(&cur[q], 1);
                    word[u] = ((uint64_t)oz << 32) | og;
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (live[u]) words[pos[u]] = word[u];
        }
    }
}

// ------------------------------------------------------------------ host

// zero offsets when the entries overflow the capacity (tiles.cu)
__global__ void k_zero_if_over(const int64_t* __restrict__ m_dev, int64_t m_cap, int32_t* __restrict__ off, int64_t nq,
                               int* err);

GroupViews* group_views_new() { return new GroupViews(); }
void group_views_free(GroupViews* gv) { delete gv; }
int64_t group_seg_base(const GroupViews* gv, int v) { return gv->seg_base[v]; }

int64_t group_views_set(GroupViews* gv, int64_t n, int nv, const gs_camera* cams, const int32_t* K)
{
    memset(gv, 0, sizeof(*gv));
    gv->nv = nv;
    gv->n = n;
    for (int v = 0; v < nv; ++v) {
        const int tx = (cams[v].width + 15) / 16, ty = (cams[v].height + 15) / 16;
        gv->K[v] = K[v];
        gv->tiles_x[v] = tx;
        gv->tiles_y[v] = ty;
        gv->tile_base[v + 1] = gv->tile_base[v] + tx * ty;
        gv->seg_base[v + 1] = gv->seg_base[v] + (int64_t)tx * ty * K[v];
        gv->row_base[v + 1] = gv->row_base[v] + ty;
        gv->layer_base[v + 1] = gv->layer_base[v] + K[v];
        gv->d_base[v + 1] = gv->d_base[v] + (int64_t)K[v] * ty * (tx + 1);
        gv->near_plane[v] = cams[v].near_plane;
        gv->far_plane[v] = cams[v].far_plane;
    }
    return gv->seg_base[nv];
}

// The group's scratch in gc->d_tiles: difference counts, cursors (also the
// staging copy of the transposed counts), row records, samples, per-view bin
// parameters and entry counts.
struct GroupScratch {
    int32_t* D;
    int32_t* cur;
    uint32_t *rs_g, *rs_ya, *rs_w, *rs_z;
    uint32_t* samples;
    BinParams* bp;
    ViewCount* vc;
    int64_t* m_views;
};

static size_t group_scratch(const GroupViews& gv, int64_t m_cap, int S, char* base, GroupScratch* s)
{
    const size_t mc = (size_t)(m_cap > 0 ? m_cap : 1);
    const size_t sizes[] = {(size_t)gv.d_base[gv.nv] * 4, (size_t)gv.seg_base[gv.nv] * 4, mc * 4, mc * 4, mc * 4,
                            mc * 4, (size_t)gv.nv * S * 4, (size_t)gv.nv * sizeof(BinParams),
                            (size_t)gv.nv * sizeof(ViewCount), (size_t)gv.nv * 8};
    size_t total = 0;
    for (size_t z : sizes) total += align256(z > 0 ? z : 4);
    if (s) {
        char* p = base;
        void** dst[] = {(void**)&s->D, (void**)&s->cur, (void**)&s->rs_g, (void**)&s->rs_ya, (void**)&s->rs_w,
                        (void**)&s->rs_z, (void**)&s->samples, (void**)&s->bp, (void**)&s->vc, (void**)&s->m_views};
        for (int k = 0; k < 10; ++k) {
            *dst[k] = p;
            p += align256(sizes[k] > 0 ? sizes[k] : 4);
        }
    }
    return total;
}

int group_reserve(gs_ctx* gc, const GroupViews* gvp, int64_t m_cap)
{
    const GroupViews& gv = *gvp;
    const int64_t N = gv.n * gv.nv, NS = gv.seg_base[gv.nv];
    int r;
    if ((r = ensure(&gc->r_proj, &gc->r_proj_cap, gs_projected_bytes(N))) != GS_OK) return r;
    if (m_cap > gc->r_m_cap) {
        if (gc->r_stream) cudaFree(gc->r_stream);
        gc->r_stream = nullptr;
        gc->r_m_cap = 0;
        size_t sb = 0;
        void* sp = nullptr;
        if ((r = ensure(&sp, &sb, (size_t)m_cap * 8)) != GS_OK) return r;
        gc->r_stream = (uint64_t*)sp;
        gc->r_m_cap = m_cap;
    }
    void* op = gc->r_off;
    if ((r = ensure(&op, &gc->r_off_cap, ((size_t)NS + 1) * 4)) != GS_OK) return r;
    gc->r_off = (int32_t*)op;
    void* tp = gc->d_tiles;
    if ((r = ensure(&tp, &gc->tiles_cap, group_scratch(gv, gc->r_m_cap, gc->cfg.sample_count, nullptr, nullptr))) !=
        GS_OK)
        return r;
    gc->d_tiles = (int32_t*)tp;
    if ((r = goff_reserve(gc, N)) != GS_OK) return r;
    return scan_reserve(gc, N > NS ? N : NS);
}

int group_binning(gs_ctx* gc, const GroupViews* gvp, int32_t flags, int64_t* h_m_views, cudaStream_t st)
{
    const GroupViews& gv = *gvp;
    const int64_t N = gv.n * gv.nv, NS = gv.seg_base[gv.nv];
    const int S = gc->cfg.sample_count;
    int r;
    if ((r = group_reserve(gc, gvp, gc->r_m_cap > 0 ? gc->r_m_cap : 1)) != GS_OK) return r;
    const ProjView pv = proj_view(gc->r_proj, N);
    // tile counts and row counts of every item, one scan (as a single frame)
    if ((r = count_rows_scan(gc, pv, N, gc->r_m, st)) != GS_OK) return r;
    if (!(flags & GS_RENDER_NO_SYNC)) {
        GS_CUDA_TRY(cudaMemcpyAsync(gc->h_m, gc->r_m, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        GS_CUDA_TRY(cudaStreamSynchronize(st));
        if (gc->h_m[0] > gc->r_m_cap && (r = group_reserve(gc, gvp, gc->h_m[0])) != GS_OK) return r;
    }
    GroupScratch s;
    group_scratch(gv, gc->r_m_cap, S, reinterpret_cast<char*>(gc->d_tiles), &s);
    const int32_t* roff = rows_offsets(gc, N);
    // per-view entry counts, samples and depth range (Alg. 2)
    k_group_counts<<<1, 32, 0, st>>>(gc->d_goff, gv.n, gv.nv, S, s.vc, s.m_views);
    if (h_m_views)
        GS_CUDA_TRY(cudaMemcpyAsync(h_m_views, s.m_views, (size_t)gv.nv * 8, cudaMemcpyDeviceToHost, st));
    if (N > 0) k_group_sample_gids<<<dim3((unsigned)((S + 255) / 256), (unsigned)gv.nv), 256, 0, st>>>(gc->d_goff, gv, s.vc, S, s.samples);
    DrArgs a;
    a.S = S;
    a.near_shift = 0;  // EXACT mode
    a.near_alpha = gc->cfg.near_alpha;
    a.near_gamma = gc->cfg.near_gamma;
    a.p_lo = gc->cfg.p_lo;
    a.p_hi = gc->cfg.p_hi;
    a.pad = gc->cfg.pad;
    a.eps = gc->cfg.eps;
    a.near_plane = a.far_plane = 0.0f;
    a.K = 0;  // set per view
    k_group_depth_range<<<(unsigned)gv.nv, kDrThreads, 0, st>>>(pv.c_o_z, gv, s.vc, s.samples, a, s.bp);
    gc->launches += N > 0 ? 3 : 2;
    // row spans and per-row difference counts, per-view prefixes, the counts
    // transposed into the group's segment order, one scan
    GS_CUDA_TRY(cudaMemsetAsync(s.D, 0, (size_t)gv.d_base[gv.nv] * 4, st));
    const CullArgs ca{pv.xy_ab, pv.c_o_z, pv.rgb, 16};
    const int64_t warps = (N + 31) / 32;
    if (warps > 0)
        k_group_row_spans<<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(pv.rect, roff, ca, gv, s.bp, gc->r_m,
                                                                       gc->r_m_cap, s.D, s.rs_g, s.rs_ya, s.rs_w,
                                                                       s.rs_z);
    k_group_layer_prefix<<<(unsigned)gv.layer_base[gv.nv], 1024, 0, st>>>(s.D, gv);
    int max_tx = 1, max_k = 1;
    for (int v = 0; v < gv.nv; ++v) {
        max_tx = gv.tiles_x[v] > max_tx ? gv.tiles_x[v] : max_tx;
        max_k = gv.K[v] > max_k ? gv.K[v] : max_k;
    }
    k_group_transpose<<<dim3((unsigned)((max_tx + 31) / 32), (unsigned)((max_k + 31) / 32), (unsigned)gv.row_base[gv.nv]),
                        256, 0, st>>>(s.D, gv, s.cur);
    gc->launches += 3;
    if ((r = scan_impl(gc, LoadI32{s.cur}, NS, gc->r_off, nullptr, st)) != GS_OK) return r;
    const unsigned g_sm = (unsigned)gc->num_sms * 8;
    k_zero_if_over<<<g_sm, 256, 0, st>>>(gc->r_m, gc->r_m_cap, gc->r_off, NS + 1, gc->d_err);
    // the scatter: every entry a slot in its view's (tile, bin) segment
    GS_CUDA_TRY(cudaMemcpyAsync(s.cur, gc->r_off, (size_t)NS * 4, cudaMemcpyDeviceToDevice, st));
    if (N > 0)
        k_group_scatter<<<g_sm * 2, 256, 0, st>>>(s.rs_g, s.rs_ya, s.rs_w, s.rs_z, roff, gv, gc->r_m, gc->r_m_cap,
                                                  s.cur, gc->r_stream);
    gc->launches += 2;
    GS_CUDA_TRY(cudaGetLastError());
    // segments longer than the raster sorts in shared memory
    return sort_long_segments(gc, NS, gc->r_off, gc->r_stream, kRasterSortCap + 1, st);
}

}  // namespace gs
