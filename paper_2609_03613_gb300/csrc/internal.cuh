// internal.cuh -- shared pieces of libtilegs (not part of the ABI).
//
// Built with -fmad=false: no multiply-add is fused unless fmaf() is written,
// so every float32 value that decides an integer (tile rectangle, alpha skip,
// transmittance stop, bin index) follows the operation order stated at its
// definition.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tilegs.h"

#define GS_CUDA_TRY(expr)                                   \
    do {                                                    \
        cudaError_t e_ = (expr);                            \
        if (e_ != cudaSuccess) return gs_cuda_fail(e_, #expr); \
    } while (0)

int gs_cuda_fail(cudaError_t e, const char* what);

namespace gs {

constexpr int kNumSMs = 152;  // GB300: 2 dies x 76 SMs (queried at runtime where it matters)

// ------------------------------------------------------------------ records
// Byte offsets of the projected fields (each 256-byte aligned).
__host__ __device__ inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct ProjView {
    float4* xy_ab;   // {mean_x, mean_y, conic_a, conic_b}
    float4* c_o_z;   // {conic_c, opacity, depth, cull_tau}
    float4* rgb;     // {r, g, b, cull_margin}
    uint2* rect;     // {tx0 | ty0 << 16, tx1 | ty1 << 16}
    int32_t* radius;
};

inline ProjView proj_view(void* base, int64_t n)
{
    char* b = static_cast<char*>(base);
    ProjView v;
    v.xy_ab = reinterpret_cast<float4*>(b + gs_projected_offset(n, GS_P_XY_AB));
    v.c_o_z = reinterpret_cast<float4*>(b + gs_projected_offset(n, GS_P_C_O_Z));
    v.rgb = reinterpret_cast<float4*>(b + gs_projected_offset(n, GS_P_RGB));
    v.rect = reinterpret_cast<uint2*>(b + gs_projected_offset(n, GS_P_RECT));
    v.radius = reinterpret_cast<int32_t*>(b + gs_projected_offset(n, GS_P_RADIUS));
    return v;
}

struct IsectView {
    uint32_t* tile;
    uint32_t* zbits;
    uint32_t* gid;
};

inline IsectView isect_view(void* base, int64_t m_cap)
{
    char* b = static_cast<char*>(base);
    IsectView v;
    v.tile = reinterpret_cast<uint32_t*>(b + gs_isect_offset(m_cap, 0));
    v.zbits = reinterpret_cast<uint32_t*>(b + gs_isect_offset(m_cap, 1));
    v.gid = reinterpret_cast<uint32_t*>(b + gs_isect_offset(m_cap, 2));
    return v;
}

// Gradient buffer of gs_rasterize_bwd: three float4 fields mirroring the
// first three fields of the projected record.
struct GradView {
    float4* xy_ab;  // {dmean_x, dmean_y, dconic_a, dconic_b}
    float4* c_o_z;  // {dconic_c, dopacity, 0, 0}
    float4* rgb;    // {dr, dg, db, 0}
};

inline GradView grad_view(void* base, int64_t n)
{
    char* b = static_cast<char*>(base);
    GradView v;
    v.xy_ab = reinterpret_cast<float4*>(b + gs_grad2d_offset(n, 0));
    v.c_o_z = reinterpret_cast<float4*>(b + gs_grad2d_offset(n, 1));
    v.rgb = reinterpret_cast<float4*>(b + gs_grad2d_offset(n, 2));
    return v;
}

// Live entry count: the device count when it fits the capacity, else 0 (the
// emitter has raised GS_ERR_CAPACITY and written nothing).
__device__ __forceinline__ int64_t live_count(const int64_t* m_dev, int64_t m_cap)
{
    const int64_t m = *m_dev;
    return (m >= 0 && m <= m_cap) ? m : 0;
}

// ------------------------------------------------------------------ device error word
// Kernels record the first device-side error here (atomicCAS from 0).
__device__ inline void raise_error(int* err, int code)
{
    if (err) atomicCAS(err, 0, code);
}

// ------------------------------------------------------------------ programmatic dependent launch
// A kernel launched by launch_k() on a context with cfg.pdl may be set up
// while its predecessor in the stream drains (its blocks are scheduled as
// the predecessor's blocks exit).  Every such kernel calls
// grid_dependency_sync() first, in every thread, before any memory access:
// it returns once the predecessor grid has completed and its writes are
// visible -- and since every kernel of the chain waits the same way, so have
// all earlier ones.  Launched the ordinary way, it is a no-op.  No kernel
// signals its successor early: a signal at kernel start (successor blocks
// resident behind the last wave) measured 0.604 ms against 0.595 ms for the
// 1080p frame graph.
__device__ __forceinline__ void grid_dependency_sync()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ------------------------------------------------------------------ elementary functions
// exp by Cody-Waite range reduction and a degree-7 Taylor polynomial (W. J.
// Cody and W. Waite, "Software Manual for the Elementary Functions", 1980):
// n = round(x log2 e) via the 1.5 * 2^23 shifter, r = x - n ln2 in two
// pieces, e^r by Horner over 1/k!, then scaled by 2^n built in the exponent
// field.  Every step is one correctly rounded float32 operation.  The core
// requires x in [-87, 88] (so that 2^n is a normal float); spec_exp clamps.
__device__ __forceinline__ float spec_exp_core(float x)
{
    const float kLog2e = 1.44269504088896341f;
    const float kLn2Hi = 0.693145751953125f;
    const float kLn2Lo = 1.42860682030941723e-6f;
    const float kShift = 12582912.0f;  // 1.5 * 2^23
    const float k = fmaf(x, kLog2e, kShift);
    const float n = __fsub_rn(k, kShift);
    float r = fmaf(n, -kLn2Hi, x);
    r = fmaf(n, -kLn2Lo, r);
    float p = 1.0f / 5040.0f;
    p = fmaf(p, r, 1.0f / 720.0f);
    p = fmaf(p, r, 1.0f / 120.0f);
    p = fmaf(p, r, 1.0f / 24.0f);
    p = fmaf(p, r, 1.0f / 6.0f);
    p = fmaf(p, r, 0.5f);
    p = fmaf(p, r, 1.0f);
    p = fmaf(p, r, 1.0f);
    // bits(k) = bits(kShift) + n for |n| < 2^22, so the exponent field of
    // 2^n is (bits(k) - bits(kShift) + 127) << 23 -- formed in unsigned
    // arithmetic, which wraps, so that x outside the core's range (the
    // raster evaluates it for every test and uses the value only inside)
    // gives some float and never an undefined signed overflow.
    const uint32_t e = (__float_as_uint(k) - 0x4B400000u + 127u) << 23;
    return __fmul_rn(p, __uint_as_float(e));
}

// Full-range variant: clamps x to [-87, 88] first.
__device__ __forceinline__ float spec_exp(float x)
{
    x = x < -87.0f ? -87.0f : x;
    x = x > 88.0f ? 88.0f : x;
    return spec_exp_core(x);
}

// 1/d for d in [2^-126, 2^126]: the hardware's approximate reciprocal (PTX
// rcp.approx.ftz.f32, within 1 ulp) refined by one Newton-Raphson step,
// r' = r + r (1 - d r), with the residual 1 - d r formed by one fused
// multiply-add (the FMA-based iteration of P. Markstein, "Computation of
// elementary functions on the IBM RISC System/6000 processor", IBM J. Res.
// Dev. 34(1), 1990): the seed's error is squared, so the result is within
// one rounding of 1/d -- the correctly rounded value or its neighbour
// (gs_reciprocal exposes it; a GPU test checks it against the correctly
// rounded reciprocal over [0.01, 1]).
__device__ __forceinline__ float rcp_newton(float d)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
    return fmaf(r, fmaf(-d, r, 1.0f), r);
}

// ln by exponent split and the atanh series (Abramowitz and Stegun 4.1.27):
// x = 2^e m, m in (sqrt(1/2), sqrt(2)], s = (m-1)/(m+1),
// ln m = 2 s (1 + s^2/3 + s^4/5 + s^6/7 + s^8/9), ln x = e ln2 + ln m.
// Defined for normal positive x.
__device__ __forceinline__ float spec_log(float x)
{
    const float kLn2Hi = 0.693145751953125f;
    const float kLn2Lo = 1.42860682030941723e-6f;
    const uint32_t u = __float_as_uint(x);
    int e = int((u >> 23) & 0xffu) - 127;
    float m = __uint_as_float((u & 0x007fffffu) | 0x3f800000u);
    if (m > 1.41421356f) {
        m = __fmul_rn(m, 0.5f);
        e = e + 1;
    }
    const float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float s2 = __fmul_rn(s, s);
    float p = 1.0f / 9.0f;
    p = fmaf(p, s2, 1.0f / 7.0f);
    p = fmaf(p, s2, 1.0f / 5.0f);
    p = fmaf(p, s2, 1.0f / 3.0f);
    p = fmaf(p, s2, 1.0f);
    const float lnm = __fmul_rn(__fmul_rn(2.0f, s), p);
    const float fe = float(e);
    return fmaf(fe, kLn2Hi, fmaf(fe, kLn2Lo, lnm));
}

// ------------------------------------------------------------------ bins
struct BinParams {
    float zmin, zmax;  // robust depth range
    float lmin, lmax;  // ln z'min, ln z'max
    int32_t K;
    int32_t nsamples;  // kept samples
    float splits[GS_MAX_K];  // K-1 log-spaced split depths (monotone map)
};

}  // namespace gs

// ------------------------------------------------------------------ context
namespace gs {
struct BatchState;
}

struct gs_ctx {
    gs_config cfg;
    int device = 0;
    int num_sms = 152;
    int* d_err = nullptr;
    // scan scratch (block sums) and the scans' last-block counter (zeroed once)
    void* d_scan = nullptr;
    size_t scan_bytes = 0;
    unsigned int* d_scan_done = nullptr;
    // a frame's scan-flag arena: scan_arena words of d_scan that the frame's
    // first kernel zeroed, handed out in order (scan_used) so that the
    // frame's scans need no memset between kernels; 0: none (every scan
    // clears its own flags).  Valid while d_scan keeps the size it had then
    // (scan_arena_bytes): a grown buffer is a new one.
    int64_t scan_arena = 0, scan_used = 0;
    size_t scan_arena_bytes = 0;
    // the same for the EXACT bin stage's difference counts and the repair's
    // long-segment counter: the zeroed pointer and its buffer's size then
    int32_t* zeroed_D = nullptr;
    size_t zeroed_D_bytes = 0;
    int32_t* zeroed_tail = nullptr;
    size_t zeroed_tail_bytes = 0;
    // the regions the frame's depth-range sampling zeroes (the projection
    // zeroes only the first scan's flags: a multi-megabyte clear there
    // lengthened it more than the sampling kernel)
    int32_t* late_p[3] = {nullptr, nullptr, nullptr};
    int64_t late_n[3] = {0, 0, 0};
    // per-Gaussian emission offsets [n+1]
    int32_t* d_goff = nullptr;
    size_t goff_cap = 0;
    // global radix sort ping-pong + histograms
    uint64_t* d_keys[2] = {nullptr, nullptr};
    uint32_t* d_vals[2] = {nullptr, nullptr};
    size_t sort_cap = 0;
    uint32_t* d_hist = nullptr;
    size_t hist_cap = 0;
    // binning
    int32_t* d_count = nullptr;  // T*K counters
    size_t count_cap = 0;
    uint8_t* d_bin = nullptr;    // per-entry bin id
    size_t bin_cap = 0;
    gs::BinParams* d_bp = nullptr;
    uint8_t* d_sel = nullptr;    // per-segment repair selection
    size_t sel_cap = 0;
    int32_t* d_tail = nullptr;   // segments too long for a shared-memory sort
    size_t tail_cap = 0;
    int32_t* d_tiles = nullptr;   // tile-count difference grid, tile offsets, cursors
    size_t tiles_cap = 0;
    uint32_t* d_samples = nullptr; // depth-range samples (their keys as float bits)
    size_t samples_cap = 0;
    int32_t* d_tiles_order = nullptr;  // persistent raster tile order
    int32_t* d_tile_counter = nullptr;
    size_t order_cap = 0;
    // whole-frame buffers (gs_render)
    void* r_proj = nullptr; size_t r_proj_cap = 0;
    void* r_isect = nullptr; int64_t r_m_cap = 0;
    uint64_t* r_stream = nullptr;
    int32_t* r_off = nullptr; size_t r_off_cap = 0;
    int64_t* r_m = nullptr;
    int64_t* h_m = nullptr;  // pinned
    float* r_scene = nullptr; size_t r_scene_cap = 0;  // device copies of host inputs
    float* r_out = nullptr; size_t r_out_cap = 0;      // device outputs for host outputs
    // pipelined host-buffer frames (GS_RENDER_PIPELINE): two slots of device
    // inputs and outputs used in turn, an upload and a download stream
    struct PipeSlot {
        float* scene = nullptr; size_t scene_cap = 0;
        float* out = nullptr; size_t out_cap = 0;
        cudaEvent_t uploaded = nullptr;    // the slot's scene is on the device
        cudaEvent_t rendered = nullptr;    // the slot's frame has finished
        cudaEvent_t downloaded = nullptr;  // the slot's outputs are in host memory
        bool used = false;
    } pipe[2];
    cudaStream_t pipe_up = nullptr, pipe_down = nullptr;
    int pipe_next = 0;
    // saved state of the last gs_render with GS_RENDER_SAVE (for gs_render_bwd)
    float* r_T = nullptr; size_t r_T_cap = 0;        // final transmittance [H,W]
    int32_t* r_tend = nullptr; size_t r_tend_cap = 0; // per-tile end of the compositing [T]
    int32_t* r_wend = nullptr; size_t r_wend_cap = 0; // per-warp end of the compositing [T][warps]
    int r_wend_valid = 0;                             // the saved frame wrote r_wend
    const int32_t* r_last = nullptr;                  // the last-id buffer that render wrote (device)
    int64_t r_n = -1;                                 // Gaussian count of that render
    gs_camera r_cam;
    float r_bg[3] = {0.f, 0.f, 0.f};
    int r_saved = 0;
    int64_t last_m = 0;
    int64_t launches = 0;  // kernels this context has launched
    int64_t* d_ops = nullptr;  // compositing ops counted by the instrumented raster
    // whole-frame CUDA graph (GS_RENDER_GRAPH)
    cudaGraphExec_t gexec = nullptr;
    unsigned char gkey[1024];
    size_t gkey_len = 0;
    int64_t glaunches = 0;
    const int32_t* g_last = nullptr;  // last-id buffer of the captured frame
    int g_wend_valid = 0;             // the captured frame writes per-warp ends
    int capturing = 0;
    // bin planner (planner.cu): MLP parameters, per-frame features and plan
    float* d_planner = nullptr;
    int planner_ready = 0;
    float* d_feat = nullptr; size_t feat_cap = 0;
    uint8_t* d_plan = nullptr; size_t plan_cap_bytes = 0;  // [T] first-pass bins, [T] completion flags, [T] row flags
    int32_t* d_plist = nullptr; size_t plist_cap = 0;      // [1 + T]: count, then the flagged tiles
    int32_t* exact_roff = nullptr;  // row-record offsets of the last planned frame's bin construction
    // batched multi-view rendering (gs_render_batch)
    gs::BatchState* batch = nullptr;
    // spatial order of a scene (order.cu)
    void* d_order_ws = nullptr;
    size_t order_ws_cap = 0;
    // timing
    int timing = 0;
    cudaEvent_t ev_b[GS_STAGE_COUNT];
    cudaEvent_t ev_e[GS_STAGE_COUNT];
    int ev_ok = 0;
    float stage_ms[GS_STAGE_COUNT];
    int stage_used[GS_STAGE_COUNT];
};

// ------------------------------------------------------------------ internal launchers
namespace gs {
// Regions (int32 words, 16-byte aligned starts) that a frame's first kernel
// zeroes for the later ones.
struct FrameZero {
    int32_t* p[3] = {nullptr, nullptr, nullptr};
    int64_t n[3] = {0, 0, 0};
};

// Zero the regions of z with the whole grid (16-byte stores, then the tail).
__device__ __forceinline__ void frame_zero(const FrameZero& z)
{
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        int32_t* p = z.p[r];
        if (!p) continue;
        const int64_t n4 = z.n[r] >> 2;
        int4* q = reinterpret_cast<int4*>(p);
        for (int64_t i = t0; i < n4; i += stride) q[i] = make_int4(0, 0, 0, 0);
        for (int64_t i = 4 * n4 + t0; i < z.n[r]; i += stride) p[i] = 0;
    }
}

// Forget the regions a frame's first kernel zeroed (the frame is over, or
// none was zeroed): every later scan, bin stage and repair clears its own.
inline void frame_zero_reset(gs_ctx* c)
{
    c->scan_arena = 0;
    c->scan_used = 0;
    c->zeroed_D = nullptr;
    c->zeroed_tail = nullptr;
    for (int k = 0; k < 3; ++k) c->late_p[k] = nullptr;
}

// Launch of a frame kernel (one that starts with grid_dependency_sync()):
// with programmatic stream serialization when the context allows it and is
// not recording stage times (an event between two overlapped kernels would
// not bound either of them).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(const gs_ctx* ctx, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                            cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t lc = {};
    lc.gridDim = grid;
    lc.blockDim = block;
    lc.dynamicSmemBytes = smem;
    lc.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    if (ctx->cfg.pdl && !ctx->timing) {
        lc.attrs = attr;
        lc.numAttrs = 1;
    }
    return cudaLaunchKernelEx(&lc, kern, static_cast<KArgs>(args)...);
}

// A whole frame of this context runs the planned two passes (EXACT, repair in
// the raster, tile cull, planner on).
inline bool frame_planned(const gs_ctx* c)
{
    return c->cfg.planner && c->cfg.mode == GS_MODE_BINNED_EXACT && c->cfg.repair_in_raster && c->cfg.tile_cull;
}

int ensure(void** p, size_t* cap, size_t bytes);
int check_config(const gs_config* cfg);

// scan.cu
// Exclusive scan of int32 counts[0..n) into out[0..n] (out[n] = total) with
// the total also stored as int64 at total64 (nullable).  3 kernels.
int exclusive_scan_i32(gs_ctx* ctx, const int32_t* counts, int64_t n, int32_t* out,
                       int64_t* total64, cudaStream_t st);
// Tile counts of the projected rects, scanned into per-Gaussian offsets.
int scan_tile_counts(gs_ctx* ctx, const uint2* rect, int64_t n, int32_t* out, int64_t* total64,
                     cudaStream_t st);

// tile counts -> per-Gaussian offsets (ctx->d_goff) and M; then the emission
int count_scan(gs_ctx* ctx, const ProjView& pv, int64_t n, int64_t* m_dev, cudaStream_t st);
// count_scan plus the EXACT row-record offsets in one pass
int count_rows_scan(gs_ctx* ctx, const ProjView& pv, int64_t n, int64_t* m_dev, cudaStream_t st);
int32_t* rows_offsets(gs_ctx* ctx, int64_t n);
int64_t* rows_total(gs_ctx* ctx, int64_t n);
// scratch of the per-Gaussian offsets and of the scans (intersect.cu)
int goff_reserve(gs_ctx* ctx, int64_t n);
int scan_reserve(gs_ctx* ctx, int64_t n);
int emit_only(gs_ctx* ctx, const ProjView& pv, int64_t n, const gs_camera* cam, const IsectView& is,
              int64_t m_cap, const int64_t* m_dev, cudaStream_t st);

// sort.cu
int global_sort(gs_ctx* ctx, const IsectView& is, int64_t m_cap, const int64_t* m_dev,
                int32_t n_tiles, uint64_t* stream_words, int32_t* offsets, cudaStream_t st);

// bins.cu
int depth_range(gs_ctx* ctx, const ProjView& pv, const float* scales, const IsectView& is,
                int64_t m_cap, const int64_t* m_dev, const gs_camera* cam, cudaStream_t st);
int bin_build(gs_ctx* ctx, const ProjView& pv, const float* scales, const IsectView& is,
              int64_t m_cap, const int64_t* m_dev, int32_t n_tiles, uint64_t* stream_words,
              int32_t* offsets, cudaStream_t st);
int repair(gs_ctx* ctx, int32_t n_tiles, const int64_t* m_dev, uint64_t* stream_words,
           const int32_t* offsets, uint8_t* selected_out, cudaStream_t st);
int set_zrange(gs_ctx* ctx, const float* zrange, cudaStream_t st);
int launch_depth_range_into(const gs_config& c, const ProjView& pv, const float* scales, const IsectView& is,
                            int64_t m_cap, const int64_t* m_dev, const gs_camera* cam, BinParams* bp,
                            cudaStream_t st);

// tiles.cu: EXACT-mode bin construction straight from the projected rects
// (with the tile cull: per-row culled spans; without: layered difference
// counts and the expansion, which needs ctx->d_goff -- computed here unless
// goff_ready).  Segments are left unsorted.
// rows_ready: count_rows_scan has also written the row-record offsets.
// With planned (the tile cull on): after the counts, the bin planner sets
// each tile's first-pass bins (plan_frame) and only entries of those bins are
// scattered; exact_scatter_rest then places the other entries of the tiles
// the first raster pass flagged.
int exact_bins(gs_ctx* ctx, const ProjView& pv, int64_t n, const gs_camera* cam, bool goff_ready, int64_t m_cap,
               const int64_t* m_dev, uint64_t* words, int32_t* offsets, cudaStream_t st, bool rows_ready = false,
               bool planned = false);
int exact_scatter_rest(gs_ctx* ctx, int64_t n, const gs_camera* cam, int64_t m_cap, const int64_t* m_dev,
                       uint64_t* words, const int32_t* offsets, cudaStream_t st);
// the regions of a tile-cull EXACT frame that its projection zeroes (tiles.cu)
int exact_frame_zero(gs_ctx* ctx, int64_t n, const gs_camera* cam, int64_t m_cap, FrameZero* fz);
// the scratch of the bin count / scatter and the repair (bins.cu)
int bins_reserve(gs_ctx* ctx, int64_t m_cap, int64_t nseg);
// tiles.cu: items of the grouped scatter's count scan (for reserving)
int64_t group_scan_items(gs_ctx* ctx, int32_t tiles_y, int K);
// bins.cu: sort segments of length >= min_len (EXACT) or the rule/budget
// selection (PAPER)
// pass 1 / 2 (EXACT, long segments only): the segments of the planned
// frame's first pass (bins below ctx->d_plan) or of its completing pass (the
// other bins of flagged tiles); 0: every segment
int repair_min(gs_ctx* ctx, int32_t n_tiles, const int64_t* m_dev, uint64_t* stream_words, const int32_t* offsets,
               uint8_t* selected_out, int32_t min_len, cudaStream_t st, int pass = 0);
// sort every segment of a flat segment array [nseg] longer than min_len - 1
// entries (the segments the raster cannot sort in shared memory)
int sort_long_segments(gs_ctx* ctx, int64_t nseg, const int32_t* offsets, uint64_t* words, int32_t min_len,
                       cudaStream_t st);
// segments longer than this are sorted before the raster when the raster
// sorts the segments it reaches
constexpr int kRasterSortCap = 2048;
// Classes of the bin planner: class c < kPlanClasses - 1 gives a tile's first
// pass the fewest bins from its front that hold at least plan_entries(c)
// entries; the last class gives it every bin.
constexpr int kPlanClasses = 6;
__host__ __device__ inline int plan_entries(int cls) { return 64 << cls; }
// What a planned raster pass reads and writes per tile: bins[t] (nullable:
// all) is the number of bins walked from the tile's front; a tile that has
// not terminated when they end while later bins hold entries is flagged
// (flag[t] = 1, flag[T + tile row] = 1, appended to list = {count,
// tiles...}) for the completing pass;
// needed[t] (the counting twin, all bins walked) receives the bins the tile
// needs: 1 + the bin holding the last entry any pixel visits.
// Which entries (or segments) a pass of bin construction handles.  pass 0:
// all; pass 1 (a planned frame's first pass): bins below the tile's planned
// bins; pass 2 (its completing pass): the other bins of the tiles the first
// raster pass flagged.
struct ScatterPass {
    const uint8_t* plan = nullptr;  // [T] planned bins, [T] flags, then per tile row a flag (any tile of it)
    int32_t T = 0;
    int pass = 0;
    __device__ __forceinline__ bool keep(int64_t t, int b) const
    {
        if (pass == 0) return true;
        const int B = __ldg(plan + t);
        return pass == 1 ? b < B : (b >= B && __ldg(plan + T + t) != 0);
    }
    // whether the completing pass has anything in tile row ty
    __device__ __forceinline__ bool row_live(int ty) const { return pass != 2 || __ldg(plan + 2 * (int64_t)T + ty) != 0; }
    // A row record (tile row | first tile << 12 | bin << 24, width) trimmed to
    // the tiles from the first to the last this pass keeps; width 0 when it
    // keeps none (the record is skipped whole).
    __device__ __forceinline__ void trim(uint32_t& ya, uint32_t& w, int tiles_x) const
    {
        if (pass == 0 || w == 0u) return;
        const int b = (int)(ya >> 24), x0 = (int)((ya >> 12) & 0xfffu);
        const int64_t t0 = (int64_t)(ya & 0xfffu) * tiles_x + x0;
        int lo = -1, hi = -1;
        for (int j = 0; j < (int)w; ++j)
            if (keep(t0 + j, b)) {
                if (lo < 0) lo = j;
                hi = j;
            }
        if (lo < 0) {
            w = 0u;
            return;
        }
        ya = (ya & ~(0xfffu << 12)) | ((uint32_t)(x0 + lo) << 12);
        w = (uint32_t)(hi - lo + 1);
    }
};
// With resume (the completing pass), bins[t] is instead where the walk
// starts, from the pixel state the first pass left in the outputs.
struct PlanView {
    const uint8_t* bins = nullptr;
    uint8_t* flag = nullptr;
    int32_t* list = nullptr;
    int32_t* needed = nullptr;
    int resume = 0;
};
// the configured chunk size of the lazy EXACT raster
inline int chunk_cap(const gs_config& cfg) { return cfg.chunk_cap > 0 ? cfg.chunk_cap : 256; }
// The plain baseline raster kernel serves GLOBAL mode without the tile cull;
// every other configuration (GLOBAL with the cull included) uses the binned
// kernel, which culls at staging when the stream was not culled when built.
inline bool baseline_raster(const gs_config& cfg) { return cfg.mode == GS_MODE_GLOBAL_SORT && !cfg.tile_cull; }
// depth range with samples mapped to gids through the per-Gaussian offsets
int depth_range_goff(gs_ctx* ctx, const ProjView& pv, const float* scales, int64_t n, int64_t m_cap,
                     const int64_t* m_dev, const gs_camera* cam, cudaStream_t st);

// raster.cu
int raster_fwd(gs_ctx* ctx, const ProjView& pv, const gs_camera* cam, uint64_t* stream_words,
               const int32_t* offsets, int32_t stride, const float* bg, float* rgb, float* alpha,
               int32_t* last, int32_t* ntests, bool baseline, cudaStream_t st, float* final_T = nullptr,
               int32_t* tile_end = nullptr, const PlanView& plan = PlanView(), int32_t* warp_end = nullptr);
// the completing pass of a planned frame: every tile of list (device {count,
// tiles...}) composited on from the bin where its first pass stopped (plan
// [T]), from the pixel state that pass left in rgb / alpha / last (EXACT,
// repair in the raster); a persistent launch that returns at once when the
// list is empty
int raster_listed(gs_ctx* ctx, const ProjView& pv, const gs_camera* cam, uint64_t* stream_words,
                  const int32_t* offsets, int32_t stride, const float* bg, float* rgb, float* alpha, int32_t* last,
                  const uint8_t* plan, const int32_t* list, cudaStream_t st, float* final_T = nullptr,
                  int32_t* tile_end = nullptr);

// one EXACT (repair in the raster, 16x16 tiles) view of a batched raster
struct RasterView {
    ProjView pv;
    gs_camera cam;
    uint64_t* words;
    const int32_t* offsets;
    int32_t stride;
    float bg[3];
    int cull, cap;
    float* rgb;
    float* alpha;
    int32_t* last;
    int32_t gid_base;  // stream words hold gid_base + the view's gid (a batch group's shared records)
};
// all views' tiles in one persistent launch, longest tiles first
// (sched: 65 device int32; order: one int32 per tile of all views)
int raster_views(gs_ctx* ctx, const RasterView* views, int nv, int32_t* sched, int32_t* order, cudaStream_t st);

// raster_bwd.cu
int raster_bwd_prepare();
// tiles.cu
int bin_offsets_prepare();
int raster_bwd(gs_ctx* ctx, const ProjView& pv, const gs_camera* cam, const uint64_t* words, const int32_t* offsets,
               int32_t stride, const float* bg, const int32_t* last, const float* final_T,
               const int32_t* tile_end, const float* dl_drgb, const float* dl_dalpha, const GradView& gv,
               cudaStream_t st, const int32_t* warp_end = nullptr);

// ctx.cu: whole-frame pieces the batched render reuses
bool camera_ok(const gs_camera* cam);
int render_buffers(gs_ctx* c, int64_t n, int64_t m_cap, int32_t T);
int render_save_buffers(gs_ctx* c, int32_t W, int32_t H, int32_t T);
int planner_buffers(gs_ctx* c, int32_t T);
// planner.cu: features, class and first-pass bins of every tile of a binned
// stream in one launch (plan [T] bins; classes [T] nullable); also clears the
// completion flags (plan + T) and list (c->d_plist) of the frame
int plan_frame(gs_ctx* c, const int32_t* offsets, int32_t K, int32_t T, uint8_t* plan, uint8_t* classes,
               cudaStream_t st);
int render_after_project(gs_ctx* c, int64_t n, const float* scales, const gs_camera* cam, const float* bg,
                         float* d_rgb, float* d_alpha, int32_t* d_last, int32_t flags, cudaStream_t st);
// the frame up to the raster: intersect, sort or bin, repair (stream and
// offsets in c->r_stream, c->r_off)
int render_binning(gs_ctx* c, int64_t n, const float* scales, const gs_camera* cam, int32_t flags,
                   cudaStream_t st);

// project.cu
constexpr int kMaxBatchViews = GS_MAX_VIEWS;
int launch_project_batch(gs_ctx* ctx, const float* means, const float* scales, const float* quats,
                         const float* opac, const float* sh, int32_t sh_degree, int64_t n, int nviews,
                         const gs_camera* cams, const int* tiles, const ProjView* pvs, cudaStream_t st);

// batch_bins.cu: EXACT binning of a group of views as one frame of V n items
// (records of view v at items [v n, (v+1) n) of the group context's
// projected buffer); the view table is opaque here
struct GroupViews;
GroupViews* group_views_new();
void group_views_free(GroupViews* gv);
// fill the table for views of n Gaussians with cameras cams[0..nv) and bin
// counts K[0..nv); returns the group's total (tile, bin) segments
int64_t group_views_set(GroupViews* gv, int64_t n, int nv, const gs_camera* cams, const int32_t* K);
int64_t group_seg_base(const GroupViews* gv, int v);
int group_reserve(gs_ctx* gc, const GroupViews* gv, int64_t m_cap);
// intersect, depth range, bins and the long-segment sort of every view of the
// group (stream and offsets in gc->r_stream, gc->r_off); per-view entry
// counts copied to the pinned host array h_m_views [nv]
int group_binning(gs_ctx* gc, const GroupViews* gv, int32_t flags, int64_t* h_m_views, cudaStream_t st);

// batch.cu: per-context batch state (sub-contexts, streams, graph)
struct BatchState;
void batch_destroy(gs_ctx* c);
int batch_error(gs_ctx* c, cudaStream_t st);
int batch_clear_error(gs_ctx* c, cudaStream_t st);
int64_t batch_launch_count(const gs_ctx* c);  // kernels launched by the batch's sub-contexts

// grow every stage's internal scratch for (n, m_cap, T) (synchronous)
int reserve_internal(gs_ctx* ctx, int64_t n, int64_t m_cap, int32_t width, int32_t height);

// timing helpers
void stage_begin(gs_ctx* ctx, int stage, cudaStream_t st);
void stage_end(gs_ctx* ctx, int stage, cudaStream_t st);

}  // namespace gs
