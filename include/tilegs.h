/*
 * tilegs.h -- C ABI of libtilegs.so, the GB300 (sm_103a) TileGS forward path.
 *
 * The method is "TileGS: Tile-Local Depth Binning for Gaussian Splatting
 * Rasterization".  A frame runs:
 *   gs_project        -> per-Gaussian 2D mean / conic / depth / tile rect / colour
 *                        (Sec. 3.1, the method's projected inputs)
 *   gs_tile_intersect -> one entry per (Gaussian, covered tile)       (Sec. 3.1)
 *   gs_sort_or_bin    -> either the baseline global (tile, depth) sort (Sec. 3.1)
 *                        or depth-range estimation + tile-local bin construction
 *                        + selective repair (Sec. 3.2, 3.3, 3.5; supplement
 *                        algorithms 2-4), both producing a tile-major stream
 *   gs_rasterize_fwd  -> front-to-back compositing over each tile's span
 *                        (Sec. 3.4; supplement algorithm 5)
 *
 * Conventions for every entry point:
 *   - All array arguments are DEVICE pointers on the current CUDA device unless
 *     the name or comment says "host".  The caller owns them; the library never
 *     frees or retains them past the call.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  All work is enqueued asynchronously on it; nothing blocks the
 *     host unless the comment says so.
 *   - Return value: GS_OK or a GS_ERR_* code.  Argument errors are detected on
 *     the host before anything is enqueued.  Errors detected on the device
 *     (capacity overflow, a bounded wait that ran out) set the context's sticky
 *     error word, read by gs_get_error() after the stream has been synchronised.
 *   - A context is used by one host thread at a time; calls that share a
 *     context and overlap on different streams race on its scratch memory.
 *   - Floating point: float32 in a fixed operation order (no fast-math), so the
 *     integer decisions (tile rectangles, alpha skips, transmittance stops, bin
 *     indices) are reproducible bit for bit.
 */
#ifndef TILEGS_H
#define TILEGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
enum {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = 1, /* bad size, null pointer, unsupported option      */
    GS_ERR_CAPACITY = 2,    /* more entries than the caller's capacity; the
                               needed count is still written to the M output */
    GS_ERR_CUDA = 3,        /* a CUDA runtime call failed                     */
    GS_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up             */
    GS_ERR_NO_MEMORY = 5,   /* scratch allocation failed                      */
    GS_ERR_NUMERIC = 6      /* non-finite input where a finite one is needed  */
};
const char* gs_status_string(int status);

/* ---------------------------------------------------------------- modes */
enum {
    /* Baseline: global stable radix sort of (tile, depth) keys, one
     * contiguous range per tile (Sec. 3.1, "globally sorted tile-depth
     * stream").  Offsets stride K = 1. */
    GS_MODE_GLOBAL_SORT = 0,
    /* Tile-local depth bins with a monotone split map (bin order never
     * inverts depth order) and every segment of length >= 2 put in (depth,
     * gid) order: the stream is identical to GS_MODE_GLOBAL_SORT's. */
    GS_MODE_BINNED_EXACT = 1,
    /* The paper's default policy: near-depth-shifted log-space bins and the
     * five selection rules with the floor(0.25 M) entry budget (Sec. 3.5,
     * table of exact-repair selection rules).  Approximate by design. */
    GS_MODE_BINNED_PAPER = 2,
    /* Bins as in PAPER mode, no repair (the "No repair" row of the paper's
     * repair ablation). */
    GS_MODE_BINNED_NOREPAIR = 3
};

/* ---------------------------------------------------------------- camera */
typedef struct gs_camera {
    float viewmat[16];  /* row-major world-to-camera, OpenCV axes (x right, y down, z forward) */
    float fx, fy, cx, cy;
    int32_t width, height;
    float near_plane, far_plane; /* Gaussians with depth outside (near, far) are culled */
} gs_camera;

/* ---------------------------------------------------------------- config */
#define GS_MAX_K 128
#define GS_MAX_VIEWS 32 /* views of one gs_render_batch call */
/* bin planner network: 8 features -> 64 -> 64 -> 6 classes (ReLU, float32) */
#define GS_PLAN_FEATURES 8
#define GS_PLAN_HIDDEN 64
#define GS_PLAN_CLASSES 6
#define GS_PLAN_PARAMS (GS_PLAN_HIDDEN * GS_PLAN_FEATURES + GS_PLAN_HIDDEN + GS_PLAN_HIDDEN * GS_PLAN_HIDDEN + \
                        GS_PLAN_HIDDEN + GS_PLAN_CLASSES * GS_PLAN_HIDDEN + GS_PLAN_CLASSES)
typedef struct gs_config {
    int32_t mode;          /* GS_MODE_* */
    int32_t tile_size;     /* 8, 16 or 32 pixels (16 = the paper's) */
    int32_t K;             /* bins per tile, 1..GS_MAX_K (64 = paper default) */
    int32_t sample_count;  /* S, depth-range samples (8192) */
    float p_lo, p_hi;      /* percentiles of the depth range (1, 99) */
    float pad;             /* padding fraction of the clipped span (0.05) */
    float near_alpha, near_gamma; /* near-depth shift (1.0, 0.25) */
    float eps;             /* numerical floor (1e-4) */
    float repair_budget_frac; /* B_rep = floor(frac * M) (0.25) */
    int32_t near_shift;    /* 1: bin on z - min(alpha s_max, gamma z) (PAPER default) */
    int32_t tile_cull;     /* 1: conservative tile-level alpha cull in the binned raster
                              (default).  GLOBAL mode defaults to 0, the plain
                              baseline raster; GLOBAL with 1 rasters the global
                              stream with the binned kernel (tile cull at staging,
                              colour staging, per-warp masks, early-out): the
                              raster's additions without binning.  Same image. */
    int32_t persistent;    /* 1: binned raster runs persistent CTAs over tiles in
                              descending span order */
    int32_t repair_in_raster; /* EXACT only, 1 (default): gs_sort_or_bin sorts only
                              segments longer than 2048 entries and gs_rasterize_fwd
                              sorts each segment it reaches in shared memory just
                              before compositing it, so segments past every
                              pixel's termination are never sorted.  The image is
                              identical either way; with 0 the stream is fully
                              sorted by gs_sort_or_bin. */
    int32_t chunk_cap;     /* EXACT with repair_in_raster: the most entries of
                              consecutive bins the raster loads and sorts at once
                              (a tile's repair bins; a single longer segment of up
                              to 2048 forms one on its own); 32..2048, 0 = 256 */
    int32_t planner;       /* EXACT with repair_in_raster and the tile cull, 1: the
                              bin planner (an MLP over the tile's depth-bin
                              statistics, weights set with gs_planner_set_weights)
                              picks how many of each tile's K bins gs_render builds
                              in a first pass; tiles that do not terminate within
                              them are completed by a second pass.  0: every bin
                              in one pass.  Changes speed only, never the image. */
    int32_t wait_polls;    /* the most polls of a bounded device-side wait (the
                              projection's TMA copy of SH coefficients) before it
                              raises GS_ERR_TIMEOUT; gs_config_default sets
                              4194304.  0 makes every such wait give up at once
                              (a test of the error path): the error is raised, the
                              copy is still drained by a second bounded wait, and
                              the frame is written.  A block whose copy never
                              lands writes nothing: after GS_ERR_TIMEOUT the
                              frame's outputs are not valid. */
    float planner_quantile; /* the planner's decision: the smallest class whose
                              cumulative softmax probability reaches this value,
                              in (0, 1] (gs_config_default: 0.9) */
    int32_t pdl;           /* 1 (gs_config_default): the kernels of a frame are
                              launched with programmatic stream serialization, so
                              each one is set up while its predecessor drains
                              (every such kernel waits for its predecessor's
                              completion before it touches memory).  0: ordinary
                              launches.  Frames that record stage times
                              (gs_enable_timing) use ordinary launches.  Changes
                              speed only. */
} gs_config;

/* Fill *cfg with the paper's defaults (supplement, default No-GW configuration
 * and default repair-threshold tables) for the given mode.  EXACT mode turns
 * the near-depth shift off (it would make the bin map non-monotone). */
void gs_config_default(gs_config* cfg, int32_t mode);

/* ---------------------------------------------------------------- context */
typedef struct gs_ctx gs_ctx;

/* Create a context on the current CUDA device.  Owns scratch memory (grown on
 * demand with cudaMalloc, so never grow it inside a stream capture: call
 * gs_reserve first), a device error word and timing events.
 * Errors: GS_ERR_INVALID_ARG (cfg out of range), GS_ERR_NO_MEMORY. */
int gs_create(gs_ctx** out, const gs_config* cfg);
int gs_destroy(gs_ctx* ctx);
int gs_set_config(gs_ctx* ctx, const gs_config* cfg);
int gs_get_config(const gs_ctx* ctx, gs_config* cfg);

/* Pre-grow scratch for up to n Gaussians, m_cap entries and an image of
 * width x height (synchronous; allocates).  The reserved capacity also picks
 * the EXACT path's bin scatter (Alg. 3): from 8192 reserved entries per tile
 * the row records are grouped by (tile row, bin) and the slots taken with
 * shared-memory atomics (deep frames), which needs 16 more bytes of scratch
 * per reserved entry; below that, one global atomic per entry.  Both give the
 * same stream up to the order inside each (tile, bin) segment, which the
 * repair sorts. */
int gs_reserve(gs_ctx* ctx, int64_t n, int64_t m_cap, int32_t width, int32_t height);

/* Sticky device error word (synchronises `stream` first; host).  Returns the
 * first GS_ERR_* raised on the device since the last gs_clear_error. */
int gs_get_error(gs_ctx* ctx, void* stream);
int gs_clear_error(gs_ctx* ctx, void* stream);

/* Per-stage device times of the last gs_render / gs_sort_or_bin call when
 * timing is enabled (host; synchronises).  ms[] receives GS_STAGE_COUNT values. */
enum { GS_STAGE_PROJECT = 0, GS_STAGE_INTERSECT, GS_STAGE_DEPTH_RANGE, GS_STAGE_BIN,
       GS_STAGE_REPAIR, GS_STAGE_SORT, GS_STAGE_RASTER,
       GS_STAGE_COMPLETE, /* a planned frame's second pass (cfg.planner) */
       GS_STAGE_COUNT };
int gs_enable_timing(gs_ctx* ctx, int32_t on);
int gs_get_stage_times(gs_ctx* ctx, float* ms);

/* ---------------------------------------------------------------- layouts */
/*
 * Projected buffer (caller-owned, gs_projected_bytes(n) bytes, 256-byte
 * aligned base).  Structure of arrays, each field 256-byte aligned at the
 * offset gs_projected_offset(n, field):
 *   GS_P_XY_AB   float4[n]  {mean_x, mean_y, conic_a, conic_b}
 *   GS_P_C_O_Z   float4[n]  {conic_c, opacity, depth, cull_tau}
 *   GS_P_RGB     float4[n]  {r, g, b, cull_margin}
 *   GS_P_RECT    uint2[n]   {tx0 | ty0 << 16, tx1 | ty1 << 16} (tiles tx0 <= tx < tx1)
 *   GS_P_RADIUS  int32[n]   pixel radius, 0 = culled
 * conic (a, b, c) is the upper triangle of the inverse 2D covariance;
 * cull_tau / cull_margin feed the conservative tile cull (ln(255 o) and a
 * rounding margin); a culled Gaussian has an empty rect.
 */
enum { GS_P_XY_AB = 0, GS_P_C_O_Z, GS_P_RGB, GS_P_RECT, GS_P_RADIUS, GS_P_NFIELDS };
size_t gs_projected_bytes(int64_t n);
size_t gs_projected_offset(int64_t n, int32_t field);

/*
 * Intersection buffer (caller-owned, gs_isect_bytes(m_cap) bytes): three
 * uint32 arrays of m_cap entries at offsets 0, m_cap*4 and m_cap*8 (rounded to
 * 256 bytes by gs_isect_bytes): tile id (ty * tiles_x + tx), depth bits
 * (float bits of the positive depth, so integer order is depth order) and
 * Gaussian id.  Emission order: gid ascending, then ty, then tx.
 */
size_t gs_isect_bytes(int64_t m_cap);
size_t gs_isect_offset(int64_t m_cap, int32_t field); /* field 0 tile, 1 zbits, 2 gid */

/* Tiles of an image: ceil(width / tile) * ceil(height / tile). */
int32_t gs_num_tiles(int32_t width, int32_t height, int32_t tile_size);

/* ---------------------------------------------------------------- stages */

/*
 * Project n Gaussians (Sec. 3.1; the projection is the 3DGS/EWA one, which
 * the paper leaves unchanged).
 *   means [n,3], scales [n,3] (linear, already activated), quats [n,4]
 *   (w,x,y,z, any non-zero norm), opacities [n] (in [0,1]), sh [n,(d+1)^2,3]
 *   with d = sh_degree in 0..3; cam is a HOST struct.
 * Writes the projected buffer.  Errors: GS_ERR_INVALID_ARG.
 */
int gs_project(gs_ctx* ctx, const float* means, const float* scales, const float* quats,
               const float* opacities, const float* sh, int32_t sh_degree, int64_t n,
               const gs_camera* cam, void* projected, void* stream);

/*
 * Tile intersection (Sec. 3.1: "emits one tile-intersection record per
 * covered tile").  Counts the tiles of every projected Gaussian, scans them
 * and emits entries into `isect` (capacity m_cap).
 *   m_dev: device int64 receiving M (always written, even past capacity).
 *   m_host: optional HOST pointer; when non-NULL the call synchronises the
 *           stream and writes M there.
 * When M > m_cap nothing past m_cap is written and GS_ERR_CAPACITY is raised
 * (returned directly when m_host is given, else via gs_get_error).
 */
int gs_tile_intersect(gs_ctx* ctx, const void* projected, int64_t n, const gs_camera* cam,
                      void* isect, int64_t m_cap, int64_t* m_dev, int64_t* m_host,
                      void* stream);

/*
 * Order the entries into a tile-major stream, per the context's mode.
 *   stream_words [m_cap] uint64: (depth_bits << 32) | gid.
 *   offsets [T*K' + 1] int32 with K' = 1 in GLOBAL mode, K' = cfg.K otherwise:
 *     tile t's span is [offsets[t*K'], offsets[(t+1)*K']), bin b of tile t is
 *     [offsets[t*K'+b], offsets[t*K'+b+1]).
 * GLOBAL: stable LSD radix sort on (tile, depth bits); ties keep gid order.
 * BINNED_*: depth range (supplement algorithm 2) -> count / scan / scatter
 *   (algorithm 3) -> repair (algorithm 4; EXACT sorts every segment).
 * `scales` [n,3] is read only when the near-depth shift is on.
 * zrange_out: optional device float[2] receiving [zmin, zmax] (binned modes).
 */
int gs_sort_or_bin(gs_ctx* ctx, const void* projected, const float* scales, int64_t n,
                   const gs_camera* cam, const void* isect, int64_t m_cap, const int64_t* m_dev,
                   uint64_t* stream_words, int32_t* offsets, float* zrange_out, void* stream);

/*
 * The binned path's steps one at a time (for inspection and tests).
 * gs_depth_range: writes zrange[2] = [zmin, zmax] (supplement algorithm 2).
 * gs_bin_build: count / exclusive scan / atomic scatter into bins (algorithm
 *   3) given zrange; the order inside a segment is unspecified.
 * gs_repair: selected_out (optional device uint8 [T*K]) receives the segments
 *   sorted: all with length >= 2 (EXACT) or the rule/budget selection (PAPER,
 *   algorithm 4); NOREPAIR sorts nothing.
 */
int gs_depth_range(gs_ctx* ctx, const void* projected, const float* scales, int64_t n,
                   const gs_camera* cam, const void* isect, int64_t m_cap, const int64_t* m_dev,
                   float* zrange, void* stream);
int gs_bin_build(gs_ctx* ctx, const void* projected, const float* scales, int64_t n,
                 const gs_camera* cam, const void* isect, int64_t m_cap, const int64_t* m_dev,
                 const float* zrange, uint64_t* stream_words, int32_t* offsets, void* stream);
int gs_repair(gs_ctx* ctx, const gs_camera* cam, const int64_t* m_dev, uint64_t* stream_words,
              const int32_t* offsets, uint8_t* selected_out, void* stream);

/*
 * gs_depth_range without a context and without allocating anything (the
 * paper has no counterpart: this is a deployment variant of gs_depth_range).
 * For callers that cannot call cudaMalloc -- an application whose device
 * memory belongs to its own allocator or fixed budget and that passes this
 * library only pre-allocated buffers, or code that must not set off
 * cudaMalloc's implicit device synchronisation while other work runs.
 *   cfg: HOST config (mode-independent fields: sample_count, p_lo, p_hi, pad,
 *        near_shift / near_alpha / near_gamma, eps, K); other arguments and
 *        the result zrange[2] as for gs_depth_range.
 * Scratch: one 536-byte bin-parameter record in a file-scope static
 * __device__ array, held by every GPU that loads the library until exit.  Its
 * limit: K <= GS_MAX_K (128) split depths and sample_count <= 8192; larger
 * values return GS_ERR_INVALID_ARG before anything is enqueued.
 * The first call on each device resolves the scratch address with
 * cudaGetSymbolAddress (and so does the first call after the device's context
 * changed, e.g. after cudaDeviceReset); make that first call before any stream
 * capture.  Calls neither cudaMalloc nor cudaFree nor any other allocating
 * routine.  All calls share the scratch, which keeps the last call's contents
 * (each call rewrites every field it reads), so calls that overlap on the GPU
 * race.
 */
int gs_depth_range_noalloc(const gs_config* cfg, const void* projected, const float* scales, int64_t n,
                           const gs_camera* cam, const void* isect, int64_t m_cap, const int64_t* m_dev,
                           float* zrange, void* stream);

/*
 * Front-to-back compositing of each tile's span (Sec. 3.4; supplement
 * algorithm 5).  Per pixel centre (x + 0.5, y + 0.5) and entry g in stream
 * order: q = 1/2 d^T conic d, alpha = min(0.99, o exp(-q)), skip alpha < 1/255,
 * stop before applying when T (1 - alpha) < 1e-4, C += c alpha T, T *= 1 - alpha.
 *   n: the Gaussian count the projected buffer was laid out for.
 *   offsets_stride: 1 for a GLOBAL stream, cfg.K for a binned one.
 *   bg: HOST float[3].  rgb [H,W,3], alpha [H,W] (= 1 - T), last [H,W] (id of
 *   the last applied Gaussian, -1 if none); ntests [H,W] optional: entries
 *   each pixel visited, the stopping one included.
 *   final_T [H,W] and tile_end [T] (both optional, for gs_rasterize_bwd): the
 *   final transmittance T of each pixel (exact; alpha = 1 - T is rounded),
 *   and per tile the stream index at which its compositing ended (the span
 *   end, or the position in compositing order where every pixel of the tile
 *   had stopped).  With tile_end, an EXACT stream whose repair runs in the
 *   raster is modified in place: the segments the raster sorted are stored
 *   back sorted, so [span start, tile_end) of every tile is left in
 *   (depth, gid) order (the stream stays valid for any later raster).
 * stream_words is only read otherwise.
 * The GLOBAL kernel is the plain baseline (gsplat-style batch staging); the
 * binned kernel adds the conservative tile-alpha cull and colour staging of
 * the paper's default configuration.  Both give identical images.
 */
int gs_rasterize_fwd(gs_ctx* ctx, const void* projected, int64_t n, const gs_camera* cam,
                     uint64_t* stream_words, const int32_t* offsets, int32_t offsets_stride,
                     const float* bg, float* rgb, float* alpha, int32_t* last, int32_t* ntests,
                     float* final_T, int32_t* tile_end, void* stream);

/*
 * Backward of gs_rasterize_fwd: the gradient of a loss L(rgb, alpha) w.r.t.
 * the projected 2D parameters.  The paper has no backward (Sec. 7 leaves it
 * to future work and asks that it follow the forward's compositing order);
 * this one walks each tile's span in the forward's order reversed, from the
 * forward's tile_end back to the span start, for the same stream (as the
 * forward that saved tile_end left it: composited prefixes sorted), offsets
 * and context configuration, and differentiates
 *   rgb = sum_i c_i a_i T_i + T_N bg,  alpha = 1 - T_N,
 *   a_i = min(0.99, o_i exp(-q_i)),  q_i = 1/2 d^T conic d,  d = mean - centre
 * over the entries the forward applied (its float32 skip tests are repeated
 * bit for bit; T_i is recovered from the saved final T as T_{i+1}/(1 - a_i);
 * a clamped a_i passes no gradient to o_i or q_i).
 *   bg: HOST float[3], the forward's.  last, final_T, tile_end: the forward's
 *   outputs for these inputs.
 *   dl_drgb [H,W,3], dl_dalpha [H,W] (nullable: 0): dL/drgb, dL/dalpha.
 *   grad: caller-owned, 256-byte aligned, gs_grad2d_bytes(n) bytes, zeroed
 *   and then written; field f at gs_grad2d_offset(n, f):
 *     0  float4[n] {dL/dmean_x, dL/dmean_y, dL/dconic_a, dL/dconic_b}
 *     1  float4[n] {dL/dconic_c, dL/dopacity, 0, 0}
 *     2  float4[n] {dL/dr, dL/dg, dL/db, 0}
 *   (the same element layout as the projected fields GS_P_XY_AB, GS_P_C_O_Z
 *   and GS_P_RGB; conic = (a, b, c) of q = 1/2 (a dx^2 + 2 b dx dy + c dy^2)).
 * Sums over pixels use float atomics: results are reproducible to rounding,
 * not bitwise.  Errors: GS_ERR_INVALID_ARG (null pointers, bad stride,
 * misaligned grad), GS_ERR_CUDA.
 */
size_t gs_grad2d_bytes(int64_t n);
size_t gs_grad2d_offset(int64_t n, int32_t field);
int gs_rasterize_bwd(gs_ctx* ctx, const void* projected, int64_t n, const gs_camera* cam,
                     const uint64_t* stream_words, const int32_t* offsets, int32_t offsets_stride,
                     const float* bg, const int32_t* last, const float* final_T, const int32_t* tile_end,
                     const float* dl_drgb, const float* dl_dalpha, void* grad, void* stream);

/*
 * The reciprocal the backward uses to recover transmittances,
 * T_i = T_{i+1} * (1 / (1 - a_i)): out[i] = 1 / x[i] by the hardware's
 * approximate reciprocal refined by one Newton-Raphson step (Markstein's
 * FMA form), within one rounding of the exact value for x in [2^-126, 2^126]
 * (the backward's arguments lie in [0.01, 1)).  x, out: n device floats
 * (caller-owned).  Exposed so that its error can be checked.  Errors:
 * GS_ERR_INVALID_ARG (n < 0, null pointers), GS_ERR_CUDA.
 */
int gs_reciprocal(const float* x, float* out, int64_t n, void* stream);

/*
 * gs_rasterize_fwd as one pass of a planned frame (EXACT with repair_in_raster):
 *   plan [T] (nullable: every bin): the number of bins, from each tile's
 *   front, that this pass walks (values above K count as K).
 *   flags [T] (nullable): set to 1 for each tile that has a pixel still
 *   compositing when its planned bins end while later bins hold entries (it
 *   must be composited again over all its bins), 0 otherwise.
 *   bins_needed [T] (nullable; requires plan == NULL): the bins each tile
 *   needs, 1 + the bin holding the last entry any of its pixels visits (the
 *   stopping entry, or the span's last for a pixel that never stops); 0 for
 *   an empty tile.  A plan with plan[t] >= bins_needed[t] flags no tile.
 * Other arguments as gs_rasterize_fwd.  Pixels of tiles that are not flagged
 * are final.  With flags, a flagged tile's pixels hold the pass's state for
 * the completing pass: C (no background) in rgb, T in alpha (negative once
 * the pixel has stopped), last.
 */
int gs_rasterize_fwd_plan(gs_ctx* ctx, const void* projected, int64_t n, const gs_camera* cam,
                          uint64_t* stream_words, const int32_t* offsets, int32_t offsets_stride,
                          const float* bg, float* rgb, float* alpha, int32_t* last, const uint8_t* plan,
                          uint8_t* flags, int32_t* bins_needed, void* stream);

/* ---------------------------------------------------------------- bin planner */
/*
 * The learned bin planner (the paper uses one bin count and spacing for every
 * tile, Sec. 5.3, and leaves distribution-dependent settings to future work,
 * Sec. 7).  Per tile, an MLP maps 8 statistics of the tile's K depth-bin
 * counts to a class c: class c < 5 gives the tile's first pass the fewest
 * bins from its front that hold at least 64 << c entries, class 5 all K.
 * The class is the smallest whose cumulative softmax probability reaches
 * cfg.planner_quantile.  The image never changes (gs_render completes every
 * tile the first pass leaves unfinished).
 *
 * gs_tile_features: features [T][GS_PLAN_FEATURES] (device) of a binned
 *   stream's offsets (stride = K): log1p(n), log1p(max bin), nonempty/K,
 *   first/K, last/K, log1p(first bin count), log1p(entries in the K/8 bins
 *   from the first nonempty one), log1p(n/nonempty).
 * gs_planner_set_weights: GS_PLAN_PARAMS floats (host or device; NULL turns
 *   the planner off), packed W1[64][8] b1 W2[64][64] b2 W3[6][64] b3.
 * gs_plan_tiles: from a binned stream's offsets, plan [T] = each tile's
 *   first-pass bins and classes [T] (nullable) = its class (device).
 * Training kernels (device buffers, batch B):
 *   gs_mlp_forward: acts [B][128] = (h1, h2), logits [B][6];
 *   gs_mlp_loss_grad: mean softmax cross entropy into loss[0] and its
 *   gradient dlogits [B][6] for labels [B] in 0..5;
 *   gs_mlp_backward: deltas [B][128] scratch, grads [GS_PLAN_PARAMS] (overwritten);
 *   gs_adam_step: one Adam update (Kingma & Ba) with bias correction, step >= 1.
 */
int gs_tile_features(gs_ctx* ctx, const gs_camera* cam, const int32_t* offsets, int32_t stride, float* features,
                     void* stream);
int gs_planner_set_weights(gs_ctx* ctx, const float* params, void* stream);
int gs_plan_tiles(gs_ctx* ctx, const gs_camera* cam, const int32_t* offsets, int32_t stride, uint8_t* plan,
                  uint8_t* classes, void* stream);
int gs_mlp_forward(const float* params, const float* X, int32_t B, float* acts, float* logits, void* stream);
int gs_mlp_loss_grad(const float* logits, const int32_t* labels, int32_t B, float* dlogits, float* loss,
                     void* stream);
int gs_mlp_backward(const float* params, const float* X, const float* acts, const float* dlogits, int32_t B,
                    float* deltas, float* grads, void* stream);
int gs_adam_step(float* params, const float* grads, float* m, float* v, int32_t n, float lr, float beta1,
                 float beta2, float eps, int32_t step, void* stream);

/* ---------------------------------------------------------------- scene order */
/*
 * Raster-order-aware storage (the geometry-layout direction of Sec. 6.2,
 * where per-Gaussian attribute gathers dominate the raster's memory traffic):
 * a once-per-scene permutation putting the Gaussians in the Z-order (Morton
 * order) of their means, so the Gaussians a tile composites lie close together
 * in every per-Gaussian array.  The order, in float32 with one correctly
 * rounded operation per step:
 *   lo_a = min_i x_ia, hi_a = max_i x_ia (a = x, y, z over all n means),
 *   s_a = 1024 / (hi_a - lo_a), or 0 when hi_a == lo_a,
 *   c_a = min(1023, trunc((x_ia - lo_a) * s_a)),
 *   code = OR over k < 10 of bit_k(c_x) << 3k | bit_k(c_y) << 3k+1 | bit_k(c_z) << 3k+2,
 *   perm = the gids 0..n-1 stably sorted by code (ties keep gid order).
 * gs_spatial_order: means [n][3] (device, finite) -> perm [n] int32 (device,
 *   caller-owned): position i of the reordered scene holds Gaussian perm[i].
 *   Context scratch grows to ~20 n bytes (allocates outside capture).
 * gs_gather_rows: dst[i][0..width) = src[perm[i]][0..width) for float rows
 *   (device; dst must not alias src).  A perm value outside [0, n) skips
 *   its row and sets GS_ERR_INVALID_ARG in the device error word.
 * Rendering the permuted scene gives the original image wherever no two
 * Gaussians of a tile have bit-identical depths (ties follow the new gids).
 */
int gs_spatial_order(gs_ctx* ctx, const float* means, int64_t n, int32_t* perm, void* stream);
int gs_gather_rows(gs_ctx* ctx, const int32_t* perm, int64_t n, const float* src, int32_t width, float* dst,
                   void* stream);

/* ---------------------------------------------------------------- whole frame */
typedef struct gs_scene {
    const float* means;
    const float* scales;
    const float* quats;
    const float* opacities;
    const float* sh;
    int32_t sh_degree;
    int64_t n;
} gs_scene;

enum {
    GS_RENDER_HOST_INPUTS = 1,  /* scene arrays are HOST memory (pinned for async copies) */
    GS_RENDER_HOST_OUTPUTS = 2, /* rgb/alpha/last are HOST memory */
    GS_RENDER_NO_SYNC = 4,      /* do not read M back: use reserved capacity only */
    GS_RENDER_SAVE = 16,        /* also keep, in the context, what gs_render_bwd needs:
                                   the final transmittance and per-tile end of this
                                   frame (the projected record, stream and offsets
                                   stay in the context until the next gs_render) */
    GS_RENDER_GRAPH = 8,        /* device buffers only: capture the frame's launches
                                   into a CUDA graph on the first call and replay it
                                   on later calls with identical arguments (pointers,
                                   sizes, camera, background, config); implies
                                   NO_SYNC, so capacity must be reserved first
                                   (gs_reserve or one plain gs_render), and
                                   needs a non-default stream */
    GS_RENDER_PIPELINE = 32     /* with HOST_INPUTS and HOST_OUTPUTS: the call
                                   returns once its copies and its frame are
                                   enqueued, and consecutive calls overlap -- the
                                   scene upload of one call with the frame and the
                                   image download of the one before (see
                                   gs_render_wait) */
};

/*
 * One whole frame: project -> intersect -> sort_or_bin -> rasterize, with all
 * intermediates in context scratch.  With GS_RENDER_HOST_* the copies run on
 * `stream` inside the call and the call returns after the outputs landed.
 * Without GS_RENDER_NO_SYNC the entry count is read back once to grow scratch.
 * last may be NULL.  Errors: as the stages.
 */
int gs_render(gs_ctx* ctx, const gs_scene* scene, const gs_camera* cam, const float* bg,
              float* rgb, float* alpha, int32_t* last, int32_t flags, void* stream);

/*
 * Pipelined host-buffer frames (GS_RENDER_PIPELINE | GS_RENDER_HOST_INPUTS |
 * GS_RENDER_HOST_OUTPUTS; implies GS_RENDER_NO_SYNC).  The context keeps two
 * slots of device inputs and outputs and two streams of its own, one for
 * uploads and one for downloads; calls alternate between the slots.  A call
 * enqueues its scene upload on the upload stream (after the frame two calls
 * back has finished reading that slot), its frame on `stream` (after its
 * upload, and after the download two calls back has emptied the slot's
 * outputs), and its image download on the download stream (after its frame),
 * then returns: the host link moves the next scene while this frame renders
 * and the previous image comes back.  Every call still copies all its inputs
 * in and all its outputs out.  Until gs_render_wait returns, the caller keeps
 * the host inputs of every pipelined call unchanged and reads none of their
 * host outputs.  All pipelined calls use the same `stream`; entry capacity
 * must have been reserved (gs_reserve or one gs_render without NO_SYNC);
 * an overflow is reported in the sticky error word (gs_get_error), as for
 * any NO_SYNC frame; gs_last_entry_count is not updated.  Errors:
 * GS_ERR_INVALID_ARG when a host flag is missing, with GS_RENDER_SAVE or
 * GS_RENDER_GRAPH, or before capacity was reserved; GS_ERR_NO_MEMORY;
 * GS_ERR_CUDA.
 *
 * gs_render_wait (host): returns once every pipelined call made so far on
 * this context has finished, its outputs in host memory.  GS_OK, or
 * GS_ERR_CUDA when a copy or the frame failed.  Also GS_OK when no pipelined
 * call was made.
 */
int gs_render_wait(gs_ctx* ctx);

/*
 * Backward of the last gs_render on this context, which must have had
 * GS_RENDER_SAVE: gs_rasterize_bwd over that frame's projected record,
 * stream, offsets, last ids, final transmittance and tile ends, with its
 * camera and background.  dl_drgb [H,W,3], dl_dalpha [H,W] (nullable) as for
 * gs_rasterize_bwd; grad: gs_grad2d_bytes(n) bytes for that frame's n,
 * 256-byte aligned, zeroed and written.  Errors: GS_ERR_INVALID_ARG (no saved
 * frame, null or misaligned pointers), GS_ERR_CUDA.
 */
int gs_render_bwd(gs_ctx* ctx, const float* dl_drgb, const float* dl_dalpha, void* grad, void* stream);

/*
 * Several views of one scene in one call (the paper renders single views; this
 * is the batched form a training or serving system needs).  Every view runs
 * the whole-frame pipeline of gs_render in its own sub-context of ctx, with
 * the configuration set for it by gs_batch_set_view_config / gs_batch_autotune
 * (default: ctx's): one projection launch serves all views (each Gaussian is
 * read once and projected n_cams times), then each view's intersect / bin /
 * repair / raster runs on its own stream, forked from and joined back into
 * `stream`.
 *   cams: HOST array [n_cams], 1 <= n_cams <= GS_MAX_VIEWS.
 *   rgb, alpha: HOST arrays [n_cams] of DEVICE pointers ([H_v,W_v,3], [H_v,W_v]);
 *   last: HOST array of DEVICE pointers (nullable array; null entries: not
 *   written).  bg: HOST float[3].  Device scene arrays only.
 *   flags: GS_RENDER_NO_SYNC (no entry-count readback; capacity from earlier
 *   calls), GS_RENDER_GRAPH (device buffers, non-default stream: the whole
 *   batch is captured once and replayed while the arguments are unchanged;
 *   every view must have been sized by an earlier call without NO_SYNC).
 *   Host-buffer, pipelined and SAVE flags are rejected.
 * Each view's image is the one gs_render gives for that camera and the view's
 * configuration.  Errors: as gs_render; GS_ERR_INVALID_ARG for bad counts.
 */
int gs_render_batch(gs_ctx* ctx, const gs_scene* scene, const gs_camera* cams, int32_t n_cams, const float* bg,
                    float* const* rgb, float* const* alpha, int32_t* const* last, int32_t flags, void* stream);

/* Configuration of batch view `view` (0 <= view < GS_MAX_VIEWS); cfg NULL
 * resets it to the context's. */
int gs_batch_set_view_config(gs_ctx* ctx, int32_t view, const gs_config* cfg);
int gs_batch_get_view_config(gs_ctx* ctx, int32_t view, gs_config* cfg);

/* Entry count of view `view` in the last gs_render_batch (host; valid after
 * the stream synchronises; -1 if the view does not exist). */
int64_t gs_batch_last_entry_count(gs_ctx* ctx, int32_t view);

/*
 * Choose each view's tile size (8, 16, 32; only when tune_tile != 0) and bin
 * count K (32, 64, 128; binned modes) by timing `iters` whole frames of that
 * view for every candidate (CUDA events on `stream`, synchronous), and set
 * them with gs_batch_set_view_config.  best_ms: HOST [n_cams] (nullable), the
 * chosen candidates' mean frame times.  With tune_tile, when a view's
 * fastest tile size is not 16 (so it would leave the group of views binned
 * and rasterised together), the assignment of each view's fastest candidate
 * and that of each view's fastest 16 x 16 candidate are also timed as whole
 * batches (`iters` gs_render_batch calls each) and the faster is kept.  K
 * never changes an EXACT image; the tile size can, for Gaussians that reach
 * alpha >= 1/255 outside their 3-sigma square (opacity above ~0.35), because
 * their tile rectangles differ.  Allocates (temporary contexts and output
 * buffers).
 */
int gs_batch_autotune(gs_ctx* ctx, const gs_scene* scene, const gs_camera* cams, int32_t n_cams,
                      int32_t tune_tile, int32_t iters, float* best_ms, void* stream);

/* Tiles the last planned gs_render (cfg.planner) left to its second pass
 * (host; synchronises `stream`); 0 without a planned frame, -1 on error. */
int32_t gs_last_flagged_tiles(gs_ctx* ctx, void* stream);

/* Entry count of the last gs_render (host; valid after the stream synchronises). */
int64_t gs_last_entry_count(gs_ctx* ctx);

/* Number of CUDA kernels this context (and its batch sub-contexts) has
 * launched so far (host counter). */
int64_t gs_launch_count(const gs_ctx* ctx);

/* Float32 operations of the compositing definition executed by the last
 * gs_rasterize_fwd call that passed an ntests buffer (host; synchronises):
 * 8 per visit, +17 when exp is evaluated, +3 when alpha passes, +4 when the
 * entry is applied.  -1 on error. */
int64_t gs_last_raster_ops(gs_ctx* ctx, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TILEGS_H */
