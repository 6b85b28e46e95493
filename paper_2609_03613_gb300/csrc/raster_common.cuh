// raster_common.cuh -- what the forward raster (raster.cu) and its backward
// (raster_bwd.cu) share: the batch staging of a tile's entries into shared
// memory (with the conservative tile-alpha cull and the per-warp strip mask)
// and the walk over a tile's span -- either the whole span at once, or, for
// EXACT streams whose repair runs in the raster, chunk by chunk with each
// segment of 2..kRasterSortCap entries sorted in shared memory by (depth bits,
// gid) right before it is composited (Sec. 3.5 selective repair; supplement,
// binned raster traversal after repair).  A forward that saves its state for
// the backward stores the sorted chunks back, so the backward walks the same
// order in place.
#pragma once
#include "device.cuh"

namespace gs {

struct RasterArgs {
    int width, height, tiles_x, n_tiles, stride;
    float bg0, bg1, bg2;
    int32_t gid_base = 0;  // stream words hold gid_base + gid (the last-id output subtracts it)
};

template <int TILE, bool BASELINE>
struct RasterShared {
    static constexpr int BS = TILE * TILE;
    static constexpr int BATCH = BS < 256 ? BS : 256;  // entries staged per batch
    static constexpr int NW = BATCH / 32;              // warps that load a batch
    static constexpr int NWT = BS / 32;                // warps of the tile
    float4 a[BATCH];                       // {mx, my, a/2, b}
    float4 b[BATCH];                       // {c/2, o, tau, gid bits}
    float4 c[BASELINE ? 1 : BATCH];        // colour (binned)
    uint32_t g[BASELINE ? BATCH : 1];      // gid (baseline colour lookup)
    uint8_t list[BASELINE ? 1 : NWT][BASELINE ? 1 : BATCH];  // per warp: staged entries its warp mask admits
};

// The staged entries (of cnt) whose warp mask admits the calling warp, in
// stage order, into sh.list[warp]; returns their count.  Whole warp.
template <int TILE>
__device__ __forceinline__ int warp_strip_list(RasterShared<TILE, false>& sh, int cnt)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int nw = 0;
    for (int j0 = 0; j0 < cnt; j0 += 32) {
        const int j = j0 + lane;
        const bool mine = j < cnt && ((__float_as_uint(sh.c[j].w) >> warp) & 1u);
        const unsigned bal = __ballot_sync(0xffffffffu, mine);
        if (mine) sh.list[warp][nw + __popc(bal & ((1u << lane) - 1u))] = (uint8_t)j;
        nw += __popc(bal);
    }
    __syncwarp();
    return nw;
}

// A warp owns an 8 x 4 pixel block of the tile: blocks are laid out TILE/8
// wide and TILE/4 tall (16x16: 2 x 4 blocks for the 8 warps; 8x8: 1 x 2;
// 32x32: 4 x 8), lanes row-major inside the block.
template <int TILE>
struct WarpBlocks {
    static constexpr int COLS = TILE / 8, ROWS = TILE / 4;
    static_assert(COLS * ROWS == TILE * TILE / 32, "one 8x4 block per warp");
    __device__ static int lx() { return ((threadIdx.x >> 5) % COLS) * 8 + (threadIdx.x & 7); }
    __device__ static int ly() { return ((threadIdx.x >> 5) / COLS) * 4 + ((threadIdx.x & 31) >> 3); }
};

// Warp mask of an entry: bit w is set when the entry's alpha >= 1/255
// ellipse (the tile cull's bound Q(d) <= tau / margin, d = mean - pixel
// centre, widened as there) reaches a pixel centre of warp w's 8 x 4 block of
// the tile (origin x0, y0).  Per band of four pixel rows the ellipse's
// x-extent over the band's centre rows (the row-span geometry of the bin
// stage: band ends and the ellipse's leftmost / rightmost points) is widened
// by 5e-3 relative + 0.05 px and tested against each block's centre columns,
// so a warp never skips a pixel the entry can reach.  The geometry takes the
// hardware's approximate division and square root (relative errors near
// 2^-22, far inside the widening).
template <int TILE>
__device__ __forceinline__ uint32_t strip_mask(float mx, float my, float ha, float hb, float hc, float tau,
                                               float margin, float x0, float y0)
{
    using WB = WarpBlocks<TILE>;
    constexpr int NWT = TILE * TILE / 32;
    const uint32_t all = NWT >= 32 ? 0xffffffffu : ((1u << NWT) - 1u);
    if (!(margin > 0.0f)) return all;
    const float D = 4.0f * ha * hc - hb * hb;
    const float tp = __fdividef(tau, margin);
    if (!(D > 0.0f) || !(tp > 0.0f)) return all;
    const float a4tp = 4.0f * ha * tp;
    const float iD = __fdividef(1.0f, D);
    float dymax, ext;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(dymax) : "f"(a4tp * iD));
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(ext) : "f"(4.0f * hc * tp * iD));
    dymax = dymax * (1.0f + 5e-3f) + 0.05f;
    const float dyl = hb * ext * __fdividef(1.0f, 2.0f * hc);  // dy of the leftmost point (dx = -ext)
    const float inv2ha = __fdividef(1.0f, 2.0f * ha);
    uint32_t m = 0u;
#pragma unroll
    for (int by = 0; by < WB::ROWS; ++by) {
        float yl = my - (y0 + (float)(4 * by) + 3.5f), yh = my - (y0 + (float)(4 * by) + 0.5f);
        yl = yl - (0.05f + 5e-3f * fabsf(yl));
        yh = yh + (0.05f + 5e-3f * fabsf(yh));
        const float ya = fmaxf(yl, -dymax), yb = fminf(yh, dymax);
        if (ya > yb) continue;  // the band misses the ellipse
        float s_a, s_b;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(s_a) : "f"(fmaxf(0.0f, a4tp - D * ya * ya)));
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(s_b) : "f"(fmaxf(0.0f, a4tp - D * yb * yb)));
        const float La = (-hb * ya - s_a) * inv2ha, Lb = (-hb * yb - s_b) * inv2ha;
        const float Ra = (-hb * ya + s_a) * inv2ha, Rb = (-hb * yb + s_b) * inv2ha;
        float dxmin = (dyl >= ya && dyl <= yb) ? -ext : fminf(La, Lb);
        float dxmax = (-dyl >= ya && -dyl <= yb) ? ext : fmaxf(Ra, Rb);
        dxmin = dxmin - (0.05f + 5e-3f * fabsf(dxmin));
        dxmax = dxmax + (0.05f + 5e-3f * fabsf(dxmax));
        // pixel centres x with mx - x in [dxmin, dxmax]
        const float xlo = mx - dxmax - x0, xhi = mx - dxmin - x0;
#pragma unroll
        for (int bx = 0; bx < WB::COLS; ++bx)
            if (xlo <= (float)(8 * bx) + 7.5f && xhi >= (float)(8 * bx) + 0.5f) m |= 1u << (by * WB::COLS + bx);
    }
    return m & all;
}

// The staged record of binned entry g from its projected fields p = xy_ab[g],
// q = c_o_z[g] and colour c = rgbv[g]: {mx, my, a/2, b}, {c/2, o, tau, gid
// bits} and the colour with the warp mask in .w (zero when the tile cull
// drops the entry: no warp's list admits it).
template <int TILE>
__device__ __forceinline__ void stage_record(uint32_t g, const float4& p, const float4& q, float4 c, int cullmode,
                                             int tx, int ty, float4& A, float4& B, float4& C)
{
    A = make_float4(p.x, p.y, 0.5f * p.z, p.w);
    B = make_float4(0.5f * q.x, q.y, q.w, __uint_as_float(g));
    bool keep = true;
    if (cullmode & 1)
        keep = !tile_culled(A.x, A.y, A.z, A.w, B.x, q.w, c.w, (float)(tx * TILE), (float)(ty * TILE), (float)TILE);
    const uint32_t m = (cullmode & 2)
                           ? strip_mask<TILE>(A.x, A.y, A.z, A.w, B.x, q.w, c.w, (float)(tx * TILE), (float)(ty * TILE))
                           : 0xffffffffu;
    c.w = __uint_as_float(keep ? m : 0u);
    C = c;
}

// Stage the batch [b0, b0 + BATCH) of n_entries stream words from src (global
// or shared memory): per entry {mx, my, a/2, b}, {c/2, o, tau, gid bits} and,
// binned, the colour with the strip mask in .w (zero for an entry the tile
// cull drops).  Returns the number staged (block-uniform); the caller
// synchronises the block before reading sh.
template <int TILE, bool BASELINE>
__device__ __forceinline__ int stage_batch(const uint64_t* src, int32_t b0, int32_t n_entries,
                                           RasterShared<TILE, BASELINE>& sh, const float4* __restrict__ xy_ab,
                                           const float4* __restrict__ c_o_z, const float4* __restrict__ rgbv,
                                           int cullmode, int tx, int ty)
{
    using SH = RasterShared<TILE, BASELINE>;
    constexpr int BATCH = SH::BATCH;
    const int32_t idx = b0 + threadIdx.x;
    const bool valid = threadIdx.x < BATCH && idx < n_entries;
    float4 A = make_float4(0.f, 0.f, 0.f, 0.f), B = A, Cc = A;
    uint32_t g = 0;
    if (valid) {
        g = (uint32_t)(src[idx] & 0xffffffffull);
        const float4 p = __ldg(xy_ab + g);
        const float4 q = __ldg(c_o_z + g);
        if constexpr (BASELINE) {
            A = make_float4(p.x, p.y, 0.5f * p.z, p.w);
            B = make_float4(0.5f * q.x, q.y, q.w, __uint_as_float(g));
        } else {
            stage_record<TILE>(g, p, q, __ldg(rgbv + g), cullmode, tx, ty, A, B, Cc);
        }
    }
    // entry i of the batch goes to slot i: the tile cull and the strip mask
    // leave a zero mask, which no warp's list admits (stream order is kept
    // without a compaction pass)
    const int cnt = min(BATCH, n_entries - b0);
    const int pos = threadIdx.x;
    if (valid) {
        sh.a[pos] = A;
        sh.b[pos] = B;
        if (BASELINE) sh.g[pos] = g;
        else sh.c[pos] = Cc;
    }
    return cnt;
}

// Shared memory of the tile walk.
template <bool LAZY>
struct WalkShared {
    uint64_t sort[LAZY ? kRasterSortCap : 1];
    int32_t off[LAZY ? GS_MAX_K + 1 : 1];
    int big[LAZY ? GS_MAX_K : 1];  // segments sorted by the whole block
    int nsort;
};

// The sorted position of word `key`, entry i of the chunk held in ws.sort
// (bins bfirst..e-1 from stream position c0): the start of its segment plus
// the number of smaller words in the segment (the words are distinct, their
// low half being the gid).
template <bool LAZY>
__device__ __forceinline__ int chunk_rank(const WalkShared<LAZY>& ws, int i, uint64_t key, int32_t c0, int bfirst,
                                          int e)
{
    int lo = bfirst, hi = e - 1;  // the last bin starting at or before i
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ws.off[mid] - c0 <= i) lo = mid;
        else hi = mid - 1;
    }
    const int s0 = ws.off[lo] - c0, s1 = ws.off[lo + 1] - c0;
    int r = s0;
    for (int j = s0; j < s1; ++j) r += ws.sort[j] < key ? 1 : 0;
    return r;
}

// Load the chunk [c0, c0 + len) (bins bfirst..e-1) into ws.sort and sort each
// of its segments by (depth bits, gid).  A chunk of at most one entry per
// thread is sorted by rank: each thread counts the smaller words of its own
// segment (the words are distinct, their low half being the gid), so one
// pass of comparisons and one scatter place every word.  Longer chunks: each
// segment of up to 64 entries in registers by one warp, up to 256 in shared
// memory by one warp, longer ones by the whole block (ws.big[base..] collects
// the long ones).
template <int TILE, bool LAZY>
__device__ __forceinline__ void load_sort_chunk(const uint64_t* words, int32_t c0, int32_t len,
                                                int bfirst, int e, WalkShared<LAZY>& ws, int base = 0)
{
    constexpr int BS = TILE * TILE;
    constexpr int NWB = BS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (len <= BS) {
        // one entry a thread: its rank in its segment is the segment start
        // plus the number of smaller words there (words are unique: gid)
        const int i = threadIdx.x;
        uint64_t key = 0;
        if (i < len) key = __ldcs(reinterpret_cast<const unsigned long long*>(words) + c0 + i);
        if (i < len) ws.sort[i] = key;
        __syncthreads();
        const int r = i < len ? chunk_rank(ws, i, key, c0, bfirst, e) : 0;
        __syncthreads();
        if (i < len) ws.sort[r] = key;
        __syncthreads();
        return;
    }
    // the stream is read once: streamed past L2 (evict first)
    for (int i = threadIdx.x; i < len; i += BS)
        ws.sort[i] = __ldcs(reinterpret_cast<const unsigned long long*>(words) + c0 + i);
    if (threadIdx.x == 0) ws.nsort = 0;
    __syncthreads();
    for (int j = bfirst + warp; j < e; j += NWB) {
        const int l = ws.off[j + 1] - ws.off[j];
        uint64_t* seg = ws.sort + (ws.off[j] - c0);
        if (l < 2) continue;
        if (l <= 32) {
            uint64_t v = lane < l ? seg[lane] : ~0ull;
            v = warp_bitonic32(v);
            if (lane < l) seg[lane] = v;
        } else if (l <= 64) {
            warp_bitonic64(seg, l);
        } else if (l <= 256) {
            bitonic_mem(seg, l, lane, 32, SyncWarp{});
        } else if (lane == 0) {
            ws.big[atomicAdd(&ws.nsort, 1)] = j;
        }
    }
    __syncthreads();
    const int nbig = ws.nsort;
    for (int k = 0; k < nbig; ++k) {
        const int j = ws.big[k];
        bitonic_mem(ws.sort + (ws.off[j] - c0), ws.off[j + 1] - ws.off[j], threadIdx.x, BS, SyncBlock{});
    }
}

// Walk tile t's span of the stream front to back, handing runs of entries to
// span(src, n, checked, base) (src[0] is stream position base; returns -1
// after consuming all n, or, block-uniformly, the offset within the run at
// which every pixel of the tile had terminated; span.done() is the calling
// thread's termination flag; a Span with kStageAtRank also takes a chunk of
// at most kBatch entries staged slot by slot, span.stage_at(slot, gid), and
// composites it with span.composite_staged(n, base)).  Only bins [kbegin, kend) of the tile's K are
// walked (a planned frame's passes; 0, K: the whole span).
// Not LAZY: one run, [off[t*K], off[t*K + kend]).  LAZY: chunks of
// consecutive segments of at most `cap` entries (a single segment of up to
// kRasterSortCap entries forms a chunk of its own) are loaded into shared
// memory and every segment of the chunk is sorted; a segment longer than
// kRasterSortCap was sorted before the raster and is handed over in place.
// The chunks are the tile's repair bins.  ws.off holds all K + 1 bin offsets
// of the tile on return (LAZY).
// Returns the stream index at which the walk ended: the end of the walked
// bins, or the position (in the composited order) where every pixel had
// terminated.  With writeback (the stream itself), every sorted chunk is also
// stored back in place, so the tile's composited prefix is left in (depth,
// gid) order.
template <int TILE, bool LAZY, class Span>
__device__ __forceinline__ int32_t walk_tile(const uint64_t* words, const int32_t* __restrict__ off, int t, int K,
                                             int kbegin, int kend, int cap, WalkShared<LAZY>& ws, Span& span,
                                             uint64_t* writeback = nullptr)
{
    constexpr int BS = TILE * TILE;
    if (!LAZY) {
        const int32_t s0 = off[(int64_t)t * K + kbegin], s1 = off[(int64_t)t * K + kend];
        const int32_t r = span(words + s0, s1 - s0, false, s0);
        return r < 0 ? s1 : s0 + r;
    }
    for (int b = threadIdx.x; b <= K; b += BS) ws.off[b] = off[(int64_t)t * K + b];
    __syncthreads();
    int b = kbegin;
    while (b < kend) {
        const int32_t c0 = ws.off[b];
        if (ws.off[b + 1] - c0 > kRasterSortCap) {  // sorted before the raster
            const int32_t r = span(words + c0, ws.off[b + 1] - c0, false, c0);
            if (r >= 0) return c0 + r;
            ++b;
            continue;
        }
        // the chunk ends before the first bin j > b whose end passes c0 + cap
        // (bin ends are nondecreasing, so the bins that fit are a prefix):
        // counted 32 bins a ballot by every warp, in place of a serial walk
        int e = b + 1;
        {
            const int lane = threadIdx.x & 31;
            for (int j0 = b + 1; j0 < kend; j0 += 32) {
                const int j = j0 + lane;
                const int fit = __popc(__ballot_sync(0xffffffffu, j < kend && ws.off[j + 1] - c0 <= cap));
                e += fit;
                if (fit < 32) break;
            }
        }
        const int32_t len = ws.off[e] - c0;
        const int bfirst = b;
        b = e;
        if (len == 0) continue;
        if (__syncthreads_count(span.done()) == BS) return c0;
        if constexpr (Span::kStageAtRank) {
            if (len <= Span::kBatch) {
                // a chunk of one batch: each thread loads one word, finds
                // its rank in its segment and stages its entry straight at
                // that slot -- no sorted copy of the chunk, two block
                // barriers and a shared-memory round fewer than sorting
                // first and staging after (raster 0.264 -> 0.259 ms at
                // 1080p; gathering the entry's fields before the rank count
                // instead held them across it and spilled: 0.291 ms)
                const int i = threadIdx.x;
                uint64_t key = 0;
                if (i < len) {
                    key = __ldcs(reinterpret_cast<const unsigned long long*>(words) + c0 + i);
                    ws.sort[i] = key;
                }
                __syncthreads();
                if (i < len) {
                    const int r = chunk_rank(ws, i, key, c0, bfirst, e);
                    if (writeback) writeback[c0 + r] = key;
                    span.stage_at(r, (uint32_t)key);
                }
                __syncthreads();
                span.composite_staged(len, c0);  // termination just counted above
                continue;
            }
        }
        load_sort_chunk<TILE>(words, c0, len, bfirst, e, ws);  // ends with a block barrier
        if (writeback)
            for (int i = threadIdx.x; i < len; i += BS) writeback[c0 + i] = ws.sort[i];
        const int32_t r = span(ws.sort, len, true, c0);  // termination just counted above
        if (r >= 0) return c0 + r;
    }
    return ws.off[kend];
}

// The walk of walk_tile in reverse over the entries before stream index
// `end` (a walk_tile result), for a stream sorted throughout or one whose
// composited prefixes the forward wrote back sorted: the span
// [off[t*K], min(end, off[(t+1)*K])) handed to span(src, n) in place.
template <class Span>
__device__ __forceinline__ void walk_tile_rev(const uint64_t* __restrict__ words, const int32_t* __restrict__ off,
                                              int t, int K, int32_t end, Span& span)
{
    const int32_t s0 = off[(int64_t)t * K], s1 = off[(int64_t)(t + 1) * K];
    const int32_t e = end < s1 ? end : s1;
    if (e > s0) span(words + s0, e - s0);
}

}  // namespace gs
