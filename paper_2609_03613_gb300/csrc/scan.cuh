// scan.cuh -- device-wide exclusive scan of items given by a load functor, in
// one pass: each block takes a ticket (its place in the scan, so every block
// it waits for has already started), scans its tile of 4096 items, publishes
// its total, and looks back over its predecessors' published totals and
// prefixes (decoupled look-back: D. Merrill and M. Garland, "Single-pass
// Parallel Prefix Scan with Decoupled Look-back", 2016) with bounded waits.
// Totals are carried in int64, so an overflowing total is detected instead of
// wrapping.
#pragma once

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

// a rect's tile count (as LoadRectCount) and its row count (rows of a
// non-empty rect, else 0)
struct LoadRectCountRows {
    const uint2* rect;
    __device__ void operator()(int64_t i, int64_t& count, int64_t& rows) const
    {
        const uint2 r = rect[i];
        const int64_t w = (int64_t)(r.y & 0xffffu) - (int64_t)(r.x & 0xffffu);
        const int64_t h = (int64_t)(r.y >> 16) - (int64_t)(r.x >> 16);
        count = w * h;
        rows = (w > 0 && h > 0) ? h : 0;
    }
};

// The block tile's items move between the striped order of coalesced global
// accesses (item k*256 + t in thread t's slot k) and the blocked order of the
// per-thread serial scan (item 16t + k) through shared memory, one padding
// word per 32 so that neither side conflicts badly on banks.
constexpr int kScanPadded = kScanTile + kScanTile / 32;
__device__ __forceinline__ int scan_pad(int j) { return j + (j >> 5); }

// ------------------------------------------------------------------ one pass
// A block's published word: status in the top two bits (0 not yet, A its
// total, P its inclusive prefix), the value below (< 2^62).
constexpr uint64_t kScanFlagA = 1ull << 62, kScanFlagP = 2ull << 62, kScanFlagMask = 3ull << 62;
constexpr int kLookbackPolls = 1 << 22;

// The exclusive prefix of block bid from the words of its predecessors, by
// one warp (in every lane): windows of 32 predecessors, each lane waiting
// (bounded; GS_ERR_TIMEOUT when it runs out) for its word, the values summed
// back to the nearest inclusive prefix.
__device__ __forceinline__ int64_t scan_lookback(const volatile uint64_t* flags, int64_t bid, int* err)
{
    const int lane = threadIdx.x & 31;
    int64_t prefix = 0;
    for (int64_t j = bid - 1; j >= 0; j -= 32) {
        const int64_t idx = j - lane;
        uint64_t w = 0;
        if (idx >= 0) {
            int it = 0;
            do {
                w = flags[idx];
            } while ((w & kScanFlagMask) == 0 && ++it < kLookbackPolls);
            if ((w & kScanFlagMask) == 0) raise_error(err, GS_ERR_TIMEOUT);
        }
        const unsigned pmask = __ballot_sync(0xffffffffu, idx >= 0 && (w & kScanFlagMask) == kScanFlagP);
        const int stop = pmask ? __ffs(pmask) - 1 : 31;  // the nearest predecessor with a prefix
        int64_t val = (idx >= 0 && lane <= stop) ? (int64_t)(w & ~kScanFlagMask) : 0;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) val += __shfl_xor_sync(0xffffffffu, val, d);
        prefix += val;
        if (pmask) break;
    }
    return prefix;
}

// Exclusive scan of the block tile's items in int32 (striped in, striped
// out): blocked transposition through shared memory, serial scan per thread,
// one block scan; returns the tile's total.
__device__ __forceinline__ int64_t scan_tile32(int32_t (&v)[kScanItems], int32_t* sm, int64_t* s_warp)
{
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) sm[scan_pad(k * kScanThreads + threadIdx.x)] = v[k];
    __syncthreads();
    int32_t run = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int32_t x = sm[scan_pad(threadIdx.x * kScanItems + k)];
        v[k] = run;
        run += x;
    }
    int64_t total;
    const int32_t off = (int32_t)block_exclusive_scan(run, s_warp, &total);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) sm[scan_pad(threadIdx.x * kScanItems + k)] = v[k] + off;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) v[k] = sm[scan_pad(k * kScanThreads + threadIdx.x)];
    __syncthreads();
    return total;
}

// NC channels of item values (one load gives all of them), each scanned into
// its own output; out[n] = total unless it exceeds INT32_MAX - 1 (then
// GS_ERR_CAPACITY and the outputs are not valid); totals[c] receives the
// int64 total.  dup0, when given, receives a second copy of channel 0's
// items 0..n-1 (it may be the load's own source: a block writes only the
// items it has read).  Per-item values and a tile's total must fit in int32.
template <int NC, class Load>
__global__ void __launch_bounds__(kScanThreads)
k_scan_onepass(Load ld, int64_t n, uint64_t* flags, int64_t nb, unsigned int* ticket, int32_t* out0, int32_t* out1,
               int64_t* tot0, int64_t* tot1, int* err, int32_t* dup0)
{
    grid_dependency_sync();
    __shared__ int32_t s_tile[kScanPadded];
    __shared__ int64_t s_warp[kScanThreads / 32];
    __shared__ int64_t s_pre[NC];
    __shared__ int64_t s_bid;
    if (threadIdx.x == 0) {
        const unsigned t = atomicAdd(ticket, 1u);
        s_bid = t;
        if ((int64_t)t == nb - 1) *ticket = 0u;  // every ticket is out: ready for the next scan
    }
    __syncthreads();
    const int64_t bid = s_bid;
    const int64_t base = bid * kScanTile;
    int32_t v[NC][kScanItems];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        int64_t x[2] = {0, 0};
        if (i < n) ld.load(i, x);
#pragma unroll
        for (int c = 0; c < NC; ++c) v[c][k] = (int32_t)x[c];
    }
    int64_t agg[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) agg[c] = scan_tile32(v[c], s_tile, s_warp);
    volatile uint64_t* vf = flags;
    if (threadIdx.x == 0)
        for (int c = 0; c < NC; ++c) vf[c * nb + bid] = (bid == 0 ? kScanFlagP : kScanFlagA) | (uint64_t)agg[c];
    if (threadIdx.x < 32) {
        for (int c = 0; c < NC; ++c) {
            const int64_t pre = bid > 0 ? scan_lookback(vf + c * nb, bid, err) : 0;
            if (threadIdx.x == 0) {
                if (bid > 0) vf[c * nb + bid] = kScanFlagP | (uint64_t)(pre + agg[c]);
                s_pre[c] = pre;
            }
        }
    }
    __syncthreads();
    int32_t* outs[2] = {out0, out1};
    int64_t* tots[2] = {tot0, tot1};
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int64_t pre = s_pre[c];
        const bool over = pre + agg[c] > (int64_t)INT32_MAX - 1;
        if (over) {
            if (threadIdx.x == 0) raise_error(err, GS_ERR_CAPACITY);
        } else {
#pragma unroll
            for (int k = 0; k < kScanItems; ++k) {
                const int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
                if (i < n) {
                    outs[c][i] = (int32_t)(pre + v[c][k]);
                    if (c == 0 && dup0) dup0[i] = (int32_t)(pre + v[c][k]);
                }
            }
        }
        if (bid == nb - 1 && threadIdx.x == 0) {
            if (!over) outs[c][n] = (int32_t)(pre + agg[c]);
            if (tots[c]) *tots[c] = pre + agg[c];
        }
    }
}

// one-value and two-value loads for the one-pass kernel
template <class Load>
struct Load1 {
    Load ld;
    __device__ void load(int64_t i, int64_t (&x)[2]) const { x[0] = ld(i); }
};
template <class Load2>
struct Load2v {
    Load2 ld;
    __device__ void load(int64_t i, int64_t (&x)[2]) const { ld(i, x[0], x[1]); }
};

// The flag words of one scan of nw words: the next piece of the frame's
// pre-zeroed arena, or (no arena, or the arena is spent) words past the arena
// cleared here.
static inline int scan_flags(gs_ctx* ctx, int64_t nw, uint64_t** flags, cudaStream_t st)
{
    if (ctx->scan_arena > 0 && ctx->scan_bytes != ctx->scan_arena_bytes) ctx->scan_arena = 0;  // reallocated
    if (ctx->scan_arena > 0 && ctx->scan_used + nw <= ctx->scan_arena) {
        *flags = static_cast<uint64_t*>(ctx->d_scan) + ctx->scan_used;
        ctx->scan_used += nw;
        return GS_OK;
    }
    const size_t bytes = ctx->scan_bytes;
    int r = ensure(&ctx->d_scan, &ctx->scan_bytes, (size_t)(ctx->scan_arena + nw + 2) * sizeof(uint64_t));
    if (r != GS_OK) return r;
    if (ctx->scan_bytes != bytes) ctx->scan_arena = 0;
    *flags = static_cast<uint64_t*>(ctx->d_scan) + ctx->scan_arena;
    GS_CUDA_TRY(cudaMemsetAsync(*flags, 0, (size_t)nw * sizeof(uint64_t), st));
    return GS_OK;
}

template <class Load2>
static inline int scan2_impl(gs_ctx* ctx, Load2 ld, int64_t n, int32_t* oa, int64_t* ta, int32_t* ob, int64_t* tb,
                             cudaStream_t st)
{
    const int64_t nb = n > 0 ? (n + kScanTile - 1) / kScanTile : 1;
    uint64_t* flags;
    int r = scan_flags(ctx, 2 * nb, &flags, st);
    if (r != GS_OK) return r;
    GS_CUDA_TRY(launch_k(ctx, (k_scan_onepass<2, Load2v<Load2>>), (unsigned)nb, kScanThreads, 0, st,
                         Load2v<Load2>{ld}, n, flags, nb, ctx->d_scan_done, oa, ob, ta, tb, ctx->d_err,
                         static_cast<int32_t*>(nullptr)));
    ctx->launches += 1;
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

template <class Load>
static inline int scan_impl(gs_ctx* ctx, Load ld, int64_t n, int32_t* out, int64_t* total64, cudaStream_t st,
                            int32_t* dup = nullptr)
{
    const int64_t nb = n > 0 ? (n + kScanTile - 1) / kScanTile : 1;
    uint64_t* flags;
    int r = scan_flags(ctx, nb, &flags, st);
    if (r != GS_OK) return r;
    GS_CUDA_TRY(launch_k(ctx, (k_scan_onepass<1, Load1<Load>>), (unsigned)nb, kScanThreads, 0, st, Load1<Load>{ld}, n,
                         flags, nb, ctx->d_scan_done, out, nullptr, total64, nullptr, ctx->d_err, dup));
    ctx->launches += 1;
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

}  // namespace gs
