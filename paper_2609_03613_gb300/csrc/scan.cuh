// scan.cuh -- device-wide exclusive scan of int64-valued items given by a
// load functor: two kernels without inter-block waits (reduce per block, the
// last block to finish scanning the block sums -> per-block rescan with the
// prefix), all in int64 so an overflowing total is detected instead of
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

// Exclusive scan of sums[0..nb) in place by one block; sums[nb] = grand total.
__device__ __forceinline__ void scan_sums_body(int64_t* sums, int64_t nb)
{
    __shared__ int64_t s_warp[kScanThreads / 32];
    int64_t carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += kScanThreads) {
        const int64_t i = b0 + threadIdx.x;
        const int64_t v = i < nb ? __ldcg(sums + i) : 0;  // written by other blocks: read at L2
        int64_t total;
        const int64_t ex = block_exclusive_scan(v, s_warp, &total);
        if (i < nb) sums[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) sums[nb] = carry;
}

// Called by every block after it stored its block sum(s): the last block to
// arrive (a counter, reset by that block) scans the sums; no block waits for
// another.  Returns true in the block that did the scan.
__device__ __forceinline__ bool last_block_scans(unsigned int* done, int64_t* sa, int64_t* sb)
{
    __shared__ bool s_last;
    __threadfence();  // this thread's sum store is visible device-wide ...
    __syncthreads();  // ... before the block counts itself done
    if (threadIdx.x == 0) s_last = atomicAdd(done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    scan_sums_body(sa, gridDim.x);
    if (sb) scan_sums_body(sb, gridDim.x);
    if (threadIdx.x == 0) *done = 0u;  // ready for the next scan on the stream
    return true;
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

// Block sums: every item of the block's tile loaded at once (coalesced,
// all in flight), summed, then reduced across the block.
template <class Load>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(Load ld, int64_t n, int64_t* sums, unsigned int* done)
{
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t v[kScanItems];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        v[k] = i < n ? ld(i) : 0;
    }
    int64_t acc = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) acc += v[k];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
    __shared__ int64_t s_warp[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_warp[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
#pragma unroll
        for (int w = 0; w < kScanThreads / 32; ++w) t += s_warp[w];
        sums[blockIdx.x] = t;
    }
    last_block_scans(done, sums, nullptr);
}


// The block tile's items move between the striped order of coalesced global
// accesses (item k*256 + t in thread t's slot k) and the blocked order of the
// per-thread serial scan (item 16t + k) through shared memory, one padding
// word per 32 so that neither side conflicts badly on banks.
constexpr int kScanPadded = kScanTile + kScanTile / 32;
__device__ __forceinline__ int scan_pad(int j) { return j + (j >> 5); }

__device__ __forceinline__ void striped_to_blocked(int64_t (&v)[kScanItems], int64_t* sm)
{
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) sm[scan_pad(k * kScanThreads + threadIdx.x)] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) v[k] = sm[scan_pad(threadIdx.x * kScanItems + k)];
    __syncthreads();
}

__device__ __forceinline__ void blocked_to_striped(int64_t (&v)[kScanItems], int64_t* sm)
{
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) sm[scan_pad(threadIdx.x * kScanItems + k)] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) v[k] = sm[scan_pad(k * kScanThreads + threadIdx.x)];
    __syncthreads();
}

// Exclusive scan of the block tile's items (striped in, striped out), offset
// by `base`: blocked transposition, serial scan per thread, one block scan.
__device__ __forceinline__ void scan_tile_striped(int64_t (&v)[kScanItems], int64_t base, int64_t* sm,
                                                  int64_t* s_warp)
{
    striped_to_blocked(v, sm);
    int64_t run = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t x = v[k];
        v[k] = run;
        run += x;
    }
    int64_t total;
    const int64_t off = base + block_exclusive_scan(run, s_warp, &total);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) v[k] += off;
    blocked_to_striped(v, sm);
}

// Per-block rescan.  out[i] (int32) = exclusive prefix; out[n] = total.  The
// int64 total goes to total64.  A total >= 2^31 raises GS_ERR_CAPACITY and
// leaves out[] unwritten.  Same tile partition as k_scan_reduce, so the
// block's prefix from the sums applies; loads and stores are coalesced.
template <class Load>
__global__ void __launch_bounds__(kScanThreads)
k_scan_down(Load ld, int64_t n, const int64_t* sums, int64_t nb, int32_t* out, int64_t* total64, int* err)
{
    __shared__ int64_t s_warp[kScanThreads / 32];
    __shared__ int64_t s_tile[kScanPadded];
    const int64_t grand = sums[nb];
    if (grand > (int64_t)INT32_MAX - 1) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            raise_error(err, GS_ERR_CAPACITY);
            if (total64) *total64 = grand;
        }
        return;
    }
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t v[kScanItems];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        v[k] = i < n ? ld(i) : 0;
    }
    scan_tile_striped(v, sums[blockIdx.x], s_tile, s_warp);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < n) out[i] = (int32_t)v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        out[n] = (int32_t)grand;
        if (total64) *total64 = grand;
    }
}

// ------------------------------------------------------------------ two scans in one pass
// Two exclusive scans of per-item values produced by one load (for example a
// rect's tile count and its row count): ld(i, a, b).  The same kernels, each
// carrying both values; sums hold [nb + 1] entries per scan.
template <class Load2>
__global__ void __launch_bounds__(kScanThreads) k_scan2_reduce(Load2 ld, int64_t n, int64_t* sa, int64_t* sb,
                                                               unsigned int* done)
{
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t acc_a = 0, acc_b = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        int64_t x = 0, y = 0;
        if (i < n) ld(i, x, y);
        acc_a += x;
        acc_b += y;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        acc_a += __shfl_down_sync(0xffffffffu, acc_a, d);
        acc_b += __shfl_down_sync(0xffffffffu, acc_b, d);
    }
    __shared__ int64_t s_warp[2][kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        s_warp[0][warp] = acc_a;
        s_warp[1][warp] = acc_b;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        int64_t t = 0;
#pragma unroll
        for (int w = 0; w < kScanThreads / 32; ++w) t += s_warp[threadIdx.x][w];
        (threadIdx.x ? sb : sa)[blockIdx.x] = t;
    }
    last_block_scans(done, sa, sb);
}

template <class Load2>
__global__ void __launch_bounds__(kScanThreads)
k_scan2_down(Load2 ld, int64_t n, const int64_t* sa, const int64_t* sb, int64_t nb, int32_t* oa, int64_t* ta,
             int32_t* ob, int64_t* tb, int* err)
{
    __shared__ int64_t s_warp[kScanThreads / 32];
    __shared__ int64_t s_tile[kScanPadded];
    const int64_t ga = sa[nb], gb = sb[nb];
    if (ga > (int64_t)INT32_MAX - 1 || gb > (int64_t)INT32_MAX - 1) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            raise_error(err, GS_ERR_CAPACITY);
            if (ta) *ta = ga;
            if (tb) *tb = gb;
        }
        return;
    }
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t va[kScanItems], vb[kScanItems];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        va[k] = vb[k] = 0;
        if (i < n) ld(i, va[k], vb[k]);
    }
    scan_tile_striped(va, sa[blockIdx.x], s_tile, s_warp);
    scan_tile_striped(vb, sb[blockIdx.x], s_tile, s_warp);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < n) {
            oa[i] = (int32_t)va[k];
            ob[i] = (int32_t)vb[k];
        }
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        oa[n] = (int32_t)ga;
        ob[n] = (int32_t)gb;
        if (ta) *ta = ga;
        if (tb) *tb = gb;
    }
}

template <class Load2>
static inline int scan2_impl(gs_ctx* ctx, Load2 ld, int64_t n, int32_t* oa, int64_t* ta, int32_t* ob, int64_t* tb,
                             cudaStream_t st)
{
    const int64_t nb = n > 0 ? (n + kScanTile - 1) / kScanTile : 1;
    int r = ensure(&ctx->d_scan, &ctx->scan_bytes, (size_t)2 * (nb + 1) * sizeof(int64_t));
    if (r != GS_OK) return r;
    int64_t* sa = static_cast<int64_t*>(ctx->d_scan);
    int64_t* sb = sa + nb + 1;
    k_scan2_reduce<Load2><<<(unsigned)nb, kScanThreads, 0, st>>>(ld, n, sa, sb, ctx->d_scan_done);
    k_scan2_down<Load2><<<(unsigned)nb, kScanThreads, 0, st>>>(ld, n, sa, sb, nb, oa, ta, ob, tb, ctx->d_err);
    ctx->launches += 2;
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

template <class Load>
static inline int scan_impl(gs_ctx* ctx, Load ld, int64_t n, int32_t* out, int64_t* total64, cudaStream_t st)
{
    const int64_t nb = n > 0 ? (n + kScanTile - 1) / kScanTile : 1;
    int r = ensure(&ctx->d_scan, &ctx->scan_bytes, (size_t)(nb + 1) * sizeof(int64_t));
    if (r != GS_OK) return r;
    int64_t* sums = static_cast<int64_t*>(ctx->d_scan);
    k_scan_reduce<Load><<<(unsigned)nb, kScanThreads, 0, st>>>(ld, n, sums, ctx->d_scan_done);
    k_scan_down<Load><<<(unsigned)nb, kScanThreads, 0, st>>>(ld, n, sums, nb, out, total64, ctx->d_err);
    ctx->launches += 2;
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}


}  // namespace gs
