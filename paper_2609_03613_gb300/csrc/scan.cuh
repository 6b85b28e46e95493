// scan.cuh -- device-wide exclusive scan of int64-valued items given by a
// load functor: three kernels without inter-block waits (reduce per block ->
// one-block scan of the block sums -> per-block rescan with the prefix), all
// in int64 so an overflowing total is detected instead of wrapping.
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
static __global__ void __launch_bounds__(kScanThreads) k_scan_sums(int64_t* sums, int64_t nb)
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

template <class Load>
static inline int scan_impl(gs_ctx* ctx, Load ld, int64_t n, int32_t* out, int64_t* total64, cudaStream_t st)
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


}  // namespace gs
