// sort.cu -- K4+K5, the baseline ordering: a stable LSD radix sort of the
// entries by the key (tile << 32 | depth bits), then per-tile ranges
// (Sec. 3.1: "globally sorted by a composite key that first groups by tile and
// then orders by depth"; the paper's baseline uses a CUB global radix sort).
//
// Emission order is gid-major, so a stable sort leaves ties in depth in gid
// order: the result is the (tile, depth, gid) order.
//
// Each 8-bit pass runs three kernels over chunks of 2048 keys:
//   histogram per chunk -> per-digit scan over chunks -> stable scatter.
// The entry count M is read on the device, so no host synchronisation is
// needed; grids are sized for the capacity and loop over the live chunks.
// Ranking inside a chunk: each warp owns 256 consecutive keys, processed in
// 8 rounds of 32; __match_any_sync groups equal digits, giving each key its
// rank among earlier equal digits; warp counts are then prefixed across warps.
#include "internal.cuh"

namespace gs {

constexpr int kRsThreads = 256;
constexpr int kRsItems = 8;
constexpr int kRsChunk = kRsThreads * kRsItems;  // 2048
constexpr int kRsWarps = kRsThreads / 32;

__device__ __forceinline__ uint32_t digit_of(uint64_t key, int shift) { return (uint32_t)(key >> shift) & 0xffu; }

__device__ __forceinline__ uint64_t load_key(int pass0, const IsectView& is, const uint64_t* keys, int64_t i)
{
    if (pass0) return ((uint64_t)is.tile[i] << 32) | is.zbits[i];
    return keys[i];
}

__global__ void __launch_bounds__(kRsThreads)
k_rs_hist(int pass0, IsectView is, const uint64_t* __restrict__ keys, const int64_t* __restrict__ m_dev,
          int64_t m_cap, int shift, uint32_t* __restrict__ H, int64_t nchunks_cap)
{
    __shared__ uint32_t s_h[256];
    const int64_t M = live_count(m_dev, m_cap);
    const int64_t nchunks = (M + kRsChunk - 1) / kRsChunk;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        s_h[threadIdx.x] = 0;
        __syncthreads();
        const int64_t base = c * kRsChunk;
#pragma unroll
        for (int k = 0; k < kRsItems; ++k) {
            const int64_t i = base + (int64_t)k * kRsThreads + threadIdx.x;
            if (i < M) atomicAdd(&s_h[digit_of(load_key(pass0, is, keys, i), shift)], 1u);
        }
        __syncthreads();
        H[(int64_t)threadIdx.x * nchunks_cap + c] = s_h[threadIdx.x];
        __syncthreads();
    }
}

// One block per digit: exclusive scan of H[d][0..nchunks) in place; the
// digit total goes to tot[d].
__global__ void __launch_bounds__(kRsThreads)
k_rs_scan(uint32_t* __restrict__ H, int64_t nchunks_cap, const int64_t* __restrict__ m_dev, int64_t m_cap,
          uint32_t* __restrict__ tot)
{
    __shared__ uint32_t s_w[kRsWarps];
    const int64_t M = live_count(m_dev, m_cap);
    const int64_t nchunks = (M + kRsChunk - 1) / kRsChunk;
    uint32_t* row = H + (int64_t)blockIdx.x * nchunks_cap;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t carry = 0;
    for (int64_t b0 = 0; b0 < nchunks; b0 += kRsThreads) {
        const int64_t i = b0 + threadIdx.x;
        const uint32_t v = i < nchunks ? row[i] : 0u;
        uint32_t incl = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += t;
        }
        if (lane == 31) s_w[warp] = incl;
        __syncthreads();
        uint32_t wp = 0, all = 0;
#pragma unroll
        for (int w = 0; w < kRsWarps; ++w) {
            const uint32_t x = s_w[w];
            if (w < warp) wp += x;
            all += x;
        }
        if (i < nchunks) row[i] = carry + wp + incl - v;
        carry += all;
        __syncthreads();
    }
    if (threadIdx.x == 0) tot[blockIdx.x] = carry;
}

__global__ void __launch_bounds__(kRsThreads)
k_rs_scatter(int pass0, int last, IsectView is, const uint64_t* __restrict__ keys_in,
             const uint32_t* __restrict__ vals_in, const int64_t* __restrict__ m_dev, int64_t m_cap, int shift,
             const uint32_t* __restrict__ H, int64_t nchunks_cap, const uint32_t* __restrict__ tot,
             uint64_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
             uint64_t* __restrict__ words_out, uint32_t* __restrict__ tiles_out)
{
    __shared__ uint64_t s_key[kRsChunk];
    __shared__ uint32_t s_val[kRsChunk];
    __shared__ uint32_t s_cnt[kRsWarps][256];
    __shared__ uint32_t s_dstart[256];
    __shared__ uint32_t s_base[256];
    __shared__ uint32_t s_w[kRsWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int64_t M = live_count(m_dev, m_cap);
    const int64_t nchunks = (M + kRsChunk - 1) / kRsChunk;

    // digit bases: exclusive scan of the digit totals
    {
        const uint32_t v = tot[threadIdx.x];
        uint32_t incl = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += t;
        }
        if (lane == 31) s_w[warp] = incl;
        __syncthreads();
        uint32_t wp = 0;
        for (int w = 0; w < warp; ++w) wp += s_w[w];
        s_base[threadIdx.x] = wp + incl - v;
        __syncthreads();
    }

    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
#pragma unroll
        for (int w = 0; w < kRsWarps; ++w) s_cnt[w][threadIdx.x] = 0;
        __syncthreads();
        const int64_t base = c * kRsChunk;
        uint64_t key[kRsItems];
        uint32_t val[kRsItems];
        uint32_t rank[kRsItems];
#pragma unroll
        for (int k = 0; k < kRsItems; ++k) {
            const int64_t i = base + warp * (32 * kRsItems) + k * 32 + lane;
            const bool ok = i < M;
            key[k] = ok ? load_key(pass0, is, keys_in, i) : ~0ull;
            val[k] = ok ? (pass0 ? is.gid[i] : vals_in[i]) : 0u;
            const uint32_t d = ok ? digit_of(key[k], shift) : 256u;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            const uint32_t before = __popc(peers & lt_mask);
            rank[k] = ok ? s_cnt[warp][d] + before : 0u;
            __syncwarp();
            if (ok && before == 0) s_cnt[warp][d] += __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // per digit: prefix over warps, chunk total; then scan over digits
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kRsWarps; ++w) {
            const uint32_t x = s_cnt[w][threadIdx.x];
            s_cnt[w][threadIdx.x] = run;
            run += x;
        }
        {
            uint32_t incl = run;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += t;
            }
            if (lane == 31) s_w[warp] = incl;
            __syncthreads();
            uint32_t wp = 0;
            for (int w = 0; w < warp; ++w) wp += s_w[w];
            s_dstart[threadIdx.x] = wp + incl - run;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kRsItems; ++k) {
            const int64_t i = base + warp * (32 * kRsItems) + k * 32 + lane;
            if (i < M) {
                const uint32_t d = digit_of(key[k], shift);
                const uint32_t lp = s_dstart[d] + s_cnt[warp][d] + rank[k];
                s_key[lp] = key[k];
                s_val[lp] = val[k];
            }
        }
        __syncthreads();
        const int cnt = (int)((M - base) < kRsChunk ? (M - base) : kRsChunk);
        for (int j = threadIdx.x; j < cnt; j += kRsThreads) {
            const uint64_t kk = s_key[j];
            const uint32_t d = digit_of(kk, shift);
            const int64_t dst = (int64_t)s_base[d] + H[(int64_t)d * nchunks_cap + c] + (j - s_dstart[d]);
            if (last) {
                words_out[dst] = ((kk & 0xffffffffull) << 32) | s_val[j];
                tiles_out[dst] = (uint32_t)(kk >> 32);
            } else {
                keys_out[dst] = kk;
                vals_out[dst] = s_val[j];
            }
        }
        __syncthreads();
    }
}

// offsets[t] = first sorted position whose tile is >= t (t = 0..T).
__global__ void k_tile_ranges(const uint32_t* __restrict__ tiles, const int64_t* __restrict__ m_dev,
                              int64_t m_cap, int32_t n_tiles, int32_t* __restrict__ offsets)
{
    const int64_t M = live_count(m_dev, m_cap);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (M == 0) {
        for (int64_t t = g; t <= n_tiles; t += stride) offsets[t] = 0;
        return;
    }
    for (int64_t p = g; p < M; p += stride) {
        const int64_t t = tiles[p];
        const int64_t tprev = p > 0 ? (int64_t)tiles[p - 1] : -1;
        for (int64_t tt = tprev + 1; tt <= t; ++tt) offsets[tt] = (int32_t)p;
        if (p == M - 1)
            for (int64_t tt = t + 1; tt <= n_tiles; ++tt) offsets[tt] = (int32_t)M;
    }
}

int sort_reserve(gs_ctx* ctx, int64_t m_cap)
{
    const int64_t nchunks_cap = m_cap > 0 ? (m_cap + kRsChunk - 1) / kRsChunk : 1;
    int r;
    const size_t need_k = (size_t)(m_cap > 0 ? m_cap : 1) * 8;
    if (ctx->sort_cap < need_k) {
        for (int b = 0; b < 2; ++b) {
            if (ctx->d_keys[b]) cudaFree(ctx->d_keys[b]);
            if (ctx->d_vals[b]) cudaFree(ctx->d_vals[b]);
            ctx->d_keys[b] = nullptr;
            ctx->d_vals[b] = nullptr;
        }
        ctx->sort_cap = 0;
        for (int b = 0; b < 2; ++b) {
            void* pk = nullptr;
            void* pv = nullptr;
            size_t ck = 0, cv = 0;
            if ((r = ensure(&pk, &ck, need_k)) != GS_OK) return r;
            ctx->d_keys[b] = (uint64_t*)pk;
            if ((r = ensure(&pv, &cv, need_k / 2)) != GS_OK) return r;
            ctx->d_vals[b] = (uint32_t*)pv;
        }
        ctx->sort_cap = need_k;
    }
    void* hp = ctx->d_hist;
    // H[256][nchunks_cap] + tot[256] + sorted tile ids [m_cap]
    if ((r = ensure(&hp, &ctx->hist_cap, ((size_t)256 * nchunks_cap + 256 + (size_t)m_cap + 64) * 4)) != GS_OK)
        return r;
    ctx->d_hist = (uint32_t*)hp;
    return GS_OK;
}

int global_sort(gs_ctx* ctx, const IsectView& is, int64_t m_cap, const int64_t* m_dev, int32_t n_tiles,
                uint64_t* stream_words, int32_t* offsets, cudaStream_t st)
{
    const int64_t nchunks_cap = m_cap > 0 ? (m_cap + kRsChunk - 1) / kRsChunk : 1;
    int r = sort_reserve(ctx, m_cap);
    if (r != GS_OK) return r;
    uint32_t* H = ctx->d_hist;
    uint32_t* tot = H + (size_t)256 * nchunks_cap;
    uint32_t* tiles_sorted = tot + 256;

    int tile_bits = 0;
    while ((1ll << tile_bits) < (long long)n_tiles) ++tile_bits;
    const int passes = 4 + (tile_bits + 7) / 8;
    const int64_t gmax = (int64_t)ctx->num_sms * 4;
    const unsigned grid = (unsigned)(nchunks_cap < gmax ? nchunks_cap : gmax);
    int cur = 0;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        const int pass0 = p == 0, last = p == passes - 1;
        const uint64_t* kin = pass0 ? nullptr : ctx->d_keys[cur];
        const uint32_t* vin = pass0 ? nullptr : ctx->d_vals[cur];
        k_rs_hist<<<grid, kRsThreads, 0, st>>>(pass0, is, kin, m_dev, m_cap, shift, H, nchunks_cap);
        k_rs_scan<<<256, kRsThreads, 0, st>>>(H, nchunks_cap, m_dev, m_cap, tot);
        k_rs_scatter<<<grid, kRsThreads, 0, st>>>(pass0, last, is, kin, vin, m_dev, m_cap, shift, H, nchunks_cap, tot,
                                                 ctx->d_keys[cur ^ 1], ctx->d_vals[cur ^ 1], stream_words,
                                                 tiles_sorted);
        cur ^= 1;
    }
    k_tile_ranges<<<(unsigned)ctx->num_sms * 4, 256, 0, st>>>(tiles_sorted, m_dev, m_cap, n_tiles, offsets);
    ctx->launches += 3 * passes + 1;
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

}  // namespace gs
