// order.cu -- raster-order-aware storage of the scene: the Gaussians in the
// Z-order (Morton order) of their means, so that the Gaussians one tile
// composites sit close together in every per-Gaussian array (the paper's
// stated next direction, Sec. 6.2: a geometry layout aligned with tile-local
// traversal).  A per-scene step, outside the frame; the image of the permuted
// scene equals the original's except where two Gaussians of one tile share a
// depth bit for bit (the (depth, gid) tie order follows the new gids).
//
// The order (float32, one correctly rounded operation per step):
//   lo_a = min_i x_ia, ext_a = hi_a - lo_a, s_a = 1024 / ext_a (0 if ext_a == 0),
//   c_a = min(1023, trunc((x_ia - lo_a) * s_a)),
//   code = sum_k bit_k(c_x) << 3k | bit_k(c_y) << (3k+1) | bit_k(c_z) << (3k+2),
// perm = the gids stably sorted by code (the baseline's radix sort).
#include "internal.cuh"

namespace gs {

constexpr int kOrderThreads = 256;

// per-block min and max of each axis (a deterministic two-level reduction)
__global__ void __launch_bounds__(kOrderThreads)
k_bounds_partial(const float* __restrict__ means, int64_t n, float* __restrict__ part)
{
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = blockIdx.x * (int64_t)kOrderThreads + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kOrderThreads) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float x = means[i * 3 + a];
            lo[a] = fminf(lo[a], x);
            hi[a] = fmaxf(hi[a], x);
        }
    }
    __shared__ float s[6][kOrderThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], d));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], d));
        }
        if (lane == 0) {
            s[a][warp] = lo[a];
            s[3 + a][warp] = hi[a];
        }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int f = threadIdx.x;
        float v = s[f][0];
        for (int w = 1; w < kOrderThreads / 32; ++w) v = f < 3 ? fminf(v, s[f][w]) : fmaxf(v, s[f][w]);
        part[(int64_t)blockIdx.x * 6 + f] = v;
    }
}

// lo[3] and the scale s[3] from the partials (one block)
__global__ void k_bounds_final(const float* __restrict__ part, int nparts, float* __restrict__ lo_s,
                               int64_t* __restrict__ m_dev, int64_t n)
{
    if (threadIdx.x < 3) {
        const int a = threadIdx.x;
        float lo = INFINITY, hi = -INFINITY;
        for (int b = 0; b < nparts; ++b) {
            lo = fminf(lo, part[b * 6 + a]);
            hi = fmaxf(hi, part[b * 6 + 3 + a]);
        }
        const float ext = __fsub_rn(hi, lo);
        lo_s[a] = lo;
        lo_s[3 + a] = ext > 0.0f ? __fdiv_rn(1024.0f, ext) : 0.0f;
    }
    if (threadIdx.x == 0) *m_dev = n;
}

__device__ __forceinline__ uint32_t spread3(uint32_t v)
{
    // bit k of v -> bit 3k (v < 1024)
    uint32_t r = 0;
#pragma unroll
    for (int k = 0; k < 10; ++k) r |= ((v >> k) & 1u) << (3 * k);
    return r;
}

__device__ __forceinline__ uint32_t cell_of(float x, float lo, float s)
{
    const float q = __fmul_rn(__fsub_rn(x, lo), s);
    const int c = (int)q;  // q >= 0: truncation is the floor
    return (uint32_t)(c < 0 ? 0 : c > 1023 ? 1023 : c);
}

// the sort's input: key (0, code), value gid
__global__ void __launch_bounds__(kOrderThreads)
k_morton(const float* __restrict__ means, int64_t n, const float* __restrict__ lo_s, IsectView is)
{
    const float lx = lo_s[0], ly = lo_s[1], lz = lo_s[2], sx = lo_s[3], sy = lo_s[4], sz = lo_s[5];
    for (int64_t i = blockIdx.x * (int64_t)kOrderThreads + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kOrderThreads) {
        const uint32_t cx = cell_of(means[i * 3 + 0], lx, sx);
        const uint32_t cy = cell_of(means[i * 3 + 1], ly, sy);
        const uint32_t cz = cell_of(means[i * 3 + 2], lz, sz);
        is.tile[i] = 0u;
        is.zbits[i] = spread3(cx) | (spread3(cy) << 1) | (spread3(cz) << 2);
        is.gid[i] = (uint32_t)i;
    }
}

__global__ void __launch_bounds__(kOrderThreads)
k_perm_from_words(const uint64_t* __restrict__ words, int64_t n, int32_t* __restrict__ perm)
{
    for (int64_t i = blockIdx.x * (int64_t)kOrderThreads + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kOrderThreads)
        perm[i] = (int32_t)(words[i] & 0xffffffffull);
}

// dst[i][0..w) = src[perm[i]][0..w); a warp per row group, lanes over the
// row's floats (coalesced for wide rows such as SH coefficients)
__global__ void __launch_bounds__(kOrderThreads)
k_gather_rows(const int32_t* __restrict__ perm, int64_t n, const float* __restrict__ src, int32_t w,
              float* __restrict__ dst, int* __restrict__ err)
{
    const int64_t total = n * (int64_t)w;
    for (int64_t e = blockIdx.x * (int64_t)kOrderThreads + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * kOrderThreads) {
        const int64_t i = e / w;
        const int32_t j = (int32_t)(e - i * w);
        const int32_t p = perm[i];
        if (p < 0 || (int64_t)p >= n) {
            raise_error(err, GS_ERR_INVALID_ARG);
            continue;
        }
        dst[e] = src[(int64_t)p * w + j];
    }
}

}  // namespace gs

using namespace gs;

extern "C" int gs_spatial_order(gs_ctx* c, const float* means, int64_t n, int32_t* perm, void* stream)
{
    if (!c || n < 0 || (n > 0 && (!means || !perm)) || n > (int64_t)INT32_MAX) return GS_ERR_INVALID_ARG;
    if (n == 0) return GS_OK;
    const cudaStream_t st = (cudaStream_t)stream;
    const int nparts = c->num_sms * 2;
    // workspace: partials [nparts][6], lo/s [6], m (int64), offsets [2],
    // sort input (gs_isect_bytes(n)), sorted words [n]
    const size_t o_part = 0;
    const size_t o_los = align256(o_part + (size_t)nparts * 6 * sizeof(float));
    const size_t o_m = align256(o_los + 6 * sizeof(float));
    const size_t o_off = align256(o_m + sizeof(int64_t));
    const size_t o_is = align256(o_off + 2 * sizeof(int32_t));
    const size_t o_words = align256(o_is + gs_isect_bytes(n));
    const size_t bytes = o_words + (size_t)n * sizeof(uint64_t);
    int r = ensure(&c->d_order_ws, &c->order_ws_cap, bytes);
    if (r != GS_OK) return r;
    char* b = static_cast<char*>(c->d_order_ws);
    float* part = reinterpret_cast<float*>(b + o_part);
    float* los = reinterpret_cast<float*>(b + o_los);
    int64_t* m_dev = reinterpret_cast<int64_t*>(b + o_m);
    int32_t* offsets = reinterpret_cast<int32_t*>(b + o_off);
    const IsectView is = isect_view(b + o_is, n);
    uint64_t* words = reinterpret_cast<uint64_t*>(b + o_words);

    const int64_t want = (n + kOrderThreads - 1) / kOrderThreads;
    const unsigned grid = (unsigned)(want < (int64_t)c->num_sms * 8 ? want : (int64_t)c->num_sms * 8);
    const unsigned pgrid = (unsigned)(want < nparts ? want : nparts);
    k_bounds_partial<<<pgrid, kOrderThreads, 0, st>>>(means, n, part);
    k_bounds_final<<<1, 32, 0, st>>>(part, (int)pgrid, los, m_dev, n);
    k_morton<<<grid, kOrderThreads, 0, st>>>(means, n, los, is);
    c->launches += 3;
    GS_CUDA_TRY(cudaGetLastError());
    if ((r = global_sort(c, is, n, m_dev, 1, words, offsets, st)) != GS_OK) return r;
    k_perm_from_words<<<grid, kOrderThreads, 0, st>>>(words, n, perm);
    c->launches += 1;
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

extern "C" int gs_gather_rows(gs_ctx* c, const int32_t* perm, int64_t n, const float* src, int32_t width,
                              float* dst, void* stream)
{
    if (!c || n < 0 || width < 1 || (n > 0 && (!perm || !src || !dst))) return GS_ERR_INVALID_ARG;
    if (n == 0) return GS_OK;
    if (src == dst) return GS_ERR_INVALID_ARG;  // a gather cannot run in place
    const int64_t total = n * (int64_t)width;
    const int64_t want = (total + kOrderThreads - 1) / kOrderThreads;
    const unsigned grid = (unsigned)(want < (int64_t)c->num_sms * 8 ? want : (int64_t)c->num_sms * 8);
    k_gather_rows<<<grid, kOrderThreads, 0, (cudaStream_t)stream>>>(perm, n, src, width, dst, c->d_err);
    c->launches += 1;
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}
