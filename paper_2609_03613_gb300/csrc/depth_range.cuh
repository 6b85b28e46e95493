// depth_range.cuh -- the robust depth-range estimate (supplement, "Robust
// depth-range estimation", Alg. 2) as the body of one block, and the bin
// parameters it feeds (the log-depth-bin formula; monotone split depths for
// EXACT mode).  Used per frame by bins.cu and per view by batch_bins.cu.
#pragma once
#include "device.cuh"

namespace gs {

// ------------------------------------------------------------------ depth range
constexpr int kDrThreads = 1024;
constexpr int kDrMaxS = 8192;

struct DrArgs {
    float near_plane, far_plane;
    int S;
    int near_shift;
    float near_alpha, near_gamma;
    float p_lo, p_hi, pad, eps;
    int K;
};

__device__ __forceinline__ float zkey_of(float z, const float* __restrict__ scales, uint32_t g, float a, float gm)
{
    const float s0 = __ldg(scales + 3 * (size_t)g), s1 = __ldg(scales + 3 * (size_t)g + 1),
                s2 = __ldg(scales + 3 * (size_t)g + 2);
    const float smax = fmaxf(fmaxf(s0, s1), s2);
    return z - fminf(a * smax, gm * z);
}

__device__ __forceinline__ int64_t rank_of(float p, int64_t n)
{
    int64_t k = (int64_t)ceil((double)p / 100.0 * (double)n);
    if (k < 1) k = 1;
    if (k > n) k = n;
    return k;
}

// Bin parameters from [zmin, zmax]: z'min = max(zmin, eps),
// z'max = max(zmax, z'min + 1e-6), lmin/lmax their logs, and K-1 log-spaced
// split depths exp(lmin + (lmax - lmin) k/K), kept non-decreasing.
__device__ __forceinline__ void write_bin_params(BinParams* bp, float zmin, float zmax, int K, float eps, int nsamples)
{
    __shared__ float s_l[2];
    if (threadIdx.x == 0) {
        const float zmn = fmaxf(zmin, eps);
        const float zmx = fmaxf(zmax, zmn + 1e-6f);
        s_l[0] = spec_log(zmn);
        s_l[1] = spec_log(zmx);
        bp->zmin = zmin;
        bp->zmax = zmax;
        bp->lmin = s_l[0];
        bp->lmax = s_l[1];
        bp->K = K;
        bp->nsamples = nsamples;
    }
    __syncthreads();
    __shared__ float s_split[GS_MAX_K];
    const float lmin = s_l[0], lmax = s_l[1];
    for (int k = 1 + threadIdx.x; k < K; k += blockDim.x) {
        const float t = (float)k / (float)K;
        s_split[k - 1] = spec_exp(lmin + (lmax - lmin) * t);
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 1; k < K - 1; ++k)
            if (s_split[k] < s_split[k - 1]) s_split[k] = s_split[k - 1];
    __syncthreads();
    for (int k = threadIdx.x; k < K - 1; k += blockDim.x) bp->splits[k] = s_split[k];
}

// ... or from a per-sample gid array (the batched views' sampling).
struct GidFromSamples {
    static constexpr bool kKeys = false;
    const uint32_t* gid;  // indexed by sample number
    __device__ uint32_t operator()(int64_t i, int64_t) const { return gid[i]; }
};

// ... or the samples' keys themselves (depth, or the near-shifted key, as
// float bits), gathered by the wide sampling kernel.
struct KeyFromSamples {
    static constexpr bool kKeys = true;
    const uint32_t* key;  // indexed by sample number
    __device__ uint32_t operator()(int64_t i, int64_t) const { return key[i]; }
};

// The key of Gaussian g's depth sample: its depth, or the near-shifted key.
__device__ __forceinline__ float sample_key(const float4* __restrict__ c_o_z, const float* __restrict__ scales,
                                            uint32_t g, const DrArgs& a)
{
    float z = c_o_z[g].z;
    if (a.near_shift) z = zkey_of(z, scales, g, a.near_alpha, a.near_gamma);
    return z;
}

// Rank search of one radix pass, by one warp: the digit d whose cumulative
// count first reaches k (k >= 1), and k minus the counts below d, written by
// the one lane that returns true.  Lane l holds digits 8l .. 8l+7.
__device__ __forceinline__ bool warp_digit_select(const uint32_t* __restrict__ h, int64_t k, uint32_t* dsel,
                                                  int64_t* krem)
{
    const int lane = threadIdx.x & 31;
    uint32_t c[8], sum = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        c[j] = h[8 * lane + j];
        sum += c[j];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += u;
    }
    const unsigned hit = __ballot_sync(0xffffffffu, (int64_t)incl >= k);
    const int L = hit ? __ffs(hit) - 1 : 31;
    const uint32_t before = __shfl_sync(0xffffffffu, incl - sum, L);
    if (lane == L) {
        int64_t kk = k - (int64_t)before;
        uint32_t d = 8u * L + 7u;
        for (int j = 0; j < 8; ++j) {
            if ((int64_t)c[j] >= kk) {
                d = 8u * L + j;
                break;
            }
            kk -= c[j];
        }
        *dsel = d;
        *krem = kk;
    }
    return lane == L;
}

// Alg. 2 by one block of kDrThreads threads over the first S' = min(S, M)
// samples gid_of(i, floor(i M / S')) of M entries: the positive depths (or
// near-shifted keys) clamped to [max(near, eps), far], their exact p_lo / p_hi
// order statistics by radix select, padded by pad of the span; the bin
// parameters of [zmin, zmax] are written to bp.
template <class GidOf>
__device__ __forceinline__ void depth_range_block(const float4* __restrict__ c_o_z, const float* __restrict__ scales,
                                                  GidOf gid_of, int64_t M, const DrArgs& a, BinParams* bp)
{
    __shared__ uint32_t s_v[kDrMaxS];
    __shared__ int s_n;
    __shared__ uint32_t s_h[2][256];
    __shared__ uint32_t s_pref[2];
    __shared__ int64_t s_k[2];
    __shared__ int s_low;
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    const int64_t ns = M < (int64_t)a.S ? M : (int64_t)a.S;
    const float lo_clamp = fmaxf(a.near_plane, a.eps);
    // every sample's key: read (the sampling kernel gathered them), or its
    // gid then its depth (and scale) gathered at once, so the dependent loads
    // cost two round trips rather than two per round
    constexpr int kPer = kDrMaxS / kDrThreads;
    float zk[kPer];
    if constexpr (GidOf::kKeys) {
#pragma unroll
        for (int r = 0; r < kPer; ++r) {
            const int64_t i = (int64_t)r * kDrThreads + threadIdx.x;
            zk[r] = i < ns ? __uint_as_float(gid_of(i, 0)) : 0.0f;
        }
    } else {
        uint32_t gk[kPer];
#pragma unroll
        for (int r = 0; r < kPer; ++r) {
            const int64_t i = (int64_t)r * kDrThreads + threadIdx.x;
            gk[r] = i < ns ? gid_of(i, (i * M) / ns) : 0u;
        }
#pragma unroll
        for (int r = 0; r < kPer; ++r) {
            const int64_t i = (int64_t)r * kDrThreads + threadIdx.x;
            zk[r] = i < ns ? sample_key(c_o_z, scales, gk[r], a) : 0.0f;
        }
    }
    // the positive keys, clamped, compacted with one shared atomic per warp
    // and round; their minimum and maximum on the way
    uint32_t lo_v = 0xffffffffu, hi_v = 0u;
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
        const int64_t i = (int64_t)r * kDrThreads + threadIdx.x;
        const float z = zk[r];
        const bool keep = i < ns && z > 0.0f;
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        const int lane = threadIdx.x & 31;
        int base = 0;
        if (lane == 0 && bal) base = atomicAdd(&s_n, __popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (keep) {
            const uint32_t v = __float_as_uint(fminf(fmaxf(z, lo_clamp), a.far_plane));
            s_v[base + __popc(bal & ((1u << lane) - 1u))] = v;
            lo_v = min(lo_v, v);
            hi_v = max(hi_v, v);
        }
    }
    __syncthreads();
    const int n = s_n;
    float zmin, zmax;
    if (n == 0) {
        zmin = lo_clamp;
        zmax = a.far_plane;
    } else {
        // the bits every sample shares (those of the block's min and max)
        // need no pass: start below the highest bit where samples differ
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        lo_v = __reduce_min_sync(0xffffffffu, lo_v);
        hi_v = __reduce_max_sync(0xffffffffu, hi_v);
        if (lane == 0) {
            s_h[0][warp] = lo_v;
            s_h[1][warp] = hi_v;
        }
        __syncthreads();
        if (warp == 0) {
            const int nw = blockDim.x >> 5;
            lo_v = __reduce_min_sync(0xffffffffu, lane < nw ? s_h[0][lane] : 0xffffffffu);
            hi_v = __reduce_max_sync(0xffffffffu, lane < nw ? s_h[1][lane] : 0u);
            if (lane == 0) {
                const int cp = lo_v == hi_v ? 32 : __clz(lo_v ^ hi_v);
                const uint32_t top = cp == 32 ? 0xffffffffu : (cp == 0 ? 0u : ~(0xffffffffu >> cp));
                s_pref[0] = s_pref[1] = lo_v & top;
                s_k[0] = rank_of(a.p_lo, n);
                s_k[1] = rank_of(a.p_hi, n);
                s_low = 32 - cp;  // bits still to select
            }
        }
        __syncthreads();
        const int low = s_low;
        uint32_t mask = low >= 32 ? 0u : ~((1u << low) - 1u);
        // radix select (positive floats: bit order = value order), <= 8 bits a pass
        for (int hi_bit = low; hi_bit > 0; hi_bit -= 8) {
            const int shift = hi_bit > 8 ? hi_bit - 8 : 0;
            const uint32_t dmask = (1u << (hi_bit - shift)) - 1u;
            for (int d = threadIdx.x; d < 512; d += blockDim.x) s_h[d >> 8][d & 255] = 0u;
            __syncthreads();
            const uint32_t p0 = s_pref[0], p1 = s_pref[1];
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const uint32_t v = s_v[i];
                const uint32_t dg = (v >> shift) & dmask;
                if ((v & mask) == p0) atomicAdd(&s_h[0][dg], 1u);
                if ((v & mask) == p1) atomicAdd(&s_h[1][dg], 1u);
            }
            __syncthreads();
            if (warp < 2) {
                uint32_t dsel = 0u;
                int64_t krem = 0;
                if (warp_digit_select(s_h[warp], s_k[warp], &dsel, &krem)) {
                    s_k[warp] = krem;
                    s_pref[warp] |= dsel << shift;
                }
            }
            mask |= dmask << shift;
            __syncthreads();
        }
        const float zlo = __uint_as_float(s_pref[0]);
        const float zhi = __uint_as_float(s_pref[1]);
        const float span = fmaxf(zhi - zlo, 1e-6f);
        zmin = fmaxf(a.near_plane, zlo - a.pad * span);
        zmax = fminf(a.far_plane, zhi + a.pad * span);
    }
    write_bin_params(bp, zmin, zmax, a.K, a.eps, n);
}

}  // namespace gs
