// device.cuh -- device helpers shared by several kernels: the warp-cooperative
// (Gaussian -> covered tiles) expansion, the monotone bin map, and the
// bitonic sorting networks used by the repair sorts.
#pragma once

#include "internal.cuh"

namespace gs {

// ------------------------------------------------------------------ expansion
// A warp owns 32 consecutive Gaussians, whose entries occupy one contiguous
// range of the emission order (their scanned offsets are consecutive).  Each
// lane takes every 32nd entry of that range, finds its Gaussian by a binary
// search over the 32 offsets held in the warp's lanes, and derives the tile
// from its index inside the Gaussian's rect (row-major).
struct WarpExpand {
    int32_t my_off;   // offset of this lane's Gaussian
    uint32_t r0, r1;  // its rect
    uint32_t zb;      // its depth bits
    int32_t base, end;
    int64_t g0;

    __device__ __forceinline__ WarpExpand(const uint2* __restrict__ rect, const float4* __restrict__ c_o_z,
                                          const int32_t* __restrict__ goff, int64_t n, int64_t g0_)
        : g0(g0_)
    {
        const int lane = threadIdx.x & 31;
        const int64_t gl = g0 + lane;
        const bool ok = gl < n;
        my_off = goff[ok ? gl : n];
        const uint2 r = ok ? rect[gl] : make_uint2(0u, 0u);
        r0 = r.x;
        r1 = r.y;
        zb = ok ? __float_as_uint(c_o_z[gl].z) : 0u;
        base = __shfl_sync(0xffffffffu, my_off, 0);
        end = goff[(g0 + 32) < n ? (g0 + 32) : n];
    }

    // Entry e (all lanes call it together): gid, tile and depth bits.
    __device__ __forceinline__ void entry(int32_t e, int tiles_x, uint32_t* gid, uint32_t* tile, uint32_t* z) const
    {
        int k = 0;
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) {
            const int32_t v = __shfl_sync(0xffffffffu, my_off, (k + s) & 31);
            if (k + s < 32 && v <= e) k += s;
        }
        const uint32_t a = __shfl_sync(0xffffffffu, r0, k), b = __shfl_sync(0xffffffffu, r1, k);
        const int32_t o = __shfl_sync(0xffffffffu, my_off, k);
        *z = __shfl_sync(0xffffffffu, zb, k);
        const uint32_t tx0 = a & 0xffffu, ty0 = a >> 16, w = (b & 0xffffu) - tx0;
        const uint32_t l = (uint32_t)(e - o);
        const uint32_t dy = w ? l / w : 0u, dx = l - dy * w;
        *tile = (ty0 + dy) * (uint32_t)tiles_x + tx0 + dx;
        *gid = (uint32_t)(g0 + k);
    }
};


// ------------------------------------------------------------------ bin maps
// Monotone map: the number of split depths <= z (binary search over the
// non-decreasing split list).
__device__ __forceinline__ int bin_split(float z, const float* s_split, int K)
{
    int lo = 0, hi = K - 1;  // answer in [0, K-1]
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (s_split[mid] <= z) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}


// ------------------------------------------------------------------ segment sorts
// All sorts order the 64-bit words (depth bits << 32 | gid) ascending.
// Bitonic networks in the form where every compare-exchange puts the minimum
// at the lower index (a mirrored compare at the first step of each merge), so
// positions past the segment end behave as +infinity and can be skipped.

__device__ __forceinline__ void cex(uint64_t* a, int i, int l)
{
    const uint64_t x = a[i], y = a[l];
    if (y < x) {
        a[i] = y;
        a[l] = x;
    }
}

struct SyncWarp {
    __device__ void operator()() const { __syncwarp(); }
};
struct SyncBlock {
    __device__ void operator()() const { __syncthreads(); }
};

// Sort a[0..n) held in (shared or global) memory by `nthreads` cooperating
// threads with index `tid`; `sync` is called between steps.
template <class Sync>
__device__ void bitonic_mem(uint64_t* a, int n, int tid, int nthreads, Sync sync)
{
    int P = 1, lp = 0;
    while (P < n) {
        P <<= 1;
        ++lp;
    }
    // all strides are powers of two: index arithmetic by shifts and masks
    for (int lk = 1; lk <= lp; ++lk) {
        const int k = 1 << lk, h = k >> 1;
        for (int t = tid; t < P / 2; t += nthreads) {
            const int r = t & (h - 1);
            const int i = ((t >> (lk - 1)) << lk) + r, l = i + (k - 1 - 2 * r);
            if (l < n) cex(a, i, l);
        }
        sync();
        for (int lj = lk - 2; lj >= 0; --lj) {
            const int j = 1 << lj;
            for (int t = tid; t < P / 2; t += nthreads) {
                const int i = ((t >> lj) << (lj + 1)) | (t & (j - 1)), l = i + j;
                if (l < n) cex(a, i, l);
            }
            sync();
        }
    }
}

// 32 words, one per lane, sorted ascending across the warp.
__device__ __forceinline__ uint64_t warp_bitonic32(uint64_t v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const uint64_t o = __shfl_xor_sync(0xffffffffu, v, j);
            const bool up = ((lane & k) == 0);
            const bool lower = ((lane & j) == 0);
            // lower lane of an ascending pair keeps the min, etc.
            const bool take_min = (lower == up);
            v = take_min ? (o < v ? o : v) : (o > v ? o : v);
        }
    }
    return v;
}


// 33..64 words a[0..n) sorted ascending by one warp in registers: lane l
// holds positions l and l + 32 (past n: +infinity, above every word, whose
// depth bits are those of a finite float), one bitonic network over the 64
// positions; a stride-32 step pairs the two words of one lane.
__device__ __forceinline__ void warp_bitonic64(uint64_t* a, int n)
{
    const int lane = threadIdx.x & 31;
    uint64_t x0 = a[lane];
    uint64_t x1 = lane + 32 < n ? a[lane + 32] : ~0ull;
#pragma unroll
    for (int k = 2; k <= 64; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j == 32) {  // k = 64: ascending
                const uint64_t lo = x1 < x0 ? x1 : x0, hi = x1 < x0 ? x0 : x1;
                x0 = lo;
                x1 = hi;
                continue;
            }
            const bool lower = (lane & j) == 0;
            // position i = h * 32 + lane sorts ascending when (i & k) == 0
            const bool up0 = k == 64 || (lane & k) == 0;
            const bool up1 = k == 64 || (k < 32 && (lane & k) == 0);
            const uint64_t o0 = __shfl_xor_sync(0xffffffffu, x0, j);
            const uint64_t o1 = __shfl_xor_sync(0xffffffffu, x1, j);
            x0 = (lower == up0) ? (o0 < x0 ? o0 : x0) : (o0 > x0 ? o0 : x0);
            x1 = (lower == up1) ? (o1 < x1 ? o1 : x1) : (o1 > x1 ? o1 : x1);
        }
    }
    a[lane] = x0;
    if (lane + 32 < n) a[lane + 32] = x1;
}

// ------------------------------------------------------------------ tile cull
// True when no pixel centre of the tile can give alpha >= 1/255 (nor a
// q < 0 skip would change anything).  Minimum of the quadratic
// Q = ha dx^2 + hb dx dy + hc dy^2 over the tile's (slightly widened) box of
// pixel offsets; the unconstrained minimum (0) outside the box puts the
// constrained one on an edge.  margin < 1 covers float32 cancellation in the
// per-pixel q (it shrinks with the conditioning of the conic; 0 = never cull).
__device__ __forceinline__ bool tile_culled(float mx, float my, float ha, float hb, float hc, float tau,
                                            float margin, float x0, float y0, float span)
{
    if (!(margin > 0.0f)) return false;
    float xl = mx - (x0 + span - 0.5f), xh = mx - (x0 + 0.5f);
    float yl = my - (y0 + span - 0.5f), yh = my - (y0 + 0.5f);
    xl = xl - 1e-3f * (1.0f + fabsf(xl));
    xh = xh + 1e-3f * (1.0f + fabsf(xh));
    yl = yl - 1e-3f * (1.0f + fabsf(yl));
    yh = yh + 1e-3f * (1.0f + fabsf(yh));
    if (xl <= 0.0f && xh >= 0.0f && yl <= 0.0f && yh >= 0.0f) return false;
    const float ry = -hb / (2.0f * hc), rx = -hb / (2.0f * ha);
    float qmin = 3.0e38f;
    {
        const float X = xl, Yc = fminf(fmaxf(ry * X, yl), yh);
        qmin = fminf(qmin, ha * X * X + hb * X * Yc + hc * Yc * Yc);
    }
    {
        const float X = xh, Yc = fminf(fmaxf(ry * X, yl), yh);
        qmin = fminf(qmin, ha * X * X + hb * X * Yc + hc * Yc * Yc);
    }
    {
        const float Y = yl, Xc = fminf(fmaxf(rx * Y, xl), xh);
        qmin = fminf(qmin, ha * Xc * Xc + hb * Xc * Y + hc * Y * Y);
    }
    {
        const float Y = yh, Xc = fminf(fmaxf(rx * Y, xl), xh);
        qmin = fminf(qmin, ha * Xc * Xc + hb * Xc * Y + hc * Y * Y);
    }
    return qmin * margin > tau;
}

// The same test for entry (g, tile t) straight from the projected records.
__device__ __forceinline__ bool entry_culled(const float4* __restrict__ xy_ab, const float4* __restrict__ c_o_z,
                                             const float4* __restrict__ rgbv, uint32_t g, uint32_t t, int tiles_x,
                                             int tile)
{
    const float4 p = __ldg(xy_ab + g);
    const float4 q = __ldg(c_o_z + g);
    const float margin = __ldg(&rgbv[g].w);
    const int tx = (int)(t % (uint32_t)tiles_x), ty = (int)(t / (uint32_t)tiles_x);
    return tile_culled(p.x, p.y, 0.5f * p.z, p.w, 0.5f * q.x, q.w, margin, (float)(tx * tile), (float)(ty * tile),
                       (float)tile);
}

}  // namespace gs
