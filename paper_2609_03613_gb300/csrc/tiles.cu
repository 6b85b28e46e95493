// tiles.cu -- bin construction for EXACT mode (Sec. 3.3; supplement Alg. 3),
// arranged for GB300.  With the monotone split map every entry of a Gaussian
// falls in the same bin b(z_g), so:
//
//   1. count[t, b]: each Gaussian adds its tile rect to layer b of a stack of
//      K 2D difference arrays over the tile grid (four atomics per Gaussian
//      instead of one per entry); per-layer 2D prefix sums give the counts;
//   2. exclusive scan of count in tile-major, bin-minor order -> bin offsets
//      (the same array Alg. 3's global count/scan produces);
//   3. scatter: each entry takes a slot in its (t, b) segment from an atomic
//      cursor -- straight from the Gaussians' rects (warp-cooperative
//      expansion, the emission-order entries are never written) or from
//      materialised entries.
//
// The order inside a segment is left to the repair (Alg. 4): an eager sort of
// every segment, or the raster's in-shared-memory sort of each segment it
// reaches (segments too long for its buffer are sorted here, eagerly).
#include "device.cuh"
#include "rows.cuh"
#include "scan.cuh"

namespace gs {

// ------------------------------------------------------------------ counts
// Per visible Gaussian: its bin (kept in gbin) and its rect added to layer b.
__global__ void __launch_bounds__(256)
k_bin_diff(const uint2* __restrict__ rect, const float4* __restrict__ c_o_z, int64_t n, int tiles_x, int tiles_y,
           const BinParams* __restrict__ bp, int K, int32_t* __restrict__ D, uint8_t* __restrict__ gbin)
{
    __shared__ float s_split[GS_MAX_K];
    for (int k = threadIdx.x; k < K - 1; k += blockDim.x) s_split[k] = bp->splits[k];
    __syncthreads();
    const int W1 = tiles_x + 1;
    const int64_t layer = (int64_t)(tiles_y + 1) * W1;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += stride) {
        const uint2 r = rect[g];
        const int tx0 = r.x & 0xffff, ty0 = r.x >> 16, tx1 = r.y & 0xffff, ty1 = r.y >> 16;
        if (tx0 >= tx1 || ty0 >= ty1) continue;
        const int b = bin_split(c_o_z[g].z, s_split, K);
        gbin[g] = (uint8_t)b;
        int32_t* L = D + b * layer;
        atomicAdd(&L[ty0 * W1 + tx0], 1);
        atomicAdd(&L[ty0 * W1 + tx1], -1);
        atomicAdd(&L[ty1 * W1 + tx0], -1);
        atomicAdd(&L[ty1 * W1 + tx1], 1);
    }
}

// One block per layer: 2D inclusive prefix (columns, then rows) in place.
__global__ void __launch_bounds__(1024)
k_layer_prefix(int32_t* __restrict__ D, int tiles_x, int tiles_y)
{
    const int W1 = tiles_x + 1;
    int32_t* L = D + (int64_t)blockIdx.x * (tiles_y + 1) * W1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int x = threadIdx.x; x < tiles_x; x += blockDim.x) {
        int32_t run = 0;
        for (int y = 0; y < tiles_y; ++y) {
            run += L[y * W1 + x];
            L[y * W1 + x] = run;
        }
    }
    __syncthreads();
    for (int y = warp; y < tiles_y; y += blockDim.x / 32) {
        int32_t carry = 0;
        for (int x0 = 0; x0 < tiles_x; x0 += 32) {
            const int x = x0 + lane;
            int32_t v = x < tiles_x ? L[y * W1 + x] : 0;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int32_t u = __shfl_up_sync(0xffffffffu, v, d);
                if (lane >= d) v += u;
            }
            if (x < tiles_x) L[y * W1 + x] = carry + v;
            carry += __shfl_sync(0xffffffffu, v, 31);
        }
    }
}

// ------------------------------------------------------------------ row spans (tile cull): rows.cuh

struct LoadRectRows {
    const uint2* rect;
    __device__ int64_t operator()(int64_t i) const
    {
        const uint2 r = rect[i];
        const int64_t w = (int64_t)(r.y & 0xffffu) - (int64_t)(r.x & 0xffffu);
        const int64_t h = (int64_t)(r.y >> 16) - (int64_t)(r.x >> 16);
        return (w > 0 && h > 0) ? h : 0;
    }
};

// Warp-cooperative over (Gaussian, row) pairs: a warp owns 32 consecutive
// Gaussians, whose rows are consecutive records [roff[g0], roff[g0 + 32)).
// Each lane holds its Gaussian (record, bin); every row record is computed by
// one lane from the owner's values (shuffled): the row's culled span, the
// record (gid, row | start, width), and +1 / -1 at the span ends of layer b's
// row (a per-row difference array).
__global__ void __launch_bounds__(256)
k_row_spans(const uint2* __restrict__ rect, int64_t n, const int32_t* __restrict__ roff, CullArgs ca, int tiles_x,
            const BinParams* __restrict__ bp, int K, const int64_t* __restrict__ m_dev, int64_t m_cap,
            int32_t* __restrict__ Drow, int64_t layer, uint8_t* __restrict__ gbin, uint32_t* __restrict__ rs_g,
            uint32_t* __restrict__ rs_ya, uint32_t* __restrict__ rs_w, uint32_t* __restrict__ rs_z)
{
    grid_dependency_sync();
    __shared__ float s_split[GS_MAX_K];
    for (int k = threadIdx.x; k < K - 1; k += blockDim.x) s_split[k] = bp->splits[k];
    __syncthreads();
    if (*m_dev > m_cap) return;
    const int64_t g0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32;
    if (g0 >= n) return;
    const int lane = threadIdx.x & 31;
    const int64_t gl = g0 + lane;
    const bool ok = gl < n;
    const int32_t my_off = roff[ok ? gl : n];
    const int32_t base = __shfl_sync(0xffffffffu, my_off, 0);
    const int32_t end = roff[(g0 + 32) < n ? (g0 + 32) : n];
    uint2 r = make_uint2(0u, 0u);
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f), q = p;
    float margin = 0.0f;
    uint32_t bin = 0u;
    if (ok) {
        r = rect[gl];
        if ((r.x & 0xffffu) < (r.y & 0xffffu) && (r.x >> 16) < (r.y >> 16)) {
            p = __ldg(ca.xy_ab + gl);
            q = __ldg(ca.c_o_z + gl);
            margin = __ldg(&ca.rgb[gl].w);
            bin = (uint32_t)bin_split(q.z, s_split, K);
            gbin[gl] = (uint8_t)bin;
        }
    }
    const RowGeom mine = row_geom(0.5f * p.z, p.w, 0.5f * q.x, q.w, margin, p.y);
    const float inv_tile = 1.0f / (float)ca.tile;  // exact: tiles are 8, 16 or 32
    const int W1 = tiles_x + 1;
    for (int32_t e0 = base; e0 < end; e0 += 32) {
        const int32_t e = e0 + lane;
        int k = 0;
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) {
            const int32_t v = __shfl_sync(0xffffffffu, my_off, (k + s) & 31);
            if (k + s < 32 && v <= e) k += s;
        }
        const uint32_t ra = __shfl_sync(0xffffffffu, r.x, k), rb = __shfl_sync(0xffffffffu, r.y, k);
        const float mx = __shfl_sync(0xffffffffu, p.x, k);
        RowGeom g;
        g.my = __shfl_sync(0xffffffffu, mine.my, k);
        g.hb = __shfl_sync(0xffffffffu, mine.hb, k);
        g.inv2ha = __shfl_sync(0xffffffffu, mine.inv2ha, k);
        g.a4tp = __shfl_sync(0xffffffffu, mine.a4tp, k);
        g.D = __shfl_sync(0xffffffffu, mine.D, k);
        g.dymax = __shfl_sync(0xffffffffu, mine.dymax, k);
        g.ext = __shfl_sync(0xffffffffu, mine.ext, k);
        g.dyl = __shfl_sync(0xffffffffu, mine.dyl, k);
        const uint32_t zb = __shfl_sync(0xffffffffu, __float_as_uint(q.z), k);
        const uint32_t b = __shfl_sync(0xffffffffu, bin, k);
        const int32_t o = __shfl_sync(0xffffffffu, my_off, k);
        if (e < end) {
            const int tx0 = ra & 0xffff, ty0 = ra >> 16, tx1 = rb & 0xffff;
            const int ty = ty0 + (e - o);
            int a, x1;
            row_span(mx, g, ty, ca.tile, inv_tile, tx0, tx1, &a, &x1);
            rs_g[e] = (uint32_t)(g0 + k);
            rs_ya[e] = row_record(ty, a, b);
            rs_w[e] = (uint32_t)(x1 - a);
            rs_z[e] = zb;
            if (x1 > a) {
                int32_t* L = Drow + b * layer;
                atomicAdd(&L[ty * W1 + a], 1);
                atomicAdd(&L[ty * W1 + x1], -1);
            }
        }
    }
}

// One block per layer: inclusive prefix along each row.
__global__ void __launch_bounds__(1024)
k_layer_rows_prefix(int32_t* __restrict__ D, int tiles_x, int tiles_y, int64_t layer)
{
    grid_dependency_sync();
    const int W1 = tiles_x + 1;
    int32_t* L = D + (int64_t)blockIdx.x * layer;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int y = warp; y < tiles_y; y += blockDim.x / 32) {
        int32_t carry = 0;
        for (int x0 = 0; x0 < tiles_x; x0 += 32) {
            const int x = x0 + lane;
            int32_t v = x < tiles_x ? L[y * W1 + x] : 0;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int32_t u = __shfl_up_sync(0xffffffffu, v, d);
                if (lane >= d) v += u;
            }
            if (x < tiles_x) L[y * W1 + x] = carry + v;
            carry += __shfl_sync(0xffffffffu, v, 31);
        }
    }
}

// Warp-cooperative over the entries of 64 consecutive row records, two a
// lane: a warp scans the lanes' record widths and keeps its records (gid,
// tile row | first tile | bin, depth bits, first entry) in shared memory;
// then, a window of 384 entries at a time, each record marks the window's
// entries that are its own in a per-warp owner map, and each lane takes
// every 32nd entry, reads its record through the map and takes a slot in the
// entry's (tile, bin) segment -- the cursors start at the segment offsets, so
// the atomic returns the slot itself.  Twelve entries per lane are in flight:
// the kernel waits on its atomics' returns.  Measured at 1080p against a
// binary search over the warp's prefix with the fields shuffled from the
// owning lane: one record a lane and four in flight 13.6 us slower, two
// records and twelve in flight 6.7 us slower (short-scoreboard stalls on
// the shuffles); with the owner map, four records a lane were slower.  The
// records carry the Gaussian's bin and depth bits, so nothing is gathered.
constexpr int kScatRL = 2;                 // row records a lane
constexpr int kScatIF = 12;                // entries a lane has in flight
constexpr int kScatWin = 32 * kScatIF;     // entries a warp places a round

__global__ void __launch_bounds__(256)
k_bin_scatter_rows(const uint32_t* __restrict__ rs_g, const uint32_t* __restrict__ rs_ya, const uint32_t* __restrict__ rs_w,
                   const uint32_t* __restrict__ rs_z, const int32_t* __restrict__ roff, int64_t n, int tiles_x, int K,
                   const int64_t* __restrict__ m_dev, int64_t m_cap, int32_t* __restrict__ cur,
                   uint64_t* __restrict__ words, const ScatterPass sp, const int32_t* __restrict__ flagged)
{
    grid_dependency_sync();
    // per warp: its 64 records {gid, tile row | first tile | bin, depth bits,
    // first entry}, and for a round's window of entries the record of each
    __shared__ uint4 s_rec[8][32 * kScatRL];
    __shared__ uint8_t s_own[8][kScatWin];
    if (*m_dev > m_cap) return;
    if (sp.pass == 2 && flagged[0] == 0) return;  // no tile to complete
    const int64_t R = roff[n];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint4* rec = s_rec[warp];
    uint8_t* own = s_own[warp];
    const int64_t nchunks = (R + 32 * kScatRL - 1) / (32 * kScatRL);
    const int64_t wstride = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; c < nchunks; c += wstride) {
        uint32_t w[kScatRL], g[kScatRL], ya[kScatRL], z[kScatRL];
#pragma unroll
        for (int h = 0; h < kScatRL; ++h) {
            w[h] = g[h] = ya[h] = z[h] = 0;
            const int64_t k = c * (32 * kScatRL) + kScatRL * lane + h;
            if (k < R) {  // read once: streamed past L2
                ya[h] = __ldcs(rs_ya + k);
                w[h] = __ldcs(rs_w + k);
                g[h] = __ldcs(rs_g + k);
                z[h] = __ldcs(rs_z + k);
                if (sp.row_live((int)(ya[h] & 0xfffu))) sp.trim(ya[h], w[h], tiles_x);
                else w[h] = 0;
            }
        }
        uint32_t wl = 0;
#pragma unroll
        for (int h = 0; h < kScatRL; ++h) wl += w[h];
        uint32_t incl = wl;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += u;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        uint32_t st[kScatRL];
        st[0] = incl - wl;
#pragma unroll
        for (int h = 1; h < kScatRL; ++h) st[h] = st[h - 1] + w[h - 1];
#pragma unroll
        for (int h = 0; h < kScatRL; ++h) rec[kScatRL * lane + h] = make_uint4(g[h], ya[h], z[h], st[h]);
        for (uint32_t e0 = 0; e0 < total; e0 += kScatWin) {
            // each record marks the entries of this window that are its own
#pragma unroll
            for (int h = 0; h < kScatRL; ++h) {
                const uint32_t lo = st[h] > e0 ? st[h] : e0;
                const uint32_t end = st[h] + w[h], wend = e0 + kScatWin;
                const uint32_t hi = end < wend ? end : wend;
                for (uint32_t x = lo; x < hi; ++x) own[x - e0] = (uint8_t)(kScatRL * lane + h);
            }
            __syncwarp();
            int32_t p[kScatIF];
            uint64_t word[kScatIF];
            bool live[kScatIF];
#pragma unroll
            for (int u = 0; u < kScatIF; ++u) {
                const uint32_t e = e0 + 32 * u + lane;
                live[u] = e < total;
                if (live[u]) {
                    const uint4 r = rec[own[e - e0]];
                    const uint32_t oya = r.y;
                    const int ty = (int)(oya & 0xfffu), tx = (int)((oya >> 12) & 0xfffu) + (int)(e - r.w);
                    const int64_t t = (int64_t)ty * tiles_x + tx;
                    live[u] = sp.keep(t, (int)(oya >> 24));
                    if (live[u]) {
                        p[u] = atomicAdd(&cur[t * K + (oya >> 24)], 1);
                        word[u] = ((uint64_t)r.z << 32) | r.x;
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kScatIF; ++u)
                if (live[u]) words[p[u]] = word[u];
            __syncwarp();  // the window's owner map is read before the next one is written
        }
        __syncwarp();  // the records are read before the next chunk's are written
    }
}

// The completing pass's cursors: those of every flagged tile start at its
// segment offsets (the first pass placed none of the bins it leaves).
__global__ void k_flagged_cursors(const int32_t* __restrict__ list, const int32_t* __restrict__ offsets, int K,
                                  int32_t* __restrict__ cur)
{
    grid_dependency_sync();
    const int32_t nl = list[0];
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nl * K; i += gridDim.x * blockDim.x) {
        const int64_t q = (int64_t)list[1 + i / K] * K + i % K;
        cur[q] = offsets[q];
    }
}

// ------------------------------------------------------------------ scatter by (row, bin) groups
// For deep frames the per-entry cursor atomics in global memory are the
// bin construction's limit.  Here the row records are first grouped by
// (tile row, bin) -- a counting pass and a writing pass over C slices of the
// records with block histograms in shared memory, one scan in between -- and
// then one block per group holds the cursors of that row's tiles for that bin
// (tiles_x words) and takes every slot with a shared-memory atomic.
constexpr int kGroupThreads = 1024;
constexpr int kMaxGroupKeys = 12288;  // (tile row, bin) keys in 48 KB of shared memory
// reserved entries per tile from which the grouped scatter is used: measured
// slower at ~3k (1M Gaussians, 1080p: bin stage 0.228 vs 0.210 ms), faster at
// ~19k (3M, 1080p: 0.60 vs 0.83 ms) and ~43k (6M, 4K: 3.74 vs 7.6 ms)
constexpr int64_t kGroupedMinPerTile = 8192;

__host__ __device__ inline int group_slices(int num_sms) { return 2 * num_sms; }

// the record slice [r0, r1) of slice c out of C
__device__ __forceinline__ void record_slice(int64_t R, int C, int c, int64_t* r0, int64_t* r1)
{
    *r0 = R * c / C;
    *r1 = R * (c + 1) / C;
}

// key of a row record: (tile row, bin)
__device__ __forceinline__ int group_key(uint32_t ya, int K) { return (int)(ya & 0xfffu) * K + (int)(ya >> 24); }

// pass 1: H[key * C + c] = non-empty records of slice c with that key
__global__ void __launch_bounds__(kGroupThreads)
k_group_count(const uint32_t* __restrict__ rs_ya, const uint32_t* __restrict__ rs_w, const int32_t* __restrict__ roff,
              int64_t n, int K, int nkeys, const int64_t* __restrict__ m_dev, int64_t m_cap, int32_t* __restrict__ H,
              const ScatterPass sp, int tiles_x)
{
    grid_dependency_sync();
    extern __shared__ int32_t s_h[];
    const int C = gridDim.x, c = blockIdx.x;
    for (int i = threadIdx.x; i < nkeys; i += blockDim.x) s_h[i] = 0;
    __syncthreads();
    if (*m_dev <= m_cap) {
        int64_t r0, r1;
        record_slice(roff[n], C, c, &r0, &r1);
        for (int64_t k = r0 + threadIdx.x; k < r1; k += blockDim.x) {
            uint32_t w = rs_w[k], ya = rs_ya[k];
            sp.trim(ya, w, tiles_x);
            if (w != 0u) atomicAdd(&s_h[group_key(ya, K)], 1);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nkeys; i += blockDim.x) H[(int64_t)i * C + c] = s_h[i];
}

// pass 2: list[Hs[key * C + c] + rank] = the record {gid, row word, width,
// depth bits} (any order within a key), so the scatter reads its group
// contiguously
__global__ void __launch_bounds__(kGroupThreads)
k_group_write(const uint32_t* __restrict__ rs_g, const uint32_t* __restrict__ rs_ya,
              const uint32_t* __restrict__ rs_w, const uint32_t* __restrict__ rs_z, const int32_t* __restrict__ roff,
              int64_t n, int K, int nkeys, const int64_t* __restrict__ m_dev, int64_t m_cap,
              const int32_t* __restrict__ Hs, uint4* __restrict__ list, const ScatterPass sp, int tiles_x)
{
    grid_dependency_sync();
    extern __shared__ int32_t s_h[];  // [nkeys] next slot, from the slice's base
    const int C = gridDim.x, c = blockIdx.x;
    if (*m_dev > m_cap) return;
    for (int i = threadIdx.x; i < nkeys; i += blockDim.x) s_h[i] = Hs[(int64_t)i * C + c];
    __syncthreads();
    int64_t r0, r1;
    record_slice(roff[n], C, c, &r0, &r1);
    for (int64_t k = r0 + threadIdx.x; k < r1; k += blockDim.x) {
        uint32_t w = rs_w[k], ya = rs_ya[k];
        sp.trim(ya, w, tiles_x);
        if (w == 0u) continue;
        list[atomicAdd(&s_h[group_key(ya, K)], 1)] = make_uint4(rs_g[k], ya, w, rs_z[k]);
    }
}

// one block per (tile row, bin): that bin's cursor of every tile of the row
// (1024 threads: the groups' sizes vary widely, and the largest bound the
// kernel's tail); a thread takes a record and walks its span of tiles
constexpr int kScatterGroupThreads = 1024;

__global__ void __launch_bounds__(kScatterGroupThreads)
k_scatter_groups(const uint4* __restrict__ list, const int32_t* __restrict__ Hs, int C,
                 const int32_t* __restrict__ offsets, int tiles_x, int K, const int64_t* __restrict__ m_dev,
                 int64_t m_cap, uint64_t* __restrict__ words, const ScatterPass sp,
                 const int32_t* __restrict__ flagged)
{
    grid_dependency_sync();
    extern __shared__ int32_t s_cur[];  // [tiles_x]
    const int key = blockIdx.x;
    if (*m_dev > m_cap) return;
    if (sp.pass == 2 && flagged[0] == 0) return;  // no tile to complete
    const int ty = key / K, b = key - ty * K;
    const int32_t L0 = Hs[(int64_t)key * C], L1 = Hs[(int64_t)(key + 1) * C];
    if (L1 <= L0) return;
    int any = 0;
    for (int x = threadIdx.x; x < tiles_x; x += blockDim.x) {
        const int64_t t = (int64_t)ty * tiles_x + x;
        s_cur[x] = offsets[t * K + b];
        any |= sp.keep(t, b) ? 1 : 0;
    }
    // a planned pass skips the groups no tile of the row takes in this pass
    if (!__syncthreads_or(any)) return;
    for (int32_t i = L0 + (int32_t)threadIdx.x; i < L1; i += (int32_t)blockDim.x) {
        const uint4 rec = list[i];
        const uint64_t word = ((uint64_t)rec.w << 32) | rec.x;
        const int a = (int)((rec.y >> 12) & 0xfffu);
        for (int j = 0; j < (int)rec.z; ++j) {
            if (!sp.keep((int64_t)ty * tiles_x + a + j, b)) continue;
            const int32_t slot = atomicAdd(&s_cur[a + j], 1);
            words[slot] = word;
        }
    }
}

// ------------------------------------------------------------------ scatter
// Without the tile cull: straight from the rects with the warp-cooperative
// expansion, four entries per lane in flight so the returning atomics overlap.
__global__ void __launch_bounds__(256)
k_bin_scatter_rects(const uint2* __restrict__ rect, const float4* __restrict__ c_o_z,
                    const int32_t* __restrict__ goff, const uint8_t* __restrict__ gbin, int64_t n, int tiles_x,
                    int K, const int64_t* __restrict__ m_dev, int64_t m_cap, const int32_t* __restrict__ off,
                    int32_t* __restrict__ cur, uint64_t* __restrict__ words)
{
    if (*m_dev > m_cap) return;  // capacity error raised by the caller's check
    const int64_t g0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32;
    if (g0 >= n) return;
    const WarpExpand wx(rect, c_o_z, goff, n, g0);
    const int lane = threadIdx.x & 31;
    const int64_t gl = g0 + lane;
    const uint32_t mybin = (gl < n && ((wx.r1 & 0xffffu) > (wx.r0 & 0xffffu))) ? gbin[gl] : 0u;
    for (int32_t e0 = wx.base; e0 < wx.end; e0 += 128) {
        uint32_t g[4], t[4], z[4], b[4];
        int32_t p[4];
        bool live[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            wx.entry(e0 + 32 * u + lane, tiles_x, &g[u], &t[u], &z[u]);
            b[u] = __shfl_sync(0xffffffffu, mybin, (int)(g[u] - (uint32_t)g0) & 31);
            live[u] = e0 + 32 * u + lane < wx.end;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (live[u]) {
                const int64_t q = (int64_t)t[u] * K + b[u];
                p[u] = atomicAdd(&cur[q], 1);
            }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (live[u]) words[p[u]] = ((uint64_t)z[u] << 32) | g[u];
    }
}

// Count of segment q = t*K + b from the prefixed layers (tile-major order).
// count[t, b] from the layer-major row prefix D [b][y][x] into C [t][b]
// (t = y * tiles_x + x): 32 x 32 (x, b) blocks through shared memory, so both
// the reads (along x) and the writes (along b) are coalesced.
__global__ void __launch_bounds__(256)
k_transpose_counts(const int32_t* __restrict__ D, int tiles_x, int tiles_y, int K, int64_t layer,
                   int32_t* __restrict__ C)
{
    grid_dependency_sync();
    __shared__ int32_t s[32][33];
    const int y = blockIdx.z;
    const int x0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
    const int W1 = tiles_x + 1;
    const int lx = threadIdx.x & 31;
    for (int r = threadIdx.x >> 5; r < 32; r += blockDim.x >> 5) {
        const int b = b0 + r, x = x0 + lx;
        s[r][lx] = (b < K && x < tiles_x) ? D[b * layer + (int64_t)y * W1 + x] : 0;
    }
    __syncthreads();
    for (int r = threadIdx.x >> 5; r < 32; r += blockDim.x >> 5) {
        const int x = x0 + r, b = b0 + lx;
        if (x < tiles_x && b < K) C[((int64_t)y * tiles_x + x) * K + b] = s[lx][r];
    }
}

// The (tile, bin) segment offsets from the layered row differences
// D[b][ty][x] in one pass, tile-major (t = ty tiles_x + x, bins inside): one
// block per tile row (taken in ticket order) forms its counts by a prefix
// along x per bin, scans them in tile-major order, finds the rows before it
// by decoupled look-back over the rows' published totals (bounded waits),
// and writes offsets and, when given, the scatter cursors.  Over capacity
// (or past INT32_MAX) every offset is written 0 and GS_ERR_CAPACITY raised,
// so nothing downstream reads out of bounds.  Replaces a per-layer prefix,
// a transposition, a device-wide scan and the over-capacity pass.
constexpr int kOffThreads = 1024;
constexpr size_t kOffMaxSmem = 160 * 1024;
__host__ __device__ inline size_t bin_offsets_smem(int tiles_x, int K) { return (size_t)tiles_x * (K + 1) * 4; }

__global__ void __launch_bounds__(kOffThreads)
k_bin_offsets(const int32_t* __restrict__ D, int tiles_x, int tiles_y, int K, int64_t layer,
              const int64_t* __restrict__ m_dev, int64_t m_cap, uint64_t* flags, unsigned int* ticket,
              int32_t* __restrict__ off, int32_t* __restrict__ cur, int* err)
{
    grid_dependency_sync();
    extern __shared__ int32_t s_c[];  // [tiles_x][K + 1]: counts, then exclusive offsets in the row
    __shared__ int32_t s_warp[kOffThreads / 32];
    __shared__ int64_t s_pre;
    __shared__ int s_row;
    if (threadIdx.x == 0) {
        const unsigned t = atomicAdd(ticket, 1u);
        s_row = (int)t;
        if ((int)t == tiles_y - 1) *ticket = 0u;  // every ticket is out: ready for the next scan
    }
    __syncthreads();
    const int ty = s_row;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int KP = K + 1;
    // counts: per bin, the inclusive prefix of the row's differences
    for (int b = warp; b < K; b += kOffThreads / 32) {
        const int32_t* row = D + (int64_t)b * layer + (int64_t)ty * (tiles_x + 1);
        int32_t carry = 0;
        for (int x0 = 0; x0 < tiles_x; x0 += 32) {
            const int x = x0 + lane;
            int32_t v = x < tiles_x ? row[x] : 0;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int32_t u = __shfl_up_sync(0xffffffffu, v, d);
                if (lane >= d) v += u;
            }
            if (x < tiles_x) s_c[x * KP + b] = carry + v;
            carry += __shfl_sync(0xffffffffu, v, 31);
        }
    }
    __syncthreads();
    // the row's exclusive scan in tile-major order: a run of items a thread
    const int items = tiles_x * K;
    const int per = (items + kOffThreads - 1) / kOffThreads;
    const int j0 = threadIdx.x * per;
    int32_t run = 0;
    {
        int x = j0 / K, b = j0 - (j0 / K) * K;
        for (int k = 0; k < per && j0 + k < items; ++k) {
            run += s_c[x * KP + b];
            if (++b == K) { b = 0; ++x; }
        }
    }
    int32_t incl = run;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int32_t u = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += u;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        constexpr int NW = kOffThreads / 32;
        int32_t w = lane < NW ? s_warp[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t u = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += u;
        }
        if (lane < NW) s_warp[lane] = w;  // inclusive warp totals
    }
    __syncthreads();
    const int64_t total = s_warp[kOffThreads / 32 - 1];
    int32_t e = (warp > 0 ? s_warp[warp - 1] : 0) + incl - run;
    {
        int x = j0 / K, b = j0 - (j0 / K) * K;
        for (int k = 0; k < per && j0 + k < items; ++k) {
            const int32_t c = s_c[x * KP + b];
            s_c[x * KP + b] = e;
            e += c;
            if (++b == K) { b = 0; ++x; }
        }
    }
    // the rows before: publish this row's total, look back over theirs
    volatile uint64_t* vf = flags;
    if (threadIdx.x == 0) vf[ty] = (ty == 0 ? kScanFlagP : kScanFlagA) | (uint64_t)total;
    if (warp == 0) {
        const int64_t pre = ty > 0 ? scan_lookback(vf, ty, err) : 0;
        if (lane == 0) {
            if (ty > 0) vf[ty] = kScanFlagP | (uint64_t)(pre + total);
            s_pre = pre;
        }
    }
    __syncthreads();
    const int64_t pre = s_pre;
    const bool over = *m_dev > m_cap || pre + total > (int64_t)INT32_MAX - 1;
    if (over && threadIdx.x == 0) raise_error(err, GS_ERR_CAPACITY);
    const int64_t base = (int64_t)ty * items;
    for (int j = threadIdx.x; j < items; j += kOffThreads) {
        const int x = j / K, b = j - x * K;
        const int32_t v = over ? 0 : (int32_t)(pre + s_c[x * KP + b]);
        off[base + j] = v;
        if (cur) cur[base + j] = v;
    }
    if (ty == tiles_y - 1 && threadIdx.x == 0) off[(int64_t)tiles_y * items] = over ? 0 : (int32_t)(pre + total);
}

struct LoadPlainCount {
    const int32_t* C;
    __device__ int64_t operator()(int64_t q) const { return C[q]; }
};

struct LoadLayerCount {
    const int32_t* D;
    int K, tiles_x, W1;
    int64_t layer;
    __device__ int64_t operator()(int64_t q) const
    {
        const int64_t t = q / K;
        const int b = (int)(q - t * K);
        const int y = (int)(t / tiles_x), x = (int)(t - (int64_t)y * tiles_x);
        return D[b * layer + (int64_t)y * W1 + x];
    }
};

__global__ void k_zero_if_over(const int64_t* __restrict__ m_dev, int64_t m_cap, int32_t* __restrict__ off, int64_t nq,
                               int* err)
{
    grid_dependency_sync();
    if (*m_dev <= m_cap) return;  // over capacity: empty stream, nothing out of bounds downstream
    if (blockIdx.x == 0 && threadIdx.x == 0) raise_error(err, GS_ERR_CAPACITY);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x)
        off[q] = 0;
}

// The grouped scatter pays off once the frame is deep: decided on the host
// from the reserved entry capacity per tile (the entry count itself lives on
// the device).
static bool grouped_scatter(int64_t m_cap, int64_t T)
{
    return T > 0 && m_cap / T >= kGroupedMinPerTile;
}

struct ExactScratch {
    int32_t* D;      // K layers of (tiles_y + 1) x (tiles_x + 1) difference counts
    int32_t* cur;    // T*K scatter cursors
    uint8_t* gbin;   // n per-Gaussian bins
    int32_t* roff;   // n + 1 row-record offsets
    uint32_t *rs_g, *rs_ya, *rs_w, *rs_z;  // row records (<= m_cap)
    int64_t* total;  // scratch count
    int32_t *H, *Hs; // per ((tile row, bin) key, slice) record counts and their exclusive scan
    uint4* list;     // the records grouped by key (<= m_cap)
};

static size_t exact_scratch(gs_ctx* ctx, int64_t n, int64_t m_cap, int32_t tiles_x, int32_t tiles_y, int K,
                            ExactScratch* v)
{
    const size_t layer = (size_t)(tiles_x + 1) * (tiles_y + 1);
    const size_t T = (size_t)tiles_x * tiles_y;
    const size_t mc = (size_t)(m_cap > 0 ? m_cap : 1), nn = (size_t)(n > 0 ? n : 1);
    const size_t nh = (size_t)tiles_y * K * group_slices(ctx->num_sms);
    const size_t sizes[] = {layer * K * 4, T * K * 4, nn, (nn + 1) * 4, mc * 4, mc * 4, mc * 4, mc * 4, 8,
                            nh * 4, (nh + 1) * 4, grouped_scatter(m_cap, (int64_t)T) ? mc * 16 : 16};
    size_t total = 0;
    for (size_t s : sizes) total += align256(s);
    if (v) {
        char* b = (char*)ctx->d_tiles;
        void** dst[] = {(void**)&v->D, (void**)&v->cur, (void**)&v->gbin, (void**)&v->roff, (void**)&v->rs_g,
                        (void**)&v->rs_ya, (void**)&v->rs_w, (void**)&v->rs_z, (void**)&v->total,
                        (void**)&v->H, (void**)&v->Hs, (void**)&v->list};
        for (int k = 0; k < 12; ++k) {
            *dst[k] = b;
            b += align256(sizes[k]);
        }
    }
    return total;
}

// items of the grouped scatter's count scan (for reserving the scan's sums)
int64_t group_scan_items(gs_ctx* ctx, int32_t tiles_y, int K)
{
    return (int64_t)tiles_y * K * group_slices(ctx->num_sms);
}

int exact_bins_reserve(gs_ctx* ctx, int64_t n, int64_t m_cap, int32_t tiles_x, int32_t tiles_y, int K)
{
    void* p = ctx->d_tiles;
    int r = ensure(&p, &ctx->tiles_cap, exact_scratch(ctx, n, m_cap, tiles_x, tiles_y, K, nullptr));
    ctx->d_tiles = (int32_t*)p;
    return r;
}

// Whether a first-pass scatter takes the grouped path (records grouped by
// (tile row, bin), cursors in shared memory) rather than per-entry global
// cursors.
static bool grouped_path(int64_t m_cap, int32_t tiles_x, int32_t tiles_y, int K)
{
    return grouped_scatter(m_cap, (int64_t)tiles_x * tiles_y) && tiles_y * K <= kMaxGroupKeys;
}

// The record scatter of the tile-cull path, for one pass (grouped by (tile
// row, bin) on deep frames, else per-entry global cursors, `cur` being
// initialised from the offsets before the first pass -- unless the offsets'
// scan already wrote them there, cur_ready).
static int exact_scatter(gs_ctx* ctx, const ExactScratch& v, int64_t n, int32_t tiles_x, int32_t tiles_y, int K,
                         int64_t m_cap, const int64_t* m_dev, uint64_t* words, const int32_t* offsets,
                         const ScatterPass& sp, cudaStream_t st, bool cur_ready = false)
{
    const int64_t T = (int64_t)tiles_x * tiles_y;
    const int nkeys = tiles_y * K;
    const unsigned g_sm = (unsigned)ctx->num_sms * 8;
    const int32_t* flagged = sp.pass ? ctx->d_plist : nullptr;
    if (n <= 0) return GS_OK;
    if (sp.pass != 2 && grouped_path(m_cap, tiles_x, tiles_y, K)) {
        // records grouped by (tile row, bin), then cursors in shared memory
        // (a planned first pass groups only the records it keeps)
        const int C = group_slices(ctx->num_sms);
        const size_t hsm = (size_t)nkeys * 4;
        GS_CUDA_TRY(launch_k(ctx, k_group_count, (unsigned)C, kGroupThreads, hsm, st, v.rs_ya, v.rs_w, v.roff, n, K, nkeys, m_dev, m_cap,
                                                                v.H, sp, tiles_x));
        ctx->launches += 1;
        int r;
        if ((r = scan_impl(ctx, LoadI32{v.H}, (int64_t)nkeys * C, v.Hs, nullptr, st)) != GS_OK) return r;
        GS_CUDA_TRY(launch_k(ctx, k_group_write, (unsigned)C, kGroupThreads, hsm, st, v.rs_g, v.rs_ya, v.rs_w, v.rs_z, v.roff, n, K, nkeys,
                                                                m_dev, m_cap, v.Hs, v.list, sp, tiles_x));
        GS_CUDA_TRY(launch_k(ctx, k_scatter_groups, (unsigned)nkeys, kScatterGroupThreads, (size_t)tiles_x * 4, st, 
            v.list, v.Hs, C, offsets, tiles_x, K, m_dev, m_cap, words, sp, flagged));
        ctx->launches += 2;
    } else {
        // per-entry cursors in global memory: all of them from the offsets
        // before a first pass, those of the flagged tiles before the
        // completing pass (few entries: no grouping)
        if (sp.pass != 2) {
            if (!cur_ready)
                GS_CUDA_TRY(cudaMemcpyAsync(v.cur, offsets, (size_t)T * K * 4, cudaMemcpyDeviceToDevice, st));
        } else {
            GS_CUDA_TRY(launch_k(ctx, k_flagged_cursors, (unsigned)ctx->num_sms * 2, 256, 0, st, flagged, offsets, K, v.cur));
            ctx->launches += 1;
        }
        GS_CUDA_TRY(launch_k(ctx, k_bin_scatter_rows, g_sm * 2, 256, 0, st, v.rs_g, v.rs_ya, v.rs_w, v.rs_z, v.roff, n, tiles_x, K, m_dev,
                                                     m_cap, v.cur, words, sp, flagged));
        ctx->launches += 1;
    }
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

// The regions a frame of the tile-cull EXACT path needs zeroed, so that no
// memset sits between its kernels: the frame's scan-flag arena (the row-count
// scan, the offsets scan and, on deep frames, the grouped scatter's count
// scan), the bin stage's difference counts, the repair's long-segment
// counter.  The projection (*fz) clears the row-count scan's flags, the
// depth-range sampling (ctx->late_*) the rest.  Reserves the scratch they
// live in.
int exact_frame_zero(gs_ctx* ctx, int64_t n, const gs_camera* cam, int64_t m_cap, FrameZero* fz)
{
    const int tile = ctx->cfg.tile_size, K = ctx->cfg.K;
    const int32_t tiles_x = (cam->width + tile - 1) / tile, tiles_y = (cam->height + tile - 1) / tile;
    const int64_t T = (int64_t)tiles_x * tiles_y, nseg = T * K;
    int r;
    if ((r = exact_bins_reserve(ctx, n, m_cap, tiles_x, tiles_y, K)) != GS_OK) return r;
    if ((r = bins_reserve(ctx, 1, nseg)) != GS_OK) return r;
    ExactScratch v;
    exact_scratch(ctx, n, m_cap, tiles_x, tiles_y, K, &v);
    auto blocks = [](int64_t items) { return items > 0 ? (items + kScanTile - 1) / kScanTile : 1; };
    int64_t words = 2 * blocks(n) + (blocks(nseg) > tiles_y ? blocks(nseg) : tiles_y);
    if (grouped_path(m_cap, tiles_x, tiles_y, K))
        words += blocks((int64_t)tiles_y * K * group_slices(ctx->num_sms));
    if ((size_t)(words + 2) * sizeof(uint64_t) > ctx->scan_bytes) {
        if (ctx->capturing) return GS_OK;  // no allocation inside a capture: the scans clear their own flags
        if ((r = ensure(&ctx->d_scan, &ctx->scan_bytes, (size_t)(words + 2) * sizeof(uint64_t))) != GS_OK) return r;
    }
    const int64_t w2 = 2 * blocks(n);  // the row-count scan's flags: cleared by the projection
    fz->p[0] = static_cast<int32_t*>(ctx->d_scan);
    fz->n[0] = 2 * w2;
    ctx->late_p[0] = v.D;
    ctx->late_n[0] = (int64_t)(tiles_x + 1) * (tiles_y + 1) * K;
    ctx->late_p[1] = static_cast<int32_t*>(ctx->d_scan) + 2 * w2;
    ctx->late_n[1] = 2 * (words - w2);
    ctx->late_p[2] = ctx->d_tail;
    ctx->late_n[2] = 1;
    ctx->scan_arena = words;
    ctx->scan_used = 0;
    ctx->scan_arena_bytes = ctx->scan_bytes;
    ctx->zeroed_D = v.D;
    ctx->zeroed_D_bytes = ctx->tiles_cap;
    ctx->zeroed_tail = ctx->d_tail;
    ctx->zeroed_tail_bytes = ctx->tail_cap;
    return GS_OK;
}

// The one-pass offsets kernel takes up to kOffMaxSmem of dynamic shared
// memory (tile rows of up to kOffMaxSmem / 4 / (K + 1) tiles): set once per
// context, on its device.
int bin_offsets_prepare()
{
    GS_CUDA_TRY(cudaFuncSetAttribute(k_bin_offsets, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOffMaxSmem));
    return GS_OK;
}

int exact_scatter_rest(gs_ctx* ctx, int64_t n, const gs_camera* cam, int64_t m_cap, const int64_t* m_dev,
                       uint64_t* words, const int32_t* offsets, cudaStream_t st)
{
    const int tile = ctx->cfg.tile_size, K = ctx->cfg.K;
    const int32_t tiles_x = (cam->width + tile - 1) / tile, tiles_y = (cam->height + tile - 1) / tile;
    ExactScratch v;
    exact_scratch(ctx, n, m_cap, tiles_x, tiles_y, K, &v);
    v.roff = ctx->exact_roff;  // the first pass's row records (the fused scan's offsets on the render path)
    ScatterPass sp;
    sp.plan = ctx->d_plan;
    sp.T = tiles_x * tiles_y;
    sp.pass = 2;
    return exact_scatter(ctx, v, n, tiles_x, tiles_y, K, m_cap, m_dev, words, offsets, sp, st);
}

int exact_bins(gs_ctx* ctx, const ProjView& pv, int64_t n, const gs_camera* cam, bool goff_ready, int64_t m_cap,
               const int64_t* m_dev, uint64_t* words, int32_t* offsets, cudaStream_t st, bool rows_ready,
               bool planned)
{
    const int tile = ctx->cfg.tile_size, K = ctx->cfg.K;
    const int32_t tiles_x = (cam->width + tile - 1) / tile, tiles_y = (cam->height + tile - 1) / tile;
    const int64_t T = (int64_t)tiles_x * tiles_y, nseg = T * K;
    int r;
    if ((r = exact_bins_reserve(ctx, n, m_cap, tiles_x, tiles_y, K)) != GS_OK) return r;
    ExactScratch v;
    exact_scratch(ctx, n, m_cap, tiles_x, tiles_y, K, &v);
    const size_t layer = (size_t)(tiles_x + 1) * (tiles_y + 1);
    if (tiles_x > 4096 || tiles_y > 4096) return GS_ERR_INVALID_ARG;  // row-record packing
    if (!(ctx->zeroed_D == v.D && ctx->zeroed_D_bytes == ctx->tiles_cap))
        GS_CUDA_TRY(cudaMemsetAsync(v.D, 0, layer * K * 4, st));
    ctx->zeroed_D = nullptr;  // zeroed by the frame's first kernel once, for this call
    const unsigned g_sm = (unsigned)ctx->num_sms * 8;
    if (ctx->cfg.tile_cull) {
        // rows of every rect, each row's culled span, per-row difference counts
        const int64_t rlayer = (int64_t)tiles_y * (tiles_x + 1);
        if (rows_ready && goff_ready) {
            v.roff = rows_offsets(ctx, n);
            v.total = rows_total(ctx, n);
        } else if ((r = scan_impl(ctx, LoadRectRows{pv.rect}, n, v.roff, v.total, st)) != GS_OK) {
            return r;
        }
        CullArgs ca{pv.xy_ab, pv.c_o_z, pv.rgb, tile};
        const int64_t warps = (n + 31) / 32;
        if (warps > 0)
            GS_CUDA_TRY(launch_k(ctx, k_row_spans, (unsigned)((warps + 7) / 8), 256, 0, st, pv.rect, n, v.roff, ca, tiles_x, ctx->d_bp, K,
                                                                     m_dev, m_cap, v.D, rlayer, v.gbin, v.rs_g,
                                                                     v.rs_ya, v.rs_w, v.rs_z));
        ctx->launches += 1;
        // the per-entry scatter starts its cursors at the offsets
        const bool cur_ready = n > 0 && !grouped_path(m_cap, tiles_x, tiles_y, K);
        const size_t osm = bin_offsets_smem(tiles_x, K);
        if (osm <= kOffMaxSmem) {
            // one pass: counts, tile-major scan, look-back over tile rows
            uint64_t* flags;
            if ((r = scan_flags(ctx, tiles_y, &flags, st)) != GS_OK) return r;
            GS_CUDA_TRY(launch_k(ctx, k_bin_offsets, (unsigned)tiles_y, kOffThreads, osm, st, v.D, tiles_x, tiles_y,
                                 K, rlayer, m_dev, m_cap, flags, ctx->d_scan_done, offsets,
                                 cur_ready ? v.cur : nullptr, ctx->d_err));
            ctx->launches += 1;
        } else {
            // rows too wide for one block's shared memory: per-layer prefix,
            // the counts tile-major (the cursor array serves as the staging
            // copy; the scan rewrites it with the offsets when the per-entry
            // scatter will start its cursors there), a coalesced scan
            GS_CUDA_TRY(launch_k(ctx, k_layer_rows_prefix, (unsigned)K, 1024, 0, st, v.D, tiles_x, tiles_y, rlayer));
            GS_CUDA_TRY(launch_k(ctx, k_transpose_counts,
                                 dim3((unsigned)((tiles_x + 31) / 32), (unsigned)((K + 31) / 32), (unsigned)tiles_y),
                                 256, 0, st, v.D, tiles_x, tiles_y, K, rlayer, v.cur));
            ctx->launches += 2;
            if ((r = scan_impl(ctx, LoadPlainCount{v.cur}, nseg, offsets, nullptr, st, cur_ready ? v.cur : nullptr)) !=
                GS_OK)
                return r;
            GS_CUDA_TRY(launch_k(ctx, k_zero_if_over, g_sm, 256, 0, st, m_dev, m_cap, offsets, nseg + 1, ctx->d_err));
            ctx->launches += 1;
        }
        ScatterPass sp;
        if (planned) {
            ctx->exact_roff = v.roff;
            // the bin planner sets each tile's first-pass bins from the counts
            if ((r = plan_frame(ctx, offsets, K, (int32_t)T, ctx->d_plan, nullptr, st)) != GS_OK) return r;
            sp.plan = ctx->d_plan;
            sp.T = (int32_t)T;
            sp.pass = 1;
        }
        if ((r = exact_scatter(ctx, v, n, tiles_x, tiles_y, K, m_cap, m_dev, words, offsets, sp, st, cur_ready)) !=
            GS_OK)
            return r;
    } else {
        // whole rects per bin layer: four atomics per Gaussian, 2D prefix sums
        if (!goff_ready && (r = count_scan(ctx, pv, n, v.total, st)) != GS_OK) return r;
        if (n > 0) k_bin_diff<<<g_sm, 256, 0, st>>>(pv.rect, pv.c_o_z, n, tiles_x, tiles_y, ctx->d_bp, K, v.D, v.gbin);
        k_layer_prefix<<<(unsigned)K, 1024, 0, st>>>(v.D, tiles_x, tiles_y);
        ctx->launches += 2;
        if ((r = scan_impl(ctx, LoadLayerCount{v.D, K, tiles_x, tiles_x + 1, (int64_t)layer}, nseg, offsets, nullptr,
                           st)) != GS_OK)
            return r;
        GS_CUDA_TRY(launch_k(ctx, k_zero_if_over, g_sm, 256, 0, st, m_dev, m_cap, offsets, nseg + 1, ctx->d_err));
        GS_CUDA_TRY(cudaMemcpyAsync(v.cur, offsets, (size_t)nseg * 4, cudaMemcpyDeviceToDevice, st));
        const int64_t warps = (n + 31) / 32;
        if (warps > 0)
            k_bin_scatter_rects<<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(pv.rect, pv.c_o_z, ctx->d_goff, v.gbin, n,
                                                                             tiles_x, K, m_dev, m_cap, offsets, v.cur,
                                                                             words);
        ctx->launches += 2;
    }
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

}  // namespace gs
