// planner.cu -- K23: the learned bin planner.  The paper uses one bin count
// and spacing for every tile (Sec. 5.3 ablates K for the whole frame; Sec. 7
// leaves settings that follow the depth distribution or the resolution to
// future work).  Here a small MLP picks, per tile, how many of the tile's K
// depth bins (the monotone split depths of EXACT mode) the frame builds in
// its first pass: only the entries of those bins are scattered and
// composited.  A tile whose pixels have not all terminated when its bins run
// out, and which has entries in later bins, is completed by a second pass
// (the rest of its bins scattered, the tile composited again from its
// front).  So every plan gives the same image; a good plan skips the
// scattering of entries behind the point where a tile saturates.
//
// Features per tile, from its culled span and the K bin counts n_b:
//   f0 log1p(n)        n = entries of the tile
//   f1 log1p(max n_b)
//   f2 nonempty / K
//   f3 first nonempty bin / K      (1 when the tile is empty)
//   f4 last nonempty bin / K       (0 when empty)
//   f5 log1p(n_first)              count of the first nonempty bin
//   f6 log1p(front)                entries in the K/8 bins from the first nonempty one
//   f7 log1p(n / nonempty)         mean occupancy of a nonempty bin
// Network: 8 -> 64 -> 64 -> 6, ReLU, float32; parameters packed as
//   W1[64][8] b1[64] W2[64][64] b2[64] W3[6][64] b3[6]  (5126 floats).
// Class c < 5 keeps the fewest bins from the tile's front holding at least
// 64 << c entries; class 5 keeps all K.  The decision is the smallest class
// whose cumulative softmax probability reaches the configured quantile q
// (a calibrated network then needs the second pass for about 1 - q of the
// tiles).  Training runs on the GPU with the kernels below (forward, softmax
// cross entropy, backward, Adam) on labels the raster itself logs: each
// tile's bins needed (the counting raster, gs_rasterize_fwd_plan).
#include "internal.cuh"

namespace gs {

constexpr int kF = GS_PLAN_FEATURES, kH = GS_PLAN_HIDDEN, kC = GS_PLAN_CLASSES;
constexpr int oW1 = 0, oB1 = oW1 + kH * kF, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH, oB3 = oW3 + kC * kH;
static_assert(oB3 + kC == GS_PLAN_PARAMS, "parameter layout");
static_assert(kC == kPlanClasses, "plan classes");

// The features of tile t, in every lane of the calling warp (K <= GS_MAX_K,
// so at most 4 bins per lane).  All the tile's offsets are loaded in one
// round: a lane holds o[b] and o[b + 1] of its bins b = lane + 32 j.
__device__ __forceinline__ void warp_tile_features(const int32_t* __restrict__ off, int K, int t, float (&f)[kF])
{
    const int lane = threadIdx.x & 31;
    const int32_t* o = off + (int64_t)t * K;
    int lo[4], hi[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int b = lane + 32 * j;
        lo[j] = b < K ? __ldg(o + b) : 0;
        hi[j] = b < K ? __ldg(o + b + 1) : 0;
    }
    const int o0 = __ldg(o), oK = __ldg(o + K);
    int cnt[4];
    int mx = 0, ne = 0, first = K, last = -1;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int b = lane + 32 * j;
        cnt[j] = hi[j] - lo[j];
        mx = max(mx, cnt[j]);
        if (cnt[j] > 0) {
            ++ne;
            first = min(first, b);
            last = max(last, b);
        }
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, s));
        ne += __shfl_xor_sync(0xffffffffu, ne, s);
        first = min(first, __shfl_xor_sync(0xffffffffu, first, s));
        last = max(last, __shfl_xor_sync(0xffffffffu, last, s));
    }
    const int span = K / 8 > 0 ? K / 8 : 1;
    int front = 0, nfirst = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int b = lane + 32 * j;
        if (b >= first && b < first + span) front += cnt[j];
        if (b == first) nfirst = cnt[j];
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        front += __shfl_xor_sync(0xffffffffu, front, s);
        nfirst += __shfl_xor_sync(0xffffffffu, nfirst, s);
    }
    const int n = oK - o0;
    const float fk = (float)K;
    f[0] = log1pf((float)n);
    f[1] = log1pf((float)mx);
    f[2] = (float)ne / fk;
    f[3] = ne > 0 ? (float)first / fk : 1.0f;
    f[4] = ne > 0 ? (float)last / fk : 0.0f;
    f[5] = log1pf((float)nfirst);
    f[6] = log1pf((float)front);
    f[7] = ne > 0 ? log1pf((float)n / (float)ne) : 0.0f;
}

// one warp per tile
__global__ void k_tile_features(const int32_t* __restrict__ off, int K, int T, float* __restrict__ feat)
{
    const int t = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (t >= T) return;
    float f[kF];
    warp_tile_features(off, K, t, f);
    if ((threadIdx.x & 31) < kF) {
        float v = f[0];
#pragma unroll
        for (int i = 1; i < kF; ++i)
            if ((threadIdx.x & 31) == i) v = f[i];
        feat[(int64_t)t * kF + (threadIdx.x & 31)] = v;
    }
}

// Inference parameters in shared memory, laid out so that lane l reads
// consecutive words: W1t[i][j] = W1[j][i], W2t[i][j] = W2[j][i].  The same
// layout is kept in device memory (written once by gs_planner_set_weights),
// so a block stages it with contiguous 16-byte copies.
struct __align__(16) PlanShared {
    float W1t[kF * kH];
    float b1[kH];
    float W2t[kH * kH];
    float b2[kH];
    float W3[kC * kH];
    float b3[kC];
    float pad[2];
};
static_assert(sizeof(PlanShared) % 16 == 0, "16-byte staging");
constexpr int kPlanLayoutFloats = (int)(sizeof(PlanShared) / 4);

// the inference layout of packed parameters P (one block)
__global__ void k_plan_layout(const float* __restrict__ P, PlanShared* __restrict__ s)
{
    for (int k = threadIdx.x; k < kF * kH; k += blockDim.x) {
        const int j = k / kF, i = k % kF;
        s->W1t[i * kH + j] = P[oW1 + k];
    }
    for (int k = threadIdx.x; k < kH * kH; k += blockDim.x) {
        const int j = k / kH, i = k % kH;
        s->W2t[i * kH + j] = P[oW2 + k];
    }
    for (int k = threadIdx.x; k < kH; k += blockDim.x) {
        s->b1[k] = P[oB1 + k];
        s->b2[k] = P[oB2 + k];
    }
    for (int k = threadIdx.x; k < kC * kH; k += blockDim.x) s->W3[k] = P[oW3 + k];
    for (int k = threadIdx.x; k < kC; k += blockDim.x) s->b3[k] = P[oB3 + k];
    if (threadIdx.x < 2) s->pad[threadIdx.x] = 0.0f;
}

__device__ __forceinline__ void stage_plan_params(const PlanShared* __restrict__ L, PlanShared& s)
{
    const float4* src = reinterpret_cast<const float4*>(L);
    float4* dst = reinterpret_cast<float4*>(&s);
    constexpr int n4 = kPlanLayoutFloats / 4;
#pragma unroll 6
    for (int k = threadIdx.x; k < n4; k += blockDim.x) dst[k] = __ldg(src + k);
    __syncthreads();
}

// The planner network for one tile by one warp (features in every lane):
// lane l holds hidden units l and l + 32 of both layers; the logits are warp
// sums.  Returns, in every lane, the smallest class whose cumulative softmax
// probability reaches q.
__device__ __forceinline__ int warp_plan(const PlanShared& P, const float (&f)[kF], float q)
{
    const int lane = threadIdx.x & 31;
    float h1[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int j = lane + 32 * u;
        float a = P.b1[j];
#pragma unroll
        for (int i = 0; i < kF; ++i) a = fmaf(P.W1t[i * kH + j], f[i], a);
        h1[u] = fmaxf(a, 0.0f);
    }
    float a0 = P.b2[lane], a1 = P.b2[lane + 32];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll 8
        for (int i0 = 0; i0 < 32; ++i0) {
            const int i = 32 * u + i0;
            const float hi = __shfl_sync(0xffffffffu, h1[u], i0);
            a0 = fmaf(P.W2t[i * kH + lane], hi, a0);
            a1 = fmaf(P.W2t[i * kH + lane + 32], hi, a1);
        }
    const float h20 = fmaxf(a0, 0.0f), h21 = fmaxf(a1, 0.0f);
    float z[kC];
#pragma unroll
    for (int c = 0; c < kC; ++c) {
        float v = fmaf(P.W3[c * kH + lane], h20, P.W3[c * kH + lane + 32] * h21);
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
        z[c] = v + P.b3[c];
    }
    float m = z[0];
#pragma unroll
    for (int c = 1; c < kC; ++c) m = fmaxf(m, z[c]);
    float e[kC], sum = 0.0f;
#pragma unroll
    for (int c = 0; c < kC; ++c) {
        e[c] = expf(z[c] - m);
        sum += e[c];
    }
    int cls = kC - 1;
    float cum = 0.0f;
#pragma unroll
    for (int c = 0; c < kC - 1; ++c) {
        cum += e[c];
        if (cls == kC - 1 && cum >= q * sum) cls = c;
    }
    return cls;
}

// First-pass bins of class c for the tile whose bin offsets start at o (K + 1
// of them), in every lane: the fewest bins from the front holding at least
// plan_entries(c) entries (K if the tile has fewer); K for the last class.
__device__ __forceinline__ int warp_class_bins(const int32_t* __restrict__ o, int K, int c)
{
    if (c >= kC - 1) return K;
    const int need = plan_entries(c);
    const int lane = threadIdx.x & 31;
    const int32_t s0 = o[0];
    for (int j0 = 0; j0 < K; j0 += 32) {
        const int b = j0 + lane;
        const unsigned hit = __ballot_sync(0xffffffffu, b < K && o[b + 1] - s0 >= need);
        if (hit) return j0 + __ffs(hit);
    }
    return K;
}

// Features, class and first-pass bins of every tile in one launch: blocks
// of 8 warps stage the parameters once and loop over tiles, a warp per tile.
// Also clears the frame's completion flags, row flags and list.
__global__ void __launch_bounds__(256, 8) k_plan_fused(const int32_t* __restrict__ off, int K, int T,
                                                    const PlanShared* __restrict__ params, float q,
                                                    uint8_t* __restrict__ plan, uint8_t* __restrict__ classes,
                                                    uint8_t* __restrict__ flag, int32_t* __restrict__ list)
{
    grid_dependency_sync();
    __shared__ PlanShared P;
    stage_plan_params(params, P);
    if (list && blockIdx.x == 0 && threadIdx.x == 0) list[0] = 0;
    const int warps = blockDim.x >> 5;
    for (int t = blockIdx.x * warps + (threadIdx.x >> 5); t < T; t += gridDim.x * warps) {
        float f[kF];
        warp_tile_features(off, K, t, f);
        const int c = warp_plan(P, f, q);
        const int B = warp_class_bins(off + (int64_t)t * K, K, c);
        if ((threadIdx.x & 31) == 0) {
            plan[t] = (uint8_t)B;
            if (classes) classes[t] = (uint8_t)c;
            if (flag) {
                flag[t] = 0;
                flag[T + t] = 0;  // the row flags (tile rows <= T)
            }
        }
    }
}

// hidden activations of one sample (ReLU outputs)
__device__ __forceinline__ void mlp_hidden(const float* __restrict__ P, const float* x, float* h1, float* h2)
{
    for (int j = 0; j < kH; ++j) {
        float a = P[oB1 + j];
#pragma unroll
        for (int i = 0; i < kF; ++i) a = fmaf(P[oW1 + j * kF + i], x[i], a);
        h1[j] = fmaxf(a, 0.0f);
    }
    for (int j = 0; j < kH; ++j) {
        float a = P[oB2 + j];
        for (int i = 0; i < kH; ++i) a = fmaf(P[oW2 + j * kH + i], h1[i], a);
        h2[j] = fmaxf(a, 0.0f);
    }
}

__device__ __forceinline__ void mlp_logits(const float* __restrict__ P, const float* h2, float* z)
{
#pragma unroll
    for (int c = 0; c < kC; ++c) {
        float a = P[oB3 + c];
        for (int i = 0; i < kH; ++i) a = fmaf(P[oW3 + c * kH + i], h2[i], a);
        z[c] = a;
    }
}

// training forward: acts [B][2H] = (h1, h2), logits [B][C]
__global__ void k_mlp_forward(const float* __restrict__ P, const float* __restrict__ X, int B,
                              float* __restrict__ acts, float* __restrict__ logits)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B) return;
    float x[kF], h1[kH], h2[kH], z[kC];
#pragma unroll
    for (int i = 0; i < kF; ++i) x[i] = X[(int64_t)s * kF + i];
    mlp_hidden(P, x, h1, h2);
    mlp_logits(P, h2, z);
    float* a = acts + (int64_t)s * 2 * kH;
    for (int j = 0; j < kH; ++j) {
        a[j] = h1[j];
        a[kH + j] = h2[j];
    }
#pragma unroll
    for (int c = 0; c < kC; ++c) logits[(int64_t)s * kC + c] = z[c];
}

// mean softmax cross entropy over the batch: dlogits = (softmax - onehot) / B,
// loss[0] += sum of per-sample losses / B
__global__ void k_mlp_xent(const float* __restrict__ logits, const int32_t* __restrict__ labels, int B,
                           float* __restrict__ dlogits, float* __restrict__ loss)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.0f;
    if (s < B) {
        const float* z = logits + (int64_t)s * kC;
        float m = z[0];
#pragma unroll
        for (int c = 1; c < kC; ++c) m = fmaxf(m, z[c]);
        float e[kC], sum = 0.0f;
#pragma unroll
        for (int c = 0; c < kC; ++c) {
            e[c] = expf(z[c] - m);
            sum += e[c];
        }
        const int y = min(max(labels[s], 0), kC - 1);  // labels outside 0..5 count as the nearest class
        const float inv = 1.0f / (sum * (float)B);
#pragma unroll
        for (int c = 0; c < kC; ++c) dlogits[(int64_t)s * kC + c] = e[c] * inv - (c == y ? 1.0f / (float)B : 0.0f);
        l = (logf(sum) + m - z[y]) / (float)B;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.0f) atomicAdd(loss, l);
}

// per-sample deltas of the two hidden layers: d2 = (W3^T dz) * [h2 > 0],
// d1 = (W2^T d2) * [h1 > 0]; deltas [B][2H] = (d1, d2)
__global__ void k_mlp_deltas(const float* __restrict__ P, const float* __restrict__ acts,
                             const float* __restrict__ dlogits, int B, float* __restrict__ deltas)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B) return;
    const float* a = acts + (int64_t)s * 2 * kH;
    const float* dz = dlogits + (int64_t)s * kC;
    float d2[kH];
    for (int i = 0; i < kH; ++i) {
        float g = 0.0f;
#pragma unroll
        for (int c = 0; c < kC; ++c) g = fmaf(P[oW3 + c * kH + i], dz[c], g);
        d2[i] = a[kH + i] > 0.0f ? g : 0.0f;
    }
    float* d = deltas + (int64_t)s * 2 * kH;
    for (int i = 0; i < kH; ++i) {
        float g = 0.0f;
        for (int j = 0; j < kH; ++j) g = fmaf(P[oW2 + j * kH + i], d2[j], g);
        d[i] = a[i] > 0.0f ? g : 0.0f;
        d[kH + i] = d2[i];
    }
}

// parameter gradients, one thread per parameter, summed over the batch:
// dW1 = d1 x^T, db1 = sum d1, dW2 = d2 h1^T, db2 = sum d2, dW3 = dz h2^T, db3 = sum dz
__global__ void k_mlp_wgrad(const float* __restrict__ X, const float* __restrict__ acts,
                            const float* __restrict__ deltas, const float* __restrict__ dlogits, int B,
                            float* __restrict__ grads)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= GS_PLAN_PARAMS) return;
    float g = 0.0f;
    if (p < oB1) {
        const int j = (p - oW1) / kF, i = (p - oW1) % kF;
        for (int s = 0; s < B; ++s) g = fmaf(deltas[(int64_t)s * 2 * kH + j], X[(int64_t)s * kF + i], g);
    } else if (p < oW2) {
        const int j = p - oB1;
        for (int s = 0; s < B; ++s) g += deltas[(int64_t)s * 2 * kH + j];
    } else if (p < oB2) {
        const int j = (p - oW2) / kH, i = (p - oW2) % kH;
        for (int s = 0; s < B; ++s) g = fmaf(deltas[(int64_t)s * 2 * kH + kH + j], acts[(int64_t)s * 2 * kH + i], g);
    } else if (p < oW3) {
        const int j = p - oB2;
        for (int s = 0; s < B; ++s) g += deltas[(int64_t)s * 2 * kH + kH + j];
    } else if (p < oB3) {
        const int c = (p - oW3) / kH, i = (p - oW3) % kH;
        for (int s = 0; s < B; ++s) g = fmaf(dlogits[(int64_t)s * kC + c], acts[(int64_t)s * 2 * kH + kH + i], g);
    } else {
        const int c = p - oB3;
        for (int s = 0; s < B; ++s) g += dlogits[(int64_t)s * kC + c];
    }
    grads[p] = g;
}

// Adam (Kingma & Ba, 2015) with bias correction, step t >= 1
__global__ void k_adam(float* __restrict__ params, const float* __restrict__ grads, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = grads[i];
    const float mi = b1 * m[i] + (1.0f - b1) * g;
    const float vi = b2 * v[i] + (1.0f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    params[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace gs

using namespace gs;

extern "C" int gs_tile_features(gs_ctx* c, const gs_camera* cam, const int32_t* offsets, int32_t stride,
                                float* features, void* stream)
{
    if (!c || !cam || !offsets || !features || stride < 1 || stride > GS_MAX_K) return GS_ERR_INVALID_ARG;
    const int T = gs_num_tiles(cam->width, cam->height, c->cfg.tile_size);
    if (T <= 0) return GS_ERR_INVALID_ARG;
    const int threads = 256;
    const unsigned grid = (unsigned)(((int64_t)T * 32 + threads - 1) / threads);
    k_tile_features<<<grid, threads, 0, (cudaStream_t)stream>>>(offsets, stride, T, features);
    c->launches += 1;
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

namespace gs {
// device copy of the planner: the packed parameters, then (16-byte aligned)
// their inference layout
constexpr size_t kPlannerLayoutOffset = ((GS_PLAN_PARAMS + 3) / 4) * 4;
constexpr size_t kPlannerDeviceFloats = kPlannerLayoutOffset + kPlanLayoutFloats;
static PlanShared* planner_layout(gs_ctx* c) { return reinterpret_cast<PlanShared*>(c->d_planner + kPlannerLayoutOffset); }

int plan_frame(gs_ctx* c, const int32_t* offsets, int32_t K, int32_t T, uint8_t* plan, uint8_t* classes,
               cudaStream_t st)
{
    if (!c->planner_ready) return GS_ERR_INVALID_ARG;
    if (T <= 0) return GS_OK;
    // about one tile a warp: each warp's loads of its tile's offsets are one
    // dependent chain, so parallelism over tiles, not fewer weight stagings,
    // sets the time
    const int grid = min((T + 7) / 8, c->num_sms * 8);
    GS_CUDA_TRY(launch_k(c, k_plan_fused, (unsigned)grid, 256, 0, st, offsets, K, T, planner_layout(c), c->cfg.planner_quantile, plan, classes,
                                                 plan + T, c->d_plist));
    c->launches += 1;
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}
}  // namespace gs

extern "C" int gs_planner_set_weights(gs_ctx* c, const float* params, void* stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (!params) {
        c->planner_ready = 0;
        return GS_OK;
    }
    if (!c->d_planner) {
        void* p = nullptr;
        size_t cap = 0;
        const int r = ensure(&p, &cap, kPlannerDeviceFloats * sizeof(float));
        if (r != GS_OK) return r;
        c->d_planner = (float*)p;
    }
    GS_CUDA_TRY(cudaMemcpyAsync(c->d_planner, params, GS_PLAN_PARAMS * sizeof(float), cudaMemcpyDefault,
                                (cudaStream_t)stream));
    k_plan_layout<<<1, 256, 0, (cudaStream_t)stream>>>(c->d_planner, planner_layout(c));
    GS_CUDA_TRY(cudaGetLastError());
    // 20 KB of parameters per block: let as many blocks share an SM as its
    // threads allow (the kernel's time is its tiles' load latency)
    GS_CUDA_TRY(cudaFuncSetAttribute(k_plan_fused, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared));
    c->planner_ready = 1;
    return GS_OK;
}

extern "C" int gs_plan_tiles(gs_ctx* c, const gs_camera* cam, const int32_t* offsets, int32_t stride, uint8_t* plan,
                             uint8_t* classes, void* stream)
{
    if (!c || !cam || !offsets || !plan || stride < 1 || stride > GS_MAX_K) return GS_ERR_INVALID_ARG;
    if (!c->planner_ready) return GS_ERR_INVALID_ARG;
    const int T = gs_num_tiles(cam->width, cam->height, c->cfg.tile_size);
    if (T <= 0) return GS_ERR_INVALID_ARG;
    const int grid = min((T + 7) / 8, c->num_sms * 8);
    GS_CUDA_TRY(launch_k(c, k_plan_fused, (unsigned)grid, 256, 0, (cudaStream_t)stream, offsets, stride, T, planner_layout(c),
                                                                   c->cfg.planner_quantile, plan, classes, nullptr,
                                                                   nullptr));
    c->launches += 1;
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

extern "C" int gs_mlp_forward(const float* params, const float* X, int32_t B, float* acts, float* logits,
                              void* stream)
{
    if (!params || !X || !acts || !logits || B < 1) return GS_ERR_INVALID_ARG;
    k_mlp_forward<<<(unsigned)((B + 127) / 128), 128, 0, (cudaStream_t)stream>>>(params, X, B, acts, logits);
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

extern "C" int gs_mlp_loss_grad(const float* logits, const int32_t* labels, int32_t B, float* dlogits, float* loss,
                                void* stream)
{
    if (!logits || !labels || !dlogits || !loss || B < 1) return GS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    GS_CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(float), st));
    k_mlp_xent<<<(unsigned)((B + 127) / 128), 128, 0, st>>>(logits, labels, B, dlogits, loss);
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

extern "C" int gs_mlp_backward(const float* params, const float* X, const float* acts, const float* dlogits,
                               int32_t B, float* deltas, float* grads, void* stream)
{
    if (!params || !X || !acts || !dlogits || !deltas || !grads || B < 1) return GS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    k_mlp_deltas<<<(unsigned)((B + 127) / 128), 128, 0, st>>>(params, acts, dlogits, B, deltas);
    k_mlp_wgrad<<<(unsigned)((GS_PLAN_PARAMS + 127) / 128), 128, 0, st>>>(X, acts, deltas, dlogits, B, grads);
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

extern "C" int gs_adam_step(float* params, const float* grads, float* m, float* v, int32_t n, float lr, float beta1,
                            float beta2, float eps, int32_t step, void* stream)
{
    if (!params || !grads || !m || !v || n < 1 || step < 1 || !(lr > 0.0f)) return GS_ERR_INVALID_ARG;
    const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
    k_adam<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(params, grads, m, v, n, lr, beta1, beta2,
                                                                          eps, c1, c2);
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}
