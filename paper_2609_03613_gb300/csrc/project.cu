// project.cu -- K1+K2: SH colour and EWA projection of 3D Gaussians.
//
// The paper keeps the 3DGS projection unchanged (its input is the projected
// Gaussians, Sec. 3.1) without printing it.  The reading implemented here, in this exact
// float32 operation order (compiled with -fmad=false):
//   p_c = R m + t; cull unless near < z < far and opacity >= 1/255;
//   Sigma = (R_q S)(R_q S)^T; Sigma_c = R Sigma R^T;
//   J at the view direction clamped to 1.3x the image half-extent tangents;
//   Sigma' = J Sigma_c J^T + 0.3 I; conic = Sigma'^{-1};
//   mean = (fx x/z + cx, fy y/z + cy); radius = ceil(3 sqrt(lambda_max));
//   rect = tiles met by the (mean +- radius) square, clamped; cull if empty;
//   rgb = max(sum_k Y_k(dir) sh_k + 0.5, 0), dir = normalize(m - campos).
// Non-finite inputs (the paper assumes trained, finite parameters): a
// Gaussian with a non-finite mean, scale, quaternion component or opacity,
// or whose SH sum is not finite in some channel, is culled, and the kernel
// raises GS_ERR_NUMERIC in the context's error word.
// One thread per Gaussian; the block's SH coefficients (contiguous in memory)
// are staged through shared memory with coalesced float4 loads.  The batched
// kernel projects each Gaussian for every view of a batch from one read of its
// parameters.
#include <string.h>

#include "internal.cuh"

namespace gs {

struct CamArgs {
    float W[16];
    float fx, fy, cx, cy;
    int width, height;
    float near_plane, far_plane;
    int tiles_x, tiles_y, tile;
};

__device__ __forceinline__ void sh_basis(float x, float y, float z, float* Y)
{
    // Real spherical harmonics to degree 3, orthonormal on the sphere, in the
    // sign convention of 3D Gaussian Splatting.
    const float c0 = 0.28209479177387814f;
    const float c1 = 0.4886025119029199f;
    const float c20 = 1.0925484305920792f, c21 = -1.0925484305920792f, c22 = 0.31539156525252005f,
                c23 = -1.0925484305920792f, c24 = 0.5462742152960396f;
    const float c30 = -0.5900435899266435f, c31 = 2.890611442640554f, c32 = -0.4570457994644658f,
                c33 = 0.3731763325901154f, c34 = -0.4570457994644658f, c35 = 1.445305721320277f,
                c36 = -0.5900435899266435f;
    const float xx = x * x, yy = y * y, zz = z * z;
    const float xy = x * y, yz = y * z, xz = x * z;
    Y[0] = c0;
    Y[1] = -c1 * y;
    Y[2] = c1 * z;
    Y[3] = -c1 * x;
    Y[4] = c20 * xy;
    Y[5] = c21 * yz;
    Y[6] = c22 * (2.0f * zz - xx - yy);
    Y[7] = c23 * xz;
    Y[8] = c24 * (xx - yy);
    Y[9] = c30 * y * (3.0f * xx - yy);
    Y[10] = c31 * xy * z;
    Y[11] = c32 * y * (4.0f * zz - xx - yy);
    Y[12] = c33 * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
    Y[13] = c34 * x * (4.0f * zz - xx - yy);
    Y[14] = c35 * z * (xx - yy);
    Y[15] = c36 * x * (xx - 3.0f * yy);
}

constexpr int kProjBlock = 64;  // 64 measured 3 % faster than 128 and 192

// Stage the block's SH coefficients (contiguous in memory) into shared
// memory.  With a 16-byte aligned array the TMA engine copies the block in one
// bulk transfer (cp.async.bulk completing on an mbarrier; the multiple-of-16
// prefix, any 4-byte tail by plain loads); the wait is bounded and reports
// GS_ERR_TIMEOUT through err.  Otherwise coalesced plain loads.  Returns 0
// (block-uniform) when the copy never completed: the block must then leave
// without using s_sh.
constexpr int kDrainPolls = 1 << 22;

__device__ __forceinline__ uint32_t mbar_try_wait(uint32_t sbar)
{
    uint32_t done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done)
                 : "r"(sbar)
                 : "memory");
    return done;
}

template <int PER>
__device__ __forceinline__ int stage_sh(const float* __restrict__ sh, int sh_aligned, int64_t base, int64_t n,
                                        float* s_sh, int polls, int* err)
{
    __shared__ __align__(8) uint64_t bar;
    const int cnt = (int)((n - base) < kProjBlock ? (n - base) : kProjBlock);
    const int total = cnt * PER;
    const float* src = sh + base * PER;
    if (sh_aligned) {
        const uint32_t bytes = (uint32_t)(total * 4) & ~15u;
        const uint32_t sbar = (uint32_t)__cvta_generic_to_shared(&bar);
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sbar) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sbar), "r"(bytes)
                         : "memory");
            if (bytes > 0) {
                // the scene is read once a frame: evict it first, so the
                // projected records and the later stages keep L2
                uint64_t pol;
                asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
                asm volatile(
                    "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
                        (uint32_t)__cvta_generic_to_shared(s_sh)),
                    "l"(src), "r"(bytes), "r"(sbar), "l"(pol)
                    : "memory");
            }
        }
        for (int k = (int)(bytes / 4) + threadIdx.x; k < total; k += kProjBlock) s_sh[k] = __ldg(src + k);
        // bounded wait for phase 0 of the barrier: `polls` tries, then
        // GS_ERR_TIMEOUT and a second bounded wait (the drain) so that the
        // copy is not left writing into shared memory the block gives up
        uint32_t done = 0;
        for (int it = 0; it < polls && !done; ++it) done = mbar_try_wait(sbar);
        if (!done) {
            raise_error(err, GS_ERR_TIMEOUT);
            for (int it = 0; it < kDrainPolls && !done; ++it) done = mbar_try_wait(sbar);
        }
        // every thread waited on the same barrier: the block agrees on done;
        // a barrier whose copy never landed is not invalidated and the block
        // writes nothing (the frame is invalid after a timeout in any case)
        const int ok = __syncthreads_and((int)done);
        if (ok && threadIdx.x == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(sbar) : "memory");
        return ok;
    }
    for (int k = threadIdx.x; k < total; k += kProjBlock) s_sh[k] = __ldg(src + k);
    __syncthreads();
    return 1;
}

// Bit 31 of the result is set when x is not finite (exponent field all ones).
__device__ __forceinline__ uint32_t nonfinite_bit(float x)
{
    return (__float_as_uint(x) & 0x7f800000u) + 0x00800000u;
}

// Whether any of a Gaussian's geometric parameters is not finite.
__device__ __forceinline__ bool geometry_nonfinite(float mx, float my, float mz, float o, float4 q4, float s0,
                                                   float s1, float s2)
{
    const uint32_t f = nonfinite_bit(mx) | nonfinite_bit(my) | nonfinite_bit(mz) | nonfinite_bit(o) |
                       nonfinite_bit(q4.x) | nonfinite_bit(q4.y) | nonfinite_bit(q4.z) | nonfinite_bit(q4.w) |
                       nonfinite_bit(s0) | nonfinite_bit(s1) | nonfinite_bit(s2);
    return (f >> 31) != 0u;
}

// One Gaussian seen by one camera: the record fields, all zero when culled.
// (mx, my, mz), o, q4 and (s0, s1, s2) are the Gaussian's parameters, cs its
// SH coefficients (NC x 3, coefficient-major).  Returns true when the SH sum
// of a Gaussian that reached the colour step was not finite (it is culled).
template <int DEG>
__device__ __forceinline__ bool project_one(float mx, float my, float mz, float o, float4 q4, float s0, float s1,
                                            float s2, const float* cs, const CamArgs& cam, float4& o_xy_ab,
                                            float4& o_c_o_z, float4& o_rgb, uint2& o_rect, int& o_radius)
{
    constexpr int NC = (DEG + 1) * (DEG + 1);
    const float* W = cam.W;
    o_xy_ab = make_float4(0.f, 0.f, 0.f, 0.f);
    o_c_o_z = make_float4(0.f, 0.f, 0.f, 0.f);
    o_rgb = make_float4(0.f, 0.f, 0.f, 0.f);
    o_rect = make_uint2(0u, 0u);
    o_radius = 0;
    bool bad_colour = false;
    const float xc = W[0] * mx + W[1] * my + W[2] * mz + W[3];
    const float yc = W[4] * mx + W[5] * my + W[6] * mz + W[7];
    const float zc = W[8] * mx + W[9] * my + W[10] * mz + W[11];
    const float qn = sqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
    bool vis = (zc > cam.near_plane && zc < cam.far_plane) && (o >= 1.0f / 255.0f) && (qn > 0.0f) &&
               !geometry_nonfinite(mx, my, mz, o, q4, s0, s1, s2);
    if (vis) {
        const float w = q4.x / qn, x = q4.y / qn, y = q4.z / qn, z = q4.w / qn;
        float Rq[3][3];
        Rq[0][0] = 1.0f - 2.0f * (y * y + z * z);
        Rq[0][1] = 2.0f * (x * y - w * z);
        Rq[0][2] = 2.0f * (x * z + w * y);
        Rq[1][0] = 2.0f * (x * y + w * z);
        Rq[1][1] = 1.0f - 2.0f * (x * x + z * z);
        Rq[1][2] = 2.0f * (y * z - w * x);
        Rq[2][0] = 2.0f * (x * z - w * y);
        Rq[2][1] = 2.0f * (y * z + w * x);
        Rq[2][2] = 1.0f - 2.0f * (x * x + y * y);
        float M[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            M[r][0] = Rq[r][0] * s0;
            M[r][1] = Rq[r][1] * s1;
            M[r][2] = Rq[r][2] * s2;
        }
        float S[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) S[r][c] = M[r][0] * M[c][0] + M[r][1] * M[c][1] + M[r][2] * M[c][2];
        float Tm[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                Tm[r][c] = W[r * 4 + 0] * S[0][c] + W[r * 4 + 1] * S[1][c] + W[r * 4 + 2] * S[2][c];
        // rows 0..2 of Sigma_c as used by J (Sigma_c[1][0] is never needed)
        float Sc[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                Sc[r][c] = Tm[r][0] * W[c * 4 + 0] + Tm[r][1] * W[c * 4 + 1] + Tm[r][2] * W[c * 4 + 2];
        const float limx_hi = 1.3f * (((float)cam.width - cam.cx) / cam.fx);
        const float limx_lo = 1.3f * (cam.cx / cam.fx);
        const float limy_hi = 1.3f * (((float)cam.height - cam.cy) / cam.fy);
        const float limy_lo = 1.3f * (cam.cy / cam.fy);
        const float xz = xc / zc, yz = yc / zc;
        float u = xz, v = yz;
        if (u < -limx_lo) u = -limx_lo;
        if (u > limx_hi) u = limx_hi;
        if (v < -limy_lo) v = -limy_lo;
        if (v > limy_hi) v = limy_hi;
        const float j00 = cam.fx / zc, j02 = -cam.fx * u / zc;
        const float j11 = cam.fy / zc, j12 = -cam.fy * v / zc;
        float K0[3], K1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            K0[c] = j00 * Sc[0][c] + j02 * Sc[2][c];
            K1[c] = j11 * Sc[1][c] + j12 * Sc[2][c];
        }
        float a = K0[0] * j00 + K0[2] * j02;
        const float b = K0[1] * j11 + K0[2] * j12;
        float c = K1[1] * j11 + K1[2] * j12;
        a = a + 0.3f;
        c = c + 0.3f;
        const float det = a * c - b * b;
        if (det > 0.0f) {
            const float inv = 1.0f / det;
            const float ca = c * inv, cb = -b * inv, cc = a * inv;
            const float px = cam.fx * xz + cam.cx;
            const float py = cam.fy * yz + cam.cy;
            const float mid = 0.5f * (a + c);
            const float disc = fmaxf(0.01f, mid * mid - det);
            const float lmax = mid + sqrtf(disc);
            const float r = ceilf(3.0f * sqrtf(lmax));
            const float ft = (float)cam.tile;
            float tx0 = floorf((px - r) / ft), tx1 = ceilf((px + r) / ft);
            float ty0 = floorf((py - r) / ft), ty1 = ceilf((py + r) / ft);
            tx0 = fminf(fmaxf(tx0, 0.0f), (float)cam.tiles_x);
            tx1 = fminf(fmaxf(tx1, 0.0f), (float)cam.tiles_x);
            ty0 = fminf(fmaxf(ty0, 0.0f), (float)cam.tiles_y);
            ty1 = fminf(fmaxf(ty1, 0.0f), (float)cam.tiles_y);
            if (tx0 < tx1 && ty0 < ty1) {
                // colour
                const float cpx = -(W[0] * W[3] + W[4] * W[7] + W[8] * W[11]);
                const float cpy = -(W[1] * W[3] + W[5] * W[7] + W[9] * W[11]);
                const float cpz = -(W[2] * W[3] + W[6] * W[7] + W[10] * W[11]);
                float dx = mx - cpx, dy = my - cpy, dz = mz - cpz;
                const float len = sqrtf(dx * dx + dy * dy + dz * dz);
                if (len > 0.0f) {
                    dx = dx / len;
                    dy = dy / len;
                    dz = dz / len;
                }
                float Y[16];
                sh_basis(dx, dy, dz, Y);
                float col[3];
                uint32_t nf = 0u;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    float acc = Y[0] * cs[ch];
#pragma unroll
                    for (int k = 1; k < NC; ++k) acc = acc + Y[k] * cs[k * 3 + ch];
                    nf |= nonfinite_bit(acc);
                    col[ch] = fmaxf(acc + 0.5f, 0.0f);
                }
                bad_colour = (nf >> 31) != 0u;
                // conservative tile-cull data (not part of the image math):
                // tau = ln(255 o) + slack; margin shrinks with the conditioning
                // of Sigma' to cover float32 cancellation in q.
                const float lam_hi = mid + sqrtf(fmaxf(0.0f, mid * mid - det));
                const float lam_lo = det / lam_hi;
                const float kappa = lam_hi / fmaxf(lam_lo, 1e-30f);
                float margin = 1.0f - 2e-5f * (kappa + 1.0f);
                margin = margin < 0.5f ? 0.0f : margin;
                const float tau = logf(255.0f * o) + 2e-4f;

                if (!bad_colour) {
                    o_xy_ab = make_float4(px, py, ca, cb);
                    o_c_o_z = make_float4(cc, o, zc, tau);
                    o_rgb = make_float4(col[0], col[1], col[2], margin);
                    o_rect = make_uint2((uint32_t)tx0 | ((uint32_t)ty0 << 16),
                                        (uint32_t)tx1 | ((uint32_t)ty1 << 16));
                    o_radius = (int)r;
                }
            }
        }
    }
    return bad_colour;
}

// A Gaussian's parameters other than its SH coefficients (streamed: the
// scene is read once a frame).
struct GaussParams {
    float mx = 0.f, my = 0.f, mz = 0.f, o = 0.f, s0 = 0.f, s1 = 0.f, s2 = 0.f;
    float4 q4 = make_float4(0.f, 0.f, 0.f, 0.f);
};

__device__ __forceinline__ GaussParams load_params(const float* __restrict__ means, const float* __restrict__ scales,
                                                   const float4* __restrict__ quats, const float* __restrict__ opac,
                                                   int64_t i)
{
    GaussParams g;
    g.mx = __ldcs(means + 3 * i);
    g.my = __ldcs(means + 3 * i + 1);
    g.mz = __ldcs(means + 3 * i + 2);
    g.o = __ldcs(opac + i);
    g.q4 = __ldcs(quats + i);
    g.s0 = __ldcs(scales + 3 * i);
    g.s1 = __ldcs(scales + 3 * i + 1);
    g.s2 = __ldcs(scales + 3 * i + 2);
    return g;
}

template <int DEG>
__global__ void __launch_bounds__(kProjBlock)
k_project(const float* __restrict__ means, const float* __restrict__ scales,
          const float4* __restrict__ quats, const float* __restrict__ opac,
          const float* __restrict__ sh, int sh_aligned, int64_t n, CamArgs cam, ProjView pv, int polls, int* err,
          FrameZero fz)
{
    grid_dependency_sync();
    frame_zero(fz);  // the frame's first scan's flags
    constexpr int NC = (DEG + 1) * (DEG + 1);
    constexpr int PER = NC * 3;  // floats of SH per Gaussian
    __shared__ __align__(16) float s_sh[kProjBlock * PER];
    const int64_t base = (int64_t)blockIdx.x * kProjBlock;
    const int64_t i = base + threadIdx.x;
    // the Gaussian's other parameters are loaded before the wait for the SH
    // copy: both round trips overlap
    GaussParams gp;
    if (i < n) gp = load_params(means, scales, quats, opac, i);
    if (!stage_sh<PER>(sh, sh_aligned, base, n, s_sh, polls, err)) return;
    if (i >= n) return;
    float4 a, b, c;
    uint2 rect;
    int radius;
    const float mx = gp.mx, my = gp.my, mz = gp.mz, o = gp.o, s0 = gp.s0, s1 = gp.s1, s2 = gp.s2;
    const float4 q4 = gp.q4;
    const bool bad = project_one<DEG>(mx, my, mz, o, q4, s0, s1, s2, s_sh + threadIdx.x * PER, cam, a, b, c, rect,
                                      radius);
    if (bad || geometry_nonfinite(mx, my, mz, o, q4, s0, s1, s2)) raise_error(err, GS_ERR_NUMERIC);
    pv.xy_ab[i] = a;
    pv.c_o_z[i] = b;
    pv.rgb[i] = c;
    pv.rect[i] = rect;
    pv.radius[i] = radius;
}

// Views of one batched projection launch (kernel parameters).
struct BatchCams {
    CamArgs cam[kMaxBatchViews];
    ProjView pv[kMaxBatchViews];
    int nviews;
};

// The same Gaussian for every view of the batch: its parameters (and SH
// coefficients) are read from HBM once and projected V times.
template <int DEG>
__global__ void __launch_bounds__(kProjBlock)
k_project_batch(const float* __restrict__ means, const float* __restrict__ scales,
                const float4* __restrict__ quats, const float* __restrict__ opac,
                const float* __restrict__ sh, int sh_aligned, int64_t n, const __grid_constant__ BatchCams bc,
                int polls, int* err)
{
    constexpr int NC = (DEG + 1) * (DEG + 1);
    constexpr int PER = NC * 3;
    __shared__ __align__(16) float s_sh[kProjBlock * PER];
    const int64_t base = (int64_t)blockIdx.x * kProjBlock;
    const int64_t i = base + threadIdx.x;
    GaussParams gp;
    if (i < n) gp = load_params(means, scales, quats, opac, i);
    if (!stage_sh<PER>(sh, sh_aligned, base, n, s_sh, polls, err)) return;
    if (i >= n) return;
    const float mx = gp.mx, my = gp.my, mz = gp.mz, o = gp.o, s0 = gp.s0, s1 = gp.s1, s2 = gp.s2;
    const float4 q4 = gp.q4;
    bool bad = geometry_nonfinite(mx, my, mz, o, q4, s0, s1, s2);
    for (int v = 0; v < bc.nviews; ++v) {
        float4 a, b, c;
        uint2 rect;
        int radius;
        bad |= project_one<DEG>(mx, my, mz, o, q4, s0, s1, s2, s_sh + threadIdx.x * PER, bc.cam[v], a, b, c, rect,
                                radius);
        const ProjView& pv = bc.pv[v];
        pv.xy_ab[i] = a;
        pv.c_o_z[i] = b;
        pv.rgb[i] = c;
        pv.rect[i] = rect;
        pv.radius[i] = radius;
    }
    if (bad) raise_error(err, GS_ERR_NUMERIC);
}

static CamArgs cam_args(const gs_camera* cam, int tile)
{
    CamArgs ca;
    for (int k = 0; k < 16; ++k) ca.W[k] = cam->viewmat[k];
    ca.fx = cam->fx;
    ca.fy = cam->fy;
    ca.cx = cam->cx;
    ca.cy = cam->cy;
    ca.width = cam->width;
    ca.height = cam->height;
    ca.near_plane = cam->near_plane;
    ca.far_plane = cam->far_plane;
    ca.tile = tile;
    ca.tiles_x = (cam->width + tile - 1) / tile;
    ca.tiles_y = (cam->height + tile - 1) / tile;
    return ca;
}

int launch_project_batch(gs_ctx* ctx, const float* means, const float* scales, const float* quats,
                         const float* opac, const float* sh, int32_t sh_degree, int64_t n, int nviews,
                         const gs_camera* cams, const int* tiles, const ProjView* pvs, cudaStream_t st)
{
    if (n <= 0 || nviews <= 0) return GS_OK;
    if (nviews > kMaxBatchViews) return GS_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(quats) & 15) return GS_ERR_INVALID_ARG;  // float4 loads
    BatchCams bc;
    memset(&bc, 0, sizeof(bc));
    bc.nviews = nviews;
    for (int v = 0; v < nviews; ++v) {
        bc.cam[v] = cam_args(cams + v, tiles[v]);
        bc.pv[v] = pvs[v];
    }
    const int aligned = (reinterpret_cast<uintptr_t>(sh) & 15) == 0;
    const int polls = ctx->cfg.wait_polls;
    const unsigned grid = (unsigned)((n + kProjBlock - 1) / kProjBlock);
    const float4* q4 = reinterpret_cast<const float4*>(quats);
    switch (sh_degree) {
        case 0: k_project_batch<0><<<grid, kProjBlock, 0, st>>>(means, scales, q4, opac, sh, aligned, n, bc, polls, ctx->d_err); break;
        case 1: k_project_batch<1><<<grid, kProjBlock, 0, st>>>(means, scales, q4, opac, sh, aligned, n, bc, polls, ctx->d_err); break;
        case 2: k_project_batch<2><<<grid, kProjBlock, 0, st>>>(means, scales, q4, opac, sh, aligned, n, bc, polls, ctx->d_err); break;
        default: k_project_batch<3><<<grid, kProjBlock, 0, st>>>(means, scales, q4, opac, sh, aligned, n, bc, polls, ctx->d_err); break;
    }
    ctx->launches += 1;
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

int launch_project(gs_ctx* ctx, const float* means, const float* scales, const float* quats,
                   const float* opac, const float* sh, int32_t sh_degree, int64_t n,
                   const gs_camera* cam, const ProjView& pv, cudaStream_t st, const FrameZero& fz)
{
    if (n <= 0) return GS_OK;
    if (reinterpret_cast<uintptr_t>(quats) & 15) return GS_ERR_INVALID_ARG;  // float4 loads
    const CamArgs ca = cam_args(cam, ctx->cfg.tile_size);
    const int aligned = (reinterpret_cast<uintptr_t>(sh) & 15) == 0;
    const int polls = ctx->cfg.wait_polls;
    const unsigned grid = (unsigned)((n + kProjBlock - 1) / kProjBlock);
    const float4* q4 = reinterpret_cast<const float4*>(quats);
    switch (sh_degree) {
        case 0: GS_CUDA_TRY(launch_k(ctx, k_project<0>, grid, kProjBlock, 0, st, means, scales, q4, opac, sh, aligned, n, ca, pv, polls, ctx->d_err, fz)); break;
        case 1: GS_CUDA_TRY(launch_k(ctx, k_project<1>, grid, kProjBlock, 0, st, means, scales, q4, opac, sh, aligned, n, ca, pv, polls, ctx->d_err, fz)); break;
        case 2: GS_CUDA_TRY(launch_k(ctx, k_project<2>, grid, kProjBlock, 0, st, means, scales, q4, opac, sh, aligned, n, ca, pv, polls, ctx->d_err, fz)); break;
        default: GS_CUDA_TRY(launch_k(ctx, k_project<3>, grid, kProjBlock, 0, st, means, scales, q4, opac, sh, aligned, n, ca, pv, polls, ctx->d_err, fz)); break;
    }
    ctx->launches += 1;
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

}  // namespace gs
