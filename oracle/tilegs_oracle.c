/*
 * tilegs_oracle.c -- plain, slow CPU oracle for the TileGS forward path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  The
 * product path (the CUDA library) never calls it, and the two share no code.
 *
 * What it computes (paper: "TileGS: Tile-Local Depth Binning for Gaussian
 * Splatting Rasterization"):
 *   - projection of 3D Gaussians to 2D mean / conic / depth / tile rectangle
 *     and SH colour (Sec. 3.1: the paper keeps the 3DGS/EWA projection
 *     unchanged and does not print it; the reading used is written out below);
 *   - the per-tile candidate lists in exact (depth, gid) order (Sec. 3.1,
 *     baseline globally sorted tile-depth stream);
 *   - front-to-back alpha compositing per pixel (Sec. 3.1 and the supplement's
 *     binned raster traversal algorithm: same splat test and compositing as
 *     the baseline);
 *   - robust depth-range estimation (supplement, algorithm "Robust depth-range
 *     estimation");
 *   - the clamped log-space depth-to-bin map and tile-local bin construction
 *     (supplement, algorithm "Tile-local bin construction" and the
 *     log-depth-bin formula beside it);
 *   - selective-repair selection with the fixed rules and greedy entry budget
 *     (Sec. 3.5, table of exact-repair selection rules; supplement, algorithm
 *     "Selective repair selection and local exact sorting").
 *
 * Precision: float32 where a floating-point value decides an integer outcome
 * (tile rectangle, alpha skip, transmittance stop, bin index), evaluated in
 * the exact operation order written here; build with -ffp-contract=off so no
 * multiply-add is fused unless fmaf() is written.  An fp64 twin of the
 * projection and compositing (orc64_*) serves the invariant and closed-form
 * checks.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Elementary functions of the spec.                                         */
/* ------------------------------------------------------------------------ */

static float f_from_bits(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }
static uint32_t bits_of(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

/* exp(x) by Cody-Waite range reduction and a degree-7 Taylor polynomial
 * (W. J. Cody, W. Waite, "Software Manual for the Elementary Functions",
 * 1980).  x = n ln2 + r with n = round(x log2 e), |r| <= ln2/2;
 * e^r = sum_{k<=7} r^k/k! by Horner; result = e^r * 2^n.
 * Valid on [-87, 88] (clamped).  Rounding of n uses the 1.5*2^23 shifter. */
float orc_expf(float x)
{
    const float LOG2E = 1.44269504088896341f;
    const float LN2_HI = 0.693145751953125f;      /* ln 2 to 16 leading bits */
    const float LN2_LO = 1.42860682030941723e-6f; /* ln 2 - LN2_HI */
    const float SHIFT = 12582912.0f;              /* 1.5 * 2^23 */
    if (x < -87.0f) x = -87.0f;
    if (x > 88.0f) x = 88.0f;
    float k = fmaf(x, LOG2E, SHIFT);
    float n = k - SHIFT;
    float r = fmaf(n, -LN2_HI, x);
    r = fmaf(n, -LN2_LO, r);
    float p = 1.0f / 5040.0f;
    p = fmaf(p, r, 1.0f / 720.0f);
    p = fmaf(p, r, 1.0f / 120.0f);
    p = fmaf(p, r, 1.0f / 24.0f);
    p = fmaf(p, r, 1.0f / 6.0f);
    p = fmaf(p, r, 0.5f);
    p = fmaf(p, r, 1.0f);
    p = fmaf(p, r, 1.0f);
    int32_t ni = (int32_t)n;
    float scale = f_from_bits((uint32_t)(ni + 127) << 23);
    return p * scale;
}

/* ln(x) for normal x > 0: x = 2^e m with m in (sqrt(1/2), sqrt(2)],
 * ln m = 2 atanh(s) = 2 (s + s^3/3 + s^5/5 + s^7/7 + s^9/9), s = (m-1)/(m+1)
 * (Abramowitz & Stegun 4.1.27); ln x = e ln2 + ln m. */
float orc_logf(float x)
{
    const float LN2_HI = 0.693145751953125f;
    const float LN2_LO = 1.42860682030941723e-6f;
    uint32_t u = bits_of(x);
    int32_t e = (int32_t)((u >> 23) & 0xffu) - 127;
    float m = f_from_bits((u & 0x007fffffu) | 0x3f800000u);
    if (m > 1.41421356f) { m = m * 0.5f; e = e + 1; }
    float s = (m - 1.0f) / (m + 1.0f);
    float s2 = s * s;
    float p = 1.0f / 9.0f;
    p = fmaf(p, s2, 1.0f / 7.0f);
    p = fmaf(p, s2, 1.0f / 5.0f);
    p = fmaf(p, s2, 1.0f / 3.0f);
    p = fmaf(p, s2, 1.0f);
    float lnm = (2.0f * s) * p;
    float fe = (float)e;
    return fmaf(fe, LN2_HI, fmaf(fe, LN2_LO, lnm));
}

/* ------------------------------------------------------------------------ */
/* Projection (Sec. 3.1: the method starts from 3DGS's projected Gaussians). */
/* ------------------------------------------------------------------------ */

/* Real spherical-harmonic basis up to degree 3 (orthonormal on the unit
 * sphere, the sign convention of 3D Gaussian Splatting). */
static const float SH_C0 = 0.28209479177387814f;
static const float SH_C1 = 0.4886025119029199f;
static const float SH_C2[5] = {1.0925484305920792f, -1.0925484305920792f,
                               0.31539156525252005f, -1.0925484305920792f,
                               0.5462742152960396f};
static const float SH_C3[7] = {-0.5900435899266435f, 2.890611442640554f,
                               -0.4570457994644658f, 0.3731763325901154f,
                               -0.4570457994644658f, 1.445305721320277f,
                               -0.5900435899266435f};

void orc_sh_basis(float x, float y, float z, float* Y)
{
    float xx = x * x, yy = y * y, zz = z * z;
    float xy = x * y, yz = y * z, xz = x * z;
    Y[0] = SH_C0;
    Y[1] = -SH_C1 * y;
    Y[2] = SH_C1 * z;
    Y[3] = -SH_C1 * x;
    Y[4] = SH_C2[0] * xy;
    Y[5] = SH_C2[1] * yz;
    Y[6] = SH_C2[2] * (2.0f * zz - xx - yy);
    Y[7] = SH_C2[3] * xz;
    Y[8] = SH_C2[4] * (xx - yy);
    Y[9] = SH_C3[0] * y * (3.0f * xx - yy);
    Y[10] = SH_C3[1] * xy * z;
    Y[11] = SH_C3[2] * y * (4.0f * zz - xx - yy);
    Y[12] = SH_C3[3] * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
    Y[13] = SH_C3[4] * x * (4.0f * zz - xx - yy);
    Y[14] = SH_C3[5] * z * (xx - yy);
    Y[15] = SH_C3[6] * x * (xx - 3.0f * yy);
}

/*
 * Project n Gaussians through one pinhole camera (OpenCV axes).
 *   means [n,3], scales [n,3] (linear), quats [n,4] (w,x,y,z, any norm > 0),
 *   opac [n] in [0,1], sh [n, (deg+1)^2, 3]; viewmat row-major world->camera.
 * Outputs per Gaussian: mean2d [n,2], conic [n,3] (upper triangle of the
 * inverse 2D covariance: a, b, c), depth [n], radius [n], rect [n,4]
 * (tx0, ty0, tx1, ty1; tiles tx0 <= tx < tx1), rgb [n,3], visible [n].
 * Invisible Gaussians get radius 0, an empty rect and zeros elsewhere.
 *
 * The reading (Sec. 3.1 leaves it to 3DGS/EWA splatting):
 *   p_c = R m + t; cull unless near < z < far; cull if opacity < 1/255
 *   (such a Gaussian can never reach the alpha test); Sigma = (R_q S)(R_q S)^T;
 *   Sigma_c = R Sigma R^T; J evaluated at the direction clamped to 1.3x the
 *   image half-extent tangents; Sigma' = J Sigma_c J^T + 0.3 I;
 *   conic = Sigma'^{-1}; mean2d = (fx x/z + cx, fy y/z + cy);
 *   radius = ceil(3 sqrt(lambda_max)); rect = tiles touched by the
 *   (mean +- radius) square, clamped to the grid; cull if empty;
 *   rgb = max(sum_k Y_k(dir) sh_k + 0.5, 0) with dir = normalize(m - campos).
 * Non-finite inputs (a reading: the paper assumes trained, finite
 * parameters and says nothing of others): a Gaussian with a non-finite
 * mean, scale, quaternion component or opacity is culled, and so is one whose
 * SH sum is not finite in some channel.
 */
void orc_project(int64_t n, const float* means, const float* scales, const float* quats,
                 const float* opac, const float* sh, int sh_degree, const float* W,
                 float fx, float fy, float cx, float cy, int width, int height,
                 float near_plane, float far_plane, int tile,
                 float* mean2d, float* conic, float* depth, int32_t* radius,
                 int32_t* rect, float* rgb, uint8_t* visible)
{
    const int tiles_x = (width + tile - 1) / tile;
    const int tiles_y = (height + tile - 1) / tile;
    const float ftile = (float)tile;
    const int ncoef = (sh_degree + 1) * (sh_degree + 1);
    /* camera centre in world coordinates: -R^T t */
    float campos[3];
    for (int j = 0; j < 3; ++j)
        campos[j] = -(W[0 * 4 + j] * W[3] + W[1 * 4 + j] * W[7] + W[2 * 4 + j] * W[11]);
    const float limx_hi = 1.3f * (((float)width - cx) / fx);
    const float limx_lo = 1.3f * (cx / fx);
    const float limy_hi = 1.3f * (((float)height - cy) / fy);
    const float limy_lo = 1.3f * (cy / fy);

    for (int64_t i = 0; i < n; ++i) {
        mean2d[2 * i] = mean2d[2 * i + 1] = 0.0f;
        conic[3 * i] = conic[3 * i + 1] = conic[3 * i + 2] = 0.0f;
        depth[i] = 0.0f;
        radius[i] = 0;
        rect[4 * i] = rect[4 * i + 1] = rect[4 * i + 2] = rect[4 * i + 3] = 0;
        rgb[3 * i] = rgb[3 * i + 1] = rgb[3 * i + 2] = 0.0f;
        visible[i] = 0;

        const float mx = means[3 * i], my = means[3 * i + 1], mz = means[3 * i + 2];
        int finite = isfinite(mx) && isfinite(my) && isfinite(mz) && isfinite(opac[i]);
        for (int k = 0; k < 4; ++k) finite = finite && isfinite(quats[4 * i + k]);
        for (int k = 0; k < 3; ++k) finite = finite && isfinite(scales[3 * i + k]);
        if (!finite) continue;
        const float xc = W[0] * mx + W[1] * my + W[2] * mz + W[3];
        const float yc = W[4] * mx + W[5] * my + W[6] * mz + W[7];
        const float zc = W[8] * mx + W[9] * my + W[10] * mz + W[11];
        if (!(zc > near_plane && zc < far_plane)) continue;
        const float o = opac[i];
        if (!(o >= 1.0f / 255.0f)) continue;

        /* rotation from the normalised quaternion */
        float qw = quats[4 * i], qx = quats[4 * i + 1], qy = quats[4 * i + 2], qz = quats[4 * i + 3];
        float qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
        if (!(qn > 0.0f)) continue;
        float w = qw / qn, x = qx / qn, y = qy / qn, z = qz / qn;
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
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) M[r][c] = Rq[r][c] * scales[3 * i + c];
        float S[3][3];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) S[r][c] = M[r][0] * M[c][0] + M[r][1] * M[c][1] + M[r][2] * M[c][2];
        /* camera-space covariance R S R^T */
        float Tm[3][3], Sc[3][3];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                Tm[r][c] = W[r * 4 + 0] * S[0][c] + W[r * 4 + 1] * S[1][c] + W[r * 4 + 2] * S[2][c];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                Sc[r][c] = Tm[r][0] * W[c * 4 + 0] + Tm[r][1] * W[c * 4 + 1] + Tm[r][2] * W[c * 4 + 2];
        /* perspective Jacobian at the clamped direction */
        const float xz = xc / zc, yz = yc / zc;
        float u = xz, v = yz;
        if (u < -limx_lo) u = -limx_lo;
        if (u > limx_hi) u = limx_hi;
        if (v < -limy_lo) v = -limy_lo;
        if (v > limy_hi) v = limy_hi;
        const float j00 = fx / zc, j02 = -fx * u / zc;
        const float j11 = fy / zc, j12 = -fy * v / zc;
        float K0[3], K1[3];
        for (int c = 0; c < 3; ++c) {
            K0[c] = j00 * Sc[0][c] + j02 * Sc[2][c];
            K1[c] = j11 * Sc[1][c] + j12 * Sc[2][c];
        }
        float a = K0[0] * j00 + K0[2] * j02;
        float b = K0[1] * j11 + K0[2] * j12;
        float c = K1[1] * j11 + K1[2] * j12;
        a = a + 0.3f;
        c = c + 0.3f;
        const float det = a * c - b * b;
        if (!(det > 0.0f)) continue;
        const float inv = 1.0f / det;
        const float ca = c * inv, cb = -b * inv, cc = a * inv;
        const float px = fx * xz + cx;
        const float py = fy * yz + cy;
        const float mid = 0.5f * (a + c);
        const float disc = fmaxf(0.01f, mid * mid - det);
        const float lmax = mid + sqrtf(disc);
        const float r = ceilf(3.0f * sqrtf(lmax));
        float tx0 = floorf((px - r) / ftile), tx1 = ceilf((px + r) / ftile);
        float ty0 = floorf((py - r) / ftile), ty1 = ceilf((py + r) / ftile);
        tx0 = fminf(fmaxf(tx0, 0.0f), (float)tiles_x);
        tx1 = fminf(fmaxf(tx1, 0.0f), (float)tiles_x);
        ty0 = fminf(fmaxf(ty0, 0.0f), (float)tiles_y);
        ty1 = fminf(fmaxf(ty1, 0.0f), (float)tiles_y);
        if (!(tx0 < tx1 && ty0 < ty1)) continue;

        /* view-dependent colour */
        float dx = mx - campos[0], dy = my - campos[1], dz = mz - campos[2];
        float len = sqrtf(dx * dx + dy * dy + dz * dz);
        if (len > 0.0f) { dx = dx / len; dy = dy / len; dz = dz / len; }
        float Y[16];
        orc_sh_basis(dx, dy, dz, Y);
        float col[3];
        int colour_finite = 1;
        for (int ch = 0; ch < 3; ++ch) {
            float acc = Y[0] * sh[(i * ncoef + 0) * 3 + ch];
            for (int k = 1; k < ncoef; ++k) acc = acc + Y[k] * sh[(i * ncoef + k) * 3 + ch];
            colour_finite = colour_finite && isfinite(acc);
            col[ch] = fmaxf(acc + 0.5f, 0.0f);
        }
        if (!colour_finite) continue;
        for (int ch = 0; ch < 3; ++ch) rgb[3 * i + ch] = col[ch];

        mean2d[2 * i] = px;
        mean2d[2 * i + 1] = py;
        conic[3 * i] = ca;
        conic[3 * i + 1] = cb;
        conic[3 * i + 2] = cc;
        depth[i] = zc;
        radius[i] = (int32_t)r;
        rect[4 * i] = (int32_t)tx0;
        rect[4 * i + 1] = (int32_t)ty0;
        rect[4 * i + 2] = (int32_t)tx1;
        rect[4 * i + 3] = (int32_t)ty1;
        visible[i] = 1;
    }
}

/* ------------------------------------------------------------------------ */
/* Tile intersection and the baseline tile lists (Sec. 3.1).                 */
/* ------------------------------------------------------------------------ */

int64_t orc_count_entries(int64_t n, const int32_t* rect)
{
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i)
        m += (int64_t)(rect[4 * i + 2] - rect[4 * i]) * (int64_t)(rect[4 * i + 3] - rect[4 * i + 1]);
    return m;
}

/* One entry per (Gaussian, covered tile), in emission order: gid ascending,
 * then tile rows ty ascending, then tx ascending.  zbits = float bits of the
 * depth (positive, so bit order is numeric order). */
void orc_emit(int64_t n, const int32_t* rect, const float* depth, int tiles_x,
              uint32_t* tile, uint32_t* zbits, uint32_t* gid)
{
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int ty = rect[4 * i + 1]; ty < rect[4 * i + 3]; ++ty)
            for (int tx = rect[4 * i]; tx < rect[4 * i + 2]; ++tx) {
                tile[m] = (uint32_t)(ty * tiles_x + tx);
                zbits[m] = bits_of(depth[i]);
                gid[m] = (uint32_t)i;
                ++m;
            }
}

typedef struct { uint32_t tile, zbits, gid; } orc_entry;

static int cmp_entry(const void* pa, const void* pb)
{
    const orc_entry* a = (const orc_entry*)pa;
    const orc_entry* b = (const orc_entry*)pb;
    if (a->tile != b->tile) return a->tile < b->tile ? -1 : 1;
    if (a->zbits != b->zbits) return a->zbits < b->zbits ? -1 : 1;
    if (a->gid != b->gid) return a->gid < b->gid ? -1 : 1;
    return 0;
}

/* Baseline order: every tile's entries contiguous, tiles ascending, and each
 * tile's list in (depth, gid) order.  offsets[T+1] bound tile t's span; the
 * stream word is (zbits << 32) | gid. */
void orc_sort_tiles(int64_t m, const uint32_t* tile, const uint32_t* zbits, const uint32_t* gid,
                    int32_t n_tiles, int32_t* offsets, uint64_t* stream)
{
    orc_entry* e = (orc_entry*)malloc((size_t)(m > 0 ? m : 1) * sizeof(orc_entry));
    for (int64_t k = 0; k < m; ++k) { e[k].tile = tile[k]; e[k].zbits = zbits[k]; e[k].gid = gid[k]; }
    qsort(e, (size_t)m, sizeof(orc_entry), cmp_entry);
    for (int32_t t = 0; t <= n_tiles; ++t) offsets[t] = 0;
    for (int64_t k = 0; k < m; ++k) offsets[e[k].tile + 1] += 1;
    for (int32_t t = 0; t < n_tiles; ++t) offsets[t + 1] += offsets[t];
    for (int64_t k = 0; k < m; ++k) stream[k] = ((uint64_t)e[k].zbits << 32) | e[k].gid;
    free(e);
}

/* ------------------------------------------------------------------------ */
/* Front-to-back compositing (Sec. 3.1; supplement, binned raster traversal: */
/* the binned raster keeps the baseline's per-pixel opacity/conic test).     */
/* ------------------------------------------------------------------------ */

/*
 * For every pixel of the listed tiles (all tiles when tiles_sel == NULL),
 * composite the tile's span [offsets[t*K], offsets[(t+1)*K]) of `stream`
 * front to back:
 *   d = mean2d - (x + 0.5, y + 0.5);
 *   q = fmaf(dx, fmaf(a/2, dx, b*dy), ((c/2)*dy)*dy)      (= 1/2 d^T conic d)
 *   skip unless q >= 0;  alpha = min(0.99, o * exp(-q));  skip if alpha < 1/255;
 *   Tn = T (1 - alpha); stop (without applying) if Tn < 1e-4;
 *   C = fmaf(col, alpha*T, C); T = Tn; last = gid of the applied entry.
 * out_rgb = fmaf(T, bg, C), out_alpha = 1 - T.  out_ntests (nullable) counts
 * the entries a pixel visits, the stopping one included.
 */
void orc_composite(const float* mean2d, const float* conic, const float* opac, const float* rgb,
                   const int32_t* offsets, int K, const uint64_t* stream,
                   int width, int height, int tile, const float* bg,
                   const int32_t* tiles_sel, int64_t n_sel,
                   float* out_rgb, float* out_alpha, int32_t* out_last, int32_t* out_ntests)
{
    const int tiles_x = (width + tile - 1) / tile;
    const int tiles_y = (height + tile - 1) / tile;
    const int64_t n_iter = tiles_sel ? n_sel : (int64_t)tiles_x * tiles_y;
    /* tiles are independent; the thread count changes nothing in the result */
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t it = 0; it < n_iter; ++it) {
        const int32_t t = tiles_sel ? tiles_sel[it] : (int32_t)it;
        const int tx = t % tiles_x, ty = t / tiles_x;
        const int32_t s0 = offsets[(int64_t)t * K], s1 = offsets[(int64_t)(t + 1) * K];
        for (int j = ty * tile; j < ty * tile + tile && j < height; ++j)
            for (int i = tx * tile; i < tx * tile + tile && i < width; ++i) {
                const float pxc = (float)i + 0.5f, pyc = (float)j + 0.5f;
                float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
                int32_t last = -1, ntests = 0;
                for (int32_t s = s0; s < s1; ++s) {
                    const uint32_t g = (uint32_t)(stream[s] & 0xffffffffu);
                    ntests += 1;
                    const float dx = mean2d[2 * g] - pxc;
                    const float dy = mean2d[2 * g + 1] - pyc;
                    const float ha = 0.5f * conic[3 * g], hb = conic[3 * g + 1], hc = 0.5f * conic[3 * g + 2];
                    const float q = fmaf(dx, fmaf(ha, dx, hb * dy), (hc * dy) * dy);
                    if (!(q >= 0.0f)) continue;
                    const float e = orc_expf(-q);
                    const float alpha = fminf(0.99f, opac[g] * e);
                    if (alpha < 1.0f / 255.0f) continue;
                    const float Tn = T * (1.0f - alpha);
                    if (Tn < 1e-4f) break;
                    const float wgt = alpha * T;
                    C0 = fmaf(rgb[3 * g], wgt, C0);
                    C1 = fmaf(rgb[3 * g + 1], wgt, C1);
                    C2 = fmaf(rgb[3 * g + 2], wgt, C2);
                    T = Tn;
                    last = (int32_t)g;
                }
                const int64_t p = (int64_t)j * width + i;
                out_rgb[3 * p] = fmaf(T, bg[0], C0);
                out_rgb[3 * p + 1] = fmaf(T, bg[1], C1);
                out_rgb[3 * p + 2] = fmaf(T, bg[2], C2);
                out_alpha[p] = 1.0f - T;
                out_last[p] = last;
                if (out_ntests) out_ntests[p] = ntests;
            }
    }
}

/* ------------------------------------------------------------------------ */
/* Robust depth range (supplement, algorithm "Robust depth-range estimation") */
/* ------------------------------------------------------------------------ */

/* Near-depth-shifted binning key of one Gaussian:
 * z_key = z - min(alpha * s_max, gamma * z), s_max = largest linear scale. */
float orc_zkey(float z, const float* s3, float near_alpha, float near_gamma)
{
    float smax = fmaxf(fmaxf(s3[0], s3[1]), s3[2]);
    return z - fminf(near_alpha * smax, near_gamma * z);
}

static int cmp_float(const void* pa, const void* pb)
{
    float a = *(const float*)pa, b = *(const float*)pb;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* k-th smallest (1-based) with the torch.kthvalue rank convention, the rank
 * being k = ceil(p/100 * n) clamped to [1, n], evaluated in double. */
static int64_t rank_of(double p, int64_t n)
{
    int64_t k = (int64_t)ceil(p / 100.0 * (double)n);
    if (k < 1) k = 1;
    if (k > n) k = n;
    return k;
}

/*
 * Samples: S' = min(S, M) emitted entries, the i-th at index floor(i*M/S')
 * (integer arithmetic), each contributing the depth of its Gaussian; with the
 * near-depth shift on, each sample becomes z_key.  Samples with z_key <= 0 are
 * discarded, the rest clamped to [max(near, eps), far].  z_lo / z_hi are the
 * exact p_lo / p_hi order statistics; span = max(z_hi - z_lo, 1e-6);
 * zmin = max(near, z_lo - pad*span), zmax = min(far, z_hi + pad*span).
 * With no sample left: zmin = max(near, eps), zmax = far.
 * Returns the number of kept samples.
 */
int64_t orc_depth_range(int64_t m, const uint32_t* entry_gid, const float* depth, const float* scales,
                        float near_plane, float far_plane, int S, int near_shift,
                        float near_alpha, float near_gamma, float p_lo, float p_hi,
                        float pad, float eps, float* zrange)
{
    int64_t ns = m < (int64_t)S ? m : (int64_t)S;
    float* v = (float*)malloc((size_t)(ns > 0 ? ns : 1) * sizeof(float));
    const float lo_clamp = fmaxf(near_plane, eps);
    int64_t kept = 0;
    for (int64_t i = 0; i < ns; ++i) {
        int64_t j = (i * m) / ns; /* i < 8192 and m < 2^40: no overflow */
        uint32_t g = entry_gid[j];
        float z = depth[g];
        if (near_shift) z = orc_zkey(z, scales + 3 * (int64_t)g, near_alpha, near_gamma);
        if (!(z > 0.0f)) continue;
        z = fminf(fmaxf(z, lo_clamp), far_plane);
        v[kept++] = z;
    }
    if (kept == 0) {
        zrange[0] = lo_clamp;
        zrange[1] = far_plane;
        free(v);
        return 0;
    }
    qsort(v, (size_t)kept, sizeof(float), cmp_float);
    const float zlo = v[rank_of((double)p_lo, kept) - 1];
    const float zhi = v[rank_of((double)p_hi, kept) - 1];
    const float span = fmaxf(zhi - zlo, 1e-6f);
    zrange[0] = fmaxf(near_plane, zlo - pad * span);
    zrange[1] = fminf(far_plane, zhi + pad * span);
    free(v);
    return kept;
}

/* ------------------------------------------------------------------------ */
/* Depth-to-bin maps (supplement, the log-depth-bin formula).                 */
/* ------------------------------------------------------------------------ */

/* Shared set-up: z'min = max(zmin, eps), z'max = max(zmax, z'min + 1e-6),
 * lmin = ln z'min, lmax = ln z'max.  splits[k-1] for k = 1..K-1 are the
 * log-spaced depths exp(lmin + (lmax - lmin) * (k/K)) used by the monotone
 * map, as a running maximum. */
void orc_bin_params(float zmin, float zmax, int K, float eps, float* lmin_out, float* lmax_out,
                    float* splits)
{
    const float zmn = fmaxf(zmin, eps);
    const float zmx = fmaxf(zmax, zmn + 1e-6f);
    const float lmin = orc_logf(zmn), lmax = orc_logf(zmx);
    *lmin_out = lmin;
    *lmax_out = lmax;
    for (int k = 1; k < K; ++k) {
        const float t = (float)k / (float)K;
        splits[k - 1] = orc_expf(lmin + (lmax - lmin) * t);
    }
    /* keep the list non-decreasing (a no-op unless exp rounding ever broke
     * monotonicity), so "number of splits <= z" is also a binary search */
    for (int k = 1; k < K - 1; ++k)
        if (splits[k] < splits[k - 1]) splits[k] = splits[k - 1];
}

/* The paper's map: u = clamp((ln max(z, eps) - lmin) / (lmax - lmin), 0,
 * 1 - 1e-6); b = clamp(floor(K u), 0, K - 1). */
int orc_bin_log(float z, float lmin, float lmax, int K, float eps)
{
    float u = (orc_logf(fmaxf(z, eps)) - lmin) / (lmax - lmin);
    u = fminf(fmaxf(u, 0.0f), 1.0f - 1e-6f);
    int b = (int)floorf((float)K * u);
    if (b < 0) b = 0;
    if (b > K - 1) b = K - 1;
    return b;
}

/* Monotone map: the number of split depths <= z.  Non-decreasing in z for any
 * split set, so bin order never inverts depth order. */
int orc_bin_split(float z, const float* splits, int K)
{
    int b = 0;
    for (int k = 0; k < K - 1; ++k)
        if (splits[k] <= z) ++b;
    return b;
}

/*
 * Tile-local bin construction (supplement, "Tile-local bin construction"):
 * count[t, b] over the entries, exclusive scan over the T*K histogram in
 * tile-major / bin-minor order -> bin_offsets[T*K + 1], scatter each entry's
 * word (zbits << 32 | gid) into its (t, b) segment.  This oracle scatters in
 * emission order (a stable counting sort); the paper's atomic scatter leaves
 * any order inside a segment, so only segment multisets are comparable.
 *   map_mode 0: monotone split map on the entry depth;
 *   map_mode 1: the paper's log map on the near-shifted key of the entry's
 *               Gaussian (zkey[gid], precomputed by the caller).
 */
void orc_bin_build(int64_t m, const uint32_t* tile, const uint32_t* zbits, const uint32_t* gid,
                   const float* zkey, int map_mode, float lmin, float lmax, const float* splits,
                   float eps, int32_t n_tiles, int K, int32_t* bin_offsets, uint64_t* stream)
{
    const int64_t nseg = (int64_t)n_tiles * K;
    int32_t* bins = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    int64_t* cursor = (int64_t*)calloc((size_t)nseg + 1, sizeof(int64_t));
    for (int64_t s = 0; s <= nseg; ++s) bin_offsets[s] = 0;
    for (int64_t k = 0; k < m; ++k) {
        int b;
        if (map_mode == 0) b = orc_bin_split(f_from_bits(zbits[k]), splits, K);
        else b = orc_bin_log(zkey[gid[k]], lmin, lmax, K, eps);
        bins[k] = b;
        bin_offsets[(int64_t)tile[k] * K + b + 1] += 1;
    }
    for (int64_t s = 0; s < nseg; ++s) bin_offsets[s + 1] += bin_offsets[s];
    for (int64_t s = 0; s < nseg; ++s) cursor[s] = bin_offsets[s];
    for (int64_t k = 0; k < m; ++k) {
        int64_t seg = (int64_t)tile[k] * K + bins[k];
        stream[cursor[seg]++] = ((uint64_t)zbits[k] << 32) | gid[k];
    }
    free(bins);
    free(cursor);
}

/* ------------------------------------------------------------------------ */
/* Selective repair (Sec. 3.5; supplement, "Selective repair selection and    */
/* local exact sorting"; thresholds from the default repair-threshold table). */
/* ------------------------------------------------------------------------ */

/*
 * Visit segments q = t*K + b in order.  Skip l <= 1.  keep if any of
 *   (i) l >= 320, (ii) l > 512, (iii) l / l_tile >= 45 %,
 *   (iv) 129 <= l <= 256 and l / l_tile >= 10 %, (v) b < 2 and l >= 16;
 * share tests in exact integer form (100 l >= 45 l_tile).  A kept segment is
 * selected when used + l <= B (B = floor(budget_frac * M), in double), and
 * then used += l; a segment that would overflow is skipped and later ones are
 * still considered.  Writes selected[q] in {0,1}; returns used.
 */
int64_t orc_repair_select(int32_t n_tiles, int K, const int32_t* bin_offsets, int64_t m,
                          double budget_frac, uint8_t* selected)
{
    const int64_t B = (int64_t)floor(budget_frac * (double)m);
    int64_t used = 0;
    for (int32_t t = 0; t < n_tiles; ++t) {
        const int64_t ltile = (int64_t)bin_offsets[(int64_t)(t + 1) * K] - bin_offsets[(int64_t)t * K];
        for (int b = 0; b < K; ++b) {
            const int64_t q = (int64_t)t * K + b;
            selected[q] = 0;
            const int64_t l = (int64_t)bin_offsets[q + 1] - bin_offsets[q];
            if (l <= 1) continue;
            int keep = 0;
            if (l >= 320) keep = 1;
            if (l > 512) keep = 1;
            if (100 * l >= 45 * ltile) keep = 1;
            if (l >= 129 && l <= 256 && 100 * l >= 10 * ltile) keep = 1;
            if (b < 2 && l >= 16) keep = 1;
            if (keep && used + l <= B) {
                selected[q] = 1;
                used += l;
            }
        }
    }
    return used;
}

static int cmp_u64(const void* pa, const void* pb)
{
    uint64_t a = *(const uint64_t*)pa, b = *(const uint64_t*)pb;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* Sort segments by the baseline key: selected[q] != 0, or every segment when
 * selected == NULL.  The word (zbits << 32 | gid) orders by depth then gid. */
void orc_sort_segments(int64_t nseg, const int32_t* bin_offsets, const uint8_t* selected,
                       uint64_t* stream)
{
    for (int64_t q = 0; q < nseg; ++q) {
        if (selected && !selected[q]) continue;
        const int64_t l = (int64_t)bin_offsets[q + 1] - bin_offsets[q];
        if (l > 1) qsort(stream + bin_offsets[q], (size_t)l, sizeof(uint64_t), cmp_u64);
    }
}

/* ------------------------------------------------------------------------ */
/* fp64 twin of the projection and the compositing (for pins only).          */
/* ------------------------------------------------------------------------ */

/* Same reading as orc_project, in double with libm; returns mean2d, conic,
 * depth, radius (double), rgb.  No culling beyond near/far and det > 0. */
void orc64_project(int64_t n, const float* means, const float* scales, const float* quats,
                   const float* sh, int sh_degree, const float* Wf,
                   double fx, double fy, double cx, double cy, int width, int height,
                   double* mean2d, double* conic, double* depth, double* radius, double* rgb,
                   uint8_t* ok)
{
    double W[16];
    for (int k = 0; k < 16; ++k) W[k] = Wf[k];
    const int ncoef = (sh_degree + 1) * (sh_degree + 1);
    double campos[3];
    for (int j = 0; j < 3; ++j)
        campos[j] = -(W[0 * 4 + j] * W[3] + W[1 * 4 + j] * W[7] + W[2 * 4 + j] * W[11]);
    const double limx_hi = 1.3 * ((width - cx) / fx), limx_lo = 1.3 * (cx / fx);
    const double limy_hi = 1.3 * ((height - cy) / fy), limy_lo = 1.3 * (cy / fy);
    for (int64_t i = 0; i < n; ++i) {
        ok[i] = 0;
        const double mx = means[3 * i], my = means[3 * i + 1], mz = means[3 * i + 2];
        const double xc = W[0] * mx + W[1] * my + W[2] * mz + W[3];
        const double yc = W[4] * mx + W[5] * my + W[6] * mz + W[7];
        const double zc = W[8] * mx + W[9] * my + W[10] * mz + W[11];
        if (!(zc > 0.01)) continue;
        double qw = quats[4 * i], qx = quats[4 * i + 1], qy = quats[4 * i + 2], qz = quats[4 * i + 3];
        double qn = sqrt(qw * qw + qx * qx + qy * qy + qz * qz);
        double w = qw / qn, x = qx / qn, y = qy / qn, z = qz / qn;
        double Rq[3][3] = {
            {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
            {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
            {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
        double M[3][3], S[3][3], Tm[3][3], Sc[3][3];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) M[r][c] = Rq[r][c] * (double)scales[3 * i + c];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) S[r][c] = M[r][0] * M[c][0] + M[r][1] * M[c][1] + M[r][2] * M[c][2];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                Tm[r][c] = W[r * 4] * S[0][c] + W[r * 4 + 1] * S[1][c] + W[r * 4 + 2] * S[2][c];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                Sc[r][c] = Tm[r][0] * W[c * 4] + Tm[r][1] * W[c * 4 + 1] + Tm[r][2] * W[c * 4 + 2];
        double u = xc / zc, v = yc / zc;
        u = fmin(fmax(u, -limx_lo), limx_hi);
        v = fmin(fmax(v, -limy_lo), limy_hi);
        const double j00 = fx / zc, j02 = -fx * u / zc, j11 = fy / zc, j12 = -fy * v / zc;
        double a = j00 * j00 * Sc[0][0] + 2 * j00 * j02 * Sc[0][2] + j02 * j02 * Sc[2][2] + 0.3;
        double b = j00 * j11 * Sc[0][1] + j00 * j12 * Sc[0][2] + j02 * j11 * Sc[2][1] + j02 * j12 * Sc[2][2];
        double c = j11 * j11 * Sc[1][1] + 2 * j11 * j12 * Sc[1][2] + j12 * j12 * Sc[2][2] + 0.3;
        const double det = a * c - b * b;
        if (!(det > 0)) continue;
        conic[3 * i] = c / det;
        conic[3 * i + 1] = -b / det;
        conic[3 * i + 2] = a / det;
        mean2d[2 * i] = fx * xc / zc + cx;
        mean2d[2 * i + 1] = fy * yc / zc + cy;
        depth[i] = zc;
        const double mid = 0.5 * (a + c);
        radius[i] = ceil(3.0 * sqrt(mid + sqrt(fmax(0.01, mid * mid - det))));
        double dx = mx - campos[0], dy = my - campos[1], dz = mz - campos[2];
        double len = sqrt(dx * dx + dy * dy + dz * dz);
        dx /= len; dy /= len; dz /= len;
        double xx = dx * dx, yy = dy * dy, zz = dz * dz;
        double Y[16] = {0.28209479177387814,
                        -0.4886025119029199 * dy, 0.4886025119029199 * dz, -0.4886025119029199 * dx,
                        1.0925484305920792 * dx * dy, -1.0925484305920792 * dy * dz,
                        0.31539156525252005 * (2 * zz - xx - yy), -1.0925484305920792 * dx * dz,
                        0.5462742152960396 * (xx - yy),
                        -0.5900435899266435 * dy * (3 * xx - yy), 2.890611442640554 * dx * dy * dz,
                        -0.4570457994644658 * dy * (4 * zz - xx - yy),
                        0.3731763325901154 * dz * (2 * zz - 3 * xx - 3 * yy),
                        -0.4570457994644658 * dx * (4 * zz - xx - yy),
                        1.445305721320277 * dz * (xx - yy), -0.5900435899266435 * dx * (xx - 3 * yy)};
        for (int ch = 0; ch < 3; ++ch) {
            double acc = 0;
            for (int k = 0; k < ncoef; ++k) acc += Y[k] * sh[(i * ncoef + k) * 3 + ch];
            rgb[3 * i + ch] = fmax(acc + 0.5, 0.0);
        }
        ok[i] = 1;
    }
}

/* fp64 compositing of one pixel centre over an explicit ordered gid list,
 * with libm exp and the same thresholds.  Returns T; writes C[3]. */
double orc64_composite_pixel(double pxc, double pyc, const double* mean2d, const double* conic,
                             const float* opac, const double* rgb, const uint32_t* gids, int64_t n,
                             double* C)
{
    double T = 1.0;
    C[0] = C[1] = C[2] = 0.0;
    for (int64_t s = 0; s < n; ++s) {
        const uint32_t g = gids[s];
        const double dx = mean2d[2 * g] - pxc, dy = mean2d[2 * g + 1] - pyc;
        const double q = 0.5 * (conic[3 * g] * dx * dx + conic[3 * g + 2] * dy * dy) + conic[3 * g + 1] * dx * dy;
        if (q < 0) continue;
        const double alpha = fmin(0.99, opac[g] * exp(-q));
        if (alpha < 1.0 / 255.0) continue;
        const double Tn = T * (1.0 - alpha);
        if (Tn < 1e-4) break;
        for (int ch = 0; ch < 3; ++ch) C[ch] += rgb[3 * g + ch] * alpha * T;
        T = Tn;
    }
    return T;
}

/* Threads used by the compositing loop (1 = serial). */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Backward of the compositing (gradient of the image w.r.t. the projected    */
/* 2D parameters).  The paper leaves the backward to future work (Sec. 7):    */
/* it has to follow the order the forward composites in.                      */
/* ------------------------------------------------------------------------ */

/*
 * For every pixel of every tile: replay the forward over the tile's span of
 * `stream` with its float32 decisions (which entries are skipped, where the
 * pixel stops, whether alpha is clamped -- exactly orc_composite's), then
 * accumulate in double the derivatives of
 *   out_rgb = sum_i c_i a_i T_i + T_N bg,  out_alpha = 1 - T_N,
 *   a_i = min(0.99, o_i exp(-q_i)),  q_i = 1/2 (a dx^2 + 2 b dx dy + c dy^2),
 *   T_{i+1} = T_i (1 - a_i),  d = mean - pixel centre,
 * w.r.t. mean2d, conic (a, b, c), opacity and rgb, weighted by dl_drgb [H,W,3]
 * and dl_dalpha [H,W] (nullable), over the pixels of the listed tiles
 * (tiles_sel[n_sel], each listed once; all tiles when NULL -- the same as a
 * zero incoming gradient elsewhere).  A clamped alpha (o exp(-q) > 0.99 in
 * float32) passes no gradient to o or q.  Gradients are added into
 * g_mean2d [n,2], g_conic [n,3], g_opac [n], g_rgb [n,3] (double,
 * caller-zeroed); g_abs [n,9] (nullable) receives, in the order
 * (mx, my, a, b, c, o, r, g, b), the error scale of a float32 evaluation:
 * the sums over pixels of each term's magnitude with dL/da replaced by
 * |G.c| T_i + (|G|.S_i + |dA| T_N) / (1 - a_i) -- the magnitudes of the two
 * parts dL/da is the difference of (|G| and S taken per channel, S the
 * colour behind the entry, background included).
 * at_f32 = 0: every value in double from the float32 inputs (the derivative
 * of the exact compositing, pinned by finite differences).  at_f32 = 1: the
 * same formulas, in double, at the float32 forward's own exp(-q), alpha and
 * transmittances (recorded by the replay): the gradient of the image the
 * float32 forward produced, without the forward's own rounding drift.
 */
void orc_composite_grad(const float* mean2d, const float* conic, const float* opac, const float* rgb,
                        const int32_t* offsets, int K, const uint64_t* stream, int width, int height,
                        int tile, const float* bg, const float* dl_drgb, const float* dl_dalpha,
                        const int32_t* tiles_sel, int64_t n_sel, int at_f32,
                        double* g_mean2d, double* g_conic, double* g_opac, double* g_rgb, double* g_abs)
{
    const int tiles_x = (width + tile - 1) / tile;
    const int tiles_y = (height + tile - 1) / tile;
    const int64_t nt = tiles_sel ? n_sel : (int64_t)tiles_x * tiles_y;
    int32_t* applied = NULL;
    unsigned char* clamped = NULL;
    float *ap_e = NULL, *ap_a = NULL, *ap_T = NULL; /* the float32 forward's exp(-q), alpha, T before */
    int64_t cap = 0;
    for (int64_t it = 0; it < nt; ++it) {
        const int32_t t = tiles_sel ? tiles_sel[it] : (int32_t)it;
        const int tx = t % tiles_x, ty = t / tiles_x;
        const int32_t s0 = offsets[(int64_t)t * K], s1 = offsets[(int64_t)(t + 1) * K];
        if (s1 - s0 > cap) {
            cap = s1 - s0;
            applied = (int32_t*)realloc(applied, (size_t)cap * sizeof(int32_t));
            clamped = (unsigned char*)realloc(clamped, (size_t)cap);
            ap_e = (float*)realloc(ap_e, (size_t)cap * sizeof(float));
            ap_a = (float*)realloc(ap_a, (size_t)cap * sizeof(float));
            ap_T = (float*)realloc(ap_T, (size_t)cap * sizeof(float));
        }
        for (int j = ty * tile; j < ty * tile + tile && j < height; ++j)
            for (int i = tx * tile; i < tx * tile + tile && i < width; ++i) {
                const float pxc = (float)i + 0.5f, pyc = (float)j + 0.5f;
                /* pass 1: the forward's float32 decisions */
                float T = 1.0f;
                int64_t na = 0;
                for (int32_t s = s0; s < s1; ++s) {
                    const uint32_t g = (uint32_t)(stream[s] & 0xffffffffu);
                    const float dx = mean2d[2 * g] - pxc, dy = mean2d[2 * g + 1] - pyc;
                    const float ha = 0.5f * conic[3 * g], hb = conic[3 * g + 1], hc = 0.5f * conic[3 * g + 2];
                    const float q = fmaf(dx, fmaf(ha, dx, hb * dy), (hc * dy) * dy);
                    if (!(q >= 0.0f)) continue;
                    const float e = orc_expf(-q);
                    const float oe = opac[g] * e;
                    const float alpha = fminf(0.99f, oe);
                    if (alpha < 1.0f / 255.0f) continue;
                    const float Tn = T * (1.0f - alpha);
                    if (Tn < 1e-4f) break;
                    clamped[na] = oe > 0.99f;
                    ap_e[na] = e;
                    ap_a[na] = alpha;
                    ap_T[na] = T;
                    T = Tn;
                    applied[na++] = (int32_t)g;
                }
                /* pass 2: double-precision values and derivatives over the applied list */
                const int64_t p = (int64_t)j * width + i;
                const double px = (double)i + 0.5, py = (double)j + 0.5;
                double Tf = 1.0;
                if (at_f32) {
                    Tf = T;
                } else {
                    for (int64_t k = 0; k < na; ++k) {
                        const int32_t g = applied[k];
                        const double dx = mean2d[2 * g] - px, dy = mean2d[2 * g + 1] - py;
                        const double q = 0.5 * (conic[3 * g] * dx * dx + conic[3 * g + 2] * dy * dy) + conic[3 * g + 1] * dx * dy;
                        const double a = clamped[k] ? 0.99 : opac[g] * exp(-q);
                        Tf *= 1.0 - a;
                    }
                }
                const double dA = dl_dalpha ? dl_dalpha[p] : 0.0;
                /* back to front: S = colour composited behind the entry (incl. background) */
                double S[3] = {Tf * bg[0], Tf * bg[1], Tf * bg[2]};
                double Tb = Tf; /* transmittance after the entry */
                double Gabs[3], dCmag = 0.0;
                for (int ch = 0; ch < 3; ++ch) Gabs[ch] = fabs((double)dl_drgb[3 * p + ch]);
                for (int64_t k = na - 1; k >= 0; --k) {
                    const int32_t g = applied[k];
                    const double dx = mean2d[2 * g] - px, dy = mean2d[2 * g + 1] - py;
                    const double ca = conic[3 * g], cb = conic[3 * g + 1], cc = conic[3 * g + 2];
                    const double q = 0.5 * (ca * dx * dx + cc * dy * dy) + cb * dx * dy;
                    const double G = at_f32 ? (double)ap_e[k] : exp(-q);
                    const double a = at_f32 ? (double)ap_a[k] : clamped[k] ? 0.99 : opac[g] * G;
                    /* transmittance before the entry */
                    const double Ti = at_f32 ? (double)ap_T[k] : Tb / (1.0 - a);
                    double dl_da = dA * Tf / (1.0 - a);
                    double term[9], absdl = fabs(dA) * Tf;
                    dCmag = 0.0;
                    for (int ch = 0; ch < 3; ++ch) {
                        const double dC = dl_drgb[3 * p + ch];
                        term[6 + ch] = dC * a * Ti;
                        dl_da += dC * (rgb[3 * g + ch] * Ti - S[ch] / (1.0 - a));
                        dCmag += Gabs[ch] * fabs((double)rgb[3 * g + ch]);
                        absdl += Gabs[ch] * fabs(S[ch]);
                    }
                    absdl = dCmag * Ti + absdl / (1.0 - a);
                    /* dL/dq = -dL/da o G; q's partials w.r.t. (mx, my, a, b, c) */
                    const double dq[5] = {ca * dx + cb * dy, cb * dx + cc * dy, 0.5 * dx * dx, dx * dy, 0.5 * dy * dy};
                    double mag[9];
                    for (int v = 0; v < 5; ++v) {
                        term[v] = clamped[k] ? 0.0 : -dl_da * opac[g] * G * dq[v];
                        mag[v] = clamped[k] ? 0.0 : absdl * opac[g] * G * fabs(dq[v]);
                    }
                    term[5] = clamped[k] ? 0.0 : dl_da * G;
                    mag[5] = clamped[k] ? 0.0 : absdl * G;
                    for (int v = 6; v < 9; ++v) mag[v] = fabs(term[v]);
                    g_mean2d[2 * (int64_t)g] += term[0];
                    g_mean2d[2 * (int64_t)g + 1] += term[1];
                    for (int v = 0; v < 3; ++v) g_conic[3 * (int64_t)g + v] += term[2 + v];
                    g_opac[g] += term[5];
                    for (int v = 0; v < 3; ++v) g_rgb[3 * (int64_t)g + v] += term[6 + v];
                    if (g_abs)
                        for (int v = 0; v < 9; ++v) g_abs[9 * (int64_t)g + v] += mag[v];
                    for (int ch = 0; ch < 3; ++ch) S[ch] += rgb[3 * g + ch] * a * Ti;
                    Tb = Ti;
                }
            }
    }
    free(applied);
    free(clamped);
    free(ap_e);
    free(ap_a);
    free(ap_T);
}

/*
 * The double-precision forward over frozen per-pixel lists: applied_off
 * [P+1] / applied [..] give, per pixel (row-major), the gids the forward
 * applied, in order.  No threshold decision is taken, so the map from the 2D
 * parameters to (out_rgb, out_alpha) is smooth and central finite differences
 * of it check orc_composite_grad.
 */
void orc64_composite_frozen(const double* mean2d, const double* conic, const double* opac, const double* rgb,
                            const int64_t* applied_off, const int32_t* applied, int width, int height,
                            const double* bg, double* out_rgb, double* out_alpha)
{
    for (int j = 0; j < height; ++j)
        for (int i = 0; i < width; ++i) {
            const int64_t p = (int64_t)j * width + i;
            const double px = (double)i + 0.5, py = (double)j + 0.5;
            double T = 1.0, C[3] = {0.0, 0.0, 0.0};
            for (int64_t k = applied_off[p]; k < applied_off[p + 1]; ++k) {
                const int32_t g = applied[k];
                const double dx = mean2d[2 * g] - px, dy = mean2d[2 * g + 1] - py;
                const double q = 0.5 * (conic[3 * g] * dx * dx + conic[3 * g + 2] * dy * dy) + conic[3 * g + 1] * dx * dy;
                const double a = fmin(0.99, opac[g] * exp(-q));
                for (int ch = 0; ch < 3; ++ch) C[ch] += rgb[3 * g + ch] * a * T;
                T *= 1.0 - a;
            }
            for (int ch = 0; ch < 3; ++ch) out_rgb[3 * p + ch] = C[ch] + T * bg[ch];
            out_alpha[p] = 1.0 - T;
        }
}

/* The applied lists of the float32 forward (for the frozen forward above):
 * returns the total count; writes applied_off [P+1] and applied (capacity cap). */
int64_t orc_applied_lists(const float* mean2d, const float* conic, const float* opac, const int32_t* offsets,
                          int K, const uint64_t* stream, int width, int height, int tile,
                          int64_t* applied_off, int32_t* applied, int64_t cap)
{
    const int tiles_x = (width + tile - 1) / tile;
    int64_t na = 0;
    for (int j = 0; j < height; ++j)
        for (int i = 0; i < width; ++i) {
            const int64_t p = (int64_t)j * width + i;
            applied_off[p] = na;
            const int32_t t = (j / tile) * tiles_x + (i / tile);
            const int32_t s0 = offsets[(int64_t)t * K], s1 = offsets[(int64_t)(t + 1) * K];
            const float pxc = (float)i + 0.5f, pyc = (float)j + 0.5f;
            float T = 1.0f;
            for (int32_t s = s0; s < s1; ++s) {
                const uint32_t g = (uint32_t)(stream[s] & 0xffffffffu);
                const float dx = mean2d[2 * g] - pxc, dy = mean2d[2 * g + 1] - pyc;
                const float ha = 0.5f * conic[3 * g], hb = conic[3 * g + 1], hc = 0.5f * conic[3 * g + 2];
                const float q = fmaf(dx, fmaf(ha, dx, hb * dy), (hc * dy) * dy);
                if (!(q >= 0.0f)) continue;
                const float alpha = fminf(0.99f, opac[g] * orc_expf(-q));
                if (alpha < 1.0f / 255.0f) continue;
                const float Tn = T * (1.0f - alpha);
                if (Tn < 1e-4f) break;
                T = Tn;
                if (na < cap) applied[na] = (int32_t)g;
                ++na;
            }
        }
    applied_off[(int64_t)width * height] = na;
    return na;
}
