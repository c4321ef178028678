/*
 * gs_oracle.c -- plain, slow CPU oracle for one 3D Gaussian Splatting
 * training step (VkSplat, arxiv 2605.00219).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code:
 * only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * arm load it.  It shares no code, header or constant table with the CUDA
 * library; both sides are written independently from the paper and from the
 * written readings of it.
 *
 * Two parts:
 *   1. FP32 binning (bit-specified): projection quantities needed for tile
 *      culling, the scan-line tile culling of Sec. 4.1 / Fig. 1, the 32-bit
 *      (tile, depth) keys of Sec. 4.4, a stable sort and the tile ranges.
 *      Every floating-point operation is one IEEE binary32 operation rounded
 *      to nearest, in the order written; the file is compiled with
 *      -ffp-contract=off so no multiply-add is fused.  No library
 *      transcendental function appears (scales are stored activated,
 *      Sec. 4.3); the one logarithm, of the opacity-aware cull radius, is a
 *      fixed series written out below.
 *   2. FP64 reference of what the step computes (Sec. 2 "Related works",
 *      Sec. 4.2, Sec. 4.3): EWA projection with the 0.3 low-pass and degree-3
 *      SH colour, front-to-back compositing over the tile lists, the analytic
 *      backward of compositing and projection, and Adam in log-scale /
 *      logit-opacity space.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PSTRIDE 24     /* doubles per projected Gaussian record */
#define ORC_NTHETA 59      /* optimised scalars per Gaussian */

typedef struct {
    float R[9];            /* world -> camera rotation, row-major */
    float t[3];            /* world -> camera translation */
    float fx, fy, cx, cy;  /* pinhole intrinsics, pixels */
    int32_t width, height; /* image size, pixels */
    int32_t tile_w, tile_h;/* tile size, pixels */
} orc_cam;

/* ------------------------------------------------------------------------- */
/* Part 1: FP32 bit-specified binning                                        */
/* ------------------------------------------------------------------------- */

/* Natural logarithm in FP32 as a fixed sequence of rounded operations
 * (argument reduction x = 2^e m, m in [sqrt(1/2), sqrt(2)), then
 * ln m = 2 atanh(s) with s = (m - 1) / (m + 1) by the odd Taylor series of
 * atanh to s^9; |s| <= 0.1716 leaves a truncation error below 1e-9).  For
 * finite normal x > 0 only; the absolute error is about 2e-7 over [1, 256]. */
float orc_log32(float x)
{
    uint32_t u;
    memcpy(&u, &x, 4);
    int e = (int)(u >> 23) - 127;
    u = (u & 0x7FFFFFu) | 0x3F800000u;
    float m;
    memcpy(&m, &u, 4);
    if (m > 1.41421356f) {
        m = 0.5f * m;
        e += 1;
    }
    float s = (m - 1.0f) / (m + 1.0f);
    float s2 = s * s;
    float p = s2 * 0.111111111f + 0.142857143f;
    p = s2 * p + 0.2f;
    p = s2 * p + 0.333333333f;
    p = s2 * p + 1.0f;
    return (float)e * 0.693147181f + (2.0f * s) * p;
}

/* r^2 of the culling ellipse for opacity o (Sec. 4.1): a pixel takes part
 * only if d^2 <= 9 and o exp(-d^2 / 2) >= 1/255, i.e. d^2 <= min(9,
 * 2 ln(255 o)); widened by 2^-10 relative and 2^-10 absolute so that the FP32
 * culling stays conservative against the raster's own tests.  Returns a
 * negative value when 255 o <= 1 (alpha never reaches 1/255). */
float orc_cull_r2(float o)
{
    float x = 255.0f * o;
    if (!(x > 1.0f)) return -1.0f;
    float r = fminf(9.0f, 2.0f * orc_log32(x));
    return r * 1.0009765625f + 0.0009765625f;
}

typedef struct {
    int valid;
    float mx, my;          /* pixel-space mean */
    float a, b, c;         /* 2D covariance incl. low-pass */
    float det;
    float tz;
    float r2;              /* cull radius^2 (orc_cull_r2) */
    uint32_t mant;         /* 23-bit depth code */
} orc_bin;

static int orc_ceil_log2(int64_t n)
{
    int b = 0;
    while (((int64_t)1 << b) < n) b++;
    return b;
}

static int orc_tiles_x(const orc_cam* c) { return (c->width + c->tile_w - 1) / c->tile_w; }
static int orc_tiles_y(const orc_cam* c) { return (c->height + c->tile_h - 1) / c->tile_h; }

/* Steps B1-B14 of the binning specification. */
static void orc_bin_project(const float* mu, const float* q, const float* s, float op,
                            const orc_cam* cam, orc_bin* o)
{
    o->valid = 0;
    float r2 = orc_cull_r2(op);
    if (!(r2 > 0.0f)) return;
    float n2 = ((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3];
    if (!(n2 > 0.0f)) return;
    float r = sqrtf(n2);
    float w = q[0] / r, x = q[1] / r, y = q[2] / r, z = q[3] / r;
    float xx = x * x, yy = y * y, zz = z * z;
    float xy = x * y, xz = x * z, yz = y * z;
    float wx = w * x, wy = w * y, wz = w * z;
    float R[9];
    R[0] = 1.0f - 2.0f * (yy + zz); R[1] = 2.0f * (xy - wz);        R[2] = 2.0f * (xz + wy);
    R[3] = 2.0f * (xy + wz);        R[4] = 1.0f - 2.0f * (xx + zz); R[5] = 2.0f * (yz - wx);
    R[6] = 2.0f * (xz - wy);        R[7] = 2.0f * (yz + wx);        R[8] = 1.0f - 2.0f * (xx + yy);
    float M[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) M[3 * i + j] = R[3 * i + j] * s[j];
    float S[9];
    for (int i = 0; i < 3; i++)
        for (int j = i; j < 3; j++) {
            float v = (M[3 * i + 0] * M[3 * j + 0] + M[3 * i + 1] * M[3 * j + 1]) + M[3 * i + 2] * M[3 * j + 2];
            S[3 * i + j] = v;
            S[3 * j + i] = v;
        }
    const float* C = cam->R;
    float t[3];
    for (int i = 0; i < 3; i++)
        t[i] = ((C[3 * i + 0] * mu[0] + C[3 * i + 1] * mu[1]) + C[3 * i + 2] * mu[2]) + cam->t[i];
    if (!(t[2] >= 0.01f)) return;
    float limx = 1.3f * ((0.5f * (float)cam->width) / cam->fx);
    float limy = 1.3f * ((0.5f * (float)cam->height) / cam->fy);
    float ux = t[0] / t[2], uy = t[1] / t[2];
    ux = fminf(fmaxf(ux, -limx), limx);
    uy = fminf(fmaxf(uy, -limy), limy);
    float j00 = cam->fx / t[2], j11 = cam->fy / t[2];
    float j02 = -((cam->fx * ux) / t[2]);
    float j12 = -((cam->fy * uy) / t[2]);
    float T[6];
    for (int k = 0; k < 3; k++) {
        T[k] = j00 * C[k] + j02 * C[6 + k];
        T[3 + k] = j11 * C[3 + k] + j12 * C[6 + k];
    }
    float U[6];
    for (int i = 0; i < 2; i++)
        for (int k = 0; k < 3; k++)
            U[3 * i + k] = (T[3 * i + 0] * S[k] + T[3 * i + 1] * S[3 + k]) + T[3 * i + 2] * S[6 + k];
    float a = ((U[0] * T[0] + U[1] * T[1]) + U[2] * T[2]) + 0.3f;
    float b = (U[0] * T[3] + U[1] * T[4]) + U[2] * T[5];
    float c = ((U[3] * T[3] + U[4] * T[4]) + U[5] * T[5]) + 0.3f;
    float det = a * c - b * b;
    if (!(det > 0.0f)) return;
    float mx = (cam->fx * t[0]) / t[2] + cam->cx;
    float my = (cam->fy * t[1]) / t[2] + cam->cy;
    if (!(fabsf(mx) < 1e30f) || !(fabsf(my) < 1e30f) || !(a < 1e30f) || !(c < 1e30f) || !(det < 1e30f)) return;
    float qd = (2.0f * t[2] + 1.0f) / (t[2] + 1.0f);
    uint32_t bits;
    memcpy(&bits, &qd, 4);
    uint32_t mant = bits & 0x7FFFFFu;
    if (qd >= 2.0f) mant = 0x7FFFFFu;
    o->valid = 1;
    o->mx = mx; o->my = my; o->a = a; o->b = b; o->c = c; o->det = det;
    o->tz = t[2]; o->mant = mant; o->r2 = r2;
}

/* First tile whose pixel-centre hull reaches coordinate v from above, and the
 * last tile whose hull starts at or below v, clamped to the image. */
static int orc_tile_lo(float v, int T, int n)
{
    float f = ceilf((v + 0.5f - (float)T) / (float)T);
    f = fminf(fmaxf(f, -1.0f), (float)n);
    int i = (int)f;
    return i < 0 ? 0 : i;
}

static int orc_tile_hi(float v, int T, int n)
{
    float f = floorf((v - 0.5f) / (float)T);
    f = fminf(fmaxf(f, -1.0f), (float)n);
    int i = (int)f;
    return i > n - 1 ? n - 1 : i;
}

/* Scan-line tile culling (Sec. 4.1, Fig. 1).  Counts the tiles whose
 * pixel-centre rectangle meets the ellipse d^2 <= r2; when `tiles` is not
 * NULL the tile ids are written in traversal order.  Iterates over the
 * shorter tile dimension of the bounding box. */
static uint32_t orc_bin_scan(const orc_bin* g, const orc_cam* cam, uint32_t* tiles)
{
    if (!g->valid) return 0;
    int TW = orc_tiles_x(cam), TH = orc_tiles_y(cam);
    int tw = cam->tile_w, th = cam->tile_h;
    const float r2 = g->r2;
    float ex = sqrtf(r2 * g->a);
    float ey = sqrtf(r2 * g->c);
    int txl = orc_tile_lo(g->mx - ex, tw, TW), txh = orc_tile_hi(g->mx + ex, tw, TW);
    int tyl = orc_tile_lo(g->my - ey, th, TH), tyh = orc_tile_hi(g->my + ey, th, TH);
    if (txl > txh || tyl > tyh) return 0;
    uint32_t count = 0;
    if (tyh - tyl <= txh - txl) {
        /* rows: for each band of tile rows, the ellipse's x-range */
        float ystar = g->b * sqrtf(r2 / g->a);
        for (int ty = tyl; ty <= tyh; ty++) {
            float y0 = ((float)(ty * th) + 0.5f) - g->my;
            float y1 = ((float)((ty + 1) * th) - 0.5f) - g->my;
            float dlo = fmaxf(y0, -ey), dhi = fminf(y1, ey);
            if (!(dlo <= dhi)) continue;
            float dR = fminf(fmaxf(ystar, dlo), dhi);
            float dL = fminf(fmaxf(-ystar, dlo), dhi);
            float hR = sqrtf(fmaxf(0.0f, g->det * (r2 * g->c - dR * dR)));
            float hL = sqrtf(fmaxf(0.0f, g->det * (r2 * g->c - dL * dL)));
            float xR = g->mx + (g->b * dR + hR) / g->c;
            float xL = g->mx + (g->b * dL - hL) / g->c;
            int lo = orc_tile_lo(xL, tw, TW), hi = orc_tile_hi(xR, tw, TW);
            for (int tx = lo; tx <= hi; tx++) {
                if (tiles) tiles[count] = (uint32_t)(ty * TW + tx);
                count++;
            }
        }
    } else {
        /* columns: for each band of tile columns, the ellipse's y-range */
        float xstar = g->b * sqrtf(r2 / g->c);
        for (int tx = txl; tx <= txh; tx++) {
            float x0 = ((float)(tx * tw) + 0.5f) - g->mx;
            float x1 = ((float)((tx + 1) * tw) - 0.5f) - g->mx;
            float dlo = fmaxf(x0, -ex), dhi = fminf(x1, ex);
            if (!(dlo <= dhi)) continue;
            float dT = fminf(fmaxf(xstar, dlo), dhi);
            float dB = fminf(fmaxf(-xstar, dlo), dhi);
            float hT = sqrtf(fmaxf(0.0f, g->det * (r2 * g->a - dT * dT)));
            float hB = sqrtf(fmaxf(0.0f, g->det * (r2 * g->a - dB * dB)));
            float yT = g->my + (g->b * dT + hT) / g->a;
            float yB = g->my + (g->b * dB - hB) / g->a;
            int lo = orc_tile_lo(yB, th, TH), hi = orc_tile_hi(yT, th, TH);
            for (int ty = lo; ty <= hi; ty++) {
                if (tiles) tiles[count] = (uint32_t)(ty * TW + tx);
                count++;
            }
        }
    }
    return count;
}

/* 32-bit key of Sec. 4.4: tile id in the top ceil(log2(tiles)) bits, the high
 * bits of the depth code below it. */
static uint32_t orc_key(uint32_t tile, uint32_t mant, int tb)
{
    if (tb >= 9) return (tile << (32 - tb)) | (mant >> (tb - 9));
    return (tile << 23) | mant;
}

/* Per-Gaussian FP32 binning record and tile count.
 * out_bin: n x 8 floats (valid, mx, my, a, b, c, det, tz); out_mant: n. */
void orc_bin32_count(int64_t n, const float* means, const float* quats, const float* scales,
                     const float* opac, const orc_cam* cam, uint32_t* count, float* out_bin,
                     uint32_t* out_mant)
{
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < n; g++) {
        orc_bin b;
        orc_bin_project(means + 3 * g, quats + 4 * g, scales + 3 * g, opac[g], cam, &b);
        count[g] = orc_bin_scan(&b, cam, NULL);
        if (out_bin) {
            float* o = out_bin + 8 * g;
            o[0] = (float)b.valid; o[1] = b.mx; o[2] = b.my; o[3] = b.a; o[4] = b.b;
            o[5] = b.c; o[6] = b.det; o[7] = b.tz;
        }
        if (out_mant) out_mant[g] = b.valid ? b.mant : 0u;
    }
}

/* Emit (key, Gaussian) pairs in (Gaussian, traversal) order at the exclusive
 * offsets of the counts.  Returns the number of pairs. */
int64_t orc_bin32_emit(int64_t n, const float* means, const float* quats, const float* scales,
                       const float* opac, const orc_cam* cam, const int64_t* offset, uint32_t* keys,
                       uint32_t* gidx)
{
    int tb = orc_ceil_log2((int64_t)orc_tiles_x(cam) * orc_tiles_y(cam));
    int64_t total = 0;
#pragma omp parallel for schedule(static) reduction(+ : total)
    for (int64_t g = 0; g < n; g++) {
        orc_bin b;
        orc_bin_project(means + 3 * g, quats + 4 * g, scales + 3 * g, opac[g], cam, &b);
        uint32_t* tl = keys + offset[g];
        uint32_t cnt = orc_bin_scan(&b, cam, tl);
        for (uint32_t i = 0; i < cnt; i++) {
            tl[i] = orc_key(tl[i], b.mant, tb);
            gidx[offset[g] + i] = (uint32_t)g;
        }
        total += cnt;
    }
    return total;
}

/* Stable sort of (key, value) pairs by key: bottom-up merge sort. */
void orc_stable_sort(int64_t K, uint32_t* keys, uint32_t* vals)
{
    if (K < 2) return;
    uint32_t* tk = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)K);
    uint32_t* tv = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)K);
    uint32_t *sk = keys, *sv = vals, *dk = tk, *dv = tv;
    for (int64_t w = 1; w < K; w *= 2) {
        for (int64_t lo = 0; lo < K; lo += 2 * w) {
            int64_t mid = lo + w < K ? lo + w : K;
            int64_t hi = lo + 2 * w < K ? lo + 2 * w : K;
            int64_t i = lo, j = mid, o = lo;
            while (i < mid && j < hi) {
                if (sk[j] < sk[i]) { dk[o] = sk[j]; dv[o++] = sv[j++]; }
                else { dk[o] = sk[i]; dv[o++] = sv[i++]; }
            }
            while (i < mid) { dk[o] = sk[i]; dv[o++] = sv[i++]; }
            while (j < hi) { dk[o] = sk[j]; dv[o++] = sv[j++]; }
        }
        uint32_t* t;
        t = sk; sk = dk; dk = t;
        t = sv; sv = dv; dv = t;
    }
    if (sk != keys) {
        memcpy(keys, sk, sizeof(uint32_t) * (size_t)K);
        memcpy(vals, sv, sizeof(uint32_t) * (size_t)K);
    }
    free(tk);
    free(tv);
}

/* [start, end) of each tile in the sorted key list; tiles with no entry get
 * (0, 0). ranges: 2 x number of tiles. */
void orc_tile_ranges(int64_t K, const uint32_t* keys, const orc_cam* cam, int64_t* ranges)
{
    int64_t ntiles = (int64_t)orc_tiles_x(cam) * orc_tiles_y(cam);
    int tb = orc_ceil_log2(ntiles);
    int shift = tb >= 9 ? 32 - tb : 23;
    memset(ranges, 0, sizeof(int64_t) * 2 * (size_t)ntiles);
    for (int64_t k = 0; k < K; k++) {
        uint32_t tile = keys[k] >> shift;
        if (k == 0 || (keys[k - 1] >> shift) != tile) ranges[2 * tile] = k;
        if (k == K - 1 || (keys[k + 1] >> shift) != tile) ranges[2 * tile + 1] = k + 1;
    }
}

/* ------------------------------------------------------------------------- */
/* Part 2: FP64 reference                                                    */
/* ------------------------------------------------------------------------- */

/* Real spherical harmonics up to degree 3 in the sign convention of the 3DGS
 * family; constants are the orthonormalisation factors sqrt((2l+1)/(4pi) ...)
 * written out from their definitions. */
static void orc_sh_consts(double C[16])
{
    const double pi = 3.14159265358979323846;
    C[0] = 0.5 * sqrt(1.0 / pi);
    C[1] = -sqrt(3.0 / (4.0 * pi));
    C[2] = sqrt(3.0 / (4.0 * pi));
    C[3] = -sqrt(3.0 / (4.0 * pi));
    C[4] = sqrt(15.0 / (4.0 * pi));
    C[5] = -sqrt(15.0 / (4.0 * pi));
    C[6] = sqrt(5.0 / (16.0 * pi));
    C[7] = -sqrt(15.0 / (4.0 * pi));
    C[8] = sqrt(15.0 / (16.0 * pi));
    C[9] = -sqrt(35.0 / (32.0 * pi));
    C[10] = sqrt(105.0 / (4.0 * pi));
    C[11] = -sqrt(21.0 / (32.0 * pi));
    C[12] = sqrt(7.0 / (16.0 * pi));
    C[13] = -sqrt(21.0 / (32.0 * pi));
    C[14] = sqrt(105.0 / (16.0 * pi));
    C[15] = -sqrt(35.0 / (32.0 * pi));
}

/* Basis values Y[k] at a unit direction d, and (if dY != NULL) their partial
 * derivatives with respect to the three components of d (d treated as a free
 * 3-vector; the normalisation is differentiated by the caller). */
void orc_sh_basis(const double* d, double* Y, double* dY)
{
    double C[16];
    orc_sh_consts(C);
    double x = d[0], y = d[1], z = d[2];
    double P[16], dP[16][3];
    P[0] = 1;               dP[0][0] = 0;        dP[0][1] = 0;         dP[0][2] = 0;
    P[1] = y;               dP[1][0] = 0;        dP[1][1] = 1;         dP[1][2] = 0;
    P[2] = z;               dP[2][0] = 0;        dP[2][1] = 0;         dP[2][2] = 1;
    P[3] = x;               dP[3][0] = 1;        dP[3][1] = 0;         dP[3][2] = 0;
    P[4] = x * y;           dP[4][0] = y;        dP[4][1] = x;         dP[4][2] = 0;
    P[5] = y * z;           dP[5][0] = 0;        dP[5][1] = z;         dP[5][2] = y;
    P[6] = 2 * z * z - x * x - y * y;
    dP[6][0] = -2 * x; dP[6][1] = -2 * y; dP[6][2] = 4 * z;
    P[7] = x * z;           dP[7][0] = z;        dP[7][1] = 0;         dP[7][2] = x;
    P[8] = x * x - y * y;   dP[8][0] = 2 * x;    dP[8][1] = -2 * y;    dP[8][2] = 0;
    P[9] = y * (3 * x * x - y * y);
    dP[9][0] = 6 * x * y; dP[9][1] = 3 * x * x - 3 * y * y; dP[9][2] = 0;
    P[10] = x * y * z;
    dP[10][0] = y * z; dP[10][1] = x * z; dP[10][2] = x * y;
    P[11] = y * (4 * z * z - x * x - y * y);
    dP[11][0] = -2 * x * y; dP[11][1] = 4 * z * z - x * x - 3 * y * y; dP[11][2] = 8 * y * z;
    P[12] = z * (2 * z * z - 3 * x * x - 3 * y * y);
    dP[12][0] = -6 * x * z; dP[12][1] = -6 * y * z; dP[12][2] = 6 * z * z - 3 * x * x - 3 * y * y;
    P[13] = x * (4 * z * z - x * x - y * y);
    dP[13][0] = 4 * z * z - 3 * x * x - y * y; dP[13][1] = -2 * x * y; dP[13][2] = 8 * x * z;
    P[14] = z * (x * x - y * y);
    dP[14][0] = 2 * x * z; dP[14][1] = -2 * y * z; dP[14][2] = x * x - y * y;
    P[15] = x * (x * x - 3 * y * y);
    dP[15][0] = 3 * x * x - 3 * y * y; dP[15][1] = -6 * x * y; dP[15][2] = 0;
    for (int k = 0; k < 16; k++) {
        Y[k] = C[k] * P[k];
        if (dY)
            for (int i = 0; i < 3; i++) dY[3 * k + i] = C[k] * dP[k][i];
    }
}

/* Rotation matrix of the normalised quaternion (w, x, y, z). */
static void orc_quat_rot(const double* qn, double* R)
{
    double w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Camera centre in world space: -R^T t. */
static void orc_cam_centre(const orc_cam* cam, double* cp)
{
    for (int j = 0; j < 3; j++) {
        cp[j] = 0;
        for (int i = 0; i < 3; i++) cp[j] -= (double)cam->R[3 * i + j] * (double)cam->t[i];
    }
}

/* Projected record layout (ORC_PSTRIDE doubles):
 * 0 valid, 1-3 t (camera space), 4-5 mean2D, 6-8 cov2D (a,b,c), 9-11 conic,
 * 12 opacity, 13-15 raw colour (before clamp), 16-18 clamped colour,
 * 19-21 unit view direction, 22 distance |mu - campos|, 23 unused. */
static void orc_project_one(const double* mu, const double* q, const double* s, double op,
                            const double* sh, const orc_cam* cam, const double* cp, double* P)
{
    memset(P, 0, sizeof(double) * ORC_PSTRIDE);
    double qn2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    if (!(qn2 > 0)) return;
    double qr = sqrt(qn2), qn[4] = {q[0] / qr, q[1] / qr, q[2] / qr, q[3] / qr};
    double R[9];
    orc_quat_rot(qn, R);
    double M[9], S[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) M[3 * i + j] = R[3 * i + j] * s[j];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            S[3 * i + j] = 0;
            for (int k = 0; k < 3; k++) S[3 * i + j] += M[3 * i + k] * M[3 * j + k];
        }
    double C[9], t[3];
    for (int i = 0; i < 9; i++) C[i] = cam->R[i];
    for (int i = 0; i < 3; i++) t[i] = C[3 * i] * mu[0] + C[3 * i + 1] * mu[1] + C[3 * i + 2] * mu[2] + cam->t[i];
    if (!(t[2] >= 0.01)) return;
    double fx = cam->fx, fy = cam->fy;
    double limx = 1.3 * (0.5 * cam->width / fx), limy = 1.3 * (0.5 * cam->height / fy);
    double ux = t[0] / t[2], uy = t[1] / t[2];
    ux = fmin(fmax(ux, -limx), limx);
    uy = fmin(fmax(uy, -limy), limy);
    double J[6] = {fx / t[2], 0, -fx * ux / t[2], 0, fy / t[2], -fy * uy / t[2]};
    double T[6];
    for (int i = 0; i < 2; i++)
        for (int k = 0; k < 3; k++)
            T[3 * i + k] = J[3 * i] * C[k] + J[3 * i + 1] * C[3 + k] + J[3 * i + 2] * C[6 + k];
    double V[4] = {0, 0, 0, 0};
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 2; j++)
            for (int k = 0; k < 3; k++)
                for (int l = 0; l < 3; l++) V[2 * i + j] += T[3 * i + k] * S[3 * k + l] * T[3 * j + l];
    double a = V[0] + 0.3, b = V[1], c = V[3] + 0.3;
    double det = a * c - b * b;
    if (!(det > 0)) return;
    P[0] = 1;
    P[1] = t[0]; P[2] = t[1]; P[3] = t[2];
    P[4] = fx * t[0] / t[2] + cam->cx;
    P[5] = fy * t[1] / t[2] + cam->cy;
    P[6] = a; P[7] = b; P[8] = c;
    P[9] = c / det; P[10] = -b / det; P[11] = a / det;
    P[12] = op;
    double d[3] = {mu[0] - cp[0], mu[1] - cp[1], mu[2] - cp[2]};
    double dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double dir[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
    double Y[16];
    orc_sh_basis(dir, Y, NULL);
    for (int ch = 0; ch < 3; ch++) {
        double v = 0.5;
        for (int k = 0; k < 16; k++) v += sh[3 * k + ch] * Y[k];
        P[13 + ch] = v;
        P[16 + ch] = v < 0 ? 0 : v;
    }
    P[19] = dir[0]; P[20] = dir[1]; P[21] = dir[2];
    P[22] = dist;
}

/* FP64 projection of n Gaussians for one camera.  Parameters are given in
 * activated form (scales s > 0, opacity o in (0,1)). */
void orc_project64(int64_t n, const double* means, const double* quats, const double* scales,
                   const double* opac, const double* sh, const orc_cam* cam, double* proj)
{
    double cp[3];
    orc_cam_centre(cam, cp);
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < n; g++)
        orc_project_one(means + 3 * g, quats + 4 * g, scales + 3 * g, opac[g], sh + 48 * g, cam, cp,
                        proj + ORC_PSTRIDE * g);
}

/* Contribution of projected Gaussian P at pixel centre (px, py): returns the
 * clamped alpha, or 0 when the pair is outside 3 sigma or below 1/255.
 * *flag is set when a decision that changes the image lies within `margin`
 * (relative) of its threshold: the 3-sigma cut (only when alpha there would
 * reach 1/255) or the 1/255 skip.  *gflag is set when only this Gaussian's
 * own gradient is affected: alpha near the 0.99 clamp (alpha is continuous
 * there, its derivative is not).  *Gout and *clamped report the Gaussian
 * value and clamp state. */
static double orc_alpha(const double* P, double px, double py, double margin, int* flag, int* gflag,
                        double* Gout, int* clamped, double* dx_out, double* dy_out)
{
    double dx = px - P[4], dy = py - P[5];
    double d2 = P[9] * dx * dx + 2 * P[10] * dx * dy + P[11] * dy * dy;
    if (fabs(d2 - 9.0) <= margin * 9.0 && P[12] * exp(-4.5) >= (1.0 - margin) / 255.0) *flag = 1;
    if (d2 > 9.0) return 0;
    double G = exp(-0.5 * d2);
    double araw = P[12] * G;
    if (fabs(araw - 0.99) <= margin * 0.99) *gflag = 1;
    int cl = araw > 0.99;
    double al = cl ? 0.99 : araw;
    if (fabs(al - 1.0 / 255.0) <= margin / 255.0) *flag = 1;
    if (al < 1.0 / 255.0) return 0;
    *Gout = G;
    *clamped = cl;
    *dx_out = dx;
    *dy_out = dy;
    return al;
}

/* Front-to-back compositing over each tile's sorted list (FP64).
 * image: H*W*3 (row-major, channel-last); tfinal: H*W; nlast: H*W, the list
 * position (relative to the tile's start) one past the last blended entry.
 * unstable_px / unstable_g (optional) mark pixels and Gaussians with a
 * decision within `margin` of a threshold.  Returns the blended pair count. */
int64_t orc_render64(const orc_cam* cam, int64_t n, const double* proj, const uint32_t* sorted_g,
                     const int64_t* ranges, const double* bg, double* image, double* tfinal,
                     int32_t* nlast, double margin, uint8_t* unstable_px, uint8_t* unstable_g)
{
    (void)n;
    int W = cam->width, H = cam->height, TW = orc_tiles_x(cam);
    int64_t blended = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : blended)
    for (int64_t pix = 0; pix < (int64_t)W * H; pix++) {
        int x = (int)(pix % W), y = (int)(pix / W);
        int64_t tile = (int64_t)(y / cam->tile_h) * TW + x / cam->tile_w;
        int64_t s0 = ranges[2 * tile], s1 = ranges[2 * tile + 1];
        double T = 1, Cc[3] = {0, 0, 0};
        int32_t last = 0;
        int uflag = 0;
        for (int64_t k = s0; k < s1; k++) {
            uint32_t g = sorted_g[k];
            const double* P = proj + ORC_PSTRIDE * g;
            if (!P[0]) { uflag = 1; if (unstable_g) unstable_g[g] = 1; continue; }
            int flag = 0, gflag = 0, cl;
            double G, dx, dy;
            double al = orc_alpha(P, x + 0.5, y + 0.5, margin, &flag, &gflag, &G, &cl, &dx, &dy);
            double Tn = T * (1 - al);
            if (al > 0 && fabs(Tn - 1e-4) <= margin * 1e-4) flag = 1;
            if (flag) uflag = 1;
            if ((flag || gflag) && unstable_g) unstable_g[g] = 1;
            if (al == 0) continue;
            if (Tn < 1e-4) break;
            for (int ch = 0; ch < 3; ch++) Cc[ch] += P[16 + ch] * al * T;
            T = Tn;
            last = (int32_t)(k - s0 + 1);
            blended++;
        }
        for (int ch = 0; ch < 3; ch++) image[3 * pix + ch] = Cc[ch] + T * bg[ch];
        tfinal[pix] = T;
        nlast[pix] = last;
        if (unstable_px) unstable_px[pix] = (uint8_t)uflag;
    }
    return blended;
}

/* Brute-force compositing: every pixel walks the whole `order` list (all
 * Gaussians, in one global depth order) with the same contribution rule. */
int64_t orc_render64_brute(const orc_cam* cam, const double* proj, int64_t n_order,
                           const uint32_t* order, const double* bg, double* image, double* tfinal)
{
    int W = cam->width, H = cam->height;
    int64_t blended = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : blended)
    for (int64_t pix = 0; pix < (int64_t)W * H; pix++) {
        int x = (int)(pix % W), y = (int)(pix / W);
        double T = 1, Cc[3] = {0, 0, 0};
        for (int64_t k = 0; k < n_order; k++) {
            const double* P = proj + ORC_PSTRIDE * order[k];
            if (!P[0]) continue;
            int flag = 0, gflag = 0, cl;
            double G, dx, dy;
            double al = orc_alpha(P, x + 0.5, y + 0.5, 0.0, &flag, &gflag, &G, &cl, &dx, &dy);
            if (al == 0) continue;
            double Tn = T * (1 - al);
            if (Tn < 1e-4) break;
            for (int ch = 0; ch < 3; ch++) Cc[ch] += P[16 + ch] * al * T;
            T = Tn;
            blended++;
        }
        for (int ch = 0; ch < 3; ch++) image[3 * pix + ch] = Cc[ch] + T * bg[ch];
        tfinal[pix] = T;
    }
    return blended;
}

/* Analytic backward of the compositing (FP64), per Gaussian of this view:
 * grad2d: n x 9 = dL/d(mean2D x, y), dL/d(conic a, b, c) with b the
 * off-diagonal value, dL/d(opacity), dL/d(clamped colour r, g, b).
 * For pair i of a pixel: dC/dc_i = alpha_i T_i and
 * dC/dalpha_i = c_i T_i - S_i / (1 - alpha_i), S_i = sum_{j>i} c_j alpha_j T_j
 * + T_final bg. */
void orc_raster_bwd64(const orc_cam* cam, int64_t n, const double* proj, const uint32_t* sorted_g,
                      const int64_t* ranges, const double* bg, const double* dLdC, double* grad2d)
{
    int W = cam->width, H = cam->height, TW = orc_tiles_x(cam);
    memset(grad2d, 0, sizeof(double) * 9 * (size_t)n);
    /* serial over pixels: the per-Gaussian sums are accumulated in a fixed
     * order, so the result does not depend on the thread count */
    int64_t cap = 0;
    for (int64_t t = 0; t < (int64_t)TW * orc_tiles_y(cam); t++) {
        int64_t len = ranges[2 * t + 1] - ranges[2 * t];
        if (len > cap) cap = len;
    }
    if (cap == 0) return;
    double* al_l = (double*)malloc(sizeof(double) * (size_t)cap);
    double* T_l = (double*)malloc(sizeof(double) * (size_t)cap);
    double* G_l = (double*)malloc(sizeof(double) * (size_t)cap);
    double* dx_l = (double*)malloc(sizeof(double) * (size_t)cap);
    double* dy_l = (double*)malloc(sizeof(double) * (size_t)cap);
    int* cl_l = (int*)malloc(sizeof(int) * (size_t)cap);
    int64_t* k_l = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);
    for (int64_t pix = 0; pix < (int64_t)W * H; pix++) {
        int x = (int)(pix % W), y = (int)(pix / W);
        int64_t tile = (int64_t)(y / cam->tile_h) * TW + x / cam->tile_w;
        int64_t s0 = ranges[2 * tile], s1 = ranges[2 * tile + 1];
        double T = 1;
        int m = 0;
        for (int64_t k = s0; k < s1; k++) {
            const double* P = proj + ORC_PSTRIDE * sorted_g[k];
            if (!P[0]) continue;
            int flag = 0, gflag = 0, cl;
            double G, dx, dy;
            double al = orc_alpha(P, x + 0.5, y + 0.5, 0.0, &flag, &gflag, &G, &cl, &dx, &dy);
            if (al == 0) continue;
            double Tn = T * (1 - al);
            if (Tn < 1e-4) break;
            al_l[m] = al; T_l[m] = T; G_l[m] = G; cl_l[m] = cl; dx_l[m] = dx; dy_l[m] = dy; k_l[m] = k;
            m++;
            T = Tn;
        }
        const double* dl = dLdC + 3 * pix;
        double S[3] = {T * bg[0], T * bg[1], T * bg[2]};
        for (int i = m - 1; i >= 0; i--) {
            uint32_t g = sorted_g[k_l[i]];
            const double* P = proj + ORC_PSTRIDE * g;
            double* gr = grad2d + 9 * g;
            double al = al_l[i], Ti = T_l[i];
            double dal = 0;
            for (int ch = 0; ch < 3; ch++) {
                gr[6 + ch] += al * Ti * dl[ch];
                dal += dl[ch] * (P[16 + ch] * Ti - S[ch] / (1 - al));
            }
            for (int ch = 0; ch < 3; ch++) S[ch] += P[16 + ch] * al * Ti;
            if (cl_l[i]) continue;
            double G = G_l[i], dx = dx_l[i], dy = dy_l[i];
            gr[5] += dal * G;
            double dpow = dal * P[12] * G;
            /* power = -0.5 (ca dx^2 + 2 cb dx dy + cc dy^2), dx = px - mx */
            gr[2] += -0.5 * dx * dx * dpow;
            gr[3] += -dx * dy * dpow;
            gr[4] += -0.5 * dy * dy * dpow;
            gr[0] += (P[9] * dx + P[10] * dy) * dpow;
            gr[1] += (P[10] * dx + P[11] * dy) * dpow;
        }
    }
    free(al_l); free(T_l); free(G_l); free(dx_l); free(dy_l); free(cl_l); free(k_l);
}

/* Analytic backward of the projection (FP64) for one camera: accumulates
 * into grad (n x ORC_NTHETA) the gradient with respect to
 * theta = (mean 3, quaternion 4, log-scale 3, logit-opacity 1, SH 48), where
 * the SH index is 3*k + channel.  grad2d comes from orc_raster_bwd64. */
void orc_project_bwd64(int64_t n, const double* means, const double* quats, const double* scales,
                       const double* opac, const double* sh, const orc_cam* cam, const double* proj,
                       const double* grad2d, double* grad)
{
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < n; g++) {
        const double* P = proj + ORC_PSTRIDE * g;
        const double* g2 = grad2d + 9 * g;
        double* out = grad + ORC_NTHETA * g;
        if (!P[0]) continue;
        const double* mu = means + 3 * g;
        const double* q = quats + 4 * g;
        const double* s = scales + 3 * g;
        const double* shg = sh + 48 * g;
        double fx = cam->fx, fy = cam->fy;
        double C[9];
        for (int i = 0; i < 9; i++) C[i] = cam->R[i];
        double tx = P[1], ty = P[2], tz = P[3];

        /* colour: clamp, SH coefficients, view direction */
        double draw[3];
        for (int ch = 0; ch < 3; ch++) draw[ch] = P[13 + ch] < 0 ? 0 : g2[6 + ch];
        double Y[16], dY[48];
        orc_sh_basis(P + 19, Y, dY);
        for (int k = 0; k < 16; k++)
            for (int ch = 0; ch < 3; ch++) out[11 + 3 * k + ch] += Y[k] * draw[ch];
        double ddir[3] = {0, 0, 0};
        for (int k = 0; k < 16; k++)
            for (int ch = 0; ch < 3; ch++)
                for (int i = 0; i < 3; i++) ddir[i] += shg[3 * k + ch] * draw[ch] * dY[3 * k + i];
        const double* dir = P + 19;
        double dd = ddir[0] * dir[0] + ddir[1] * dir[1] + ddir[2] * dir[2];
        for (int i = 0; i < 3; i++) out[i] += (ddir[i] - dir[i] * dd) / P[22];

        /* opacity */
        out[10] += g2[5] * opac[g] * (1 - opac[g]);

        /* conic -> 2D covariance: dL/dV = -Q G Q with G symmetric */
        double Q[4] = {P[9], P[10], P[10], P[11]};
        double Gq[4] = {g2[2], 0.5 * g2[3], 0.5 * g2[3], g2[4]};
        double QG[4], dV[4];
        for (int i = 0; i < 2; i++)
            for (int j = 0; j < 2; j++) QG[2 * i + j] = Q[2 * i] * Gq[j] + Q[2 * i + 1] * Gq[2 + j];
        for (int i = 0; i < 2; i++)
            for (int j = 0; j < 2; j++) dV[2 * i + j] = -(QG[2 * i] * Q[j] + QG[2 * i + 1] * Q[2 + j]);

        /* rebuild J, T = J C, Sigma */
        double limx = 1.3 * (0.5 * cam->width / fx), limy = 1.3 * (0.5 * cam->height / fy);
        double ux = tx / tz, uy = ty / tz;
        int inx = (ux >= -limx && ux <= limx), iny = (uy >= -limy && uy <= limy);
        double uxc = fmin(fmax(ux, -limx), limx), uyc = fmin(fmax(uy, -limy), limy);
        double J[6] = {fx / tz, 0, -fx * uxc / tz, 0, fy / tz, -fy * uyc / tz};
        double T[6];
        for (int i = 0; i < 2; i++)
            for (int k = 0; k < 3; k++)
                T[3 * i + k] = J[3 * i] * C[k] + J[3 * i + 1] * C[3 + k] + J[3 * i + 2] * C[6 + k];
        double qr = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        double qn[4] = {q[0] / qr, q[1] / qr, q[2] / qr, q[3] / qr};
        double R[9], M[9], S[9];
        orc_quat_rot(qn, R);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) M[3 * i + j] = R[3 * i + j] * s[j];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                S[3 * i + j] = 0;
                for (int k = 0; k < 3; k++) S[3 * i + j] += M[3 * i + k] * M[3 * j + k];
            }

        /* V = T S T^T: dL/dS = T^T dV T, dL/dT = 2 dV T S */
        double dS[9], TS[6], dT[6];
        for (int k = 0; k < 3; k++)
            for (int l = 0; l < 3; l++) {
                double v = 0;
                for (int i = 0; i < 2; i++)
                    for (int j = 0; j < 2; j++) v += T[3 * i + k] * dV[2 * i + j] * T[3 * j + l];
                dS[3 * k + l] = v;
            }
        for (int i = 0; i < 2; i++)
            for (int l = 0; l < 3; l++) {
                TS[3 * i + l] = 0;
                for (int k = 0; k < 3; k++) TS[3 * i + l] += T[3 * i + k] * S[3 * k + l];
            }
        for (int i = 0; i < 2; i++)
            for (int l = 0; l < 3; l++)
                dT[3 * i + l] = 2 * (dV[2 * i] * TS[l] + dV[2 * i + 1] * TS[3 + l]);
        /* T = J C: dL/dJ = dT C^T */
        double dJ[6];
        for (int i = 0; i < 2; i++)
            for (int k = 0; k < 3; k++) {
                double v = 0;
                for (int l = 0; l < 3; l++) v += dT[3 * i + l] * C[3 * k + l];
                dJ[3 * i + k] = v;
            }
        /* J entries as functions of t */
        double dt[3] = {0, 0, 0};
        dt[2] += -fx / (tz * tz) * dJ[0];
        dt[2] += -fy / (tz * tz) * dJ[4];
        /* J02 = -fx uxc / tz */
        dt[2] += fx * uxc / (tz * tz) * dJ[2];
        if (inx) {
            dt[0] += -fx / (tz * tz) * dJ[2];
            dt[2] += fx * tx / (tz * tz * tz) * dJ[2];
        }
        dt[2] += fy * uyc / (tz * tz) * dJ[5];
        if (iny) {
            dt[1] += -fy / (tz * tz) * dJ[5];
            dt[2] += fy * ty / (tz * tz * tz) * dJ[5];
        }
        /* mean2D */
        dt[0] += fx / tz * g2[0];
        dt[1] += fy / tz * g2[1];
        dt[2] += -fx * tx / (tz * tz) * g2[0] - fy * ty / (tz * tz) * g2[1];
        /* t = C mu + tvec */
        for (int j = 0; j < 3; j++) out[j] += C[j] * dt[0] + C[3 + j] * dt[1] + C[6 + j] * dt[2];

        /* S = M M^T: dL/dM = (dS + dS^T) M */
        double dM[9];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double v = 0;
                for (int k = 0; k < 3; k++) v += (dS[3 * i + k] + dS[3 * k + i]) * M[3 * k + j];
                dM[3 * i + j] = v;
            }
        /* M = R diag(s) */
        double dR[9];
        for (int j = 0; j < 3; j++) {
            double v = 0;
            for (int i = 0; i < 3; i++) v += dM[3 * i + j] * R[3 * i + j];
            out[7 + j] += v * s[j]; /* d/d(log s) = s d/ds */
        }
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) dR[3 * i + j] = dM[3 * i + j] * s[j];
        /* R(qn) */
        double w = qn[0], x = qn[1], y = qn[2], z = qn[3];
        double dqn[4];
        dqn[0] = 2 * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
        dqn[1] = 2 * (y * dR[1] + z * dR[2] + y * dR[3] - w * dR[5] + z * dR[6] + w * dR[7])
                 - 4 * x * (dR[4] + dR[8]);
        dqn[2] = 2 * (x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] + z * dR[7])
                 - 4 * y * (dR[0] + dR[8]);
        dqn[3] = 2 * (-w * dR[1] + x * dR[2] + w * dR[3] + y * dR[5] + x * dR[6] + y * dR[7])
                 - 4 * z * (dR[0] + dR[4]);
        double dqq = dqn[0] * qn[0] + dqn[1] * qn[1] + dqn[2] * qn[2] + dqn[3] * qn[3];
        for (int i = 0; i < 4; i++) out[3 + i] += (dqn[i] - qn[i] * dqq) / qr;
    }
}

/* One Adam step (PyTorch semantics, dense) on theta (n x ORC_NTHETA).
 * lr[6]: mean, quaternion, log-scale, logit-opacity, SH degree 0, SH rest. */
void orc_adam64(int64_t n, double* theta, double* m, double* v, const double* grad,
                const double* lr, double b1, double b2, double eps, int step)
{
    double bc1 = 1 - pow(b1, step), bc2 = 1 - pow(b2, step);
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < n; g++) {
        for (int j = 0; j < ORC_NTHETA; j++) {
            int grp = j < 3 ? 0 : j < 7 ? 1 : j < 10 ? 2 : j < 11 ? 3 : j < 14 ? 4 : 5;
            int64_t i = ORC_NTHETA * g + j;
            m[i] = b1 * m[i] + (1 - b1) * grad[i];
            v[i] = b2 * v[i] + (1 - b2) * grad[i] * grad[i];
            double mh = m[i] / bc1, vh = v[i] / bc2;
            theta[i] -= lr[grp] * mh / (sqrt(vh) + eps);
        }
    }
}

/* Thread count of the OpenMP loops above, for timing the oracle on one core
 * or on all of them; no result depends on it.  n <= 0 leaves it unchanged.
 * Returns the count in effect. */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
