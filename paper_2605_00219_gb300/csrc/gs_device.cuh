// gs_device.cuh -- device-side descriptors and helpers shared by the step
// kernels (sm_103a).  Nothing here is shared with the CPU oracle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gs_step.h"

namespace gs {

constexpr int kMaxViews = GS_MAX_VIEWS;
constexpr int kMaxScenes = GS_MAX_SCENES;

// Static shape of one view, passed by value in kernel parameters.
struct ViewDesc {
    int32_t W, H;          // pixels
    int32_t TX, TY;        // tiles
    int32_t scene;
    int32_t shift;         // key >> shift = tile id
    int32_t drop;          // depth code >> drop = low key bits
    int32_t rank;          // index of this view among its scene's views
    int64_t pair_base;     // first (view, Gaussian) pair of this view
    int64_t tile_base;     // first global tile of this view
    int64_t pix_base;      // first pixel of this view
};

// Two orders of the (view, Gaussian) pairs:
//  - view-major pair index p = pair_base[v] + g (projected records, the
//    pair index the sorted lists carry);
//  - Gaussian-major index q = qbase[s] + g * nv[s] + rank[v] (tile counts,
//    their offsets and so the emission slots of the intersections): a
//    Gaussian's intersections in all views of its scene are contiguous.
struct Views {
    int32_t n;
    int32_t tw, th;        // tile size, pixels
    int32_t n_scenes;
    int64_t pairs, tiles, pixels;
    ViewDesc v[kMaxViews];
    int64_t qbase[kMaxScenes + 1];
    int32_t nv[kMaxScenes];             // views of each scene
    uint8_t view_of[kMaxScenes][kMaxViews];   // view of each (scene, rank)
};

struct SceneDesc {
    int64_t n;
    int64_t base;          // first Gaussian of this scene in concatenated order
    float4* geom;          // float4[3][n]
    void* sh;              // float4[12][n] or uint4[6][n]
    void* m;               // float4[15][n] or uint2[15][n]
    void* v;
    float2* stats;         // NULL or densification statistics, float2[n]
};

struct Scenes {
    int32_t n;
    int32_t sh_bf16, mom_bf16;
    int32_t pad;
    int64_t total;
    SceneDesc s[kMaxScenes];
};

// Workspace header (device memory, first bytes of the workspace).
struct WsHeader {
    uint32_t status;
    int32_t step;
    unsigned long long k_required;
    unsigned long long blended;
    uint32_t k_eff;            // k_required if it fits the capacity, else 0
    uint32_t loss_counter;
    float loss;
    uint32_t pad;
    float bg[4];                  // background colour of the last raster_fwd
    uint32_t sort_class[4];       // tiles per list-size class (long, medium, short, tiny), by k_tile_order
};

// Projected record of one (view, Gaussian) pair, read by the raster kernels.
//   a = (mean x, mean y, conic a, conic b)
//   b = (conic c, opacity, red, green)
//   c = (blue, depth, mean x residual, mean y residual)
// The mean is the bit-specified binning value; the residuals make
// mean + residual the pixel-space mean to about 1e-12 relative, so pixel
// offsets near x ~ 2000 px keep full FP32 accuracy.
struct __align__(16) ProjRec {
    float4 a, b, c;
};

// Gradient record of one intersection, written by raster_bwd.
//   a = dL/d(mean x, mean y, conic a, conic b); b = (conic c, opacity, r, g);
//   c = (b, 0, 0, 0)
struct __align__(16) GradRec {
    float4 a, b, c;
};

// Bounds checks of the GS_DEBUG build: GS_DCHECK(cond, status) is true in
// the normal build; with GS_DEBUG defined it evaluates cond and, when cond is
// false, sets GS_STATUS_BOUNDS in *status so the caller can skip the access.
#ifdef GS_DEBUG
__device__ __forceinline__ bool gs_dcheck(bool ok, uint32_t* status)
{
    if (!ok) atomicOr(status, GS_STATUS_BOUNDS);
    return ok;
}
#define GS_DCHECK(cond, status) gs_dcheck((cond), (status))
#else
#define GS_DCHECK(cond, status) true
#endif

// Projected record of a sorted entry's pair; in the GS_DEBUG build an index
// outside the records gives an all-zero record (opacity 0: no warp block
// takes it) and sets GS_STATUS_BOUNDS.
__device__ __forceinline__ ProjRec rec_at(const ProjRec* __restrict__ rec, uint32_t pid, int64_t pairs,
                                          uint32_t* status)
{
#ifdef GS_DEBUG
    if (!gs_dcheck((int64_t)pid < pairs, status)) {
        ProjRec z;
        z.a = z.b = z.c = make_float4(0.f, 0.f, 0.f, 0.f);
        return z;
    }
#else
    (void)pairs;
    (void)status;
#endif
    return rec[pid];
}

// A tile's list range, checked against the capacity in the GS_DEBUG build
// (an out-of-range list is treated as empty).
__device__ __forceinline__ uint2 range_at(const uint2* __restrict__ ranges, int64_t gt, uint32_t cap,
                                          uint32_t* status)
{
    uint2 r = ranges[gt];
#ifdef GS_DEBUG
    if (!gs_dcheck(r.x <= r.y && r.y <= cap, status)) r = make_uint2(0u, 0u);
#else
    (void)cap;
    (void)status;
#endif
    return r;
}

__device__ __forceinline__ int view_of_pair(const Views& V, int64_t p)
{
    int v = 0;
    while (v + 1 < V.n && V.v[v + 1].pair_base <= p) v++;
    return v;
}

__device__ __forceinline__ int view_of_tile(const Views& V, int64_t t)
{
    int v = 0;
    while (v + 1 < V.n && V.v[v + 1].tile_base <= t) v++;
    return v;
}

// --------------------------------------------------------------------------
// FP32 binning, bit-specified: every operation is one correctly rounded
// binary32 operation in the written order (explicit _rn intrinsics, which the
// compiler never fuses or reorders).
// --------------------------------------------------------------------------

#define FM(a, b) __fmul_rn((a), (b))
#define FA(a, b) __fadd_rn((a), (b))
#define FS(a, b) __fsub_rn((a), (b))
#define FD(a, b) __fdiv_rn((a), (b))
#define FQ(a) __fsqrt_rn(a)

// Natural logarithm of a finite normal x > 0 as a fixed sequence of rounded
// binary32 operations, so that the cull radius below is the same bit pattern
// wherever it is evaluated: x = 2^e m with m in [sqrt(1/2), sqrt(2)), and
// ln m = 2 atanh(s), s = (m - 1) / (m + 1), by the odd Taylor series of atanh
// to s^9 (|s| <= 0.1716: truncation below 1e-9; about 2e-7 absolute error
// over [1, 256]).
__device__ __forceinline__ float bin_log(float x)
{
    uint32_t u = __float_as_uint(x);
    int e = (int)(u >> 23) - 127;
    float m = __uint_as_float((u & 0x7FFFFFu) | 0x3F800000u);
    if (m > 1.41421356f) {
        m = FM(0.5f, m);
        e += 1;
    }
    const float sv = FD(FS(m, 1.0f), FA(m, 1.0f));
    const float s2 = FM(sv, sv);
    float p = FA(FM(s2, 0.111111111f), 0.142857143f);
    p = FA(FM(s2, p), 0.2f);
    p = FA(FM(s2, p), 0.333333333f);
    p = FA(FM(s2, p), 1.0f);
    return FA(FM((float)e, 0.693147181f), FM(FM(2.0f, sv), p));
}

// Cull radius^2 for opacity o (Sec. 4.1): a pixel takes part only if
// d^2 <= 9 and o exp(-d^2 / 2) >= 1/255, i.e. d^2 <= min(9, 2 ln(255 o));
// widened by 2^-10 relative and 2^-10 absolute so that the FP32 culling stays
// conservative against the raster's own tests.  Negative when 255 o <= 1.
__device__ __forceinline__ float cull_r2(float o)
{
    const float x = FM(255.0f, o);
    if (!(x > 1.0f)) return -1.0f;
    const float r = fminf(9.0f, FM(2.0f, bin_log(x)));
    return FA(FM(r, 1.0009765625f), 0.0009765625f);
}

struct BinGeom {
    float mx, my, a, b, c, det, tz, r2;
    uint32_t mant;
    int valid;
};

// View-independent part of the bit-specified binning of one Gaussian: the
// cull radius^2 and the 3D covariance S = (R(q) diag(s))(R(q) diag(s))^T
// (upper triangle S00, S01, S02, S11, S12, S22).  valid = 0 when the
// Gaussian is never listed (255 o <= 1, or a zero quaternion).
struct BinGauss {
    float S[6];
    float r2;
    int valid;
};

__device__ __forceinline__ void bin_gauss(float4 q, float4 s, BinGauss& o)
{
    o.valid = 0;
    const float r2 = cull_r2(s.w);
    if (!(r2 > 0.0f)) return;
    float n2 = FA(FA(FA(FM(q.x, q.x), FM(q.y, q.y)), FM(q.z, q.z)), FM(q.w, q.w));
    if (!(n2 > 0.0f)) return;
    float r = FQ(n2);
    float w = FD(q.x, r), x = FD(q.y, r), y = FD(q.z, r), z = FD(q.w, r);
    float xx = FM(x, x), yy = FM(y, y), zz = FM(z, z);
    float xy = FM(x, y), xz = FM(x, z), yz = FM(y, z);
    float wx = FM(w, x), wy = FM(w, y), wz = FM(w, z);
    float R[9];
    R[0] = FS(1.0f, FM(2.0f, FA(yy, zz)));
    R[1] = FM(2.0f, FS(xy, wz));
    R[2] = FM(2.0f, FA(xz, wy));
    R[3] = FM(2.0f, FA(xy, wz));
    R[4] = FS(1.0f, FM(2.0f, FA(xx, zz)));
    R[5] = FM(2.0f, FS(yz, wx));
    R[6] = FM(2.0f, FS(xz, wy));
    R[7] = FM(2.0f, FA(yz, wx));
    R[8] = FS(1.0f, FM(2.0f, FA(xx, yy)));
    const float sv[3] = {s.x, s.y, s.z};
    float M[9];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) M[3 * i + j] = FM(R[3 * i + j], sv[j]);
    int k = 0;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = i; j < 3; j++)
            o.S[k++] = FA(FA(FM(M[3 * i], M[3 * j]), FM(M[3 * i + 1], M[3 * j + 1])), FM(M[3 * i + 2], M[3 * j + 2]));
    o.r2 = r2;
    o.valid = 1;
}

// Field-of-view clamp limits of a view, 1.3 x the half extent in normalised
// image coordinates: (1.3 (W/2) / fx, 1.3 (H/2) / fy).
__device__ __forceinline__ float2 fov_limits(const float* cam, int W, int H)
{
    return make_float2(FM(1.3f, FD(FM(0.5f, (float)W), cam[12])), FM(1.3f, FD(FM(0.5f, (float)H), cam[13])));
}

// View-dependent part: camera transform, near-plane cull, EWA covariance
// with the field-of-view clamp (lim = fov_limits of the view), conic
// determinant, pixel mean and depth code, from the view-independent part.
__device__ __forceinline__ void bin_view(float4 mu, const BinGauss& bgs, const float* cam, float2 lim, BinGeom& o)
{
    o.valid = 0;
    if (!bgs.valid) return;
    const float S[9] = {bgs.S[0], bgs.S[1], bgs.S[2], bgs.S[1], bgs.S[3], bgs.S[4], bgs.S[2], bgs.S[4], bgs.S[5]};
    const float r2 = bgs.r2;
    const float* C = cam;          // R row-major
    const float mv[3] = {mu.x, mu.y, mu.z};
    float t[3];
#pragma unroll
    for (int i = 0; i < 3; i++)
        t[i] = FA(FA(FA(FM(C[3 * i], mv[0]), FM(C[3 * i + 1], mv[1])), FM(C[3 * i + 2], mv[2])), cam[9 + i]);
    if (!(t[2] >= 0.01f)) return;
    const float fx = cam[12], fy = cam[13], cx = cam[14], cy = cam[15];
    const float limx = lim.x, limy = lim.y;
    float ux = fminf(fmaxf(FD(t[0], t[2]), -limx), limx);
    float uy = fminf(fmaxf(FD(t[1], t[2]), -limy), limy);
    float j00 = FD(fx, t[2]), j11 = FD(fy, t[2]);
    float j02 = -FD(FM(fx, ux), t[2]);
    float j12 = -FD(FM(fy, uy), t[2]);
    float T[6];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        T[k] = FA(FM(j00, C[k]), FM(j02, C[6 + k]));
        T[3 + k] = FA(FM(j11, C[3 + k]), FM(j12, C[6 + k]));
    }
    float U[6];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int k = 0; k < 3; k++)
            U[3 * i + k] = FA(FA(FM(T[3 * i], S[k]), FM(T[3 * i + 1], S[3 + k])), FM(T[3 * i + 2], S[6 + k]));
    float a = FA(FA(FA(FM(U[0], T[0]), FM(U[1], T[1])), FM(U[2], T[2])), 0.3f);
    float b = FA(FA(FM(U[0], T[3]), FM(U[1], T[4])), FM(U[2], T[5]));
    float c = FA(FA(FA(FM(U[3], T[3]), FM(U[4], T[4])), FM(U[5], T[5])), 0.3f);
    float det = FS(FM(a, c), FM(b, b));
    if (!(det > 0.0f)) return;
    float mx = FA(FD(FM(fx, t[0]), t[2]), cx);
    float my = FA(FD(FM(fy, t[1]), t[2]), cy);
    if (!(fabsf(mx) < 1e30f) || !(fabsf(my) < 1e30f) || !(a < 1e30f) || !(c < 1e30f) || !(det < 1e30f)) return;
    float qd = FD(FA(FM(2.0f, t[2]), 1.0f), FA(t[2], 1.0f));
    uint32_t mant = __float_as_uint(qd) & 0x7FFFFFu;
    if (qd >= 2.0f) mant = 0x7FFFFFu;
    o.valid = 1;
    o.mx = mx; o.my = my; o.a = a; o.b = b; o.c = c; o.det = det; o.tz = t[2]; o.mant = mant; o.r2 = r2;
}

// 1/T for a power of two T (exponent arithmetic: exact).
__device__ __forceinline__ float inv_pow2(int T) { return __int_as_float(0x7F000000 - __float_as_int((float)T)); }

// Tile index bounds of a pixel-centre coordinate: the tile sizes are powers
// of two (8, 16, 32), so the correctly rounded division by T equals the
// product with the exact reciprocal 1/T, bit for bit.
__device__ __forceinline__ int tile_lo(float v, int T, int n)
{
    float f = ceilf(FM(FS(FA(v, 0.5f), (float)T), inv_pow2(T)));
    f = fminf(fmaxf(f, -1.0f), (float)n);
    int i = (int)f;
    return i < 0 ? 0 : i;
}

__device__ __forceinline__ int tile_hi(float v, int T, int n)
{
    float f = floorf(FM(FS(v, 0.5f), inv_pow2(T)));
    f = fminf(fmaxf(f, -1.0f), (float)n);
    int i = (int)f;
    return i > n - 1 ? n - 1 : i;
}

// Scan-line traversal (Sec. 4.1) of the tiles whose pixel-centre rectangle
// meets the ellipse d^2 <= g.r2, band by band along the shorter dimension of
// the tile bounding box: calls band(rows, coord, lo, hi) for every band that
// meets a tile, in traversal order -- rows: bands are tile rows (coord = ty,
// tiles tx = lo..hi), else tile columns (coord = tx, tiles ty = lo..hi).
// Returns the number of tiles.
template <typename Band>
__device__ __forceinline__ uint32_t scanline_bands(const BinGeom& g, int tw, int th, int TX, int TY, Band band)
{
    const float r2 = g.r2;
    float ex = FQ(FM(r2, g.a));
    float ey = FQ(FM(r2, g.c));
    int txl = tile_lo(FS(g.mx, ex), tw, TX), txh = tile_hi(FA(g.mx, ex), tw, TX);
    int tyl = tile_lo(FS(g.my, ey), th, TY), tyh = tile_hi(FA(g.my, ey), th, TY);
    if (txl > txh || tyl > tyh) return 0;
    uint32_t count = 0;
    if (tyh - tyl <= txh - txl) {
        float ystar = FM(g.b, FQ(FD(r2, g.a)));
        float r2c = FM(r2, g.c);
        for (int ty = tyl; ty <= tyh; ty++) {
            float y0 = FS(FA((float)(ty * th), 0.5f), g.my);
            float y1 = FS(FS((float)((ty + 1) * th), 0.5f), g.my);
            float dlo = fmaxf(y0, -ey), dhi = fminf(y1, ey);
            if (!(dlo <= dhi)) continue;
            float dR = fminf(fmaxf(ystar, dlo), dhi);
            float dL = fminf(fmaxf(-ystar, dlo), dhi);
            float hR = FQ(fmaxf(0.0f, FM(g.det, FS(r2c, FM(dR, dR)))));
            float hL = FQ(fmaxf(0.0f, FM(g.det, FS(r2c, FM(dL, dL)))));
            float xR = FA(g.mx, FD(FA(FM(g.b, dR), hR), g.c));
            float xL = FA(g.mx, FD(FS(FM(g.b, dL), hL), g.c));
            int lo = tile_lo(xL, tw, TX), hi = tile_hi(xR, tw, TX);
            if (lo > hi) continue;
            band(true, ty, lo, hi);
            count += (uint32_t)(hi - lo + 1);
        }
    } else {
        float xstar = FM(g.b, FQ(FD(r2, g.c)));
        float r2a = FM(r2, g.a);
        for (int tx = txl; tx <= txh; tx++) {
            float x0 = FS(FA((float)(tx * tw), 0.5f), g.mx);
            float x1 = FS(FS((float)((tx + 1) * tw), 0.5f), g.mx);
            float dlo = fmaxf(x0, -ex), dhi = fminf(x1, ex);
            if (!(dlo <= dhi)) continue;
            float dT = fminf(fmaxf(xstar, dlo), dhi);
            float dB = fminf(fmaxf(-xstar, dlo), dhi);
            float hT = FQ(fmaxf(0.0f, FM(g.det, FS(r2a, FM(dT, dT)))));
            float hB = FQ(fmaxf(0.0f, FM(g.det, FS(r2a, FM(dB, dB)))));
            float yT = FA(g.my, FD(FA(FM(g.b, dT), hT), g.a));
            float yB = FA(g.my, FD(FS(FM(g.b, dB), hB), g.a));
            int lo = tile_lo(yB, th, TY), hi = tile_hi(yT, th, TY);
            if (lo > hi) continue;
            band(false, tx, lo, hi);
            count += (uint32_t)(hi - lo + 1);
        }
    }
    return count;
}

// The same traversal tile by tile: emit(i, tile id) for the i-th tile.
template <typename Emit>
__device__ __forceinline__ uint32_t scanline_tiles(const BinGeom& g, int tw, int th, int TX, int TY, Emit emit)
{
    uint32_t i = 0;
    return scanline_bands(g, tw, th, TX, TY, [&](bool rows, int coord, int lo, int hi) {
        for (int t = lo; t <= hi; t++, i++) emit(i, rows ? (uint32_t)(coord * TX + t) : (uint32_t)(t * TX + coord));
    });
}

// Tile span of a pair, written by the projection's traversal and read by
// the emission, so that the emission repeats no traversal arithmetic
// (16 bytes, Gaussian-major pair order).  x: depth code (bits 0-22), number
// of bands nb (bits 24-25), band orientation (bit 26: 1 = tile rows), ranked
// (bit 27: the projection took the pair's place in each of its tiles' lists,
// kRankMax tiles at most).  With nb <= 2: y = coord0 | coord1 << 16,
// z = lo0 | hi0 << 16, w = lo1 | hi1 << 16 (tile coordinates < 2^16).
// nb = 3 marks a pair with more than two bands: y, z, w then hold the
// binning conic's a, b, c bits, from which the emission repeats the
// traversal.
constexpr uint32_t kSpanMany = 3u;
constexpr uint32_t kRankMax = 4u;

__device__ __forceinline__ uint4 span_pack(uint32_t mant, uint32_t nb, bool rows, bool ranked, uint32_t c0,
                                           uint32_t c1, uint32_t r0, uint32_t r1, const BinGeom& g)
{
    if (nb > 2) return make_uint4(mant | (kSpanMany << 24), __float_as_uint(g.a), __float_as_uint(g.b),
                                  __float_as_uint(g.c));
    return make_uint4(mant | (nb << 24) | (rows ? 1u << 26 : 0u) | (ranked ? 1u << 27 : 0u), c0 | (c1 << 16), r0,
                      r1);
}

// The i-th tile (local id) of a span of one or two bands.
__device__ __forceinline__ uint32_t span_tile(uint32_t i, bool rows, uint32_t TX, uint32_t c0, uint32_t c1,
                                              uint32_t r0, uint32_t r1)
{
    const uint32_t lo0 = r0 & 0xFFFFu, n0 = (r0 >> 16) - lo0 + 1u;
    const bool second = i >= n0;
    const uint32_t t = second ? (r1 & 0xFFFFu) + (i - n0) : lo0 + i;
    const uint32_t cd = second ? c1 : c0;
    return rows ? cd * TX + t : t * TX + cd;
}

// --------------------------------------------------------------------------
// Pair evaluation shared by raster forward and backward: identical
// instruction sequence in both kernels, so both take the same decisions.
// --------------------------------------------------------------------------


__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Conservative mask of the warp blocks (8 x BH pixels; BH = 4 x the pixels
// each lane owns) of a tile (WPR blocks per row, RPB rows of blocks;
// WPR * RPB <= 16) that a Gaussian (mean, conic, opacity) can contribute to.  A pair needs d^2 <= 9 and
// o exp(-d^2/2) >= 1/255, i.e. d^2 <= r^2 = min(9, 2 ln(255 o)); the
// half-extents sqrt(r^2 c / det), sqrt(r^2 a / det) of that ellipse, widened
// by 0.1% of r^2, 1e-5 relative and 0.01 px (which also cover the hardware
// divide and square root), give a box that is intersected with the blocks.
// (ox, oy) is the tile's first pixel.  Pairs in a masked-out block would be
// skipped by the raster's own tests, so skipping them changes no result.
__device__ __forceinline__ uint32_t warp_block_mask(float mx, float my, float ca, float cb, float cc, float op,
                                                    int ox, int oy, int WPR, int RPB, int BH = 4)
{
    if (!(op * 255.0f > 1.0f)) return 0u;  // alpha never reaches 1/255
    const float det = ca * cc - cb * cb;
    if (!(det > 0.0f)) return 0xffffffffu;
    const float r2 = fminf(9.0f, 2.0f * __logf(op * 255.0f)) * 1.002f + 1e-3f;
    const float s = __fdividef(r2, det);
    const float ex = fmaf(sqrt_approx(s * cc), 1.00001f, 0.01f);
    const float ey = fmaf(sqrt_approx(s * ca), 1.00001f, 0.01f);
    // pixel-centre coordinates relative to the tile's first centre
    const float mxr = mx - ((float)ox + 0.5f), myr = my - ((float)oy + 0.5f);
    const float xl = fminf(fmaxf(mxr - ex, -1e4f), 1e4f);
    const float xh = fminf(fmaxf(mxr + ex, -1e4f), 1e4f);
    const float yl = fminf(fmaxf(myr - ey, -1e4f), 1e4f);
    const float yh = fminf(fmaxf(myr + ey, -1e4f), 1e4f);
    const int bx0 = max(0, (int)ceilf((xl - 7.0f) * 0.125f)), bx1 = min(WPR - 1, (int)floorf(xh * 0.125f));
    const float ibh = 1.0f / (float)BH;   // BH a power of two: exact
    const int by0 = max(0, (int)ceilf((yl - (float)(BH - 1)) * ibh)), by1 = min(RPB - 1, (int)floorf(yh * ibh));
    if (bx0 > bx1 || by0 > by1) return 0u;
    // columns bx0..bx1 of one row, times one bit per row by0..by1
    uint32_t rows = 0;
    for (int by = 0; by < RPB; by++) rows |= 1u << (by * WPR);
    rows &= ~((1u << (by0 * WPR)) - 1u) & ((1u << ((by1 + 1) * WPR)) - 1u);
    return ((2u << bx1) - (1u << bx0)) * rows;
}

// Exponent in base 2: power2 = log2(e) * power = A dx^2 + B dx dy + C dy^2
// with (A, B, C) = -log2(e) (ca / 2, cb, cc / 2), prescaled once per staged
// list entry; G = 2^power2 by the hardware exp2.  Raster forward and backward
// use these same helpers, so they take the same decisions.  The opacity test
// o G >= 1/255 is taken before the 0.99 clamp (the same decision, since
// 0.99 > 1/255).
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kPow2Min = -4.5f * 1.4426950408889634f;   // d^2 = 9

__device__ __forceinline__ float4 pair_coefs(float mx, float my, float ca, float cb, float cc)
{
    return make_float4(mx, my, __fmul_rn(-0.5f * kLog2e, ca), __fmul_rn(-kLog2e, cb));
}

__device__ __forceinline__ float pair_c2(float cc) { return __fmul_rn(-0.5f * kLog2e, cc); }

// The exponent as dy (C dy + B dx) + (A dx) dx: the two dx terms are shared
// by the pixels of one column.
struct PowX {
    float adx2, bdx;
};

__device__ __forceinline__ PowX pair_power2_x(float dx, float A, float B)
{
    return PowX{__fmul_rn(__fmul_rn(A, dx), dx), __fmul_rn(B, dx)};
}

__device__ __forceinline__ float pair_power2_y(const PowX& x, float dy, float C)
{
    return __fmaf_rn(dy, __fmaf_rn(C, dy, x.bdx), x.adx2);
}

__device__ __forceinline__ float pair_power2(float dx, float dy, float A, float B, float C)
{
    return pair_power2_y(pair_power2_x(dx, A, B), dy, C);
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// A Gaussian's mean (hi + residual lo) relative to a tile's first pixel o,
// rounded once to FP32 when a list entry is staged: (hi - o) + lo.  Its
// error is at most about one ulp of the tile-relative mean (1e-6 px within
// 16 px of the tile), like the two roundings of (p - hi) - lo.
__device__ __forceinline__ float tile_mean(float m_hi, float m_lo, int o)
{
    return __fadd_rn(__fsub_rn(m_hi, (float)o), m_lo);
}

// Pixel-centre offset from a Gaussian's mean, both relative to the tile's
// first pixel: one subtraction per pair.  The raster forward and every
// backward use these two helpers, so they agree bit for bit.
__device__ __forceinline__ float pix_offset(float pc_tile, float m_tile)
{
    return __fsub_rn(pc_tile, m_tile);
}

// Error-free transforms (Knuth TwoSum, FMA-based TwoProduct) for the
// compensated pixel-space mean.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// mean2D = f * t_u / t_z + c with t = R mu + tcam, to about 1e-12 relative:
// returns hi + lo (hi is a rounded value, lo the residual).
__device__ __forceinline__ void accurate_mean2d(const float* cam, float4 mu, float& mx, float& mx_lo, float& my,
                                                float& my_lo)
{
    float th[3], tl[3];
    const float mv[3] = {mu.x, mu.y, mu.z};
#pragma unroll
    for (int i = 0; i < 3; i++) {
        float p[3], e[3];
#pragma unroll
        for (int j = 0; j < 3; j++) {
            p[j] = __fmul_rn(cam[3 * i + j], mv[j]);
            e[j] = __fmaf_rn(cam[3 * i + j], mv[j], -p[j]);
        }
        float s1, e1, s2, e2, s3, e3;
        two_sum(p[0], p[1], s1, e1);
        two_sum(s1, p[2], s2, e2);
        two_sum(s2, cam[9 + i], s3, e3);
        th[i] = s3;
        tl[i] = ((e[0] + e[1]) + (e[2] + e1)) + (e2 + e3);
    }
    // the low-order correction needs no correctly rounded division
    const float itz = __fdividef(1.0f, th[2]);
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const float f = cam[12 + k], c = cam[14 + k];
        const float q = __fdiv_rn(th[k], th[2]);
        const float rem = __fmaf_rn(-q, th[2], th[k]);                   // exact
        const float ql = (rem + tl[k] - q * tl[2]) * itz;
        const float p = __fmul_rn(f, q);
        const float pe = __fmaf_rn(f, q, -p);
        float s, se;
        two_sum(p, c, s, se);
        const float lo = pe + f * ql + se;
        float hi, hl;
        two_sum(s, lo, hi, hl);
        if (k == 0) { mx = hi; mx_lo = hl; } else { my = hi; my_lo = hl; }
    }
}

// Transmittance before a list entry from the one after it, as a compensated
// FP32 pair (Th + Tl) / (1 - alpha): 1 - alpha is split exactly into
// om + om_err (Fast2Sum, 1 >= alpha), the quotient q = Th r uses the hardware
// reciprocal r, the remainder Th - q om is exact (one FMA), and the low part
// (remainder + Tl - q om_err) r carries what q misses, so the pair stays close
// to the exact quotient through hundreds of divisions.  The pair is not
// renormalised: Th is always the last quotient and Tl stays near its ulp,
// since each step's remainder is at most about an ulp of Th.  Returns r.
__device__ __forceinline__ float div_one_minus(float alpha, float& Th, float& Tl)
{
    const float om = __fsub_rn(1.0f, alpha);
    const float om_err = __fsub_rn(-alpha, __fsub_rn(om, 1.0f));
    const float r = __fdividef(1.0f, om);
    const float q = __fmul_rn(Th, r);
    const float rem = __fmaf_rn(-q, om, Th);
    Tl = __fmul_rn(__fmaf_rn(-q, om_err, __fadd_rn(rem, Tl)), r);
    Th = q;
    return r;
}

constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;

// --------------------------------------------------------------------------
// Real SH basis up to degree 3 (3DGS sign convention).
// --------------------------------------------------------------------------
__device__ __forceinline__ void sh_basis(float x, float y, float z, float* Y)
{
    const float c0 = 0.28209479177387814f, c1 = 0.4886025119029199f;
    const float c20 = 1.0925484305920792f, c22 = 0.31539156525252005f, c24 = 0.5462742152960396f;
    const float c30 = 0.5900435899266435f, c31 = 2.890611442640554f, c32 = 0.4570457994644658f;
    const float c33 = 0.3731763325901154f, c35 = 1.445305721320277f;
    float xx = x * x, yy = y * y, zz = z * z;
    Y[0] = c0;
    Y[1] = -c1 * y;
    Y[2] = c1 * z;
    Y[3] = -c1 * x;
    Y[4] = c20 * x * y;
    Y[5] = -c20 * y * z;
    Y[6] = c22 * (2.0f * zz - xx - yy);
    Y[7] = -c20 * x * z;
    Y[8] = c24 * (xx - yy);
    Y[9] = -c30 * y * (3.0f * xx - yy);
    Y[10] = c31 * x * y * z;
    Y[11] = -c32 * y * (4.0f * zz - xx - yy);
    Y[12] = c33 * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
    Y[13] = -c32 * x * (4.0f * zz - xx - yy);
    Y[14] = c35 * z * (xx - yy);
    Y[15] = -c30 * x * (xx - 3.0f * yy);
}

// d/d(x, y, z) of sum_k w[k] Y_k, with the direction treated as a free vector.
__device__ __forceinline__ void sh_basis_vjp(float x, float y, float z, const float* w, float& gx, float& gy,
                                             float& gz)
{
    const float c1 = 0.4886025119029199f;
    const float c20 = 1.0925484305920792f, c22 = 0.31539156525252005f, c24 = 0.5462742152960396f;
    const float c30 = 0.5900435899266435f, c31 = 2.890611442640554f, c32 = 0.4570457994644658f;
    const float c33 = 0.3731763325901154f, c35 = 1.445305721320277f;
    float xx = x * x, yy = y * y, zz = z * z;
    gx = 0.f; gy = 0.f; gz = 0.f;
    gy += -c1 * w[1];
    gz += c1 * w[2];
    gx += -c1 * w[3];
    gx += c20 * y * w[4];           gy += c20 * x * w[4];
    gy += -c20 * z * w[5];          gz += -c20 * y * w[5];
    gx += -2.f * c22 * x * w[6];    gy += -2.f * c22 * y * w[6];   gz += 4.f * c22 * z * w[6];
    gx += -c20 * z * w[7];          gz += -c20 * x * w[7];
    gx += 2.f * c24 * x * w[8];     gy += -2.f * c24 * y * w[8];
    gx += -c30 * 6.f * x * y * w[9];
    gy += -c30 * (3.f * xx - 3.f * yy) * w[9];
    gx += c31 * y * z * w[10];      gy += c31 * x * z * w[10];     gz += c31 * x * y * w[10];
    gx += -c32 * (-2.f * x * y) * w[11];
    gy += -c32 * (4.f * zz - xx - 3.f * yy) * w[11];
    gz += -c32 * (8.f * y * z) * w[11];
    gx += c33 * (-6.f * x * z) * w[12];
    gy += c33 * (-6.f * y * z) * w[12];
    gz += c33 * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
    gx += -c32 * (4.f * zz - 3.f * xx - yy) * w[13];
    gy += -c32 * (-2.f * x * y) * w[13];
    gz += -c32 * (8.f * x * z) * w[13];
    gx += c35 * 2.f * x * z * w[14];
    gy += -c35 * 2.f * y * z * w[14];
    gz += c35 * (xx - yy) * w[14];
    gx += -c30 * (3.f * xx - 3.f * yy) * w[15];
    gy += -c30 * (-6.f * x * y) * w[15];
}

__device__ __forceinline__ float bf16_lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t u) { return __uint_as_float(u & 0xFFFF0000u); }

}  // namespace gs
