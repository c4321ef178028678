// project_fwd.cu -- projection forward fused with the exact tile count
// (VkSplat Sec. 4.1: the number of intersected tiles is computed in the
// projection-forward pass).  One thread per Gaussian, looping over the views
// of its scene: the parameters are read from HBM once, the SH coefficients
// once per surviving (view, Gaussian) pair from the first read's cached
// lines; SoA float4 loads; the records of pair (v, g) go to the view-major
// pair pair_base[v] + g, so consecutive threads write consecutive records,
// and its tile count to the Gaussian-major pair q (a Gaussian's counts for
// all views of its scene side by side).  The traversal that counts the tiles
// also adds one to the counter of every tile it meets (the per-tile list
// lengths from which the sort places each tile's list), keeping the old value
// as the pair's rank in that tile's list when the pair meets few tiles, and
// keeps the pair's tile span for the emission.
#include "gs_internal.cuh"

namespace gs {

// One (view, Gaussian) pair: tile count, and for a pair that meets a tile its
// projected record and binning geometry.
__device__ __forceinline__ void project_pair(const ViewDesc& vd, int tw, int th, const SceneDesc& sc, int sh_bf16,
                                             const float* __restrict__ camp, float2 lim, int64_t g, int64_t p,
                                             int64_t qi,
                                             const float4& mu, const BinGauss& bgs, const float4& so,
                                             uint32_t* __restrict__ count, uint32_t* __restrict__ tile_cnt,
                                             uint32_t* __restrict__ tile_over, ProjRec* __restrict__ rec,
                                             uint4* __restrict__ span, uint4* __restrict__ rank)
{
    float cam[16];
#pragma unroll
    for (int i = 0; i < 16; i++) cam[i] = __ldg(camp + i);
    BinGeom bg;
    bin_view(mu, bgs, cam, lim, bg);
    uint32_t cnt = 0;
    // The first two bands of the traversal are kept for the emission; the
    // tiles of any later band (the pair is then not ranked, below) are
    // counted as they are met.
    uint32_t nb = 0, c0 = 0, c1 = 0, r0 = 0, r1 = 0;
    bool rows = true;
    const uint32_t TX = (uint32_t)vd.TX;
    uint32_t* __restrict__ to = tile_over + vd.tile_base;
    if (bg.valid)
        cnt = scanline_bands(bg, tw, th, vd.TX, vd.TY, [&](bool rw, int coord, int lo, int hi) {
            rows = rw;
            const uint32_t pk = (uint32_t)lo | ((uint32_t)hi << 16);
            if (nb == 0) { c0 = (uint32_t)coord; r0 = pk; }
            else if (nb == 1) { c1 = (uint32_t)coord; r1 = pk; }
            else
                for (int t = lo; t <= hi; t++) atomicAdd(to + (rw ? coord * TX + t : t * TX + coord), 1u);
            nb = min(nb + 1u, 3u);
        });
    count[qi] = cnt;
    if (cnt == 0) return;
    // A pair of at most kRankMax tiles in one or two bands takes its place in
    // each tile's list here (the counter's old value), so that the emission
    // needs no atomic for it; the others are counted apart and placed by the
    // emission after the ranked entries.
    const bool ranked = cnt <= kRankMax && nb <= 2;
    uint32_t rk[kRankMax] = {0u, 0u, 0u, 0u};
    if (ranked) {
        uint32_t* __restrict__ tc = tile_cnt + vd.tile_base;
#pragma unroll
        for (uint32_t u = 0; u < kRankMax; u++)
            if (u < cnt) rk[u] = atomicAdd(tc + span_tile(u, rows, TX, c0, c1, r0, r1), 1u);
    } else {
        // the tiles of the first two bands
        const uint32_t n01 = ((r0 >> 16) - (r0 & 0xFFFFu) + 1u) + (nb > 1 ? (r1 >> 16) - (r1 & 0xFFFFu) + 1u : 0u);
        for (uint32_t u = 0; u < n01; u++) atomicAdd(to + span_tile(u, rows, TX, c0, c1, r0, r1), 1u);
    }
    span[qi] = span_pack(bg.mant, nb, rows, ranked, c0, c1, r0, r1, bg);
    // stored at once (holding the ranks through the colour computation
    // measured slower: the registers they take cost spills)
    if (ranked) rank[qi] = make_uint4(rk[0], rk[1], rk[2], rk[3]);

    // conic = inverse of the 2D covariance (one hardware reciprocal of the
    // determinant, det >= 0.09 by the low-pass: a few ulp)
    const float idet = __fdividef(1.0f, bg.det);
    const float ca = bg.c * idet, cb = -bg.b * idet, cc = bg.a * idet;

    // colour from degree-3 SH at the view direction (mu - camera centre)
    const float cpx = -(cam[0] * cam[9] + cam[3] * cam[10] + cam[6] * cam[11]);
    const float cpy = -(cam[1] * cam[9] + cam[4] * cam[10] + cam[7] * cam[11]);
    const float cpz = -(cam[2] * cam[9] + cam[5] * cam[10] + cam[8] * cam[11]);
    float dx = mu.x - cpx, dy = mu.y - cpy, dz = mu.z - cpz;
    const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
    dx *= inv; dy *= inv; dz *= inv;
    float Y[16];
    sh_basis(dx, dy, dz, Y);
    // coefficient i = 3 k + c adds to channel c in k order, one stored
    // chunk at a time (the 48 values are never live together)
    float col[3] = {0.5f, 0.5f, 0.5f};
    if (sh_bf16) {
        const uint4* s8 = reinterpret_cast<const uint4*>(sc.sh);
#pragma unroll
        for (int j = 0; j < 6; j++) {
            const uint4 c = s8[j * sc.n + g];
            const uint32_t w[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
            for (int h = 0; h < 8; h++) {
                const int i = 8 * j + h;
                const float v = (h & 1) ? bf16_hi(w[h >> 1]) : bf16_lo(w[h >> 1]);
                col[i % 3] = fmaf(v, Y[i / 3], col[i % 3]);
            }
        }
    } else {
        const float4* s4 = reinterpret_cast<const float4*>(sc.sh);
#pragma unroll
        for (int j = 0; j < 12; j++) {
            const float4 c = s4[j * sc.n + g];
            const float w[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
            for (int h = 0; h < 4; h++) {
                const int i = 4 * j + h;
                col[i % 3] = fmaf(w[h], Y[i / 3], col[i % 3]);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 3; c++) col[c] = fmaxf(col[c], 0.0f);
    // residuals of the binning mean against the compensated mean
    float amx, amx_lo, amy, amy_lo;
    accurate_mean2d(cam, mu, amx, amx_lo, amy, amy_lo);
    const float rx = (amx - bg.mx) + amx_lo, ry = (amy - bg.my) + amy_lo;
    ProjRec r;
    r.a = make_float4(bg.mx, bg.my, ca, cb);
    r.b = make_float4(cc, so.w, col[0], col[1]);
    r.c = make_float4(col[2], bg.tz, rx, ry);
    rec[p] = r;
}

// 4 CTAs per SM: the register cap (64) costs some spills but raises occupancy
// (0.636 vs 0.651 ms at 3 CTAs and 80 registers for 3M Gaussians, 4 views)
__global__ void __launch_bounds__(256, 4) k_project_fwd(Views V, Scenes S, const float* __restrict__ cams,
                                                     uint32_t* __restrict__ count, uint32_t* __restrict__ tile_cnt,
                                                     ProjRec* __restrict__ rec, uint4* __restrict__ span,
                                                     uint4* __restrict__ rank,
                                                     WsHeader* __restrict__ hdr)
{
    // the views' field-of-view limits, once per block (two correctly
    // rounded divisions a view instead of a pair)
    __shared__ float2 slim[kMaxViews];
    for (int v = threadIdx.x; v < V.n; v += blockDim.x) slim[v] = fov_limits(cams + 16 * v, V.v[v].W, V.v[v].H);
    __syncthreads();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= S.total) return;
    int s = 0;
    while (s + 1 < S.n && t >= S.s[s + 1].base) s++;
    const SceneDesc& sc = S.s[s];
    const int64_t g = t - sc.base;
    const int64_t n = sc.n;
    const float4 mu = sc.geom[g];
    const float4 q = sc.geom[n + g];
    const float4 so = sc.geom[2 * n + g];
    const bool finite = isfinite(mu.x) && isfinite(mu.y) && isfinite(mu.z) && isfinite(q.x) && isfinite(q.y) &&
                        isfinite(q.z) && isfinite(q.w) && isfinite(so.x) && isfinite(so.y) && isfinite(so.z) &&
                        isfinite(so.w);
    if (!finite) atomicOr(&hdr->status, GS_STATUS_NONFINITE);
    const int nv = V.nv[s];
    const int64_t q0 = V.qbase[s] + g * nv;
    // the view-independent part of the binning (cull radius, 3D covariance)
    BinGauss bgs;
    bin_gauss(q, so, bgs);
    for (int k = 0; k < nv; k++) {
        const int v = V.view_of[s][k];
        const ViewDesc& vd = V.v[v];
        const int64_t p = vd.pair_base + g;
        if (!finite) {
            count[q0 + k] = 0;
            continue;
        }
        project_pair(vd, V.tw, V.th, sc, S.sh_bf16, cams + 16 * v, slim[v], g, p, q0 + k, mu, bgs, so, count,
                     tile_cnt, tile_cnt + V.tiles, rec, span, rank);
    }
}

void launch_project_fwd(const Plan& P, const Scenes& S, const float* cams, const WsPtrs& w, cudaStream_t st)
{
    const int T = 256;
    const int64_t blocks = (S.total + T - 1) / T;
    if (blocks == 0) return;
    k_project_fwd<<<(unsigned)blocks, T, 0, st>>>(P.views, S, cams, w.count, w.tile_cnt, w.rec, w.span, w.rank, w.hdr);
}

}  // namespace gs
