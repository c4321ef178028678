// raster_bwd.cu -- rasterization backward parallel over Gaussians (VkSplat
// Sec. 4.2, first implementation; Fig. 2), with no pixel-level atomics.
//
// One CTA (4 warps) per tile.  The tile's list (up to the largest n_last of
// its pixels) is processed in batches of S Gaussians, S chosen per tile by
// the paper's rule S = roundup32(sqrt(N P)) capped at 128 (N = list length,
// P = pixels), or fixed by the tuning.  For each batch:
//
//  Phase A (pixels across threads): transmittance is recomputed front to
//    back from the running per-pixel state -- T as a compensated FP32 pair,
//    the blended colour prefix with Neumaier compensation -- and the state
//    (T, S) at the end of every 32-Gaussian sub-batch is kept in shared
//    memory, where S = C_image - prefix is the colour still to come.
//  Phase B (Gaussians across threads): warp k takes sub-batch k, lane l its
//    l-th Gaussian.  The lanes form a wavefront over the pixels: at step s
//    lane l handles pixel s - (31 - l), receives (T, S) from lane l + 1 by
//    warp shuffle, walks back over its own Gaussian (T_before = T / (1 - a),
//    S += c a T_before) and hands the state on.  Each lane accumulates its
//    Gaussian's nine gradients in registers; when S < 128 the warps split the
//    pixels instead and the partial sums are added in a fixed order.
//
// Output: one gradient record per intersection, at its emission slot, so
// the projection backward reads each Gaussian's records contiguously.  The
// result is deterministic (no atomics, fixed summation order).
#include "gs_internal.cuh"

namespace gs {

struct BwdSmem {
    float4* runA;   // [P] (T hi, T lo, prefix r, prefix g)
    float4* runB;   // [P] (prefix b, comp r, comp g, comp b)
    float4* pimg;   // [P] (C r, g, b, -)
    float4* pdl;    // [P] (dL/dC r, g, b, n_last bits)
    float4* st;     // [4][P] state (T, S r, S g, S b) after each sub-batch
    float4* gA;     // [128] (mx, my relative to the tile's first pixel, ca, cb)
    float4* gB;     // [128] (cc, o, r, g)
    float* gC;      // [128] blue
    uint32_t* ge;   // [128] emission slot
    float* red;     // [128][9] partial gradients
    int* misc;
};

__host__ __device__ constexpr size_t bwd_smem_bytes(int P)
{
    return (size_t)16 * P * 4 + (size_t)16 * 4 * P + 128 * (16 + 16 + 4 + 4) + 128 * 9 * 4 + 16;
}

__device__ __forceinline__ void neumaier_add(float& s, float& c, float x)
{
    const float t = s + x;
    c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
    s = t;
}

template <int P>
__global__ void __launch_bounds__(kBwdThreads) k_raster_bwd(Views V, const uint32_t* __restrict__ order,
                                                            const uint2* __restrict__ ranges,
                                                            const uint32_t* __restrict__ vals_sorted,
                                                            const uint32_t* __restrict__ pid_sorted,
                                                            const ProjRec* __restrict__ rec,
                                                            const float* __restrict__ image,
                                                            const float* __restrict__ dl,
                                                            const uint32_t* __restrict__ nlast,
                                                            GradRec* __restrict__ gradrec, int fixed_S)
{
    extern __shared__ float4 smem4[];
    BwdSmem sm;
    sm.runA = smem4;
    sm.runB = sm.runA + P;
    sm.pimg = sm.runB + P;
    sm.pdl = sm.pimg + P;
    sm.st = sm.pdl + P;
    sm.gA = sm.st + 4 * P;
    sm.gB = sm.gA + 128;
    sm.gC = reinterpret_cast<float*>(sm.gB + 128);
    sm.ge = reinterpret_cast<uint32_t*>(sm.gC + 128);
    sm.red = reinterpret_cast<float*>(sm.ge + 128);
    sm.misc = reinterpret_cast<int*>(sm.red + 128 * 9);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t gt = order[blockIdx.x];   // longest lists first
    const int v = view_of_tile(V, gt);
    const ViewDesc& vd = V.v[v];
    const int lt = (int)(gt - vd.tile_base);
    const int tw = V.tw;
    const int ox = (lt % vd.TX) * tw, oy = (lt / vd.TX) * V.th;
    const uint2 r = ranges[gt];
    const uint32_t start = r.x, ntile = r.y - r.x;

    if (tid == 0) sm.misc[0] = 0;
    __syncthreads();
    // per-pixel inputs
    int my_max = 0;
    for (int pi = tid; pi < P; pi += kBwdThreads) {
        const int px = ox + pi % tw, py = oy + pi / tw;
        float4 im = make_float4(0.f, 0.f, 0.f, 0.f), d = make_float4(0.f, 0.f, 0.f, 0.f);
        uint32_t nl = 0;
        if (px < vd.W && py < vd.H) {
            const int64_t pix = vd.pix_base + (int64_t)py * vd.W + px;
            im = make_float4(image[3 * pix], image[3 * pix + 1], image[3 * pix + 2], 0.f);
            d = make_float4(dl[3 * pix], dl[3 * pix + 1], dl[3 * pix + 2], 0.f);
            nl = nlast[pix];
        }
        d.w = __uint_as_float(nl);
        sm.pimg[pi] = im;
        sm.pdl[pi] = d;
        sm.runA[pi] = make_float4(1.f, 0.f, 0.f, 0.f);
        sm.runB[pi] = make_float4(0.f, 0.f, 0.f, 0.f);
        my_max = max(my_max, (int)nl);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) my_max = max(my_max, __shfl_xor_sync(0xffffffffu, my_max, o));
    if (lane == 0) atomicMax(&sm.misc[0], my_max);
    __syncthreads();
    const uint32_t L = min(ntile, (uint32_t)sm.misc[0]);

    int S = fixed_S;
    if (S <= 0) {
        const float x = sqrtf((float)L * (float)P);
        S = ((int)ceilf(x) + 31) & ~31;
    }
    S = min(max(S, 32), 128);
    const int nsub = S / 32;
    const int ngroups = (nsub == 3) ? 1 : 4 / nsub;
    const int glen = P / ngroups;

    for (uint32_t bb = 0; bb < L; bb += S) {
        const int cnt = (int)min((uint32_t)S, L - bb);
        if (tid < cnt) {
            const uint32_t k = start + bb + tid;
            const ProjRec q = rec[pid_sorted[k]];
            sm.gA[tid] = make_float4(tile_mean(q.a.x, q.c.z, ox), tile_mean(q.a.y, q.c.w, oy), q.a.z, q.a.w);
            sm.gB[tid] = q.b;
            sm.gC[tid] = q.c.x;
            sm.ge[tid] = vals_sorted[k];
        }
        __syncthreads();

        // ---------------- Phase A: pixel-parallel forward recompute ----------------
        const int nsub_used = (cnt + 31) >> 5;
        for (int pi = tid; pi < P; pi += kBwdThreads) {
            float4 ra = sm.runA[pi], rb = sm.runB[pi];
            float Th = ra.x, Tl = ra.y;
            float ps0 = ra.z, ps1 = ra.w, ps2 = rb.x, pc0 = rb.y, pc1 = rb.z, pc2 = rb.w;
            const float4 d = sm.pdl[pi];
            const float4 im = sm.pimg[pi];
            const uint32_t nl = __float_as_uint(d.w);
            // pixel centre relative to the tile's first pixel (the staged means are too)
            const float fx = (float)(pi % tw) + 0.5f, fy = (float)(pi / tw) + 0.5f;
            for (int k = 0; k < nsub_used; k++) {
                const int j1 = min(cnt, 32 * k + 32);
                for (int j = 32 * k; j < j1; j++) {
                    if (bb + j >= nl) break;
                    const float4 a = sm.gA[j];
                    const float4 b = sm.gB[j];
                    const float dx = pix_offset(fx, a.x), dy = pix_offset(fy, a.y);
                    const float4 pc = pair_coefs(a.x, a.y, a.z, a.w, b.x);
                    const float p2 = pair_power2(dx, dy, pc.z, pc.w, pair_c2(b.x));
                    if (p2 < kPow2Min) continue;
                    const float G = ex2_approx(p2);
                    const float araw = __fmul_rn(b.y, G);
                    if (araw < kAlphaMin) continue;
                    const float alpha = fminf(kAlphaMax, araw);
                    const float wgt = alpha * Th;
                    neumaier_add(ps0, pc0, b.z * wgt);
                    neumaier_add(ps1, pc1, b.w * wgt);
                    neumaier_add(ps2, pc2, sm.gC[j] * wgt);
                    const float om = __fsub_rn(1.0f, alpha);
                    const float om_err = __fsub_rn(-alpha, __fsub_rn(om, 1.0f));
                    const float pr = __fmul_rn(Th, om);
                    const float pe = __fmaf_rn(Th, om, -pr);
                    const float lo = __fmaf_rn(Th, om_err, __fmaf_rn(Tl, om, pe));
                    const float hi = __fadd_rn(pr, lo);
                    Tl = __fsub_rn(lo, __fsub_rn(hi, pr));
                    Th = hi;
                }
                sm.st[k * P + pi] =
                    make_float4(Th + Tl, (im.x - ps0) - pc0, (im.y - ps1) - pc1, (im.z - ps2) - pc2);
            }
            sm.runA[pi] = make_float4(Th, Tl, ps0, ps1);
            sm.runB[pi] = make_float4(ps2, pc0, pc1, pc2);
        }
        __syncthreads();

        // ---------------- Phase B: Gaussian-parallel wavefront ----------------
        const int sub = warp % nsub;
        const int pg = warp / nsub;
        const bool warp_on = (nsub != 3 || warp < 3) && sub < nsub_used;
        const int j = sub * 32 + lane;
        const bool act = warp_on && j < cnt;
        float g_mx = 0.f, g_my = 0.f, g_ca = 0.f, g_cb = 0.f, g_cc = 0.f, g_o = 0.f, g_r = 0.f, g_g = 0.f,
              g_b = 0.f;
        if (warp_on) {
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
            float cbl = 0.f;
            if (act) { a = sm.gA[j]; b = sm.gB[j]; cbl = sm.gC[j]; }
            const uint32_t myidx = bb + j;
            const int p0 = pg * glen;
            float T = 1.f, S0 = 0.f, S1 = 0.f, S2 = 0.f;
            const int nsteps = glen + 31;
            for (int s = 0; s < nsteps; s++) {
                float Ti = __shfl_down_sync(0xffffffffu, T, 1);
                float Si0 = __shfl_down_sync(0xffffffffu, S0, 1);
                float Si1 = __shfl_down_sync(0xffffffffu, S1, 1);
                float Si2 = __shfl_down_sync(0xffffffffu, S2, 1);
                if (lane == 31 && s < glen) {
                    const float4 q = sm.st[sub * P + p0 + s];
                    Ti = q.x; Si0 = q.y; Si1 = q.z; Si2 = q.w;
                }
                const int pl = s - (31 - lane);
                if (act && pl >= 0 && pl < glen) {
                    const int pi = p0 + pl;
                    const float4 d = sm.pdl[pi];
                    if (myidx < __float_as_uint(d.w)) {
                        const float dx = pix_offset((float)(pi % tw) + 0.5f, a.x);
                        const float dy = pix_offset((float)(pi / tw) + 0.5f, a.y);
                        const float4 pc = pair_coefs(a.x, a.y, a.z, a.w, b.x);
                        const float p2 = pair_power2(dx, dy, pc.z, pc.w, pair_c2(b.x));
                        if (p2 >= kPow2Min) {
                            const float G = ex2_approx(p2);
                            const float araw = __fmul_rn(b.y, G);
                            const float alpha = fminf(kAlphaMax, araw);
                            if (araw >= kAlphaMin) {
                                const float om = 1.0f - alpha;
                                const float rom = 1.0f / om;
                                const float Tb = Ti * rom;
                                const float wgt = alpha * Tb;
                                g_r = fmaf(wgt, d.x, g_r);
                                g_g = fmaf(wgt, d.y, g_g);
                                g_b = fmaf(wgt, d.z, g_b);
                                float da = d.x * (b.z * Tb - Si0 * rom);
                                da = fmaf(d.y, b.w * Tb - Si1 * rom, da);
                                da = fmaf(d.z, cbl * Tb - Si2 * rom, da);
                                Si0 = fmaf(b.z, wgt, Si0);
                                Si1 = fmaf(b.w, wgt, Si1);
                                Si2 = fmaf(cbl, wgt, Si2);
                                Ti = Tb;
                                if (araw <= kAlphaMax) {
                                    g_o = fmaf(da, G, g_o);
                                    const float dp = da * araw;
                                    g_ca = fmaf(-0.5f * dx * dx, dp, g_ca);
                                    g_cb = fmaf(-dx * dy, dp, g_cb);
                                    g_cc = fmaf(-0.5f * dy * dy, dp, g_cc);
                                    g_mx = fmaf(fmaf(a.z, dx, a.w * dy), dp, g_mx);
                                    g_my = fmaf(fmaf(a.w, dx, b.x * dy), dp, g_my);
                                }
                            }
                        }
                    }
                }
                T = Ti; S0 = Si0; S1 = Si1; S2 = Si2;
            }
        }
        if (ngroups == 1) {
            if (act) {
                GradRec o;
                o.a = make_float4(g_mx, g_my, g_ca, g_cb);
                o.b = make_float4(g_cc, g_o, g_r, g_g);
                o.c = make_float4(g_b, 0.f, 0.f, 0.f);
                gradrec[sm.ge[j]] = o;
            }
        } else {
            if (act) {
                float* rr = sm.red + (pg * S + j) * 9;
                rr[0] = g_mx; rr[1] = g_my; rr[2] = g_ca; rr[3] = g_cb; rr[4] = g_cc;
                rr[5] = g_o; rr[6] = g_r; rr[7] = g_g; rr[8] = g_b;
            }
            __syncthreads();
            if (tid < cnt) {
                float acc[9];
#pragma unroll
                for (int i = 0; i < 9; i++) acc[i] = 0.f;
                for (int q = 0; q < ngroups; q++) {
                    const float* rr = sm.red + (q * S + tid) * 9;
#pragma unroll
                    for (int i = 0; i < 9; i++) acc[i] += rr[i];
                }
                GradRec o;
                o.a = make_float4(acc[0], acc[1], acc[2], acc[3]);
                o.b = make_float4(acc[4], acc[5], acc[6], acc[7]);
                o.c = make_float4(acc[8], 0.f, 0.f, 0.f);
                gradrec[sm.ge[tid]] = o;
            }
        }
        __syncthreads();
    }
    // entries past every pixel's last blended pair receive zero gradients
    for (uint32_t k = start + L + tid; k < r.y; k += kBwdThreads) {
        GradRec o;
        o.a = o.b = o.c = make_float4(0.f, 0.f, 0.f, 0.f);
        gradrec[vals_sorted[k]] = o;
    }
}

void launch_raster_bwd_px(const Plan& P, const WsPtrs& w, const float* bg, const float* dl, cudaStream_t st);

void launch_raster_bwd(const Plan& P, const WsPtrs& w, const float* image, const float* dl, cudaStream_t st)
{
    if (P.tuning.bwd_impl == 0 || P.tuning.bwd_impl == 2) {
        const float* bg = reinterpret_cast<const float*>(reinterpret_cast<const char*>(w.hdr) + offsetof(WsHeader, bg));
        if (P.tuning.bwd_impl == 0) launch_raster_bwd_px(P, w, bg, dl, st);
        else launch_raster_bwd2(P, w, bg, dl, st);
        return;
    }
    const Views& V = P.views;
    const int np = V.tw * V.th;
    const unsigned grid = (unsigned)V.tiles;
    const int fixed = P.tuning.bwd_batch;
#define GS_RB(NP)                                                                                           \
    do {                                                                                                    \
        const size_t sb = bwd_smem_bytes(NP);                                                               \
        static bool attr_set = false;                                                                       \
        if (!attr_set) {                                                                                    \
            cudaFuncSetAttribute(k_raster_bwd<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);   \
            attr_set = true;                                                                                \
        }                                                                                                   \
        k_raster_bwd<NP><<<grid, kBwdThreads, sb, st>>>(V, w.tile_order, w.ranges, w.vals_sorted, w.pid_sorted, w.rec, image, \
                                                        dl, w.nlast, w.gradrec, fixed);                     \
    } while (0)
    if (np == 64) GS_RB(64);
    else if (np == 256) GS_RB(256);
    else GS_RB(512);
#undef GS_RB
}

}  // namespace gs

// ===========================================================================
// Second implementation: pixels across threads, per-Gaussian gradients
// reduced across each warp's pixels by shuffles (no atomics).
//
// One CTA per tile, one thread per pixel, each warp an 8x4 pixel block (so a
// small Gaussian touches few warps).  Every pixel walks its own list prefix
// back to front from its last blended entry: T before an entry is recovered
// by a compensated division of T after it by (1 - alpha) (div_one_minus:
// hardware reciprocal, exact remainder, carried low part), and the colour
// still to come S grows from T_final * bg without cancellation; only its
// projection U = dL/dC . S is carried, since dL/dalpha needs no more.  The
// list is staged BB entries at a time with a mask of the warp blocks each
// entry's 3-sigma box touches; a warp visits only its entries, and for an
// entry that
// at least one of its pixels blended it sums nine values over its 32 pixels
// with a halving butterfly (12 shuffles; afterwards nine lanes each hold one
// fully reduced value) into its own shared-memory slot: the opacity and
// colour gradients and the moments dx dp, dy dp, dx^2 dp, dx dy dp, dy^2 dp
// of dp = dL/dpower, from which the mean and conic gradients follow per
// entry (the mean gradient is the conic times the first two).  After each
// batch the warps' slots are added in warp order and written to each entry's
// emission slot, so the result does not depend on scheduling.
// ===========================================================================

namespace gs {

// Halving-butterfly reduction of nine per-lane values over a warp: returns
// the lane's share of the result; `vi` (from bfly_index) says which of the
// nine sums it is (-1: none).
__device__ __forceinline__ float bfly9(const float* v, int lane)
{
    const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4, h1 = lane & 2;
    float k[5];
#pragma unroll
    for (int i = 0; i < 5; i++) {
        const float lo = v[i], hi = i < 4 ? v[5 + i] : 0.f;
        k[i] = (h4 ? hi : lo) + __shfl_xor_sync(0xffffffffu, h4 ? lo : hi, 16);
    }
    float m[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const float lo = k[i], hi = i < 2 ? k[3 + i] : 0.f;
        m[i] = (h3 ? hi : lo) + __shfl_xor_sync(0xffffffffu, h3 ? lo : hi, 8);
    }
    float nn[2];
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const float lo = m[i], hi = i < 1 ? m[2 + i] : 0.f;
        nn[i] = (h2 ? hi : lo) + __shfl_xor_sync(0xffffffffu, h2 ? lo : hi, 4);
    }
    float p = (h1 ? nn[1] : nn[0]) + __shfl_xor_sync(0xffffffffu, h1 ? nn[0] : nn[1], 2);
    return p + __shfl_xor_sync(0xffffffffu, p, 1);
}

__device__ __forceinline__ int bfly_index(int lane)
{
    if (lane & 1) return -1;
    const int mi = ((lane & 4) ? 2 : 0) + ((lane & 2) ? 1 : 0);
    if (mi == 3) return -1;
    const int ki = (lane & 8) ? (mi < 2 ? 3 + mi : -1) : mi;
    if (ki < 0) return -1;
    return (lane & 16) ? (ki < 4 ? 5 + ki : -1) : ki;
}

// BS threads per tile, each owning PPT pixels of its warp's 8 x (4 PPT)
// block (lane (x, y) holds rows y, y + 4, ...): the PPT pixels' nine values
// are summed in the lane before one butterfly per visit.
template <int BS, int TW, int PPT>
__global__ void __launch_bounds__(BS) k_raster_bwd_px(Views V, const uint32_t* __restrict__ order,
                                                      const uint2* __restrict__ ranges,
                                                      const uint32_t* __restrict__ vals_sorted,
                                                      const uint32_t* __restrict__ pid_sorted,
                                                      const ProjRec* __restrict__ rec,
                                                      const float* __restrict__ tfinal,
                                                      const float* __restrict__ bg, const float* __restrict__ dl,
                                                      const uint32_t* __restrict__ nlast,
                                                      GradRec* __restrict__ gradrec, uint32_t* __restrict__ status,
                                                      uint32_t cap)
{
    constexpr int NW = BS / 32;
    constexpr int BH = 4 * PPT;            // warp block height, pixels
    constexpr int TH = BS * PPT / TW;      // tile height, pixels
    constexpr int WPR = TW / 8;            // warp blocks per tile row
    constexpr int RPB = TH / BH;           // rows of warp blocks
    constexpr int BB = NW <= 8 ? 96 : 64;  // list entries per staged batch
    constexpr int IPT = (BB + BS - 1) / BS;   // staged entries per thread
    __shared__ float4 sA[2][BB];
    __shared__ float4 sB[2][BB];
    __shared__ float4 sD[2][BB];          // (conic a, b, c, blue)
    __shared__ uint32_t sE[2][BB];
    __shared__ uint32_t sM[2][BB];
    __shared__ float part[NW][BB][9];
    __shared__ int smax[NW];

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t gt = order[blockIdx.x];   // longest lists first
    const int v = view_of_tile(V, gt);
    const ViewDesc& vd = V.v[v];
    const int lt = (int)(gt - vd.tile_base);
    const int ox = (lt % vd.TX) * TW, oy = (lt / vd.TX) * TH;
    const int px = ox + (w % WPR) * 8 + (lane & 7);
    const int py0 = oy + (w / WPR) * BH + (lane >> 3);
    const uint32_t wbit = 1u << w;
    const uint2 r = range_at(ranges, gt, cap, status);
    // pixel centres relative to the tile's first pixel (the staged means are too)
    const float fx = (float)(px - ox) + 0.5f;
    const int vi = bfly_index(lane);

    // per pixel k (row py0 + 4k): last blended entry, compensated T after
    // it, dL/dC, and U = sum_c dL/dC_c S_c with S_c the colour still to come
    // behind an entry (from T_final bg_c): dL/dalpha = T dL/dC . col -
    // U / (1 - alpha)
    uint32_t nl[PPT];
    float Th[PPT], Tl[PPT], d0[PPT], d1[PPT], d2[PPT], U[PPT], fy[PPT];
    int mx_nl = 0;
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        const int py = py0 + 4 * k;
        fy[k] = (float)(py - oy) + 0.5f;
        nl[k] = 0;
        Th[k] = 1.f; Tl[k] = 0.f; d0[k] = 0.f; d1[k] = 0.f; d2[k] = 0.f; U[k] = 0.f;
        if (px < vd.W && py < vd.H) {
            const int64_t pix = vd.pix_base + (int64_t)py * vd.W + px;
            nl[k] = nlast[pix];
            Th[k] = tfinal[pix];
            d0[k] = dl[3 * pix]; d1[k] = dl[3 * pix + 1]; d2[k] = dl[3 * pix + 2];
        }
        if (bg) U[k] = Th[k] * fmaf(d0[k], bg[0], fmaf(d1[k], bg[1], d2[k] * bg[2]));
        mx_nl = max(mx_nl, (int)nl[k]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx_nl = max(mx_nl, __shfl_xor_sync(0xffffffffu, mx_nl, o));
    if (lane == 0) smax[w] = mx_nl;
    __syncthreads();
    int L = 0;
#pragma unroll
    for (int i = 0; i < NW; i++) L = max(L, smax[i]);
    L = min(L, (int)(r.y - r.x));

    // Batches from the back; the batch below the current one is gathered into
    // registers while the current one is processed, then stored to the other
    // buffer: two barriers per batch.  An entry's mask keeps the warps whose
    // block its box touches and one of whose pixels blended at or past it:
    // exactly the warps that visit it.
    auto stage = [&](int bbx, int buf, int i, const ProjRec& q, uint32_t e) {
        uint32_t live = 0;
#pragma unroll
        for (int k = 0; k < NW; k++) live |= (bbx + i < smax[k] ? 1u : 0u) << k;
        sA[buf][i] = pair_coefs(tile_mean(q.a.x, q.c.z, ox), tile_mean(q.a.y, q.c.w, oy), q.a.z, q.a.w, q.b.x);
        sB[buf][i] = make_float4(pair_c2(q.b.x), q.b.y, q.b.z, q.b.w);
        sD[buf][i] = make_float4(q.a.z, q.a.w, q.b.x, q.c.x);
        sE[buf][i] = e;
        sM[buf][i] = warp_block_mask(q.a.x, q.a.y, q.a.z, q.a.w, q.b.x, q.b.y, ox, oy, WPR, RPB, BH) & live;
    };
    int bb = ((L + BB - 1) / BB - 1) * BB;
    if (bb >= 0) {
        const int cnt0 = min(BB, L - bb);
        for (int i = tid; i < cnt0; i += BS) {
            const uint32_t k = r.x + bb + i;
            stage(bb, 0, i, rec_at(rec, pid_sorted[k], V.pairs, status), vals_sorted[k]);
        }
    }
    __syncthreads();
    for (int cur = 0; bb >= 0; bb -= BB, cur ^= 1) {
        const int cnt = min(BB, L - bb);
        const float4* __restrict__ cA = sA[cur];
        const float4* __restrict__ cB = sB[cur];
        const float4* __restrict__ cD = sD[cur];
        const uint32_t* __restrict__ cM = sM[cur];
        // gathers for the next (lower) batch, all entries full since bb > 0
        ProjRec qn[IPT];
        uint32_t en[IPT];
        if (bb > 0) {
#pragma unroll
            for (int u = 0; u < IPT; u++) {
                const int i = tid + u * BS;
                if (i < BB) {
                    const uint32_t k = r.x + bb - BB + i;
                    en[u] = vals_sorted[k];
                    qn[u] = rec_at(rec, pid_sorted[k], V.pairs, status);
                }
            }
        }
        for (int c = (cnt - 1) >> 5; c >= 0; c--) {
            // entries of this chunk whose box touches this warp's block,
            // before the last pair any of the warp's pixels blended
            const int jl = 32 * c + lane;
            uint32_t bits = __ballot_sync(0xffffffffu, jl < cnt && (cM[jl] & wbit));
            while (bits) {
                const int jj = 31 - __clz(bits);
                bits &= ~(1u << jj);
                const int j = 32 * c + jj;
                const float4 a = cA[j];
                const float4 b = cB[j];
                const float dx = pix_offset(fx, a.x);
                const PowX px2 = pair_power2_x(dx, a.z, a.w);   // shared by the lane's pixels
                // the skip tests of the lane's pixels first; the nine sums
                // are zeroed and formed only when a pixel of the warp blends
                float dyk[PPT], Gk[PPT], ak[PPT];
                bool hk[PPT], any = false;
#pragma unroll
                for (int k = 0; k < PPT; k++) {
                    dyk[k] = pix_offset(fy[k], a.y);
                    const float p2 = pair_power2_y(px2, dyk[k], b.x);
                    Gk[k] = ex2_approx(p2);
                    ak[k] = __fmul_rn(b.y, Gk[k]);
                    // one test for the pixel's three skips (exp2 taken for
                    // every pixel): no nested divergent branches
                    hk[k] = bb + j < (int)nl[k] && p2 >= kPow2Min && ak[k] >= kAlphaMin;
                    any |= hk[k];
                }
                float x = 0.f;
                if (__any_sync(0xffffffffu, any)) {
                    float g[9];
#pragma unroll
                    for (int i = 0; i < 9; i++) g[i] = 0.f;
#pragma unroll
                    for (int k = 0; k < PPT; k++) {
                        if (!hk[k]) continue;
                        const float araw = ak[k], G = Gk[k], dy = dyk[k];
                        const float alpha = fminf(kAlphaMax, araw);
                        const float cb = cD[j].w;
                        // compensated T before this entry
                        const float rom = div_one_minus(alpha, Th[k], Tl[k]);
                        const float wgt = alpha * Th[k];
                        g[6] = fmaf(wgt, d0[k], g[6]);
                        g[7] = fmaf(wgt, d1[k], g[7]);
                        g[8] = fmaf(wgt, d2[k], g[8]);
                        const float dcol = fmaf(d0[k], b.z, fmaf(d1[k], b.w, d2[k] * cb));
                        const float da = fmaf(Th[k], dcol, -U[k] * rom);
                        U[k] = fmaf(wgt, dcol, U[k]);
                        // moments of dp = dL/dpower (zero where the 0.99
                        // clamp holds); the conic and the constant factors
                        // are applied per entry after the reduction
                        const float dam = araw <= kAlphaMax ? da : 0.f;
                        g[5] = fmaf(dam, G, g[5]);
                        const float dp = dam * araw;
                        const float ydp = dy * dp;
                        g[0] += dp;
                        g[1] += ydp;
                        g[4] = fmaf(dy, ydp, g[4]);
                    }
                    // the lane's pixels share dx: sum dx dp = dx S, sum dx^2 dp
                    // = dx (dx S), sum dx dy dp = dx sum dy dp
                    g[0] *= dx;
                    g[2] = dx * g[0];
                    g[3] = dx * g[1];
                    x = bfly9(g, lane);
                }
                // every visiting warp fills its slot (zeros when none of its
                // pixels blended the entry)
                if (vi >= 0) part[w][j][vi] = x;
            }
        }
        __syncthreads();
        // one thread per entry adds the visiting warps' partial sums in warp
        // order and writes the entry's record (two 16-byte stores and one
        // 4-byte store).  Slots 0-4 hold sums of dp (dx, dy, dx^2, dx dy,
        // dy^2): dL/dmean = conic (sum dx dp, sum dy dp) and dL/dconic =
        // -(sum dx^2 dp / 2, sum dx dy dp, sum dy^2 dp / 2).
        for (int j = tid; j < cnt; j += BS) {
            float sm[9];
#pragma unroll
            for (int c = 0; c < 9; c++) sm[c] = 0.f;
            for (uint32_t m = sM[cur][j]; m; m &= m - 1u) {     // visiting warps, in warp order
                const int i = __ffs(m) - 1;
#pragma unroll
                for (int c = 0; c < 9; c++) sm[c] += part[i][j][c];
            }
            const float4 cd = sD[cur][j];
            const uint32_t e = sE[cur][j];
            if (GS_DCHECK(e < cap, status)) {
                float4* o = reinterpret_cast<float4*>(gradrec + e);
                o[0] = make_float4(fmaf(cd.x, sm[0], cd.y * sm[1]), fmaf(cd.y, sm[0], cd.z * sm[1]), -0.5f * sm[2],
                                   -sm[3]);
                o[1] = make_float4(-0.5f * sm[4], sm[5], sm[6], sm[7]);
                reinterpret_cast<float*>(o + 2)[0] = sm[8];
            }
        }
        if (bb > 0) {
#pragma unroll
            for (int u = 0; u < IPT; u++) {
                const int i = tid + u * BS;
                if (i < BB) stage(bb - BB, cur ^ 1, i, qn[u], en[u]);
            }
        }
        __syncthreads();
    }
    // entries past every pixel's last blended pair receive zero gradients
    for (uint32_t k = r.x + (uint32_t)L + tid; k < r.y; k += BS) {
        GradRec o;
        o.a = o.b = o.c = make_float4(0.f, 0.f, 0.f, 0.f);
        const uint32_t e = vals_sorted[k];
        if (GS_DCHECK(e < cap, status)) gradrec[e] = o;
    }
}

void launch_raster_bwd_px(const Plan& P, const WsPtrs& w, const float* bg, const float* dl, cudaStream_t st)
{
    const Views& V = P.views;
    const unsigned grid = (unsigned)V.tiles;
    const int ppt = tile_ppt(P);
#define GS_RBP(BS, TW, PPT)                                                                                  \
    k_raster_bwd_px<BS, TW, PPT><<<grid, BS, 0, st>>>(V, w.tile_order, w.ranges, w.vals_sorted, w.pid_sorted, \
                                                      w.rec, w.tfinal, bg, dl, w.nlast, w.gradrec, &w.hdr->status,   \
                                                      (uint32_t)P.cap)
    if (V.tw == 8) {
        if (ppt == 1) GS_RBP(64, 8, 1);
        else GS_RBP(32, 8, 2);
    } else if (V.th == 16) {
        if (ppt == 1) GS_RBP(256, 16, 1);
        else if (ppt == 2) GS_RBP(128, 16, 2);
        else GS_RBP(64, 16, 4);
    } else {
        if (ppt == 1) GS_RBP(512, 16, 1);
        else if (ppt == 2) GS_RBP(256, 16, 2);
        else GS_RBP(128, 16, 4);
    }
#undef GS_RBP
}

}  // namespace gs
