// raster_bwd2.cu -- rasterization backward, the paper's second implementation
// (VkSplat Sec. 4.2): for each batch of a tile's list, a pass parallel over
// pixels computes every (Gaussian, pixel) pair's transmittance terms and
// stores them in shared memory, then a pass parallel over Gaussians sums each
// Gaussian's gradient from them -- every lane busy, no cross-lane reduction,
// no atomics.
//
// GB300 form.  One CTA per tile, one thread per pixel, each warp an 8x4
// pixel block, as in the forward.  The list is staged BB entries at a time
// (double-buffered) with a mask of the warp blocks each entry can reach; a
// (Gaussian, block) pair is one unit of work.  A staged chunk is cut from its
// back into sub-batches of at most NP pairs:
//   phase 1 (pixels): each warp walks its entries of the sub-batch back to
//     front, continuing its pixels' state (T recovered by a compensated
//     division by 1 - alpha, colour still to come S carried as its
//     projection dL/dC . S), and stores per pixel the blend
//     weight w = alpha T and A = dL/dalpha * G (zero where the 0.99 clamp
//     holds) at [pixel][pair] (odd row stride: no bank conflicts);
//   phase 2 (pairs): TPP threads per pair each sum PPT pixels of the pair's
//     block: dL/dcolour += w dL/dC, dL/dopacity += A, and with
//     dL/dpower = o A the mean and conic terms from the pixel offset;
//   combine: each entry's partial sums, in block order, go to its gradient
//     record at its emission slot (deterministic).
// The per-pair phase replaces the nine-value warp butterfly of the
// pixel-parallel implementation with plain per-lane accumulation.
#include "gs_internal.cuh"

namespace gs {

template <int BS>
struct Bwd2Cfg {
    static constexpr int NW = BS / 32;             // warps = 8x4 blocks per tile
    static constexpr int TPP = BS >= 512 ? 4 : 2;  // phase-2 threads per pair
    static constexpr int NP = BS / TPP;            // pairs per sub-batch
    static constexpr int NPS = NP + 1;             // odd row stride
    static constexpr int PPT = 32 / TPP;           // pixels per phase-2 thread
    static constexpr int BB = 64;                  // staged entries per chunk
};

template <int BS>
struct Bwd2Smem {
    using C = Bwd2Cfg<BS>;
    float pw[32 * C::NPS];        // alpha T per [pixel in block][pair]
    float pa[32 * C::NPS];        // dL/dalpha * G per [pixel in block][pair]
    float pr[9][BS + 1];          // phase-2 sums per thread
    float4 sd[32][C::NW];         // dL/dC per [pixel in block][block]
    float4 sA[2][C::BB];          // mean (relative to the tile's first pixel), prescaled conic a, b
    float4 sB[2][C::BB];          // prescaled conic c, opacity, red, green
    float4 sD[2][C::BB];          // conic a, b, c, blue
    uint32_t sE[2][C::BB];        // emission slot
    uint32_t sM[2][C::BB];        // warp-block mask
    int pbase[C::BB + 1];         // first pair of each entry of the current chunk
    uint8_t pj[C::NP];            // entry (in the chunk) of each pair of the sub-batch
    uint8_t pb[C::NP];            // block of each pair
    int smax[C::NW];
};

template <int BS>
constexpr size_t bwd2_smem_bytes() { return sizeof(Bwd2Smem<BS>); }

// Exclusive prefix of the chunk's per-entry pair counts (one warp).
template <int BB>
__device__ __forceinline__ void bwd2_pbase(const uint32_t* __restrict__ m, int cnt, int* __restrict__ pbase, int lane)
{
    int run = 0;
    for (int j0 = 0; j0 < BB; j0 += 32) {
        const int j = j0 + lane;
        const int c = j < cnt ? __popc(m[j]) : 0;
        int x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        pbase[j] = run + x - c;
        run += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) pbase[BB] = run;
}

// Smallest lo in [0, hi] with pbase[hi] - pbase[lo] <= np (pbase is
// non-decreasing).
__device__ __forceinline__ int bwd2_sub_lo(const int* __restrict__ pbase, int hi, int np)
{
    const int need = pbase[hi] - np;
    int lo = 0, up = hi;
    while (lo < up) {
        const int mid = (lo + up) >> 1;
        if (pbase[mid] >= need) up = mid;
        else lo = mid + 1;
    }
    return lo;
}

template <int BS, int TW>
__global__ void __launch_bounds__(BS) k_raster_bwd2(Views V, const uint32_t* __restrict__ order,
                                                    const uint2* __restrict__ ranges,
                                                    const uint32_t* __restrict__ vals_sorted,
                                                    const uint32_t* __restrict__ pid_sorted,
                                                    const ProjRec* __restrict__ rec,
                                                    const float* __restrict__ tfinal,
                                                    const float* __restrict__ bg, const float* __restrict__ dl,
                                                    const uint32_t* __restrict__ nlast,
                                                    GradRec* __restrict__ gradrec)
{
    using C = Bwd2Cfg<BS>;
    constexpr int NW = C::NW, BB = C::BB, NP = C::NP, NPS = C::NPS, TPP = C::TPP, PPT = C::PPT;
    constexpr int WPR = TW / 8;            // 8x4 warp blocks per tile row
    constexpr int RPB = BS / TW / 4;       // rows of warp blocks
    constexpr int IPT = (BB + BS - 1) / BS;
    extern __shared__ __align__(16) unsigned char bwd2_raw[];
    Bwd2Smem<BS>& S = *reinterpret_cast<Bwd2Smem<BS>*>(bwd2_raw);

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t gt = order[blockIdx.x];   // longest lists first
    const int v = view_of_tile(V, gt);
    const ViewDesc& vd = V.v[v];
    const int lt = (int)(gt - vd.tile_base);
    const int ox = (lt % vd.TX) * TW, oy = (lt / vd.TX) * (BS / TW);
    const int px = ox + (w % WPR) * 8 + (lane & 7);
    const int py = oy + (w / WPR) * 4 + (lane >> 3);
    const uint32_t wbit = 1u << w;
    const bool inside = px < vd.W && py < vd.H;
    const uint2 r = ranges[gt];
    // pixel centre relative to the tile's first pixel (the staged means are too)
    const float fx = (float)(px - ox) + 0.5f, fy = (float)(py - oy) + 0.5f;

    uint32_t nl = 0;
    float Th = 1.f, Tl = 0.f, d0 = 0.f, d1 = 0.f, d2 = 0.f;
    if (inside) {
        const int64_t pix = vd.pix_base + (int64_t)py * vd.W + px;
        nl = nlast[pix];
        Th = tfinal[pix];
        d0 = dl[3 * pix]; d1 = dl[3 * pix + 1]; d2 = dl[3 * pix + 2];
    }
    S.sd[lane][w] = make_float4(d0, d1, d2, 0.f);
    // U = sum_c dL/dC_c S_c, S_c the colour still to come behind an entry
    // (from T_final bg_c): dL/dalpha = T sum_c dL/dC_c col_c - U / (1 - alpha)
    float U = 0.f;
    if (bg) U = Th * fmaf(d0, bg[0], fmaf(d1, bg[1], d2 * bg[2]));
    int mx_nl = (int)nl;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx_nl = max(mx_nl, __shfl_xor_sync(0xffffffffu, mx_nl, o));
    if (lane == 0) S.smax[w] = mx_nl;
    __syncthreads();
    int L = 0;
#pragma unroll
    for (int i = 0; i < NW; i++) L = max(L, S.smax[i]);
    L = min(L, (int)(r.y - r.x));

    // warps whose pixels blended past list position pos (a pair is only
    // formed for those)
    auto live = [&](int pos) {
        uint32_t m = 0;
#pragma unroll
        for (int i = 0; i < NW; i++) m |= (pos < S.smax[i] ? 1u : 0u) << i;
        return m;
    };
    auto stage = [&](int buf, int i, int pos, const ProjRec& q, uint32_t e) {
        S.sA[buf][i] = pair_coefs(tile_mean(q.a.x, q.c.z, ox), tile_mean(q.a.y, q.c.w, oy), q.a.z, q.a.w, q.b.x);
        S.sB[buf][i] = make_float4(pair_c2(q.b.x), q.b.y, q.b.z, q.b.w);
        S.sD[buf][i] = make_float4(q.a.z, q.a.w, q.b.x, q.c.x);
        S.sE[buf][i] = e;
        S.sM[buf][i] = warp_block_mask(q.a.x, q.a.y, q.a.z, q.a.w, q.b.x, q.b.y, ox, oy, WPR, RPB) & live(pos);
    };
    int bb = ((L + BB - 1) / BB - 1) * BB;
    if (bb >= 0) {
        const int cnt0 = min(BB, L - bb);
        for (int i = tid; i < cnt0; i += BS) {
            const uint32_t k = r.x + bb + i;
            stage(0, i, bb + i, rec[pid_sorted[k]], vals_sorted[k]);
        }
    }
    __syncthreads();
    for (int cur = 0; bb >= 0; bb -= BB, cur ^= 1) {
        const int cnt = min(BB, L - bb);
        if (w == 0) bwd2_pbase<BB>(S.sM[cur], cnt, S.pbase, lane);
        // gathers for the next (lower) chunk, all entries full since bb > 0
        ProjRec qn[IPT];
        uint32_t en[IPT];
        if (bb > 0) {
#pragma unroll
            for (int u = 0; u < IPT; u++) {
                const int i = tid + u * BS;
                if (i < BB) {
                    const uint32_t k = r.x + bb - BB + i;
                    en[u] = vals_sorted[k];
                    qn[u] = rec[pid_sorted[k]];
                }
            }
        }
        __syncthreads();
        const float4* __restrict__ cA = S.sA[cur];
        const float4* __restrict__ cB = S.sB[cur];
        const float4* __restrict__ cD = S.sD[cur];
        const uint32_t* __restrict__ cM = S.sM[cur];
        // sub-batches of at most NP pairs, cut from the back (a short last
        // one leaves most warps free for other CTAs in its phase 2)
        int hi = cnt;
        while (hi > 0) {
            const int lo = bwd2_sub_lo(S.pbase, hi, NP);
            const int p0 = S.pbase[lo];
            // ---- phase 1: pixels, back to front over entries [lo, hi)
            for (int c = (hi - 1) >> 5; c >= (lo >> 5); c--) {
                const int jl = 32 * c + lane;
                uint32_t bits = __ballot_sync(0xffffffffu, jl >= lo && jl < hi && (cM[jl] & wbit));
                while (bits) {
                    const int jj = 31 - __clz(bits);
                    bits &= ~(1u << jj);
                    const int j = 32 * c + jj;
                    const int idx = S.pbase[j] - p0 + __popc(cM[j] & (wbit - 1u));
                    float wv = 0.f, av = 0.f;
                    if (bb + j < (int)nl) {
                        const float4 a = cA[j];
                        const float4 b = cB[j];
                        const float dx = pix_offset(fx, a.x), dy = pix_offset(fy, a.y);
                        const float p2 = pair_power2(dx, dy, a.z, a.w, b.x);
                        if (p2 >= kPow2Min) {
                            const float G = ex2_approx(p2);
                            const float araw = __fmul_rn(b.y, G);
                            const float alpha = fminf(kAlphaMax, araw);
                            if (araw >= kAlphaMin) {
                                const float cb = cD[j].w;
                                // compensated T before this entry
                                const float rom = div_one_minus(alpha, Th, Tl);
                                wv = alpha * Th;
                                const float dcol = fmaf(d0, b.z, fmaf(d1, b.w, d2 * cb));
                                const float da = fmaf(Th, dcol, -U * rom);
                                U = fmaf(wv, dcol, U);
                                if (araw <= kAlphaMax) av = da * G;
                            }
                        }
                    }
                    S.pw[lane * NPS + idx] = wv;
                    S.pa[lane * NPS + idx] = av;
                    if (lane == 0) {
                        S.pj[idx] = (uint8_t)j;
                        S.pb[idx] = (uint8_t)w;
                    }
                }
            }
            __syncthreads();
            // ---- phase 2: (Gaussian, block) pairs, TPP threads each
            const int npair = S.pbase[hi] - p0;
            {
                const int pq = tid / TPP, part = tid - TPP * (tid / TPP);
                float acc[9];
#pragma unroll
                for (int i = 0; i < 9; i++) acc[i] = 0.f;
                if (pq < npair) {
                    const int j = S.pj[pq], b = S.pb[pq];
                    const float4 a = cA[j];
                    const float op = cB[j].y;
                    const float bx = (float)((b % WPR) * 8) + 0.5f, by = (float)((b / WPR) * 4) + 0.5f;
#pragma unroll
                    for (int i = 0; i < PPT; i++) {
                        const int k = part * PPT + i;
                        const float wv = S.pw[k * NPS + pq], av = S.pa[k * NPS + pq];
                        const float4 dv = S.sd[k][b];
                        const float dx = pix_offset(bx + (float)(k & 7), a.x);
                        const float dy = pix_offset(by + (float)(k >> 3), a.y);
                        acc[6] = fmaf(wv, dv.x, acc[6]);
                        acc[7] = fmaf(wv, dv.y, acc[7]);
                        acc[8] = fmaf(wv, dv.z, acc[8]);
                        acc[5] += av;
                        // moments of dp = dL/dpower (conic and constant
                        // factors applied per entry in the combine)
                        const float dp = av * op;
                        const float ex = dx * dp, ey = dy * dp;
                        acc[0] += ex;
                        acc[1] += ey;
                        acc[2] = fmaf(dx, ex, acc[2]);
                        acc[3] = fmaf(dx, ey, acc[3]);
                        acc[4] = fmaf(dy, ey, acc[4]);
                    }
                }
#pragma unroll
                for (int i = 0; i < 9; i++) S.pr[i][tid] = acc[i];
            }
            __syncthreads();
            // ---- combine: each entry's pairs in block order (deterministic).
            // Slots 0-4 hold sums of dp (dx, dy, dx^2, dx dy, dy^2):
            // dL/dmean = conic (sum dx dp, sum dy dp), dL/dconic =
            // -(sum dx^2 dp / 2, sum dx dy dp, sum dy^2 dp / 2).
            for (int t = tid; t < (hi - lo) * 9; t += BS) {
                const int e = lo + t / 9, comp = t - 9 * (t / 9);
                const int comp2 = comp < 2 ? comp ^ 1 : comp;
                float s = 0.f, s2 = 0.f;
                const int q1 = (S.pbase[e + 1] - p0) * TPP;
                for (int q = (S.pbase[e] - p0) * TPP; q < q1; q++) {
                    s += S.pr[comp][q];
                    s2 += S.pr[comp2][q];
                }
                float out = s;
                if (comp < 2) {
                    const float4 cd = cD[e];
                    out = comp == 0 ? fmaf(cd.x, s, cd.y * s2) : fmaf(cd.y, s2, cd.z * s);
                } else if (comp < 5) {
                    out = comp == 3 ? -s : -0.5f * s;
                }
                reinterpret_cast<float*>(gradrec + S.sE[cur][e])[comp] = out;
            }
            hi = lo;
        }
        if (bb > 0) {
#pragma unroll
            for (int u = 0; u < IPT; u++) {
                const int i = tid + u * BS;
                if (i < BB) stage(cur ^ 1, i, bb - BB + i, qn[u], en[u]);
            }
        }
        __syncthreads();
    }
    // entries past every pixel's last blended pair receive zero gradients
    for (uint32_t k = r.x + (uint32_t)L + tid; k < r.y; k += BS) {
        GradRec o;
        o.a = o.b = o.c = make_float4(0.f, 0.f, 0.f, 0.f);
        gradrec[vals_sorted[k]] = o;
    }
}

void launch_raster_bwd2(const Plan& P, const WsPtrs& w, const float* bg, const float* dl, cudaStream_t st)
{
    const Views& V = P.views;
    const unsigned grid = (unsigned)V.tiles;
#define GS_RB2(BS, TW)                                                                                        \
    do {                                                                                                      \
        constexpr size_t sb = bwd2_smem_bytes<BS>();                                                          \
        static bool attr_set = false;                                                                         \
        if (!attr_set) {                                                                                      \
            cudaFuncSetAttribute(k_raster_bwd2<BS, TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb); \
            attr_set = true;                                                                                  \
        }                                                                                                     \
        k_raster_bwd2<BS, TW><<<grid, BS, sb, st>>>(V, w.tile_order, w.ranges, w.vals_sorted, w.pid_sorted, w.rec, w.tfinal, \
                                                     bg, dl, w.nlast, w.gradrec);                             \
    } while (0)
    if (V.tw == 8) GS_RB2(64, 8);
    else if (V.th == 16) GS_RB2(256, 16);
    else GS_RB2(512, 16);
#undef GS_RB2
}

}  // namespace gs
