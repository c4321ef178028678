// raster_fwd.cu -- front-to-back alpha compositing per tile (VkSplat Sec. 2
// pipeline, Table 2 "Rasterization Fwd"), and the L1 loss gradient
// (Sec. 4.5, L1 term).
//
// One CTA per tile, one thread per pixel, each warp an 8x4 pixel block.  The
// tile's sorted list is staged through shared memory one CTA-width chunk at a
// time (coalesced reads of the sorted pair indices, then 48-byte record
// gathers); with each entry the loader stores a mask of the warp blocks its
// 3-sigma box touches, and each warp walks only its entries (ballot over 32
// entries, then the set bits in order).  Transmittance is a compensated FP32 pair
// (TwoProduct with fmaf, the low part carried alongside), so the product over
// hundreds of factors keeps close to full FP32 accuracy.
#include "gs_internal.cuh"

namespace gs {

// 16x16 tiles: 6 CTAs per SM (40 registers) instead of 4 at 55 registers;
// more resident warps hide the chunk barriers (2.23 -> 2.01 ms at 3M Gaussians,
// 4x1080p; 7 CTAs spill and lose)
template <int BS, int TW>
__global__ void __launch_bounds__(BS, (BS == 256 ? 6 : 1)) k_raster_fwd(Views V, const uint32_t* __restrict__ order,
                                                                       const uint2* __restrict__ ranges,
                                                   const uint32_t* __restrict__ pid_sorted,
                                                   const ProjRec* __restrict__ rec, const float* __restrict__ bg,
                                                   float* __restrict__ image, float* __restrict__ tfinal,
                                                   uint32_t* __restrict__ nlast, WsHeader* __restrict__ hdr,
                                                   uint32_t cap)
{
    constexpr int CH = BS > 256 ? 256 : BS;   // list entries per staged chunk
    __shared__ float4 sA[2][CH];
    __shared__ float4 sB[2][CH];
    __shared__ float sCb[2][CH];   // blue
    __shared__ uint32_t sM[2][CH];
    __shared__ unsigned long long sblend[BS / 32];
    constexpr int WPR = TW / 8, RPB = BS / TW / 4;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t wbit = 1u << w;
    const int64_t gt = order[blockIdx.x];   // longest lists first
    const int v = view_of_tile(V, gt);
    const ViewDesc& vd = V.v[v];
    const int lt = (int)(gt - vd.tile_base);
    const int ox = (lt % vd.TX) * TW, oy = (lt / vd.TX) * (BS / TW);
    const int px = ox + (w % WPR) * 8 + (lane & 7);
    const int py = oy + (w / WPR) * 4 + (lane >> 3);
    const bool inside = px < vd.W && py < vd.H;
    // pixel centre relative to the tile's first pixel (the staged means are too)
    const float fx = (float)(px - ox) + 0.5f, fy = (float)(py - oy) + 0.5f;
    const uint2 r = range_at(ranges, gt, cap, &hdr->status);

    float Th = 1.0f, Tl = 0.0f;
    float C0 = 0.f, C1 = 0.f, C2 = 0.f;
    uint32_t last = 0, nbl = 0;
    int done = !inside;
    // chunk 0 staged directly; afterwards chunk i+1's records are gathered
    // while chunk i is composited (pair indices one chunk further ahead)
    if (threadIdx.x < CH && r.x + threadIdx.x < r.y) {
        const ProjRec q = rec_at(rec, pid_sorted[r.x + threadIdx.x], V.pairs, &hdr->status);
        sA[0][threadIdx.x] = pair_coefs(tile_mean(q.a.x, q.c.z, ox), tile_mean(q.a.y, q.c.w, oy), q.a.z, q.a.w, q.b.x);
        sB[0][threadIdx.x] = make_float4(pair_c2(q.b.x), q.b.y, q.b.z, q.b.w);
        sCb[0][threadIdx.x] = q.c.x;
        sM[0][threadIdx.x] = warp_block_mask(q.a.x, q.a.y, q.a.z, q.a.w, q.b.x, q.b.y, ox, oy, WPR, RPB);
    }
    uint32_t pid_next = threadIdx.x < CH && r.x + CH + threadIdx.x < r.y ? pid_sorted[r.x + CH + threadIdx.x] : 0u;
    int cur = 0;
    for (uint32_t base = r.x; base < r.y; base += CH, cur ^= 1) {
        if (__syncthreads_count(done) == BS) break;
        const bool have_next = threadIdx.x < CH && base + CH + threadIdx.x < r.y;
        ProjRec qn;
        if (have_next) qn = rec_at(rec, pid_next, V.pairs, &hdr->status);
        if (threadIdx.x < CH && base + 2 * CH + threadIdx.x < r.y) pid_next = pid_sorted[base + 2 * CH + threadIdx.x];
        const float4* __restrict__ cA = sA[cur];
        const float4* __restrict__ cB = sB[cur];
        const float* __restrict__ cCb = sCb[cur];
        const uint32_t* __restrict__ cM = sM[cur];
        const int cnt = (int)min((uint32_t)CH, r.y - base);
        for (int c0 = 0; c0 < cnt; c0 += 32) {
            uint32_t bits = __ballot_sync(0xffffffffu, c0 + lane < cnt && (cM[c0 + lane] & wbit));
            if (done) continue;
            while (bits) {
                const int j = c0 + __ffs(bits) - 1;
                bits &= bits - 1;
                const float4 a = cA[j];
                const float blue = cCb[j];   // read on every visit: faster than on the blend path
                const float dx = pix_offset(fx, a.x), dy = pix_offset(fy, a.y);
                const float4 b = cB[j];
                const float p2 = pair_power2(dx, dy, a.z, a.w, b.x);
                // one test for both skips (exp2 taken for every pair)
                const float G = ex2_approx(p2);
                const float araw = __fmul_rn(b.y, G);
                if (!(p2 >= kPow2Min && araw >= kAlphaMin)) continue;
                const float alpha = fminf(kAlphaMax, araw);
                // compensated T * (1 - alpha); the pair is carried without
                // renormalising (Th the rounded product, Tl its low part),
                // and the stop test takes their sum
                const float om = __fsub_rn(1.0f, alpha);
                const float om_err = __fsub_rn(-alpha, __fsub_rn(om, 1.0f));
                const float pr = __fmul_rn(Th, om);
                const float pe = __fmaf_rn(Th, om, -pr);
                const float lo = __fmaf_rn(Th, om_err, __fmaf_rn(Tl, om, pe));
                if (__fadd_rn(pr, lo) < kTMin) {
                    done = 1;
                    break;
                }
                const float wgt = alpha * Th;
                C0 = fmaf(b.z, wgt, C0);
                C1 = fmaf(b.w, wgt, C1);
                C2 = fmaf(blue, wgt, C2);
                Tl = lo;
                Th = pr;
                last = base - r.x + j + 1;
                nbl++;
            }
        }
        if (have_next) {
            const int nb = cur ^ 1;
            sA[nb][threadIdx.x] = pair_coefs(tile_mean(qn.a.x, qn.c.z, ox), tile_mean(qn.a.y, qn.c.w, oy), qn.a.z, qn.a.w,
                                             qn.b.x);
            sB[nb][threadIdx.x] = make_float4(pair_c2(qn.b.x), qn.b.y, qn.b.z, qn.b.w);
            sCb[nb][threadIdx.x] = qn.c.x;
            sM[nb][threadIdx.x] = warp_block_mask(qn.a.x, qn.a.y, qn.a.z, qn.a.w, qn.b.x, qn.b.y, ox, oy, WPR, RPB);
        }
    }
    if (gt == 0 && threadIdx.x < 3) hdr->bg[threadIdx.x] = bg ? bg[threadIdx.x] : 0.f;
    if (inside) {
        const int64_t pix = vd.pix_base + (int64_t)py * vd.W + px;
        const float T = Th + Tl;
        float b0 = 0.f, b1 = 0.f, b2 = 0.f;
        if (bg) { b0 = bg[0]; b1 = bg[1]; b2 = bg[2]; }
        image[3 * pix + 0] = fmaf(T, b0, C0);
        image[3 * pix + 1] = fmaf(T, b1, C1);
        image[3 * pix + 2] = fmaf(T, b2, C2);
        tfinal[pix] = T;
        nlast[pix] = last;
    }
    // blended pair count: warp reduce, one atomic per CTA
    unsigned long long c = nbl;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) sblend[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int i = 0; i < BS / 32; i++) s += sblend[i];
        if (s) atomicAdd(&hdr->blended, s);
    }
}

void launch_raster_fwd(const Plan& P, const WsPtrs& w, const float* bg, float* image, cudaStream_t st)
{
    const Views& V = P.views;
    const int bs = V.tw * V.th;
    const unsigned grid = (unsigned)V.tiles;
#define GS_RF(BS, TW) k_raster_fwd<BS, TW><<<grid, BS, 0, st>>>(V, w.tile_order, w.ranges, w.pid_sorted, w.rec, bg, image, \
                                                                w.tfinal, w.nlast, w.hdr, (uint32_t)P.cap)
    if (bs == 64) GS_RF(64, 8);
    else if (bs == 256) GS_RF(256, 16);
    else GS_RF(512, 16);
#undef GS_RF
}

// ---------------------------------------------------------------------------
// L1 loss and gradient
// ---------------------------------------------------------------------------

constexpr int kLossThreads = 256;
constexpr int kLossItems = 8;

__device__ __forceinline__ float l1_sign(float d, float inv_n) { return d > 0.f ? inv_n : (d < 0.f ? -inv_n : 0.f); }

// VEC: the three arrays are 16-byte aligned; each thread takes kLossItems / 2
// float4 (a block 2 x kLossThreads x kLossItems values), the ragged end
// value by value.
template <bool VEC>
__global__ void __launch_bounds__(kLossThreads) k_loss_l1(const float* __restrict__ image,
                                                          const float* __restrict__ target, float* __restrict__ dl,
                                                          int64_t n, float inv_n, float* __restrict__ part,
                                                          WsHeader* __restrict__ hdr)
{
    __shared__ float ws[kLossThreads / 32];
    __shared__ bool is_last;
    float s = 0.f;
    if (VEC) {
        const int64_t base4 = (int64_t)blockIdx.x * kLossThreads * (kLossItems / 2);
#pragma unroll
        for (int i = 0; i < kLossItems / 2; i++) {
            const int64_t i4 = base4 + i * kLossThreads + threadIdx.x, e = 4 * i4;
            if (e + 3 < n) {
                const float4 a = reinterpret_cast<const float4*>(image)[i4];
                const float4 b = reinterpret_cast<const float4*>(target)[i4];
                const float d0 = a.x - b.x, d1 = a.y - b.y, d2 = a.z - b.z, d3 = a.w - b.w;
                reinterpret_cast<float4*>(dl)[i4] =
                    make_float4(l1_sign(d0, inv_n), l1_sign(d1, inv_n), l1_sign(d2, inv_n), l1_sign(d3, inv_n));
                s += (fabsf(d0) + fabsf(d1)) + (fabsf(d2) + fabsf(d3));
            } else {
                for (int64_t k = e; k < n && k < e + 4; k++) {
                    const float d = image[k] - target[k];
                    dl[k] = l1_sign(d, inv_n);
                    s += fabsf(d);
                }
            }
        }
    } else {
        const int64_t base = (int64_t)blockIdx.x * kLossThreads * kLossItems;
#pragma unroll
        for (int i = 0; i < kLossItems; i++) {
            const int64_t idx = base + i * kLossThreads + threadIdx.x;
            if (idx < n) {
                const float d = image[idx] - target[idx];
                dl[idx] = l1_sign(d, inv_n);
                s += fabsf(d);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int i = 0; i < kLossThreads / 32; i++) t += ws[i];
        part[blockIdx.x] = t;
        __threadfence();
        const uint32_t done = atomicAdd(&hdr->loss_counter, 1u);
        is_last = done == gridDim.x - 1;
    }
    __syncthreads();
    if (is_last) {
        // the last CTA sums the partials: thread t takes indices t, t + 256,
        // ... (Kahan-compensated), then a fixed-order tree -- deterministic
        __threadfence();
        float t = 0.f, comp = 0.f;
        for (unsigned i = threadIdx.x; i < gridDim.x; i += kLossThreads) {
            const float y = ((volatile float*)part)[i] - comp;
            const float u = t + y;
            comp = (u - t) - y;
            t = u;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = t;
        __syncthreads();
        if (threadIdx.x == 0) {
            float tt = 0.f;
            for (int i = 0; i < kLossThreads / 32; i++) tt += ws[i];
            hdr->loss = tt * inv_n;
            hdr->loss_counter = 0;
        }
    }
}

void launch_loss_l1(const Plan& P, const WsPtrs& w, const float* image, const float* target, float* dl,
                    cudaStream_t st)
{
    const int64_t n = 3 * P.views.pixels;
    const bool vec = ((reinterpret_cast<uintptr_t>(image) | reinterpret_cast<uintptr_t>(target) |
                       reinterpret_cast<uintptr_t>(dl)) & 15u) == 0;
    const int64_t per_block = (int64_t)kLossThreads * kLossItems * (vec ? 2 : 1);
    const int64_t blocks = (n + per_block - 1) / per_block;
    if (vec)
        k_loss_l1<true><<<(unsigned)blocks, kLossThreads, 0, st>>>(image, target, dl, n, 1.0f / (float)n,
                                                                   w.loss_part, w.hdr);
    else
        k_loss_l1<false><<<(unsigned)blocks, kLossThreads, 0, st>>>(image, target, dl, n, 1.0f / (float)n,
                                                                    w.loss_part, w.hdr);
}

}  // namespace gs
