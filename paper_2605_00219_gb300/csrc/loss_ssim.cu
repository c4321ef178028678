// loss_ssim.cu -- fused gradient of the weighted L1 + SSIM loss on
// channel-last renders with an 8-bit RGBA reference (VkSplat Sec. 4.5).
//
//   L = (1 - lam) mean|x - y| + lam (1 - mean SSIM),
// SSIM per channel with an 11x11 Gaussian window (sigma 1.5), zero padding,
// C1 = 0.01^2, C2 = 0.03^2, means over 3 x all pixels of all views.
//
// With the window moments mu_x, mu_y, E[x^2], E[y^2], E[xy] at q,
//   dSSIM_sum / dx_p = (w * A)(p) + 2 x_p (w * B)(p) + y_p (w * Cc)(p),
// A = dSSIM/dmu_x, B = dSSIM/dE[x^2], Cc = dSSIM/dE[xy] at each q (the window
// is symmetric).  One CTA per 16x16 tile of a view: x and y are staged with a
// 10-pixel halo, separable 11-tap passes give the five moments at the 26x26
// positions whose windows reach the tile, then A, B, Cc there, and two more
// separable passes give the gradient at the tile's pixels -- one kernel, no
// intermediate image in global memory, no layout conversion.
//
// The moments are taken about a per-tile shift (x and y at the tile's centre
// pixel): variances and the covariance are shift-invariant, and with values
// near the local mean E[x^2] - mu_x^2 no longer cancels in FP32 on flat
// image regions.  Zero padding becomes padding with -shift.
#include "gs_internal.cuh"

namespace gs {

constexpr int kSsT = 16;                 // output tile
constexpr int kSsR = 5;                  // window radius
constexpr int kSsQ = kSsT + 2 * kSsR;    // 26: positions whose window reaches the tile
constexpr int kSsX = kSsT + 4 * kSsR;    // 36: staged pixels per side
constexpr float kSsC1 = 0.01f * 0.01f;

// Window tap k (0..10): exp(-(k - 5)^2 / (2 * 1.5^2)) normalised to unit sum,
// evaluated in FP64 and rounded to FP32; with unrolled tap loops these become
// immediate operands of the FMAs.
__host__ __device__ constexpr float ssim_w(int k)
{
    return (k == 0 || k == 10) ? 0.0010283801f
         : (k == 1 || k == 9)  ? 0.0075987582f
         : (k == 2 || k == 8)  ? 0.036000773f
         : (k == 3 || k == 7)  ? 0.10936069f
         : (k == 4 || k == 6)  ? 0.21300554f
                               : 0.26601171f;
}
constexpr float kSsC2 = 0.03f * 0.03f;

__device__ __forceinline__ int ssim_view_of_tile(const Views& V, int64_t t, int64_t& first)
{
    int64_t base = 0;
    for (int v = 0; v < V.n; v++) {
        const int64_t nt = (int64_t)((V.v[v].W + kSsT - 1) / kSsT) * ((V.v[v].H + kSsT - 1) / kSsT);
        if (t < base + nt || v == V.n - 1) {
            first = base;
            return v;
        }
        base += nt;
    }
    first = 0;
    return 0;
}

__device__ __forceinline__ float target_channel(uchar4 t, int c)
{
    return (float)(c == 0 ? t.x : (c == 1 ? t.y : t.z)) * (1.0f / 255.0f);
}

// Alpha masking (MASK): the loss is taken on the render and the reference
// both multiplied by the reference's alpha m = A / 255, so masked-out pixels
// add nothing; the gradient with respect to the render carries the factor m.
template <bool MASK>
__device__ __forceinline__ float pix_mask(uchar4 t)
{
    return MASK ? (float)t.w * (1.0f / 255.0f) : 1.0f;
}

template <bool MASK>
__global__ void __launch_bounds__(256) k_loss_l1_ssim(Views V, const float* __restrict__ image,
                                                      const uchar4* __restrict__ target, float lam,
                                                      float inv_n, float* __restrict__ dl,
                                                      float* __restrict__ part, WsHeader* __restrict__ hdr)
{
    __shared__ float2 sxy[kSsX][kSsX + 1];   // (x, y) about the shift
    // moments and partials interleaved, so each tap of the next pass reads
    // them with vector loads: (mu_x, mu_y, E[x^2], E[y^2]), E[xy]; (A, B), Cc
    __shared__ float4 hm03[kSsX][kSsQ];
    __shared__ float hm4[kSsX][kSsQ];
    __shared__ float2 abc01[kSsQ][kSsQ];
    __shared__ float abc2[kSsQ][kSsQ + 1];
    __shared__ float2 habc01[kSsQ][kSsT];
    __shared__ float habc2[kSsQ][kSsT];
    __shared__ float red[2][8];
    __shared__ bool is_last;

    const int tid = threadIdx.x;
    int64_t first;
    const int v = ssim_view_of_tile(V, blockIdx.x, first);
    const ViewDesc& vd = V.v[v];
    const int lt = (int)(blockIdx.x - first);
    const int TX = (vd.W + kSsT - 1) / kSsT;
    const int ox = (lt % TX) * kSsT, oy = (lt / TX) * kSsT;
    const int pc = tid % kSsT, pr = tid / kSsT;
    const int px = ox + pc, py = oy + pr;
    const bool pin = px < vd.W && py < vd.H;
    const int64_t ppix = vd.pix_base + (int64_t)py * vd.W + px;
    float l1 = 0.f, ss = 0.f;

    const int64_t cpix = vd.pix_base + (int64_t)min(oy + kSsT / 2, vd.H - 1) * vd.W + min(ox + kSsT / 2, vd.W - 1);
    for (int c = 0; c < 3; c++) {
        const uchar4 tc = target[cpix];
        const float mc = pix_mask<MASK>(tc);
        const float shx = image[3 * cpix + c] * mc, shy = target_channel(tc, c) * mc;
        __syncthreads();
        for (int i = tid; i < kSsX * kSsX; i += 256) {
            const int r = i / kSsX, col = i % kSsX;
            const int x = ox - 2 * kSsR + col, y = oy - 2 * kSsR + r;
            float a = 0.f, b = 0.f;
            if (x >= 0 && y >= 0 && x < vd.W && y < vd.H) {
                const int64_t pix = vd.pix_base + (int64_t)y * vd.W + x;
                const uchar4 t4 = target[pix];
                const float m = pix_mask<MASK>(t4);
                a = image[3 * pix + c] * m;
                b = target_channel(t4, c) * m;
            }
            sxy[r][col] = make_float2(a - shx, b - shy);
        }
        __syncthreads();
        // horizontal pass: 5 moments at 36 rows x 26 columns
        for (int i = tid; i < kSsX * kSsQ; i += 256) {
            const int r = i / kSsQ, q = i % kSsQ;
            float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f, m4 = 0.f;
#pragma unroll
            for (int k = 0; k <= 2 * kSsR; k++) {
                const float w = ssim_w(k);
                const float2 xy = sxy[r][q + k];
                const float a = xy.x, b = xy.y;
                m0 = fmaf(w, a, m0);
                m1 = fmaf(w, b, m1);
                m2 = fmaf(w, a * a, m2);
                m3 = fmaf(w, b * b, m3);
                m4 = fmaf(w, a * b, m4);
            }
            hm03[r][q] = make_float4(m0, m1, m2, m3);
            hm4[r][q] = m4;
        }
        __syncthreads();
        // vertical pass, SSIM and its partials at 26 x 26 positions
        for (int i = tid; i < kSsQ * kSsQ; i += 256) {
            const int qr = i / kSsQ, qc = i % kSsQ;
            float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k <= 2 * kSsR; k++) {
                const float w = ssim_w(k);
                const float4 a = hm03[qr + k][qc];
                m[0] = fmaf(w, a.x, m[0]);
                m[1] = fmaf(w, a.y, m[1]);
                m[2] = fmaf(w, a.z, m[2]);
                m[3] = fmaf(w, a.w, m[3]);
                m[4] = fmaf(w, hm4[qr + k][qc], m[4]);
            }
            const int x = ox - kSsR + qc, y = oy - kSsR + qr;
            float A = 0.f, B = 0.f, Cc = 0.f;
            if (x >= 0 && y >= 0 && x < vd.W && y < vd.H) {
                const float mx = m[0] + shx, my = m[1] + shy;
                const float vx = m[2] - m[0] * m[0], vy = m[3] - m[1] * m[1], cxy = m[4] - m[0] * m[1];
                const float a1 = 2.f * mx * my + kSsC1, a2 = 2.f * cxy + kSsC2;
                const float b1 = mx * mx + my * my + kSsC1, b2 = vx + vy + kSsC2;
                const float ib = 1.0f / (b1 * b2);
                const float s = a1 * a2 * ib;
                A = 2.f * my * (a2 - a1) * ib - 2.f * mx * s / b1 + 2.f * mx * s / b2;
                B = -s / b2;
                Cc = 2.f * a1 * ib;
                if (qr >= kSsR && qr < kSsR + kSsT && qc >= kSsR && qc < kSsR + kSsT) ss += s;
            }
            abc01[qr][qc] = make_float2(A, B);
            abc2[qr][qc] = Cc;
        }
        __syncthreads();
        // horizontal pass of A, B, Cc: 26 rows x 16 columns
        for (int i = tid; i < kSsQ * kSsT; i += 256) {
            const int r = i / kSsT, q = i % kSsT;
            float a = 0.f, b = 0.f, d = 0.f;
#pragma unroll
            for (int k = 0; k <= 2 * kSsR; k++) {
                const float w = ssim_w(k);
                const float2 ab = abc01[r][q + k];
                a = fmaf(w, ab.x, a);
                b = fmaf(w, ab.y, b);
                d = fmaf(w, abc2[r][q + k], d);
            }
            habc01[r][q] = make_float2(a, b);
            habc2[r][q] = d;
        }
        __syncthreads();
        // vertical pass at the tile's pixel; combine with the L1 term
        float wa = 0.f, wb = 0.f, wc = 0.f;
#pragma unroll
        for (int k = 0; k <= 2 * kSsR; k++) {
            const float w = ssim_w(k);
            const float2 ab = habc01[pr + k][pc];
            wa = fmaf(w, ab.x, wa);
            wb = fmaf(w, ab.y, wb);
            wc = fmaf(w, habc2[pr + k][pc], wc);
        }
        if (pin) {
            const uchar4 t4 = target[ppix];
            const float m = pix_mask<MASK>(t4);
            const float x = image[3 * ppix + c] * m, y = target_channel(t4, c) * m;
            const float d = x - y;
            const float dS = wa + 2.f * x * wb + y * wc;
            const float sg = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
            dl[3 * ppix + c] = MASK ? m * (((1.f - lam) * sg - lam * dS) * inv_n) : ((1.f - lam) * sg - lam * dS) * inv_n;
            l1 += fabsf(d);
        }
    }
    // per-CTA partial sums (L1, SSIM), then the last CTA adds them in order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        l1 += __shfl_down_sync(0xffffffffu, l1, o);
        ss += __shfl_down_sync(0xffffffffu, ss, o);
    }
    if ((tid & 31) == 0) { red[0][tid >> 5] = l1; red[1][tid >> 5] = ss; }
    __syncthreads();
    if (tid == 0) {
        float a = 0.f, b = 0.f;
        for (int i = 0; i < 8; i++) { a += red[0][i]; b += red[1][i]; }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
        __threadfence();
        is_last = atomicAdd(&hdr->loss_counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (is_last) {
        __threadfence();
        float a = 0.f, b = 0.f;
        for (unsigned i = tid; i < gridDim.x; i += 256) {
            a += ((volatile float*)part)[2 * i];
            b += ((volatile float*)part)[2 * i + 1];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
        __syncthreads();
        if ((tid & 31) == 0) { red[0][tid >> 5] = a; red[1][tid >> 5] = b; }
        __syncthreads();
        if (tid == 0) {
            float ta = 0.f, tb = 0.f;
            for (int i = 0; i < 8; i++) { ta += red[0][i]; tb += red[1][i]; }
            hdr->loss = (1.f - lam) * ta * inv_n + lam * (1.f - tb * inv_n);
            hdr->loss_counter = 0;
        }
    }
}

int64_t ssim_tiles(const Views& V)
{
    int64_t t = 0;
    for (int v = 0; v < V.n; v++) t += (int64_t)((V.v[v].W + kSsT - 1) / kSsT) * ((V.v[v].H + kSsT - 1) / kSsT);
    return t;
}

void launch_loss_l1_ssim(const Plan& P, const WsPtrs& w, const float* image, const void* target_rgba8, float lam,
                         bool alpha_mask, float* dl, cudaStream_t st)
{
    const int64_t tiles = ssim_tiles(P.views);
    const float inv_n = 1.0f / (float)(3 * P.views.pixels);
    const uchar4* t = static_cast<const uchar4*>(target_rgba8);
    if (alpha_mask)
        k_loss_l1_ssim<true><<<(unsigned)tiles, 256, 0, st>>>(P.views, image, t, lam, inv_n, dl, w.loss_part, w.hdr);
    else
        k_loss_l1_ssim<false><<<(unsigned)tiles, 256, 0, st>>>(P.views, image, t, lam, inv_n, dl, w.loss_part, w.hdr);
}

}  // namespace gs
