// project_bwd_adam.cu -- projection backward fused with Adam in one pass
// (VkSplat Sec. 4.3; Table 2 "Proj Bwd + Optim").
//
// One thread per Gaussian.  For every view of its scene the thread sums the
// Gaussian's intersection gradient records (contiguous at its emission
// offset), back-propagates through the SH colour (with the clamp), the view
// direction, the conic inverse, the EWA Jacobian (with the FOV clamp) and the
// camera transform, accumulating dL/dmean and the symmetric dL/dSigma of the
// 3D covariance in registers; the covariance backward (scale, quaternion with
// its normalisation) then runs once on the sum over views.  Then one
// Adam step per parameter group; scale and opacity move to log / logit space
// inside the optimiser and are written back activated, SH degree 0 and
// degrees 1-3 take their own learning rates.  No gradient tensor is stored.
//
// The bias corrections are folded into per-CTA constants (one powf pair per
// CTA), and the update uses the hardware square root and reciprocal
// approximations (about 2 ulp each): the update's relative error stays near
// 1e-7, far below the step's parameter tolerance, at a third of the cost of
// the correctly rounded sequences.
#include "gs_internal.cuh"

namespace gs {

struct AdamArgs {
    float lr[6];
    float b1, b2, eps;
    int step;        // > 0: use it; otherwise the workspace counter + 1
    int grad_only;
    uint32_t seed;   // stochastic rounding of bf16 storage
};

// Per-step Adam constants, computed once per CTA: with bias corrections
// c1 = 1 - b1^t, c2 = 1 - b2^t the update lr (m / c1) / (sqrt(v / c2) + eps)
// equals alpha_g m / (sqrt(v) + eps'), alpha_g = lr_g sqrt(c2) / c1 and
// eps' = eps sqrt(c2).
struct AdamConst {
    float alpha[6];
    float epsp, b1, b2, omb1, omb2;
};

__device__ __forceinline__ void adam1(float& th, float& m, float& v, float g, float alpha, const AdamConst& K)
{
    m = fmaf(K.b1, m, K.omb1 * g);
    v = fmaf(K.b2, v, K.omb2 * (g * g));
    th -= __fdividef(alpha * m, sqrt_approx(v) + K.epsp);
}

// Rotation R of the normalised quaternion q = (w, x, y, z) and
// M = R diag(s); returns 1 / |q|.
__device__ __forceinline__ float rot_scale(float4 q, float4 so, float* R, float* M, float& w, float& x, float& y,
                                           float& z)
{
    const float qn_r = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    w = q.x * qn_r; x = q.y * qn_r; y = q.z * qn_r; z = q.w * qn_r;
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
    const float sv[3] = {so.x, so.y, so.z};
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) M[3 * i + j] = R[3 * i + j] * sv[j];
    return qn_r;
}

// 3D covariance Sigma = M M^T as (S00, S01, S02, S11, S12, S22); it does
// not depend on the view, so it is formed once per Gaussian.
__device__ __forceinline__ void covariance3d(float4 q, float4 so, float* Sg)
{
    float R[9], M[9], w, x, y, z;
    rot_scale(q, so, R, M, w, x, y, z);
    auto dot = [&](int i, int j) { return M[3 * i] * M[3 * j] + M[3 * i + 1] * M[3 * j + 1] + M[3 * i + 2] * M[3 * j + 2]; };
    Sg[0] = dot(0, 0); Sg[1] = dot(0, 1); Sg[2] = dot(0, 2);
    Sg[3] = dot(1, 1); Sg[4] = dot(1, 2); Sg[5] = dot(2, 2);
}

// Backward of Sigma = M M^T, M = R(q) diag(s), once per Gaussian from the
// sum over views of dL/dSigma (symmetric, as stored by covariance3d):
// accumulates dq (raw quaternion) and ds (activated scale).
__device__ __forceinline__ void covariance3d_bwd(float4 q, float4 so, const float* dSg, float* dq, float* ds)
{
    float R[9], M[9], w, x, y, z;
    const float qn_r = rot_scale(q, so, R, M, w, x, y, z);
    const float dS[9] = {dSg[0], dSg[1], dSg[2], dSg[1], dSg[3], dSg[4], dSg[2], dSg[4], dSg[5]};
    const float sv[3] = {so.x, so.y, so.z};
    float dR[9];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const float dM = 2.f * (dS[3 * i] * M[j] + dS[3 * i + 1] * M[3 + j] + dS[3 * i + 2] * M[6 + j]);
            dR[3 * i + j] = dM * sv[j];
            ds[j] += dM * R[3 * i + j];
        }
    float dqn[4];
    dqn[0] = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
    dqn[1] = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - w * dR[5] + z * dR[6] + w * dR[7]) - 4.f * x * (dR[4] + dR[8]);
    dqn[2] = 2.f * (x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] + z * dR[7]) - 4.f * y * (dR[0] + dR[8]);
    dqn[3] = 2.f * (-w * dR[1] + x * dR[2] + w * dR[3] + y * dR[5] + x * dR[6] + y * dR[7]) - 4.f * z * (dR[0] + dR[4]);
    const float dqq = dqn[0] * w + dqn[1] * x + dqn[2] * y + dqn[3] * z;
    dq[0] += (dqn[0] - w * dqq) * qn_r;
    dq[1] += (dqn[1] - x * dqq) * qn_r;
    dq[2] += (dqn[2] - y * dqq) * qn_r;
    dq[3] += (dqn[3] - z * dqq) * qn_r;
}

// A Gaussian's SH coefficients in its thread's shared-memory row, chunk j =
// coefficients 4j .. 4j + 3: FP32 rows of 13 float4, or BF16 rows of 7 uint4
// (two chunks per uint4) for BF16 storage.  The strides make the 16-byte
// accesses of 8 consecutive threads cover all 32 banks once.
template <bool SH16> struct ShRow;
template <> struct ShRow<false> {
    static constexpr int kRowBytes = 13 * 16;
    const float4* r;
    __device__ __forceinline__ float4 operator()(int j) const { return r[j]; }
};
template <> struct ShRow<true> {
    static constexpr int kRowBytes = 7 * 16;
    const uint4* r;
    __device__ __forceinline__ float4 operator()(int j) const
    {
        const uint4 u = r[j >> 1];
        const uint32_t a = (j & 1) ? u.z : u.x, b = (j & 1) ? u.w : u.y;
        return make_float4(bf16_lo(a), bf16_hi(a), bf16_lo(b), bf16_hi(b));
    }
};

// Per-view backward of one Gaussian through projection and colour:
// accumulates dmu, dSg (dL/dSigma, symmetric) and dop (activated opacity),
// and adds this view's SH gradient Y[k] draw[c] (basis at the view
// direction times dL/d(raw colour)) to the thread's row sgrow.
// The SH coefficients are read twice (clamp test, then the direction
// gradient) from the thread's shared-memory row instead of being held in
// registers.
template <typename Row>
__device__ __forceinline__ void proj_bwd_view(const float* cam, int W, int H, float4 mu, const float* Sg,
                                              const Row& shrow, const float* g2, float* dmu, float* dSg,
                                              float& dop, float4* sgrow)
{
    const float fx = cam[12], fy = cam[13];
    const float* C = cam;
    const float tx = fmaf(C[0], mu.x, fmaf(C[1], mu.y, fmaf(C[2], mu.z, cam[9])));
    const float ty = fmaf(C[3], mu.x, fmaf(C[4], mu.y, fmaf(C[5], mu.z, cam[10])));
    const float tz = fmaf(C[6], mu.x, fmaf(C[7], mu.y, fmaf(C[8], mu.z, cam[11])));
    const float itz = __fdividef(1.0f, tz);   // hardware reciprocal: a few ulp, far inside the gradient bound

    // ---- colour: SH and view direction
    const float cpx = -(C[0] * cam[9] + C[3] * cam[10] + C[6] * cam[11]);
    const float cpy = -(C[1] * cam[9] + C[4] * cam[10] + C[7] * cam[11]);
    const float cpz = -(C[2] * cam[9] + C[5] * cam[10] + C[8] * cam[11]);
    const float ddx = mu.x - cpx, ddy = mu.y - cpy, ddz = mu.z - cpz;
    const float idist = rsqrtf(ddx * ddx + ddy * ddy + ddz * ddz);
    const float dirx = ddx * idist, diry = ddy * idist, dirz = ddz * idist;
    float Y[16];
    sh_basis(dirx, diry, dirz, Y);
    float raw[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
    for (int j = 0; j < 12; j++) {
        const float4 c4 = shrow(j);
        const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
        for (int i = 0; i < 4; i++) raw[(4 * j + i) % 3] = fmaf(cv[i], Y[(4 * j + i) / 3], raw[(4 * j + i) % 3]);
    }
    float draw[3];
#pragma unroll
    for (int c = 0; c < 3; c++) draw[c] = raw[c] < 0.0f ? 0.0f : g2[6 + c];
    // SH gradient of this view, Y[k] draw[c], added to the thread's row now
    // so that the basis values are dead during the covariance part
#pragma unroll
    for (int j = 0; j < 12; j++) {
        float4 a = sgrow[j];
        a.x = fmaf(Y[(4 * j) / 3], draw[(4 * j) % 3], a.x);
        a.y = fmaf(Y[(4 * j + 1) / 3], draw[(4 * j + 1) % 3], a.y);
        a.z = fmaf(Y[(4 * j + 2) / 3], draw[(4 * j + 2) % 3], a.z);
        a.w = fmaf(Y[(4 * j + 3) / 3], draw[(4 * j + 3) % 3], a.w);
        sgrow[j] = a;
    }
    float wk[16];
#pragma unroll
    for (int k = 0; k < 16; k++) wk[k] = 0.f;
#pragma unroll
    for (int j = 0; j < 12; j++) {
        const float4 c4 = shrow(j);
        const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
        for (int i = 0; i < 4; i++) wk[(4 * j + i) / 3] = fmaf(cv[i], draw[(4 * j + i) % 3], wk[(4 * j + i) / 3]);
    }
    float gdx, gdy, gdz;
    sh_basis_vjp(dirx, diry, dirz, wk, gdx, gdy, gdz);
    const float dd = gdx * dirx + gdy * diry + gdz * dirz;
    dmu[0] += (gdx - dirx * dd) * idist;
    dmu[1] += (gdy - diry * dd) * idist;
    dmu[2] += (gdz - dirz * dd) * idist;

    // ---- opacity
    dop += g2[5];

    // ---- EWA Jacobian (with the 1.3x FOV clamp) and T = J C
    const float limx = 1.3f * (0.5f * (float)W / fx), limy = 1.3f * (0.5f * (float)H / fy);
    const float ux = tx * itz, uy = ty * itz;
    const bool inx = ux >= -limx && ux <= limx, iny = uy >= -limy && uy <= limy;
    const float uxc = fminf(fmaxf(ux, -limx), limx), uyc = fminf(fmaxf(uy, -limy), limy);
    const float j00 = fx * itz, j11 = fy * itz, j02 = -fx * uxc * itz, j12 = -fy * uyc * itz;
    float T[6];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        T[k] = j00 * C[k] + j02 * C[6 + k];
        T[3 + k] = j11 * C[3 + k] + j12 * C[6 + k];
    }
    const float Sf[9] = {Sg[0], Sg[1], Sg[2], Sg[1], Sg[3], Sg[4], Sg[2], Sg[4], Sg[5]};
    float TS[6];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int l = 0; l < 3; l++) TS[3 * i + l] = T[3 * i] * Sf[l] + T[3 * i + 1] * Sf[3 + l] + T[3 * i + 2] * Sf[6 + l];
    const float va = TS[0] * T[0] + TS[1] * T[1] + TS[2] * T[2] + 0.3f;
    const float vb = TS[0] * T[3] + TS[1] * T[4] + TS[2] * T[5];
    const float vc = TS[3] * T[3] + TS[4] * T[4] + TS[5] * T[5] + 0.3f;
    const float idet = __fdividef(1.0f, va * vc - vb * vb);
    const float qa = vc * idet, qb = -vb * idet, qc = va * idet;
    // dL/dV = -Q G Q, G = [[dca, dcb/2], [dcb/2, dcc]] (symmetric)
    const float ga = g2[2], gb = 0.5f * g2[3], gc = g2[4];
    const float m00 = qa * ga + qb * gb, m01 = qa * gb + qb * gc;
    const float m11 = qb * gb + qc * gc;
    const float dV00 = -(m00 * qa + m01 * qb), dV01 = -(m00 * qb + m01 * qc);
    const float dV11 = -((qb * ga + qc * gb) * qb + m11 * qc);
    // dSigma += T^T dV T (upper triangle)
    {
        float U0[3], U1[3];     // rows of dV T
#pragma unroll
        for (int l = 0; l < 3; l++) {
            U0[l] = dV00 * T[l] + dV01 * T[3 + l];
            U1[l] = dV01 * T[l] + dV11 * T[3 + l];
        }
        dSg[0] += T[0] * U0[0] + T[3] * U1[0];
        dSg[1] += T[0] * U0[1] + T[3] * U1[1];
        dSg[2] += T[0] * U0[2] + T[3] * U1[2];
        dSg[3] += T[1] * U0[1] + T[4] * U1[1];
        dSg[4] += T[1] * U0[2] + T[4] * U1[2];
        dSg[5] += T[2] * U0[2] + T[5] * U1[2];
    }
    // dT = 2 dV T Sigma, dJ = dT C^T
    float dT[6];
#pragma unroll
    for (int l = 0; l < 3; l++) {
        dT[l] = 2.f * (dV00 * TS[l] + dV01 * TS[3 + l]);
        dT[3 + l] = 2.f * (dV01 * TS[l] + dV11 * TS[3 + l]);
    }
    const float dJ00 = dT[0] * C[0] + dT[1] * C[1] + dT[2] * C[2];
    const float dJ02 = dT[0] * C[6] + dT[1] * C[7] + dT[2] * C[8];
    const float dJ11 = dT[3] * C[3] + dT[4] * C[4] + dT[5] * C[5];
    const float dJ12 = dT[3] * C[6] + dT[4] * C[7] + dT[5] * C[8];
    const float itz2 = itz * itz;
    float dtx = fx * itz * g2[0];
    float dty = fy * itz * g2[1];
    float dtz = -(fx * tx * g2[0] + fy * ty * g2[1]) * itz2;
    dtz += -fx * itz2 * dJ00 - fy * itz2 * dJ11 + fx * uxc * itz2 * dJ02 + fy * uyc * itz2 * dJ12;
    if (inx) {
        dtx += -fx * itz2 * dJ02;
        dtz += fx * tx * itz2 * itz * dJ02;
    }
    if (iny) {
        dty += -fy * itz2 * dJ12;
        dtz += fy * ty * itz2 * itz * dJ12;
    }
    dmu[0] += C[0] * dtx + C[3] * dty + C[6] * dtz;
    dmu[1] += C[1] * dtx + C[4] * dty + C[7] * dtz;
    dmu[2] += C[2] * dtx + C[5] * dty + C[8] * dtz;
}

// Stochastic rounding to bf16 (storage form of SH and Adam moments): each
// value becomes one of its two neighbouring bf16 values with probabilities
// proportional to closeness, by the conversion instruction with stochastic
// rounding (cvt.rs, saturating to the largest finite value), two values per
// instruction from 32 random bits.  The random bits are a function of
// (seed, step, Gaussian, element), so the rounding is reproducible.
__device__ __forceinline__ uint32_t fmix32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x85ebca6bu;
    x ^= x >> 13;
    x *= 0xc2b2ae35u;
    x ^= x >> 16;
    return x;
}

// bf16 pair (lo in bits 0-15, hi in bits 16-31) by stochastic rounding
__device__ __forceinline__ uint32_t bf16x2_sr(float lo, float hi, uint32_t rbits)
{
    uint32_t d;
    asm("cvt.rs.satfinite.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
    return d;
}

// Per-thread stream key: one hash of (seed, step, Gaussian), uniform over
// 32 bits.  Draw ctr of the stream is one multiply-xorshift round of
// key + ctr * 0x9E3779B9: for each ctr a bijection of the key, hence uniform
// as well, which is what unbiased stochastic rounding needs; its 32 bits
// serve two bf16 roundings.
__device__ __forceinline__ uint32_t sr_key(uint32_t seed, int step, int64_t gi)
{
    return fmix32(seed ^ fmix32((uint32_t)step * 0x9E3779B9u ^ (uint32_t)gi ^ (uint32_t)(gi >> 32) * 0xc2b2ae35u));
}

__device__ __forceinline__ uint32_t sr_bits(uint32_t key, uint32_t ctr)
{
    uint32_t x = key + ctr * 0x9E3779B9u;
    x ^= x >> 16;
    x *= 0x7feb352du;
    return x ^ (x >> 15);
}

// Moment chunk ci (4 values) of Gaussian g: FP32 float4 or 4 x bf16.
template <bool MOM16>
__device__ __forceinline__ float4 load_mom(const void* base, int64_t idx)
{
    if (!MOM16) return reinterpret_cast<const float4*>(base)[idx];
    const uint2 u = reinterpret_cast<const uint2*>(base)[idx];
    return make_float4(bf16_lo(u.x), bf16_hi(u.x), bf16_lo(u.y), bf16_hi(u.y));
}

// The stored words of one moment chunk, loaded ahead of their use.
template <bool MOM16> struct MomWords { float4 w; };
template <> struct MomWords<true> { uint2 w; };

template <bool MOM16>
__device__ __forceinline__ MomWords<MOM16> load_mom_words(const void* base, int64_t idx)
{
    MomWords<MOM16> r;
    if constexpr (MOM16) r.w = reinterpret_cast<const uint2*>(base)[idx];
    else r.w = reinterpret_cast<const float4*>(base)[idx];
    return r;
}

template <bool MOM16>
__device__ __forceinline__ float4 mom_value(const MomWords<MOM16>& r)
{
    if constexpr (MOM16) return make_float4(bf16_lo(r.w.x), bf16_hi(r.w.x), bf16_lo(r.w.y), bf16_hi(r.w.y));
    else return r.w;
}

template <bool MOM16>
__device__ __forceinline__ void store_mom(void* base, int64_t idx, float4 m, uint32_t key, uint32_t ctr)
{
    if (!MOM16) {
        reinterpret_cast<float4*>(base)[idx] = m;
        return;
    }
    const uint32_t r0 = sr_bits(key, 2u * ctr), r1 = sr_bits(key, 2u * ctr + 1u);
    reinterpret_cast<uint2*>(base)[idx] = make_uint2(bf16x2_sr(m.x, m.y, r0), bf16x2_sr(m.z, m.w, r1));
}

constexpr int kPbaThreads = 128;

__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Phase 1 (one thread per Gaussian): sum the intersection records per view,
// back-propagate through projection and colour, apply Adam to mean,
// quaternion and (log-scale, logit-opacity); the 48 SH gradients accumulate
// in the thread's own row of shared memory.  Phase 2: Adam on the SH chunks,
// streaming coefficients and moments with few live registers.
template <bool SH16, bool MOM16>
__global__ void __launch_bounds__(kPbaThreads, 4) k_project_bwd_adam(Views V, Scenes S, const float* __restrict__ cams,
                                                                  const uint32_t* __restrict__ count,
                                                                  const uint32_t* __restrict__ offset,
                                                                  const GradRec* __restrict__ gradrec, AdamArgs A,
                                                                  float4* __restrict__ grads_out,
                                                                  const WsHeader* __restrict__ hdr, uint32_t cap)
{
    // per thread, a row of 12 float4 (stride 13 float4: the 16-byte accesses
    // of 8 consecutive threads cover all 32 banks once) for the SH gradients,
    // and a row of the Gaussian's 48 SH coefficients as stored (FP32 or BF16,
    // ShRow), read from HBM once and used by every view and by the SH update.
    // (53 KB per block with FP32 rows, 41 KB with BF16 rows)
    extern __shared__ float4 pba_smem[];
    float4 (*sG)[13] = reinterpret_cast<float4 (*)[13]>(pba_smem);
    float4 (*sS)[13] = reinterpret_cast<float4 (*)[13]>(pba_smem + kPbaThreads * 13);    // FP32 rows
    uint4 (*sS16)[7] = reinterpret_cast<uint4 (*)[7]>(pba_smem + kPbaThreads * 13);      // BF16 rows
    __shared__ AdamConst sK;
    const int tid = threadIdx.x;
    const int64_t gi = (int64_t)blockIdx.x * kPbaThreads + tid;
    const int t = A.step > 0 ? A.step : hdr->step + 1;
    const uint32_t key = MOM16 || SH16 ? sr_key(A.seed, t, gi) : 0u;
    if (tid == 0) {
        const float c1 = 1.0f - powf(A.b1, (float)t), c2 = 1.0f - powf(A.b2, (float)t);
        const float sc2 = sqrtf(c2);
#pragma unroll
        for (int i = 0; i < 6; i++) sK.alpha[i] = A.lr[i] * sc2 / c1;
        sK.epsp = A.eps * sc2;
        sK.b1 = A.b1;
        sK.b2 = A.b2;
        sK.omb1 = 1.0f - A.b1;
        sK.omb2 = 1.0f - A.b2;
    }
#pragma unroll
    for (int j = 0; j < 12; j++) sG[tid][j] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();

    if (gi < S.total) {
        int s = 0;
        while (s + 1 < S.n && S.s[s + 1].base <= gi) s++;
        const SceneDesc& sc = S.s[s];
        const int64_t g = gi - sc.base;
        const int64_t n = sc.n;
        float4 mu = sc.geom[g];
        float4 q = sc.geom[n + g];
        float4 so = sc.geom[2 * n + g];
        if (!A.grad_only) {
            // the moments are read only after the projection backward of
            // every view: request their lines into L2 now (no registers held)
#pragma unroll
            for (int ci = 0; ci < 15; ci++) {
                prefetch_l2(reinterpret_cast<const char*>(sc.m) + ((int64_t)ci * n + g) * (MOM16 ? 8 : 16));
                prefetch_l2(reinterpret_cast<const char*>(sc.v) + ((int64_t)ci * n + g) * (MOM16 ? 8 : 16));
            }
        }
        if (!SH16) {
#pragma unroll
            for (int j = 0; j < 12; j++) sS[tid][j] = reinterpret_cast<const float4*>(sc.sh)[(int64_t)j * n + g];
        } else {
#pragma unroll
            for (int jp = 0; jp < 6; jp++) sS16[tid][jp] = reinterpret_cast<const uint4*>(sc.sh)[(int64_t)jp * n + g];
        }
        float dmu[3] = {0.f, 0.f, 0.f}, dSg[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, dop = 0.f;
        float Sg[6];
        covariance3d(q, so, Sg);
        float st_sum = 0.f, st_cnt = 0.f;   // densification statistics of this step
        // the Gaussian's intersection records of all views of its scene are
        // consecutive from its first emission slot (Gaussian-major slot
        // order); the next view's count is loaded while this view is
        // processed
        const int nv = V.nv[s];
        const int64_t q0 = V.qbase[s] + g * nv;
        uint32_t e_next = offset[q0];
        uint32_t cnt_n = count[q0];
        {
            // the records of every view form [offset[q0], offset[q0 + nv]):
            // request their lines into L2 before the first view needs them
            const uint32_t e_end = min(offset[q0 + nv], cap);
            const char* p0 = reinterpret_cast<const char*>(gradrec + e_next);
            const char* p1 = reinterpret_cast<const char*>(gradrec + max(e_end, e_next));
            for (int l = 0; l < 16 && p0 + 128 * l < p1; l++) prefetch_l2(p0 + 128 * l);
        }
        for (int k = 0; k < nv; k++) {
            const int v = V.view_of[s][k];
            const uint32_t cnt = cnt_n, off = e_next;
            e_next += cnt;
            if (k + 1 < nv) cnt_n = count[q0 + k + 1];
            if (cnt == 0) continue;
            const ViewDesc& vd = V.v[v];
            const uint32_t end = min(off + cnt, cap);
            float g2[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            // two records' loads in flight at a time
#pragma unroll 2
            for (uint32_t e = off; e < end; e++) {
                const GradRec r = gradrec[e];
                g2[0] += r.a.x; g2[1] += r.a.y; g2[2] += r.a.z; g2[3] += r.a.w;
                g2[4] += r.b.x; g2[5] += r.b.y; g2[6] += r.b.z; g2[7] += r.b.w;
                g2[8] += r.c.x;
            }
            if (sc.stats) {
                // dL/d(mean2D) in half-image units, as if this view's loss
                // were the mean over its own pixels
                const float fac = (float)V.pixels / ((float)vd.W * (float)vd.H);
                const float gx = g2[0] * (0.5f * (float)vd.W) * fac, gy = g2[1] * (0.5f * (float)vd.H) * fac;
                st_sum += sqrtf(gx * gx + gy * gy);
                st_cnt += 1.0f;
            }
            float cam[16];
#pragma unroll
            for (int i = 0; i < 16; i++) cam[i] = __ldg(cams + 16 * v + i);
            if (SH16) proj_bwd_view(cam, vd.W, vd.H, mu, Sg, ShRow<true>{sS16[tid]}, g2, dmu, dSg, dop, sG[tid]);
            else proj_bwd_view(cam, vd.W, vd.H, mu, Sg, ShRow<false>{sS[tid]}, g2, dmu, dSg, dop, sG[tid]);
        }
        float dq[4] = {0.f, 0.f, 0.f, 0.f}, ds[3] = {0.f, 0.f, 0.f};
        covariance3d_bwd(q, so, dSg, dq, ds);
        if (sc.stats) {
            float2 st = sc.stats[g];
            st.x += st_sum;
            st.y += st_cnt;
            sc.stats[g] = st;
        }
        if (A.grad_only) {
            const int64_t N = S.total;
            grads_out[0 * N + gi] = make_float4(dmu[0], dmu[1], dmu[2], 0.f);
            grads_out[1 * N + gi] = make_float4(dq[0], dq[1], dq[2], dq[3]);
            grads_out[2 * N + gi] = make_float4(ds[0], ds[1], ds[2], dop);
        } else {
            const AdamConst K = sK;
            {
                float4 m = load_mom<MOM16>(sc.m, g), vv = load_mom<MOM16>(sc.v, g);
                adam1(mu.x, m.x, vv.x, dmu[0], K.alpha[0], K);
                adam1(mu.y, m.y, vv.y, dmu[1], K.alpha[0], K);
                adam1(mu.z, m.z, vv.z, dmu[2], K.alpha[0], K);
                store_mom<MOM16>(sc.m, g, m, key, 0u);
                store_mom<MOM16>(sc.v, g, vv, key, 1u);
                sc.geom[g] = mu;
            }
            {
                float4 m = load_mom<MOM16>(sc.m, n + g), vv = load_mom<MOM16>(sc.v, n + g);
                adam1(q.x, m.x, vv.x, dq[0], K.alpha[1], K);
                adam1(q.y, m.y, vv.y, dq[1], K.alpha[1], K);
                adam1(q.z, m.z, vv.z, dq[2], K.alpha[1], K);
                adam1(q.w, m.w, vv.w, dq[3], K.alpha[1], K);
                store_mom<MOM16>(sc.m, n + g, m, key, 2u);
                store_mom<MOM16>(sc.v, n + g, vv, key, 3u);
                sc.geom[n + g] = q;
            }
            {
                float4 m = load_mom<MOM16>(sc.m, 2 * n + g), vv = load_mom<MOM16>(sc.v, 2 * n + g);
                float th0 = logf(so.x), th1 = logf(so.y), th2 = logf(so.z);
                float tho = logf(so.w) - log1pf(-so.w);
                adam1(th0, m.x, vv.x, ds[0] * so.x, K.alpha[2], K);
                adam1(th1, m.y, vv.y, ds[1] * so.y, K.alpha[2], K);
                adam1(th2, m.z, vv.z, ds[2] * so.z, K.alpha[2], K);
                adam1(tho, m.w, vv.w, dop * so.w * (1.0f - so.w), K.alpha[3], K);
                store_mom<MOM16>(sc.m, 2 * n + g, m, key, 4u);
                store_mom<MOM16>(sc.v, 2 * n + g, vv, key, 5u);
                sc.geom[2 * n + g] = make_float4(expf(th0), expf(th1), expf(th2), 1.0f / (1.0f + expf(-tho)));
            }
        }
    }
    // ---------------- Phase 2: SH chunks ----------------
    if (gi >= S.total) return;
    int s = 0;
    while (s + 1 < S.n && S.s[s + 1].base <= gi) s++;
    const SceneDesc& sc = S.s[s];
    const int64_t g = gi - sc.base;
    const int64_t n = sc.n;
    if (A.grad_only) {
        const int64_t N = S.total;
#pragma unroll
        for (int j = 0; j < 12; j++)
            grads_out[(3 + j) * N + gi] = sG[tid][j];
        return;
    }
    const AdamConst K = sK;
    // the moments of the next pair of chunks are loaded while this pair is
    // updated
    MomWords<MOM16> nw[4];
    {
        const int64_t c0 = 3 * n + g;
        nw[0] = load_mom_words<MOM16>(sc.m, c0);
        nw[1] = load_mom_words<MOM16>(sc.v, c0);
        nw[2] = load_mom_words<MOM16>(sc.m, c0 + n);
        nw[3] = load_mom_words<MOM16>(sc.v, c0 + n);
    }
#pragma unroll 1
    for (int jp = 0; jp < 6; jp++) {          // pairs of chunks = 8 coefficients
        MomWords<MOM16> cw[4];
#pragma unroll
        for (int i = 0; i < 4; i++) cw[i] = nw[i];
        if (jp < 5) {
            const int64_t c0 = (int64_t)(3 + 2 * jp + 2) * n + g;
            nw[0] = load_mom_words<MOM16>(sc.m, c0);
            nw[1] = load_mom_words<MOM16>(sc.v, c0);
            nw[2] = load_mom_words<MOM16>(sc.m, c0 + n);
            nw[3] = load_mom_words<MOM16>(sc.v, c0 + n);
        }
        float th[8];
        if (SH16) {
            const uint4 c = sS16[tid][jp];
            th[0] = bf16_lo(c.x); th[1] = bf16_hi(c.x); th[2] = bf16_lo(c.y); th[3] = bf16_hi(c.y);
            th[4] = bf16_lo(c.z); th[5] = bf16_hi(c.z); th[6] = bf16_lo(c.w); th[7] = bf16_hi(c.w);
        } else {
            const float4 a = sS[tid][2 * jp], b = sS[tid][2 * jp + 1];
            th[0] = a.x; th[1] = a.y; th[2] = a.z; th[3] = a.w; th[4] = b.x; th[5] = b.y; th[6] = b.z; th[7] = b.w;
        }
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int j = 2 * jp + h;
            const int64_t ci = (int64_t)(3 + j) * n + g;
            float4 m = mom_value<MOM16>(cw[2 * h]), vv = mom_value<MOM16>(cw[2 * h + 1]);
            const float4 g4 = sG[tid][j];
            float* mp = &m.x;
            float* vp = &vv.x;
            const float* gp = &g4.x;
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const int f = 4 * j + i;
                adam1(th[4 * h + i], mp[i], vp[i], gp[i], f < 3 ? K.alpha[4] : K.alpha[5], K);
            }
            store_mom<MOM16>(sc.m, ci, m, key, 6u + 2u * j);
            store_mom<MOM16>(sc.v, ci, vv, key, 7u + 2u * j);
        }
        if (!SH16) {
            reinterpret_cast<float4*>(sc.sh)[(int64_t)(2 * jp) * n + g] = make_float4(th[0], th[1], th[2], th[3]);
            reinterpret_cast<float4*>(sc.sh)[(int64_t)(2 * jp + 1) * n + g] = make_float4(th[4], th[5], th[6], th[7]);
        } else {
            uint32_t u[4];
#pragma unroll
            for (int i = 0; i < 4; i++) u[i] = bf16x2_sr(th[2 * i], th[2 * i + 1], sr_bits(key, 64u + 8u * jp + 2 * i));
            reinterpret_cast<uint4*>(sc.sh)[(int64_t)jp * n + g] = make_uint4(u[0], u[1], u[2], u[3]);
        }
    }
}

void launch_project_bwd_adam(const Plan& P, const Scenes& S, const float* cams, const WsPtrs& w,
                             const gs_adam* adam, float* grads_out, cudaStream_t st)
{
    AdamArgs A;
    for (int i = 0; i < 6; i++) A.lr[i] = adam ? adam->lr[i] : 0.f;
    A.b1 = adam ? adam->beta1 : 0.9f;
    A.b2 = adam ? adam->beta2 : 0.999f;
    A.eps = adam ? adam->eps : 1e-15f;
    A.step = adam ? adam->step : 1;
    A.grad_only = grads_out != nullptr;
    A.seed = adam ? adam->seed : 0u;
    const int64_t blocks = (S.total + kPbaThreads - 1) / kPbaThreads;
#define GS_PBA(SH, MO)                                                                                              \
    do {                                                                                                            \
        /* 53 KB (FP32 rows) or 41 KB: above the default 48 KB for FP32 */                                          \
        const size_t smem = (sizeof(float4) * 13 + ShRow<SH>::kRowBytes) * kPbaThreads;                              \
        cudaFuncSetAttribute(k_project_bwd_adam<SH, MO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);   \
        k_project_bwd_adam<SH, MO><<<(unsigned)blocks, kPbaThreads, smem, st>>>(P.views, S, cams, w.count, w.offset, \
                              w.gradrec, A, reinterpret_cast<float4*>(grads_out), w.hdr, (uint32_t)P.cap);         \
    } while (0)
    if (!P.sh_bf16 && !P.mom_bf16) GS_PBA(false, false);
    else if (P.sh_bf16 && P.mom_bf16) GS_PBA(true, true);
    else if (P.sh_bf16) GS_PBA(true, false);
    else GS_PBA(false, true);
#undef GS_PBA
}

}  // namespace gs
