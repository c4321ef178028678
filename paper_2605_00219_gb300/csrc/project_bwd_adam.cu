// project_bwd_adam.cu -- projection backward fused with Adam in one pass
// (VkSplat Sec. 4.3; Table 2 "Proj Bwd + Optim").
//
// One thread per Gaussian.  For every view of its scene the thread sums the
// Gaussian's intersection gradient records (contiguous at its emission
// offset), back-propagates through the SH colour (with the clamp), the view
// direction, the conic inverse, the EWA Jacobian (with the FOV clamp), the
// camera transform and the covariance (scale, quaternion with its
// normalisation), accumulating the parameter gradient in registers.  Then one
// Adam step per parameter group; scale and opacity move to log / logit space
// inside the optimiser and are written back activated, SH degree 0 and
// degrees 1-3 take their own learning rates.  No gradient tensor is stored.
#include "gs_internal.cuh"

namespace gs {

struct AdamArgs {
    float lr[6];
    float b1, b2, eps;
    int step;        // > 0: use it; otherwise the workspace counter + 1
    int grad_only;
};

__device__ __forceinline__ void adam1(float& th, float& m, float& v, float g, float lr, float b1, float b2,
                                      float eps, float ibc1, float ibc2)
{
    m = fmaf(b1, m, (1.0f - b1) * g);
    v = fmaf(b2, v, (1.0f - b2) * g * g);
    th -= lr * (m * ibc1) / (sqrtf(v * ibc2) + eps);
}

// SH coefficient chunk j (flat indices 4j..4j+3) of Gaussian g.
__device__ __forceinline__ float4 sh_chunk(const SceneDesc& sc, int bf16, int64_t g, int j)
{
    if (!bf16) return reinterpret_cast<const float4*>(sc.sh)[(int64_t)j * sc.n + g];
    const uint4 c = reinterpret_cast<const uint4*>(sc.sh)[(int64_t)(j >> 1) * sc.n + g];
    const uint32_t u0 = (j & 1) ? c.z : c.x, u1 = (j & 1) ? c.w : c.y;
    return make_float4(bf16_lo(u0), bf16_hi(u0), bf16_lo(u1), bf16_hi(u1));
}

// Per-view backward of one Gaussian through projection and colour:
// accumulates dmu, dq, ds (activated scale) and dop (activated opacity), and
// returns the SH basis at the view direction (Y) and dL/d(raw colour) (draw)
// so that the SH gradient sum_v Y_v[k] draw_v[c] can be formed later.  The
// SH coefficients are streamed twice (clamp test, then the direction
// gradient) instead of being held in registers.
__device__ __forceinline__ void proj_bwd_view(const float* cam, int W, int H, float4 mu, float4 q, float4 so,
                                              const SceneDesc& sc, int bf16, int64_t g, const float* g2,
                                              float* dmu, float* dq, float* ds, float& dop, float* Y, float* draw)
{
    const float fx = cam[12], fy = cam[13];
    const float* C = cam;
    const float tx = fmaf(C[0], mu.x, fmaf(C[1], mu.y, fmaf(C[2], mu.z, cam[9])));
    const float ty = fmaf(C[3], mu.x, fmaf(C[4], mu.y, fmaf(C[5], mu.z, cam[10])));
    const float tz = fmaf(C[6], mu.x, fmaf(C[7], mu.y, fmaf(C[8], mu.z, cam[11])));
    const float itz = 1.0f / tz;

    // ---- colour: SH and view direction
    const float cpx = -(C[0] * cam[9] + C[3] * cam[10] + C[6] * cam[11]);
    const float cpy = -(C[1] * cam[9] + C[4] * cam[10] + C[7] * cam[11]);
    const float cpz = -(C[2] * cam[9] + C[5] * cam[10] + C[8] * cam[11]);
    const float ddx = mu.x - cpx, ddy = mu.y - cpy, ddz = mu.z - cpz;
    const float idist = rsqrtf(ddx * ddx + ddy * ddy + ddz * ddz);
    const float dirx = ddx * idist, diry = ddy * idist, dirz = ddz * idist;
    sh_basis(dirx, diry, dirz, Y);
    float raw[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
    for (int j = 0; j < 12; j++) {
        const float4 c4 = sh_chunk(sc, bf16, g, j);
        const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
        for (int i = 0; i < 4; i++) raw[(4 * j + i) % 3] = fmaf(cv[i], Y[(4 * j + i) / 3], raw[(4 * j + i) % 3]);
    }
#pragma unroll
    for (int c = 0; c < 3; c++) draw[c] = raw[c] < 0.0f ? 0.0f : g2[6 + c];
    float wk[16];
#pragma unroll
    for (int k = 0; k < 16; k++) wk[k] = 0.f;
#pragma unroll
    for (int j = 0; j < 12; j++) {
        const float4 c4 = sh_chunk(sc, bf16, g, j);
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

    // ---- rotation, scale, 3D covariance
    const float qn_r = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    const float w = q.x * qn_r, x = q.y * qn_r, y = q.z * qn_r, z = q.w * qn_r;
    float R[9];
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
    const float sv[3] = {so.x, so.y, so.z};
    float M[9], Sg[9];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) M[3 * i + j] = R[3 * i + j] * sv[j];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) Sg[3 * i + j] = M[3 * i] * M[3 * j] + M[3 * i + 1] * M[3 * j + 1] + M[3 * i + 2] * M[3 * j + 2];

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
    float TS[6];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int l = 0; l < 3; l++) TS[3 * i + l] = T[3 * i] * Sg[l] + T[3 * i + 1] * Sg[3 + l] + T[3 * i + 2] * Sg[6 + l];
    const float va = TS[0] * T[0] + TS[1] * T[1] + TS[2] * T[2] + 0.3f;
    const float vb = TS[0] * T[3] + TS[1] * T[4] + TS[2] * T[5];
    const float vc = TS[3] * T[3] + TS[4] * T[4] + TS[5] * T[5] + 0.3f;
    const float idet = 1.0f / (va * vc - vb * vb);
    const float qa = vc * idet, qb = -vb * idet, qc = va * idet;
    // dL/dV = -Q G Q, G = [[dca, dcb/2], [dcb/2, dcc]]
    const float ga = g2[2], gb = 0.5f * g2[3], gc = g2[4];
    const float m00 = qa * ga + qb * gb, m01 = qa * gb + qb * gc;
    const float m10 = qb * ga + qc * gb, m11 = qb * gb + qc * gc;
    const float dV00 = -(m00 * qa + m01 * qb), dV01 = -(m00 * qb + m01 * qc);
    const float dV10 = -(m10 * qa + m11 * qb), dV11 = -(m10 * qb + m11 * qc);
    // dSigma = T^T dV T
    float dS[9];
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
        for (int l = 0; l < 3; l++)
            dS[3 * k + l] = T[k] * (dV00 * T[l] + dV01 * T[3 + l]) + T[3 + k] * (dV10 * T[l] + dV11 * T[3 + l]);
    // dT = 2 dV T Sigma, dJ = dT C^T
    float dT[6];
#pragma unroll
    for (int l = 0; l < 3; l++) {
        dT[l] = 2.f * (dV00 * TS[l] + dV01 * TS[3 + l]);
        dT[3 + l] = 2.f * (dV10 * TS[l] + dV11 * TS[3 + l]);
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

    // ---- Sigma = M M^T, M = R diag(s)
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

// MAXV: views of one scene whose (Y, draw) are kept for the SH update; a
// scene with more views than MAXV uses the MAXV = kMaxViews instance.
template <int MAXV>
__global__ void __launch_bounds__(128) k_project_bwd_adam(Views V, Scenes S, const float* __restrict__ cams,
                                                          const uint32_t* __restrict__ count,
                                                          const uint32_t* __restrict__ offset,
                                                          const GradRec* __restrict__ gradrec, AdamArgs A,
                                                          float4* __restrict__ grads_out,
                                                          const WsHeader* __restrict__ hdr, uint32_t cap)
{
    const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= S.total) return;
    int s = 0;
    while (s + 1 < S.n && S.s[s + 1].base <= gi) s++;
    const SceneDesc& sc = S.s[s];
    const int64_t g = gi - sc.base;
    const int64_t n = sc.n;
    float4 mu = sc.geom[g];
    float4 q = sc.geom[n + g];
    float4 so = sc.geom[2 * n + g];

    float dmu[3] = {0.f, 0.f, 0.f}, dq[4] = {0.f, 0.f, 0.f, 0.f}, ds[3] = {0.f, 0.f, 0.f}, dop = 0.f;
    float Yv[MAXV][16], drawv[MAXV][3];
    int nvis = 0;
    for (int v = 0; v < V.n; v++) {
        const ViewDesc& vd = V.v[v];
        if (vd.scene != s) continue;
        const int64_t p = vd.pair_base + g;
        const uint32_t cnt = count[p];
        if (cnt == 0) continue;
        const uint32_t off = offset[p];
        const uint32_t end = min(off + cnt, cap);
        float g2[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (uint32_t e = off; e < end; e++) {
            const GradRec r = gradrec[e];
            g2[0] += r.a.x; g2[1] += r.a.y; g2[2] += r.a.z; g2[3] += r.a.w;
            g2[4] += r.b.x; g2[5] += r.b.y; g2[6] += r.b.z; g2[7] += r.b.w;
            g2[8] += r.c.x;
        }
        float cam[16];
#pragma unroll
        for (int i = 0; i < 16; i++) cam[i] = __ldg(cams + 16 * v + i);
        float Y[16], draw[3];
        proj_bwd_view(cam, vd.W, vd.H, mu, q, so, sc, S.sh_bf16, g, g2, dmu, dq, ds, dop, Y, draw);
        if (nvis < MAXV) {
#pragma unroll
            for (int k = 0; k < 16; k++) Yv[nvis][k] = Y[k];
            drawv[nvis][0] = draw[0]; drawv[nvis][1] = draw[1]; drawv[nvis][2] = draw[2];
            nvis++;
        }
    }

    // SH gradient of flat coefficient f = 3k + c: sum over views of Y_v[k] draw_v[c]
    auto dsh = [&](int f) {
        float acc = 0.f;
#pragma unroll
        for (int i = 0; i < MAXV; i++)
            if (i < nvis) acc = fmaf(Yv[i][f / 3], drawv[i][f % 3], acc);
        return acc;
    };

    if (A.grad_only) {
        float4* go = grads_out;
        const int64_t N = S.total;
        go[0 * N + gi] = make_float4(dmu[0], dmu[1], dmu[2], 0.f);
        go[1 * N + gi] = make_float4(dq[0], dq[1], dq[2], dq[3]);
        go[2 * N + gi] = make_float4(ds[0], ds[1], ds[2], dop);
#pragma unroll
        for (int j = 0; j < 12; j++)
            go[(3 + j) * N + gi] = make_float4(dsh(4 * j), dsh(4 * j + 1), dsh(4 * j + 2), dsh(4 * j + 3));
        return;
    }

    // ---- Adam (FP32 moments), theta = (mean, quat, log s, logit o, SH)
    const int t = A.step > 0 ? A.step : hdr->step + 1;
    const float ibc1 = 1.0f / (1.0f - powf(A.b1, (float)t));
    const float ibc2 = 1.0f / (1.0f - powf(A.b2, (float)t));
    float4* m4 = reinterpret_cast<float4*>(sc.m);
    float4* v4 = reinterpret_cast<float4*>(sc.v);
    {
        float4 m = m4[g], vv = v4[g];
        adam1(mu.x, m.x, vv.x, dmu[0], A.lr[0], A.b1, A.b2, A.eps, ibc1, ibc2);
        adam1(mu.y, m.y, vv.y, dmu[1], A.lr[0], A.b1, A.b2, A.eps, ibc1, ibc2);
        adam1(mu.z, m.z, vv.z, dmu[2], A.lr[0], A.b1, A.b2, A.eps, ibc1, ibc2);
        m4[g] = m; v4[g] = vv;
        sc.geom[g] = mu;
    }
    {
        float4 m = m4[n + g], vv = v4[n + g];
        adam1(q.x, m.x, vv.x, dq[0], A.lr[1], A.b1, A.b2, A.eps, ibc1, ibc2);
        adam1(q.y, m.y, vv.y, dq[1], A.lr[1], A.b1, A.b2, A.eps, ibc1, ibc2);
        adam1(q.z, m.z, vv.z, dq[2], A.lr[1], A.b1, A.b2, A.eps, ibc1, ibc2);
        adam1(q.w, m.w, vv.w, dq[3], A.lr[1], A.b1, A.b2, A.eps, ibc1, ibc2);
        m4[n + g] = m; v4[n + g] = vv;
        sc.geom[n + g] = q;
    }
    {
        float4 m = m4[2 * n + g], vv = v4[2 * n + g];
        float th0 = logf(so.x), th1 = logf(so.y), th2 = logf(so.z);
        float tho = logf(so.w) - log1pf(-so.w);
        adam1(th0, m.x, vv.x, ds[0] * so.x, A.lr[2], A.b1, A.b2, A.eps, ibc1, ibc2);
        adam1(th1, m.y, vv.y, ds[1] * so.y, A.lr[2], A.b1, A.b2, A.eps, ibc1, ibc2);
        adam1(th2, m.z, vv.z, ds[2] * so.z, A.lr[2], A.b1, A.b2, A.eps, ibc1, ibc2);
        adam1(tho, m.w, vv.w, dop * so.w * (1.0f - so.w), A.lr[3], A.b1, A.b2, A.eps, ibc1, ibc2);
        m4[2 * n + g] = m; v4[2 * n + g] = vv;
        sc.geom[2 * n + g] = make_float4(expf(th0), expf(th1), expf(th2), 1.0f / (1.0f + expf(-tho)));
    }
    float4* s4 = reinterpret_cast<float4*>(sc.sh);
#pragma unroll
    for (int j = 0; j < 12; j++) {
        const int64_t ci = (int64_t)(3 + j) * n + g;
        float4 m = m4[ci], vv = v4[ci];
        const float4 c4 = s4[(int64_t)j * n + g];
        float th[4] = {c4.x, c4.y, c4.z, c4.w};
        float* mp = &m.x;
        float* vp = &vv.x;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const float lr = (4 * j + i) < 3 ? A.lr[4] : A.lr[5];
            adam1(th[i], mp[i], vp[i], dsh(4 * j + i), lr, A.b1, A.b2, A.eps, ibc1, ibc2);
        }
        m4[ci] = m; v4[ci] = vv;
        s4[(int64_t)j * n + g] = make_float4(th[0], th[1], th[2], th[3]);
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
    // views per scene decides how many (Y, draw) sets a thread keeps
    int per_scene[kMaxScenes] = {0};
    int maxv = 0;
    for (int v = 0; v < P.views.n; v++) maxv = std::max(maxv, ++per_scene[P.views.v[v].scene]);
    const int T = 128;
    const int64_t blocks = (S.total + T - 1) / T;
#define GS_PBA(MV) k_project_bwd_adam<MV><<<(unsigned)blocks, T, 0, st>>>(P.views, S, cams, w.count, w.offset, \
                                                                     w.gradrec, A, reinterpret_cast<float4*>(grads_out), \
                                                                     w.hdr, (uint32_t)P.cap)
    if (maxv <= 1) GS_PBA(1);
    else if (maxv <= 2) GS_PBA(2);
    else if (maxv <= 4) GS_PBA(4);
    else GS_PBA(kMaxViews);
#undef GS_PBA
}

}  // namespace gs
