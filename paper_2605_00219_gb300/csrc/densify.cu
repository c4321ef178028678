// densify.cu -- default densification (VkSplat Sec. 4.6, which follows the
// 3DGS default strategy) and the opacity reset, on the chunk-major scene
// layout.
//
// Two passes over the Gaussians: a decision pass writes three 0/1 arrays
// (kept as is, cloned, split and kept) that are scanned into output
// positions; an apply pass copies every survivor, writes the clones and the
// two products of every split to their positions, zeroes the new Gaussians'
// Adam moments and all statistics.  Decisions are binary32 comparisons of
// stored (activated) values, so they are exact.
#include "gs_internal.cuh"

namespace gs {

struct DensifyK {
    float grad_thr;     // grow_grad2d
    float small_thr;    // grow_scale3d * scene_scale (binary32 product)
    float prune_opa;
    float big_thr;      // prune_scale3d * scene_scale
    float factor;       // split_factor
    int grow, prune_big;
};

struct DensifyScratch {
    int64_t* counts;    // [4]: kept, clones, splits, total
    uint32_t *a, *b, *c;
    uint32_t *pa, *pb, *pc;
};

static int64_t ds_parts(int64_t n) { return (n + 1 + kScanBlock - 1) / kScanBlock; }

static size_t ds_align(size_t x) { return (x + 255) & ~(size_t)255; }

static size_t ds_layout(int64_t n, void* base, DensifyScratch* d)
{
    char* p = static_cast<char*>(base);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = ds_align(o + bytes);
        return p ? p + at : nullptr;
    };
    const size_t arr = 4 * (size_t)(n + 1), part = 4 * (size_t)(ds_parts(n) + 1);
    char* counts = take(4 * sizeof(int64_t));
    char* a = take(arr);
    char* b = take(arr);
    char* c = take(arr);
    char* pa = take(part);
    char* pb = take(part);
    char* pc = take(part);
    if (d) {
        d->counts = reinterpret_cast<int64_t*>(counts);
        d->a = reinterpret_cast<uint32_t*>(a);
        d->b = reinterpret_cast<uint32_t*>(b);
        d->c = reinterpret_cast<uint32_t*>(c);
        d->pa = reinterpret_cast<uint32_t*>(pa);
        d->pb = reinterpret_cast<uint32_t*>(pb);
        d->pc = reinterpret_cast<uint32_t*>(pc);
    }
    return o;
}

__global__ void k_densify_decide(int64_t n, const float4* __restrict__ geom, const float2* __restrict__ stats,
                                 DensifyK K, uint32_t* __restrict__ a, uint32_t* __restrict__ b,
                                 uint32_t* __restrict__ c)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) a[n] = b[n] = c[n] = 0u;
    if (i >= n) return;
    const float4 so = geom[2 * n + i];
    const float2 st = stats[i];
    const float avg = __fdiv_rn(st.x, fmaxf(st.y, 1.0f));
    const bool high = K.grow && avg > K.grad_thr;
    const float ms = fmaxf(fmaxf(so.x, so.y), so.z);
    const bool small = ms <= K.small_thr;
    const bool clone = high && small, split = high && !small;
    const bool low_o = so.w < K.prune_opa;
    const bool big = K.prune_big && ms > K.big_thr;
    const bool big_split = K.prune_big && __fdiv_rn(ms, K.factor) > K.big_thr;
    a[i] = (!split && !(low_o || big)) ? 1u : 0u;
    b[i] = (clone && !(low_o || big)) ? 1u : 0u;
    c[i] = (split && !(low_o || big_split)) ? 1u : 0u;
}

__global__ void k_densify_total(int64_t n, const uint32_t* __restrict__ a, const uint32_t* __restrict__ b,
                                const uint32_t* __restrict__ c, int64_t* __restrict__ counts)
{
    if (threadIdx.x == 0) {
        const int64_t na = a[n], nb = b[n], nc = c[n];
        counts[0] = na;
        counts[1] = nb;
        counts[2] = nc;
        counts[3] = na + nb + 2 * nc;
    }
}

// Copy one Gaussian's row from `in` (row i) to `out` (row j); moments copied
// or zeroed.
template <bool SH16, bool MOM16>
__device__ __forceinline__ void ds_copy(const SceneDesc& in, int64_t i, const SceneDesc& out, int64_t j, bool keep_mom,
                                        float4 g0, float4 g1, float4 g2)
{
    const int64_t n = in.n, m = out.n;
    out.geom[j] = g0;
    out.geom[m + j] = g1;
    out.geom[2 * m + j] = g2;
    if (SH16) {
        const uint4* s = static_cast<const uint4*>(in.sh);
        uint4* d = static_cast<uint4*>(out.sh);
#pragma unroll
        for (int k = 0; k < 6; k++) d[k * m + j] = s[k * n + i];
    } else {
        const float4* s = static_cast<const float4*>(in.sh);
        float4* d = static_cast<float4*>(out.sh);
#pragma unroll
        for (int k = 0; k < 12; k++) d[k * m + j] = s[k * n + i];
    }
    if (MOM16) {
        const uint2* sm = static_cast<const uint2*>(in.m);
        const uint2* sv = static_cast<const uint2*>(in.v);
        uint2* dm = static_cast<uint2*>(out.m);
        uint2* dv = static_cast<uint2*>(out.v);
#pragma unroll
        for (int k = 0; k < 15; k++) {
            dm[k * m + j] = keep_mom ? sm[k * n + i] : make_uint2(0u, 0u);
            dv[k * m + j] = keep_mom ? sv[k * n + i] : make_uint2(0u, 0u);
        }
    } else {
        const float4* sm = static_cast<const float4*>(in.m);
        const float4* sv = static_cast<const float4*>(in.v);
        float4* dm = static_cast<float4*>(out.m);
        float4* dv = static_cast<float4*>(out.v);
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 15; k++) {
            dm[k * m + j] = keep_mom ? sm[k * n + i] : z;
            dv[k * m + j] = keep_mom ? sv[k * n + i] : z;
        }
    }
    if (out.stats) out.stats[j] = make_float2(0.f, 0.f);
}

template <bool SH16, bool MOM16>
__global__ void k_densify_apply(SceneDesc in, SceneDesc out, const uint32_t* __restrict__ a,
                                const uint32_t* __restrict__ b, const uint32_t* __restrict__ c,
                                const int64_t* __restrict__ counts, const float* __restrict__ eps, float factor)
{
    const int64_t n = in.n;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || counts[3] != out.n) return;   // wrong output size: write nothing
    const bool keep = a[i + 1] != a[i], clone = b[i + 1] != b[i], split = c[i + 1] != c[i];
    if (!keep && !clone && !split) return;
    const int64_t na = a[n], nb = b[n], nc = c[n];
    const float4 g0 = in.geom[i], g1 = in.geom[n + i], g2 = in.geom[2 * n + i];
    if (keep) ds_copy<SH16, MOM16>(in, i, out, a[i], true, g0, g1, g2);
    if (clone) ds_copy<SH16, MOM16>(in, i, out, na + b[i], false, g0, g1, g2);
    if (split) {
        // R(q) of the normalised quaternion (w, x, y, z), as in the projection
        const float qn = rsqrtf(g1.x * g1.x + g1.y * g1.y + g1.z * g1.z + g1.w * g1.w);
        const float w = g1.x * qn, x = g1.y * qn, y = g1.z * qn, z = g1.w * qn;
        const float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                            2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                            2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
        const float4 g2n = make_float4(__fdiv_rn(g2.x, factor), __fdiv_rn(g2.y, factor), __fdiv_rn(g2.z, factor),
                                       g2.w);
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const float* e = eps + 6 * i + 3 * h;
            const float lx = g2.x * e[0], ly = g2.y * e[1], lz = g2.z * e[2];
            const float4 g0n = make_float4(g0.x + (R[0] * lx + R[1] * ly + R[2] * lz),
                                           g0.y + (R[3] * lx + R[4] * ly + R[5] * lz),
                                           g0.z + (R[6] * lx + R[7] * ly + R[8] * lz), g0.w);
            ds_copy<SH16, MOM16>(in, i, out, na + nb + (h ? nc : 0) + c[i], false, g0n, g1, g2n);
        }
    }
}

template <bool MOM16>
__global__ void k_reset_opacity(SceneDesc sc, float value)
{
    const int64_t n = sc.n;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 so = sc.geom[2 * n + i];
    so.w = fminf(so.w, value);
    sc.geom[2 * n + i] = so;
    if (MOM16) {
        uint2* m = static_cast<uint2*>(sc.m);
        uint2* v = static_cast<uint2*>(sc.v);
        m[2 * n + i].y &= 0x0000FFFFu;   // the fourth bf16 is the logit-opacity moment
        v[2 * n + i].y &= 0x0000FFFFu;
    } else {
        static_cast<float4*>(sc.m)[2 * n + i].w = 0.f;
        static_cast<float4*>(sc.v)[2 * n + i].w = 0.f;
    }
}

static SceneDesc ds_scene(const gs_scene_buf& b)
{
    SceneDesc s;
    s.n = b.n;
    s.base = 0;
    s.geom = static_cast<float4*>(b.geom);
    s.sh = b.sh;
    s.m = b.m;
    s.v = b.v;
    s.stats = static_cast<float2*>(b.stats);
    return s;
}

static bool ds_cfg_ok(const gs_densify_cfg* c)
{
    auto fin = [](float x) { return x == x && x - x == 0.0f; };
    return c && fin(c->grow_grad2d) && fin(c->grow_scale3d) && fin(c->prune_opa) && fin(c->prune_scale3d) &&
           fin(c->scene_scale) && fin(c->split_factor) && c->scene_scale > 0.f && c->split_factor > 0.f &&
           c->grow_grad2d >= 0.f && c->grow_scale3d > 0.f && c->prune_scale3d > 0.f;
}

static bool ds_scene_ok(const gs_scene_buf* s)
{
    return s && s->n >= 1 && s->n < ((int64_t)1 << 31) && s->geom && s->sh && s->m && s->v;
}

static gs_status ds_launch_status()
{
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // namespace gs

using namespace gs;

extern "C" {

size_t gs_densify_scratch_bytes(int64_t n)
{
    if (n < 1) return 0;
    return ds_layout(n, nullptr, nullptr);
}

gs_status gs_densify_count(const gs_scene_buf* scene, int32_t storage_flags, const gs_densify_cfg* cfg,
                           void* scratch, void* stream)
{
    (void)storage_flags;
    if (!ds_scene_ok(scene) || !scene->stats || !scratch || !ds_cfg_ok(cfg)) return GS_ERR_INVALID_ARG;
    const int64_t n = scene->n;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DensifyScratch d;
    ds_layout(n, scratch, &d);
    DensifyK K;
    K.grad_thr = cfg->grow_grad2d;
    K.small_thr = cfg->grow_scale3d * cfg->scene_scale;
    K.prune_opa = cfg->prune_opa;
    K.big_thr = cfg->prune_scale3d * cfg->scene_scale;
    K.factor = cfg->split_factor;
    K.grow = cfg->grow != 0;
    K.prune_big = cfg->prune_big != 0;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    k_densify_decide<<<blocks, 256, 0, st>>>(n, static_cast<const float4*>(scene->geom),
                                             static_cast<const float2*>(scene->stats), K, d.a, d.b, d.c);
    scan_u32(d.a, d.a, n + 1, d.pa, st);
    scan_u32(d.b, d.b, n + 1, d.pb, st);
    scan_u32(d.c, d.c, n + 1, d.pc, st);
    k_densify_total<<<1, 32, 0, st>>>(n, d.a, d.b, d.c, d.counts);
    return ds_launch_status();
}

gs_status gs_densify_counts(const void* scratch, int64_t counts[4], void* stream)
{
    if (!scratch || !counts) return GS_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(counts, scratch, 4 * sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return GS_ERR_CUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

gs_status gs_densify_apply(const gs_scene_buf* in, int32_t storage_flags, const gs_densify_cfg* cfg,
                           const float* eps, const void* scratch, gs_scene_buf* out, void* stream)
{
    if (!ds_scene_ok(in) || !ds_scene_ok(out) || !eps || !scratch || !ds_cfg_ok(cfg)) return GS_ERR_INVALID_ARG;
    const int64_t n = in->n;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DensifyScratch d;
    ds_layout(n, const_cast<void*>(scratch), &d);
    const SceneDesc si = ds_scene(*in), so = ds_scene(*out);
    const unsigned blocks = (unsigned)((n + 255) / 256);
    const bool sh16 = storage_flags & GS_STORE_SH_BF16, mom16 = storage_flags & GS_STORE_MOMENTS_BF16;
#define GS_DA(A, B) k_densify_apply<A, B><<<blocks, 256, 0, st>>>(si, so, d.a, d.b, d.c, d.counts, eps, \
                                                                  cfg->split_factor)
    if (sh16 && mom16) GS_DA(true, true);
    else if (sh16) GS_DA(true, false);
    else if (mom16) GS_DA(false, true);
    else GS_DA(false, false);
#undef GS_DA
    return ds_launch_status();
}

gs_status gs_reset_opacity(const gs_scene_buf* scene, int32_t storage_flags, float value, void* stream)
{
    if (!ds_scene_ok(scene) || !(value == value)) return GS_ERR_INVALID_ARG;
    const SceneDesc s = ds_scene(*scene);
    const unsigned blocks = (unsigned)((scene->n + 255) / 256);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (storage_flags & GS_STORE_MOMENTS_BF16) k_reset_opacity<true><<<blocks, 256, 0, st>>>(s, value);
    else k_reset_opacity<false><<<blocks, 256, 0, st>>>(s, value);
    return ds_launch_status();
}

}  // extern "C"
