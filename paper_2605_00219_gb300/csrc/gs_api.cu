// gs_api.cu -- C ABI of the training step: plan, workspace and the stage
// entry points declared in gs_step.h.
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "gs_internal.cuh"

struct gs_plan {
    gs::Plan p;
};

namespace gs {

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

static int ceil_log2(int64_t n)
{
    int b = 0;
    while (((int64_t)1 << b) < n) b++;
    return b;
}

WsPtrs carve(const Plan& P, void* ws)
{
    char* b = static_cast<char*>(ws);
    WsPtrs w;
    w.hdr = reinterpret_cast<WsHeader*>(b + P.off_hdr);
    w.count = reinterpret_cast<uint32_t*>(b + P.off_count);
    w.offset = reinterpret_cast<uint32_t*>(b + P.off_offset);
    w.rec = reinterpret_cast<ProjRec*>(b + P.off_rec);
    w.span = reinterpret_cast<uint4*>(b + P.off_span);
    w.rank = reinterpret_cast<uint4*>(b + P.off_rank);
    w.bucket = reinterpret_cast<uint2*>(b + P.off_bucket);
    w.keys_sorted = reinterpret_cast<uint32_t*>(b + P.off_keys);
    w.vals_sorted = reinterpret_cast<uint32_t*>(b + P.off_vals);
    w.pid = reinterpret_cast<uint32_t*>(b + P.off_pid);
    w.pid_sorted = reinterpret_cast<uint32_t*>(b + P.off_pid_sorted);
    w.tile_cnt = reinterpret_cast<uint32_t*>(b + P.off_tile_cnt);
    w.tile_cur = reinterpret_cast<uint32_t*>(b + P.off_tile_cur);
    w.ranges = reinterpret_cast<uint2*>(b + P.off_ranges);
    w.tile_order = reinterpret_cast<uint32_t*>(b + P.off_order);
    w.nlast = reinterpret_cast<uint32_t*>(b + P.off_nlast);
    w.tfinal = reinterpret_cast<float*>(b + P.off_tfinal);
    w.gradrec = reinterpret_cast<GradRec*>(b + P.off_gradrec);
    w.scan_part = reinterpret_cast<uint32_t*>(b + P.off_scan_part);
    w.loss_part = reinterpret_cast<float*>(b + P.off_loss_part);
    return w;
}

static bool plan_build(Plan& P, const int64_t* scene_n, int32_t n_scenes, const gs_view* views, int32_t n_views,
                       int64_t cap, const gs_tuning* tuning, int32_t flags)
{
    if (!scene_n || !views || n_scenes < 1 || n_scenes > kMaxScenes || n_views < 1 || n_views > kMaxViews)
        return false;
    memset(&P, 0, sizeof(P));
    {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
            P.sm_count = sms;
        else
            P.sm_count = 152;
        cudaGetLastError();
    }
    gs_tuning t = {16, 16, 0, 0, 0};
    if (tuning) t = *tuning;
    const bool tile_ok = (t.tile_w == 8 && t.tile_h == 8) || (t.tile_w == 16 && t.tile_h == 16) ||
                         (t.tile_w == 16 && t.tile_h == 32);
    if (!tile_ok) return false;
    if (!(t.bwd_batch == 0 || t.bwd_batch == 32 || t.bwd_batch == 64 || t.bwd_batch == 96 || t.bwd_batch == 128))
        return false;
    if (t.bwd_impl < 0 || t.bwd_impl > 2) return false;
    {
        const int np = t.tile_w * t.tile_h;
        const int tpt = t.threads_per_tile;
        const bool ok = tpt == 0 || tpt == np || tpt == np / 2 || (t.tile_w == 16 && tpt == np / 4);
        if (!ok) return false;
        if (tpt != 0 && tpt != np && t.bwd_impl != 0) return false;
        if (tpt == np) t.threads_per_tile = 0;
    }
    if (flags & ~(GS_STORE_SH_BF16 | GS_STORE_MOMENTS_BF16)) return false;
    P.tuning = t;
    P.sh_bf16 = (flags & GS_STORE_SH_BF16) ? 1 : 0;
    P.mom_bf16 = (flags & GS_STORE_MOMENTS_BF16) ? 1 : 0;
    P.n_scenes = n_scenes;
    int64_t base = 0;
    for (int s = 0; s < n_scenes; s++) {
        if (scene_n[s] < 1 || scene_n[s] > ((int64_t)1 << 31)) return false;
        P.scene_n[s] = scene_n[s];
        P.scene_base[s] = base;
        base += scene_n[s];
    }
    P.scene_base[n_scenes] = base;
    Views& V = P.views;
    V.n = n_views;
    V.tw = t.tile_w;
    V.th = t.tile_h;
    V.n_scenes = n_scenes;
    int64_t pairs = 0, tiles = 0, pixels = 0;
    int max_bits = 0;
    for (int v = 0; v < n_views; v++) {
        const gs_view& gv = views[v];
        if (gv.width < 1 || gv.height < 1 || gv.width > 16384 || gv.height > 16384) return false;
        if (gv.scene < 0 || gv.scene >= n_scenes) return false;
        ViewDesc& d = V.v[v];
        d.W = gv.width;
        d.H = gv.height;
        d.TX = (gv.width + t.tile_w - 1) / t.tile_w;
        d.TY = (gv.height + t.tile_h - 1) / t.tile_h;
        d.scene = gv.scene;
        d.rank = V.nv[gv.scene];
        V.view_of[gv.scene][d.rank] = (uint8_t)v;
        V.nv[gv.scene] += 1;
        const int tb = ceil_log2((int64_t)d.TX * d.TY);
        d.shift = tb >= 9 ? 32 - tb : 23;
        d.drop = tb >= 9 ? tb - 9 : 0;
        max_bits = std::max(max_bits, tb >= 9 ? 32 : 23 + tb);
        d.pair_base = pairs;
        d.tile_base = tiles;
        d.pix_base = pixels;
        pairs += scene_n[gv.scene];
        tiles += (int64_t)d.TX * d.TY;
        pixels += (int64_t)gv.width * gv.height;
    }
    V.pairs = pairs;
    V.tiles = tiles;
    V.pixels = pixels;
    (void)max_bits;
    {
        int64_t q = 0;
        for (int sc = 0; sc < n_scenes; sc++) {
            V.qbase[sc] = q;
            q += scene_n[sc] * V.nv[sc];
        }
        V.qbase[n_scenes] = q;
    }
    if (pairs >= ((int64_t)1 << 31) || tiles >= ((int64_t)1 << 31)) return false;
    if (cap <= 0) cap = std::max<int64_t>(4096, 8 * pairs);
    cap = align_up((size_t)cap, kCapGranule);
    if (cap >= ((int64_t)1 << 31)) return false;
    P.cap = cap;
    P.count_scan_parts = (pairs + kScanBlock - 1) / kScanBlock;
    P.tile_scan_parts = (tiles + kScanBlock - 1) / kScanBlock;
    P.raster_blocks = tiles;
    const int64_t loss_blocks = std::max<int64_t>((3 * pixels + 2047) / 2048, 2 * ssim_tiles(V));

    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes, 256);
        return at;
    };
    P.off_hdr = take(sizeof(WsHeader));
    P.off_count = take(4 * (size_t)pairs);
    P.off_offset = take(4 * (size_t)(pairs + 1));
    P.off_rec = take(sizeof(ProjRec) * (size_t)pairs);
    P.off_span = take(16 * (size_t)pairs);
    P.off_rank = take(16 * (size_t)pairs);
    P.off_bucket = take(8 * (size_t)cap);
    P.off_keys = take(4 * (size_t)cap);
    P.off_vals = take(4 * (size_t)cap);
    P.off_pid = take(4 * (size_t)cap);
    P.off_pid_sorted = take(4 * (size_t)cap);
    P.off_tile_cnt = take(4 * 2 * (size_t)tiles);   // ranked counts, then overflow counts
    P.off_tile_cur = take(4 * (size_t)(tiles + 1));
    P.off_ranges = take(8 * (size_t)tiles);
    P.off_order = take(4 * (size_t)tiles);
    P.off_nlast = take(4 * (size_t)pixels);
    P.off_tfinal = take(4 * (size_t)pixels);
    P.off_gradrec = take(sizeof(GradRec) * (size_t)cap);
    P.off_scan_part = take(4 * (size_t)(std::max(P.count_scan_parts, P.tile_scan_parts) + 1));
    P.off_loss_part = take(4 * (size_t)loss_blocks);
    P.ws_bytes = o;
    return true;
}

Scenes make_scenes(const Plan& P, const gs_scene_buf* scenes)
{
    Scenes S;
    memset(&S, 0, sizeof(S));
    S.n = P.n_scenes;
    S.sh_bf16 = P.sh_bf16;
    S.mom_bf16 = P.mom_bf16;
    S.total = P.scene_base[P.n_scenes];
    for (int s = 0; s < P.n_scenes; s++) {
        S.s[s].n = P.scene_n[s];
        S.s[s].base = P.scene_base[s];
        S.s[s].geom = static_cast<float4*>(scenes[s].geom);
        S.s[s].sh = scenes[s].sh;
        S.s[s].m = scenes[s].m;
        S.s[s].v = scenes[s].v;
        S.s[s].stats = static_cast<float2*>(scenes[s].stats);
    }
    return S;
}

// Header reset (and, with `full`, the Adam step counter); the per-tile
// counters that the projection adds to start from zero.
__global__ void k_ws_init(WsHeader* hdr, int full, uint32_t* __restrict__ tile_cnt, int64_t n_cnt)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        hdr->status = 0;
        hdr->k_required = 0;
        hdr->blended = 0;
        hdr->k_eff = 0;
        hdr->loss_counter = 0;
        hdr->loss = 0.f;
        if (full) hdr->step = 0;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_cnt; i += (int64_t)gridDim.x * blockDim.x)
        tile_cnt[i] = 0u;
}

static unsigned init_blocks(const Plan& P)
{
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((P.views.tiles + 255) / 256, (int64_t)P.sm_count * 8));
}

void launch_ws_init(const Plan& P, const WsPtrs& w, cudaStream_t st)
{
    k_ws_init<<<init_blocks(P), 256, 0, st>>>(w.hdr, 1, w.tile_cnt, 2 * P.views.tiles);
}

static void launch_step_begin(const Plan& P, const WsPtrs& w, cudaStream_t st)
{
    k_ws_init<<<init_blocks(P), 256, 0, st>>>(w.hdr, 0, w.tile_cnt, 2 * P.views.tiles);
}

__global__ void k_adam_advance(WsHeader* hdr)
{
    if (threadIdx.x == 0) hdr->step += 1;
}

void launch_adam_advance(const WsPtrs& w, cudaStream_t st) { k_adam_advance<<<1, 32, 0, st>>>(w.hdr); }

__global__ void k_set_step(WsHeader* hdr, int32_t step)
{
    if (threadIdx.x == 0) hdr->step = step;
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// NVTX range around one stage call (host-side push / pop; free when no
// profiler is attached), so a profiler timeline groups the kernels by stage.
struct StageRange {
    explicit StageRange(const char* name) { nvtxRangePushA(name); }
    ~StageRange() { nvtxRangePop(); }
};

static gs_status launch_status()
{
    return cudaPeekAtLastError() == cudaSuccess ? GS_OK : (cudaGetLastError(), GS_ERR_CUDA);
}

}  // namespace gs

using namespace gs;

extern "C" {

gs_plan* gs_plan_create(const int64_t* scene_n, int32_t n_scenes, const gs_view* views, int32_t n_views,
                        int64_t isect_capacity, const gs_tuning* tuning, int32_t storage_flags, gs_status* err)
{
    gs_plan* p = new (std::nothrow) gs_plan;
    if (!p) {
        if (err) *err = GS_ERR_INVALID_ARG;
        return nullptr;
    }
    if (!plan_build(p->p, scene_n, n_scenes, views, n_views, isect_capacity, tuning, storage_flags)) {
        delete p;
        if (err) *err = GS_ERR_INVALID_ARG;
        return nullptr;
    }
    if (err) *err = GS_OK;
    return p;
}

void gs_plan_destroy(gs_plan* plan) { delete plan; }

size_t gs_workspace_bytes(const gs_plan* plan) { return plan ? plan->p.ws_bytes : 0; }

int64_t gs_plan_query(const gs_plan* plan, int32_t what)
{
    if (!plan) return -1;
    const Plan& P = plan->p;
    switch (what) {
    case 0: return P.views.pairs;
    case 1: return P.views.tiles;
    case 2: return P.views.pixels;
    case 3: return P.cap;
    case 4: return P.views.n;
    case 5: return P.n_scenes;
    case 6: return P.views.tw;
    case 7: return P.views.th;
    default: return -1;
    }
}

gs_status gs_workspace_init(const gs_plan* plan, void* ws, void* stream)
{
    if (!plan || !ws || (reinterpret_cast<uintptr_t>(ws) & 255u)) return GS_ERR_INVALID_ARG;
    WsPtrs w = carve(plan->p, ws);
    launch_ws_init(plan->p, w, static_cast<cudaStream_t>(stream));
    return launch_status();
}

static gs_status check_scenes(const Plan& P, const gs_scene_buf* scenes, bool need_moments)
{
    if (!scenes) return GS_ERR_INVALID_ARG;
    for (int s = 0; s < P.n_scenes; s++) {
        const gs_scene_buf& b = scenes[s];
        if (b.n != P.scene_n[s] || !b.geom || !b.sh || !aligned16(b.geom) || !aligned16(b.sh))
            return GS_ERR_INVALID_ARG;
        if (need_moments && (!b.m || !b.v || !aligned16(b.m) || !aligned16(b.v))) return GS_ERR_INVALID_ARG;
    }
    return GS_OK;
}

gs_status gs_project_fwd(const gs_plan* plan, void* ws, const gs_scene_buf* scenes, const float* cams,
                         void* stream)
{
    const StageRange range("gs_project_fwd");
    if (!plan || !ws || !cams) return GS_ERR_INVALID_ARG;
    const Plan& P = plan->p;
    gs_status e = check_scenes(P, scenes, false);
    if (e != GS_OK) return e;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    WsPtrs w = carve(P, ws);
    launch_step_begin(P, w, st);
    launch_project_fwd(P, make_scenes(P, scenes), cams, w, st);
    return launch_status();
}

gs_status gs_bin_sort(const gs_plan* plan, void* ws, void* stream)
{
    const StageRange range("gs_bin_sort");
    if (!plan || !ws) return GS_ERR_INVALID_ARG;
    WsPtrs w = carve(plan->p, ws);
    launch_bin_sort(plan->p, w, static_cast<cudaStream_t>(stream));
    return launch_status();
}

gs_status gs_raster_fwd(const gs_plan* plan, void* ws, const float* bg, float* image, void* stream)
{
    const StageRange range("gs_raster_fwd");
    if (!plan || !ws || !image || !aligned16(image)) return GS_ERR_INVALID_ARG;
    WsPtrs w = carve(plan->p, ws);
    launch_raster_fwd(plan->p, w, bg, image, static_cast<cudaStream_t>(stream));
    return launch_status();
}

gs_status gs_loss_l1(const gs_plan* plan, void* ws, const float* image, const float* target, float* dL_dimage,
                     void* stream)
{
    const StageRange range("gs_loss_l1");
    if (!plan || !ws || !image || !target || !dL_dimage) return GS_ERR_INVALID_ARG;
    WsPtrs w = carve(plan->p, ws);
    launch_loss_l1(plan->p, w, image, target, dL_dimage, static_cast<cudaStream_t>(stream));
    return launch_status();
}

static gs_status loss_l1_ssim(const gs_plan* plan, void* ws, const float* image, const void* target_rgba8,
                              float lambda, bool alpha_mask, float* dL_dimage, void* stream)
{
    if (!plan || !ws || !image || !target_rgba8 || !dL_dimage) return GS_ERR_INVALID_ARG;
    if (!(lambda >= 0.f && lambda <= 1.f)) return GS_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(target_rgba8) % 4 != 0) return GS_ERR_INVALID_ARG;
    WsPtrs w = carve(plan->p, ws);
    launch_loss_l1_ssim(plan->p, w, image, target_rgba8, lambda, alpha_mask, dL_dimage,
                        static_cast<cudaStream_t>(stream));
    return launch_status();
}

gs_status gs_loss_l1_ssim(const gs_plan* plan, void* ws, const float* image, const void* target_rgba8, float lambda,
                          float* dL_dimage, void* stream)
{
    const StageRange range("gs_loss_l1_ssim");
    return loss_l1_ssim(plan, ws, image, target_rgba8, lambda, false, dL_dimage, stream);
}

gs_status gs_loss_l1_ssim_masked(const gs_plan* plan, void* ws, const float* image, const void* target_rgba8,
                                 float lambda, float* dL_dimage, void* stream)
{
    const StageRange range("gs_loss_l1_ssim_masked");
    return loss_l1_ssim(plan, ws, image, target_rgba8, lambda, true, dL_dimage, stream);
}

gs_status gs_raster_bwd(const gs_plan* plan, void* ws, const float* image, const float* dL_dimage, void* stream)
{
    const StageRange range("gs_raster_bwd");
    if (!plan || !ws || !image || !dL_dimage) return GS_ERR_INVALID_ARG;
    WsPtrs w = carve(plan->p, ws);
    launch_raster_bwd(plan->p, w, image, dL_dimage, static_cast<cudaStream_t>(stream));
    return launch_status();
}

gs_status gs_project_bwd_adam(const gs_plan* plan, void* ws, const gs_scene_buf* scenes, const float* cams,
                              const gs_adam* adam, float* grads_out, void* stream)
{
    const StageRange range("gs_project_bwd_adam");
    if (!plan || !ws || !cams) return GS_ERR_INVALID_ARG;
    const Plan& P = plan->p;
    if (!grads_out && !adam) return GS_ERR_INVALID_ARG;
    if (grads_out && !aligned16(grads_out)) return GS_ERR_INVALID_ARG;
    gs_status e = check_scenes(P, scenes, grads_out == nullptr);
    if (e != GS_OK) return e;
    WsPtrs w = carve(P, ws);
    launch_project_bwd_adam(P, make_scenes(P, scenes), cams, w, adam, grads_out, static_cast<cudaStream_t>(stream));
    return launch_status();
}

gs_status gs_adam_advance(const gs_plan* plan, void* ws, void* stream)
{
    if (!plan || !ws) return GS_ERR_INVALID_ARG;
    WsPtrs w = carve(plan->p, ws);
    launch_adam_advance(w, static_cast<cudaStream_t>(stream));
    return launch_status();
}

gs_status gs_workspace_set_step(const gs_plan* plan, void* ws, int32_t step, void* stream)
{
    if (!plan || !ws || step < 0) return GS_ERR_INVALID_ARG;
    WsPtrs w = carve(plan->p, ws);
    k_set_step<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(w.hdr, step);
    return launch_status();
}

gs_status gs_read_stats(const gs_plan* plan, const void* ws, gs_stats* out, void* stream)
{
    if (!plan || !ws || !out) return GS_ERR_INVALID_ARG;
    WsPtrs w = carve(plan->p, const_cast<void*>(ws));
    WsHeader h;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(&h, w.hdr, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess) return GS_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return GS_ERR_CUDA;
    out->status = h.status;
    out->step = h.step;
    out->k_required = (int64_t)h.k_required;
    out->k_capacity = plan->p.cap;
    out->blended_pairs = h.blended;
    out->loss = h.loss;
    out->reserved = 0.f;
    return GS_OK;
}

void* gs_workspace_buffer(const gs_plan* plan, void* ws, int32_t which)
{
    if (!plan || !ws) return nullptr;
    WsPtrs w = carve(plan->p, ws);
    switch (which) {
    case 0: return w.count;
    case 1: return w.offset;
    case 2: return w.keys_sorted;
    case 3: return w.pid_sorted;
    case 4: return w.ranges;
    case 5: return w.nlast;
    case 6: return w.tfinal;
    case 7: return w.rec;
    case 8: return w.gradrec;
    case 9: return w.vals_sorted;
    case 10: return w.span;
    case 11: return w.rank;
    case 12: return w.tile_cnt;
    default: return nullptr;
    }
}

const char* gs_status_str(gs_status s)
{
    switch (s) {
    case GS_OK: return "ok";
    case GS_ERR_INVALID_ARG: return "invalid argument";
    case GS_ERR_CAPACITY: return "intersection capacity exceeded";
    case GS_ERR_NONFINITE: return "non-finite parameter";
    case GS_ERR_TIMEOUT: return "bounded wait gave up";
    case GS_ERR_CUDA: return "CUDA launch error";
    case GS_ERR_UNIMPLEMENTED: return "not implemented";
    default: return "unknown status";
    }
}

}  // extern "C"
