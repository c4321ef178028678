// gs_internal.cuh -- host plan, workspace carving and kernel launchers.
#pragma once

#include <algorithm>
#include <cstddef>
#include <cstring>

#include "gs_device.cuh"

namespace gs {

// Intersection capacity granule (the capacity is rounded up to it).
constexpr int kCapGranule = 2048;

// Per-tile sort: lists of up to kTileSortMax entries are sorted in shared
// memory by one thread block; longer lists are sorted in chunks of that size
// and merged in global memory by the same block.
constexpr int kTileSortThreads = 512;     // 8 keys per thread
constexpr int kTileSortMax = 4096;
constexpr int kTileSortSmall = 128;       // threads for lists of up to 1024 entries

// Exclusive scan geometry: 512 threads x 8 values per block.
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanBlock = kScanThreads * kScanItems;

// Raster backward block: 4 warps.
constexpr int kBwdThreads = 128;

struct Plan {
    Views views;
    int32_t n_scenes;
    int64_t scene_n[kMaxScenes];
    int64_t scene_base[kMaxScenes + 1];
    int64_t cap;                 // intersection capacity
    gs_tuning tuning;
    int32_t sh_bf16, mom_bf16;
    int64_t count_scan_parts;    // ceil(pairs / kScanBlock)
    int64_t tile_scan_parts;     // ceil(tiles / kScanBlock)
    int64_t raster_blocks;       // total tiles
    int32_t sm_count;            // SMs of the device current at plan creation (152 if none)
    // workspace byte offsets
    size_t off_hdr, off_count, off_offset, off_rec, off_span, off_rank;
    size_t off_bucket, off_keys, off_vals, off_pid, off_pid_sorted;
    size_t off_tile_cnt, off_tile_cur;
    size_t off_ranges, off_nlast, off_tfinal, off_gradrec, off_scan_part, off_loss_part, off_order;
    size_t ws_bytes;
};

struct WsPtrs {
    WsHeader* hdr;
    uint32_t* count;           // tiles per pair, Gaussian-major order
    uint32_t* offset;          // its exclusive scan: first emission slot of each pair
    ProjRec* rec;              // projected records, view-major pair order
    uint4* span;               // tile span of each pair, Gaussian-major order
    uint4* rank;               // in-tile ranks of a ranked pair's tiles, Gaussian-major order
    uint2* bucket;             // tile lists in arrival order: (depth code, emission slot)
    uint32_t* pid;             // view-major pair of each emission slot
    uint32_t* keys_sorted;     // sorted keys (tile << shift | depth code)
    uint32_t* vals_sorted;     // emission slot of each sorted entry
    uint32_t* pid_sorted;      // pair of each sorted entry
    uint32_t* tile_cnt;        // [tiles] entries of ranked pairs per global tile, then [tiles] entries of
                               // the other pairs (after the tile scan: their scatter cursors)
    uint32_t* tile_cur;        // tile starts (exclusive scan of both counts)
    uint2* ranges;
    uint32_t* tile_order;      // tiles by decreasing list length (raster launch order)
    uint32_t* nlast;
    float* tfinal;
    GradRec* gradrec;
    uint32_t* scan_part;
    float* loss_part;
};

WsPtrs carve(const Plan& P, void* ws);

// Pixels each raster thread owns (1, 2 or 4; validated by the plan).
inline int tile_ppt(const Plan& P)
{
    const int np = P.views.tw * P.views.th;
    return P.tuning.threads_per_tile > 0 ? np / P.tuning.threads_per_tile : 1;
}

Scenes make_scenes(const Plan& P, const gs_scene_buf* scenes);

void launch_project_fwd(const Plan& P, const Scenes& S, const float* cams, const WsPtrs& w, cudaStream_t st);
void launch_bin_sort(const Plan& P, const WsPtrs& w, cudaStream_t st);
void launch_raster_fwd(const Plan& P, const WsPtrs& w, const float* bg, float* image, cudaStream_t st);
void launch_loss_l1(const Plan& P, const WsPtrs& w, const float* image, const float* target, float* dl,
                    cudaStream_t st);
// Exclusive scan of n u32 (in place allowed); the grand total lands in
// part[ceil(n / kScanBlock)].
void scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* part, cudaStream_t st);
int64_t ssim_tiles(const Views& V);  // 16x16 tiles of the fused L1 + SSIM loss
void launch_loss_l1_ssim(const Plan& P, const WsPtrs& w, const float* image, const void* target_rgba8, float lam,
                         bool alpha_mask, float* dl, cudaStream_t st);
void launch_raster_bwd(const Plan& P, const WsPtrs& w, const float* image, const float* dl, cudaStream_t st);
void launch_raster_bwd2(const Plan& P, const WsPtrs& w, const float* bg, const float* dl, cudaStream_t st);
void launch_project_bwd_adam(const Plan& P, const Scenes& S, const float* cams, const WsPtrs& w,
                             const gs_adam* adam, float* grads_out, cudaStream_t st);
void launch_fill_u32(uint32_t* p, int64_t n, uint32_t value, cudaStream_t st);
void launch_ws_init(const Plan& P, const WsPtrs& w, cudaStream_t st);
void launch_adam_advance(const WsPtrs& w, cudaStream_t st);

}  // namespace gs
