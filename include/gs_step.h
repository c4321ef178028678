/*
 * gs_step.h -- C ABI of the GB300 (sm_103a) 3D Gaussian Splatting training
 * step: the stages of one training iteration of VkSplat (arxiv 2605.00219,
 * Sec. 2 pipeline and Sec. 4), each a call on a CUDA stream.
 *
 *   gs_project_fwd      projection forward + exact tile count  (Sec. 4.1)
 *   gs_bin_sort         index offset, key generation, the stable order of
 *                       the 32-bit keys (per-tile lists), tile
 *                       ranges                                  (Sec. 4.1, 4.4)
 *   gs_raster_fwd       front-to-back alpha compositing         (Sec. 2)
 *   gs_loss_l1          L1 loss and its gradient                (Sec. 4.5, L1 term)
 *   gs_loss_l1_ssim     L1 + SSIM loss, RGBA8 reference         (Sec. 4.5)
 *   gs_loss_l1_ssim_masked  the same with the reference's alpha as mask
 *   gs_raster_bwd       per-Gaussian rasterization backward     (Sec. 4.2)
 *   gs_project_bwd_adam projection backward fused with Adam     (Sec. 4.3)
 *
 * Conventions shared by every call:
 *  - Ownership: the caller allocates every device buffer, including the
 *    workspace of gs_workspace_bytes() bytes (256-byte aligned).  The library
 *    never allocates, frees or synchronises device memory inside the step
 *    calls; only gs_plan_create/destroy allocate, and only host memory.
 *  - All step calls are asynchronous on `stream` (a cudaStream_t passed as
 *    void*, NULL = legacy default stream) and may be captured in a CUDA graph.
 *    The intersection count K never leaves the device.
 *  - Errors: invalid host-visible arguments return GS_ERR_INVALID_ARG before
 *    anything is launched; a failed launch returns GS_ERR_CUDA.  Errors the
 *    device detects (intersection capacity exceeded, non-finite parameters, a
 *    bounded wait that gave up) set bits in a status word inside the
 *    workspace, read with gs_read_stats().  No call aborts, traps or prints.
 *  - Device pointers must be 16-byte aligned.
 *
 * Data layouts (n = Gaussians of a scene; all device memory):
 *  - geom:  float4[3][n], chunk-major: chunk 0 = mean (x, y, z, unused),
 *           chunk 1 = rotation quaternion (w, x, y, z, need not be unit),
 *           chunk 2 = (scale x, y, z, opacity), stored ACTIVATED (scales > 0,
 *           opacity in (0,1)), as the paper stores them (Sec. 4.3, Sec. 4.6).
 *  - sh:    degree-3 SH, 48 coefficients per Gaussian, flat index 3*k + c
 *           (k = basis function 0..15, c = colour channel).  FP32 storage:
 *           float4[12][n] ("column-based" 128-bit chunks, Sec. 4.6), chunk j
 *           holding flat indices 4j..4j+3.  BF16 storage: uint4[6][n], chunk j
 *           holding flat indices 8j..8j+7 as bf16 (low half first).
 *  - m, v:  Adam moments of theta = (mean, quaternion, log-scale,
 *           logit-opacity, SH), in the chunk order of geom followed by sh:
 *           FP32: float4[15][n]; BF16: uint2[15][n] (4 bf16 per chunk).
 *  - cams:  float[n_views][16]: R (row-major 3x3, world -> camera, OpenCV
 *           axes x right, y down, z forward), t (3), fx, fy, cx, cy.
 *  - image: float[sum over views of H*W][3], views concatenated, each
 *           row-major, channel-last (Sec. 4.5).
 */
#ifndef GS_STEP_H
#define GS_STEP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GS_MAX_VIEWS 64
#define GS_MAX_SCENES 16

typedef enum {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = 1,
    GS_ERR_CAPACITY = 2,      /* status bit 1: more intersections than capacity */
    GS_ERR_NONFINITE = 3,     /* status bit 2: a non-finite parameter was found */
    GS_ERR_TIMEOUT = 4,       /* status bit 3: a bounded wait gave up (reserved: no kernel of
                                 this library waits on another block, so it is never set) */
    GS_ERR_CUDA = 5,
    GS_ERR_UNIMPLEMENTED = 6
} gs_status;

/* Device status word bits (gs_stats.status). */
#define GS_STATUS_CAPACITY 0x1u
#define GS_STATUS_NONFINITE 0x2u
#define GS_STATUS_TIMEOUT 0x4u     /* reserved, never set (no kernel waits) */
#define GS_STATUS_BOUNDS 0x8u      /* bounds-checked build (GS_DEBUG) only: an
                                      index read from the workspace pointed
                                      outside its buffer; that access was
                                      skipped */

/* Storage flags for gs_plan_create. */
#define GS_STORE_SH_BF16 0x1
#define GS_STORE_MOMENTS_BF16 0x2

typedef struct {
    int32_t width, height;    /* pixels */
    int32_t scene;            /* index of the scene this view renders */
} gs_view;

typedef struct {
    int32_t tile_w, tile_h;   /* 8x8, 16x16 or 16x32 pixels */
    int32_t bwd_batch;        /* per-Gaussian raster_bwd batch S: 0 = the
                                 paper's adaptive rule S = roundup32(sqrt(N P))
                                 <= 128 (Sec. 4.2); else a fixed 32, 64, 96 or
                                 128 */
    int32_t bwd_impl;         /* raster_bwd implementation: 0 = pixels across
                                 threads with per-Gaussian warp-shuffle
                                 reductions, 1 = Gaussians across threads in
                                 batches of S (the paper's first
                                 implementation, Sec. 4.2), 2 = a pass over
                                 pixels storing per-pair transmittance terms
                                 in shared memory, then a pass over
                                 (Gaussian, pixel block) pairs summing them
                                 (the paper's second implementation) */
    int32_t threads_per_tile; /* threads of a raster_bwd thread block
                                 (bwd_impl 0): 0 or tile_w x tile_h = one per
                                 pixel; half or (16-wide tiles) a quarter of
                                 that = 2 or 4 pixels per thread, each warp
                                 covering 8 x 8 or 8 x 16 pixels (Sec. 4.2: the
                                 scheduler's threads per tile).  Pixels per
                                 thread other than 1 need bwd_impl 0.  The
                                 raster forward always runs one thread per
                                 pixel. */
} gs_tuning;

typedef struct {
    int64_t n;                /* Gaussians in this scene */
    void* geom;               /* float4[3][n] */
    void* sh;                 /* float4[12][n] or uint4[6][n] (BF16) */
    void* m;                  /* float4[15][n] or uint2[15][n] (BF16) */
    void* v;                  /* same as m */
    void* stats;              /* NULL, or float2[n] densification statistics
                                 that gs_project_bwd_adam adds to: x += the
                                 norm of dL/d(mean2D) of every view in which
                                 the Gaussian is listed, in half-image units
                                 (x scaled by W/2, y by H/2) and as if that
                                 view's loss were its own mean (x P_all/P_v);
                                 y += the number of such views */
} gs_scene_buf;

typedef struct {
    float lr[6];              /* mean, quaternion, log-scale, logit-opacity,
                                 SH degree 0, SH degrees 1-3 (Sec. 4.3) */
    float beta1, beta2, eps;
    int32_t step;             /* Adam step t >= 1; 0 = take t from the
                                 workspace step counter (then advanced by
                                 gs_adam_advance), for graph replay */
    uint32_t seed;            /* stochastic-rounding seed for BF16 storage */
    int32_t reserved;
} gs_adam;

typedef struct {
    uint32_t status;          /* GS_STATUS_* bits */
    int32_t step;             /* workspace step counter */
    int64_t k_required;       /* intersections the last gs_project_fwd needed */
    int64_t k_capacity;
    uint64_t blended_pairs;   /* pairs composited by the last gs_raster_fwd */
    float loss;               /* last gs_loss_l1 / gs_loss_l1_ssim value */
    float reserved;
} gs_stats;

typedef struct gs_plan gs_plan;   /* opaque, host memory */

/* Build the static shape of a step: scenes (Gaussian counts), views
 * (resolution and scene), intersection capacity (0 = 8 x total pairs,
 * rounded), tuning (NULL = 16x16 tiles, adaptive batch) and storage flags.
 * Returns NULL on invalid arguments (and sets *err when err != NULL). */
gs_plan* gs_plan_create(const int64_t* scene_n, int32_t n_scenes, const gs_view* views,
                        int32_t n_views, int64_t isect_capacity, const gs_tuning* tuning,
                        int32_t storage_flags, gs_status* err);
void gs_plan_destroy(gs_plan* plan);

/* Workspace bytes the caller must allocate for this plan (device memory). */
size_t gs_workspace_bytes(const gs_plan* plan);

/* Plan queries: 0 pairs (sum over views of the scene's n), 1 total tiles,
 * 2 total pixels, 3 intersection capacity, 4 views, 5 scenes, 6 tile_w,
 * 7 tile_h.  Returns -1 for an unknown query. */
int64_t gs_plan_query(const gs_plan* plan, int32_t what);

/* Zero the workspace status word, statistics and step counter. */
gs_status gs_workspace_init(const gs_plan* plan, void* ws, void* stream);

/* Projection forward (EWA splatting with the 0.3 low-pass, degree-3 SH
 * colour) for every (view, Gaussian) pair, fused with the exact scan-line
 * count of intersected tiles (Sec. 4.1 counts tiles during projection and
 * emits them in a later pass).  Reads geom and sh of every scene and cams;
 * writes the projected records, the counts, the per-tile counts and each
 * pair's tile span (the bands of its traversal, for the emission) into ws. */
gs_status gs_project_fwd(const gs_plan* plan, void* ws, const gs_scene_buf* scenes,
                         const float* cams, void* stream);

/* Tiling and sorting (Sec. 4.1, Sec. 4.4, Table 2 "Tiling/Sorting"):
 * exclusive scan of the counts ("index offset"), per-tile [start, end)
 * ranges from the per-tile counts of the projection's traversal, an
 * emission of every intersected tile into its tile's list ("generate keys";
 * the tiles come from the tile spans the traversal kept, and a pair of more
 * than two bands repeats the scan-line pass), and a sort of each tile's list, so that the lists hold
 * the 32-bit keys (tile id in the top ceil(log2 tiles) bits, depth code
 * (2z+1)/(z+1) mantissa below) in the order of a stable sort of the keys,
 * view by view (ties in emission order, i.e. by Gaussian).  K stays on the
 * device; if it exceeds the capacity, GS_STATUS_CAPACITY is set and every
 * tile list is left empty. */
gs_status gs_bin_sort(const gs_plan* plan, void* ws, void* stream);

/* Front-to-back compositing per tile (Sec. 2): alpha = min(0.99, o exp(-d^2/2))
 * for d^2 <= 9, pairs below 1/255 skipped, stop before T(1-alpha) < 1e-4,
 * transmittance kept as a compensated FP32 pair.  bg: device float[3] or
 * NULL (black).  image: device float[pixels][3].  Also records per pixel the
 * final transmittance and the list position after the last blended pair. */
gs_status gs_raster_fwd(const gs_plan* plan, void* ws, const float* bg, float* image,
                        void* stream);

/* L1 loss over all pixels of all views (mean over 3 x pixels) and its
 * gradient dL/dC = sign(C - C*) / (3 x pixels) (Sec. 4.5, L1 term).
 * target: device float[pixels][3]; dL_dimage: device float[pixels][3].
 * The loss value lands in the workspace statistics. */
gs_status gs_loss_l1(const gs_plan* plan, void* ws, const float* image, const float* target,
                     float* dL_dimage, void* stream);

/* Weighted L1 + SSIM loss (Sec. 4.5) against an 8-bit RGBA reference and its
 * gradient, fused in one kernel:
 *   L = (1 - lambda) mean|C - C*| + lambda (1 - mean SSIM),
 * SSIM per colour channel with an 11x11 Gaussian window (sigma 1.5), zero
 * padding at the image border, C1 = 0.01^2, C2 = 0.03^2; means over
 * 3 x pixels of all views.  target_rgba8: device uint8[pixels][4] (R, G, B, A;
 * A ignored here, the mask of gs_loss_l1_ssim_masked; colour = byte / 255),
 * 4-byte aligned; image and dL_dimage:
 * device float[pixels][3].  lambda in [0, 1] (the paper uses 0.2), else
 * GS_ERR_INVALID_ARG.  The loss value lands in the workspace statistics.
 * Deterministic: per-tile partial sums added in a fixed order. */
gs_status gs_loss_l1_ssim(const gs_plan* plan, void* ws, const float* image,
                          const void* target_rgba8, float lambda, float* dL_dimage,
                          void* stream);

/* The same loss with alpha masking (Sec. 4.5 fuses it into the loss): the
 * reference's alpha m = A / 255 multiplies both the render and the reference
 * before the loss, so pixels with m = 0 add nothing to it, and dL_dimage
 * carries the factor m.  Arguments and errors as gs_loss_l1_ssim. */
gs_status gs_loss_l1_ssim_masked(const gs_plan* plan, void* ws, const float* image,
                                 const void* target_rgba8, float lambda, float* dL_dimage,
                                 void* stream);

/* Rasterization backward (Sec. 4.2), one thread block per tile, no atomics:
 * one 9-float gradient record (mean2D, conic, opacity, colour) per
 * intersection, summed in a fixed order (deterministic).  Transmittance is
 * recomputed per tile (nothing per pair is kept from the forward).
 * tuning.bwd_impl = 1: the paper's first implementation -- Gaussians of the
 * tile in batches of S across threads, T recomputed front to back;
 * tuning.bwd_impl = 2: the paper's second implementation -- per batch, a
 * pass over pixels stores each (Gaussian, pixel) pair's weight and
 * dL/dalpha terms in shared memory, then a pass over (Gaussian, pixel block)
 * pairs sums them;
 * tuning.bwd_impl = 0: pixels across threads walking back from their last
 * blended pair (T recovered by division by 1 - alpha), per-Gaussian gradients
 * reduced across each warp's pixels with shuffles.
 * image is the gs_raster_fwd output, dL_dimage the loss gradient. */
gs_status gs_raster_bwd(const gs_plan* plan, void* ws, const float* image,
                        const float* dL_dimage, void* stream);

/* Projection backward fused with Adam (Sec. 4.3): per Gaussian, sums its
 * intersection gradients over all views, back-propagates through colour
 * (SH), conic, EWA Jacobian and covariance to theta, and applies one Adam
 * step with scales and opacity moved to log / logit space inside the
 * optimiser; SH degree 0 and degrees 1-3 take separate learning rates.
 * Writes geom, sh, m and v in place.  If grads_out != NULL nothing is
 * updated; instead the gradient with respect to the STORED (activated)
 * parameters is written there as float4[15][sum of scene n] (chunk order of
 * geom then sh, scenes concatenated). */
gs_status gs_project_bwd_adam(const gs_plan* plan, void* ws, const gs_scene_buf* scenes,
                              const float* cams, const gs_adam* adam, float* grads_out,
                              void* stream);

/* Advance the workspace Adam step counter by one (for graph replay). */
gs_status gs_adam_advance(const gs_plan* plan, void* ws, void* stream);

/* Set the workspace Adam step counter (to carry it into a new workspace,
 * e.g. after densification changed the plan).  step >= 0. */
gs_status gs_workspace_set_step(const gs_plan* plan, void* ws, int32_t step, void* stream);

/* Synchronous: copy the workspace statistics to the host (waits on stream).
 * Not capturable. */
gs_status gs_read_stats(const gs_plan* plan, const void* ws, gs_stats* out, void* stream);

/* Device views of intermediate buffers (for tests and tools): 0 counts
 * u32[pairs] and 1 offsets u32[pairs+1] (its exclusive scan: each pair's
 * first emission slot), both in Gaussian-major pair order (scene by scene,
 * Gaussian by Gaussian, the scene's views in plan order), 2 sorted keys
 * u32[cap], 3 sorted pair index u32[cap] (view-major: the view's first pair
 * + Gaussian), 4 tile ranges u32[tiles][2], 5 n_last u32[pixels], 6 final
 * transmittance f32[pixels], 7 projected records float4[pairs][3]
 * (view-major), 8 gradient records float4[cap][3] (at emission slots),
 * 9 sorted emission slot u32[cap], 10 tile spans u32[pairs][4] (Gaussian-
 * major; written for pairs with a nonzero count: word 0 the depth code in
 * bits 0-22, the number of bands nb in bits 24-25 and the orientation in bit
 * 26 (1: bands are tile rows); with nb <= 2, word 1 the two bands' row or
 * column (low, high 16 bits) and words 2, 3 each band's first and last tile
 * along it (low, high 16 bits); nb = 3 marks more than two bands, words 1-3
 * then hold the bits of the binning conic a, b, c; bit 27 of word 0 marks a
 * ranked pair, one of at most four tiles in one or two bands), 11 ranks
 * u32[pairs][4] (Gaussian-major; for a ranked pair, its place in each of its
 * tiles' lists, in traversal order), 12 tile counters u32[2][tiles] (entries
 * of ranked pairs per tile; then, after gs_bin_sort, each tile's cursor for
 * the other pairs' entries).  Returns NULL for an unknown buffer. */
void* gs_workspace_buffer(const gs_plan* plan, void* ws, int32_t which);

const char* gs_status_str(gs_status s);

/* L1 loss and gradient without any device allocation (no plan, no
 * workspace).  The paper has no counterpart to this call: it exists for
 * callers that may not allocate device memory -- a host framework that owns
 * the GPU's memory through its own pool and forbids cudaMalloc in libraries,
 * or a frame loop that must never wait on the allocator.
 *
 * Computes the same values as gs_loss_l1 over n_values floats (3 x pixels):
 * dL_dimage[i] = sign(image[i] - target[i]) / n_values, and
 * *loss = sum |image - target| / n_values written to the DEVICE float `loss`.
 * All four pointers are device memory owned by the caller.
 *
 * Its scratch (block partial sums and a completion counter, about 128 KiB)
 * is a static array inside the library, held by every GPU that loads the
 * library until the process exits.  The first call on a device looks up that
 * array's device address (with the device current) and caches it; make that
 * first call before any stream capture.  The cached address is the one in
 * the device's primary context (the context the CUDA runtime uses): call
 * this entry point only with that context current, and not after the
 * process has reset the device (cudaDeviceReset), which invalidates it.  The array is shared by every call on
 * the device and keeps the last call's contents (the counter is cleared at
 * the start of each call), so calls whose executions overlap on the GPU race
 * and must be ordered by the caller.
 * Returns GS_ERR_INVALID_ARG for a NULL pointer or for n_values <= 0 or
 * n_values > GS_L1_NOALLOC_MAX_VALUES, GS_ERR_CUDA if the set-up or the
 * launch fails. */
#define GS_L1_NOALLOC_MAX_VALUES 67108864LL   /* 3 x 22,369,621 pixels */
gs_status gs_loss_l1_noalloc(const float* image, const float* target, float* dL_dimage, float* loss,
                             int64_t n_values, void* stream);

/* ---------------------------------------------------------------------
 * Default densification (Sec. 4.6: the 3DGS default strategy,
 * which the paper follows): every refinement interval, Gaussians whose mean
 * statistic (stats.x / max(stats.y, 1)) exceeds grow_grad2d are cloned when
 * small (max scale <= grow_scale3d * scene_scale) or split when large; then
 * Gaussians with opacity < prune_opa -- and, with prune_big, those whose max
 * scale exceeds prune_scale3d * scene_scale -- are removed.  The decisions
 * are binary32 comparisons of stored values (opacity and scales are stored
 * activated), so they are exact and reproducible.
 *
 * Output order (one Gaussian per row of every chunk-major array):
 *   [survivors that are not split, in input order]
 *   [clones of the cloned survivors, in input order]
 *   [first product of each surviving split, in input order]
 *   [second product of each surviving split, in input order]
 * A clone copies its Gaussian; a split product keeps quaternion, opacity and
 * SH, takes scale / split_factor and mean + R(q) (scale * eps), eps the
 * caller's standard normal draws.  New Gaussians start with zero Adam
 * moments; survivors keep theirs; all output statistics are zero.
 * --------------------------------------------------------------------- */
typedef struct {
    float grow_grad2d;        /* 2e-4 */
    float grow_scale3d;       /* 0.01 (x scene_scale) */
    float prune_opa;          /* 0.005 */
    float prune_scale3d;      /* 0.1 (x scene_scale), when prune_big != 0 */
    float scene_scale;        /* scene extent, world units */
    float split_factor;       /* 1.6 */
    int32_t grow;             /* 0: prune only */
    int32_t prune_big;        /* 1 once opacities have been reset */
} gs_densify_cfg;

/* Device scratch for n input Gaussians (caller-allocated, 256-byte aligned). */
size_t gs_densify_scratch_bytes(int64_t n);

/* Decides every Gaussian's fate and the output positions.  scene: one
 * scene's buffers with stats != NULL; storage_flags: GS_STORE_* of its
 * layout.  Asynchronous; read the counts with gs_densify_counts.
 * GS_ERR_INVALID_ARG for NULL pointers, n < 1, n >= 2^31 or a config with a
 * non-finite or non-positive scale, factor or threshold. */
gs_status gs_densify_count(const gs_scene_buf* scene, int32_t storage_flags, const gs_densify_cfg* cfg,
                           void* scratch, void* stream);

/* Synchronises `stream` and returns, in counts[4] (host), the number of
 * survivors kept as they are, clones, surviving splits (each giving two
 * products) and the output total. */
gs_status gs_densify_counts(const void* scratch, int64_t counts[4], void* stream);

/* Writes the densified scene into `out` (out->n = the total from
 * gs_densify_counts; buffers of that size in the same layout; out->stats
 * zeroed when not NULL).  eps: device float[in->n][6], standard normal draws
 * (two 3-vectors per input Gaussian; only the split ones are read).
 * in and out must not overlap.  If out->n differs from the total of the
 * preceding gs_densify_count on this scratch, nothing is written. */
gs_status gs_densify_apply(const gs_scene_buf* in, int32_t storage_flags, const gs_densify_cfg* cfg,
                           const float* eps, const void* scratch, gs_scene_buf* out, void* stream);

/* Opacity reset of the default strategy: o = min(o, value) for every
 * Gaussian, and the logit-opacity Adam moments (m and v) set to zero. */
gs_status gs_reset_opacity(const gs_scene_buf* scene, int32_t storage_flags, float value, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GS_STEP_H */
