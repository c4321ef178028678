// bin_sort.cu -- tiling and sorting (VkSplat Sec. 4.1, Sec. 4.4; Table 2
// "Tiling/Sorting": index offset, generate keys, sorting, tile ranges).
//
//   index offset : exclusive scan of the per-pair tile counts (reduce-then-
//                  scan, three launches, no inter-block waiting)
//   generate keys: second scan-line pass writing 32-bit keys
//                  (tile << shift | depth code >> drop) and the pair of each
//                  emitted intersection
//   sorting      : stable LSD radix sort, 8-bit digits, 2048 keys per block,
//                  warp-level match_any ranking, scatter through shared memory
//                  so that global writes are coalesced runs per digit; the
//                  payload starts as the implicit emission index; when there
//                  are several views a final pass orders the view segments;
//                  the last pass also gathers the sorted pair indices
//   tile ranges  : [start, end) per tile from key boundaries
// K never leaves the device: every kernel reads it from the workspace header
// and grids are sized by the capacity.
#include "gs_internal.cuh"

namespace gs {

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__global__ void k_fill_u32(uint32_t* __restrict__ p, int64_t n, uint32_t value)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = value;
}

void launch_fill_u32(uint32_t* p, int64_t n, uint32_t value, cudaStream_t st)
{
    if (n <= 0) return;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_fill_u32<<<(unsigned)blocks, 256, 0, st>>>(p, n, value);
}

// ---------------------------------------------------------------------------
// Exclusive scan of u32 (reduce, scan of block sums, down-sweep)
// ---------------------------------------------------------------------------

template <int T>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* warp_sums, uint32_t* total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t s = lane < T / 32 ? warp_sums[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < T / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    uint32_t before = w > 0 ? warp_sums[w - 1] : 0u;
    if (total) *total = warp_sums[T / 32 - 1];
    return before + x - v;
}

// Effective scan length: n, or (*nb) * mul when the length is known only on
// the device (the radix histograms: 256 digits x blocks holding keys).
__device__ __forceinline__ int64_t scan_len(int64_t n, const uint32_t* nb, int mul)
{
    return nb ? min(n, (int64_t)(*nb) * mul) : n;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ in, int64_t n_max,
                                                               const uint32_t* __restrict__ nb, int mul,
                                                               uint32_t* __restrict__ part)
{
    __shared__ uint32_t ws[32];
    const int64_t n = scan_len(n_max, nb, mul);
    const int64_t base = (int64_t)blockIdx.x * kScanBlock;
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        int64_t idx = base + i * kScanThreads + threadIdx.x;
        if (idx < n) s += in[idx];
    }
    uint32_t tot;
    block_excl_scan<kScanThreads>(s, ws, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// Single block: exclusive scan of the block sums in place; grand total at part[nparts].
__global__ void __launch_bounds__(1024) k_scan_part(uint32_t* __restrict__ part, int64_t nparts)
{
    __shared__ uint32_t ws[32];
    uint32_t carry = 0;
    for (int64_t b = 0; b < nparts; b += 1024) {
        int64_t i = b + threadIdx.x;
        uint32_t v = i < nparts ? part[i] : 0u;
        uint32_t tot;
        uint32_t ex = block_excl_scan<1024>(v, ws, &tot);
        if (i < nparts) part[i] = carry + ex;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) part[nparts] = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const uint32_t* in, int64_t n_max,
                                                             const uint32_t* __restrict__ nb, int mul,
                                                             const uint32_t* __restrict__ part, uint32_t* out)
{
    __shared__ uint32_t buf[kScanBlock];
    __shared__ uint32_t ws[32];
    const int64_t n = scan_len(n_max, nb, mul);
    const int64_t base = (int64_t)blockIdx.x * kScanBlock;
    if (base >= n) return;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        int64_t idx = base + i * kScanThreads + threadIdx.x;
        buf[i * kScanThreads + threadIdx.x] = idx < n ? in[idx] : 0u;
    }
    __syncthreads();
    uint32_t loc[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        loc[i] = s;
        s += buf[threadIdx.x * kScanItems + i];
    }
    uint32_t ex = block_excl_scan<kScanThreads>(s, ws, nullptr) + part[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; i++) buf[threadIdx.x * kScanItems + i] = ex + loc[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        int64_t idx = base + i * kScanThreads + threadIdx.x;
        if (idx < n) out[idx] = buf[i * kScanThreads + threadIdx.x];
    }
}

static void scan_u32_dyn(const uint32_t* in, uint32_t* out, int64_t n_max, const uint32_t* nb, int mul,
                         uint32_t* part, cudaStream_t st)
{
    const int64_t nparts = (n_max + kScanBlock - 1) / kScanBlock;
    k_scan_reduce<<<(unsigned)nparts, kScanThreads, 0, st>>>(in, n_max, nb, mul, part);
    k_scan_part<<<1, 1024, 0, st>>>(part, nparts);
    k_scan_down<<<(unsigned)nparts, kScanThreads, 0, st>>>(in, n_max, nb, mul, part, out);
}

void scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* part, cudaStream_t st)
{
    scan_u32_dyn(in, out, n, nullptr, 1, part, st);
}

// Total, capacity check and view segment starts after the count scan.
__global__ void k_count_finalize(Views V, const uint32_t* __restrict__ part, int64_t nparts,
                                 uint32_t* __restrict__ offset, WsHeader* __restrict__ hdr, uint32_t cap)
{
    const uint32_t total = part[nparts];
    if (threadIdx.x == 0) {
        hdr->k_required = total;
        hdr->k_eff = total < cap ? total : cap;
        hdr->hist_nblk = ((total < cap ? total : cap) + kRadixBlock - 1) / kRadixBlock;
        if (total > cap) atomicOr(&hdr->status, GS_STATUS_CAPACITY);
        offset[V.pairs] = total;
        hdr->seg[V.n] = total < cap ? total : cap;
    }
    for (int v = threadIdx.x; v < V.n; v += blockDim.x) {
        uint32_t s = offset[V.v[v].pair_base];
        hdr->seg[v] = s < cap ? s : cap;
    }
}

// ---------------------------------------------------------------------------
// Generate keys
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_emit(Views V, const uint32_t* __restrict__ count,
                                              const uint32_t* __restrict__ offset, const ProjRec* __restrict__ rec,
                                              const float4* __restrict__ binrec, uint32_t* __restrict__ keys,
                                              uint32_t* __restrict__ pid, uint32_t cap)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= V.pairs) return;
    const uint32_t cnt = count[p];
    if (cnt == 0) return;
    const ViewDesc& vd = V.v[view_of_pair(V, p)];
    const uint32_t off = offset[p];
    const float4 ra = rec[p].a;
    const float4 bb = binrec[p];
    BinGeom g;
    g.mx = ra.x; g.my = ra.y; g.a = bb.x; g.b = bb.y; g.c = bb.z;
    g.det = FS(FM(g.a, g.c), FM(g.b, g.b));
    g.r2 = cull_r2(rec[p].b.y);   // same bits as in the projection pass
    g.mant = __float_as_uint(bb.w);
    g.valid = 1;
    const uint32_t low = g.mant >> vd.drop;
    const int shift = vd.shift;
    scanline_tiles(g, V.tw, V.th, vd.TX, vd.TY, [&](uint32_t i, uint32_t tile) {
        uint32_t e = off + i;
        if (e < cap) {
            keys[e] = (tile << shift) | low;
            pid[e] = (uint32_t)p;
        }
    });
}

// ---------------------------------------------------------------------------
// Radix sort passes
// ---------------------------------------------------------------------------

enum { kDigitKey = 0, kDigitView = 1 };

__device__ __forceinline__ int view_of_slot(const uint32_t* seg, int nv, uint32_t e)
{
    int v = 0;
    while (v + 1 < nv && seg[v + 1] <= e) v++;
    return v;
}

// 16-byte asynchronous global -> shared copy (bypassing L1), and its group
// commit / wait (hardware waits: no spinning in this code)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int MODE>
__global__ void __launch_bounds__(kRadixThreads) k_radix_up(const uint32_t* __restrict__ keys,
                                                             const uint32_t* __restrict__ vals, bool iota,
                                                             const WsHeader* __restrict__ hdr, int shift,
                                                             uint32_t* __restrict__ hist, int nv)
{
    // digit counts of each 2048-key block: one private histogram per warp
    // (plain shared-memory atomics), summed per digit at the end.  Only the
    // blocks that hold keys take part (the grid strides over them, the next
    // block's keys loaded while this one is counted); the histogram is
    // [digit][block] over them, so its scan covers 256 x ceil(K / 2048)
    // entries.  Key arrays are padded to whole blocks.
    constexpr int W = kRadixThreads / 32;
    const uint32_t nb = hdr->hist_nblk;
    if (blockIdx.x >= nb) return;
    __shared__ uint32_t h[W][kRadixDigits];
    __shared__ uint32_t seg[kMaxViews + 1];
    const int w = threadIdx.x >> 5;
    if (MODE == kDigitView)
        for (int i = threadIdx.x; i <= nv; i += blockDim.x) seg[i] = hdr->seg[i];
    const uint32_t K = hdr->k_eff;
    const uint32_t* src = MODE == kDigitKey ? keys : vals;
    const bool load = MODE == kDigitKey || !iota;
    uint32_t d[kRadixItems];
    auto fetch = [&](uint32_t b) {
        const int64_t base = (int64_t)b * kRadixBlock;
#pragma unroll
        for (int i = 0; i < kRadixItems; i++) {
            const int64_t idx = base + i * kRadixThreads + threadIdx.x;
            d[i] = load ? src[idx] : (uint32_t)idx;
        }
    };
    fetch(blockIdx.x);
    for (uint32_t b = blockIdx.x; b < nb; b += gridDim.x) {
        uint32_t cur[kRadixItems];
#pragma unroll
        for (int i = 0; i < kRadixItems; i++) cur[i] = d[i];
        if (b + gridDim.x < nb) fetch(b + gridDim.x);
#pragma unroll
        for (int i = 0; i < W; i++) h[i][threadIdx.x] = 0;
        __syncthreads();
        const int64_t base = (int64_t)b * kRadixBlock;
#pragma unroll
        for (int i = 0; i < kRadixItems; i++) {
            if (base + i * kRadixThreads + threadIdx.x < K) {
                const uint32_t dg = MODE == kDigitKey ? (cur[i] >> shift) & 0xFFu
                                                      : (uint32_t)view_of_slot(seg, nv, cur[i]);
                atomicAdd(&h[w][dg], 1u);
            }
        }
        __syncthreads();
        uint32_t c = 0;
#pragma unroll
        for (int i = 0; i < W; i++) c += h[i][threadIdx.x];
        hist[(int64_t)threadIdx.x * nb + b] = c;
        __syncthreads();
    }
}

template <int MODE, bool IOTA, bool LAST>
__global__ void __launch_bounds__(kRadixThreads) k_radix_down(const uint32_t* __restrict__ keys_in,
                                                               const uint32_t* __restrict__ vals_in,
                                                               uint32_t* __restrict__ keys_out,
                                                               uint32_t* __restrict__ vals_out,
                                                               const uint32_t* __restrict__ hist,
                                                               int shift, const WsHeader* __restrict__ hdr, int nv,
                                                               const uint32_t* __restrict__ pid,
                                                               uint32_t* __restrict__ pid_sorted)
{
    // Blocks are double-buffered in shared memory: the next block's keys and
    // payload are copied asynchronously while this one is ranked, and this
    // block's buffer then holds its locally reordered keys for the coalesced
    // write-out.  Key arrays are padded to whole blocks.
    constexpr int W = kRadixThreads / 32;
    __shared__ uint32_t wh[W][kRadixDigits];
    __shared__ uint32_t bstart[kRadixDigits];
    __shared__ uint32_t gbase[kRadixDigits];
    __shared__ __align__(16) uint32_t sk[2][kRadixBlock];
    __shared__ __align__(16) uint32_t sv[2][kRadixBlock];
    __shared__ uint32_t seg[kMaxViews + 1];
    __shared__ uint32_t wsum[32];
    const uint32_t K = hdr->k_eff;
    const uint32_t nb = hdr->hist_nblk;
    if (blockIdx.x >= nb) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (MODE == kDigitView)
        for (int i = threadIdx.x; i <= nv; i += blockDim.x) seg[i] = hdr->seg[i];
    const uint32_t lt = lanemask_lt();
    auto issue = [&](uint32_t b, int buf) {
        const int64_t base = (int64_t)b * kRadixBlock;
        for (int c = threadIdx.x; c < kRadixBlock / 4; c += kRadixThreads) {
            cp_async16(&sk[buf][4 * c], keys_in + base + 4 * c);
            if (!IOTA) cp_async16(&sv[buf][4 * c], vals_in + base + 4 * c);
        }
        cp_async_commit();
    };
    issue(blockIdx.x, 0);
    int cur = 0;
    for (uint32_t b = blockIdx.x; b < nb; b += gridDim.x, cur ^= 1) {   // blocks holding keys
        const int64_t base = (int64_t)b * kRadixBlock;
        if (b + gridDim.x < nb) issue(b + gridDim.x, cur ^ 1);
        else cp_async_commit();                 // empty group: the wait below stays one behind
#pragma unroll
        for (int i = 0; i < W; i++) wh[i][threadIdx.x] = 0;
        cp_async_wait<1>();
        __syncthreads();

        uint32_t key[kRadixItems], val[kRadixItems], dig[kRadixItems], rank[kRadixItems];
#pragma unroll
        for (int r = 0; r < kRadixItems; r++) {
            const int li = w * (32 * kRadixItems) + r * 32 + lane;
            const int64_t idx = base + li;
            const bool valid = idx < K;
            key[r] = valid ? sk[cur][li] : 0u;
            val[r] = IOTA ? (uint32_t)idx : (valid ? sv[cur][li] : 0u);
            uint32_t d = 0xFFFFu;
            if (valid) {
                if (MODE == kDigitKey) d = (key[r] >> shift) & 0xFFu;
                else d = (uint32_t)view_of_slot(seg, nv, val[r]);
            }
            dig[r] = d;
        }
        // stable rank within the warp's contiguous 256-key range, round by round
#pragma unroll
        for (int r = 0; r < kRadixItems; r++) {
            const uint32_t d = dig[r];
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            const bool valid = d != 0xFFFFu;
            uint32_t c = valid ? wh[w][d] : 0u;
            rank[r] = c + __popc(peers & lt);
            __syncwarp();
            if (valid && lane == __ffs(peers) - 1) wh[w][d] = c + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // per digit: exclusive offsets across warps, then across digits
        {
            const int d = threadIdx.x;
            uint32_t run = 0;
#pragma unroll
            for (int i = 0; i < W; i++) {
                uint32_t c = wh[i][d];
                wh[i][d] = run;
                run += c;
            }
            uint32_t ex = block_excl_scan<kRadixThreads>(run, wsum, nullptr);
            bstart[d] = ex;
            gbase[d] = hist[(int64_t)d * nb + b];
        }
        __syncthreads();
        // every thread has its items in registers: reorder into this block's buffer
#pragma unroll
        for (int r = 0; r < kRadixItems; r++) {
            const uint32_t d = dig[r];
            if (d != 0xFFFFu) {
                const uint32_t lp = bstart[d] + wh[w][d] + rank[r];
                sk[cur][lp] = key[r];
                sv[cur][lp] = val[r];
            }
        }
        __syncthreads();
        const int nvalid = (int)min((int64_t)kRadixBlock, (int64_t)K - base);
        for (int i = threadIdx.x; i < nvalid; i += kRadixThreads) {
            const uint32_t k = sk[cur][i], v = sv[cur][i];
            const uint32_t d = MODE == kDigitKey ? ((k >> shift) & 0xFFu) : (uint32_t)view_of_slot(seg, nv, v);
            const uint32_t pos = gbase[d] + (uint32_t)i - bstart[d];
            keys_out[pos] = k;
            vals_out[pos] = v;
            if (LAST) pid_sorted[pos] = pid[v];
        }
        __syncthreads();
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Tile ranges
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_ranges(Views V, const uint32_t* __restrict__ keys,
                                                const WsHeader* __restrict__ hdr, uint2* __restrict__ ranges,
                                                uint32_t cap)
{
    __shared__ uint32_t seg[kMaxViews + 1];
    for (int i = threadIdx.x; i <= V.n; i += blockDim.x) seg[i] = hdr->seg[i];
    __syncthreads();
    const uint32_t K = hdr->k_eff;
    // four consecutive keys per thread (one 16-byte load; the capacity is a
    // multiple of 4) and their two neighbours
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * 4;
    for (int64_t k0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4; k0 < K; k0 += stride) {
        const uint4 q = *reinterpret_cast<const uint4*>(keys + k0);
        const uint32_t kk[6] = {k0 > 0 ? keys[k0 - 1] : 0u, q.x, q.y, q.z, q.w, k0 + 4 < K ? keys[k0 + 4] : 0u};
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int64_t k = k0 + i;
            if (k >= K) break;
            const int v = view_of_slot(seg, V.n, (uint32_t)k);
            const ViewDesc& vd = V.v[v];
            const uint32_t tile = kk[i + 1] >> vd.shift;
            const int64_t gt = vd.tile_base + tile;
            const bool first = (k == seg[v]) || ((kk[i] >> vd.shift) != tile);
            const bool last = (k + 1 == seg[v + 1]) || ((kk[i + 2] >> vd.shift) != tile);
            if (first) ranges[gt].x = (uint32_t)k;
            if (last) ranges[gt].y = (uint32_t)(k + 1);
        }
    }
}

// Launch order of the raster kernels: tiles by decreasing list length,
// bucketed by floor(log2(length + 1)).  Blocks are dispatched roughly in
// index order, so the longest tiles start first and the short ones fill the
// tail (longest-processing-time scheduling).  Within a bucket the order
// follows shared-memory atomics; it decides only when a tile runs, never its
// result.
__global__ void __launch_bounds__(1024) k_tile_order(int64_t tiles, const uint2* __restrict__ ranges,
                                                     uint32_t* __restrict__ order)
{
    __shared__ uint32_t cnt[32];
    if (threadIdx.x < 32) cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t t = threadIdx.x; t < tiles; t += blockDim.x) {
        const uint2 r = ranges[t];
        atomicAdd(&cnt[31 - __clz(r.y - r.x + 1u)], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int b = 31; b >= 0; b--) {
            const uint32_t c = cnt[b];
            cnt[b] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int64_t t = threadIdx.x; t < tiles; t += blockDim.x) {
        const uint2 r = ranges[t];
        order[atomicAdd(&cnt[31 - __clz(r.y - r.x + 1u)], 1u)] = (uint32_t)t;
    }
}

// ---------------------------------------------------------------------------

void launch_bin_sort(const Plan& P, const WsPtrs& w, cudaStream_t st)
{
    const Views& V = P.views;
    const uint32_t cap = (uint32_t)P.cap;
    // index offset
    scan_u32(w.count, w.offset, V.pairs, w.scan_part, st);
    k_count_finalize<<<1, 64, 0, st>>>(V, w.scan_part, P.count_scan_parts, w.offset, w.hdr, cap);
    // generate keys
    {
        const int64_t blocks = (V.pairs + 255) / 256;
        k_emit<<<(unsigned)blocks, 256, 0, st>>>(V, w.count, w.offset, w.rec, w.binrec, w.keysA, w.pid, cap);
    }
    // sorting: the radix kernels stride over the blocks that hold keys, with
    // grids of the resident CTAs (8 per SM for the counts, 4 for the
    // double-buffered reorder)
    const int64_t nblk = std::min<int64_t>(P.radix_blocks, (int64_t)P.sm_count * 8);
    const int64_t nblk_down = std::min<int64_t>(P.radix_blocks, (int64_t)P.sm_count * 4);
    const int npass = P.key_passes + P.view_pass;
    uint32_t *kin = w.keysA, *vin = w.valsA, *kout = w.keysB, *vout = w.valsB;
    for (int pass = 0; pass < npass; pass++) {
        const bool view = pass >= P.key_passes;
        const bool first = pass == 0, last = pass == npass - 1;
        const int shift = 8 * pass;
        if (view)
            k_radix_up<kDigitView><<<(unsigned)nblk, kRadixThreads, 0, st>>>(kin, vin, first, w.hdr, 0, w.hist, V.n);
        else
            k_radix_up<kDigitKey><<<(unsigned)nblk, kRadixThreads, 0, st>>>(kin, vin, first, w.hdr, shift, w.hist,
                                                                              V.n);
        scan_u32_dyn(w.hist, w.hist, (int64_t)kRadixDigits * P.radix_blocks, &w.hdr->hist_nblk, kRadixDigits,
                     w.scan_part, st);
#define GS_DOWN(MODE, IOTA, LAST)                                                                          \
    k_radix_down<MODE, IOTA, LAST><<<(unsigned)nblk_down, kRadixThreads, 0, st>>>(kin, vin, kout, vout, w.hist, shift, \
                                                                              w.hdr, V.n, w.pid, w.pid_sorted)
        if (view) {
            if (first) GS_DOWN(kDigitView, true, true);
            else GS_DOWN(kDigitView, false, true);
        } else if (first) {
            if (last) GS_DOWN(kDigitKey, true, true);
            else GS_DOWN(kDigitKey, true, false);
        } else {
            if (last) GS_DOWN(kDigitKey, false, true);
            else GS_DOWN(kDigitKey, false, false);
        }
#undef GS_DOWN
        uint32_t* t;
        t = kin; kin = kout; kout = t;
        t = vin; vin = vout; vout = t;
    }
    // tile ranges
    launch_fill_u32(reinterpret_cast<uint32_t*>(w.ranges), 2 * V.tiles, 0u, st);
    {
        int64_t blocks = ((int64_t)cap + 255) / 256;
        if (blocks > 152 * 32) blocks = 152 * 32;
        if (blocks < 1) blocks = 1;
        k_ranges<<<(unsigned)blocks, 256, 0, st>>>(V, w.keys_sorted, w.hdr, w.ranges, cap);
    }
    k_tile_order<<<1, 1024, 0, st>>>(V.tiles, w.ranges, w.tile_order);
}

}  // namespace gs
