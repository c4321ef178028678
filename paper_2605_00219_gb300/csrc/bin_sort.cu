// bin_sort.cu -- tiling and sorting (VkSplat Sec. 4.1, Sec. 4.4; Table 2
// "Tiling/Sorting": index offset, generate keys, sorting, tile ranges).
//
// The sorted lists are the 32-bit keys (tile << shift | depth code >> drop)
// of Sec. 4.4 in stable order, i.e. ordered by (view, tile, depth code,
// emission slot): the tile is the key's leading part, so the sort is done
// as a bucketing by tile followed by a sort of each tile's short list.
//
//   index offset : exclusive scan of the per-pair tile counts, in
//                  Gaussian-major pair order (reduce-then-scan, three
//                  launches, no inter-block waiting): a Gaussian's
//                  intersections in all views are consecutive emission slots
//   tile ranges  : the projection's traversal already counted the entries of
//                  every tile; their exclusive scan gives each tile's
//                  [start, end) in the sorted arrays and its scatter cursor
//   generate keys: second scan-line pass; each intersection takes the next
//                  slot of its tile (an atomic cursor) and stores its depth
//                  code and emission slot there, and its pair at the
//                  emission slot
//   sorting      : one thread block per tile sorts the tile's entries by
//                  (depth code, emission slot) -- unique, so the arrival
//                  order of the atomics does not matter -- and writes the
//                  keys, emission slots and pairs: a block merge sort in
//                  shared memory up to kTileSortMax entries; longer lists
//                  are sorted in chunks of that size and merged in global
//                  memory by rank (each entry's position in the other run by
//                  binary search)
// K never leaves the device: every kernel reads it from the workspace header
// and grids are sized by the plan.  When K exceeds the capacity nothing is
// emitted and every tile list is empty (GS_STATUS_CAPACITY reports it).
#include "gs_internal.cuh"

namespace gs {

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

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ in,
                                                               const uint32_t* __restrict__ in2, int64_t n,
                                                               uint32_t* __restrict__ part)
{
    __shared__ uint32_t ws[32];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock;
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        int64_t idx = base + i * kScanThreads + threadIdx.x;
        if (idx < n) s += in[idx] + (in2 ? in2[idx] : 0u);
    }
    uint32_t tot;
    block_excl_scan<kScanThreads>(s, ws, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// Single block: exclusive scan of the block sums in place; grand total at
// part[nparts].  With total_at (the scan of the pair counts; hdr then not
// null): the total is K, also written to total_at (the offsets' last entry),
// and the capacity check sets k_eff = K when it fits, else 0 (nothing is
// emitted) with GS_STATUS_CAPACITY.
__global__ void __launch_bounds__(1024) k_scan_part(uint32_t* __restrict__ part, int64_t nparts,
                                                    WsHeader* __restrict__ hdr, uint32_t* __restrict__ total_at,
                                                    uint32_t cap)
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
    if (threadIdx.x == 0) {
        part[nparts] = carry;
        if (total_at) {
            hdr->k_required = carry;
            hdr->k_eff = carry <= cap ? carry : 0u;
            if (carry > cap) atomicOr(&hdr->status, GS_STATUS_CAPACITY);
            *total_at = carry;
        }
    }
}

// Down-sweep: out[i] = exclusive prefix of in[i] (+ in2[i]).  With ranges
// (the scan of the tile counters, in = entries of ranked pairs, in2 = the
// others' entries; hdr then not null, its K already set): also each tile's
// range [start, start + both counts) --
// [0, 0) when empty, and every range empty when K exceeds the capacity --
// and the cursor for the other pairs' entries, start + the ranked entries,
// written over in2 (cur2, the same array).
__global__ void __launch_bounds__(kScanThreads) k_scan_down(const uint32_t* in, const uint32_t* in2, int64_t n,
                                                             const uint32_t* __restrict__ part, uint32_t* out,
                                                             uint2* __restrict__ ranges, uint32_t* cur2,
                                                             const WsHeader* __restrict__ hdr)
{
    __shared__ uint32_t buf[kScanBlock];
    __shared__ uint32_t ws[32];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock;
    if (base >= n) return;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        int64_t idx = base + i * kScanThreads + threadIdx.x;
        buf[i * kScanThreads + threadIdx.x] = idx < n ? in[idx] + (in2 ? in2[idx] : 0u) : 0u;
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
    // (the list lengths are read back before the prefixes replace them)
    uint32_t len[kScanItems];
    if (ranges) {
#pragma unroll
        for (int i = 0; i < kScanItems; i++) len[i] = buf[threadIdx.x * kScanItems + i];
    }
#pragma unroll
    for (int i = 0; i < kScanItems; i++) buf[threadIdx.x * kScanItems + i] = ex + loc[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        int64_t idx = base + i * kScanThreads + threadIdx.x;
        if (idx < n) out[idx] = buf[i * kScanThreads + threadIdx.x];
    }
    if (ranges) {
        const bool fits = hdr->k_eff == hdr->k_required;
#pragma unroll
        for (int i = 0; i < kScanItems; i++) {
            const int64_t idx = base + threadIdx.x * kScanItems + i;
            if (idx < n) {
                const uint32_t s0 = ex + loc[i], c = len[i];
                ranges[idx] = fits && c ? make_uint2(s0, s0 + c) : make_uint2(0u, 0u);
                cur2[idx] = s0 + in[idx];
            }
        }
    }
}

static void scan_launch(const uint32_t* in, const uint32_t* in2, uint32_t* out, int64_t n, uint32_t* part,
                        WsHeader* hdr, uint32_t* total_at, uint32_t cap, uint2* ranges, uint32_t* cur2,
                        cudaStream_t st)
{
    const int64_t nparts = (n + kScanBlock - 1) / kScanBlock;
    k_scan_reduce<<<(unsigned)nparts, kScanThreads, 0, st>>>(in, in2, n, part);
    k_scan_part<<<1, 1024, 0, st>>>(part, nparts, hdr, total_at, cap);
    k_scan_down<<<(unsigned)nparts, kScanThreads, 0, st>>>(in, in2, n, part, out, ranges, cur2, hdr);
}

// Offsets of the pair counts, K and the capacity check.
static void scan_pair_counts(const Plan& P, const WsPtrs& w, cudaStream_t st)
{
    scan_launch(w.count, nullptr, w.offset, P.views.pairs, w.scan_part, w.hdr, w.offset + P.views.pairs,
                (uint32_t)P.cap, nullptr, nullptr, st);
}

// Tile starts, ranges and the other pairs' cursors from the two tile
// counters (after scan_pair_counts: the ranges read K and k_eff).
static void scan_tile_counts(const Plan& P, const WsPtrs& w, cudaStream_t st)
{
    const int64_t tiles = P.views.tiles;
    scan_launch(w.tile_cnt, w.tile_cnt + tiles, w.tile_cur, tiles, w.scan_part, w.hdr, nullptr, 0u, w.ranges,
                w.tile_cnt + tiles, st);
}

void scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* part, cudaStream_t st)
{
    scan_launch(in, nullptr, out, n, part, nullptr, nullptr, 0u, nullptr, nullptr, st);
}

// ---------------------------------------------------------------------------
// Generate keys into tile buckets
// ---------------------------------------------------------------------------

// One thread per Gaussian-major pair q: its intersections take emission
// slots offset[q] + i in traversal order; each is placed in its tile's list
// (depth code and emission slot), and the view-major pair index is recorded
// at its emission slot.  The tiles come from the pair's tile span.  A ranked
// pair's entries go to tile start + the rank the projection took; the other
// pairs' entries take the next free place after the ranked ones (an atomic
// cursor per tile), and the rare pair of more than two bands repeats the
// traversal from its binning geometry.
__global__ void __launch_bounds__(256, 6) k_emit(Views V, const uint32_t* __restrict__ count,
                                                 const uint32_t* __restrict__ offset, const ProjRec* __restrict__ rec,
                                                 const uint4* __restrict__ span, const uint4* __restrict__ rank,
                                                 const uint32_t* __restrict__ tile_start, uint32_t* tile_over,
                                                 uint2* __restrict__ bucket, uint32_t* __restrict__ pid,
                                                 WsHeader* __restrict__ hdr)
{
    const int64_t qi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (qi >= V.pairs) return;
    // the pair's loads are issued together, before any of them is tested
    // (one memory round trip instead of three); span and ranks are stale
    // for a pair without tiles and a pair that is not ranked, and unused
    const uint32_t kreq = hdr->k_required, keff = hdr->k_eff;
    const uint32_t cnt = count[qi];
    const uint32_t off = offset[qi];
    const uint4 sp = span[qi];
    const uint4 rk4 = rank[qi];
    if (keff != kreq) return;     // over capacity: nothing is emitted
    if (cnt == 0) return;
    int s = 0;
    while (s + 1 < V.n_scenes && V.qbase[s + 1] <= qi) s++;
    const int nv = V.nv[s];
    const int64_t local = qi - V.qbase[s];
    const int64_t g = local / nv;
    const int v = V.view_of[s][(int)(local - g * nv)];
    const ViewDesc& vd = V.v[v];
    const uint32_t p = (uint32_t)(vd.pair_base + g);
    const uint32_t low = (sp.x & 0x7FFFFFu) >> vd.drop;
    const uint32_t nb = (sp.x >> 24) & 3u;
    uint32_t* cur = tile_over + vd.tile_base;
    if (nb == kSpanMany) {
        const float4 ra = rec[p].a;
        BinGeom gm;
        gm.mx = ra.x; gm.my = ra.y;
        gm.a = __uint_as_float(sp.y); gm.b = __uint_as_float(sp.z); gm.c = __uint_as_float(sp.w);
        gm.det = FS(FM(gm.a, gm.c), FM(gm.b, gm.b));
        gm.r2 = cull_r2(rec[p].b.y);   // same bits as in the projection pass
        gm.mant = sp.x & 0x7FFFFFu;
        gm.valid = 1;
        scanline_tiles(gm, V.tw, V.th, vd.TX, vd.TY, [&](uint32_t i, uint32_t tile) {
            const uint32_t e = off + i;
            const uint32_t slot = atomicAdd(cur + tile, 1u);
            if (GS_DCHECK(slot < hdr->k_eff && e < hdr->k_eff, &hdr->status)) {
                bucket[slot] = make_uint2(low, e);
                pid[e] = p;
            }
        });
        return;
    }
    const bool rows = (sp.x >> 26) & 1u;
    const uint32_t TX = (uint32_t)vd.TX;
    const uint32_t c0 = sp.y & 0xFFFFu, c1 = sp.y >> 16;
    if ((sp.x >> 27) & 1u) {
        // ranked: at most kRankMax tiles, no atomics
        const uint32_t rk[kRankMax] = {rk4.x, rk4.y, rk4.z, rk4.w};
        const uint32_t* __restrict__ st0 = tile_start + vd.tile_base;
#pragma unroll
        for (uint32_t u = 0; u < kRankMax; u++) {
            const uint32_t e = off + u;
            if (u < cnt) {
                const uint32_t slot = st0[span_tile(u, rows, TX, c0, c1, sp.z, sp.w)] + rk[u];
                if (GS_DCHECK(slot < hdr->k_eff && e < hdr->k_eff, &hdr->status)) {
                    bucket[slot] = make_uint2(low, e);
                    pid[e] = p;
                }
            }
        }
        return;
    }
    // one or two bands: the cursors taken four at a time so that the
    // atomics' round trips overlap
    for (uint32_t i0 = 0; i0 < cnt; i0 += 4) {
        uint32_t slot[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const uint32_t i = i0 + u;
            if (i < cnt) slot[u] = atomicAdd(cur + span_tile(i, rows, TX, c0, c1, sp.z, sp.w), 1u);
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const uint32_t i = i0 + u, e = off + i;
            if (i < cnt && GS_DCHECK(slot[u] < hdr->k_eff && e < hdr->k_eff, &hdr->status)) {
                bucket[slot[u]] = make_uint2(low, e);
                pid[e] = p;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Per-tile sort
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long sort_key(uint32_t low, uint32_t e)
{
    return ((unsigned long long)low << 32) | e;
}

// Ascending sort of N (a multiple of 8, 8 <= N <= 8 * blockDim.x) 64-bit
// keys in shared memory, block merge sort: thread t < N / 8 owns the 8 keys
// [8t, 8t + 8); it sorts them with a 19-comparator network in registers,
// then, at each merge level of run width w, finds where its 8 outputs start
// in the merge of its two runs (merge-path binary search on the output
// diagonal) and merges them sequentially.  The last run of a level may be
// short or alone (then it is already merged), so no padding to a power of
// two is sorted.  While two runs fit in one warp's 256 keys (w <= 128) only
// that warp reads and writes them, so the level synchronises the warp; a
// level that reads wider runs synchronises the group, also before its
// reads.  The caller synchronises the group before.
__device__ __forceinline__ void cmpx(unsigned long long& a, unsigned long long& b)
{
    const unsigned long long lo = a < b ? a : b, hi = a < b ? b : a;
    a = lo;
    b = hi;
}

// The threads that sort one list: the whole block, half of it (a named
// barrier of its own) or one warp.  t is the thread's index in the group.
struct SortGroup {
    int t, n, bar;
    __device__ __forceinline__ void sync() const
    {
        if (n == 32) __syncwarp();
        else if (bar == 0) __syncthreads();
        else asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(n) : "memory");
    }
};

__device__ __forceinline__ SortGroup whole_block() { return SortGroup{(int)threadIdx.x, (int)blockDim.x, 0}; }

__device__ void block_merge_sort_smem(unsigned long long* s, int N, const SortGroup& g)
{
    constexpr int IT = 8;
    const int nt = N / IT, t = g.t;
    unsigned long long r[IT];
    if (t < nt) {
#pragma unroll
        for (int k = 0; k < IT; k++) r[k] = s[IT * t + k];
        cmpx(r[0], r[1]); cmpx(r[2], r[3]); cmpx(r[4], r[5]); cmpx(r[6], r[7]);
        cmpx(r[0], r[2]); cmpx(r[1], r[3]); cmpx(r[4], r[6]); cmpx(r[5], r[7]);
        cmpx(r[1], r[2]); cmpx(r[5], r[6]);
        cmpx(r[0], r[4]); cmpx(r[1], r[5]); cmpx(r[2], r[6]); cmpx(r[3], r[7]);
        cmpx(r[2], r[4]); cmpx(r[3], r[5]);
        cmpx(r[1], r[2]); cmpx(r[3], r[4]); cmpx(r[5], r[6]);
#pragma unroll
        for (int k = 0; k < IT; k++) s[IT * t + k] = r[k];
    }
    __syncwarp();
    for (int w = IT; w < N; w <<= 1) {
        const bool in_warp = 2 * w <= 32 * IT;
        const int base = (IT * t) & ~(2 * w - 1), diag = IT * t - base;
        const int la = min(w, N - base), lb = max(0, min(w, N - base - w));
        const bool merge = t < nt && lb > 0;   // a lone last run stays in place
        if (merge) {
            const unsigned long long* A = s + base;
            const unsigned long long* B = s + base + w;
            int lo = max(0, diag - lb), hi = min(diag, la);
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (A[mid] <= B[diag - 1 - mid]) lo = mid + 1;
                else hi = mid;
            }
            int a = lo, b = diag - lo;
            unsigned long long ha = a < la ? A[a] : 0ull, hb = b < lb ? B[b] : 0ull;
#pragma unroll
            for (int k = 0; k < IT; k++) {
                const bool take_a = b >= lb || (a < la && ha <= hb);
                r[k] = take_a ? ha : hb;
                if (take_a) {
                    a++;
                    ha = a < la ? A[a] : 0ull;
                } else {
                    b++;
                    hb = b < lb ? B[b] : 0ull;
                }
            }
        }
        if (in_warp) __syncwarp();
        else g.sync();
        if (merge) {
#pragma unroll
            for (int k = 0; k < IT; k++) s[IT * t + k] = r[k];
        }
        // the next level (width 2w) reads other warps' keys unless its runs
        // still fit in one warp
        if (4 * w <= 32 * IT) __syncwarp();
        else g.sync();
    }
    g.sync();
}

// (depth code, emission slot) lists in two layouts: one uint2 per entry, or
// two u32 arrays.
struct PackedList {
    uint2* kv;
    __device__ unsigned long long get(uint32_t i) const { const uint2 x = kv[i]; return sort_key(x.x, x.y); }
    __device__ void put(uint32_t i, unsigned long long x) const { kv[i] = make_uint2((uint32_t)(x >> 32), (uint32_t)x); }
};
struct SplitList {
    uint32_t* k;
    uint32_t* v;
    __device__ unsigned long long get(uint32_t i) const { return sort_key(k[i], v[i]); }
    __device__ void put(uint32_t i, unsigned long long x) const { k[i] = (uint32_t)(x >> 32); v[i] = (uint32_t)x; }
};

// Entries of a sorted run [b, b + len) below key x (binary search; keys
// unique).
template <class L>
__device__ __forceinline__ uint32_t rank_in_run(const L& l, uint32_t b, uint32_t len, unsigned long long x)
{
    uint32_t lo = 0, hi = len;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (l.get(b + mid) < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// One merge level of run width `run` over a list of n entries at s0: each
// entry goes to its index in its own run plus its rank in the other run.
template <class Src, class Dst>
__device__ void merge_level(const Src& src, const Dst& dst, uint32_t s0, uint32_t n, uint32_t run)
{
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        const uint32_t ri = i / run, b = (ri & ~1u) * run;
        const unsigned long long x = src.get(s0 + i);
        uint32_t pos;
        if ((ri & 1u) == 0) {   // left run: rank among the right run
            const uint32_t pb = b + run, plen = pb < n ? min(run, n - pb) : 0u;
            pos = i + (plen ? rank_in_run(src, s0 + pb, plen, x) : 0u);
        } else {                // right run: rank among the left run
            pos = b + (i - ri * run) + rank_in_run(src, s0 + b, run, x);
        }
        dst.put(s0 + pos, x);
    }
    __syncthreads();
}

// One thread block per tile (launched longest lists first).  Input: the
// tile's bucket [s0, s1) of (depth code, emission slot) in atomic arrival
// order.  Output at the same positions: keys_sorted = tile << shift | depth
// code, vals_sorted = emission slot, pid_sorted = the slot's pair.
//
// One tile's list of n <= 8 g.n entries, sorted in shared memory (sk) by the
// group g.
__device__ __forceinline__ void tile_sort_group(const Views& V, int64_t gt, uint32_t s0, uint32_t n, unsigned long long* sk,
                                const SortGroup& g, uint2* bucket, const uint32_t* __restrict__ pid,
                                uint32_t* keys_sorted, uint32_t* vals_sorted, uint32_t* __restrict__ pid_sorted,
                                uint32_t* status, uint32_t cap)
{
    (void)status;
    (void)cap;
    const ViewDesc& vd = V.v[view_of_tile(V, gt)];
    const uint32_t hi_bits = (uint32_t)(gt - vd.tile_base) << vd.shift;
    const int N = (int)((n + 7u) & ~7u);    // the last thread's keys padded
    for (int i = g.t; i < N; i += g.n) {
        unsigned long long x = ~0ull;
        if (i < (int)n) {
            const uint2 b = bucket[s0 + i];
            x = sort_key(b.x, b.y);
        }
        sk[i] = x;
    }
    g.sync();
    block_merge_sort_smem(sk, N, g);
    for (int i = g.t; i < (int)n; i += g.n) {
        const unsigned long long x = sk[i];
        const uint32_t e = (uint32_t)x;
        keys_sorted[s0 + i] = hi_bits | (uint32_t)(x >> 32);
        vals_sorted[s0 + i] = e;
        pid_sorted[s0 + i] = GS_DCHECK(e < cap, status) ? pid[e] : 0u;
    }
}

// A list longer than kTileSortMax, sorted by the whole block: chunks of
// kTileSortMax sorted in shared memory, then merge levels alternating
// between the bucket and the (keys, vals) arrays, starting where an even
// number of moves ends in the bucket.
__device__ void tile_sort_chunked(const Views& V, int64_t gt, uint32_t s0, uint32_t n, unsigned long long* sk,
                                  uint2* bucket, const uint32_t* __restrict__ pid, uint32_t* keys_sorted,
                                  uint32_t* vals_sorted, uint32_t* __restrict__ pid_sorted, uint32_t* status,
                                  uint32_t cap)
{
    (void)status;
    (void)cap;
    const ViewDesc& vd = V.v[view_of_tile(V, gt)];
    const uint32_t hi_bits = (uint32_t)(gt - vd.tile_base) << vd.shift;
    const SortGroup g = whole_block();
    const PackedList pk{bucket};
    const SplitList sp{keys_sorted, vals_sorted};
    const uint32_t M = kTileSortMax;
    int levels = 0;
    for (uint32_t run = M; run < n; run <<= 1) levels++;
    const bool chunks_in_bucket = (levels & 1) == 0;
    for (uint32_t c0 = 0; c0 < n; c0 += M) {
        const uint32_t len = min(M, n - c0);
        for (uint32_t i = threadIdx.x; i < M; i += blockDim.x) sk[i] = i < len ? pk.get(s0 + c0 + i) : ~0ull;
        __syncthreads();
        block_merge_sort_smem(sk, (int)M, g);
        for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) {
            if (chunks_in_bucket) pk.put(s0 + c0 + i, sk[i]);
            else sp.put(s0 + c0 + i, sk[i]);
        }
        __syncthreads();
    }
    bool in_bucket = chunks_in_bucket;
    for (uint32_t run = M; run < n; run <<= 1) {
        if (in_bucket) merge_level(pk, sp, s0, n, run);
        else merge_level(sp, pk, s0, n, run);
        in_bucket = !in_bucket;
    }
    // the sorted list is in the bucket now
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        const unsigned long long x = pk.get(s0 + i);
        const uint32_t e = (uint32_t)x;
        keys_sorted[s0 + i] = hi_bits | (uint32_t)(x >> 32);
        vals_sorted[s0 + i] = e;
        pid_sorted[s0 + i] = GS_DCHECK(e < cap, status) ? pid[e] : 0u;
    }
}

// The tile order lists the tiles by size class (k_tile_order): long lists
// (>= 2047 entries), medium (1023-2046), short (255-1022), tiny (<= 254).
// Long and medium lists: 512-thread blocks, one long list per block (up to
// kTileSortMax entries in shared memory, longer ones chunked), or two medium
// lists per block, one per 256-thread half with a named barrier of its own.
__global__ void __launch_bounds__(kTileSortThreads) k_tile_sort_long(Views V, const uint32_t* __restrict__ order,
                                                                     const uint2* __restrict__ ranges,
                                                                     uint2* bucket, const uint32_t* __restrict__ pid,
                                                                     uint32_t* keys_sorted, uint32_t* vals_sorted,
                                                                     uint32_t* __restrict__ pid_sorted,
                                                                     const WsHeader* __restrict__ hdr,
                                                                     uint32_t* status, uint32_t cap)
{
    extern __shared__ unsigned long long sk[];
    const uint32_t n_long = hdr->sort_class[0], n_med = hdr->sort_class[1];
    const uint32_t b = blockIdx.x;
    if (b < n_long) {
        const int64_t gt = order[b];
        const uint2 r = range_at(ranges, gt, cap, status);
        const uint32_t n = r.y - r.x;
        if (n <= (uint32_t)kTileSortMax)
            tile_sort_group(V, gt, r.x, n, sk, SortGroup{(int)threadIdx.x, kTileSortThreads, 0}, bucket, pid,
                            keys_sorted, vals_sorted, pid_sorted, status, cap);
        else
            tile_sort_chunked(V, gt, r.x, n, sk, bucket, pid, keys_sorted, vals_sorted, pid_sorted, status, cap);
        return;
    }
    const uint32_t half = threadIdx.x >= kTileSortThreads / 2 ? 1u : 0u;
    const uint32_t m = 2u * (b - n_long) + half;     // medium list of this half
    if (b >= n_long + (n_med + 1u) / 2u || m >= n_med) return;
    const int64_t gt = order[n_long + m];
    const uint2 r = range_at(ranges, gt, cap, status);
    const uint32_t n = r.y - r.x;
    if (n == 0 || n > 4u * kTileSortThreads) return;
    const SortGroup g{(int)(threadIdx.x - half * (kTileSortThreads / 2)), kTileSortThreads / 2, 1 + (int)half};
    tile_sort_group(V, gt, r.x, n, sk + half * (kTileSortMax / 2), g, bucket, pid, keys_sorted, vals_sorted,
                    pid_sorted, status, cap);
}

// Short and tiny lists: 128-thread blocks, one short list per block, or four
// tiny lists per block, one per warp.
__global__ void __launch_bounds__(kTileSortSmall) k_tile_sort_short(Views V, const uint32_t* __restrict__ order,
                                                                    const uint2* __restrict__ ranges, uint2* bucket,
                                                                    const uint32_t* __restrict__ pid,
                                                                    uint32_t* keys_sorted, uint32_t* vals_sorted,
                                                                    uint32_t* __restrict__ pid_sorted,
                                                                    const WsHeader* __restrict__ hdr,
                                                                    uint32_t* status, uint32_t cap)
{
    extern __shared__ unsigned long long sk[];
    const uint32_t base = hdr->sort_class[0] + hdr->sort_class[1];
    const uint32_t n_short = hdr->sort_class[2], n_tiny = hdr->sort_class[3];
    const uint32_t b = blockIdx.x;
    if (b < n_short) {
        const int64_t gt = order[base + b];
        const uint2 r = range_at(ranges, gt, cap, status);
        const uint32_t n = r.y - r.x;
        if (n == 0 || n > 8u * kTileSortSmall) return;
        tile_sort_group(V, gt, r.x, n, sk, SortGroup{(int)threadIdx.x, kTileSortSmall, 0}, bucket, pid, keys_sorted,
                        vals_sorted, pid_sorted, status, cap);
        return;
    }
    const uint32_t w = threadIdx.x >> 5;
    const uint32_t m = 4u * (b - n_short) + w;       // tiny list of this warp
    if (b >= n_short + (n_tiny + 3u) / 4u || m >= n_tiny) return;
    const int64_t gt = order[base + n_short + m];
    const uint2 r = range_at(ranges, gt, cap, status);
    const uint32_t n = r.y - r.x;
    if (n == 0 || n > 256u) return;
    const SortGroup g{(int)(threadIdx.x & 31u), 32, 0};
    tile_sort_group(V, gt, r.x, n, sk + w * 256, g, bucket, pid, keys_sorted, vals_sorted, pid_sorted, status, cap);
}

// Launch order of the raster kernels: tiles by decreasing list length,
// bucketed by floor(log2(length + 1)).  Blocks are dispatched roughly in
// index order, so the longest tiles start first and the short ones fill the
// tail (longest-processing-time scheduling).  Within a bucket the order
// follows shared-memory atomics; it decides only when a tile runs, never its
// result.
__global__ void __launch_bounds__(1024) k_tile_order(int64_t tiles, const uint2* __restrict__ ranges,
                                                     uint32_t* __restrict__ order, WsHeader* __restrict__ hdr)
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
        // the sort's size classes are runs of buckets: long >= 2047 entries
        // (buckets 11+), medium 1023-2046 (10), short 255-1022 (8, 9), tiny
        // <= 254 (0-7)
        uint32_t cls[4] = {0u, 0u, 0u, 0u};
        for (int b = 0; b < 32; b++) cls[b >= 11 ? 0 : b == 10 ? 1 : b >= 8 ? 2 : 3] += cnt[b];
        for (int c = 0; c < 4; c++) hdr->sort_class[c] = cls[c];
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
    // index offset (Gaussian-major pair order), K and the capacity check
    scan_pair_counts(P, w, st);
    // tile starts, ranges and the other pairs' cursors from the tile counters
    scan_tile_counts(P, w, st);
    k_tile_order<<<1, 1024, 0, st>>>(V.tiles, w.ranges, w.tile_order, w.hdr);
    // generate keys into the tile buckets
    {
        const int64_t blocks = (V.pairs + 255) / 256;
        k_emit<<<(unsigned)blocks, 256, 0, st>>>(V, w.count, w.offset, w.rec, w.span, w.rank, w.tile_cur,
                                                 w.tile_cnt + V.tiles, w.bucket, w.pid, w.hdr);
    }
    // sort each tile's list
    {
        const size_t smem_l = sizeof(unsigned long long) * kTileSortMax;            // 32 KB: no opt-in needed
        const size_t smem_s = sizeof(unsigned long long) * 8 * kTileSortSmall;      // 8 KB
        k_tile_sort_long<<<(unsigned)V.tiles, kTileSortThreads, smem_l, st>>>(V, w.tile_order, w.ranges, w.bucket,
                                                                             w.pid, w.keys_sorted, w.vals_sorted,
                                                                             w.pid_sorted, w.hdr, &w.hdr->status,
                                                                             cap);
        k_tile_sort_short<<<(unsigned)V.tiles, kTileSortSmall, smem_s, st>>>(V, w.tile_order, w.ranges, w.bucket,
                                                                             w.pid, w.keys_sorted, w.vals_sorted,
                                                                             w.pid_sorted, w.hdr, &w.hdr->status,
                                                                             cap);
    }
}

}  // namespace gs
