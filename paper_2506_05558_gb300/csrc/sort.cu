// Per-tile duplication and depth ordering (K2-K4).
//
// Design: instead of one radix sort of 64-bit (tile, depth) keys over all P
// pairs, the V visible (view, Gaussian) items are first sorted by their 32-bit
// fp32 depth bits (stable), their pairs are then emitted in that order, and a
// stable sort on the global tile index alone (ceil(log2 tiles) bits, 2 passes
// at 1080p x 8 views) yields each tile's list in (depth bits, item index)
// order. Every pass is a reduce-then-scan LSD pass with 8-bit digits whose
// element count is read from device memory, so the whole sort is enqueued
// without a host sync and can be captured in a CUDA graph.
#include "common.cuh"

namespace gs {

// ---------------------------------------------------------------------------
// Device-wide exclusive scan (reduce, scan of block sums, down-sweep).
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

struct LoadU32 {
    const uint32_t* p;
    __device__ uint32_t operator()(int64_t i) const { return p[i]; }
};
struct LoadTiles {
    const int32_t* n_tiles;
    __device__ uint32_t operator()(int64_t i) const { return n_tiles[i] > 0 ? (uint32_t)n_tiles[i] : 0u; }
};
struct LoadVisible {
    const int32_t* n_tiles;
    __device__ uint32_t operator()(int64_t i) const { return n_tiles[i] > 0 ? 1u : 0u; }
};
struct LoadGatherTiles {
    const int32_t* n_tiles;
    const uint32_t* idx;
    __device__ uint32_t operator()(int64_t i) const { return (uint32_t)n_tiles[idx[i]]; }
};

__device__ __forceinline__ int64_t valid_count(int64_t n_max, const uint32_t* n_dev) {
    return n_dev ? min(n_max, (int64_t)*n_dev) : n_max;
}

// Block-wide exclusive scan of one value per thread; returns the block total.
template <int NT>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t& excl) {
    constexpr int NW = NT / 32;
    __shared__ uint32_t warp_off[NW];
    __shared__ uint32_t s_total;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = v;  // inclusive scan within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_off[w] = inc;
    __syncthreads();
    if (w == 0) {
        const uint32_t t = lane < NW ? warp_off[lane] : 0u;
        uint32_t ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += u;
        }
        if (lane < NW) warp_off[lane] = ti - t;
        if (lane == NW - 1) s_total = ti;
    }
    __syncthreads();
    excl = warp_off[w] + inc - v;
    const uint32_t total = s_total;
    __syncthreads();  // the shared words may be reused by the next call
    return total;
}

template <class Load>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(Load load, int64_t n_max, const uint32_t* n_dev,
                                                              uint32_t* partial) {
    const int64_t n = valid_count(n_max, n_dev);
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++)
        if (base + k < n) s += load(base + k);
    uint32_t excl;
    uint32_t tot = block_exclusive_scan<kScanThreads>(s, excl);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// Single CTA: exclusive scan of nb block sums in place; total -> *total.
__global__ void __launch_bounds__(1024) k_scan_top(uint32_t* partial, int64_t nb, uint32_t* total) {
    const int64_t per = (nb + 1023) / 1024;
    const int64_t b0 = (int64_t)threadIdx.x * per;
    uint32_t s = 0;
    for (int64_t i = b0; i < b0 + per && i < nb; i++) s += partial[i];
    uint32_t excl;
    uint32_t tot = block_exclusive_scan<1024>(s, excl);
    uint32_t run = excl;
    for (int64_t i = b0; i < b0 + per && i < nb; i++) {
        uint32_t t = partial[i];
        partial[i] = run;
        run += t;
    }
    if (threadIdx.x == 0 && total) *total = tot;
}

template <class Load>
__global__ void __launch_bounds__(kScanThreads) k_scan_down(Load load, uint32_t* out, int64_t n_max,
                                                            const uint32_t* n_dev, const uint32_t* partial) {
    const int64_t n = valid_count(n_max, n_dev);
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        v[k] = base + k < n ? load(base + k) : 0u;
        s += v[k];
    }
    uint32_t excl;
    block_exclusive_scan<kScanThreads>(s, excl);
    uint32_t run = excl + partial[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        if (base + k < n_max) out[base + k] = run;
        run += v[k];
    }
}

size_t scan_workspace_bytes(int64_t n_max) { return align256(sizeof(uint32_t) * (ceil_div(n_max, kScanTile) + 1)); }

template <class Load>
static void scan_exclusive(Load load, uint32_t* out, int64_t n_max, const uint32_t* n_dev, uint32_t* total, void* ws,
                           cudaStream_t s) {
    const int64_t nb = ceil_div(n_max, kScanTile);
    uint32_t* partial = (uint32_t*)ws;
    if (nb == 0) return;
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(load, n_max, n_dev, partial);
    count_launch();
    k_scan_top<<<1, 1024, 0, s>>>(partial, nb, total);
    count_launch();
    k_scan_down<<<(unsigned)nb, kScanThreads, 0, s>>>(load, out, n_max, n_dev, partial);
    count_launch();
}

void scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total, void* ws, cudaStream_t s) {
    scan_exclusive(LoadU32{in}, out, n, nullptr, total, ws, s);
}

// ---------------------------------------------------------------------------
// LSD radix sort, 8-bit digits, stable.
//
// Each CTA owns 4096 consecutive keys. The histogram pass counts digits with
// shared-memory atomics into per-warp sub-histograms. The scatter pass ranks
// keys within each warp (peers by one ballot per digit bit, running per-warp digit
// counts in shared memory), turns warp counts into block-local digit offsets,
// places keys and values in shared memory in sorted order and then writes
// each digit's run to its global offset with consecutive threads on
// consecutive addresses.
// ---------------------------------------------------------------------------
constexpr int kRadixThreads = 256;
constexpr int kRadixWarps = kRadixThreads / 32;
constexpr int kRadixIters = 16;                                 // 32-key rounds per warp
constexpr int kRadixTile = kRadixThreads * kRadixIters;         // 4096 keys per CTA
constexpr int kRadixWarpSpan = 32 * kRadixIters;                // 512 keys per warp

int64_t radix_blocks(int64_t n_max) { return ceil_div(n_max, kRadixTile); }

// Per-CTA digit histogram, stored digit-major: hist[d * nb + block].
__global__ void __launch_bounds__(kRadixThreads) k_radix_hist(const uint32_t* __restrict__ keys, int64_t n_max,
                                                              const uint32_t* n_dev, int shift, uint32_t* hist,
                                                              int64_t nb) {
    __shared__ uint32_t h[kRadixWarps][256];
    const int w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kRadixWarps * 256; i += kRadixThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    const int64_t n = valid_count(n_max, n_dev);
    const int64_t b0 = (int64_t)blockIdx.x * kRadixTile;
    if (b0 < n) {
        uint32_t k[kRadixIters];
#pragma unroll
        for (int it = 0; it < kRadixIters; it++) {
            const int64_t idx = b0 + it * kRadixThreads + threadIdx.x;
            k[it] = idx < n ? keys[idx] : 0u;
        }
#pragma unroll
        for (int it = 0; it < kRadixIters; it++)
            if (b0 + it * kRadixThreads + threadIdx.x < n) atomicAdd(&h[w][(k[it] >> shift) & 255u], 1u);
    }
    __syncthreads();
    uint32_t s = 0;
#pragma unroll
    for (int q = 0; q < kRadixWarps; q++) s += h[q][threadIdx.x];
    hist[(int64_t)threadIdx.x * nb + blockIdx.x] = s;
}

// vin == nullptr: the values are the keys' input positions (0, 1, 2, ...).
__global__ void __launch_bounds__(kRadixThreads, 3) k_radix_scatter(const uint32_t* __restrict__ kin,
                                                                 const uint32_t* __restrict__ vin,
                                                                 uint32_t* __restrict__ kout,
                                                                 uint32_t* __restrict__ vout, int64_t n_max,
                                                                 const uint32_t* n_dev, int shift,
                                                                 const uint32_t* __restrict__ hist, int64_t nb) {
    __shared__ uint32_t cnt[kRadixWarps][256];  // per-warp digit counts, then each warp's offset within the digit
    __shared__ uint32_t goff[256];              // global offset of this CTA's run of each digit
    __shared__ uint32_t dstart[256];            // block-local start of each digit
    __shared__ uint32_t s_k[kRadixTile];
    __shared__ uint32_t s_v[kRadixTile];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t n = valid_count(n_max, n_dev);
    const int64_t b0 = (int64_t)blockIdx.x * kRadixTile;
    if (b0 >= n) return;  // uniform over the CTA
    for (int i = threadIdx.x; i < kRadixWarps * 256; i += kRadixThreads) (&cnt[0][0])[i] = 0;
    goff[threadIdx.x] = hist[(int64_t)threadIdx.x * nb + blockIdx.x];
    __syncthreads();
    const int64_t base = b0 + (int64_t)w * kRadixWarpSpan;
    // this lane's keys are kin[base + lane + 32 it] for 32 it < rem
    const int64_t rem = n - base - lane;
    const uint32_t* kp = kin + base + lane;
    uint32_t kk[kRadixIters], rank[kRadixIters];  // values are loaded after ranking (fewer registers)
#pragma unroll
    for (int it = 0; it < kRadixIters; it++) kk[it] = 32 * it < rem ? kp[32 * it] : 0u;
#pragma unroll
    for (int it = 0; it < kRadixIters; it++) {
        const bool valid = 32 * it < rem;
        const unsigned d = valid ? (kk[it] >> shift) & 255u : 256u;
        // lanes holding the same digit: one ballot per bit of the 9-bit label
        // (256 marks a missing key), all in registers
        unsigned peers = 0xffffffffu;
#pragma unroll
        for (int b = 0; b < 9; b++) {
            const bool bit = (d >> b) & 1u;
            const unsigned bal = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? bal : ~bal;
        }
        const unsigned lower = peers & lanemask_lt();
        const uint32_t before = valid ? cnt[w][d] : 0u;
        __syncwarp();
        if (valid && lower == 0) cnt[w][d] = before + __popc(peers);
        __syncwarp();
        rank[it] = valid ? before + __popc(lower) : 0xFFFFFFFFu;
    }
    __syncthreads();
    uint32_t tot = 0;  // thread t handles digit t
#pragma unroll
    for (int q = 0; q < kRadixWarps; q++) {
        const uint32_t c = cnt[q][threadIdx.x];
        cnt[q][threadIdx.x] = tot;
        tot += c;
    }
    uint32_t ex;
    block_exclusive_scan<kRadixThreads>(tot, ex);
    dstart[threadIdx.x] = ex;
    __syncthreads();
    uint32_t vv[kRadixIters];
    const uint32_t* vp = vin ? vin + base + lane : nullptr;
#pragma unroll
    for (int it = 0; it < kRadixIters; it++)
        vv[it] = 32 * it < rem ? (vp ? vp[32 * it] : (uint32_t)(base + lane + 32 * it)) : 0u;
#pragma unroll
    for (int it = 0; it < kRadixIters; it++) {
        if (rank[it] != 0xFFFFFFFFu) {
            const unsigned d = (kk[it] >> shift) & 255u;
            const uint32_t pos = dstart[d] + cnt[w][d] + rank[it];
            s_k[pos] = kk[it];
            s_v[pos] = vv[it];
        }
    }
    __syncthreads();
    const int cnt_block = (int)min((int64_t)kRadixTile, n - b0);
    for (int i = threadIdx.x; i < cnt_block; i += kRadixThreads) {
        const uint32_t k = s_k[i];
        const unsigned d = (k >> shift) & 255u;
        const uint32_t dest = goff[d] + (uint32_t)i - dstart[d];
        if ((int64_t)dest < n) {  // always true for a consistent histogram; guards the scatter
            kout[dest] = k;
            vout[dest] = s_v[i];
        }
    }
}

bool radix_sort_pairs(uint32_t* ka, uint32_t* va, uint32_t* kb, uint32_t* vb, int64_t n_max, const uint32_t* n_dev,
                      int bits, uint32_t* hist, void* scan_ws, cudaStream_t s, bool va_is_position) {
    const int64_t nb = radix_blocks(n_max);
    bool in_b = false;
    if (nb == 0) return false;
    for (int shift = 0; shift < bits; shift += 8) {
        uint32_t* ki = in_b ? kb : ka;
        const uint32_t* vi = in_b ? vb : (va_is_position && shift == 0 ? nullptr : va);
        uint32_t* ko = in_b ? ka : kb;
        uint32_t* vo = in_b ? va : vb;
        k_radix_hist<<<(unsigned)nb, kRadixThreads, 0, s>>>(ki, n_max, n_dev, shift, hist, nb);
        count_launch();
        scan_exclusive(LoadU32{hist}, hist, 256 * nb, nullptr, nullptr, scan_ws, s);
        k_radix_scatter<<<(unsigned)nb, kRadixThreads, 0, s>>>(ki, vi, ko, vo, n_max, n_dev, shift, hist, nb);
        count_launch();
        in_b = !in_b;
    }
    return in_b;
}

// ---------------------------------------------------------------------------
// gs_sort stages
// ---------------------------------------------------------------------------
__global__ void k_compact_visible(const int32_t* __restrict__ n_tiles, const float4* __restrict__ rgb_depth,
                                  const uint32_t* __restrict__ pos, int64_t n_items, uint32_t* __restrict__ key,
                                  uint32_t* __restrict__ val) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_items || n_tiles[i] <= 0) return;
    const uint32_t p = pos[i];
    key[p] = __float_as_uint(rgb_depth[i].w);  // depth > near_z > 0: bits are monotone
    val[p] = (uint32_t)i;
}

// count[0] = number of pairs; n_eff = min(count, capacity); status
__global__ void k_pair_count(const uint32_t* total, int64_t capacity, int64_t* count, uint32_t* n_eff,
                             int32_t* status) {
    const uint32_t t = *total;
    *count = t;
    *n_eff = (uint32_t)min((int64_t)t, capacity);
    *status = (int64_t)t > capacity ? GS_ERR_CAPACITY : GS_OK;
}

// One (tile, item) pair per tile of each visible item's rect, the items taken
// in depth order: pair positions follow depth order (what the stable tile sort
// needs); each pair also records its item and its emission slot - in item
// order: the item's first slot (offset) plus the pair's index in the item. A warp
// owns 32 consecutive sorted items, whose pairs occupy consecutive positions,
// and writes them together: pair j of the warp's run finds its item by a
// binary search over the lanes' prefix counts, so consecutive lanes write
// consecutive positions whatever the rect sizes.
__global__ void __launch_bounds__(256) k_duplicate(const uint32_t* __restrict__ sorted_item,
                                                   const uint32_t* __restrict__ emit_off, const uint32_t* n_vis,
                                                   const ushort4* __restrict__ rect, int64_t n, gs_frame f,
                                                   int64_t capacity, const uint32_t* __restrict__ offset,
                                                   uint32_t* __restrict__ pkey, uint2* __restrict__ psrc) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nv = *n_vis;
    if (s - lane >= nv) return;  // uniform over the warp
    uint32_t item = 0, off = 0, x0 = 0, y0 = 0, wx = 1, cnt = 0, tb = 0, tx = 0, slot0 = 0;
    if (s < nv) {
        item = sorted_item[s];
        off = emit_off[s];
        slot0 = offset[item];
        const int v = (int)(item / (uint64_t)n);
        const ushort4 r = rect[item];
        tb = (uint32_t)f.tile_base[v];
        tx = (uint32_t)f.tiles_x[v];
        const uint32_t ty = (uint32_t)f.tiles_y[v];
        // rect is clamped to the view's grid by gs_project; re-clamp so foreign input cannot index past it
        x0 = min((uint32_t)r.x, tx);
        const uint32_t x1 = max(min((uint32_t)r.z, tx), x0);
        y0 = min((uint32_t)r.y, ty);
        const uint32_t y1 = max(min((uint32_t)r.w, ty), y0);
        wx = max(x1 - x0, 1u);
        cnt = (x1 - x0) * (y1 - y0);
    }
    uint32_t start = cnt;  // inclusive, then exclusive prefix of cnt over the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(FULL, start, o);
        if (lane >= o) start += t;
    }
    const uint32_t total = __shfl_sync(FULL, start, 31);
    start -= cnt;
    for (uint32_t b = 0; b < total; b += 32) {
        const uint32_t j = b + lane;
        int L = 0;  // highest lane whose prefix start is <= j
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            const uint32_t st = __shfl_sync(FULL, start, L + step);
            if (L + step < 32 && st <= j) L += step;
        }
        const uint32_t st = __shfl_sync(FULL, start, L);
        const uint32_t o = __shfl_sync(FULL, off, L);
        const uint32_t it = __shfl_sync(FULL, item, L);
        const uint32_t sl = __shfl_sync(FULL, slot0, L);
        const uint32_t ax = __shfl_sync(FULL, x0, L), ay = __shfl_sync(FULL, y0, L);
        const uint32_t aw = __shfl_sync(FULL, wx, L), atb = __shfl_sync(FULL, tb, L), atx = __shfl_sync(FULL, tx, L);
        if (j < total) {
            const uint32_t local = j - st;
            const uint32_t yy = local / aw, xx = local - yy * aw;
            const int64_t e = (int64_t)o + local;
            if (e < capacity) {
                pkey[e] = atb + (ay + yy) * atx + ax + xx;
                psrc[e] = make_uint2(it, sl + local);
            }
        }
    }
}

// Sorted pair p: its item, its emission slot (the item's first slot in item
// order plus the pair's index within the item) and the tile ranges.
__global__ void k_finish_pairs(const uint32_t* __restrict__ skey, const uint32_t* __restrict__ sval,
                               const uint2* __restrict__ psrc, const uint32_t* n_eff, uint32_t* __restrict__ src,
                               uint32_t* __restrict__ emit, uint32_t* __restrict__ range) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t cnt = *n_eff;
    if (p >= cnt) return;
    const uint2 q = psrc[sval[p]];  // (item, emission slot) of the pair at that position before the sort
    src[p] = q.x;
    emit[p] = q.y;
    const uint32_t t = skey[p];
    if (p == 0 || skey[p - 1] != t) range[2 * (int64_t)t] = (uint32_t)p;
    if (p == cnt - 1 || skey[p + 1] != t) range[2 * (int64_t)t + 1] = (uint32_t)(p + 1);
}

// Work order of the persistent schedule: tiles by decreasing pair count.
__global__ void k_tile_order_keys(const uint32_t* __restrict__ range, int64_t n_tiles, uint32_t* __restrict__ key,
                                  uint32_t* __restrict__ val) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    const uint32_t len = range[2 * t + 1] - range[2 * t];
    key[t] = 0xFFFFu - min(len, 0xFFFFu);
    val[t] = (uint32_t)t;
}

__global__ void k_copy_u32(const uint32_t* __restrict__ a, uint32_t* __restrict__ b, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i];
}

struct SortWs {
    uint32_t *scan, *vis_pos, *vk0, *vv0, *vk1, *vv1, *emit_off, *pk0, *pv0, *pk1, *pv1, *hist, *misc;
    uint2* psrc;
    uint32_t *tk0, *tv0, *tk1, *tv1;
};

static SortWs carve_sort(char* base, size_t cap_bytes, int64_t n_items, int64_t capacity, int64_t n_tiles,
                         size_t* used) {
    Carve c{base, 0, cap_bytes};
    SortWs w;
    int64_t m = n_items > capacity ? n_items : capacity;
    m = m > n_tiles ? m : n_tiles;
    w.scan = c.take<uint32_t>(scan_workspace_bytes(256 * radix_blocks(m) > m ? 256 * radix_blocks(m) : m) / 4);
    w.vis_pos = c.take<uint32_t>(n_items);
    w.vk0 = c.take<uint32_t>(n_items);
    w.vv0 = c.take<uint32_t>(n_items);
    w.vk1 = c.take<uint32_t>(n_items);
    w.vv1 = c.take<uint32_t>(n_items);
    w.emit_off = c.take<uint32_t>(n_items + 1);
    w.pk0 = c.take<uint32_t>(capacity);
    w.pv0 = c.take<uint32_t>(capacity);
    w.pk1 = c.take<uint32_t>(capacity);
    w.pv1 = c.take<uint32_t>(capacity);
    w.psrc = c.take<uint2>(capacity);
    w.hist = c.take<uint32_t>(256 * radix_blocks(m));
    w.misc = c.take<uint32_t>(8);
    w.tk0 = c.take<uint32_t>(n_tiles);
    w.tv0 = c.take<uint32_t>(n_tiles);
    w.tk1 = c.take<uint32_t>(n_tiles);
    w.tv1 = c.take<uint32_t>(n_tiles);
    *used = c.used;
    return w;
}

static int bits_for(int64_t v) {
    int b = 0;
    while (b < 32 && ((int64_t)1 << b) < v) b++;
    return b < 1 ? 1 : b;
}

}  // namespace gs

using namespace gs;

extern "C" size_t gs_sort_workspace_size(int64_t n, const gs_frame* f, int64_t capacity) {
    if (!f || n < 0 || capacity < 0) return 0;
    size_t used = 0;
    carve_sort(nullptr, 0, n * f->n_views, capacity, f->tile_base[f->n_views], &used);
    return used;
}

extern "C" int gs_sort(const gs_projected* p, int64_t n, const gs_frame* f, const gs_pairs* out, void* ws,
                       size_t ws_bytes, void* stream) {
    if (!p || !f || !out || n < 0 || f->n_views < 1 || f->n_views > GS_MAX_VIEWS) return GS_ERR_INVALID_ARG;
    const int64_t n_items = n * f->n_views;
    if (n_items > (int64_t)UINT32_MAX || out->capacity < 0 || out->capacity > (int64_t)UINT32_MAX - 1)
        return GS_ERR_INVALID_ARG;
    if (!out->count || !out->status || !out->range || (out->capacity > 0 && (!out->src || !out->emit)) ||
        (n_items > 0 && !out->offset))
        return GS_ERR_INVALID_ARG;
    size_t need = 0;
    const int64_t n_tiles_all = f->tile_base[f->n_views];
    SortWs w = carve_sort((char*)ws, ws_bytes, n_items, out->capacity, n_tiles_all, &need);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n_tiles_total = f->tile_base[f->n_views];
    uint32_t* n_vis = w.misc;        // visible item count
    uint32_t* p_total = w.misc + 1;  // pair count
    uint32_t* n_eff = w.misc + 2;    // pairs actually stored
    cudaMemsetAsync(out->range, 0, sizeof(uint32_t) * 2 * n_tiles_total, s);
    cudaMemsetAsync(w.misc, 0, 8 * sizeof(uint32_t), s);
    if (n_items == 0) {
        k_pair_count<<<1, 1, 0, s>>>(p_total, out->capacity, out->count, n_eff, out->status);
        count_launch();
        GS_CUDA_CHECK_LAUNCH();
        return GS_OK;
    }
    // 1. compact visible items (in item order) with their depth keys
    scan_exclusive(LoadVisible{p->n_tiles}, w.vis_pos, n_items, nullptr, n_vis, w.scan, s);
    k_compact_visible<<<(unsigned)ceil_div(n_items, 256), 256, 0, s>>>(p->n_tiles, (const float4*)p->rgb_depth,
                                                                       w.vis_pos, n_items, w.vk0, w.vv0);
    count_launch();
    // 2. stable sort of visible items by depth bits
    const bool in1 = radix_sort_pairs(w.vk0, w.vv0, w.vk1, w.vv1, n_items, n_vis, 32, w.hist, w.scan, s, false);
    const uint32_t* sorted_item = in1 ? w.vv1 : w.vv0;
    // 3. pair positions in depth order; pair count; emission slots in item order (each item's pairs
    //    occupy offset[item] .. offset[item] + n_tiles - 1, so the adjoint's per-item runs of the
    //    Gaussians of one view are adjacent)
    scan_exclusive(LoadGatherTiles{p->n_tiles, sorted_item}, w.emit_off, n_items, n_vis, p_total, w.scan, s);
    scan_exclusive(LoadTiles{p->n_tiles}, out->offset, n_items, nullptr, nullptr, w.scan, s);
    k_pair_count<<<1, 1, 0, s>>>(p_total, out->capacity, out->count, n_eff, out->status);
    count_launch();
    // 4. duplicate: one (tile, emission slot) pair per tile of each visible item's rect
    k_duplicate<<<(unsigned)ceil_div(n_items, 256), 256, 0, s>>>(sorted_item, w.emit_off, n_vis,
                                                                 (const ushort4*)p->rect, n, *f, out->capacity,
                                                                 out->offset, w.pk0, w.psrc);
    count_launch();
    // 5. stable sort by global tile index; 6. gather sources, tile ranges
    if (out->capacity > 0) {
        // the pairs' values are their emission slots, i.e. their positions before the sort
        const bool pin1 = radix_sort_pairs(w.pk0, w.pv0, w.pk1, w.pv1, out->capacity, n_eff,
                                           bits_for(n_tiles_total), w.hist, w.scan, s, true);
        k_finish_pairs<<<(unsigned)ceil_div(out->capacity, 256), 256, 0, s>>>(
            pin1 ? w.pk1 : w.pk0, pin1 ? w.pv1 : w.pv0, w.psrc, n_eff, out->src, out->emit, out->range);
        count_launch();
    }
    // 7. optional work order for the persistent render schedule
    if (out->order && n_tiles_total > 0) {
        k_tile_order_keys<<<(unsigned)ceil_div(n_tiles_total, 256), 256, 0, s>>>(out->range, n_tiles_total, w.tk0,
                                                                                  w.tv0);
        count_launch();
        const bool t1 = radix_sort_pairs(w.tk0, w.tv0, w.tk1, w.tv1, n_tiles_total, nullptr, 16, w.hist, w.scan, s,
                                         false);
        k_copy_u32<<<(unsigned)ceil_div(n_tiles_total, 256), 256, 0, s>>>(t1 ? w.tv1 : w.tv0, out->order,
                                                                           n_tiles_total);
        count_launch();
    }
    GS_CUDA_CHECK_LAUNCH();
    return GS_OK;
}
