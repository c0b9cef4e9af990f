// Per-tile duplication and depth ordering (K2-K4).
//
// Design: instead of one radix sort of 64-bit (tile, depth) keys over all P
// pairs, the V visible (view, Gaussian) items are first sorted by their 32-bit
// fp32 depth bits (stable), their pairs are then emitted in that order, and a
// stable sort on the global tile index alone (ceil(log2 tiles) bits, 2 passes
// at 1080p x 8 views) yields each tile's list in (depth bits, item index)
// order. gs_sort uses single-pass kernels: each scan is one launch (chunks with
// decoupled look-back) and each radix sort is one histogram launch for all its
// 8-bit digits plus one launch per digit (tiles with decoupled look-back); the
// tile sort carries every pair's (item, emission slot) and its last pass writes
// them to the output lists. Element counts are read from device memory, so the
// whole sort is enqueued without a host sync and can be captured in a CUDA
// graph. The reduce-then-scan scan and radix sort below serve the library's
// other compactions and sorts (spawning, anchors).
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
// Single-pass scans and one-sweep radix passes with decoupled look-back (the
// scheme of Merrill & Garland's single-pass prefix scan and of Adinets &
// Merrill's Onesweep radix sort). CTAs take consecutive tiles of the input by
// ticket (an atomic counter), so every tile below a CTA's own belongs to a CTA
// that started earlier. Each CTA publishes its tile's aggregate at once, then
// walks back over the earlier tiles' words - adding aggregates until it meets
// an inclusive prefix - and publishes its own inclusive prefix. A CTA only
// ever waits for earlier tiles to publish their aggregate, which they do
// before waiting on anything, so the waits always end; each poll loop is
// still bounded (kSpinLimit polls), after which the CTA records
// GS_ERR_TIMEOUT in an error word and carries on with the prefix it has.
// Look-back words are 64-bit: flag in bits 62-63, a 32-bit count below.
// ---------------------------------------------------------------------------
constexpr uint64_t kLbAgg = 1ull << 62, kLbPre = 2ull << 62, kLbFlags = 3ull << 62;
constexpr int kSpinLimit = 1 << 22;
constexpr int kMaxPasses = 4;

__device__ __forceinline__ uint64_t lb_load(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void lb_store(uint64_t* p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Exclusive prefix of tile `tile` from the look-back words of the tiles before
// it (word stride `stride` between tiles), one thread: the words of kLbWin
// earlier tiles are loaded at once, then added newest first until an
// inclusive prefix; a tile not yet published is polled again. 0 for tile 0.
constexpr int kLbWin = 8;
__device__ __forceinline__ uint32_t look_back(const uint64_t* words, int64_t tile, int64_t stride, int32_t* err) {
    uint32_t excl = 0;
    int64_t j = tile - 1;
    int spins = 0;
    while (j >= 0) {
        uint64_t v[kLbWin];
#pragma unroll
        for (int q = 0; q < kLbWin; q++) v[q] = j - q >= 0 ? lb_load(words + (j - q) * stride) : kLbPre;
        int q = 0;
        bool found = false;
#pragma unroll
        for (int r = 0; r < kLbWin; r++) {
            if (q == r) {
                if ((v[r] & kLbFlags) != 0) {
                    excl += (uint32_t)v[r];
                    q++;
                    if (v[r] & kLbPre) found = true;
                }
            }
            if (found) break;
        }
        if (found) break;
        j -= q;  // q < kLbWin: tile j - q is not published yet; poll it again
        if (q < kLbWin && ++spins > kSpinLimit) {
            if (err) atomicExch(err, GS_ERR_TIMEOUT);
            break;
        }
    }
    return excl;
}

// The same, by a whole CTA of NT threads: thread t reads the word of tile
// j - t, so each round covers NT earlier tiles (the walk back from a tile is
// about as long as the number of CTAs in flight, so it must cover many tiles
// per round). Called by every thread; returns the prefix in every thread.
template <int NT>
__device__ __forceinline__ uint32_t look_back_cta(const uint64_t* words, int64_t tile, int32_t* err) {
    constexpr int NW = NT / 32;
    __shared__ unsigned s_min[NW];
    __shared__ uint32_t s_sum[NW];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t excl = 0;
    int64_t j = tile - 1;
    int spins = 0;
    while (j >= 0) {  // uniform over the CTA
        const int64_t jj = j - threadIdx.x;
        const uint64_t v = jj >= 0 ? lb_load(words + jj) : kLbPre;  // before tile 0: an empty prefix
        // nearest inclusive prefix among the NT words
        const unsigned wm = __reduce_min_sync(FULL, (v & kLbPre) ? (unsigned)threadIdx.x : (unsigned)NT);
        if (lane == 0) s_min[w] = wm;
        __syncthreads();
        unsigned first = NT;
#pragma unroll
        for (int q = 0; q < NW; q++) first = min(first, s_min[q]);
        const bool need = (unsigned)threadIdx.x <= first;
        if (__syncthreads_or(need && (v & kLbFlags) == 0)) {  // a needed tile is not published yet
            if (++spins > kSpinLimit) {
                if (err && threadIdx.x == 0) atomicExch(err, GS_ERR_TIMEOUT);
                break;
            }
            continue;
        }
        const uint32_t ws = __reduce_add_sync(FULL, need ? (uint32_t)v : 0u);
        if (lane == 0) s_sum[w] = ws;
        __syncthreads();
#pragma unroll
        for (int q = 0; q < NW; q++) excl += s_sum[q];
        __syncthreads();  // s_min / s_sum are rewritten by the next round
        if (first < (unsigned)NT) break;
        j -= NT;
    }
    return excl;
}

// Control words of one single-pass scan or one radix sort, zeroed by the
// caller before the first kernel that uses them.
struct ScanCtl {
    uint32_t ticket;
};
struct SortCtl {
    uint32_t count[kMaxPasses][256];  // digit counts of every pass, then their exclusive sums
    uint32_t ticket[kMaxPasses];
    uint32_t hist_done;
};

// Exclusive scan of load(0..n-1) into out[0..n_max) (positions at or past the
// valid count n = min(n_max, *n_dev) get the total), total -> *total.
// Per-element step after a scan: nothing, or (visible-item compaction) the
// item's depth key and index written at its exclusive prefix.
struct NoEpilogue {
    __device__ void operator()(int64_t, uint32_t) const {}
};
struct CompactVisible {
    const int32_t* n_tiles;
    const float4* rgb_depth;
    uint32_t* key;
    uint32_t* val;
    __device__ void operator()(int64_t i, uint32_t p) const {
        if (n_tiles[i] > 0) {
            key[p] = __float_as_uint(rgb_depth[i].w);  // depth > near_z > 0: bits are monotone
            val[p] = (uint32_t)i;
        }
    }
};

// Exclusive scan of load(0..n-1) into out[0..n_max) (positions at or past the
// valid count n = min(n_max, *n_dev) get the total; out may be null), epi
// called with each valid position and its prefix, total -> *total. Each CTA
// takes one contiguous chunk: it sums the chunk, publishes the sum, looks
// back over the earlier chunks (all CTAs of the grid run at once, so the walk
// covers at most a round or two of the CTA-wide window), then scans the chunk
// tile by tile (its second read mostly hits L2).
template <class Load, class Epi>
__global__ void __launch_bounds__(kScanThreads) k_scan_single(Load load, Epi epi, uint32_t* __restrict__ out,
                                                              int64_t n_max, const uint32_t* n_dev, int64_t chunk,
                                                              ScanCtl* ctl, uint64_t* words, uint32_t* total,
                                                              int32_t* err) {
    // each tile passes through shared memory so that global loads and stores
    // are coalesced while each thread scans 8 consecutive values (one padding
    // word per 32 keeps the per-thread reads free of bank conflicts)
    __shared__ uint32_t s_v[kScanTile + kScanTile / 32];
    __shared__ uint32_t s_tile;
    if (threadIdx.x == 0) s_tile = atomicAdd(&ctl->ticket, 1u);
    __syncthreads();
    const int64_t c = s_tile;
    const int64_t c0 = c * chunk;
    if (c0 >= n_max) return;  // uniform over the CTA
    const int64_t c1 = min(c0 + chunk, n_max);
    const int64_t n = valid_count(n_max, n_dev);
    const int64_t cv = min(c1, n);  // end of the valid part of the chunk
    uint32_t sum = 0;
#pragma unroll 2
    for (int64_t i0 = c0; i0 < cv; i0 += kScanTile) {
        uint32_t part[kScanItems];
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            const int64_t i = i0 + k * kScanThreads + threadIdx.x;
            part[k] = i < cv ? load(i) : 0u;
        }
#pragma unroll
        for (int k = 0; k < kScanItems; k++) sum += part[k];
    }
    uint32_t unused;
    const uint32_t agg = block_exclusive_scan<kScanThreads>(sum, unused);
    uint64_t* mine = words + c;
    uint32_t run = 0;
    if (c == 0) {
        if (threadIdx.x == 0) lb_store(mine, kLbPre | agg);
    } else {
        if (threadIdx.x == 0) lb_store(mine, kLbAgg | agg);
        run = look_back_cta<kScanThreads>(words, c, err);
        if (threadIdx.x == 0) lb_store(mine, kLbPre | (uint32_t)(run + agg));
    }
    if (threadIdx.x == 0 && total && c1 >= n_max) *total = run + agg;
    for (int64_t t0 = c0; t0 < c1; t0 += kScanTile) {
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            const int i = k * kScanThreads + threadIdx.x;
            s_v[i + (i >> 5)] = t0 + i < cv ? load(t0 + i) : 0u;
        }
        __syncthreads();
        uint32_t v[kScanItems];
        uint32_t tsum = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            const int i = threadIdx.x * kScanItems + k;
            v[k] = s_v[i + (i >> 5)];
            tsum += v[k];
        }
        uint32_t excl;
        const uint32_t tagg = block_exclusive_scan<kScanThreads>(tsum, excl);
        uint32_t r = run + excl;
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            const int i = threadIdx.x * kScanItems + k;
            s_v[i + (i >> 5)] = r;
            r += v[k];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            const int i = k * kScanThreads + threadIdx.x;
            if (t0 + i < c1) {
                const uint32_t ex = s_v[i + (i >> 5)];
                if (out) out[t0 + i] = ex;
                if (t0 + i < n) epi(t0 + i, ex);
            }
        }
        run += tagg;
        __syncthreads();  // s_v is rewritten by the next tile
    }
}

// CTAs of the single-pass scan: four per SM (each CTA's two walks over its
// chunk are latency-bound, so shorter chunks finish sooner), each with one
// chunk of whole tiles.
static int64_t scan_ctas() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        sms = v > 0 ? v : 152;
    }
    return 4 * (int64_t)sms;
}

template <class Load, class Epi = NoEpilogue>
static void scan_single(Load load, uint32_t* out, int64_t n_max, const uint32_t* n_dev, uint32_t* total,
                        ScanCtl* ctl, uint64_t* words, int32_t* err, cudaStream_t s, Epi epi = Epi{}) {
    const int64_t tiles = ceil_div(n_max, kScanTile);
    if (tiles == 0) return;
    const int64_t g = tiles < scan_ctas() ? tiles : scan_ctas();
    const int64_t chunk = ceil_div(tiles, g) * kScanTile;
    k_scan_single<<<(unsigned)ceil_div(n_max, chunk), kScanThreads, 0, s>>>(load, epi, out, n_max, n_dev, chunk, ctl,
                                                                           words, total, err);
    count_launch();
}

// Digit counts of every pass in one read of the keys (shared-memory atomics
// into per-warp sub-histograms), then, in the last CTA to finish, their
// exclusive sums: the global start of each digit. Also zeroes the first
// pass's look-back words and the passes' tickets.
__global__ void __launch_bounds__(256) k_onesweep_hist(const uint32_t* __restrict__ keys, int64_t n_max,
                                                       const uint32_t* n_dev, int passes, SortCtl* ctl,
                                                       uint64_t* words0) {
    __shared__ uint32_t h[kRadixWarps][kMaxPasses][256];
    __shared__ bool s_last;
    const int w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kRadixWarps * kMaxPasses * 256; i += 256) (&h[0][0][0])[i] = 0;
    __syncthreads();
    const int64_t n = valid_count(n_max, n_dev);
    const int64_t stride = (int64_t)gridDim.x * 256;
    // 4096-key tiles, 16 keys per thread loaded before any is counted
    for (int64_t t0 = (int64_t)blockIdx.x * kRadixTile; t0 < n; t0 += (int64_t)gridDim.x * kRadixTile) {
        uint32_t k[kRadixIters];
#pragma unroll
        for (int it = 0; it < kRadixIters; it++) {
            const int64_t i = t0 + it * 256 + threadIdx.x;
            k[it] = i < n ? keys[i] : 0u;
        }
#pragma unroll
        for (int it = 0; it < kRadixIters; it++)
            if (t0 + it * 256 + threadIdx.x < n)
                for (int p = 0; p < passes; p++) atomicAdd(&h[w][p][(k[it] >> (8 * p)) & 255u], 1u);
    }
    const int64_t tiles = ceil_div(n, kRadixTile);
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < tiles * 256; i += stride) words0[i] = 0;
    __syncthreads();
    for (int p = 0; p < passes; p++) {
        uint32_t c = 0;
#pragma unroll
        for (int q = 0; q < kRadixWarps; q++) c += h[q][p][threadIdx.x];
        if (c) atomicAdd(&ctl->count[p][threadIdx.x], c);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&ctl->hist_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int p = 0; p < passes; p++) {
        const uint32_t c = atomicAdd(&ctl->count[p][threadIdx.x], 0u);  // read past L1
        uint32_t ex;
        block_exclusive_scan<256>(c, ex);
        ctl->count[p][threadIdx.x] = ex;
    }
    if (threadIdx.x < kMaxPasses) ctl->ticket[threadIdx.x] = 0;
}

// One 8-bit digit pass. Values of type V travel with the keys: vin ==
// nullptr means the values are the keys' input positions (V = uint32_t);
// with out_x / out_y set (V = uint2), the last pass writes the two halves of
// each value to separate arrays. Shared memory holds each key with its index
// in the tile, and the value is fetched from the tile's input range when the
// key is written out, so no value waits in registers. words: this pass's
// look-back words (256 per tile: one per digit); words_next: the next pass's,
// zeroed here for this tile (or null).
template <class V>
__global__ void __launch_bounds__(kRadixThreads, 4) k_onesweep_pass(
    const uint32_t* __restrict__ kin, const V* __restrict__ vin, uint32_t* __restrict__ kout, V* __restrict__ vout,
    uint32_t* __restrict__ out_x, uint32_t* __restrict__ out_y, int64_t n_max, const uint32_t* n_dev, int pass,
    SortCtl* ctl, uint64_t* words, uint64_t* words_next, int32_t* err) {
    __shared__ uint32_t cnt[kRadixWarps][256];  // per-warp digit counts, then each warp's offset within the digit
    __shared__ uint32_t goff[256];              // global offset of this tile's run of each digit
    __shared__ uint32_t dstart[256];            // block-local start of each digit
    __shared__ uint32_t s_k[kRadixTile];
    __shared__ uint16_t s_i[kRadixTile];        // index of the key within the tile
    __shared__ uint32_t s_tile;
    const int shift = 8 * pass;
    if (threadIdx.x == 0) s_tile = atomicAdd(&ctl->ticket[pass], 1u);
    for (int i = threadIdx.x; i < kRadixWarps * 256; i += kRadixThreads) (&cnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t tile = s_tile;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t n = valid_count(n_max, n_dev);
    const int64_t b0 = tile * kRadixTile;
    if (b0 >= n) return;  // uniform over the CTA
    if (words_next) words_next[tile * 256 + threadIdx.x] = 0;
    const int64_t base = b0 + (int64_t)w * kRadixWarpSpan;
    const int64_t rem = n - base - lane;
    const uint32_t* kp = kin + base + lane;
    uint32_t kk[kRadixIters], rank[kRadixIters];
#pragma unroll
    for (int it = 0; it < kRadixIters; it++) kk[it] = 32 * it < rem ? kp[32 * it] : 0u;
#pragma unroll
    for (int it = 0; it < kRadixIters; it++) {
        const bool valid = 32 * it < rem;
        const unsigned d = valid ? (kk[it] >> shift) & 255u : 256u;
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
    uint64_t* mine = words + tile * 256 + threadIdx.x;
    lb_store(mine, (tile == 0 ? kLbPre : kLbAgg) | tot);
    uint32_t ex;
    block_exclusive_scan<kRadixThreads>(tot, ex);
    dstart[threadIdx.x] = ex;
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kRadixIters; it++) {
        if (rank[it] != 0xFFFFFFFFu) {
            const unsigned d = (kk[it] >> shift) & 255u;
            const uint32_t pos = dstart[d] + cnt[w][d] + rank[it];
            s_k[pos] = kk[it];
            s_i[pos] = (uint16_t)(w * kRadixWarpSpan + lane + 32 * it);
        }
    }
    uint32_t pre = 0;
    if (tile > 0) {
        pre = look_back(words + threadIdx.x, tile, 256, err);
        lb_store(mine, kLbPre | (uint32_t)(pre + tot));
    }
    goff[threadIdx.x] = ctl->count[pass][threadIdx.x] + pre;
    __syncthreads();
    const int cnt_block = (int)min((int64_t)kRadixTile, n - b0);
    // the values this thread writes are fetched in batches of VB before their
    // stores, so VB loads are in flight together
    constexpr int VB = sizeof(V) == 8 ? kRadixIters / 2 : kRadixIters;
#pragma unroll
    for (int r0 = 0; r0 < kRadixIters; r0 += VB) {
        V vals[VB];
#pragma unroll
        for (int r = 0; r < VB; r++) {
            const int i = threadIdx.x + (r0 + r) * kRadixThreads;
            const uint32_t src = i < cnt_block ? s_i[i] : 0u;
            if constexpr (sizeof(V) == 4) vals[r] = vin ? vin[b0 + src] : (V)(b0 + src);
            else vals[r] = i < cnt_block ? vin[b0 + src] : V{};
        }
#pragma unroll
        for (int r = 0; r < VB; r++) {
            const int i = threadIdx.x + (r0 + r) * kRadixThreads;
            if (i >= cnt_block) break;
            const uint32_t k = s_k[i];
            const unsigned d = (k >> shift) & 255u;
            const uint32_t dest = goff[d] + (uint32_t)i - dstart[d];
            if ((int64_t)dest < n) {  // always true for consistent counts; guards the scatter after a timeout
                kout[dest] = k;
                if constexpr (sizeof(V) == 8) {
                    if (out_x) {
                        out_x[dest] = vals[r].x;
                        out_y[dest] = vals[r].y;
                        continue;
                    }
                }
                vout[dest] = vals[r];
            }
        }
    }
}

// Look-back words of one radix pass: 256 per tile of the largest input.
static int64_t onesweep_words(int64_t n_max) { return 256 * radix_blocks(n_max); }

// Stable LSD sort of (key, value) pairs on key bits [0, 8 * passes) with
// 1 + passes launches. (ka, va) hold the input, (kb, vb) are the alternates;
// va == nullptr: the input values are the positions 0, 1, 2, ... (V =
// uint32_t). With out_x set (V = uint2), the last pass writes the values'
// two halves to out_x / out_y instead of va / vb. Returns true when the
// sorted keys (and values, unless split) end in (kb, vb). ctl must be zeroed;
// wa / wb: onesweep_words(n_max) words each.
template <class V>
static bool onesweep_sort_pairs(uint32_t* ka, const V* va, uint32_t* kb, V* vb, V* va_alt, int64_t n_max,
                                const uint32_t* n_dev, int bits, SortCtl* ctl, uint64_t* wa, uint64_t* wb,
                                int32_t* err, cudaStream_t s, uint32_t* out_x = nullptr,
                                uint32_t* out_y = nullptr) {
    const int64_t nb = radix_blocks(n_max);
    if (nb == 0) return false;
    const int passes = (bits + 7) / 8;
    const unsigned hist_grid = (unsigned)(nb < 4 * 152 ? nb : 4 * 152);
    k_onesweep_hist<<<hist_grid, 256, 0, s>>>(ka, n_max, n_dev, passes, ctl, wa);
    count_launch();
    bool in_b = false;
    for (int p = 0; p < passes; p++) {
        uint32_t* ki = in_b ? kb : ka;
        const V* vi = p == 0 ? va : in_b ? vb : va_alt;
        uint32_t* ko = in_b ? ka : kb;
        V* vo = in_b ? va_alt : vb;
        const bool last = p + 1 == passes;
        uint64_t* w = (p & 1) ? wb : wa;
        uint64_t* wn = last ? nullptr : ((p & 1) ? wa : wb);
        k_onesweep_pass<V><<<(unsigned)nb, kRadixThreads, 0, s>>>(ki, vi, ko, vo, last ? out_x : nullptr,
                                                                  last ? out_y : nullptr, n_max, n_dev, p, ctl, w,
                                                                  wn, err);
        count_launch();
        in_b = !in_b;
    }
    return in_b;
}

// ---------------------------------------------------------------------------
// gs_sort stages
// ---------------------------------------------------------------------------
// count[0] = number of pairs; n_eff = min(count, capacity); status (a
// look-back timeout recorded in *err so far takes precedence)
__global__ void k_pair_count(const uint32_t* total, int64_t capacity, int64_t* count, uint32_t* n_eff,
                             int32_t* status, const int32_t* err) {
    const uint32_t t = *total;
    *count = t;
    *n_eff = (uint32_t)min((int64_t)t, capacity);
    *status = *err ? *err : (int64_t)t > capacity ? GS_ERR_CAPACITY : GS_OK;
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
    const int64_t nv = *n_vis;
    const int64_t n_chunks = ceil_div(nv, 32);
    const int64_t n_warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    // grid-stride over chunks of 32 sorted items, one warp each
    for (int64_t chunk = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; chunk < n_chunks;
         chunk += n_warps) {
        const int64_t s = chunk * 32 + lane;
        uint32_t item = 0, off = 0, x0 = 0, y0 = 0, wx = 1, cnt = 0, tb = 0, tx = 0, slot0 = 0;
        if (s < nv) {
            item = sorted_item[s];
            off = emit_off[s];
            slot0 = offset[item];
            const int v = (int)(item / (uint32_t)n);  // item < 2^32 (checked by gs_sort)
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
}

// Tile ranges of the sorted pairs (the last tile-sort pass wrote each sorted
// pair's item and emission slot).
__global__ void k_tile_ranges(const uint32_t* __restrict__ skey, const uint32_t* n_eff,
                              uint32_t* __restrict__ range, const int32_t* err, int32_t* status) {
    const int64_t p0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p0 == 0 && *err) *status = *err;
    const int64_t cnt = *n_eff;
    for (int64_t p = p0; p < cnt; p += (int64_t)gridDim.x * blockDim.x) {  // grid-stride: few CTAs
        const uint32_t t = skey[p];
        if (p == 0 || skey[p - 1] != t) range[2 * (int64_t)t] = (uint32_t)p;
        if (p == cnt - 1 || skey[p + 1] != t) range[2 * (int64_t)t + 1] = (uint32_t)(p + 1);
    }
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

__global__ void k_copy_u32(const uint32_t* __restrict__ a, uint32_t* __restrict__ b, int64_t n, const int32_t* err,
                           int32_t* status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && *err) *status = *err;
    if (i < n) b[i] = a[i];
}

struct SortWs {
    uint32_t *vk0, *vv0, *vk1, *vv1, *emit_off, *pk0, *pk1, *misc;
    uint2 *psrc, *psrc2;
    uint32_t *tk0, *tv0, *tk1, *tv1;
    // zeroed together at the start of every call: control words of the three
    // scans and the three sorts, and the scans' look-back words
    char* zero_base;
    size_t zero_bytes;
    ScanCtl* scan_ctl;     // [3]
    SortCtl* sort_ctl;     // [3]
    uint64_t* scan_words;  // [3][scan tiles]
    uint64_t *wa, *wb;     // radix look-back words (zeroed by the kernels)
};

static SortWs carve_sort(char* base, size_t cap_bytes, int64_t n_items, int64_t capacity, int64_t n_tiles,
                         size_t* used) {
    Carve c{base, 0, cap_bytes};
    SortWs w;
    int64_t m = n_items > capacity ? n_items : capacity;
    m = m > n_tiles ? m : n_tiles;
    const int64_t scan_tiles = ceil_div(n_items > n_tiles ? n_items : n_tiles, kScanTile);
    w.misc = c.take<uint32_t>(8);
    const size_t z0 = c.used;
    w.scan_ctl = c.take<ScanCtl>(3);
    w.sort_ctl = c.take<SortCtl>(3);
    w.scan_words = c.take<uint64_t>(3 * scan_tiles);
    w.zero_base = base ? base + z0 : nullptr;
    w.zero_bytes = c.used - z0;
    w.vk0 = c.take<uint32_t>(n_items);
    w.vv0 = c.take<uint32_t>(n_items);
    w.vk1 = c.take<uint32_t>(n_items);
    w.vv1 = c.take<uint32_t>(n_items);
    w.emit_off = c.take<uint32_t>(n_items + 1);
    w.pk0 = c.take<uint32_t>(capacity);
    w.pk1 = c.take<uint32_t>(capacity);
    w.psrc = c.take<uint2>(capacity);
    w.psrc2 = c.take<uint2>(capacity);
    w.tk0 = c.take<uint32_t>(n_tiles);
    w.tv0 = c.take<uint32_t>(n_tiles);
    w.tk1 = c.take<uint32_t>(n_tiles);
    w.tv1 = c.take<uint32_t>(n_tiles);
    w.wa = c.take<uint64_t>(onesweep_words(m));
    w.wb = c.take<uint64_t>(onesweep_words(m));
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
    int32_t* err = (int32_t*)(w.misc + 3);  // GS_ERR_TIMEOUT from a look-back wait
    cudaMemsetAsync(out->range, 0, sizeof(uint32_t) * 2 * n_tiles_total, s);
    cudaMemsetAsync(w.misc, 0, 8 * sizeof(uint32_t), s);
    if (n_items == 0) {
        k_pair_count<<<1, 1, 0, s>>>(p_total, out->capacity, out->count, n_eff, out->status, err);
        count_launch();
        GS_CUDA_CHECK_LAUNCH();
        return GS_OK;
    }
    cudaMemsetAsync(w.zero_base, 0, w.zero_bytes, s);
    const int64_t scan_tiles = ceil_div(n_items > n_tiles_total ? n_items : n_tiles_total, kScanTile);
    // 1. compact visible items (in item order) with their depth keys
    scan_single(LoadVisible{p->n_tiles}, nullptr, n_items, nullptr, n_vis, &w.scan_ctl[0], w.scan_words, err, s,
                CompactVisible{p->n_tiles, (const float4*)p->rgb_depth, w.vk0, w.vv0});
    // 2. stable sort of visible items by depth bits
    const bool in1 = onesweep_sort_pairs<uint32_t>(w.vk0, w.vv0, w.vk1, w.vv1, w.vv0, n_items, n_vis, 32,
                                                   &w.sort_ctl[0], w.wa, w.wb, err, s);
    const uint32_t* sorted_item = in1 ? w.vv1 : w.vv0;
    // 3. pair positions in depth order; pair count; emission slots in item order (each item's pairs
    //    occupy offset[item] .. offset[item] + n_tiles - 1, so the adjoint's per-item runs of the
    //    Gaussians of one view are adjacent)
    scan_single(LoadGatherTiles{p->n_tiles, sorted_item}, w.emit_off, n_items, n_vis, p_total, &w.scan_ctl[1],
                w.scan_words + scan_tiles, err, s);
    scan_single(LoadTiles{p->n_tiles}, out->offset, n_items, nullptr, nullptr, &w.scan_ctl[2],
                w.scan_words + 2 * scan_tiles, err, s);
    k_pair_count<<<1, 1, 0, s>>>(p_total, out->capacity, out->count, n_eff, out->status, err);
    count_launch();
    // 4. duplicate: one (tile, emission slot) pair per tile of each visible item's rect
    k_duplicate<<<(unsigned)ceil_div(n_items, 256), 256, 0, s>>>(sorted_item, w.emit_off, n_vis,
                                                                 (const ushort4*)p->rect, n, *f, out->capacity,
                                                                 out->offset, w.pk0, w.psrc);
    count_launch();
    // 5. stable sort by global tile index carrying each pair's (item, emission slot), the last pass
    //    writing them to src / emit; 6. tile ranges
    if (out->capacity > 0) {
        const bool pin1 = onesweep_sort_pairs<uint2>(w.pk0, w.psrc, w.pk1, w.psrc2, w.psrc, out->capacity, n_eff,
                                                     bits_for(n_tiles_total), &w.sort_ctl[1], w.wa, w.wb, err, s,
                                                     out->src, out->emit);
        const int64_t rg = ceil_div(out->capacity, 256);
        k_tile_ranges<<<(unsigned)(rg < 152 * 8 ? rg : 152 * 8), 256, 0, s>>>(pin1 ? w.pk1 : w.pk0, n_eff, out->range,
                                                                             err, out->status);
        count_launch();
    }
    // 7. optional work order for the persistent render schedule
    if (out->order && n_tiles_total > 0) {
        k_tile_order_keys<<<(unsigned)ceil_div(n_tiles_total, 256), 256, 0, s>>>(out->range, n_tiles_total, w.tk0,
                                                                                  w.tv0);
        count_launch();
        const bool t1 = onesweep_sort_pairs<uint32_t>(w.tk0, w.tv0, w.tk1, w.tv1, w.tv0, n_tiles_total, nullptr, 16,
                                                      &w.sort_ctl[2], w.wa, w.wb, err, s);
        k_copy_u32<<<(unsigned)ceil_div(n_tiles_total, 256), 256, 0, s>>>(t1 ? w.tv1 : w.tv0, out->order,
                                                                           n_tiles_total, err, out->status);
        count_launch();
    }
    GS_CUDA_CHECK_LAUNCH();
    return GS_OK;
}
