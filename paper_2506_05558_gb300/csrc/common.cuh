// Internal helpers shared by the sm_103a kernels of libgs (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/gs.h"

#define GS_CUDA_CHECK_LAUNCH()                         \
    do {                                               \
        if (cudaPeekAtLastError() != cudaSuccess) {    \
            (void)cudaGetLastError();                  \
            return GS_ERR_CUDA;                        \
        }                                              \
    } while (0)

namespace gs {

constexpr float kLog2e = 1.4426950408889634f;
constexpr int kWarp = 32;

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Global tile index -> view (binary search over the frame's tile bases).
__device__ __forceinline__ int view_of_tile(const gs_frame& f, int tile) {
    int lo = 0, hi = f.n_views - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (f.tile_base[mid] <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// 2^x on the MUFU unit (PTX ex2.approx, flush-to-zero for denormals).
__device__ __forceinline__ float fast_exp2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Hardware reciprocal approximation (MUFU), for x away from 0 and infinity.
__device__ __forceinline__ float fast_rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Philox4x32-10 (Salmon et al., SC'11).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; r++) {
        const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += W0;
        k.y += W1;
    }
    return c;
}

// Uniform in [0, 1) from the top 24 bits of a Philox output word.
__device__ __forceinline__ float philox_u24(uint32_t x) { return (float)(x >> 8) * (1.f / 16777216.f); }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Host-side count of kernels this library has launched (diagnostics).
void count_launch();

// Bytes rounded up to 256 so carved sub-buffers stay aligned.
__host__ __device__ inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Bump allocator over a caller-owned scratch buffer.
struct Carve {
    char* base;
    size_t used;
    size_t cap;
    template <class T>
    T* take(size_t count) {
        size_t b = align256(count * sizeof(T));
        T* p = reinterpret_cast<T*>(base ? base + used : nullptr);
        used += b;
        return p;
    }
    bool ok() const { return used <= cap; }
};

// Scratch bytes of the device-wide scan for up to n_max inputs.
size_t scan_workspace_bytes(int64_t n_max);

// Device-wide exclusive scan of n uint32 values; total (device) gets the sum.
void scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total, void* ws, cudaStream_t s);

// Stable LSD radix sort of (uint32 key, uint32 value) pairs on key bits
// [0, bits), 8 bits per pass. The pair count is min(n_max, *n_dev). Buffers
// (ka, va) hold the input; (kb, vb) are the alternates. With va_is_position
// the input values are taken to be 0, 1, 2, ... and va is not read (it is
// still needed as the alternate buffer). Returns true when the sorted result
// ends in (kb, vb). hist: 256 * radix_blocks(n_max) uint32.
int64_t radix_blocks(int64_t n_max);
bool radix_sort_pairs(uint32_t* ka, uint32_t* va, uint32_t* kb, uint32_t* vb, int64_t n_max,
                      const uint32_t* n_dev, int bits, uint32_t* hist, void* scan_ws, cudaStream_t s,
                      bool va_is_position);

// Persistent grid: as many CTAs as fit at once on all SMs. The occupancy query
// runs once per (device, kernel) so later calls, e.g. inside a stream capture,
// make no runtime queries. The cache is shared by all host threads (locked).
inline int persistent_grid(const void* fn, int threads) {
    struct Entry { const void* fn; int dev; int grid; };
    static Entry cache[64];
    static int n_cache = 0;
    static std::mutex lock;
    std::lock_guard<std::mutex> guard(lock);
    int dev = 0;
    cudaGetDevice(&dev);
    for (int i = 0; i < n_cache; i++)
        if (cache[i].fn == fn && cache[i].dev == dev) return cache[i].grid;
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0);
    const int grid = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    if (n_cache < 64) cache[n_cache++] = {fn, dev, grid};
    return grid;
}

}  // namespace gs
