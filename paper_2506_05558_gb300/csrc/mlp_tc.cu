// Tensor-core path (sm_100-family tcgen05) of the MLP's "TN" GEMM:
// C[m][n] = sum_k A[m][k] B[n][k], bf16 operands (K-major), FP32 accumulator
// in tensor memory.
//
// One CTA (4 warps) computes a 128 x Nt tile (Nt = N rounded up to 16, at most
// 256) of one K split. Per 64-wide K stage all threads copy the A (128 x 64)
// and B (Nt x 64) tiles into shared memory in the canonical no-swizzle K-major
// layout (8-row x 16-byte core matrices, K-adjacent cores 128 B apart, 8-row
// groups 1024 B apart), fence the async proxy, and one elected thread issues
// four tcgen05.mma (K = 16 each) into the TMEM accumulator and commits them to
// an mbarrier. The epilogue reads the accumulator back with tcgen05.ld (each
// warp its 32 TMEM lanes) and stores FP32 rows. Every wait on the mbarrier is
// bounded; on timeout the kernel records an error code, frees its TMEM and
// returns.
#include <cuda_bf16.h>

#include "common.cuh"

namespace gs {

constexpr int kTcM = 128;
constexpr int kTcBK = 64;
constexpr int kTcMaxN = 256;
constexpr uint32_t kTcSpinLimit = 1u << 22;

__device__ int g_tc_error;  // 0 = ok, otherwise the line of the failing wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading (K) and
// stride (M/N) byte offsets in 16-byte units, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: D f32, A and B bf16, both K-major, N, M.
__host__ __device__ constexpr uint32_t instr_desc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__global__ void __launch_bounds__(128) k_gemm_tn_tc(const __nv_bfloat16* __restrict__ A, int64_t lda,
                                                    const __nv_bfloat16* __restrict__ B, int64_t ldb,
                                                    float* __restrict__ C, int64_t ldc, int64_t M, int N, int Nt,
                                                    int64_t K, int64_t k_per_split, int64_t c_split_stride,
                                                    uint32_t tmem_cols) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    uint8_t* sA = smem;  // two buffers of A (128 x 64 bf16) followed by B (Nt x 64 bf16)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t m0 = (int64_t)blockIdx.x * kTcM;
    const int64_t kb = (int64_t)blockIdx.z * k_per_split;
    const int64_t ke = min(K, kb + k_per_split);
    const uint32_t bar = smem_u32(&s_bar);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        s_fail = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = s_tmem;
    const uint32_t idesc = instr_desc_bf16(kTcM, Nt);
    uint32_t phase = 0;
    bool first = true;
    const int rows_total = kTcM + Nt;
    const uint32_t buf_bytes = (uint32_t)rows_total * kTcBK * 2;
    // stage k0 into buffer b: 16-byte cp.async copies (zero-filled outside the matrix), one commit group
    auto issue_stage = [&](int64_t k0, int b) {
        uint8_t* sAb = sA + b * buf_bytes;
        uint8_t* sBb = sAb + kTcM * kTcBK * 2;
        for (int i = tid; i < rows_total * (kTcBK / 8); i += 128) {
            const int r = i / (kTcBK / 8), kc = i % (kTcBK / 8);
            const bool isA = r < kTcM;
            const int rr = isA ? r : r - kTcM;
            const int64_t grow = isA ? m0 + rr : rr;
            const int64_t gk = k0 + kc * 8;
            const bool row_ok = isA ? grow < M : grow < N;
            uint8_t* dst = (isA ? sAb : sBb) + (uint32_t)(((rr >> 3) * (kTcBK / 8) + kc) * 128 + (rr & 7) * 16);
            if (row_ok && gk < ke && gk + 8 > ke) {  // a K tail inside the chunk: element by element
                __nv_bfloat16 tmp[8];
                const __nv_bfloat16* src = (isA ? A + grow * lda : B + grow * ldb);
                for (int e = 0; e < 8; e++) tmp[e] = (gk + e < ke) ? src[gk + e] : __float2bfloat16_rn(0.f);
                *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<uint4*>(tmp);
                continue;
            }
            const bool ok = row_ok && gk + 8 <= ke;
            const __nv_bfloat16* src = ok ? (isA ? A + grow * lda : B + grow * ldb) + gk : A;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
                         "r"(ok ? 16 : 0)
                         : "memory");
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };

    // double-buffered: the copies of slice s + 1 are in flight while slice s is
    // waited for and multiplied; a buffer is refilled only after the MMA that
    // read it has completed (the mbarrier wait at the end of its iteration)
    if (kb < ke) issue_stage(kb, 0);
    int buf = 0;
    for (int64_t k0 = kb; k0 < ke; k0 += kTcBK) {
        const bool more = k0 + kTcBK < ke;
        if (more) issue_stage(k0 + kTcBK, buf ^ 1);
        if (more) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        else asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t a0 = smem_u32(sA + buf * buf_bytes), b0 = a0 + kTcM * kTcBK * 2;
#pragma unroll
            for (int s = 0; s < kTcBK / 16; s++) {
                const uint64_t ad = smem_desc(a0 + s * 256, 128, 1024);
                const uint64_t bd = smem_desc(b0 + s * 256, 128, 1024);
                const uint32_t acc = (first && s == 0) ? 0u : 1u;
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                         : "memory");
            uint32_t spins = 0;
            while (!mbar_try_wait(bar, phase)) {
                if (++spins > kTcSpinLimit) {
                    s_fail = 1;
                    break;
                }
            }
        }
        first = false;
        phase ^= 1u;
        buf ^= 1;
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (s_fail) {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");  // no copy may land after the exit
            break;
        }
    }

    if (!s_fail && !first) {
        // epilogue: warp w reads TMEM lanes 32w..32w+31 (rows of the tile), 16 columns at a time
        const int64_t row = m0 + 32 * warp + lane;
        float* Cz = C + (int64_t)blockIdx.z * c_split_stride;
        for (int c0 = 0; c0 < Nt; c0 += 16) {
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];\n"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            if (row < M && c0 < N) {  // N and ldc are multiples of 16: whole 16-column groups, 128-bit stores
                float4* dst = reinterpret_cast<float4*>(Cz + row * ldc + c0);
#pragma unroll
                for (int j = 0; j < 4; j++)
                    dst[j] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                         __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
            }
        }
    } else if (s_fail && tid == 0) {
        atomicCAS(&g_tc_error, 0, __LINE__);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tmem_cols) : "memory");
    }
}

int gemm_tn_tc(const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* B, int64_t ldb, float* C, int64_t ldc,
               int64_t M, int N, int64_t K, int64_t k_per_split, int64_t c_split_stride, cudaStream_t s) {
    const int Nt = (int)ceil_div(N, 16) * 16;
    if (Nt > kTcMaxN || M <= 0 || K <= 0) return GS_ERR_INVALID_ARG;
    uint32_t cols = 32;
    while (cols < (uint32_t)Nt) cols <<= 1;
    const size_t smem = 2 * (size_t)(kTcM + Nt) * kTcBK * 2;  // two stages
    static bool attr_set = false;
    if (!attr_set) {
        // at most ~115 KB of the SM's shared memory per CTA so that at most two
        // CTAs (2 x 256 TMEM columns) share an SM
        cudaFuncSetAttribute(k_gemm_tn_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
        attr_set = true;
    }
    const size_t smem_launch = smem < 80 * 1024 ? 80 * 1024 : smem;
    const int64_t splits = ceil_div(K, k_per_split);
    dim3 grid((unsigned)ceil_div(M, kTcM), 1, (unsigned)splits);
    k_gemm_tn_tc<<<grid, 128, smem_launch, s>>>(A, lda, B, ldb, C, ldc, M, N, Nt, K, k_per_split, c_split_stride,
                                                 cols);
    count_launch();
    return GS_OK;
}

}  // namespace gs

extern "C" int gs_mlp_tc_error(int32_t* out) {
    if (!out) return GS_ERR_INVALID_ARG;
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, gs::g_tc_error, sizeof(int)) != cudaSuccess) {
        (void)cudaGetLastError();
        return GS_ERR_CUDA;
    }
    *out = v;
    return GS_OK;
}

namespace gs {

// ---------------------------------------------------------------------------
// Fused inference of the whole MLP on tensor cores (tcgen05).
//
// Persistent CTAs of 256 threads, one per SM (about 206 KB of shared memory):
// each converts the four weight matrices to bfloat16 once, in the canonical
// no-swizzle K-major layout (K-adjacent 8x16-byte core matrices 128 B apart,
// 8-row groups (K/8) * 128 B apart), then walks 128-patch tiles. Per tile the
// threads gather the patch features straight from the image into the same
// layout (X, 128 x 208), and for each layer one elected thread issues the
// K/16 tcgen05.mma (M = 128 patches, N = 128 or 16, bf16 in, FP32 in a
// 128-column TMEM accumulator) and commits them to an mbarrier; the eight
// warps then read the accumulator back (warps w and w + 4 share TMEM lane
// quarter w % 4 and split the columns), add the bias, apply GELU and write the
// bf16 activations over the previous layer's buffer (that product has
// completed) as the next layer's A operand. The last layer writes (logit,
// depth, log-scale) in FP32. Every mbarrier wait is bounded; on timeout the
// kernel records the failing line in g_tc_error, frees its TMEM and returns.
// ---------------------------------------------------------------------------
constexpr int kFM = 128, kFIn = 194, kFInPad = 208, kFHid = 128, kFOut = 3, kFOutPad = 16;
constexpr int kFThreads = 256;
constexpr uint32_t kFOffW1 = 0;
constexpr uint32_t kFOffW2 = kFOffW1 + kFHid * kFInPad * 2;     // 53248
constexpr uint32_t kFOffW3 = kFOffW2 + kFHid * kFHid * 2;       // 86016
constexpr uint32_t kFOffW4 = kFOffW3 + kFHid * kFHid * 2;       // 118784
constexpr uint32_t kFOffX = kFOffW4 + kFOutPad * kFHid * 2;     // 122880
constexpr uint32_t kFOffH = kFOffX + kFM * kFInPad * 2;         // 176128
constexpr uint32_t kFOffB = kFOffH + kFM * kFHid * 2;           // 208896: biases, FP32
constexpr uint32_t kFSmem = kFOffB + (3 * kFHid + kFOutPad) * 4;

// Byte offset of element (r, k) of a K-major [rows][K] bf16 matrix, K % 8 == 0.
__device__ __forceinline__ uint32_t kmajor_off(int r, int k, int K) {
    return (uint32_t)((((r >> 3) * (K >> 3) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ uint4 pack8_bf16(const float* v) {
    uint4 u;
    uint32_t* w = reinterpret_cast<uint32_t*>(&u);
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        w[i] = *reinterpret_cast<const uint32_t*>(&h);
    }
    return u;
}

// Element j (0..7) of eight packed bfloat16 values (j a compile-time constant in
// unrolled loops, so the value stays in registers).
__device__ __forceinline__ __nv_bfloat16 bf16_at(const uint4& u, int j) {
    const uint32_t w = j < 2 ? u.x : j < 4 ? u.y : j < 6 ? u.z : u.w;
    return __ushort_as_bfloat16((unsigned short)((j & 1) ? (w >> 16) : (w & 0xFFFFu)));
}

__device__ __forceinline__ float gelu_erf(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }

// W [rows_valid][cols_valid] FP32 (nn.Linear layout) -> bf16 [rows][K] K-major at dst, zero padded.
__device__ void stage_weight(const float* __restrict__ Wm, int rows_valid, int cols_valid, int rows, int K,
                             uint8_t* dst) {
    const int chunks = rows * (K >> 3);
    for (int q = threadIdx.x; q < chunks; q += blockDim.x) {
        const int r = q / (K >> 3), kc = q % (K >> 3);
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; e++) {
            const int k = kc * 8 + e;
            v[e] = (r < rows_valid && k < cols_valid) ? Wm[(int64_t)r * cols_valid + k] : 0.f;
        }
        *reinterpret_cast<uint4*>(dst + kmajor_off(r, kc * 8, K)) = pack8_bf16(v);
    }
}

// What the training step's backward needs from the forward, written by the
// TRAIN instantiation in the layouts of the GEMM-chain forward: the features
// transposed (Xt [208][Mp], bf16), the pre-activations with their bias (Z[l]
// [Mp][128] FP32, l < 3) and the activations transposed (Ht[l] [128][Mp], bf16),
// and the output layer before its bias (Z3 [Mp][16] FP32); rows up to Mp.
struct TrainFwdOut {
    __nv_bfloat16* Xt;
    float* Z[3];
    __nv_bfloat16* Ht[3];
    float* Z3;
    int64_t Mp;
};

template <bool TRAIN>
__global__ void __launch_bounds__(kFThreads, 1) k_mlp_forward_tc(
    const float* __restrict__ image, int W, int H, const float* __restrict__ w1, const float* __restrict__ b1,
    const float* __restrict__ w2, const float* __restrict__ b2, const float* __restrict__ w3,
    const float* __restrict__ b3, const float* __restrict__ w4, const float* __restrict__ b4,
    float* __restrict__ out, TrainFwdOut to) {
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nx = W >> 3, ny = H >> 3;
    const int64_t M = (int64_t)nx * ny;
    const int64_t n_tiles = TRAIN ? to.Mp / kFM : (M + kFM - 1) / kFM;
    const uint32_t bar = smem_u32(&s_bar);
    float* s_b = reinterpret_cast<float*>(sm + kFOffB);  // b1 | b2 | b3 | b4 (padded to 16)

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                     "r"(128)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        s_fail = 0;
    }
    stage_weight(w1, kFHid, kFIn, kFHid, kFInPad, sm + kFOffW1);
    stage_weight(w2, kFHid, kFHid, kFHid, kFHid, sm + kFOffW2);
    stage_weight(w3, kFHid, kFHid, kFHid, kFHid, sm + kFOffW3);
    stage_weight(w4, kFOut, kFHid, kFOutPad, kFHid, sm + kFOffW4);
    for (int i = tid; i < 3 * kFHid + kFOutPad; i += kFThreads) {
        const int l = i / kFHid, j = i % kFHid;
        s_b[i] = l == 0 ? b1[j] : l == 1 ? b2[j] : l == 2 ? b3[j] : (j < kFOut ? b4[j] : 0.f);
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = s_tmem;
    const uint32_t sbase = smem_u32(sm);
    uint32_t phase = 0;

    for (int64_t tile = blockIdx.x; tile < n_tiles && !s_fail; tile += gridDim.x) {
        // 1. features: chunk q = (row r, 8-column group kc); a warp covers 32 patches of one group
        const int64_t p0 = tile * kFM;
        for (int q = tid; q < kFM * (kFInPad >> 3); q += kFThreads) {
            const int r = q % kFM, kc = q / kFM;
            const int64_t p = p0 + r;
            float v[8];
            if (p < M) {
                const int py = (int)(p / nx), px = (int)(p % nx);
                if (kc < 24) {  // 3 channels x 8 rows of 8 pixels
                    const int c = kc >> 3, dy = kc & 7;
                    const float4* src =
                        reinterpret_cast<const float4*>(image + ((int64_t)c * H + 8 * py + dy) * W + 8 * px);
                    const float4 a = src[0], b = src[1];
                    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
                } else {
#pragma unroll
                    for (int e = 0; e < 8; e++) v[e] = 0.f;
                    if (kc == 24) {  // patch centre in [-1, 1]^2, x first
                        v[0] = (px + 0.5f) / nx * 2.f - 1.f;
                        v[1] = (py + 0.5f) / ny * 2.f - 1.f;
                    }
                }
            } else {
#pragma unroll
                for (int e = 0; e < 8; e++) v[e] = 0.f;
            }
            const uint4 pk = pack8_bf16(v);
            *reinterpret_cast<uint4*>(sm + kFOffX + kmajor_off(r, kc * 8, kFInPad)) = pk;
            if (TRAIN) {  // X^T: for each of the 8 columns, consecutive threads write consecutive patches
#pragma unroll
                for (int e = 0; e < 8; e++) to.Xt[(int64_t)(kc * 8 + e) * to.Mp + p] = bf16_at(pk, e);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();

        for (int l = 0; l < 4; l++) {
            const int K = l == 0 ? kFInPad : kFHid;
            const int N = l == 3 ? kFOutPad : kFHid;
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t a0 = sbase + (l == 0 ? kFOffX : kFOffH);
                const uint32_t b0 = sbase + (l == 0 ? kFOffW1 : l == 1 ? kFOffW2 : l == 2 ? kFOffW3 : kFOffW4);
                const uint32_t sbo = (uint32_t)(K >> 3) * 128u;
                const uint32_t idesc = instr_desc_bf16(kFM, N);
                for (int s = 0; s < K / 16; s++) {
                    const uint64_t ad = smem_desc(a0 + s * 256, 128, sbo);
                    const uint64_t bd = smem_desc(b0 + s * 256, 128, sbo);
                    const uint32_t acc = s > 0 ? 1u : 0u;
                    asm volatile(
                        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                        : "memory");
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                                 bar)
                             : "memory");
                uint32_t spins = 0;
                while (!mbar_try_wait(bar, phase)) {
                    if (++spins > kTcSpinLimit) {
                        s_fail = __LINE__;
                        break;
                    }
                }
            }
            phase ^= 1u;
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            if (s_fail) break;
            // 2. epilogue: row r of the tile = TMEM lane 32 (warp % 4) + lane
            const int quarter = warp & 3, half = warp >> 2;
            const int r = 32 * quarter + lane;
            const uint32_t trow = tmem + ((uint32_t)(32 * quarter) << 16);
            if (l < 3) {
                for (int c0 = 64 * half; c0 < 64 * half + 64; c0 += 16) {
                    uint32_t u[16];
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
                        "%15}, [%16];\n"
                        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]),
                          "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]),
                          "=r"(u[14]), "=r"(u[15])
                        : "r"(trow + (uint32_t)c0));
                    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                    float v[16];
                    if (TRAIN) {
                        const int64_t p = p0 + r;
                        float zr[16];
#pragma unroll
                        for (int j = 0; j < 16; j++) zr[j] = __uint_as_float(u[j]) + s_b[l * kFHid + c0 + j];
                        float* Zl = l == 0 ? to.Z[0] : l == 1 ? to.Z[1] : to.Z[2];  // no dynamic index into the param
                        float4* zd = reinterpret_cast<float4*>(Zl + p * kFHid + c0);
#pragma unroll
                        for (int j = 0; j < 4; j++) zd[j] = make_float4(zr[4 * j], zr[4 * j + 1], zr[4 * j + 2], zr[4 * j + 3]);
#pragma unroll
                        for (int j = 0; j < 16; j++) v[j] = gelu_erf(zr[j]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; j++) v[j] = gelu_erf(__uint_as_float(u[j]) + s_b[l * kFHid + c0 + j]);
                    }
                    const uint4 h0 = pack8_bf16(v), h1 = pack8_bf16(v + 8);
                    *reinterpret_cast<uint4*>(sm + kFOffH + kmajor_off(r, c0, kFHid)) = h0;
                    *reinterpret_cast<uint4*>(sm + kFOffH + kmajor_off(r, c0 + 8, kFHid)) = h1;
                    if (TRAIN) {  // H^T: per column, the warp's 32 consecutive patches
                        const int64_t p = p0 + r;
                        __nv_bfloat16* Hl = l == 0 ? to.Ht[0] : l == 1 ? to.Ht[1] : to.Ht[2];
#pragma unroll
                        for (int j = 0; j < 8; j++) {
                            Hl[(int64_t)(c0 + j) * to.Mp + p] = bf16_at(h0, j);
                            Hl[(int64_t)(c0 + 8 + j) * to.Mp + p] = bf16_at(h1, j);
                        }
                    }
                }
            } else if (half == 0) {
                uint32_t u[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
                    "%15}, [%16];\n"
                    : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
                      "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]),
                      "=r"(u[15])
                    : "r"(trow));
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                const int64_t p = p0 + r;
                if (TRAIN) {  // the output layer before its bias, all 16 padded columns, every row up to Mp
                    float4* zd = reinterpret_cast<float4*>(to.Z3 + p * kFOutPad);
#pragma unroll
                    for (int j = 0; j < 4; j++)
                        zd[j] = make_float4(__uint_as_float(u[4 * j]), __uint_as_float(u[4 * j + 1]),
                                            __uint_as_float(u[4 * j + 2]), __uint_as_float(u[4 * j + 3]));
                } else if (p < M) {
#pragma unroll
                    for (int j = 0; j < kFOut; j++) out[p * kFOut + j] = __uint_as_float(u[j]) + s_b[3 * kFHid + j];
                }
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncthreads();
        }
    }
    if (s_fail && tid == 0) atomicCAS(&g_tc_error, 0, s_fail);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(128) : "memory");
    }
}

static int fused_sms() {
    static int n_sm = 0;
    if (n_sm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(k_mlp_forward_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFSmem);
        cudaFuncSetAttribute(k_mlp_forward_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFSmem);
    }
    return n_sm > 0 ? n_sm : 1;
}

int mlp_forward_fused(const float* const* w, const float* const* b, const float* image, int W, int H, float* out,
                      cudaStream_t s) {
    const int n_sm = fused_sms();
    const int64_t M = (int64_t)(W / 8) * (H / 8);
    const int64_t n_tiles = (M + kFM - 1) / kFM;
    if (n_tiles == 0) return GS_OK;
    const int grid = (int)(n_tiles < n_sm ? n_tiles : n_sm);
    TrainFwdOut none{};
    k_mlp_forward_tc<false><<<grid, kFThreads, kFSmem, s>>>(image, W, H, w[0], b[0], w[1], b[1], w[2], b[2], w[3],
                                                            b[3], out, none);
    count_launch();
    return GS_OK;
}

// The training step's forward in one launch: as mlp_forward_fused, writing the
// tensors the backward reads (Mp = patches rounded up to a multiple of 128).
int mlp_train_forward_fused(const float* const* w, const float* const* b, const float* image, int W, int H,
                            __nv_bfloat16* Xt, float* const* Z, __nv_bfloat16* const* Ht, float* Z3, int64_t Mp,
                            cudaStream_t s) {
    const int n_sm = fused_sms();
    const int64_t n_tiles = Mp / kFM;
    if (n_tiles == 0) return GS_OK;
    const int grid = (int)(n_tiles < n_sm ? n_tiles : n_sm);
    TrainFwdOut to{Xt, {Z[0], Z[1], Z[2]}, {Ht[0], Ht[1], Ht[2]}, Z3, Mp};
    k_mlp_forward_tc<true><<<grid, kFThreads, kFSmem, s>>>(image, W, H, w[0], b[0], w[1], b[1], w[2], b[2], w[3],
                                                           b[3], nullptr, to);
    count_launch();
    return GS_OK;
}

}  // namespace gs
