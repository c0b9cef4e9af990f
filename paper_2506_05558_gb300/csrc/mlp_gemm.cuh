// "TN" GEMM for the learned-proposal MLP: C[m][n] = sum_k A[m][k] B[n][k] with
// A [M][lda] and B [N][ldb] bfloat16, K-major, FP32 accumulation and output.
// With k_per_split < K the product is split over K: split z covers
// [z k_per_split, (z+1) k_per_split) and writes C + z * c_split_stride.
//
// Path 0: warp-level mma.sync m16n8k16 (bf16 in, f32 accumulate) on 64x64
// tiles staged in shared memory. Path 1: tcgen05.mma with the accumulator in
// tensor memory (mlp_tc.cuh).
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace gs {

constexpr int kGM = 64, kGN = 64, kGK = 32, kGPad = 8;

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                               uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Loads a ROWS x kGK bf16 tile (rows r0.., columns k0..k0+kGK) into shared
// memory, zero outside [0, nrows) x [k0, kend).
template <int ROWS>
__device__ __forceinline__ void load_tile(const __nv_bfloat16* __restrict__ src, int64_t ld, int r0, int nrows,
                                          int k0, int kend, __nv_bfloat16 (*dst)[kGK + kGPad]) {
    for (int i = threadIdx.x; i < ROWS * (kGK / 8); i += blockDim.x) {
        const int r = i / (kGK / 8), c8 = (i % (kGK / 8)) * 8;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        const int gr = r0 + r, gk = k0 + c8;
        if (gr < nrows && gk + 8 <= kend) {
            v = *reinterpret_cast<const uint4*>(src + (int64_t)gr * ld + gk);
        } else if (gr < nrows) {
            __nv_bfloat16 tmp[8];
            for (int e = 0; e < 8; e++) tmp[e] = (gk + e < kend) ? src[(int64_t)gr * ld + gk + e] : __float2bfloat16_rn(0.f);
            v = *reinterpret_cast<uint4*>(tmp);
        }
        *reinterpret_cast<uint4*>(&dst[r][c8]) = v;
    }
}

__global__ void __launch_bounds__(128) k_gemm_tn_mma(const __nv_bfloat16* __restrict__ A, int64_t lda,
                                                     const __nv_bfloat16* __restrict__ B, int64_t ldb,
                                                     float* __restrict__ C, int64_t ldc, int M, int N, int K,
                                                     int k_per_split, int64_t c_split_stride) {
    __shared__ __align__(16) __nv_bfloat16 sA[kGM][kGK + kGPad];
    __shared__ __align__(16) __nv_bfloat16 sB[kGN][kGK + kGPad];
    const int m0 = blockIdx.x * kGM, n0 = blockIdx.y * kGN;
    const int kb = blockIdx.z * k_per_split;
    const int ke = min(K, kb + k_per_split);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; i++) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
    for (int k0 = kb; k0 < ke; k0 += kGK) {
        load_tile<kGM>(A, lda, m0, M, k0, ke, sA);
        load_tile<kGN>(B, ldb, n0, N, k0, ke, sB);
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kGK; kk += 16) {
            const int ar = warp * 16;
            const uint32_t a0 = *reinterpret_cast<const uint32_t*>(&sA[ar + g][kk + 2 * t]);
            const uint32_t a1 = *reinterpret_cast<const uint32_t*>(&sA[ar + g + 8][kk + 2 * t]);
            const uint32_t a2 = *reinterpret_cast<const uint32_t*>(&sA[ar + g][kk + 2 * t + 8]);
            const uint32_t a3 = *reinterpret_cast<const uint32_t*>(&sA[ar + g + 8][kk + 2 * t + 8]);
#pragma unroll
            for (int nt = 0; nt < 8; nt++) {
                const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&sB[nt * 8 + g][kk + 2 * t]);
                const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&sB[nt * 8 + g][kk + 2 * t + 8]);
                mma_bf16_16816(acc[nt], a0, a1, a2, a3, b0, b1);
            }
        }
        __syncthreads();
    }
    float* Cz = C + (int64_t)blockIdx.z * c_split_stride;
    const int r_lo = m0 + warp * 16 + g, r_hi = r_lo + 8;
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
        const int c = n0 + nt * 8 + 2 * t;
        if (r_lo < M) {
            if (c < N) Cz[(int64_t)r_lo * ldc + c] = acc[nt][0];
            if (c + 1 < N) Cz[(int64_t)r_lo * ldc + c + 1] = acc[nt][1];
        }
        if (r_hi < M) {
            if (c < N) Cz[(int64_t)r_hi * ldc + c] = acc[nt][2];
            if (c + 1 < N) Cz[(int64_t)r_hi * ldc + c + 1] = acc[nt][3];
        }
    }
}

int gemm_tn_tc(const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* B, int64_t ldb, float* C, int64_t ldc,
               int64_t M, int N, int64_t K, int64_t k_per_split, int64_t c_split_stride, cudaStream_t s);

inline int gemm_tn(int path, const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* B, int64_t ldb, float* C,
                   int64_t ldc, int64_t M, int N, int64_t K, int64_t k_per_split, int64_t c_split_stride,
                   cudaStream_t s) {
    if (k_per_split <= 0 || k_per_split > K) k_per_split = K;
    if (path == 1) return gemm_tn_tc(A, lda, B, ldb, C, ldc, M, N, K, k_per_split, c_split_stride, s);
    const int64_t splits = ceil_div(K, k_per_split);
    dim3 grid((unsigned)ceil_div(M, kGM), (unsigned)ceil_div(N, kGN), (unsigned)splits);
    k_gemm_tn_mma<<<grid, 128, 0, s>>>(A, lda, B, ldb, C, ldc, (int)M, N, (int)K, (int)k_per_split, c_split_stride);
    count_launch();
    return GS_OK;
}

}  // namespace gs
