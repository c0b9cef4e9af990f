// Throughput probes of the two SM units the compositing kernels use: the FP32
// FMA pipe and the MUFU (special function) pipe. They do no part of the
// method; they measure the peaks against which the compositing kernels'
// evaluations are reported, on the GPU and at the clock at hand.
#include "common.cuh"

namespace gs {

// Each thread runs 8 independent FMA chains, 16 rounds unrolled per loop trip
// (128 FMAs per trip), so the issue slots go almost entirely to FFMA.
__global__ void __launch_bounds__(256) k_probe_fma(float* __restrict__ out, int iters, float a, float b) {
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; j++) x[j] = 1e-3f * (float)threadIdx.x + (float)j;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int r = 0; r < 16; r++)
#pragma unroll
            for (int j = 0; j < 8; j++) x[j] = __fmaf_rn(x[j], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; j++) s += x[j];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// 8 independent chains alternating 2^x and 1/x (both MUFU), 8 steps per chain
// per loop trip (64 MUFU operations); the values stay within [0.5, 2].
__global__ void __launch_bounds__(256) k_probe_mufu(float* __restrict__ out, int iters) {
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; j++) x[j] = 0.5f + 0.01f * (float)j + 1e-5f * (float)threadIdx.x;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
            for (int j = 0; j < 8; j++) x[j] = fast_rcp(fast_exp2(x[j]));
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; j++) s += x[j];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace gs

using namespace gs;

extern "C" int gs_probe_fma(float* out, int32_t blocks, int32_t iters, void* stream) {
    if (!out || blocks < 1 || iters < 1) return GS_ERR_INVALID_ARG;
    k_probe_fma<<<blocks, 256, 0, (cudaStream_t)stream>>>(out, iters, 0.9999999f, 1e-7f);
    count_launch();
    GS_CUDA_CHECK_LAUNCH();
    return GS_OK;
}

extern "C" int gs_probe_mufu(float* out, int32_t blocks, int32_t iters, void* stream) {
    if (!out || blocks < 1 || iters < 1) return GS_ERR_INVALID_ARG;
    k_probe_mufu<<<blocks, 256, 0, (cudaStream_t)stream>>>(out, iters);
    count_launch();
    GS_CUDA_CHECK_LAUNCH();
    return GS_OK;
}
