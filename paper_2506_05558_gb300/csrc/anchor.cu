// Anchor trigger and offload (Sec. 4.4). A Gaussian's on-screen size seen from
// a camera is S / D with S its largest scale and D the distance of its mean to
// the camera centre; in pixels, fx * S / D. An anchor is due when more than
// 40% of the active Gaussians are smaller than tau_min = 1 px from the
// previous camera; the active set and its optimiser state are then copied to
// host memory.
#include "common.cuh"

namespace gs {

__global__ void __launch_bounds__(256) k_anchor_check(const float4* __restrict__ mean_opa,
                                                      const float4* __restrict__ scale, int64_t n,
                                                      const gs_camera* __restrict__ cam, float tau_px,
                                                      uint8_t* __restrict__ too_fine,
                                                      unsigned long long* __restrict__ count) {
    __shared__ unsigned int s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool fine = false;
    if (g < n) {
        const gs_camera& c = *cam;
        // camera centre = -R^T t
        const float cx = -(c.R[0] * c.t[0] + c.R[3] * c.t[1] + c.R[6] * c.t[2]);
        const float cy = -(c.R[1] * c.t[0] + c.R[4] * c.t[1] + c.R[7] * c.t[2]);
        const float cz = -(c.R[2] * c.t[0] + c.R[5] * c.t[1] + c.R[8] * c.t[2]);
        const float4 mo = mean_opa[g];
        const float4 s4 = scale[g];
        const float dx = mo.x - cx, dy = mo.y - cy, dz = mo.z - cz;
        const float D = sqrtf(dx * dx + dy * dy + dz * dz);
        const float S = expf(fmaxf(s4.x, fmaxf(s4.y, s4.z)));
        fine = c.fx * S < tau_px * D;  // fx S / D < tau, without dividing by D
        too_fine[g] = fine ? 1 : 0;
    }
    // integer counts are order-independent, so the total is exact and reproducible
    const unsigned int b = __popc(__ballot_sync(0xffffffffu, fine));
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(&s_cnt, b);
    __syncthreads();
    if (threadIdx.x == 0 && s_cnt) atomicAdd(count, (unsigned long long)s_cnt);
}

}  // namespace gs

using namespace gs;

extern "C" int gs_anchor_check(const gs_gaussians* g, const gs_camera* cam, float tau_px, uint8_t* too_fine,
                               int64_t* count, void* stream) {
    if (!g || !cam || !too_fine || !count || g->n < 0 || !(tau_px > 0.f)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemsetAsync(count, 0, sizeof(int64_t), s);
    if (g->n > 0) {
        k_anchor_check<<<(unsigned)ceil_div(g->n, 256), 256, 0, s>>>((const float4*)g->mean_opa,
                                                                     (const float4*)g->scale, g->n, cam, tau_px,
                                                                     too_fine, (unsigned long long*)count);
        count_launch();
    }
    GS_CUDA_CHECK_LAUNCH();
    return GS_OK;
}

static int copy_set(const gs_gaussians* dst, const gs_gaussians* src, cudaMemcpyKind kind, cudaStream_t s) {
    if (!dst || !src || dst->n != src->n || src->n < 0) return GS_ERR_INVALID_ARG;
    const size_t n = (size_t)src->n;
    if (n == 0) return GS_OK;
    const struct { float* d; const float* s; size_t bytes; } parts[4] = {
        {dst->mean_opa, src->mean_opa, n * 16}, {dst->scale, src->scale, n * 16},
        {dst->quat, src->quat, n * 16}, {dst->sh, src->sh, n * 192}};
    for (const auto& p : parts) {
        if (!p.d || !p.s) return GS_ERR_INVALID_ARG;
        if (cudaMemcpyAsync(p.d, p.s, p.bytes, kind, s) != cudaSuccess) {
            (void)cudaGetLastError();
            return GS_ERR_CUDA;
        }
    }
    return GS_OK;
}

extern "C" int gs_anchor_offload(const gs_gaussians* params, const gs_gaussians* m, const gs_gaussians* v,
                                 const gs_gaussians* host_params, const gs_gaussians* host_m,
                                 const gs_gaussians* host_v, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    int rc = copy_set(host_params, params, cudaMemcpyDeviceToHost, s);
    if (rc == GS_OK && m && host_m) rc = copy_set(host_m, m, cudaMemcpyDeviceToHost, s);
    if (rc == GS_OK && v && host_v) rc = copy_set(host_v, v, cudaMemcpyDeviceToHost, s);
    return rc;
}

extern "C" int gs_anchor_load(const gs_gaussians* host_params, const gs_gaussians* host_m,
                              const gs_gaussians* host_v, const gs_gaussians* params, const gs_gaussians* m,
                              const gs_gaussians* v, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    int rc = copy_set(params, host_params, cudaMemcpyHostToDevice, s);
    if (rc == GS_OK && m && host_m) rc = copy_set(m, host_m, cudaMemcpyHostToDevice, s);
    if (rc == GS_OK && v && host_v) rc = copy_set(v, host_v, cudaMemcpyHostToDevice, s);
    return rc;
}
