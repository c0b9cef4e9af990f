// Optimiser step of the joint optimisation (Sec. 4.3): sparse Adam over the
// Gaussians visible in the step's views, Adam + SE(3) retraction for the
// camera poses, and the L1 photometric loss with its gradient.
#include "common.cuh"

namespace gs {

// One thread per 16-byte parameter row. Rows are laid out segment by segment
// (mean_opa | scale | quat | sh) so every warp reads contiguous memory.
__global__ void __launch_bounds__(256) k_adam(float4* __restrict__ p_mo, float4* __restrict__ p_sc,
                                              float4* __restrict__ p_q, float4* __restrict__ p_sh,
                                              const float4* __restrict__ g_mo, const float4* __restrict__ g_sc,
                                              const float4* __restrict__ g_q, const float4* __restrict__ g_sh,
                                              float4* __restrict__ m_mo, float4* __restrict__ m_sc,
                                              float4* __restrict__ m_q, float4* __restrict__ m_sh,
                                              float4* __restrict__ v_mo, float4* __restrict__ v_sc,
                                              float4* __restrict__ v_q, float4* __restrict__ v_sh,
                                              const uint8_t* __restrict__ visible, int64_t n, gs_adam_config c,
                                              float bc1, float bc2, const int32_t* __restrict__ step_dev,
                                              const float* __restrict__ lr_scale) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 15 * n) return;
    if (step_dev) {  // bias corrections of the step number held on the device
        const float t = (float)*step_dev;
        bc1 = 1.f - powf(c.beta1, t);
        bc2 = 1.f - powf(c.beta2, t);
    }
    int64_t g, row;
    float4 *P, *M, *V;
    const float4* G;
    float4 lr;
    if (i < n) {
        g = i; row = i; P = p_mo; G = g_mo; M = m_mo; V = v_mo;
        lr = make_float4(c.lr_mean, c.lr_mean, c.lr_mean, c.lr_opacity);
    } else if (i < 2 * n) {
        g = i - n; row = g; P = p_sc; G = g_sc; M = m_sc; V = v_sc;
        lr = make_float4(c.lr_scale, c.lr_scale, c.lr_scale, 0.f);
    } else if (i < 3 * n) {
        g = i - 2 * n; row = g; P = p_q; G = g_q; M = m_q; V = v_q;
        lr = make_float4(c.lr_rot, c.lr_rot, c.lr_rot, c.lr_rot);
    } else {
        row = i - 3 * n; g = row / 12; P = p_sh; G = g_sh; M = m_sh; V = v_sh;
        lr = (row % 12 == 0) ? make_float4(c.lr_sh_dc, c.lr_sh_dc, c.lr_sh_dc, c.lr_sh_rest)
                             : make_float4(c.lr_sh_rest, c.lr_sh_rest, c.lr_sh_rest, c.lr_sh_rest);
    }
    if (!visible[g]) return;
    if (lr_scale) {
        const float ls = lr_scale[g];
        lr.x *= ls; lr.y *= ls; lr.z *= ls; lr.w *= ls;
    }
    float4 p = P[row], gr = G[row], m = M[row], v = V[row];
    float* pp = &p.x;
    float* gg = &gr.x;
    float* mm = &m.x;
    float* vv = &v.x;
    const float* ll = &lr.x;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        mm[k] = c.beta1 * mm[k] + (1.f - c.beta1) * gg[k];
        vv[k] = c.beta2 * vv[k] + (1.f - c.beta2) * gg[k] * gg[k];
        pp[k] -= ll[k] * (mm[k] / bc1) / (sqrtf(vv[k] / bc2) + c.eps);
    }
    P[row] = p;
    M[row] = m;
    V[row] = v;
}

// One thread per view: Adam on the 6-vector, then T_cw <- exp(delta^) T_cw.
__global__ void k_pose_step(gs_camera* cams, int nv, const float* __restrict__ grad, float* m, float* v, float lr_t,
                            float lr_r, float b1, float b2, float eps, float bc1, float bc2,
                            const int32_t* __restrict__ step_dev) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    if (step_dev) {
        const float t = (float)*step_dev;
        bc1 = 1.f - powf(b1, t);
        bc2 = 1.f - powf(b2, t);
    }
    float d[6];
    for (int k = 0; k < 6; k++) {
        const float g = grad[6 * i + k];
        const float mk = b1 * m[6 * i + k] + (1.f - b1) * g;
        const float vk = b2 * v[6 * i + k] + (1.f - b2) * g * g;
        m[6 * i + k] = mk;
        v[6 * i + k] = vk;
        d[k] = -(k < 3 ? lr_t : lr_r) * (mk / bc1) / (sqrtf(vk / bc2) + eps);
    }
    // exp of (rho, phi): R = I + A K + B K^2, t = (I + B K + C K^2) rho with
    // A = sin(th)/th, B = (1 - cos th)/th^2, C = (th - sin th)/th^3
    const float wx = d[3], wy = d[4], wz = d[5];
    const float th2 = wx * wx + wy * wy + wz * wz;
    const float th = sqrtf(th2);
    float A, B, C;
    if (th < 1e-4f) {
        A = 1.f - th2 / 6.f;
        B = 0.5f - th2 / 24.f;
        C = 1.f / 6.f - th2 / 120.f;
    } else {
        A = sinf(th) / th;
        B = (1.f - cosf(th)) / th2;
        C = (th - sinf(th)) / (th2 * th);
    }
    const float K[9] = {0.f, -wz, wy, wz, 0.f, -wx, -wy, wx, 0.f};
    float K2[9];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) K2[3 * r + c] = K[3 * r] * K[c] + K[3 * r + 1] * K[3 + c] + K[3 * r + 2] * K[6 + c];
    float dR[9], Vm[9];
    for (int k = 0; k < 9; k++) {
        const float I = (k % 4 == 0) ? 1.f : 0.f;
        dR[k] = I + A * K[k] + B * K2[k];
        Vm[k] = I + B * K[k] + C * K2[k];
    }
    gs_camera& cam = cams[i];
    float R[9], t[3];
    for (int k = 0; k < 9; k++) R[k] = cam.R[k];
    for (int k = 0; k < 3; k++) t[k] = cam.t[k];
    for (int r = 0; r < 3; r++) {
        for (int c = 0; c < 3; c++) cam.R[3 * r + c] = dR[3 * r] * R[c] + dR[3 * r + 1] * R[3 + c] + dR[3 * r + 2] * R[6 + c];
        cam.t[r] = dR[3 * r] * t[0] + dR[3 * r + 1] * t[1] + dR[3 * r + 2] * t[2] + Vm[3 * r] * d[0] +
                   Vm[3 * r + 1] * d[1] + Vm[3 * r + 2] * d[2];
    }
}

constexpr int kLossThreads = 256;
constexpr int kLossMaxBlocks = 4096;

__global__ void __launch_bounds__(kLossThreads) k_l1(const float4* __restrict__ c4, const float4* __restrict__ t4,
                                                     float4* __restrict__ g4, int64_t n4, const float* __restrict__ c,
                                                     const float* __restrict__ t, float* __restrict__ gd, int64_t n,
                                                     float inv_n, float* __restrict__ partial) {
    __shared__ float s[kLossThreads / 32];
    float acc = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const float4 a = c4[i], b = t4[i];
        const float d0 = a.x - b.x, d1 = a.y - b.y, d2 = a.z - b.z, d3 = a.w - b.w;
        acc += fabsf(d0) + fabsf(d1) + fabsf(d2) + fabsf(d3);
        auto sg = [](float x) { return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f); };
        g4[i] = make_float4(sg(d0) * inv_n, sg(d1) * inv_n, sg(d2) * inv_n, sg(d3) * inv_n);
    }
    // scalar tail
    for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float d = c[i] - t[i];
        acc += fabsf(d);
        gd[i] = (d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f)) * inv_n;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float b = 0.f;
        for (int k = 0; k < kLossThreads / 32; k++) b += s[k];
        partial[blockIdx.x] = b;
    }
}

__global__ void __launch_bounds__(1024) k_l1_final(const float* __restrict__ partial, int nb, float inv_n,
                                                   float* __restrict__ loss) {
    __shared__ float s[1024];
    float a = 0.f;
    for (int k = threadIdx.x; k < nb; k += 1024) a += partial[k];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int h = 512; h > 0; h >>= 1) {
        if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = s[0] * inv_n;
}

}  // namespace gs

using namespace gs;

__global__ void k_counter_add(int32_t* c, int32_t d) { *c += d; }

extern "C" int gs_counter_add(int32_t* counter, int32_t delta, void* stream) {
    if (!counter) return GS_ERR_INVALID_ARG;
    k_counter_add<<<1, 1, 0, (cudaStream_t)stream>>>(counter, delta);
    count_launch();
    GS_CUDA_CHECK_LAUNCH();
    return GS_OK;
}

// Each processed Gaussian's rate multiplier decays after the update (a
// separate launch: every parameter row of a Gaussian reads the old value).
__global__ void k_lr_decay(float* __restrict__ lr_scale, const uint8_t* __restrict__ visible, int64_t n, float d) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && visible[i]) lr_scale[i] *= d;
}

extern "C" int gs_adam_step(const gs_gaussians* params, const gs_grads* grads, const gs_gaussians* m,
                            const gs_gaussians* v, const gs_adam_config* cfg, int32_t step, const int32_t* step_dev,
                            float* lr_scale, void* stream) {
    if (!params || !grads || !m || !v || !cfg || (step < 1 && !step_dev) || params->n < 0) return GS_ERR_INVALID_ARG;
    if (m->n != params->n || v->n != params->n || !grads->visible) return GS_ERR_INVALID_ARG;
    const int64_t n = params->n;
    if (n == 0) return GS_OK;
    const float bc1 = (float)(1.0 - pow((double)cfg->beta1, step < 1 ? 1 : step));
    const float bc2 = (float)(1.0 - pow((double)cfg->beta2, step < 1 ? 1 : step));
    k_adam<<<(unsigned)ceil_div(15 * n, 256), 256, 0, (cudaStream_t)stream>>>(
        (float4*)params->mean_opa, (float4*)params->scale, (float4*)params->quat, (float4*)params->sh,
        (const float4*)grads->mean_opa, (const float4*)grads->scale, (const float4*)grads->quat,
        (const float4*)grads->sh, (float4*)m->mean_opa, (float4*)m->scale, (float4*)m->quat, (float4*)m->sh,
        (float4*)v->mean_opa, (float4*)v->scale, (float4*)v->quat, (float4*)v->sh, grads->visible, n, *cfg, bc1, bc2,
        step_dev, lr_scale);
    count_launch();
    if (lr_scale && cfg->decay != 1.f) {
        k_lr_decay<<<(unsigned)ceil_div(n, 256), 256, 0, (cudaStream_t)stream>>>(lr_scale, grads->visible, n,
                                                                                 cfg->decay);
        count_launch();
    }
    GS_CUDA_CHECK_LAUNCH();
    return GS_OK;
}

extern "C" int gs_pose_step(gs_camera* cams, int32_t n_views, const float* dL_dpose, float* m, float* v, float lr_t,
                            float lr_r, float beta1, float beta2, float eps, int32_t step, const int32_t* step_dev,
                            void* stream) {
    if (!cams || !dL_dpose || !m || !v || n_views < 1 || n_views > GS_MAX_VIEWS || (step < 1 && !step_dev))
        return GS_ERR_INVALID_ARG;
    const float bc1 = (float)(1.0 - pow((double)beta1, step < 1 ? 1 : step));
    const float bc2 = (float)(1.0 - pow((double)beta2, step < 1 ? 1 : step));
    k_pose_step<<<1, 64, 0, (cudaStream_t)stream>>>(cams, n_views, dL_dpose, m, v, lr_t, lr_r, beta1, beta2, eps, bc1,
                                                    bc2, step_dev);
    count_launch();
    GS_CUDA_CHECK_LAUNCH();
    return GS_OK;
}

// SE(3) exponential and left Jacobian in FP64. With K = phi^, th = |phi|:
// exp: R = I + a K + b K^2, t = V rho, V = I + b K + c K^2, and the left
// Jacobian [[V, Q], [0, V]] with
// Q = rho^/2 + c (K P + P K + K P K) + d (K K P + P K K - 3 K P K)
//     + e (K P K K + K K P K),  P = rho^,
// a = sin th / th, b = (1 - cos th) / th^2, c = (th - sin th) / th^3,
// d = (th^2 + 2 cos th - 2) / (2 th^4), e = (2 th - 3 sin th + th cos th) / (2 th^5)
// (Taylor series below th = 1e-3).
struct Se3Coef {
    double a, b, c, d, e;
};

__device__ Se3Coef se3_coef(double th) {
    const double t2 = th * th;
    Se3Coef k;
    if (th < 1e-3) {
        k.a = 1.0 - t2 / 6.0;
        k.b = 0.5 - t2 / 24.0;
        k.c = 1.0 / 6.0 - t2 / 120.0;
        k.d = 1.0 / 24.0 - t2 / 720.0;
        k.e = 1.0 / 120.0 - t2 / 2520.0;
    } else {
        const double s = sin(th), co = cos(th);
        k.a = s / th;
        k.b = (1.0 - co) / t2;
        k.c = (th - s) / (t2 * th);
        k.d = (t2 + 2.0 * co - 2.0) / (2.0 * t2 * t2);
        k.e = (2.0 * th - 3.0 * s + th * co) / (2.0 * t2 * t2 * th);
    }
    return k;
}

__device__ void hat3(const double* w, double* K) {
    K[0] = 0.0, K[1] = -w[2], K[2] = w[1];
    K[3] = w[2], K[4] = 0.0, K[5] = -w[0];
    K[6] = -w[1], K[7] = w[0], K[8] = 0.0;
}

__device__ void mul3(const double* A, const double* B, double* C) {
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) C[3 * r + c] = A[3 * r] * B[c] + A[3 * r + 1] * B[3 + c] + A[3 * r + 2] * B[6 + c];
}

__global__ void k_pose_apply(const gs_camera* __restrict__ ref, const float* __restrict__ xi, int nv,
                             gs_camera* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    double rho[3], phi[3];
    for (int k = 0; k < 3; k++) rho[k] = xi[6 * i + k], phi[k] = xi[6 * i + 3 + k];
    const Se3Coef c = se3_coef(sqrt(phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2]));
    double K[9], K2[9];
    hat3(phi, K);
    mul3(K, K, K2);
    gs_camera cam = ref[i];
    double R[9], t[3];
    for (int k = 0; k < 9; k++) R[k] = cam.R[k];
    for (int k = 0; k < 3; k++) t[k] = cam.t[k];
    double dR[9], V[9];
    for (int k = 0; k < 9; k++) {
        const double I = (k % 4 == 0) ? 1.0 : 0.0;
        dR[k] = I + c.a * K[k] + c.b * K2[k];
        V[k] = I + c.b * K[k] + c.c * K2[k];
    }
    for (int r = 0; r < 3; r++) {
        for (int q = 0; q < 3; q++)
            cam.R[3 * r + q] = (float)(dR[3 * r] * R[q] + dR[3 * r + 1] * R[3 + q] + dR[3 * r + 2] * R[6 + q]);
        cam.t[r] = (float)(dR[3 * r] * t[0] + dR[3 * r + 1] * t[1] + dR[3 * r + 2] * t[2] + V[3 * r] * rho[0] +
                           V[3 * r + 1] * rho[1] + V[3 * r + 2] * rho[2]);
    }
    out[i] = cam;
}

__global__ void k_pose_tangent_grad(const float* __restrict__ xi, const float* g_delta, int nv, float* g_xi) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    double rho[3], phi[3], g[6];
    for (int k = 0; k < 3; k++) rho[k] = xi[6 * i + k], phi[k] = xi[6 * i + 3 + k];
    for (int k = 0; k < 6; k++) g[k] = g_delta[6 * i + k];
    const Se3Coef c = se3_coef(sqrt(phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2]));
    double K[9], P[9], K2[9], KP[9], PK[9], KPK[9], KKP[9], PKK[9], KPKK[9], KKPK[9];
    hat3(phi, K);
    hat3(rho, P);
    mul3(K, K, K2);
    mul3(K, P, KP);
    mul3(P, K, PK);
    mul3(KP, K, KPK);
    mul3(K2, P, KKP);
    mul3(P, K2, PKK);
    mul3(KPK, K, KPKK);
    mul3(K, KPK, KKPK);
    double V[9], Q[9];
    for (int k = 0; k < 9; k++) {
        const double I = (k % 4 == 0) ? 1.0 : 0.0;
        V[k] = I + c.b * K[k] + c.c * K2[k];
        Q[k] = 0.5 * P[k] + c.c * (KP[k] + PK[k] + KPK[k]) + c.d * (KKP[k] + PKK[k] - 3.0 * KPK[k]) +
               c.e * (KPKK[k] + KKPK[k]);
    }
    // [g_rho; g_phi] <- [[V^T, 0], [Q^T, V^T]] [g_rho; g_phi]
    double o[6];
    for (int q = 0; q < 3; q++) {
        o[q] = V[q] * g[0] + V[3 + q] * g[1] + V[6 + q] * g[2];
        o[3 + q] = Q[q] * g[0] + Q[3 + q] * g[1] + Q[6 + q] * g[2] + V[q] * g[3] + V[3 + q] * g[4] + V[6 + q] * g[5];
    }
    for (int k = 0; k < 6; k++) g_xi[6 * i + k] = (float)o[k];
}

extern "C" int gs_pose_apply(const gs_camera* cams_ref, const float* xi, int32_t n_views, gs_camera* cams_out,
                             void* stream) {
    if (!cams_ref || !xi || !cams_out || n_views < 1 || n_views > GS_MAX_VIEWS) return GS_ERR_INVALID_ARG;
    k_pose_apply<<<1, 64, 0, (cudaStream_t)stream>>>(cams_ref, xi, n_views, cams_out);
    count_launch();
    GS_CUDA_CHECK_LAUNCH();
    return GS_OK;
}

extern "C" int gs_pose_tangent_grad(const float* xi, const float* dL_ddelta, int32_t n_views, float* dL_dxi,
                                    void* stream) {
    if (!xi || !dL_ddelta || !dL_dxi || n_views < 1 || n_views > GS_MAX_VIEWS) return GS_ERR_INVALID_ARG;
    k_pose_tangent_grad<<<1, 64, 0, (cudaStream_t)stream>>>(xi, dL_ddelta, n_views, dL_dxi);
    count_launch();
    GS_CUDA_CHECK_LAUNCH();
    return GS_OK;
}

// Coarse-to-fine training image: out [3][ceil(H/f)][ceil(W/f)], each pixel the
// mean of the input pixels of its f x f block (partial blocks at ragged edges).
__global__ void k_downsample(const float* __restrict__ in, int W, int H, int f, int w, int h,
                             float* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3LL * w * h) return;
    const int ch = (int)(i / ((int64_t)w * h));
    const int64_t rem = i % ((int64_t)w * h);
    const int I = (int)(rem / w), J = (int)(rem % w);
    const int y1 = min(H, (I + 1) * f), x1 = min(W, (J + 1) * f);
    const float* src = in + (int64_t)ch * W * H;
    float acc = 0.f;
    for (int y = I * f; y < y1; y++)
        for (int x = J * f; x < x1; x++) acc += src[(int64_t)y * W + x];
    out[i] = acc / (float)((y1 - I * f) * (x1 - J * f));
}

extern "C" int gs_downsample(const float* image, int32_t width, int32_t height, int32_t factor, float* out,
                             void* stream) {
    if (!image || !out || width < 1 || height < 1 || factor < 1) return GS_ERR_INVALID_ARG;
    const int w = (width + factor - 1) / factor, h = (height + factor - 1) / factor;
    const int64_t n = 3LL * w * h;
    k_downsample<<<(unsigned)ceil_div(n, 256), 256, 0, (cudaStream_t)stream>>>(image, width, height, factor, w, h,
                                                                               out);
    count_launch();
    GS_CUDA_CHECK_LAUNCH();
    return GS_OK;
}

extern "C" int gs_l1_loss(const float* color, const float* target, int64_t count, float* dL_dcolor, float* loss,
                          void* ws, size_t ws_bytes, void* stream) {
    if (!color || !target || !dL_dcolor || !loss || count < 1 || !ws || ws_bytes < 4 * kLossMaxBlocks)
        return GS_ERR_INVALID_ARG;
    const bool vec = (((uintptr_t)color | (uintptr_t)target | (uintptr_t)dL_dcolor) & 15) == 0;
    const int64_t n4 = vec ? count / 4 : 0;
    int64_t nb = ceil_div(count, kLossThreads * 8);
    if (nb > kLossMaxBlocks) nb = kLossMaxBlocks;
    const float inv_n = (float)(1.0 / (double)count);
    cudaStream_t s = (cudaStream_t)stream;
    k_l1<<<(unsigned)nb, kLossThreads, 0, s>>>((const float4*)color, (const float4*)target, (float4*)dL_dcolor, n4,
                                                color, target, dL_dcolor, count, inv_n, (float*)ws);
    count_launch();
    k_l1_final<<<1, 1024, 0, s>>>((const float*)ws, (int)nb, inv_n, loss);
    count_launch();
    GS_CUDA_CHECK_LAUNCH();
    return GS_OK;
}
