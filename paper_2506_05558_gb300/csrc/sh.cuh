// Real spherical harmonics up to degree 3 (orthonormal, Condon-Shortley phase),
// written as homogeneous polynomials in the unit view direction (x, y, z).
// Index k = l^2 + l + m. Constants: K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!),
// times sqrt(2) for m != 0, times the polynomial's leading factor.
#pragma once

namespace gs {

// degree-wise constants
constexpr float kSH0 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
constexpr float kSH1 = 0.4886025119029199f;    // sqrt(3/(4 pi))
constexpr float kSH2a = 1.0925484305920792f;   // sqrt(15/pi)/2
constexpr float kSH2b = 0.31539156525252005f;  // sqrt(5/pi)/4
constexpr float kSH2c = 0.5462742152960396f;   // sqrt(15/pi)/4
constexpr float kSH3a = 0.5900435899266435f;   // sqrt(35/(2 pi))/4
constexpr float kSH3b = 2.890611442640554f;    // sqrt(105/pi)/2
constexpr float kSH3c = 0.4570457994644658f;   // sqrt(21/(2 pi))/4
constexpr float kSH3d = 0.3731763325901154f;   // sqrt(7/pi)/4
constexpr float kSH3e = 1.445305721320277f;    // sqrt(105/pi)/4

__device__ __forceinline__ void sh_eval_basis(int deg, float x, float y, float z, float* Y) {
    Y[0] = kSH0;
    if (deg < 1) return;
    Y[1] = -kSH1 * y;
    Y[2] = kSH1 * z;
    Y[3] = -kSH1 * x;
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = kSH2a * x * y;
    Y[5] = -kSH2a * y * z;
    Y[6] = kSH2b * (2.f * zz - xx - yy);
    Y[7] = -kSH2a * x * z;
    Y[8] = kSH2c * (xx - yy);
    if (deg < 3) return;
    Y[9] = -kSH3a * y * (3.f * xx - yy);
    Y[10] = kSH3b * x * y * z;
    Y[11] = -kSH3c * y * (4.f * zz - xx - yy);
    Y[12] = kSH3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
    Y[13] = -kSH3c * x * (4.f * zz - xx - yy);
    Y[14] = kSH3e * z * (xx - yy);
    Y[15] = -kSH3a * x * (xx - 3.f * yy);
}

// Gradient of each basis polynomial w.r.t. (x, y, z): dY[k] = (d/dx, d/dy, d/dz).
__device__ __forceinline__ void sh_basis_grad(int deg, float x, float y, float z, float3* dY) {
    dY[0] = make_float3(0.f, 0.f, 0.f);
    if (deg < 1) return;
    dY[1] = make_float3(0.f, -kSH1, 0.f);
    dY[2] = make_float3(0.f, 0.f, kSH1);
    dY[3] = make_float3(-kSH1, 0.f, 0.f);
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    dY[4] = make_float3(kSH2a * y, kSH2a * x, 0.f);
    dY[5] = make_float3(0.f, -kSH2a * z, -kSH2a * y);
    dY[6] = make_float3(-2.f * kSH2b * x, -2.f * kSH2b * y, 4.f * kSH2b * z);
    dY[7] = make_float3(-kSH2a * z, 0.f, -kSH2a * x);
    dY[8] = make_float3(2.f * kSH2c * x, -2.f * kSH2c * y, 0.f);
    if (deg < 3) return;
    dY[9] = make_float3(-kSH3a * 6.f * x * y, -kSH3a * (3.f * xx - 3.f * yy), 0.f);
    dY[10] = make_float3(kSH3b * y * z, kSH3b * x * z, kSH3b * x * y);
    dY[11] = make_float3(kSH3c * 2.f * x * y, -kSH3c * (4.f * zz - xx - 3.f * yy), -kSH3c * 8.f * y * z);
    dY[12] = make_float3(-kSH3d * 6.f * x * z, -kSH3d * 6.f * y * z, kSH3d * (6.f * zz - 3.f * xx - 3.f * yy));
    dY[13] = make_float3(-kSH3c * (4.f * zz - 3.f * xx - yy), kSH3c * 2.f * x * y, -kSH3c * 8.f * x * z);
    dY[14] = make_float3(kSH3e * 2.f * x * z, -kSH3e * 2.f * y * z, kSH3e * (xx - yy));
    dY[15] = make_float3(-kSH3a * (3.f * xx - 3.f * yy), kSH3a * 6.f * x * y, 0.f);
}

// Unclamped colour 0.5 + sum_k Y_k sh_k for one Gaussian (sh: its 12 float4 rows).
__device__ __forceinline__ float3 sh_color(const float4* __restrict__ sh, int deg, const float* Y) {
    const int ncoef = (deg + 1) * (deg + 1);
    float c[48];
    const int nrow = (3 * ncoef + 3) / 4;
#pragma unroll
    for (int r = 0; r < 12; r++) {
        if (r < nrow) {
            const float4 q = sh[r];
            c[4 * r] = q.x; c[4 * r + 1] = q.y; c[4 * r + 2] = q.z; c[4 * r + 3] = q.w;
        } else {
            c[4 * r] = c[4 * r + 1] = c[4 * r + 2] = c[4 * r + 3] = 0.f;
        }
    }
    float3 o = make_float3(0.5f, 0.5f, 0.5f);
#pragma unroll
    for (int k = 0; k < 16; k++) {
        if (k < ncoef) {
            o.x += Y[k] * c[3 * k];
            o.y += Y[k] * c[3 * k + 1];
            o.z += Y[k] * c[3 * k + 2];
        }
    }
    return o;
}

}  // namespace gs
