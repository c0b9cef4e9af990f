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

// Gradient of f = sum_k w_k Y_k with respect to the direction components
// (x, y, z) of the basis polynomials, accumulated term by term (w_0 unused:
// Y_0 is constant).
__device__ __forceinline__ float3 sh_weighted_grad(int deg, float x, float y, float z, const float* w) {
    float gx = 0.f, gy = 0.f, gz = 0.f;
    if (deg < 1) return make_float3(gx, gy, gz);
    gy -= kSH1 * w[1];
    gz += kSH1 * w[2];
    gx -= kSH1 * w[3];
    if (deg < 2) return make_float3(gx, gy, gz);
    gx += kSH2a * w[4] * y;  // Y4 = a x y
    gy += kSH2a * w[4] * x;
    gy -= kSH2a * w[5] * z;  // Y5 = -a y z
    gz -= kSH2a * w[5] * y;
    gx -= 2.f * kSH2b * w[6] * x;  // Y6 = b (2 zz - xx - yy)
    gy -= 2.f * kSH2b * w[6] * y;
    gz += 4.f * kSH2b * w[6] * z;
    gx -= kSH2a * w[7] * z;  // Y7 = -a x z
    gz -= kSH2a * w[7] * x;
    gx += 2.f * kSH2c * w[8] * x;  // Y8 = c (xx - yy)
    gy -= 2.f * kSH2c * w[8] * y;
    if (deg < 3) return make_float3(gx, gy, gz);
    const float xx = x * x, yy = y * y, zz = z * z;
    gx -= kSH3a * w[9] * 6.f * x * y;  // Y9 = -a y (3 xx - yy)
    gy -= kSH3a * w[9] * (3.f * xx - 3.f * yy);
    gx += kSH3b * w[10] * y * z;  // Y10 = b x y z
    gy += kSH3b * w[10] * x * z;
    gz += kSH3b * w[10] * x * y;
    gx += kSH3c * w[11] * 2.f * x * y;  // Y11 = -c y (4 zz - xx - yy)
    gy -= kSH3c * w[11] * (4.f * zz - xx - 3.f * yy);
    gz -= kSH3c * w[11] * 8.f * y * z;
    gx -= kSH3d * w[12] * 6.f * x * z;  // Y12 = d z (2 zz - 3 xx - 3 yy)
    gy -= kSH3d * w[12] * 6.f * y * z;
    gz += kSH3d * w[12] * (6.f * zz - 3.f * xx - 3.f * yy);
    gx -= kSH3c * w[13] * (4.f * zz - 3.f * xx - yy);  // Y13 = -c x (4 zz - xx - yy)
    gy += kSH3c * w[13] * 2.f * x * y;
    gz -= kSH3c * w[13] * 8.f * x * z;
    gx += kSH3e * w[14] * 2.f * x * z;  // Y14 = e z (xx - yy)
    gy -= kSH3e * w[14] * 2.f * y * z;
    gz += kSH3e * w[14] * (xx - yy);
    gx -= kSH3a * w[15] * (3.f * xx - 3.f * yy);  // Y15 = -a x (xx - 3 yy)
    gy += kSH3a * w[15] * 6.f * x * y;
    return make_float3(gx, gy, gz);
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
