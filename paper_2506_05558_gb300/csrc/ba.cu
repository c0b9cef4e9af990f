// Mini bundle adjustment of the initial pose estimation (Sec. 4.1 and App. A.1):
// Levenberg-Marquardt over a shared focal length, the poses of frames 1..F-1
// (frame 0 fixed: the gauge) and P points, each observed in all F frames - the
// fixed-size layout that makes every block of the problem a fixed-size
// computation. One iteration:
//   k_ba_residual   residual norms e of all P F observations
//   (radix sorts)   lower median of e and of |e - median|: threshold median + 4 MAD
//   k_ba_normal     per 32-point chunk: each point's Huber-weighted 3x3 block
//                   (damped), gradient and coupling rows K (Nc x 3) are staged
//                   in shared memory; threads owning entries of the reduced
//                   camera system accumulate H_cc - sum_p K H_pp^-1 K^T and its
//                   right-hand side in FP64, in a fixed order (deterministic)
//   k_ba_solve      one CTA: sum of the chunk partials, Marquardt damping,
//                   Cholesky and the two triangular solves in FP64
//   k_ba_backsub    point steps dp = -H_pp^-1 (g_p + K^T dc) and the trial state
//   k_ba_trial_cost robust cost of the trial state on the same observation set
//   k_ba_accept     accept (state <- trial, lam /= nu) or reject (lam *= nu)
// Everything stays on the device, so the iterations can be captured into one
// CUDA graph and replayed without host work.
#include "common.cuh"

namespace gs {

constexpr int kBaMaxF = 8;
constexpr int kBaMaxNc = 6 * (kBaMaxF - 1) + 1;  // 43 camera parameters
constexpr int kBaPts = 32;                       // points per chunk of k_ba_normal
constexpr int kBaThreads = 128;

__device__ __forceinline__ int ba_nc(int F) { return 6 * (F - 1) + 1; }
__device__ __forceinline__ int ba_nup(int nc) { return nc * (nc + 1) / 2; }
__device__ __forceinline__ int ba_stride(int nc) { return ba_nup(nc) + 2 * nc + 1; }  // S_up | H diag | rhs | cost

struct BaObs {
    float r[2], e, w;
    float jq[2][3];  // d pixel / d q (camera-space point)
    float q[3];
};

// Residual of point X in frame (R, t) against its observation, with the
// derivative of the projection with respect to the camera-space point.
__device__ __forceinline__ void ba_observe(const float* Rt, float4 X, float fl, float cx, float cy, float2 uv,
                                           BaObs& o) {
    const float x = Rt[0] * X.x + Rt[1] * X.y + Rt[2] * X.z + Rt[9];
    const float y = Rt[3] * X.x + Rt[4] * X.y + Rt[5] * X.z + Rt[10];
    const float z = Rt[6] * X.x + Rt[7] * X.y + Rt[8] * X.z + Rt[11];
    const float iz = 1.f / z;
    o.q[0] = x; o.q[1] = y; o.q[2] = z;
    o.r[0] = fl * x * iz + cx - uv.x;
    o.r[1] = fl * y * iz + cy - uv.y;
    o.e = sqrtf(o.r[0] * o.r[0] + o.r[1] * o.r[1]);
    const float a = fl * iz;
    o.jq[0][0] = a; o.jq[0][1] = 0.f; o.jq[0][2] = -a * x * iz;
    o.jq[1][0] = 0.f; o.jq[1][1] = a; o.jq[1][2] = -a * y * iz;
}

// Huber weight and cost of an observation kept by the median + 4 MAD rule.
__device__ __forceinline__ float ba_weight(float e, bool keep, float delta) {
    return keep ? (e <= delta ? 1.f : delta / e) : 0.f;
}
__device__ __forceinline__ double ba_cost(float e, bool keep, float delta) {
    if (!keep) return 0.0;
    return e <= delta ? 0.5 * (double)e * e : (double)delta * ((double)e - 0.5 * delta);
}

__device__ __forceinline__ float ba_threshold(const uint32_t* sorted_e, const uint32_t* sorted_d, int64_t n) {
    const int64_t mid = (n - 1) / 2;
    return __uint_as_float(sorted_e[mid]) + 4.f * __uint_as_float(sorted_d[mid]);
}

__global__ void k_ba_residual(const float2* __restrict__ obs, const float* __restrict__ poses,
                              const float4* __restrict__ pts, const float* __restrict__ fl, float cx, float cy,
                              int F, int64_t P, float* __restrict__ e_out, uint32_t* __restrict__ key,
                              uint32_t* __restrict__ val) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * F) return;
    const int64_t p = i / F;
    const int f = (int)(i % F);
    BaObs o;
    ba_observe(poses + 12 * f, pts[p], *fl, cx, cy, obs[i], o);
    e_out[i] = o.e;
    key[i] = __float_as_uint(o.e);  // e >= 0: the bit pattern orders like the value
    val[i] = (uint32_t)i;
}

__global__ void k_ba_dev_keys(const float* __restrict__ e, const uint32_t* __restrict__ sorted_e, int64_t n,
                              uint32_t* __restrict__ key, uint32_t* __restrict__ val) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float med = __uint_as_float(sorted_e[(n - 1) / 2]);
    key[i] = __float_as_uint(fabsf(e[i] - med));
    val[i] = (uint32_t)i;
}

// Per-point system: damped H_pp, gradient g_p, coupling rows K (camera
// parameter c -> 3-vector), the per-observation camera Jacobian rows (for
// H_cc), and the point's robust cost.
struct BaPoint {
    double Hinv[6];  // symmetric 3x3 inverse: 00 01 02 11 12 22
    float g[3];
    double cost;
};

__device__ void ba_point_system(int64_t p, int F, const float2* __restrict__ obs, const float* s_pose,
                                const float4* __restrict__ pts, float fl, float cx, float cy, const float* __restrict__ e_cur,
                                float thr, float delta, float lam, float (*K)[3] /* [Nc][3] or null */,
                                float (*Jc)[2][8] /* [F][2][8] or null */, float* wout /* [F] or null */, BaPoint& bp) {
    const int nc = ba_nc(F);
    const float4 X = pts[p];
    float H[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float g[3] = {0.f, 0.f, 0.f};
    double cost = 0.0;
    if (K)
        for (int c = 0; c < nc; c++) K[c][0] = K[c][1] = K[c][2] = 0.f;
    for (int f = 0; f < F; f++) {
        const float* Rt = s_pose + 12 * f;
        BaObs o;
        ba_observe(Rt, X, fl, cx, cy, obs[p * F + f], o);
        const bool keep = e_cur[p * F + f] <= thr;
        const float w = ba_weight(o.e, keep, delta);
        cost += ba_cost(o.e, keep, delta);
        // point Jacobian Jp = jq R (2 x 3)
        float Jp[2][3];
        for (int k = 0; k < 2; k++)
            for (int c = 0; c < 3; c++) Jp[k][c] = o.jq[k][0] * Rt[c] + o.jq[k][1] * Rt[3 + c] + o.jq[k][2] * Rt[6 + c];
        H[0] += w * (Jp[0][0] * Jp[0][0] + Jp[1][0] * Jp[1][0]);
        H[1] += w * (Jp[0][0] * Jp[0][1] + Jp[1][0] * Jp[1][1]);
        H[2] += w * (Jp[0][0] * Jp[0][2] + Jp[1][0] * Jp[1][2]);
        H[3] += w * (Jp[0][1] * Jp[0][1] + Jp[1][1] * Jp[1][1]);
        H[4] += w * (Jp[0][1] * Jp[0][2] + Jp[1][1] * Jp[1][2]);
        H[5] += w * (Jp[0][2] * Jp[0][2] + Jp[1][2] * Jp[1][2]);
        for (int c = 0; c < 3; c++) g[c] += w * (Jp[0][c] * o.r[0] + Jp[1][c] * o.r[1]);
        // camera Jacobian rows: pose (rho: jq, phi: jq (-q^)) for f > 0, focal (x/z, y/z)
        float jc[2][7];
        const float qx = o.q[0], qy = o.q[1], qz = o.q[2];
        for (int k = 0; k < 2; k++) {
            const float a0 = o.jq[k][0], a1 = o.jq[k][1], a2 = o.jq[k][2];
            jc[k][0] = a0; jc[k][1] = a1; jc[k][2] = a2;
            // row of jq (-q^): -q^ = [[0, qz, -qy], [-qz, 0, qx], [qy, -qx, 0]]
            jc[k][3] = -a1 * qz + a2 * qy;
            jc[k][4] = a0 * qz - a2 * qx;
            jc[k][5] = -a0 * qy + a1 * qx;
            jc[k][6] = (k == 0 ? qx : qy) / qz;
        }
        if (Jc) {
            for (int k = 0; k < 2; k++) {
                for (int a = 0; a < 6; a++) Jc[f][k][a] = f > 0 ? jc[k][a] : 0.f;
                Jc[f][k][6] = jc[k][6];
                Jc[f][k][7] = w * o.r[k];
            }
            wout[f] = w;
        }
        if (K) {
            for (int a = 0; a < 6 && f > 0; a++) {
                float* kr = K[6 * (f - 1) + a];
                for (int c = 0; c < 3; c++) kr[c] += w * (jc[0][a] * Jp[0][c] + jc[1][a] * Jp[1][c]);
            }
            float* kf = K[nc - 1];
            for (int c = 0; c < 3; c++) kf[c] += w * (jc[0][6] * Jp[0][c] + jc[1][6] * Jp[1][c]);
        }
    }
    // Marquardt damping with the absolute floor, then the symmetric 3x3 inverse (FP64)
    const double a = (double)H[0] * (1.0 + lam) + 1e-9, b = H[1], c = H[2];
    const double d = (double)H[3] * (1.0 + lam) + 1e-9, e = H[4];
    const double ff = (double)H[5] * (1.0 + lam) + 1e-9;
    const double c00 = d * ff - e * e, c01 = c * e - b * ff, c02 = b * e - c * d;
    const double c11 = a * ff - c * c, c12 = b * c - a * e, c22 = a * d - b * b;
    const double idet = 1.0 / (a * c00 + b * c01 + c * c02);
    bp.Hinv[0] = c00 * idet; bp.Hinv[1] = c01 * idet; bp.Hinv[2] = c02 * idet;
    bp.Hinv[3] = c11 * idet; bp.Hinv[4] = c12 * idet; bp.Hinv[5] = c22 * idet;
    bp.g[0] = g[0]; bp.g[1] = g[1]; bp.g[2] = g[2];
    bp.cost = cost;
}

__device__ __forceinline__ void sym3_mul(const double* S, const float* v, double* o) {
    o[0] = S[0] * v[0] + S[1] * v[1] + S[2] * v[2];
    o[1] = S[1] * v[0] + S[3] * v[1] + S[4] * v[2];
    o[2] = S[2] * v[0] + S[4] * v[1] + S[5] * v[2];
}

// Upper-triangle index e -> (i, j), i <= j, row-major over i.
__device__ __forceinline__ void up_ij(int e, int nc, int& i, int& j) {
    int r = 0, left = e;
    while (left >= nc - r) { left -= nc - r; r++; }
    i = r;
    j = r + left;
}

__global__ void __launch_bounds__(kBaThreads) k_ba_normal(const float2* __restrict__ obs,
                                                          const float* __restrict__ poses,
                                                          const float4* __restrict__ pts,
                                                          const float* __restrict__ fl_p, float cx, float cy, int F,
                                                          int64_t P, const float* __restrict__ e_cur,
                                                          const uint32_t* __restrict__ sorted_e,
                                                          const uint32_t* __restrict__ sorted_d, float delta,
                                                          const float* __restrict__ lam_p,
                                                          double* __restrict__ partial) {
    extern __shared__ float sm[];
    const int nc = ba_nc(F);
    float* s_pose = sm;                                              // [F][12]
    float(*s_K)[kBaMaxNc][3] = (float(*)[kBaMaxNc][3])(s_pose + 12 * kBaMaxF);  // [pts][Nc][3]
    double(*s_V)[kBaMaxNc][3] = (double(*)[kBaMaxNc][3])(s_K + kBaPts);         // H^-1 K rows
    double(*s_u)[3] = (double(*)[3])(s_V + kBaPts);                              // H^-1 g
    float(*s_J)[kBaMaxF][2][8] = (float(*)[kBaMaxF][2][8])(s_u + kBaPts);         // camera rows
    float(*s_w)[kBaMaxF] = (float(*)[kBaMaxF])(s_J + kBaPts);
    double* s_cost = (double*)(s_w + kBaPts);  // [kBaPts]
    const int tid = threadIdx.x;
    for (int i = tid; i < 12 * F; i += blockDim.x) s_pose[i] = poses[i];
    __syncthreads();
    const int64_t p0 = (int64_t)blockIdx.x * kBaPts;
    const int np = (int)min((int64_t)kBaPts, P - p0);
    const float thr = ba_threshold(sorted_e, sorted_d, P * F);
    const float fl = *fl_p, lam = *lam_p;
    if (tid < kBaPts) {
        if (tid < np) {
            BaPoint bp;
            ba_point_system(p0 + tid, F, obs, s_pose, pts, fl, cx, cy, e_cur, thr, delta, lam, s_K[tid], s_J[tid],
                            s_w[tid], bp);
            for (int c = 0; c < nc; c++) {
                double v[3];
                sym3_mul(bp.Hinv, s_K[tid][c], v);
                s_V[tid][c][0] = v[0]; s_V[tid][c][1] = v[1]; s_V[tid][c][2] = v[2];
            }
            double u[3];
            sym3_mul(bp.Hinv, bp.g, u);
            s_u[tid][0] = u[0]; s_u[tid][1] = u[1]; s_u[tid][2] = u[2];
            s_cost[tid] = bp.cost;
        } else {
            s_cost[tid] = 0.0;
        }
    }
    __syncthreads();
    const int nup = ba_nup(nc);
    double* out = partial + (int64_t)blockIdx.x * ba_stride(nc);
    // frame and local index of camera parameter c (focal: frame -1)
    auto cam_of = [&](int c, int& fr, int& a) {
        if (c == nc - 1) { fr = -1; a = 6; } else { fr = c / 6 + 1; a = c % 6; }
    };
    for (int e = tid; e < nup; e += blockDim.x) {
        int i, j;
        up_ij(e, nc, i, j);
        int fi, ai, fj, aj;
        cam_of(i, fi, ai);
        cam_of(j, fj, aj);
        double h = 0.0;  // H_cc entry from the observations
        for (int pt = 0; pt < np; pt++) {
            for (int f = 0; f < F; f++) {
                if ((fi >= 0 && fi != f) || (fj >= 0 && fj != f)) continue;
                const float w = s_w[pt][f];
                h += (double)w * ((double)s_J[pt][f][0][ai] * s_J[pt][f][0][aj] +
                                  (double)s_J[pt][f][1][ai] * s_J[pt][f][1][aj]);
            }
        }
        double sch = 0.0;  // sum_p K_i . H^-1 K_j
        for (int pt = 0; pt < np; pt++)
            sch += (double)s_K[pt][i][0] * s_V[pt][j][0] + (double)s_K[pt][i][1] * s_V[pt][j][1] +
                   (double)s_K[pt][i][2] * s_V[pt][j][2];
        out[e] = h - sch;
        if (i == j) out[nup + i] = h;
    }
    for (int c = tid; c < nc; c += blockDim.x) {
        int fc, ac;
        cam_of(c, fc, ac);
        double gc = 0.0, ku = 0.0;
        for (int pt = 0; pt < np; pt++) {
            for (int f = 0; f < F; f++) {
                if (fc >= 0 && fc != f) continue;
                gc += (double)s_J[pt][f][0][ac] * s_J[pt][f][0][7] + (double)s_J[pt][f][1][ac] * s_J[pt][f][1][7];
            }
            ku += (double)s_K[pt][c][0] * s_u[pt][0] + (double)s_K[pt][c][1] * s_u[pt][1] +
                  (double)s_K[pt][c][2] * s_u[pt][2];
        }
        out[nup + nc + c] = -gc + ku;  // rhs of the reduced system
    }
    if (tid == 0) {
        double cst = 0.0;
        for (int pt = 0; pt < kBaPts; pt++) cst += s_cost[pt];
        out[nup + 2 * nc] = cst;
    }
}

constexpr int kBaSolveThreads = 256;

// One CTA: fixed-order sum of the chunk partials, damping, Cholesky, solves.
__global__ void __launch_bounds__(kBaSolveThreads) k_ba_solve(const double* __restrict__ partial, int nb, int F,
                                                               const float* __restrict__ lam_p,
                                                               double* __restrict__ dc, double* __restrict__ cost_cur,
                                                               int* __restrict__ fail) {
    __shared__ double s_tot[kBaMaxNc * (kBaMaxNc + 1) / 2 + 2 * kBaMaxNc + 1];
    __shared__ double L[kBaMaxNc][kBaMaxNc + 1];
    __shared__ double y[kBaMaxNc];
    __shared__ int s_bad;
    const int nc = ba_nc(F), nup = ba_nup(nc), stride = ba_stride(nc);
    const int tid = threadIdx.x;
    for (int v = tid; v < stride; v += blockDim.x) {
        double a = 0.0;
        for (int b = 0; b < nb; b++) a += partial[(int64_t)b * stride + v];
        s_tot[v] = a;
    }
    if (tid == 0) s_bad = 0;
    __syncthreads();
    const double lam = *lam_p;
    for (int e = tid; e < nup; e += blockDim.x) {
        int i, j;
        up_ij(e, nc, i, j);
        double v = s_tot[e];
        if (i == j) v += lam * s_tot[nup + i] + 1e-9;
        L[i][j] = v;
        L[j][i] = v;
    }
    __syncthreads();
    for (int k = 0; k < nc; k++) {  // right-looking Cholesky, lower triangle
        if (tid == 0) {
            const double d = L[k][k];
            if (!(d > 0.0)) s_bad = 1;
            L[k][k] = d > 0.0 ? sqrt(d) : 1.0;
        }
        __syncthreads();
        for (int i = k + 1 + tid; i < nc; i += blockDim.x) L[i][k] /= L[k][k];
        __syncthreads();
        const int m = nc - k - 1;
        for (int e = tid; e < m * m; e += blockDim.x) {
            const int i = k + 1 + e / m, j = k + 1 + e % m;
            if (j <= i) L[i][j] -= L[i][k] * L[j][k];
        }
        __syncthreads();
    }
    if (tid < 32) {  // forward and back substitution by one warp
        const int lane = tid;
        for (int i = 0; i < nc; i++) {
            double s = 0.0;
            for (int j = lane; j < i; j += 32) s += L[i][j] * y[j];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) y[i] = (s_tot[nup + nc + i] - s) / L[i][i];
            __syncwarp();
        }
        for (int i = nc - 1; i >= 0; i--) {
            double s = 0.0;
            for (int j = i + 1 + lane; j < nc; j += 32) s += L[j][i] * y[j];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) y[i] = (y[i] - s) / L[i][i];
            __syncwarp();
        }
    }
    __syncthreads();
    for (int c = tid; c < nc; c += blockDim.x) dc[c] = s_bad ? 0.0 : y[c];
    if (tid == 0) {
        *cost_cur = s_tot[nup + 2 * nc];
        if (s_bad) atomicExch(fail, 1);
    }
}

// T <- exp(d^) T for d = (rho, phi), in FP64.
__device__ void ba_retract(const float* Rt, const double* d, float* out) {
    const double wx = d[3], wy = d[4], wz = d[5];
    const double th2 = wx * wx + wy * wy + wz * wz, th = sqrt(th2);
    double A, B, Cc;
    if (th < 1e-4) {
        A = 1.0 - th2 / 6.0; B = 0.5 - th2 / 24.0; Cc = 1.0 / 6.0 - th2 / 120.0;
    } else {
        A = sin(th) / th; B = (1.0 - cos(th)) / th2; Cc = (th - sin(th)) / (th2 * th);
    }
    const double K[9] = {0.0, -wz, wy, wz, 0.0, -wx, -wy, wx, 0.0};
    double K2[9];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) K2[3 * r + c] = K[3 * r] * K[c] + K[3 * r + 1] * K[3 + c] + K[3 * r + 2] * K[6 + c];
    double dR[9], V[9];
    for (int k = 0; k < 9; k++) {
        const double I = (k % 4 == 0) ? 1.0 : 0.0;
        dR[k] = I + A * K[k] + B * K2[k];
        V[k] = I + B * K[k] + Cc * K2[k];
    }
    for (int r = 0; r < 3; r++) {
        for (int c = 0; c < 3; c++)
            out[3 * r + c] = (float)(dR[3 * r] * Rt[c] + dR[3 * r + 1] * Rt[3 + c] + dR[3 * r + 2] * Rt[6 + c]);
        out[9 + r] = (float)(dR[3 * r] * Rt[9] + dR[3 * r + 1] * Rt[10] + dR[3 * r + 2] * Rt[11] + V[3 * r] * d[0] +
                             V[3 * r + 1] * d[1] + V[3 * r + 2] * d[2]);
    }
}

__global__ void __launch_bounds__(kBaThreads) k_ba_backsub(const float2* __restrict__ obs,
                                                           const float* __restrict__ poses,
                                                           const float4* __restrict__ pts,
                                                           const float* __restrict__ fl_p, float cx, float cy, int F,
                                                           int64_t P, const float* __restrict__ e_cur,
                                                           const uint32_t* __restrict__ sorted_e,
                                                           const uint32_t* __restrict__ sorted_d, float delta,
                                                           const float* __restrict__ lam_p,
                                                           const double* __restrict__ dc, float* __restrict__ poses_t,
                                                           float4* __restrict__ pts_t, float* __restrict__ fl_t) {
    __shared__ float s_pose[12 * kBaMaxF];
    const int nc = ba_nc(F);
    for (int i = threadIdx.x; i < 12 * F; i += blockDim.x) s_pose[i] = poses[i];
    __syncthreads();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x == 0 && threadIdx.x < F) {  // trial camera state
        const int f = threadIdx.x;
        if (f == 0) {
            for (int k = 0; k < 12; k++) poses_t[k] = s_pose[k];
            *fl_t = (float)((double)*fl_p + dc[nc - 1]);
        } else {
            ba_retract(s_pose + 12 * f, dc + 6 * (f - 1), poses_t + 12 * f);
        }
    }
    if (p >= P) return;
    float K[kBaMaxNc][3];
    BaPoint bp;
    const float thr = ba_threshold(sorted_e, sorted_d, P * F);
    ba_point_system(p, F, obs, s_pose, pts, *fl_p, cx, cy, e_cur, thr, delta, *lam_p, K, nullptr, nullptr, bp);
    double rhs[3] = {bp.g[0], bp.g[1], bp.g[2]};
    for (int c = 0; c < nc; c++)
        for (int k = 0; k < 3; k++) rhs[k] += (double)K[c][k] * dc[c];
    const double* S = bp.Hinv;
    const double dx = -(S[0] * rhs[0] + S[1] * rhs[1] + S[2] * rhs[2]);
    const double dy = -(S[1] * rhs[0] + S[3] * rhs[1] + S[4] * rhs[2]);
    const double dz = -(S[2] * rhs[0] + S[4] * rhs[1] + S[5] * rhs[2]);
    const float4 X = pts[p];
    pts_t[p] = make_float4((float)(X.x + dx), (float)(X.y + dy), (float)(X.z + dz), 0.f);
}

__global__ void __launch_bounds__(256) k_ba_trial_cost(const float2* __restrict__ obs,
                                                        const float* __restrict__ poses_t,
                                                        const float4* __restrict__ pts_t,
                                                        const float* __restrict__ fl_t, float cx, float cy, int F,
                                                        int64_t P, const float* __restrict__ e_cur,
                                                        const uint32_t* __restrict__ sorted_e,
                                                        const uint32_t* __restrict__ sorted_d, float delta,
                                                        double* __restrict__ partial) {
    __shared__ double s[256];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double c = 0.0;
    if (i < P * F) {
        const float thr = ba_threshold(sorted_e, sorted_d, P * F);
        BaObs o;
        ba_observe(poses_t + 12 * (i % F), pts_t[i / F], *fl_t, cx, cy, obs[i], o);
        c = ba_cost(o.e, e_cur[i] <= thr, delta);
    }
    s[threadIdx.x] = c;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = s[0];
}

__global__ void k_ba_accept(const double* __restrict__ trial_partial, int nb, const double* __restrict__ cost_cur,
                            int F, int64_t P, const float* __restrict__ poses_t, const float4* __restrict__ pts_t,
                            const float* __restrict__ fl_t, float* __restrict__ poses, float4* __restrict__ pts,
                            float* __restrict__ fl, float* __restrict__ lam, float nu, float* __restrict__ history,
                            int* __restrict__ iter) {
    double tc = 0.0;  // every thread sums in the same order
    for (int b = 0; b < nb; b++) tc += trial_partial[b];
    const double cur = *cost_cur;
    const bool acc = tc < cur;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (acc) {
        if (i < P) pts[i] = pts_t[i];
        if (i < 12 * F) poses[i] = poses_t[i];
        if (i == 0) *fl = *fl_t;
    }
    if (i == 0) {
        *lam = acc ? *lam / nu : *lam * nu;
        if (history) {
            const int it = *iter;
            history[3 * it] = (float)cur;
            history[3 * it + 1] = (float)tc;
            history[3 * it + 2] = acc ? 1.f : 0.f;
        }
        *iter += 1;
    }
}

struct BaWs {
    float *e, *poses_t, *fl_t;
    float4* pts_t;
    uint32_t *k0, *v0, *k1, *v1, *d0, *dv0, *d1, *dv1, *hist;
    void* scan;
    double *partial, *trial_partial, *dc, *cost_cur;
    int *iter, *fail;
};

static BaWs carve_ba(char* base, size_t cap, int F, int64_t P, size_t* used) {
    Carve c{base, 0, cap};
    BaWs w;
    const int64_t n = P * F;
    const int nc = 6 * (F - 1) + 1;
    const int64_t nb = ceil_div(P, kBaPts), nt = ceil_div(n, 256);
    w.e = c.take<float>(n);
    w.poses_t = c.take<float>(12 * kBaMaxF);
    w.fl_t = c.take<float>(4);
    w.pts_t = c.take<float4>(P);
    w.k0 = c.take<uint32_t>(n); w.v0 = c.take<uint32_t>(n);
    w.k1 = c.take<uint32_t>(n); w.v1 = c.take<uint32_t>(n);
    w.d0 = c.take<uint32_t>(n); w.dv0 = c.take<uint32_t>(n);
    w.d1 = c.take<uint32_t>(n); w.dv1 = c.take<uint32_t>(n);
    w.hist = c.take<uint32_t>(256 * radix_blocks(n));
    const int64_t sn = 256 * radix_blocks(n) > n ? 256 * radix_blocks(n) : n;
    w.scan = c.take<char>(scan_workspace_bytes(sn));
    w.partial = c.take<double>(nb * (nc * (nc + 1) / 2 + 2 * nc + 1));
    w.trial_partial = c.take<double>(nt);
    w.dc = c.take<double>(kBaMaxNc);
    w.cost_cur = c.take<double>(1);
    w.iter = c.take<int>(1);
    w.fail = c.take<int>(1);
    *used = c.used;
    return w;
}

static size_t ba_normal_smem() {
    return sizeof(float) * 12 * kBaMaxF + sizeof(float) * kBaPts * kBaMaxNc * 3 +
           sizeof(double) * kBaPts * kBaMaxNc * 3 + sizeof(double) * kBaPts * 3 +
           sizeof(float) * kBaPts * kBaMaxF * 2 * 8 + sizeof(float) * kBaPts * kBaMaxF + sizeof(double) * kBaPts;
}

}  // namespace gs

using namespace gs;

extern "C" size_t gs_ba_workspace_size(int32_t n_frames, int64_t n_points) {
    if (n_frames < 2 || n_frames > kBaMaxF || n_points < 1) return 0;
    size_t used = 0;
    carve_ba(nullptr, 0, n_frames, n_points, &used);
    return used;
}

extern "C" int gs_ba_lm(const float* obs, int32_t n_frames, int64_t n_points, float cx, float cy, float* fl,
                        float* poses, float* points, float* lam, int32_t iterations, float huber_delta, float nu,
                        float* history, int32_t* failed, void* ws, size_t ws_bytes, void* stream) {
    const int F = n_frames;
    const int64_t P = n_points;
    if (!obs || !fl || !poses || !points || !lam || F < 2 || F > kBaMaxF || P < 1 || iterations < 0 ||
        !(huber_delta > 0.f) || !(nu > 1.f) || P * F > (int64_t)UINT32_MAX || !failed)
        return GS_ERR_INVALID_ARG;
    size_t need = 0;
    BaWs w = carve_ba((char*)ws, ws_bytes, F, P, &need);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255) || ((uintptr_t)points & 15) || ((uintptr_t)obs & 7))
        return GS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = P * F;
    const int nc = 6 * (F - 1) + 1;
    const int nb = (int)ceil_div(P, kBaPts), nt = (int)ceil_div(n, 256);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_ba_normal, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ba_normal_smem());
        attr_set = true;
    }
    const float2* ob = (const float2*)obs;
    float4* pts = (float4*)points;
    cudaMemsetAsync(w.iter, 0, sizeof(int), s);
    cudaMemsetAsync(w.fail, 0, sizeof(int), s);
    for (int it = 0; it < iterations; it++) {
        k_ba_residual<<<nt, 256, 0, s>>>(ob, poses, pts, fl, cx, cy, F, P, w.e, w.k0, w.v0);
        count_launch();
        const bool e1 = radix_sort_pairs(w.k0, w.v0, w.k1, w.v1, n, nullptr, 32, w.hist, w.scan, s, false);
        const uint32_t* se = e1 ? w.k1 : w.k0;
        k_ba_dev_keys<<<nt, 256, 0, s>>>(w.e, se, n, w.d0, w.dv0);
        count_launch();
        const bool d1 = radix_sort_pairs(w.d0, w.dv0, w.d1, w.dv1, n, nullptr, 32, w.hist, w.scan, s, false);
        const uint32_t* sd = d1 ? w.d1 : w.d0;
        k_ba_normal<<<nb, kBaThreads, ba_normal_smem(), s>>>(ob, poses, pts, fl, cx, cy, F, P, w.e, se, sd,
                                                             huber_delta, lam, w.partial);
        count_launch();
        k_ba_solve<<<1, kBaSolveThreads, 0, s>>>(w.partial, nb, F, lam, w.dc, w.cost_cur, w.fail);
        count_launch();
        k_ba_backsub<<<(unsigned)ceil_div(P, kBaThreads), kBaThreads, 0, s>>>(
            ob, poses, pts, fl, cx, cy, F, P, w.e, se, sd, huber_delta, lam, w.dc, w.poses_t, w.pts_t, w.fl_t);
        count_launch();
        k_ba_trial_cost<<<nt, 256, 0, s>>>(ob, w.poses_t, w.pts_t, w.fl_t, cx, cy, F, P, w.e, se, sd, huber_delta,
                                           w.trial_partial);
        count_launch();
        const int64_t na = P > 12 * F ? P : 12 * F;
        k_ba_accept<<<(unsigned)ceil_div(na, 256), 256, 0, s>>>(w.trial_partial, nt, w.cost_cur, F, P, w.poses_t,
                                                                w.pts_t, w.fl_t, poses, pts, fl, lam, nu, history,
                                                                w.iter);
        count_launch();
    }
    cudaMemcpyAsync(failed, w.fail, sizeof(int), cudaMemcpyDeviceToDevice, s);
    (void)nc;
    GS_CUDA_CHECK_LAUNCH();
    return GS_OK;
}
