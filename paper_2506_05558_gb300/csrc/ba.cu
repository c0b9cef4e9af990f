// Mini bundle adjustment of the initial pose estimation (Sec. 4.1 and App. A.1):
// Levenberg-Marquardt over a shared focal length, the poses of frames 1..F-1
// (frame 0 fixed: the gauge) and P points, each observed in all F frames - the
// fixed-size layout that makes every block of the problem a fixed-size
// computation. One iteration:
//   k_ba_residual   residual norms e of all P F observations
//   k_ba_median_mad lower median of e and of |e - median| by radix select in one
//                   CTA: median + 4 MAD
//   k_ba_normal     per 32-point chunk: each point's Huber-weighted 3x3 block
//                   (damped), gradient and coupling rows K (Nc x 3) are staged
//                   in shared memory; threads owning entries of the reduced
//                   camera system accumulate H_cc - sum_p K H_pp^-1 K^T and its
//                   right-hand side in FP64, in a fixed order (deterministic)
//   k_ba_reduce     fixed-order sum of the chunk partials
//   k_ba_solve      one CTA: Marquardt damping, L D L^T factorisation and the
//                   two triangular solves in FP64
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

__global__ void k_ba_residual(const float2* __restrict__ obs, const float* __restrict__ poses,
                              const float4* __restrict__ pts, const float* __restrict__ fl, float cx, float cy,
                              int F, int64_t P, float* __restrict__ e_out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * F) return;
    const int64_t p = i / F;
    const int f = (int)(i % F);
    BaObs o;
    ba_observe(poses + 12 * f, pts[p], *fl, cx, cy, obs[i], o);
    e_out[i] = o.e;
}

// Median + 4 MAD threshold in one CTA: radix select (8 bits per pass, most
// significant first) of the lower median of e, then of |e - median|; the
// values are re-read from global memory (L1-resident) on every pass, so any
// P F fits. Non-negative floats order like their bits. The residual norms share
// a handful of exponents, so the first pass would pile every atomic onto a few
// bins: each lane counts into its own copy of the histogram (row stride 257,
// so equal digits of one warp fall into distinct banks).
constexpr int kBaSelThreads = 1024;
constexpr int64_t kBaMaxObs = int64_t(1) << 26;  // P F bound: 32-bit indexing everywhere
constexpr int kBaHistStride = 257;

template <bool kAbsDev>
__device__ uint32_t select_rank(const float* __restrict__ e, int n, float med, int rank, uint32_t* hist,
                                uint32_t* s_wsum, uint32_t* s_pref) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t* my = hist + lane * kBaHistStride;
    uint32_t prefix = 0, mask = 0;
    int k = rank;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int i = tid; i < 32 * kBaHistStride; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        for (int i = tid; i < n; i += blockDim.x) {
            const float x = kAbsDev ? fabsf(e[i] - med) : e[i];
            const uint32_t u = __float_as_uint(x);
            if ((u & mask) == prefix) atomicAdd(&my[(u >> shift) & 255u], 1u);
        }
        __syncthreads();
        uint32_t c = 0, incl = 0;
        if (tid < 256) {  // bin tid over the 32 copies, then a block scan of the 256 bins
            for (int l = 0; l < 32; l++) c += hist[l * kBaHistStride + tid];
            incl = c;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            if (lane == 31) s_wsum[warp] = incl;
        }
        __syncthreads();
        if (tid < 256) {
            for (int w = 0; w < warp; w++) incl += s_wsum[w];
            const uint32_t excl = incl - c;
            if (excl <= (uint32_t)k && (uint32_t)k < incl) {  // exactly one bin holds rank k
                s_pref[0] = prefix | ((uint32_t)tid << shift);
                s_pref[1] = (uint32_t)k - excl;
            }
        }
        __syncthreads();
        prefix = s_pref[0];
        k = (int)s_pref[1];
        mask |= 255u << shift;
        __syncthreads();
    }
    return prefix;
}

__global__ void __launch_bounds__(kBaSelThreads) k_ba_median_mad(const float* __restrict__ e, int n,
                                                                 float* __restrict__ thr) {
    __shared__ uint32_t hist[32 * kBaHistStride];
    __shared__ uint32_t s_wsum[8];
    __shared__ uint32_t s_pref[2];
    const float med = __uint_as_float(select_rank<false>(e, n, 0.f, (n - 1) / 2, hist, s_wsum, s_pref));
    const float mad = __uint_as_float(select_rank<true>(e, n, med, (n - 1) / 2, hist, s_wsum, s_pref));
    if (threadIdx.x == 0) *thr = med + 4.f * mad;
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
                                                          const float* __restrict__ thr_p, float delta,
                                                          const float* __restrict__ lam_p,
                                                          double* __restrict__ partial) {
    extern __shared__ float sm[];
    const int nc = ba_nc(F);
    float* s_pose = sm;                                              // [F][12]
    float(*s_K)[kBaMaxNc][3] = (float(*)[kBaMaxNc][3])(s_pose + 12 * kBaMaxF);  // [pts][Nc][3]
    float(*s_V)[kBaMaxNc][3] = (float(*)[kBaMaxNc][3])(s_K + kBaPts);           // H^-1 K rows
    double(*s_u)[3] = (double(*)[3])(s_V + kBaPts);                              // H^-1 g
    float(*s_J)[kBaMaxF][2][8] = (float(*)[kBaMaxF][2][8])(s_u + kBaPts);         // camera rows
    float(*s_w)[kBaMaxF] = (float(*)[kBaMaxF])(s_J + kBaPts);
    double* s_cost = (double*)(s_w + kBaPts);  // [kBaPts]
    const int tid = threadIdx.x;
    for (int i = tid; i < 12 * F; i += blockDim.x) s_pose[i] = poses[i];
    __syncthreads();
    const int64_t p0 = (int64_t)blockIdx.x * kBaPts;
    const int np = (int)min((int64_t)kBaPts, P - p0);
    const float thr = *thr_p;
    const float fl = *fl_p, lam = *lam_p;
    if (tid < kBaPts) {
        if (tid < np) {
            BaPoint bp;
            ba_point_system(p0 + tid, F, obs, s_pose, pts, fl, cx, cy, e_cur, thr, delta, lam, s_K[tid], s_J[tid],
                            s_w[tid], bp);
            for (int c = 0; c < nc; c++) {
                double v[3];
                sym3_mul(bp.Hinv, s_K[tid][c], v);
                s_V[tid][c][0] = (float)v[0]; s_V[tid][c][1] = (float)v[1]; s_V[tid][c][2] = (float)v[2];
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
        // H_cc entry from the observations: poses of two different frames share
        // none; a pose entry involves its own frame only; focal-focal all frames
        double h = 0.0;
        if (fi < 0 || fj < 0 || fi == fj) {
            const int f_lo = fi >= 0 ? fi : (fj >= 0 ? fj : 0);
            const int f_hi = fi >= 0 ? fi + 1 : (fj >= 0 ? fj + 1 : F);
            for (int pt = 0; pt < np; pt++) {
                float hp = 0.f;  // this point's terms in FP32
                for (int f = f_lo; f < f_hi; f++)
                    hp += s_w[pt][f] * (s_J[pt][f][0][ai] * s_J[pt][f][0][aj] + s_J[pt][f][1][ai] * s_J[pt][f][1][aj]);
                h += (double)hp;
            }
        }
        double sch = 0.0;  // sum_p K_i . H^-1 K_j: each point's dot product in FP32, the sum in FP64
        for (int pt = 0; pt < np; pt++)
            sch += (double)(s_K[pt][i][0] * s_V[pt][j][0] + s_K[pt][i][1] * s_V[pt][j][1] +
                            s_K[pt][i][2] * s_V[pt][j][2]);
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

// Fixed-order sum of the chunk partials: a block of 32 x 8 threads takes 32
// values; each of the 8 rows sums a contiguous segment of the chunks, then the
// 8 segment sums are added in order.
__global__ void __launch_bounds__(256) k_ba_reduce(const double* __restrict__ partial, int nb, int stride,
                                                   double* __restrict__ tot) {
    __shared__ double s[8][33];
    const int v = blockIdx.x * 32 + threadIdx.x;
    const int seg = (nb + 7) / 8, b0 = threadIdx.y * seg, b1 = min(nb, b0 + seg);
    double a = 0.0;
    if (v < stride)
        for (int b = b0; b < b1; b++) a += partial[(int64_t)b * stride + v];
    s[threadIdx.y][threadIdx.x] = a;
    __syncthreads();
    if (threadIdx.y == 0 && v < stride) {
        double t = 0.0;
        for (int r = 0; r < 8; r++) t += s[r][threadIdx.x];
        tot[v] = t;
    }
}

// Fixed-order sum of the trial-cost block partials (one CTA).
__global__ void k_ba_sum(const double* __restrict__ part, int nb, double* __restrict__ out) {
    __shared__ double s[256];
    double a = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) a += part[b];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

// One CTA: damping, L D L^T factorisation and solves (FP64).
__global__ void __launch_bounds__(kBaSolveThreads) k_ba_solve(const double* __restrict__ tot, int F,
                                                               const float* __restrict__ lam_p,
                                                               double* __restrict__ dc, double* __restrict__ cost_cur,
                                                               int* __restrict__ fail) {
    __shared__ double s_tot[kBaMaxNc * (kBaMaxNc + 1) / 2 + 2 * kBaMaxNc + 1];
    __shared__ double L[kBaMaxNc][kBaMaxNc + 1];
    __shared__ double y[kBaMaxNc];
    __shared__ double s_dinv[kBaMaxNc];
    __shared__ int s_bad;
    const int nc = ba_nc(F), nup = ba_nup(nc), stride = ba_stride(nc);
    const int tid = threadIdx.x;
    for (int v = tid; v < stride; v += blockDim.x) s_tot[v] = tot[v];
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
    // right-looking L D L^T (unit lower L): one reciprocal per column, no square
    // roots; the trailing update uses the unscaled column, scaled at the end
    for (int k = 0; k < nc; k++) {
        if (tid == 0) {
            const double d = L[k][k];
            if (!(d > 0.0)) s_bad = 1;
            s_dinv[k] = d > 0.0 ? 1.0 / d : 0.0;
        }
        __syncthreads();
        const double dinv = s_dinv[k];
        const int m = nc - k - 1;
        for (int e = tid; e < m * m; e += blockDim.x) {
            const int i = k + 1 + e / m, j = k + 1 + e % m;
            if (j <= i) L[i][j] -= L[i][k] * L[j][k] * dinv;
        }
        __syncthreads();
    }
    for (int e = tid; e < nc * nc; e += blockDim.x) {
        const int i = e / nc, k = e % nc;
        if (i > k) L[i][k] *= s_dinv[k];
    }
    __syncthreads();
    if (tid < 32) {  // L y = rhs, then L^T x = D^-1 y, by one warp
        const int lane = tid;
        for (int i = 0; i < nc; i++) {
            double a = 0.0;
            for (int j = lane; j < i; j += 32) a += L[i][j] * y[j];
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0) y[i] = s_tot[nup + nc + i] - a;
            __syncwarp();
        }
        for (int i = lane; i < nc; i += 32) y[i] *= s_dinv[i];
        __syncwarp();
        for (int i = nc - 1; i >= 0; i--) {
            double a = 0.0;
            for (int j = i + 1 + lane; j < nc; j += 32) a += L[j][i] * y[j];
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0) y[i] -= a;
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
                                                           const float* __restrict__ thr_p, float delta,
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
    ba_point_system(p, F, obs, s_pose, pts, *fl_p, cx, cy, e_cur, *thr_p, delta, *lam_p, K, nullptr, nullptr, bp);
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
                                                        const float* __restrict__ thr_p, float delta,
                                                        double* __restrict__ partial) {
    __shared__ double s[256];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double c = 0.0;
    if (i < P * F) {
        BaObs o;
        ba_observe(poses_t + 12 * (i % F), pts_t[i / F], *fl_t, cx, cy, obs[i], o);
        c = ba_cost(o.e, e_cur[i] <= *thr_p, delta);
    }
    s[threadIdx.x] = c;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = s[0];
}

__global__ void k_ba_accept(const double* __restrict__ trial_total, const double* __restrict__ cost_cur,
                            int F, int64_t P, const float* __restrict__ poses_t, const float4* __restrict__ pts_t,
                            const float* __restrict__ fl_t, float* __restrict__ poses, float4* __restrict__ pts,
                            float* __restrict__ fl, float* __restrict__ lam, float nu, float* __restrict__ history,
                            int* __restrict__ iter) {
    const double tc = *trial_total;
    const double cur = *cost_cur;
    const bool acc = tc < cur;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (acc) {
        if (i < P) pts[i] = pts_t[i];
        if (i < 12 * F) poses[i] = poses_t[i];
        if (i == 0) *fl = *fl_t;
    }
    if (i == 0) {
        // lam is kept within [1e-12, 1e10]: a converged run rejects every further
        // step, and unbounded growth would reach infinity
        *lam = fminf(1e10f, fmaxf(1e-12f, acc ? *lam / nu : *lam * nu));
        if (history) {
            const int it = *iter;
            history[3 * it] = (float)cur;
            history[3 * it + 1] = (float)tc;
            history[3 * it + 2] = acc ? 1.f : 0.f;
        }
        *iter += 1;
    }
}

__global__ void k_ba_project(const float* __restrict__ poses, const float4* __restrict__ pts,
                             const float* __restrict__ fl, float cx, float cy, int F, int64_t P,
                             float2* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * F) return;
    BaObs o;
    ba_observe(poses + 12 * (i % F), pts[i / F], *fl, cx, cy, make_float2(0.f, 0.f), o);
    out[i] = make_float2(o.r[0], o.r[1]);
}

struct BaWs {
    float *e, *poses_t, *fl_t;
    float4* pts_t;
    double *partial, *trial_partial, *dc, *cost_cur, *tot, *trial_total;
    float* thr;
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
    w.partial = c.take<double>(nb * (nc * (nc + 1) / 2 + 2 * nc + 1));
    w.trial_partial = c.take<double>(nt);
    w.dc = c.take<double>(kBaMaxNc);
    w.cost_cur = c.take<double>(1);
    w.tot = c.take<double>(nc * (nc + 1) / 2 + 2 * nc + 1);
    w.trial_total = c.take<double>(1);
    w.thr = c.take<float>(1);
    w.iter = c.take<int>(1);
    w.fail = c.take<int>(1);
    *used = c.used;
    return w;
}

// ---------------------------------------------------------------------------
// Pose refinement of a new frame (Sec. 4.1, subsequent frames): the same
// robust iteration over one pose, points and focal length fixed. The 6 x 6
// normal equations are summed per CTA (FP32 products, FP64 warp and CTA sums
// in a fixed order); one CTA then damps, factors (L D L^T, FP64) and retracts.
// The residual, median / MAD, trial-cost and accept kernels are the bundle
// adjustment's with one frame.
// ---------------------------------------------------------------------------
constexpr int kBpThreads = 256;
constexpr int kBpVals = 28;  // H upper triangle (21) | g (6) | cost

__global__ void __launch_bounds__(kBpThreads) k_bp_normal(const float2* __restrict__ obs,
                                                           const float* __restrict__ pose,
                                                           const float4* __restrict__ pts,
                                                           const float* __restrict__ fl_p, float cx, float cy,
                                                           int64_t M, const float* __restrict__ e_cur,
                                                           const float* __restrict__ thr_p, float delta,
                                                           double* __restrict__ partial) {
    __shared__ float s_pose[12];
    __shared__ double s_w[kBpThreads / 32][kBpVals];
    if (threadIdx.x < 12) s_pose[threadIdx.x] = pose[threadIdx.x];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double v[kBpVals];
#pragma unroll
    for (int k = 0; k < kBpVals; k++) v[k] = 0.0;
    if (i < M) {
        BaObs o;
        ba_observe(s_pose, pts[i], *fl_p, cx, cy, obs[i], o);
        const bool keep = e_cur[i] <= *thr_p;
        const float w = ba_weight(o.e, keep, delta);
        float J[2][6];
        const float qx = o.q[0], qy = o.q[1], qz = o.q[2];
        for (int k = 0; k < 2; k++) {  // rho: jq; phi: jq (-q^), -q^ = [[0, qz, -qy], [-qz, 0, qx], [qy, -qx, 0]]
            const float a0 = o.jq[k][0], a1 = o.jq[k][1], a2 = o.jq[k][2];
            J[k][0] = a0; J[k][1] = a1; J[k][2] = a2;
            J[k][3] = -a1 * qz + a2 * qy;
            J[k][4] = a0 * qz - a2 * qx;
            J[k][5] = -a0 * qy + a1 * qx;
        }
        int e = 0;
#pragma unroll
        for (int a = 0; a < 6; a++)
#pragma unroll
            for (int b = a; b < 6; b++) v[e++] = (double)(w * (J[0][a] * J[0][b] + J[1][a] * J[1][b]));
#pragma unroll
        for (int a = 0; a < 6; a++) v[21 + a] = (double)(w * (J[0][a] * o.r[0] + J[1][a] * o.r[1]));
        v[27] = ba_cost(o.e, keep, delta);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kBpVals; k++) {
        double a = v[k];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) s_w[warp][k] = a;
    }
    __syncthreads();
    if (threadIdx.x < kBpVals) {
        double a = 0.0;
        for (int wi = 0; wi < kBpThreads / 32; wi++) a += s_w[wi][threadIdx.x];
        partial[(int64_t)blockIdx.x * kBpVals + threadIdx.x] = a;
    }
}

// One thread: damping (H + lam diag(H) + 1e-9 I), L D L^T of the 6 x 6 system
// in FP64, the step d = -A^-1 g and the retracted trial pose.
__global__ void k_bp_solve(const double* __restrict__ tot, const float* __restrict__ pose,
                           const float* __restrict__ lam_p, float* __restrict__ pose_t,
                           double* __restrict__ cost_cur, int* __restrict__ fail) {
    if (threadIdx.x != 0) return;
    const double lam = *lam_p;
    double A[6][6], g[6];
    int e = 0;
    for (int a = 0; a < 6; a++)
        for (int b = a; b < 6; b++) { A[a][b] = tot[e]; A[b][a] = tot[e]; e++; }
    for (int a = 0; a < 6; a++) { A[a][a] += lam * A[a][a] + 1e-9; g[a] = tot[21 + a]; }
    bool bad = false;
    double dinv[6];
    for (int k = 0; k < 6; k++) {  // L D L^T, unit lower L stored below the diagonal
        const double d = A[k][k];
        if (!(d > 0.0)) bad = true;
        dinv[k] = d > 0.0 ? 1.0 / d : 0.0;
        double col[6];
        for (int i = k + 1; i < 6; i++) col[i] = A[i][k];  // unscaled column k
        for (int i = k + 1; i < 6; i++)
            for (int j = k + 1; j <= i; j++) A[i][j] -= col[i] * col[j] * dinv[k];
        for (int i = k + 1; i < 6; i++) A[i][k] = col[i] * dinv[k];
    }
    double y[6];
    for (int i = 0; i < 6; i++) {
        double a = -g[i];
        for (int j = 0; j < i; j++) a -= A[i][j] * y[j];
        y[i] = a;
    }
    for (int i = 0; i < 6; i++) y[i] *= dinv[i];
    for (int i = 5; i >= 0; i--)
        for (int j = i + 1; j < 6; j++) y[i] -= A[j][i] * y[j];
    if (bad)
        for (int i = 0; i < 6; i++) y[i] = 0.0;
    if (bad) *fail = 1;
    ba_retract(pose, y, pose_t);
    *cost_cur = tot[27];
}

struct BpWs {
    float *e, *pose_t, *fl_t, *thr;
    double *partial, *tot, *trial_partial, *trial_total, *cost_cur;
    int *iter, *fail;
};

static BpWs carve_bp(char* base, size_t cap, int64_t M, size_t* used) {
    Carve c{base, 0, cap};
    BpWs w;
    const int64_t nb = ceil_div(M, kBpThreads), nt = ceil_div(M, 256);
    w.e = c.take<float>(M);
    w.pose_t = c.take<float>(12);
    w.fl_t = c.take<float>(4);
    w.thr = c.take<float>(1);
    w.partial = c.take<double>(nb * kBpVals);
    w.tot = c.take<double>(kBpVals);
    w.trial_partial = c.take<double>(nt);
    w.trial_total = c.take<double>(1);
    w.cost_cur = c.take<double>(1);
    w.iter = c.take<int>(1);
    w.fail = c.take<int>(1);
    *used = c.used;
    return w;
}

static size_t ba_normal_smem() {
    return sizeof(float) * 12 * kBaMaxF + sizeof(float) * kBaPts * kBaMaxNc * 3 +
           sizeof(float) * kBaPts * kBaMaxNc * 3 + sizeof(double) * kBaPts * 3 +
           sizeof(float) * kBaPts * kBaMaxF * 2 * 8 + sizeof(float) * kBaPts * kBaMaxF + sizeof(double) * kBaPts;
}

}  // namespace gs

using namespace gs;

extern "C" size_t gs_ba_workspace_size(int32_t n_frames, int64_t n_points) {
    if (n_frames < 2 || n_frames > kBaMaxF || n_points < 1 || n_points * n_frames > kBaMaxObs) return 0;
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
        !(huber_delta > 0.f) || !(nu > 1.f) || P * F > kBaMaxObs || !failed)
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
        cudaFuncSetAttribute(k_ba_median_mad, cudaFuncAttributePreferredSharedMemoryCarveout, 25);
        attr_set = true;
    }
    const int stride = nc * (nc + 1) / 2 + 2 * nc + 1;
    const float2* ob = (const float2*)obs;
    float4* pts = (float4*)points;
    cudaMemsetAsync(w.iter, 0, sizeof(int), s);
    cudaMemsetAsync(w.fail, 0, sizeof(int), s);
    for (int it = 0; it < iterations; it++) {
        k_ba_residual<<<nt, 256, 0, s>>>(ob, poses, pts, fl, cx, cy, F, P, w.e);
        count_launch();
        k_ba_median_mad<<<1, kBaSelThreads, 0, s>>>(w.e, (int)n, w.thr);
        count_launch();
        k_ba_normal<<<nb, kBaThreads, ba_normal_smem(), s>>>(ob, poses, pts, fl, cx, cy, F, P, w.e, w.thr,
                                                             huber_delta, lam, w.partial);
        count_launch();
        k_ba_reduce<<<(unsigned)ceil_div(stride, 32), dim3(32, 8), 0, s>>>(w.partial, nb, stride, w.tot);
        count_launch();
        k_ba_solve<<<1, kBaSolveThreads, 0, s>>>(w.tot, F, lam, w.dc, w.cost_cur, w.fail);
        count_launch();
        k_ba_backsub<<<(unsigned)ceil_div(P, kBaThreads), kBaThreads, 0, s>>>(
            ob, poses, pts, fl, cx, cy, F, P, w.e, w.thr, huber_delta, lam, w.dc, w.poses_t, w.pts_t, w.fl_t);
        count_launch();
        k_ba_trial_cost<<<nt, 256, 0, s>>>(ob, w.poses_t, w.pts_t, w.fl_t, cx, cy, F, P, w.e, w.thr, huber_delta,
                                           w.trial_partial);
        count_launch();
        k_ba_sum<<<1, 256, 0, s>>>(w.trial_partial, nt, w.trial_total);
        count_launch();
        const int64_t na = P > 12 * F ? P : 12 * F;
        k_ba_accept<<<(unsigned)ceil_div(na, 256), 256, 0, s>>>(w.trial_total, w.cost_cur, F, P, w.poses_t,
                                                                w.pts_t, w.fl_t, poses, pts, fl, lam, nu, history,
                                                                w.iter);
        count_launch();
    }
    cudaMemcpyAsync(failed, w.fail, sizeof(int), cudaMemcpyDeviceToDevice, s);
    (void)nc;
    GS_CUDA_CHECK_LAUNCH();
    return GS_OK;
}

extern "C" int gs_ba_project(const float* fl, const float* poses, const float* points, int32_t n_frames,
                             int64_t n_points, float cx, float cy, float* obs, void* stream) {
    if (!fl || !poses || !points || !obs || n_frames < 1 || n_frames > kBaMaxF || n_points < 1 ||
        ((uintptr_t)points & 15) || ((uintptr_t)obs & 7))
        return GS_ERR_INVALID_ARG;
    const int64_t n = n_points * n_frames;
    k_ba_project<<<(unsigned)ceil_div(n, 256), 256, 0, (cudaStream_t)stream>>>(
        poses, (const float4*)points, fl, cx, cy, n_frames, n_points, (float2*)obs);
    count_launch();
    GS_CUDA_CHECK_LAUNCH();
    return GS_OK;
}

extern "C" size_t gs_ba_pose_workspace_size(int64_t n_obs) {
    if (n_obs < 1 || n_obs > kBaMaxObs) return 0;
    size_t used = 0;
    carve_bp(nullptr, 0, n_obs, &used);
    return used;
}

extern "C" int gs_ba_pose_lm(const float* points, const float* obs, int64_t n_obs, const float* fl, float cx,
                             float cy, float* pose, float* lam, int32_t iterations, float huber_delta, float nu,
                             float* history, int32_t* failed, void* ws, size_t ws_bytes, void* stream) {
    const int64_t M = n_obs;
    if (!points || !obs || !fl || !pose || !lam || !failed || M < 1 || M > kBaMaxObs || iterations < 0 ||
        !(huber_delta > 0.f) || !(nu > 1.f))
        return GS_ERR_INVALID_ARG;
    size_t need = 0;
    BpWs w = carve_bp((char*)ws, ws_bytes, M, &need);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255) || ((uintptr_t)points & 15) || ((uintptr_t)obs & 7))
        return GS_ERR_INVALID_ARG;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_ba_median_mad, cudaFuncAttributePreferredSharedMemoryCarveout, 25);
        attr_set = true;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = (int)ceil_div(M, kBpThreads), nt = (int)ceil_div(M, 256);
    const float2* ob = (const float2*)obs;
    const float4* pts = (const float4*)points;
    cudaMemcpyAsync(w.fl_t, fl, sizeof(float), cudaMemcpyDeviceToDevice, s);
    cudaMemsetAsync(w.iter, 0, sizeof(int), s);
    cudaMemsetAsync(w.fail, 0, sizeof(int), s);
    for (int it = 0; it < iterations; it++) {
        k_ba_residual<<<nt, 256, 0, s>>>(ob, pose, pts, w.fl_t, cx, cy, 1, M, w.e);
        count_launch();
        k_ba_median_mad<<<1, kBaSelThreads, 0, s>>>(w.e, (int)M, w.thr);
        count_launch();
        k_bp_normal<<<nb, kBpThreads, 0, s>>>(ob, pose, pts, w.fl_t, cx, cy, M, w.e, w.thr, huber_delta, w.partial);
        count_launch();
        k_ba_reduce<<<1, dim3(32, 8), 0, s>>>(w.partial, nb, kBpVals, w.tot);
        count_launch();
        k_bp_solve<<<1, 32, 0, s>>>(w.tot, pose, lam, w.pose_t, w.cost_cur, w.fail);
        count_launch();
        k_ba_trial_cost<<<nt, 256, 0, s>>>(ob, w.pose_t, pts, w.fl_t, cx, cy, 1, M, w.e, w.thr, huber_delta,
                                           w.trial_partial);
        count_launch();
        k_ba_sum<<<1, 256, 0, s>>>(w.trial_partial, nt, w.trial_total);
        count_launch();
        k_ba_accept<<<1, 32, 0, s>>>(w.trial_total, w.cost_cur, 1, 0, w.pose_t, nullptr, w.fl_t, pose, nullptr,
                                     w.fl_t, lam, nu, history, w.iter);
        count_launch();
    }
    cudaMemcpyAsync(failed, w.fail, sizeof(int), cudaMemcpyDeviceToDevice, s);
    GS_CUDA_CHECK_LAUNCH();
    return GS_OK;
}

