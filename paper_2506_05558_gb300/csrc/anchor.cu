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

// ---------------------------------------------------------------------------
// Merging at an anchor (Sec. 4.4): a random 1/(k+1) of the too-fine Gaussians
// each absorb their k nearest too-fine neighbours.
//
// Selection: Philox counter (i, 0, 2, 0). Neighbour search: the candidates
// (too fine, not selected) are radix-sorted by a 31-bit hash of their grid
// cell (cell size = the search radius), so every point within the radius of a
// query lies in one of the 27 cells around it; each of those cells' hash is
// found by binary search and every entry is distance-checked, which makes hash
// collisions harmless. Claims: a candidate proposed by several selected
// Gaussians goes to the lowest index (atomicMin, order-independent). Merge:
// moment matching with weights opacity x (product of the two largest scales),
// covariance eigen-decomposed by cyclic Jacobi rotations.
// ---------------------------------------------------------------------------
constexpr int kMergeMaxK = 8;

__device__ __forceinline__ uint32_t cell_hash(int cx, int cy, int cz) {
    return ((uint32_t)cx * 73856093u ^ (uint32_t)cy * 19349663u ^ (uint32_t)cz * 83492791u) & 0x7FFFFFFFu;
}

__device__ __forceinline__ int cell_coord(float v, float inv_h) {
    return (int)fminf(fmaxf(floorf(v * inv_h), -1.0e9f), 1.0e9f);
}

__global__ void k_merge_select(const float4* __restrict__ mean_opa, const uint8_t* __restrict__ too_fine, int64_t n,
                               uint2 key, float thresh, float inv_h, uint32_t* __restrict__ sel,
                               uint32_t* __restrict__ hkey, uint32_t* __restrict__ hval) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool fine = too_fine[i] != 0;
    const float u = philox_u24(philox4x32_10(make_uint4((uint32_t)i, 0u, 2u, 0u), key).x);
    const bool s = fine && u < thresh;
    sel[i] = s ? 1u : 0u;
    uint32_t h = 0xFFFFFFFFu;  // not a candidate: sorts after every cell hash
    if (fine && !s) {
        const float4 m = mean_opa[i];
        h = cell_hash(cell_coord(m.x, inv_h), cell_coord(m.y, inv_h), cell_coord(m.z, inv_h));
    }
    hkey[i] = h;
    hval[i] = (uint32_t)i;
}

__device__ __forceinline__ int64_t lower_bound_u32(const uint32_t* __restrict__ a, int64_t n, uint32_t v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void k_merge_knn(const float4* __restrict__ mean_opa, const uint32_t* __restrict__ sel, int64_t n,
                            const uint32_t* __restrict__ skey, const uint32_t* __restrict__ sval, float radius,
                            int k, int32_t* __restrict__ prop) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !sel[i]) return;
    const float4 m = mean_opa[i];
    const float inv_h = 1.f / radius, r2 = radius * radius;
    const int cx = cell_coord(m.x, inv_h), cy = cell_coord(m.y, inv_h), cz = cell_coord(m.z, inv_h);
    float bd[kMergeMaxK];
    int32_t bi[kMergeMaxK];
    for (int t = 0; t < k; t++) { bd[t] = INFINITY; bi[t] = -1; }
    for (int dz = -1; dz <= 1; dz++)
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                const uint32_t h = cell_hash(cx + dx, cy + dy, cz + dz);
                for (int64_t j = lower_bound_u32(skey, n, h); j < n && skey[j] == h; j++) {
                    const int32_t c = (int32_t)sval[j];
                    const float4 q = mean_opa[c];
                    const float ex = q.x - m.x, ey = q.y - m.y, ez = q.z - m.z;
                    const float d2 = ex * ex + ey * ey + ez * ez;
                    if (!(d2 <= r2)) continue;
                    bool dup = false;  // a colliding hash may list a cell twice
                    for (int t = 0; t < k; t++) dup |= bi[t] == c;
                    if (dup) continue;
                    // insert into the sorted top-k by (distance, index)
                    int t = k - 1;
                    if (!(d2 < bd[t] || (d2 == bd[t] && c < bi[t]))) continue;
                    while (t > 0 && (d2 < bd[t - 1] || (d2 == bd[t - 1] && c < bi[t - 1]))) {
                        bd[t] = bd[t - 1];
                        bi[t] = bi[t - 1];
                        t--;
                    }
                    bd[t] = d2;
                    bi[t] = c;
                }
            }
    for (int t = 0; t < k; t++) prop[i * k + t] = bi[t];
}

__global__ void k_merge_claim(const uint32_t* __restrict__ sel, const int32_t* __restrict__ prop, int64_t n, int k,
                              uint32_t* __restrict__ claim) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !sel[i]) return;
    for (int t = 0; t < k; t++) {
        const int32_t c = prop[i * k + t];
        if (c >= 0) atomicMin(&claim[c], (uint32_t)i);
    }
}

__global__ void k_merge_keep(const uint32_t* __restrict__ claim, int64_t n, uint32_t* __restrict__ keep) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) keep[i] = claim[i] == 0xFFFFFFFFu ? 1u : 0u;
}

// Eigen-decomposition of a symmetric 3x3 matrix by cyclic Jacobi rotations:
// A = V diag(lam) V^T, V orthonormal (columns = eigenvectors).
__device__ void eig_sym3(float A[3][3], float lam[3], float V[3][3]) {
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) V[r][c] = r == c ? 1.f : 0.f;
    const int P[3] = {0, 0, 1}, Q[3] = {1, 2, 2};
    for (int sweep = 0; sweep < 10; sweep++) {
        const float off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        const float diag = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
        if (off <= 1e-14f * diag) break;
        for (int e = 0; e < 3; e++) {
            const int p = P[e], q = Q[e];
            const float apq = A[p][q];
            if (fabsf(apq) <= 1e-30f) continue;
            // rotation angle zeroing A[p][q]: t = tan(phi) from cot(2 phi) = (A_qq - A_pp) / (2 A_pq)
            const float theta = (A[q][q] - A[p][p]) / (2.f * apq);
            const float t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
            const float c = rsqrtf(t * t + 1.f), s = t * c;
            for (int k = 0; k < 3; k++) {  // columns p, q of A J
                const float akp = A[k][p], akq = A[k][q];
                A[k][p] = c * akp - s * akq;
                A[k][q] = s * akp + c * akq;
            }
            for (int k = 0; k < 3; k++) {  // rows p, q of J^T (A J)
                const float apk = A[p][k], aqk = A[q][k];
                A[p][k] = c * apk - s * aqk;
                A[q][k] = s * apk + c * aqk;
            }
            for (int k = 0; k < 3; k++) {
                const float vkp = V[k][p], vkq = V[k][q];
                V[k][p] = c * vkp - s * vkq;
                V[k][q] = s * vkp + c * vkq;
            }
        }
    }
    for (int k = 0; k < 3; k++) lam[k] = A[k][k];
}

// Unit quaternion (w, x, y, z) of a rotation matrix, from its largest
// diagonal combination (numerically stable for every rotation).
__device__ float4 rot_to_quat(const float R[3][3]) {
    const float tr = R[0][0] + R[1][1] + R[2][2];
    float4 q;
    if (tr > fmaxf(R[0][0], fmaxf(R[1][1], R[2][2]))) {
        const float w = 0.5f * sqrtf(fmaxf(1.f + tr, 0.f)), f = 0.25f / w;
        q = make_float4(w, (R[2][1] - R[1][2]) * f, (R[0][2] - R[2][0]) * f, (R[1][0] - R[0][1]) * f);
    } else if (R[0][0] >= R[1][1] && R[0][0] >= R[2][2]) {
        const float x = 0.5f * sqrtf(fmaxf(1.f + R[0][0] - R[1][1] - R[2][2], 0.f)), f = 0.25f / x;
        q = make_float4((R[2][1] - R[1][2]) * f, x, (R[0][1] + R[1][0]) * f, (R[0][2] + R[2][0]) * f);
    } else if (R[1][1] >= R[2][2]) {
        const float y = 0.5f * sqrtf(fmaxf(1.f - R[0][0] + R[1][1] - R[2][2], 0.f)), f = 0.25f / y;
        q = make_float4((R[0][2] - R[2][0]) * f, (R[0][1] + R[1][0]) * f, y, (R[1][2] + R[2][1]) * f);
    } else {
        const float z = 0.5f * sqrtf(fmaxf(1.f - R[0][0] - R[1][1] + R[2][2], 0.f)), f = 0.25f / z;
        q = make_float4((R[1][0] - R[0][1]) * f, (R[0][2] + R[2][0]) * f, (R[1][2] + R[2][1]) * f, z);
    }
    return q;
}

__device__ void quat_rot(float4 q, float R[3][3]) {
    const float n = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    const float w = q.x * n, x = q.y * n, y = q.z * n, z = q.w * n;
    R[0][0] = 1.f - 2.f * (y * y + z * z); R[0][1] = 2.f * (x * y - w * z); R[0][2] = 2.f * (x * z + w * y);
    R[1][0] = 2.f * (x * y + w * z); R[1][1] = 1.f - 2.f * (x * x + z * z); R[1][2] = 2.f * (y * z - w * x);
    R[2][0] = 2.f * (x * z - w * y); R[2][1] = 2.f * (y * z + w * x); R[2][2] = 1.f - 2.f * (x * x + y * y);
}

__device__ __forceinline__ float merge_weight(float4 mo, float4 sc) {
    const float o = 1.f / (1.f + expf(-mo.w));
    const float a = expf(sc.x), b = expf(sc.y), c = expf(sc.z);
    return o * (a * b * c / fminf(a, fminf(b, c)));  // opacity x product of the two largest scales
}

__global__ void k_merge_write(const float4* __restrict__ mo_in, const float4* __restrict__ sc_in,
                              const float4* __restrict__ q_in, const float4* __restrict__ sh_in,
                              const float4* __restrict__ m_mo, const float4* __restrict__ m_sc,
                              const float4* __restrict__ m_q, const float4* __restrict__ m_sh,
                              const float4* __restrict__ v_mo, const float4* __restrict__ v_sc,
                              const float4* __restrict__ v_q, const float4* __restrict__ v_sh,
                              const uint32_t* __restrict__ sel, const int32_t* __restrict__ prop,
                              const uint32_t* __restrict__ claim, const uint32_t* __restrict__ keep,
                              const uint32_t* __restrict__ pos, int64_t n, int k, const float* __restrict__ lr_in,
                              float* __restrict__ lr_out, float4* __restrict__ o_mo,
                              float4* __restrict__ o_sc, float4* __restrict__ o_q, float4* __restrict__ o_sh,
                              float4* __restrict__ om_mo, float4* __restrict__ om_sc, float4* __restrict__ om_q,
                              float4* __restrict__ om_sh, float4* __restrict__ ov_mo, float4* __restrict__ ov_sc,
                              float4* __restrict__ ov_q, float4* __restrict__ ov_sh) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !keep[i]) return;
    const int64_t o = pos[i];
    const bool moments = om_mo != nullptr;
    if (lr_out) lr_out[o] = sel[i] ? 1.f : lr_in[i];  // a merged Gaussian is a new primitive
    if (!sel[i]) {  // unchanged, with its optimiser state
        o_mo[o] = mo_in[i]; o_sc[o] = sc_in[i]; o_q[o] = q_in[i];
        for (int r = 0; r < 12; r++) o_sh[12 * o + r] = sh_in[12 * i + r];
        if (moments) {
            om_mo[o] = m_mo[i]; om_sc[o] = m_sc[i]; om_q[o] = m_q[i];
            ov_mo[o] = v_mo[i]; ov_sc[o] = v_sc[i]; ov_q[o] = v_q[i];
            for (int r = 0; r < 12; r++) { om_sh[12 * o + r] = m_sh[12 * i + r]; ov_sh[12 * o + r] = v_sh[12 * i + r]; }
        }
        return;
    }
    int64_t grp[kMergeMaxK + 1];
    int g = 0;
    grp[g++] = i;
    for (int t = 0; t < k; t++) {
        const int32_t c = prop[i * k + t];
        if (c >= 0 && claim[c] == (uint32_t)i) grp[g++] = c;
    }
    // weighted mean, then second moment about it
    float W = 0.f, mx = 0.f, my = 0.f, mz = 0.f;
    for (int j = 0; j < g; j++) {
        const float4 a = mo_in[grp[j]];
        const float w = merge_weight(a, sc_in[grp[j]]);
        W += w; mx += w * a.x; my += w * a.y; mz += w * a.z;
    }
    mx /= W; my /= W; mz /= W;
    float C[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    for (int j = 0; j < g; j++) {
        const float4 a = mo_in[grp[j]], sc = sc_in[grp[j]];
        const float w = merge_weight(a, sc);
        float R[3][3];
        quat_rot(q_in[grp[j]], R);
        const float s2[3] = {expf(2.f * sc.x), expf(2.f * sc.y), expf(2.f * sc.z)};
        const float d[3] = {a.x - mx, a.y - my, a.z - mz};
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++)
                C[r][c] += w * (R[r][0] * s2[0] * R[c][0] + R[r][1] * s2[1] * R[c][1] + R[r][2] * s2[2] * R[c][2] +
                                d[r] * d[c]);
    }
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) C[r][c] /= W;
    float lam[3], V[3][3];
    eig_sym3(C, lam, V);
    const float det = V[0][0] * (V[1][1] * V[2][2] - V[1][2] * V[2][1]) -
                      V[0][1] * (V[1][0] * V[2][2] - V[1][2] * V[2][0]) +
                      V[0][2] * (V[1][0] * V[2][1] - V[1][1] * V[2][0]);
    if (det < 0.f)
        for (int r = 0; r < 3; r++) V[r][2] = -V[r][2];
    const float sd[3] = {sqrtf(fmaxf(lam[0], 1e-30f)), sqrtf(fmaxf(lam[1], 1e-30f)), sqrtf(fmaxf(lam[2], 1e-30f))};
    const float area = sd[0] * sd[1] * sd[2] / fminf(sd[0], fminf(sd[1], sd[2]));
    const float op = fminf(0.99f, W / area);
    o_mo[o] = make_float4(mx, my, mz, logf(op / (1.f - op)));
    o_sc[o] = make_float4(logf(sd[0]), logf(sd[1]), logf(sd[2]), 0.f);
    o_q[o] = rot_to_quat(V);
    for (int r = 0; r < 12; r++) {
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int j = 0; j < g; j++) {
            const float w = merge_weight(mo_in[grp[j]], sc_in[grp[j]]);
            const float4 v = sh_in[12 * grp[j] + r];
            acc.x += w * v.x; acc.y += w * v.y; acc.z += w * v.z; acc.w += w * v.w;
        }
        o_sh[12 * o + r] = make_float4(acc.x / W, acc.y / W, acc.z / W, acc.w / W);
    }
    if (moments) {  // a new primitive starts with fresh optimiser state
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        om_mo[o] = z; om_sc[o] = z; om_q[o] = z; ov_mo[o] = z; ov_sc[o] = z; ov_q[o] = z;
        for (int r = 0; r < 12; r++) { om_sh[12 * o + r] = z; ov_sh[12 * o + r] = z; }
    }
}

__global__ void k_merge_count(const uint32_t* total, int64_t* n_out) { *n_out = *total; }

__global__ void k_cull_keep(const float4* __restrict__ mean_opa, int64_t n, float min_opacity,
                            uint32_t* __restrict__ keep) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) keep[i] = 1.f / (1.f + expf(-mean_opa[i].w)) >= min_opacity ? 1u : 0u;
}

// Copies the kept rows (and, when given, their Adam moments and rate
// multipliers) to their compacted positions.
__global__ void k_compact_rows(const uint32_t* __restrict__ keep, const uint32_t* __restrict__ pos, int64_t n,
                               const float4* __restrict__ mo, const float4* __restrict__ sc,
                               const float4* __restrict__ q, const float4* __restrict__ sh,
                               const float4* __restrict__ m_mo, const float4* __restrict__ m_sc,
                               const float4* __restrict__ m_q, const float4* __restrict__ m_sh,
                               const float4* __restrict__ v_mo, const float4* __restrict__ v_sc,
                               const float4* __restrict__ v_q, const float4* __restrict__ v_sh,
                               const float* __restrict__ lr_in, float4* __restrict__ o_mo, float4* __restrict__ o_sc,
                               float4* __restrict__ o_q, float4* __restrict__ o_sh, float4* __restrict__ om_mo,
                               float4* __restrict__ om_sc, float4* __restrict__ om_q, float4* __restrict__ om_sh,
                               float4* __restrict__ ov_mo, float4* __restrict__ ov_sc, float4* __restrict__ ov_q,
                               float4* __restrict__ ov_sh, float* __restrict__ lr_out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !keep[i]) return;
    const int64_t o = pos[i];
    o_mo[o] = mo[i]; o_sc[o] = sc[i]; o_q[o] = q[i];
    for (int r = 0; r < 12; r++) o_sh[12 * o + r] = sh[12 * i + r];
    if (om_mo) {
        om_mo[o] = m_mo[i]; om_sc[o] = m_sc[i]; om_q[o] = m_q[i];
        ov_mo[o] = v_mo[i]; ov_sc[o] = v_sc[i]; ov_q[o] = v_q[i];
        for (int r = 0; r < 12; r++) { om_sh[12 * o + r] = m_sh[12 * i + r]; ov_sh[12 * o + r] = v_sh[12 * i + r]; }
    }
    if (lr_out) lr_out[o] = lr_in[i];
}

__global__ void k_scale_opacity(float4* __restrict__ mean_opa, int64_t n, float w) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 m = mean_opa[i];
    const float o = w / (1.f + expf(-m.w));
    m.w = logf(o / (1.f - o));
    mean_opa[i] = m;
}

struct MergeWs {
    uint32_t *sel, *k0, *v0, *k1, *v1, *hist, *claim, *keep, *pos, *total;
    int32_t* prop;
    void* scan;
};

static MergeWs carve_merge(char* base, size_t cap, int64_t n, int k, size_t* used) {
    Carve c{base, 0, cap};
    MergeWs w;
    w.sel = c.take<uint32_t>(n);
    w.k0 = c.take<uint32_t>(n);
    w.v0 = c.take<uint32_t>(n);
    w.k1 = c.take<uint32_t>(n);
    w.v1 = c.take<uint32_t>(n);
    w.hist = c.take<uint32_t>(256 * radix_blocks(n));
    const int64_t sn = 256 * radix_blocks(n) > n ? 256 * radix_blocks(n) : n;
    w.scan = c.take<char>(scan_workspace_bytes(sn));
    w.prop = c.take<int32_t>(n * k);
    w.claim = c.take<uint32_t>(n);
    w.keep = c.take<uint32_t>(n);
    w.pos = c.take<uint32_t>(n);
    w.total = c.take<uint32_t>(4);
    *used = c.used;
    return w;
}

}  // namespace gs

using namespace gs;

extern "C" float gs_anchor_blend_weight(float d1, float d2, float overlap) {
    if (!(d1 >= 0.f) || !(d2 >= d1) || !(d2 > 0.f) || !(overlap > 0.f) || !(overlap < 0.5f)) return NAN;
    const float r = d1 / d2;
    return r < 1.f - overlap ? 1.f : 1.f - (r - (1.f - overlap)) * 0.5f / overlap;
}

extern "C" int gs_scale_opacity(float* mean_opa, int64_t n, float w, void* stream) {
    if (!mean_opa || n < 0 || !(w >= 0.f) || !(w <= 1.f)) return GS_ERR_INVALID_ARG;
    if (n > 0) {
        k_scale_opacity<<<(unsigned)ceil_div(n, 256), 256, 0, (cudaStream_t)stream>>>((float4*)mean_opa, n, w);
        count_launch();
    }
    GS_CUDA_CHECK_LAUNCH();
    return GS_OK;
}

extern "C" size_t gs_cull_opacity_workspace_size(int64_t n) {
    if (n < 0) return 0;
    Carve c{nullptr, 0, 0};
    c.take<uint32_t>(n);
    c.take<uint32_t>(n);
    c.take<uint32_t>(4);
    c.take<char>(scan_workspace_bytes(n));
    return c.used;
}

extern "C" int gs_cull_opacity(const gs_gaussians* in, const gs_gaussians* m_in, const gs_gaussians* v_in,
                               const float* lr_in, float min_opacity, const gs_gaussians* out,
                               const gs_gaussians* m_out, const gs_gaussians* v_out, float* lr_out, int64_t* n_out,
                               void* ws, size_t ws_bytes, void* stream) {
    auto ok = [](const gs_gaussians* g) { return g && g->mean_opa && g->scale && g->quat && g->sh; };
    if (!ok(in) || !ok(out) || !n_out || in->n < 0 || out->n < in->n || !(min_opacity >= 0.f) ||
        in->n > (int64_t)UINT32_MAX || !lr_in != !lr_out)
        return GS_ERR_INVALID_ARG;
    const bool moments = m_in || v_in || m_out || v_out;
    if (moments && !(ok(m_in) && ok(v_in) && ok(m_out) && ok(v_out) && m_in->n == in->n && v_in->n == in->n &&
                     m_out->n >= in->n && v_out->n >= in->n))
        return GS_ERR_INVALID_ARG;
    const int64_t n = in->n;
    Carve c{(char*)ws, 0, ws_bytes};
    uint32_t* keep = c.take<uint32_t>(n);
    uint32_t* pos = c.take<uint32_t>(n);
    uint32_t* total = c.take<uint32_t>(4);
    void* scan_ws = c.take<char>(scan_workspace_bytes(n));
    if (!ws || !c.ok() || ((uintptr_t)ws & 255)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        cudaMemsetAsync(n_out, 0, sizeof(int64_t), s);
        GS_CUDA_CHECK_LAUNCH();
        return GS_OK;
    }
    const unsigned nb = (unsigned)ceil_div(n, 256);
    k_cull_keep<<<nb, 256, 0, s>>>((const float4*)in->mean_opa, n, min_opacity, keep);
    count_launch();
    scan_exclusive_u32(keep, pos, n, total, scan_ws, s);
    auto f4 = [](const gs_gaussians* g, int f) -> const float4* {
        if (!g) return nullptr;
        return (const float4*)(f == 0 ? g->mean_opa : f == 1 ? g->scale : f == 2 ? g->quat : g->sh);
    };
    auto o4 = [](const gs_gaussians* g, int f) -> float4* {
        if (!g) return nullptr;
        return (float4*)(f == 0 ? g->mean_opa : f == 1 ? g->scale : f == 2 ? g->quat : g->sh);
    };
    k_compact_rows<<<nb, 256, 0, s>>>(keep, pos, n, f4(in, 0), f4(in, 1), f4(in, 2), f4(in, 3), f4(m_in, 0),
                                      f4(m_in, 1), f4(m_in, 2), f4(m_in, 3), f4(v_in, 0), f4(v_in, 1), f4(v_in, 2),
                                      f4(v_in, 3), lr_in, o4(out, 0), o4(out, 1), o4(out, 2), o4(out, 3),
                                      o4(m_out, 0), o4(m_out, 1), o4(m_out, 2), o4(m_out, 3), o4(v_out, 0),
                                      o4(v_out, 1), o4(v_out, 2), o4(v_out, 3), lr_out);
    count_launch();
    k_merge_count<<<1, 1, 0, s>>>(total, n_out);
    count_launch();
    GS_CUDA_CHECK_LAUNCH();
    return GS_OK;
}

extern "C" size_t gs_anchor_merge_workspace_size(int64_t n, int32_t k) {
    if (n < 0 || k < 1 || k > kMergeMaxK) return 0;
    size_t used = 0;
    carve_merge(nullptr, 0, n, k, &used);
    return used;
}

static bool set_ok(const gs_gaussians* g) { return g && g->mean_opa && g->scale && g->quat && g->sh; }

extern "C" int gs_anchor_merge(const gs_gaussians* in, const gs_gaussians* m_in, const gs_gaussians* v_in,
                               const float* lr_in, const uint8_t* too_fine, float radius, int32_t k, uint64_t seed,
                               const gs_gaussians* out, const gs_gaussians* m_out, const gs_gaussians* v_out,
                               float* lr_out, int64_t* n_out, void* ws, size_t ws_bytes, void* stream) {
    if (!set_ok(in) || !set_ok(out) || !too_fine || !n_out || in->n < 0 || out->n < in->n || !(radius > 0.f) ||
        k < 1 || k > kMergeMaxK || in->n > (int64_t)INT32_MAX)
        return GS_ERR_INVALID_ARG;
    const bool moments = m_in || v_in || m_out || v_out;
    if (moments && !(set_ok(m_in) && set_ok(v_in) && set_ok(m_out) && set_ok(v_out) && m_in->n == in->n &&
                     v_in->n == in->n && m_out->n >= in->n && v_out->n >= in->n))
        return GS_ERR_INVALID_ARG;
    if (!lr_in != !lr_out) return GS_ERR_INVALID_ARG;
    const int64_t n = in->n;
    size_t need = 0;
    MergeWs w = carve_merge((char*)ws, ws_bytes, n, k, &need);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        cudaMemsetAsync(n_out, 0, sizeof(int64_t), s);
        GS_CUDA_CHECK_LAUNCH();
        return GS_OK;
    }
    const unsigned nb = (unsigned)ceil_div(n, 256);
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    k_merge_select<<<nb, 256, 0, s>>>((const float4*)in->mean_opa, too_fine, n, key, 1.f / (float)(k + 1),
                                      1.f / radius, w.sel, w.k0, w.v0);
    count_launch();
    const bool in1 = radix_sort_pairs(w.k0, w.v0, w.k1, w.v1, n, nullptr, 32, w.hist, w.scan, s, false);
    const uint32_t* skey = in1 ? w.k1 : w.k0;
    const uint32_t* sval = in1 ? w.v1 : w.v0;
    k_merge_knn<<<nb, 256, 0, s>>>((const float4*)in->mean_opa, w.sel, n, skey, sval, radius, k, w.prop);
    count_launch();
    cudaMemsetAsync(w.claim, 0xFF, sizeof(uint32_t) * n, s);
    k_merge_claim<<<nb, 256, 0, s>>>(w.sel, w.prop, n, k, w.claim);
    count_launch();
    k_merge_keep<<<nb, 256, 0, s>>>(w.claim, n, w.keep);
    count_launch();
    scan_exclusive_u32(w.keep, w.pos, n, w.total, w.scan, s);
    auto f4 = [](const float* p) { return (const float4*)p; };
    auto o4 = [](float* p) { return (float4*)p; };
    k_merge_write<<<nb, 256, 0, s>>>(
        f4(in->mean_opa), f4(in->scale), f4(in->quat), f4(in->sh), moments ? f4(m_in->mean_opa) : nullptr,
        moments ? f4(m_in->scale) : nullptr, moments ? f4(m_in->quat) : nullptr, moments ? f4(m_in->sh) : nullptr,
        moments ? f4(v_in->mean_opa) : nullptr, moments ? f4(v_in->scale) : nullptr,
        moments ? f4(v_in->quat) : nullptr, moments ? f4(v_in->sh) : nullptr, w.sel, w.prop, w.claim, w.keep, w.pos,
        n, k, lr_in, lr_out, o4(out->mean_opa), o4(out->scale), o4(out->quat), o4(out->sh),
        moments ? o4(m_out->mean_opa) : nullptr, moments ? o4(m_out->scale) : nullptr,
        moments ? o4(m_out->quat) : nullptr, moments ? o4(m_out->sh) : nullptr,
        moments ? o4(v_out->mean_opa) : nullptr, moments ? o4(v_out->scale) : nullptr,
        moments ? o4(v_out->quat) : nullptr, moments ? o4(v_out->sh) : nullptr);
    count_launch();
    k_merge_count<<<1, 1, 0, s>>>(w.total, n_out);
    count_launch();
    GS_CUDA_CHECK_LAUNCH();
    return GS_OK;
}

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
