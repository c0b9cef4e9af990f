// Adjoint of the projection (K7) and the per-view pose reduction.
//
// A CTA holds 32 Gaussians (one per lane) and up to 8 views (one per warp).
// Each warp sums its (view, Gaussian) items' pair partials (contiguous
// emission slots written by the compositing adjoint), recomputes the
// projection, applies the chain rule and leaves per item in shared memory the
// 12 geometry gradients, a visibility mark, the clamp-masked colour gradient
// (3) and the 16 SH basis values. The views are then summed in a fixed order;
// the SH coefficient gradients are formed there as sum_v gc_v[ch] Y_v[k], so
// the per-item record is 32 values instead of 64. Each gradient row is
// written once, without atomics. Each view's pose gradient is reduced per CTA
// in a fixed order and then across CTAs by k_pose_reduce: the whole backward
// pass is deterministic.
#include "common.cuh"
#include "sh.cuh"

namespace gs {

constexpr int kPBGauss = 32;                   // Gaussians per CTA group, one per lane
constexpr int kPBWarps = 8;                    // views processed at once, one per warp
constexpr int kPBThreads = kPBGauss * kPBWarps;
// per-item record: 0-3 mean xyz + opacity logit, 4-7 log-scale xyz + 0, 8-11
// quaternion, 12 visible, 13-15 clamp-masked colour gradient, 16-31 SH basis
constexpr int kSlots = 32;
constexpr int kSlotVis = 12, kSlotGc = 13, kSlotY = 16;
constexpr int kSlotPitch = kPBGauss + 1;       // +1 word: conflict-free column access
// output values per Gaussian: 12 geometry, visible, 48 SH coefficient gradients
constexpr int kOut = 61;
constexpr int kAcc = (kOut * kPBGauss + kPBThreads - 1) / kPBThreads;
constexpr size_t kPBSmem = sizeof(float) * kPBWarps * kSlots * kSlotPitch;

// Output value o (0..60) of lane gl, summed over warps w0 .. w0 + nw - 1 of the
// slot array in a fixed order.
__device__ __forceinline__ float out_value(const float* s_slot, int w0, int nw, int o, int gl) {
    float a = 0.f;
    if (o <= kSlotVis) {
        for (int w = w0; w < w0 + nw; w++) a += s_slot[(w * kSlots + o) * kSlotPitch + gl];
    } else {
        const int c = o - (kSlotVis + 1), k = c / 3, ch = c - 3 * k;
        for (int w = w0; w < w0 + nw; w++)
            a += s_slot[(w * kSlots + kSlotGc + ch) * kSlotPitch + gl] *
                 s_slot[(w * kSlots + kSlotY + k) * kSlotPitch + gl];
    }
    return a;
}

__global__ void __launch_bounds__(kPBThreads, 3) k_project_bwd(
    const float4* __restrict__ mean_opa, const float4* __restrict__ scale, const float4* __restrict__ quat,
    const float4* __restrict__ sh, int64_t n, const gs_camera* __restrict__ cams, gs_frame f, gs_config cfg,
    const int32_t* __restrict__ n_tiles, const uint32_t* __restrict__ offset, const float4* __restrict__ part0,
    const float4* __restrict__ part1, const float* __restrict__ part2, int64_t capacity,
    float4* __restrict__ g_mean_opa, float4* __restrict__ g_scale, float4* __restrict__ g_quat,
    float4* __restrict__ g_sh, uint8_t* __restrict__ visible, float* __restrict__ d_proj,
    float* __restrict__ pose_part) {
    extern __shared__ float s_slot[];  // [kPBWarps][kSlots][kSlotPitch]
    __shared__ gs_camera s_cam[GS_MAX_VIEWS];
    const unsigned FULL = 0xffffffffu;
    const int nv = f.n_views;
    for (int i = threadIdx.x; i < nv * (int)(sizeof(gs_camera) / 4); i += kPBThreads)
        reinterpret_cast<float*>(s_cam)[i] = reinterpret_cast<const float*>(cams)[i];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // With fewer than 8 views the CTA takes several groups of 32 Gaussians:
    // warp w handles group w / nvw and, each round, view round * nvw + w % nvw.
    const int nvw = nv < kPBWarps ? nv : kPBWarps;
    const int G = kPBWarps / nvw;
    const int group = w / nvw, vw = w % nvw;
    const int64_t gi = (int64_t)blockIdx.x * G + group;  // global group index
    const int64_t n_groups = ceil_div(n, kPBGauss);
    const int64_t g = gi * kPBGauss + lane;
    const bool valid = group < G && g < n;
    float4 mo = make_float4(0.f, 0.f, 0.f, 0.f), s4 = mo, q4 = make_float4(1.f, 0.f, 0.f, 0.f);
    if (valid) { mo = mean_opa[g]; s4 = scale[g]; q4 = quat[g]; }
    // parameter-space quantities shared by all views
    const float qi = rsqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
    const float qw = q4.x * qi, qx = q4.y * qi, qy = q4.z * qi, qz = q4.w * qi;
    float Rq[9];
    Rq[0] = 1.f - 2.f * (qy * qy + qz * qz); Rq[1] = 2.f * (qx * qy - qw * qz); Rq[2] = 2.f * (qx * qz + qw * qy);
    Rq[3] = 2.f * (qx * qy + qw * qz); Rq[4] = 1.f - 2.f * (qx * qx + qz * qz); Rq[5] = 2.f * (qy * qz - qw * qx);
    Rq[6] = 2.f * (qx * qz - qw * qy); Rq[7] = 2.f * (qy * qz + qw * qx); Rq[8] = 1.f - 2.f * (qx * qx + qy * qy);
    const float sv[3] = {expf(s4.x), expf(s4.y), expf(s4.z)};
    const float opa = 1.f / (1.f + expf(-mo.w));
    const int ncoef = (cfg.sh_degree + 1) * (cfg.sh_degree + 1);
    float* col = s_slot + (w * kSlots) * kSlotPitch + lane;  // this item's record
    auto put = [&](int c, float v) { col[c * kSlotPitch] = v; };
    // G == 1 (8 views or more): thread t accumulates output values t + 256 i over rounds
    float acc[kAcc];
#pragma unroll
    for (int i = 0; i < kAcc; i++) acc[i] = 0.f;
    __syncthreads();

    for (int v0 = 0; v0 < nv; v0 += nvw) {
        const int v = v0 + vw;
        const int64_t item = (int64_t)v * n + g;
        const int nt = (valid && v < nv) ? n_tiles[item] : 0;
        float pose[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (nt <= 0) {
#pragma unroll 4
            for (int c = 0; c < kSlots; c++) put(c, 0.f);  // all of it: 0 x stale data could be NaN
        } else {
            const gs_camera& c = s_cam[v];
            // the SH rows are needed after the partial sums: start fetching them into L2 now
            const float4* shg = sh + 12 * g;
            if (ncoef > 1) {
                asm volatile("prefetch.global.L2 [%0];" ::"l"(shg));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(shg + 6));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(shg + 11));
            }
            // 1. sum this item's pair partials (contiguous emission slots)
            const uint32_t off = offset[item];
            float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
            float a2 = 0.f;
            // slots past the pair buffer's capacity were never written (overflowed sort)
            const int run = (int)max((int64_t)0, min((int64_t)nt, capacity - (int64_t)off));
            const float4* q0 = part0 + off;
            const float4* q1 = part1 + off;
            const float* q2 = part2 + off;
            int k = 0;
            for (; k + 4 <= run; k += 4) {  // four pairs' loads in flight, summed in slot order
                float4 p0[4], p1[4];
                float p2[4];
#pragma unroll
                for (int u = 0; u < 4; u++) { p0[u] = q0[k + u]; p1[u] = q1[k + u]; p2[u] = q2[k + u]; }
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    a0.x += p0[u].x; a0.y += p0[u].y; a0.z += p0[u].z; a0.w += p0[u].w;
                    a1.x += p1[u].x; a1.y += p1[u].y; a1.z += p1[u].z; a1.w += p1[u].w;
                    a2 += p2[u];
                }
            }
            for (; k < run; k++) {
                const float4 p0 = q0[k], p1 = q1[k];
                a0.x += p0.x; a0.y += p0.y; a0.z += p0.z; a0.w += p0.w;
                a1.x += p1.x; a1.y += p1.y; a1.z += p1.z; a1.w += p1.w;
                a2 += q2[k];
            }
            const float du = a0.x, dv = a0.y, dA = a0.z, dB = a0.w, dC = a1.x, dop = a1.y;
            const float dr = a1.z, dg = a1.w, db = a2;
            if (d_proj) {
                float* o = d_proj + 9 * item;
                o[0] = du; o[1] = dv; o[2] = dA; o[3] = dB; o[4] = dC; o[5] = dop; o[6] = dr; o[7] = dg; o[8] = db;
            }

            // 2. colour: rgb = max(0.5 + sum_k Y_k(d) sh_k, 0), d = (mu - centre)/|mu - centre|
            const float ccx = -(c.R[0] * c.t[0] + c.R[3] * c.t[1] + c.R[6] * c.t[2]);
            const float ccy = -(c.R[1] * c.t[0] + c.R[4] * c.t[1] + c.R[7] * c.t[2]);
            const float ccz = -(c.R[2] * c.t[0] + c.R[5] * c.t[1] + c.R[8] * c.t[2]);
            float ddx = mo.x - ccx, ddy = mo.y - ccy, ddz = mo.z - ccz;
            const float il = rsqrtf(ddx * ddx + ddy * ddy + ddz * ddz);
            ddx *= il; ddy *= il; ddz *= il;
            float gc[3];
            {
                float Y[16];
                sh_eval_basis(cfg.sh_degree, ddx, ddy, ddz, Y);
                float raw0 = 0.5f, raw1 = 0.5f, raw2 = 0.5f;
#pragma unroll
                for (int r = 0; r < 12; r++) {
                    if (4 * r < 3 * ncoef) {
                        const float4 q = shg[r];
                        const float cq[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                        for (int u = 0; u < 4; u++) {
                            const int idx = 4 * r + u, kk = idx / 3, ch = idx % 3;
                            if (kk < ncoef) {
                                if (ch == 0) raw0 += Y[kk] * cq[u];
                                else if (ch == 1) raw1 += Y[kk] * cq[u];
                                else raw2 += Y[kk] * cq[u];
                            }
                        }
                    }
                }
                gc[0] = raw0 > 0.f ? dr : 0.f;
                gc[1] = raw1 > 0.f ? dg : 0.f;
                gc[2] = raw2 > 0.f ? db : 0.f;
#pragma unroll
                for (int kk = 0; kk < 16; kk++) put(kSlotY + kk, kk < ncoef ? Y[kk] : 0.f);
            }
            put(kSlotGc, gc[0]);
            put(kSlotGc + 1, gc[1]);
            put(kSlotGc + 2, gc[2]);
            float gmx = 0.f, gmy = 0.f, gmz = 0.f;
            if (cfg.sh_degree > 0) {
                // direction gradient of sum_k w_k Y_k(d), w_k = sum_ch gc[ch] sh[k][ch]
                float wk[16];
#pragma unroll
                for (int kk = 0; kk < 16; kk++) wk[kk] = 0.f;
#pragma unroll
                for (int r = 0; r < 12; r++) {
                    if (4 * r < 3 * ncoef) {
                        const float4 q = shg[r];
                        const float cq[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                        for (int u = 0; u < 4; u++) {
                            const int idx = 4 * r + u, kk = idx / 3, ch = idx % 3;
                            if (kk >= 1 && kk < ncoef) wk[kk] += gc[ch] * cq[u];
                        }
                    }
                }
                const float3 gd = sh_weighted_grad(cfg.sh_degree, ddx, ddy, ddz, wk);
                const float dd = gd.x * ddx + gd.y * ddy + gd.z * ddz;
                gmx = (gd.x - ddx * dd) * il; gmy = (gd.y - ddy * dd) * il; gmz = (gd.z - ddz * dd) * il;
                if (cfg.pose_grad_through_sh) {
                    // centre = -R^T t moves by -R^T rho under exp(xi^): dL/drho += R dL/ddir
                    pose[0] += c.R[0] * gmx + c.R[1] * gmy + c.R[2] * gmz;
                    pose[1] += c.R[3] * gmx + c.R[4] * gmy + c.R[5] * gmz;
                    pose[2] += c.R[6] * gmx + c.R[7] * gmy + c.R[8] * gmz;
                }
            }

            // 3. recompute the projection
            const float x = c.R[0] * mo.x + c.R[1] * mo.y + c.R[2] * mo.z + c.t[0];
            const float y = c.R[3] * mo.x + c.R[4] * mo.y + c.R[5] * mo.z + c.t[1];
            const float z = c.R[6] * mo.x + c.R[7] * mo.y + c.R[8] * mo.z + c.t[2];
            float T[9];  // R_cam Rq diag(s)
#pragma unroll
            for (int r = 0; r < 3; r++)
#pragma unroll
                for (int kk = 0; kk < 3; kk++)
                    T[3 * r + kk] =
                        (c.R[3 * r] * Rq[kk] + c.R[3 * r + 1] * Rq[3 + kk] + c.R[3 * r + 2] * Rq[6 + kk]) * sv[kk];
            const float limx = 1.3f * 0.5f * (float)c.width / c.fx;
            const float limy = 1.3f * 0.5f * (float)c.height / c.fy;
            const float iz = 1.f / z;
            const float xz = x * iz, yz = y * iz;
            const bool clx = xz < -limx || xz > limx, cly = yz < -limy || yz > limy;
            const float txz = fminf(limx, fmaxf(-limx, xz)), tyz = fminf(limy, fmaxf(-limy, yz));
            const float J00 = c.fx * iz, J02 = -c.fx * txz * iz, J11 = c.fy * iz, J12 = -c.fy * tyz * iz;
            float M0[3], M1[3];  // rows of M = J T
#pragma unroll
            for (int kk = 0; kk < 3; kk++) {
                M0[kk] = J00 * T[kk] + J02 * T[6 + kk];
                M1[kk] = J11 * T[3 + kk] + J12 * T[6 + kk];
            }
            const float Sa0 = M0[0] * M0[0] + M0[1] * M0[1] + M0[2] * M0[2];
            const float Sb = M0[0] * M1[0] + M0[1] * M1[1] + M0[2] * M1[2];
            const float Sc0 = M1[0] * M1[0] + M1[1] * M1[1] + M1[2] * M1[2];
            const float Sa = Sa0 + cfg.dilation, Sc = Sc0 + cfg.dilation;
            const float idet = 1.f / (Sa * Sc - Sb * Sb);
            const float Qa = Sc * idet, Qb = -Sb * idet, Qc = Sa * idet;
            // filter factor f = sqrt(rho), rho = det(Sigma2D) / det(Sigma2D + dil I) (1 without the filter)
            float fmip = 1.f, g_rho = 0.f, rho = 1.f;
            if (cfg.mip_filter) {
                // det Sigma2D = |M0 x M1|^2 (no cancellation for thin splats)
                const float k0 = M0[1] * M1[2] - M0[2] * M1[1], k1 = M0[2] * M1[0] - M0[0] * M1[2];
                const float k2 = M0[0] * M1[1] - M0[1] * M1[0];
                rho = (k0 * k0 + k1 * k1 + k2 * k2) * idet;
                fmip = sqrtf(rho > 1e-6f ? rho : 1e-6f);
                if (rho > 1e-6f) g_rho = dop * opa / (2.f * fmip);  // dL/drho through opacity o f
            }

            // 4. conic = S^-1: dL/dS = -Q dL/dQ Q, dL/dQ = [[dA, dB/2], [dB/2, dC]]
            const float hB = 0.5f * dB;
            const float t00 = Qa * dA + Qb * hB, t01 = Qa * hB + Qb * dC;
            const float t10 = Qb * dA + Qc * hB, t11 = Qb * hB + Qc * dC;
            // plus the filter factor's rho = ((A - dil)(C - dil) - B^2) / (A C - B^2), S = [[A, B], [B, C]]
            const float GS00 = -(t00 * Qa + t01 * Qb) + g_rho * (Sc0 - rho * Sc) * idet;
            const float GS01 = -(t00 * Qb + t01 * Qc) - g_rho * Sb * (1.f - rho) * idet;
            const float GS11 = -(t10 * Qb + t11 * Qc) + g_rho * (Sa0 - rho * Sa) * idet;
            // 5. S = M M^T + dil I: dL/dM = 2 GS M
            float GM0[3], GM1[3];
#pragma unroll
            for (int kk = 0; kk < 3; kk++) {
                GM0[kk] = 2.f * (GS00 * M0[kk] + GS01 * M1[kk]);
                GM1[kk] = 2.f * (GS01 * M0[kk] + GS11 * M1[kk]);
            }
            // 6. M = J T: dL/dJ = GM T^T (entries J00, J02, J11, J12), dL/dT = J^T GM
            const float GJ00 = GM0[0] * T[0] + GM0[1] * T[1] + GM0[2] * T[2];
            const float GJ02 = GM0[0] * T[6] + GM0[1] * T[7] + GM0[2] * T[8];
            const float GJ11 = GM1[0] * T[3] + GM1[1] * T[4] + GM1[2] * T[5];
            const float GJ12 = GM1[0] * T[6] + GM1[1] * T[7] + GM1[2] * T[8];
            float GT[9];
#pragma unroll
            for (int kk = 0; kk < 3; kk++) {
                GT[kk] = J00 * GM0[kk];
                GT[3 + kk] = J11 * GM1[kk];
                GT[6 + kk] = J02 * GM0[kk] + J12 * GM1[kk];
            }
            // 7. T = R Rq diag(s): dL/d(Rq diag s) = R^T GT -> log-scale and rotation matrix
            float gRq[9];
#pragma unroll
            for (int kk = 0; kk < 3; kk++) {
                float gsk = 0.f;
#pragma unroll
                for (int r = 0; r < 3; r++) {
                    const float h = c.R[r] * GT[kk] + c.R[3 + r] * GT[3 + kk] + c.R[6 + r] * GT[6 + kk];
                    gsk += h * Rq[3 * r + kk];
                    gRq[3 * r + kk] = h * sv[kk];
                }
                put(4 + kk, gsk * sv[kk]);
            }
            put(7, 0.f);
            // rotation matrix -> normalised quaternion -> raw quaternion
            float gq[4];
            gq[0] = 2.f * (-qz * gRq[1] + qy * gRq[2] + qz * gRq[3] - qx * gRq[5] - qy * gRq[6] + qx * gRq[7]);
            gq[1] = 2.f * (qy * gRq[1] + qz * gRq[2] + qy * gRq[3] - 2.f * qx * gRq[4] - qw * gRq[5] + qz * gRq[6] +
                           qw * gRq[7] - 2.f * qx * gRq[8]);
            gq[2] = 2.f * (-2.f * qy * gRq[0] + qx * gRq[1] + qw * gRq[2] + qx * gRq[3] + qz * gRq[5] - qw * gRq[6] +
                           qz * gRq[7] - 2.f * qy * gRq[8]);
            gq[3] = 2.f * (-2.f * qz * gRq[0] - qw * gRq[1] + qx * gRq[2] + qw * gRq[3] - 2.f * qz * gRq[4] +
                           qy * gRq[5] + qx * gRq[6] + qy * gRq[7]);
            const float qd = gq[0] * qw + gq[1] * qx + gq[2] * qy + gq[3] * qz;
            put(8, (gq[0] - qw * qd) * qi);
            put(9, (gq[1] - qx * qd) * qi);
            put(10, (gq[2] - qy * qd) * qi);
            put(11, (gq[3] - qz * qd) * qi);
            // 8. p = (x, y, z): through the 2D mean and J
            float gpx = du * c.fx * iz, gpy = dv * c.fy * iz;
            float gpz = -(du * c.fx * x + dv * c.fy * y) * iz * iz;
            gpz += -(GJ00 * c.fx + GJ11 * c.fy) * iz * iz;
            if (clx) {
                gpz += GJ02 * c.fx * txz * iz * iz;
            } else {
                gpx += -GJ02 * c.fx * iz * iz;
                gpz += 2.f * GJ02 * c.fx * x * iz * iz * iz;
            }
            if (cly) {
                gpz += GJ12 * c.fy * tyz * iz * iz;
            } else {
                gpy += -GJ12 * c.fy * iz * iz;
                gpz += 2.f * GJ12 * c.fy * y * iz * iz * iz;
            }
            // mean: p = R mu + t (plus the SH view-direction term)
            put(0, gmx + c.R[0] * gpx + c.R[3] * gpy + c.R[6] * gpz);
            put(1, gmy + c.R[1] * gpx + c.R[4] * gpy + c.R[7] * gpz);
            put(2, gmz + c.R[2] * gpx + c.R[5] * gpy + c.R[8] * gpz);
            put(3, dop * fmip * opa * (1.f - opa));
            put(kSlotVis, 1.f);
            // 9. pose, left perturbation: dp = rho + phi x p, dT = phi^ T
            pose[0] += gpx; pose[1] += gpy; pose[2] += gpz;
            pose[3] += y * gpz - z * gpy;
            pose[4] += z * gpx - x * gpz;
            pose[5] += x * gpy - y * gpx;
            // tr(T GT^T phi^): N = T GT^T, dphi = (N12 - N21, N20 - N02, N01 - N10)
            float N01 = 0.f, N10 = 0.f, N02 = 0.f, N20 = 0.f, N12 = 0.f, N21 = 0.f;
#pragma unroll
            for (int kk = 0; kk < 3; kk++) {
                N01 += T[kk] * GT[3 + kk]; N10 += T[3 + kk] * GT[kk];
                N02 += T[kk] * GT[6 + kk]; N20 += T[6 + kk] * GT[kk];
                N12 += T[3 + kk] * GT[6 + kk]; N21 += T[6 + kk] * GT[3 + kk];
            }
            pose[3] += N12 - N21;
            pose[4] += N20 - N02;
            pose[5] += N01 - N10;
        }
        // this view's pose partial over the CTA's 32 Gaussians (fixed xor tree)
#pragma unroll
        for (int c = 0; c < 6; c++)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) pose[c] += __shfl_xor_sync(FULL, pose[c], o);
        if (group < G && gi < n_groups && v < nv && lane < 6) {
            float pv = pose[0];
#pragma unroll
            for (int c = 1; c < 6; c++) pv = (lane == c) ? pose[c] : pv;
            pose_part[((int64_t)v * n_groups + gi) * 6 + lane] = pv;
        }
        __syncthreads();
        if (G == 1) {  // possibly several rounds: accumulate this round's views in registers
#pragma unroll
            for (int i = 0; i < kAcc; i++) {
                const int idx = threadIdx.x + kPBThreads * i;
                if (idx < kOut * kPBGauss) acc[i] += out_value(s_slot, 0, nvw, idx >> 5, idx & 31);
            }
            __syncthreads();
        }
    }
    if (G == 1) {  // stage the totals as [kOut][kSlotPitch] at the start of the slot array
#pragma unroll
        for (int i = 0; i < kAcc; i++) {
            const int idx = threadIdx.x + kPBThreads * i;
            if (idx < kOut * kPBGauss) s_slot[(idx >> 5) * kSlotPitch + (idx & 31)] = acc[i];
        }
        __syncthreads();
    }
    // output value o of group grp's lane gl: the staged total (G == 1) or the
    // sum over the group's warps (G > 1, a single round)
    auto total = [&](int grp, int o, int gl) -> float {
        return G == 1 ? s_slot[o * kSlotPitch + gl] : out_value(s_slot, grp * nvw, nvw, o, gl);
    };
    // write rows, coalesced across each group's 32 Gaussians: 3 geometry rows and
    // 12 SH rows (output value 13 + c holds SH element c = 3 k + ch)
    for (int ri = threadIdx.x; ri < G * 15 * kPBGauss; ri += kPBThreads) {
        const int grp = ri / (15 * kPBGauss), rr = ri % (15 * kPBGauss);
        const int64_t g0 = ((int64_t)blockIdx.x * G + grp) * kPBGauss;
        int gl, o0;
        float4* dst;
        if (rr < 3 * kPBGauss) {
            gl = rr % kPBGauss;
            const int arr = rr / kPBGauss;
            o0 = 4 * arr;
            dst = (arr == 0 ? g_mean_opa : arr == 1 ? g_scale : g_quat) + (g0 + gl);
        } else {
            const int r = rr - 3 * kPBGauss;
            gl = r / 12;
            o0 = kSlotVis + 1 + 4 * (r % 12);
            dst = g_sh + (g0 + gl) * 12 + (r % 12);
        }
        if (g0 + gl >= n) continue;
        float4 val = make_float4(total(grp, o0, gl), total(grp, o0 + 1, gl), total(grp, o0 + 2, gl),
                                 total(grp, o0 + 3, gl));
        if (cfg.accumulate) {
            const float4 old = *dst;
            val.x += old.x; val.y += old.y; val.z += old.z; val.w += old.w;
        }
        *dst = val;
    }
    for (int t = threadIdx.x; t < G * kPBGauss; t += kPBThreads) {
        const int grp = t / kPBGauss, gl = t % kPBGauss;
        const int64_t gg = ((int64_t)blockIdx.x * G + grp) * kPBGauss + gl;
        if (gg >= n) continue;
        const bool vis = total(grp, kSlotVis, gl) > 0.f;
        uint8_t* vd = visible + gg;
        *vd = (vis || (cfg.accumulate && *vd)) ? 1 : 0;
    }
}

// dL/dxi of view v = sum over CTAs of pose_part[v][b][6], fixed tree order.
__global__ void __launch_bounds__(256) k_pose_reduce(const float* __restrict__ pose_part, int64_t nb,
                                                     float* __restrict__ dL_dpose) {
    __shared__ float s[256][6];
    const int v = blockIdx.x;
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int64_t b = threadIdx.x; b < nb; b += 256)
#pragma unroll
        for (int c = 0; c < 6; c++) acc[c] += pose_part[((int64_t)v * nb + b) * 6 + c];
#pragma unroll
    for (int c = 0; c < 6; c++) s[threadIdx.x][c] = acc[c];
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h)
#pragma unroll
            for (int c = 0; c < 6; c++) s[threadIdx.x][c] += s[threadIdx.x + h][c];
        __syncthreads();
    }
    if (threadIdx.x < 6) dL_dpose[v * 6 + threadIdx.x] = s[0][threadIdx.x];
}

int launch_render_bwd(const gs_projected* p, const gs_pairs* pairs, const gs_frame* f, const gs_config* cfg,
                      const gs_image* fwd, const float* dL_dcolor, float4* part0, float4* part1, float* part2,
                      uint32_t* counter, cudaStream_t s);

struct BwdWs {
    float4 *part0, *part1;
    float *part2, *pose_part;
    uint32_t* counter;
};

static BwdWs carve_bwd(char* base, size_t cap, int64_t n, int n_views, int64_t capacity, size_t* used) {
    Carve c{base, 0, cap};
    BwdWs w;
    w.part0 = c.take<float4>(capacity);
    w.part1 = c.take<float4>(capacity);
    w.part2 = c.take<float>(capacity);
    w.pose_part = c.take<float>((size_t)n_views * ceil_div(n, kPBGauss) * 6);
    w.counter = c.take<uint32_t>(4);
    *used = c.used;
    return w;
}

}  // namespace gs

using namespace gs;

extern "C" size_t gs_backward_workspace_size(int64_t n, const gs_frame* f, int64_t capacity) {
    if (!f || n < 0 || capacity < 0) return 0;
    size_t used = 0;
    carve_bwd(nullptr, 0, n, f->n_views, capacity, &used);
    return used;
}

static int check_bwd_common(const gs_frame* f, const gs_config* cfg) {
    if (!f || !cfg || f->n_views < 1 || f->n_views > GS_MAX_VIEWS || cfg->tile != f->tile ||
        cfg->sh_degree < 0 || cfg->sh_degree > 3)
        return GS_ERR_INVALID_ARG;
    return GS_OK;
}

extern "C" int gs_composite_bwd(const gs_projected* p, const gs_pairs* pairs, const gs_frame* f,
                                const gs_config* cfg, const gs_image* fwd, const float* dL_dcolor, int64_t n,
                                void* ws, size_t ws_bytes, void* stream) {
    if (!p || !pairs || !fwd || !dL_dcolor || n < 0 || check_bwd_common(f, cfg) != GS_OK) return GS_ERR_INVALID_ARG;
    size_t need = 0;
    BwdWs w = carve_bwd((char*)ws, ws_bytes, n, f->n_views, pairs->capacity, &need);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255)) return GS_ERR_INVALID_ARG;
    if (n == 0) return GS_OK;
    return launch_render_bwd(p, pairs, f, cfg, fwd, dL_dcolor, w.part0, w.part1, w.part2, w.counter,
                             (cudaStream_t)stream);
}

extern "C" int gs_project_bwd(const gs_gaussians* g, const gs_camera* cams, const gs_projected* p,
                              const gs_pairs* pairs, const gs_frame* f, const gs_config* cfg, const gs_grads* grads,
                              float* dL_dpose, float* d_proj, void* ws, size_t ws_bytes, void* stream) {
    if (!g || !cams || !p || !pairs || !grads || !dL_dpose || g->n < 0 || check_bwd_common(f, cfg) != GS_OK)
        return GS_ERR_INVALID_ARG;
    if (!grads->mean_opa || !grads->scale || !grads->quat || !grads->sh || !grads->visible) return GS_ERR_INVALID_ARG;
    size_t need = 0;
    BwdWs w = carve_bwd((char*)ws, ws_bytes, g->n, f->n_views, pairs->capacity, &need);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (g->n == 0) {
        cudaMemsetAsync(dL_dpose, 0, sizeof(float) * 6 * f->n_views, s);
        GS_CUDA_CHECK_LAUNCH();
        return GS_OK;
    }
    const int64_t nb = ceil_div(g->n, kPBGauss);  // groups of 32 Gaussians (pose partials per view)
    const int nvw = f->n_views < kPBWarps ? f->n_views : kPBWarps;
    const int64_t grid = ceil_div(nb, kPBWarps / nvw);
    static bool attr_set = false;  // the smem opt-in is per function and device-independent here
    if (!attr_set) {
        cudaFuncSetAttribute(k_project_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPBSmem);
        attr_set = true;
    }
    k_project_bwd<<<(unsigned)grid, kPBThreads, kPBSmem, s>>>(
        (const float4*)g->mean_opa, (const float4*)g->scale, (const float4*)g->quat, (const float4*)g->sh, g->n, cams,
        *f, *cfg, p->n_tiles, pairs->offset, w.part0, w.part1, w.part2, pairs->capacity, (float4*)grads->mean_opa,
        (float4*)grads->scale, (float4*)grads->quat, (float4*)grads->sh, grads->visible, d_proj, w.pose_part);
    count_launch();
    k_pose_reduce<<<f->n_views, 256, 0, s>>>(w.pose_part, nb, dL_dpose);
    count_launch();
    GS_CUDA_CHECK_LAUNCH();
    return GS_OK;
}

extern "C" int gs_render_bwd(const gs_gaussians* g, const gs_camera* cams, const gs_projected* p,
                             const gs_pairs* pairs, const gs_frame* f, const gs_config* cfg, const gs_image* fwd,
                             const float* dL_dcolor, const gs_grads* grads, float* dL_dpose, float* d_proj, void* ws,
                             size_t ws_bytes, void* stream) {
    if (!g || !fwd || !dL_dcolor) return GS_ERR_INVALID_ARG;
    int rc = gs_composite_bwd(p, pairs, f, cfg, fwd, dL_dcolor, g->n, ws, ws_bytes, stream);
    if (rc != GS_OK) return rc;
    return gs_project_bwd(g, cams, p, pairs, f, cfg, grads, dL_dpose, d_proj, ws, ws_bytes, stream);
}
