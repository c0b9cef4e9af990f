// Adjoint of the projection (K7) and the per-view pose reduction.
//
// Two kernels. k_item_partials: one thread per (view, Gaussian) item sums the
// item's pair partials - a run of emission slots, which gs_sort assigns in
// item order, so neighbouring threads' runs are adjacent and the loads are
// coalesced - into a 48-byte record, written in item order. k_project_bwd:
// one thread per Gaussian loads its parameters once and walks the views in
// order; per visible view it reads the item's record (coalesced across the
// warp's 32 Gaussians), recomputes the projection, applies the chain rule and
// adds the result to per-Gaussian accumulators - the mean and opacity terms
// and H = sum_v R_v^T dL/dT_v, from which the scale and rotation gradients
// are formed once after the last view, and for SH degree d the 3 (d + 1)^2
// coefficient gradients gc_v[ch] Y_v[k] (summed after the view loop from
// shared memory for up to 16 views) - so each gradient row is written once,
// without atomics. Each view's pose gradient is summed over the warp's 32
// Gaussians by a fixed xor tree and over the CTA's four warps in order into
// one partial per (view, CTA), and those are summed by k_pose_reduce in a
// fixed order: the whole backward pass
// is deterministic. After a pair-buffer overflow (sort status) some slots were
// never written, and the gradients are zero.
#include "common.cuh"
#include "sh.cuh"

namespace gs {

constexpr int kPBThreads = 128;  // threads (Gaussians) per CTA of k_project_bwd, one pose partial per view

// Record of item i: (du dv dA dB | dC dop dr dg | db 0 0 0), written only for
// items with pairs (zeros after a pair-buffer overflow); also the 9 values to
// d_proj (when given).
// The runs of a warp's 32 consecutive items form one contiguous slot range:
// the warp loads it window by window into shared memory with coalesced loads,
// then each lane adds the slots of its own run in slot order.
constexpr int kGatherWin = 128;  // slots per window and warp
constexpr int kGatherWarps = 8;

__global__ void __launch_bounds__(32 * kGatherWarps) k_item_partials(
    int64_t n_items, const int32_t* __restrict__ n_tiles, const uint32_t* __restrict__ offset,
    const float4* __restrict__ part0, const float4* __restrict__ part1, const float* __restrict__ part2,
    int64_t capacity, const int32_t* __restrict__ sort_status, float4* __restrict__ rec, float* __restrict__ d_proj) {
    __shared__ float4 s0[kGatherWarps][kGatherWin];
    __shared__ float4 s1[kGatherWarps][kGatherWin];
    __shared__ float s2[kGatherWarps][kGatherWin];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = item < n_items;
    int nt = in ? n_tiles[item] : 0;
    const uint32_t off = in ? offset[item] : 0u;
    const bool ok = *sort_status == GS_OK;  // after an overflow some slots were never written: no gradient
    // slots past the pair buffer's capacity were never written (overflowed sort)
    const int64_t run = (ok && nt > 0) ? max((int64_t)0, min((int64_t)nt, capacity - (int64_t)off)) : 0;
    const int64_t beg = off, end = off + run;
    const int64_t lo = __reduce_min_sync(FULL, run > 0 ? (unsigned)beg : 0xffffffffu);
    const int64_t hi = __reduce_max_sync(FULL, run > 0 ? (unsigned)end : 0u);
    float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
    float a2 = 0.f;
    for (int64_t base = lo; base < hi; base += kGatherWin) {
        const int cnt = (int)min((int64_t)kGatherWin, hi - base);
        for (int j = lane; j < cnt; j += 32) {
            s0[w][j] = part0[base + j];
            s1[w][j] = part1[base + j];
            s2[w][j] = part2[base + j];
        }
        __syncwarp();
        const int64_t from = max(beg, base), to = min(end, base + cnt);
        for (int64_t q = from; q < to; q++) {
            const float4 p0 = s0[w][q - base], p1 = s1[w][q - base];
            a0.x += p0.x; a0.y += p0.y; a0.z += p0.z; a0.w += p0.w;
            a1.x += p1.x; a1.y += p1.y; a1.z += p1.z; a1.w += p1.w;
            a2 += s2[w][q - base];
        }
        __syncwarp();
    }
    if (!in || nt <= 0) return;  // an item without pairs has no record (its reader skips it)
    rec[3 * item] = a0;
    rec[3 * item + 1] = a1;
    rec[3 * item + 2] = make_float4(a2, 0.f, 0.f, 0.f);
    if (d_proj && nt > 0) {
        float* o = d_proj + 9 * item;
        o[0] = a0.x; o[1] = a0.y; o[2] = a0.z; o[3] = a0.w; o[4] = a1.x; o[5] = a1.y; o[6] = a1.z; o[7] = a1.w;
        o[8] = a2;
    }
}

// Rotation matrix (row-major) of the unit quaternion (w, x, y, z).
__device__ __forceinline__ void quat_rotation(float qw, float qx, float qy, float qz, float (&R)[9]) {
    R[0] = 1.f - 2.f * (qy * qy + qz * qz); R[1] = 2.f * (qx * qy - qw * qz); R[2] = 2.f * (qx * qz + qw * qy);
    R[3] = 2.f * (qx * qy + qw * qz); R[4] = 1.f - 2.f * (qx * qx + qz * qz); R[5] = 2.f * (qy * qz - qw * qx);
    R[6] = 2.f * (qx * qz - qw * qy); R[7] = 2.f * (qy * qz + qw * qx); R[8] = 1.f - 2.f * (qx * qx + qy * qy);
}

// DV > 0 (at most DV views): each view's colour gradient is kept in shared
// memory and the SH-coefficient sums are formed after the view loop (the view
// direction computed again there), so their 3 (d + 1)^2 accumulators are not
// live across it: 128 registers (a few bytes spilled), four CTAs per SM;
// DV = 0: accumulated view by view.
constexpr int kPBDeferViews = 16;

template <int SHD, int DV>
__global__ void __launch_bounds__(kPBThreads, DV > 0 ? 4 : 1) k_project_bwd(
    const float4* __restrict__ mean_opa, const float4* __restrict__ scale, const float4* __restrict__ quat,
    const float4* __restrict__ sh, int64_t n, const float* __restrict__ filter3d, const gs_camera* __restrict__ cams,
    gs_frame f, gs_config cfg,
    const int32_t* __restrict__ n_tiles, const float4* __restrict__ rec, float4* __restrict__ g_mean_opa,
    float4* __restrict__ g_scale, float4* __restrict__ g_quat, float4* __restrict__ g_sh,
    uint8_t* __restrict__ visible, float* __restrict__ pose_part) {
    constexpr int NC = (SHD + 1) * (SHD + 1);  // SH coefficients per channel
    constexpr int NR = (3 * NC + 3) / 4;       // float4 rows of SH coefficients in use
    constexpr int NWP = kPBThreads / 32;
    __shared__ gs_camera s_cam[GS_MAX_VIEWS];
    __shared__ float s_pose[GS_MAX_VIEWS][NWP][6];  // each warp's pose partial per view
    const unsigned FULL = 0xffffffffu;
    const int nv = f.n_views;
    for (int i = threadIdx.x; i < nv * (int)(sizeof(gs_camera) / 4); i += kPBThreads)
        reinterpret_cast<float*>(s_cam)[i] = reinterpret_cast<const float*>(cams)[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int64_t g = (int64_t)blockIdx.x * kPBThreads + threadIdx.x;
    const bool valid = g < n;
    float4 mo = make_float4(0.f, 0.f, 0.f, 0.f), s4 = mo, q4 = make_float4(1.f, 0.f, 0.f, 0.f);
    if (valid) { mo = mean_opa[g]; s4 = scale[g]; q4 = quat[g]; }
    // parameter-space quantities shared by all views (the rotation and scales are read again
    // after the view loop, so that they are not held in registers across it)
    float RS[9];  // Rq diag(s'): the Gaussian's principal axes in world space
    {
        const float qi = rsqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
        quat_rotation(q4.x * qi, q4.y * qi, q4.z * qi, q4.w * qi, RS);
    }
    // with the 3-D filter the projection sees scales s' = sqrt(s^2 + v) and the opacity
    // factor f3 = prod s / s' (both formed again after the view loop for the log-scale chain)
    float sv[3] = {expf(s4.x), expf(s4.y), expf(s4.z)};
    float f3 = 1.f;
    if (filter3d && valid) {
        const float fv = filter3d[g];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const float p = sqrtf(sv[k] * sv[k] + fv);
            f3 *= sv[k] / p;
            sv[k] = p;
        }
    }
#pragma unroll
    for (int k = 0; k < 9; k++) RS[k] *= sv[k % 3];
    const float opa = 1.f / (1.f + expf(-mo.w));
    float a3 = 0.f;  // sum over views of dL/d(opacity) x the 2-D filter factor
    const float4* shg = sh + 12 * g;
    // per-Gaussian sums over the views (in view order)
    // and H = sum_v R_v^T dL/dT_v (T_v = R_v Rq diag(s')): the scale and rotation gradients are
    // linear in H and are formed once, after the view loop
    float am[3] = {0.f, 0.f, 0.f}, alogit = 0.f, aH[9];
#pragma unroll
    for (int k = 0; k < 9; k++) aH[k] = 0.f;
    float ash[3 * NC];
    if constexpr (DV == 0) {
#pragma unroll
        for (int c = 0; c < 3 * NC; c++) ash[c] = 0.f;
    }
    __shared__ float s_gd[DV > 0 ? DV : 1][3][kPBThreads];  // per view: the colour gradient gc[3]
    uint32_t vmask = 0;                                       // views whose entries are set
    bool vis = false;
    // the next view's tile count and record are loaded while this view is processed (a record
    // is used only when its item has pairs: the others were never written)
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    int nt_nx = valid ? n_tiles[g] : 0;
    float4 r0_nx = valid ? rec[3 * g] : zero4, r1_nx = valid ? rec[3 * g + 1] : zero4;
    float4 r2_nx = valid ? rec[3 * g + 2] : zero4;

    for (int v = 0; v < nv; v++) {
        const int64_t item = (int64_t)v * n + g;
        const int nt = nt_nx;
        const float4 r0 = r0_nx, r1 = r1_nx, r2 = r2_nx;
        if (valid && v + 1 < nv) {
            const int64_t nx = item + n;
            nt_nx = n_tiles[nx];
            r0_nx = rec[3 * nx];
            r1_nx = rec[3 * nx + 1];
            r2_nx = rec[3 * nx + 2];
        }
        float pose[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (nt > 0) {
            vis = true;
            const gs_camera& c = s_cam[v];
            const float du = r0.x, dv = r0.y, dA = r0.z, dB = r0.w, dC = r1.x, dop = r1.y;
            const float dr = r1.z, dg = r1.w, db = r2.x;

            // colour: rgb = max(0.5 + sum_k Y_k(d) sh_k, 0), d = (mu - centre)/|mu - centre|
            const float ccx = -(c.R[0] * c.t[0] + c.R[3] * c.t[1] + c.R[6] * c.t[2]);
            const float ccy = -(c.R[1] * c.t[0] + c.R[4] * c.t[1] + c.R[7] * c.t[2]);
            const float ccz = -(c.R[2] * c.t[0] + c.R[5] * c.t[1] + c.R[8] * c.t[2]);
            float ddx = mo.x - ccx, ddy = mo.y - ccy, ddz = mo.z - ccz;
            const float il = rsqrtf(ddx * ddx + ddy * ddy + ddz * ddz);
            ddx *= il; ddy *= il; ddz *= il;
            float Y[16];
            sh_eval_basis(SHD, ddx, ddy, ddz, Y);
            float cq[4 * NR];
#pragma unroll
            for (int r = 0; r < NR; r++) {
                const float4 q = shg[r];
                cq[4 * r] = q.x; cq[4 * r + 1] = q.y; cq[4 * r + 2] = q.z; cq[4 * r + 3] = q.w;
            }
            float raw[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
            for (int kk = 0; kk < NC; kk++)
#pragma unroll
                for (int ch = 0; ch < 3; ch++) raw[ch] += Y[kk] * cq[3 * kk + ch];
            const float gc[3] = {raw[0] > 0.f ? dr : 0.f, raw[1] > 0.f ? dg : 0.f, raw[2] > 0.f ? db : 0.f};
            if constexpr (DV == 0) {
#pragma unroll
                for (int kk = 0; kk < NC; kk++)
#pragma unroll
                    for (int ch = 0; ch < 3; ch++) ash[3 * kk + ch] += gc[ch] * Y[kk];
            } else {
                const int t = threadIdx.x;
                s_gd[v][0][t] = gc[0]; s_gd[v][1][t] = gc[1]; s_gd[v][2][t] = gc[2];
                vmask |= 1u << v;
            }
            float gmx = 0.f, gmy = 0.f, gmz = 0.f;
            if (SHD > 0) {
                // direction gradient of sum_k w_k Y_k(d), w_k = sum_ch gc[ch] sh[k][ch]
                float wk[16];
#pragma unroll
                for (int kk = 0; kk < 16; kk++) wk[kk] = 0.f;
#pragma unroll
                for (int kk = 1; kk < NC; kk++)
#pragma unroll
                    for (int ch = 0; ch < 3; ch++) wk[kk] += gc[ch] * cq[3 * kk + ch];
                const float3 gd = sh_weighted_grad(SHD, ddx, ddy, ddz, wk);
                const float dd = gd.x * ddx + gd.y * ddy + gd.z * ddz;
                gmx = (gd.x - ddx * dd) * il; gmy = (gd.y - ddy * dd) * il; gmz = (gd.z - ddz * dd) * il;
                if (cfg.pose_grad_through_sh) {
                    // centre = -R^T t moves by -R^T rho under exp(xi^): dL/drho += R dL/ddir
                    pose[0] += c.R[0] * gmx + c.R[1] * gmy + c.R[2] * gmz;
                    pose[1] += c.R[3] * gmx + c.R[4] * gmy + c.R[5] * gmz;
                    pose[2] += c.R[6] * gmx + c.R[7] * gmy + c.R[8] * gmz;
                }
            }

            // recompute the projection
            const float x = c.R[0] * mo.x + c.R[1] * mo.y + c.R[2] * mo.z + c.t[0];
            const float y = c.R[3] * mo.x + c.R[4] * mo.y + c.R[5] * mo.z + c.t[1];
            const float z = c.R[6] * mo.x + c.R[7] * mo.y + c.R[8] * mo.z + c.t[2];
            float T[9];  // R_cam Rq diag(s)
#pragma unroll
            for (int r = 0; r < 3; r++)
#pragma unroll
                for (int kk = 0; kk < 3; kk++)
                    T[3 * r + kk] = c.R[3 * r] * RS[kk] + c.R[3 * r + 1] * RS[3 + kk] + c.R[3 * r + 2] * RS[6 + kk];
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
                if (rho > 1e-6f) g_rho = dop * f3 * opa / (2.f * fmip);  // dL/drho through opacity o f
            }

            // conic = S^-1: dL/dS = -Q dL/dQ Q, dL/dQ = [[dA, dB/2], [dB/2, dC]]
            const float hB = 0.5f * dB;
            const float t00 = Qa * dA + Qb * hB, t01 = Qa * hB + Qb * dC;
            const float t10 = Qb * dA + Qc * hB, t11 = Qb * hB + Qc * dC;
            // plus the filter factor's rho = ((A - dil)(C - dil) - B^2) / (A C - B^2), S = [[A, B], [B, C]]
            const float GS00 = -(t00 * Qa + t01 * Qb) + g_rho * (Sc0 - rho * Sc) * idet;
            const float GS01 = -(t00 * Qb + t01 * Qc) - g_rho * Sb * (1.f - rho) * idet;
            const float GS11 = -(t10 * Qb + t11 * Qc) + g_rho * (Sa0 - rho * Sa) * idet;
            // S = M M^T + dil I: dL/dM = 2 GS M
            float GM0[3], GM1[3];
#pragma unroll
            for (int kk = 0; kk < 3; kk++) {
                GM0[kk] = 2.f * (GS00 * M0[kk] + GS01 * M1[kk]);
                GM1[kk] = 2.f * (GS01 * M0[kk] + GS11 * M1[kk]);
            }
            // M = J T: dL/dJ = GM T^T (entries J00, J02, J11, J12), dL/dT = J^T GM
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
            // T = R (Rq diag s'): dL/d(Rq diag s') = R^T GT, summed over the views
#pragma unroll
            for (int r = 0; r < 3; r++)
#pragma unroll
                for (int kk = 0; kk < 3; kk++)
                    aH[3 * r + kk] += c.R[r] * GT[kk] + c.R[3 + r] * GT[3 + kk] + c.R[6 + r] * GT[6 + kk];
            // p = (x, y, z): through the 2D mean and J
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
            am[0] += gmx + c.R[0] * gpx + c.R[3] * gpy + c.R[6] * gpz;
            am[1] += gmy + c.R[1] * gpx + c.R[4] * gpy + c.R[7] * gpz;
            am[2] += gmz + c.R[2] * gpx + c.R[5] * gpy + c.R[8] * gpz;
            alogit += dop * f3 * fmip * opa * (1.f - opa);
            a3 += dop * fmip;
            // pose, left perturbation: dp = rho + phi x p, dT = phi^ T
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
        // this view's pose partial over the warp's 32 Gaussians (fixed xor tree)
#pragma unroll
        for (int c = 0; c < 6; c++)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) pose[c] += __shfl_xor_sync(FULL, pose[c], o);
        if (lane < 6) {
            float pv = pose[0];
#pragma unroll
            for (int c = 1; c < 6; c++) pv = (lane == c) ? pose[c] : pv;
            s_pose[v][wp][lane] = pv;
        }
    }
    // one pose partial per (view, CTA): the CTA's warps summed in order
    __syncthreads();
    for (int i = threadIdx.x; i < nv * 6; i += kPBThreads) {
        const int v = i / 6, c = i % 6;
        float pv = 0.f;
#pragma unroll
        for (int q = 0; q < NWP; q++) pv += s_pose[v][q][c];
        pose_part[((int64_t)v * gridDim.x + blockIdx.x) * 6 + c] = pv;
    }
    if (!valid) return;
    if constexpr (DV > 0) {
        // the SH-coefficient gradients, summed over the views in order as above
#pragma unroll
        for (int c = 0; c < 3 * NC; c++) ash[c] = 0.f;
        const int t = threadIdx.x;
        const float4 me = mean_opa[g];
        for (int v = 0; v < nv; v++) {
            if (!((vmask >> v) & 1u)) continue;
            const float gc[3] = {s_gd[v][0][t], s_gd[v][1][t], s_gd[v][2][t]};
            // the view direction exactly as in the view loop
            const gs_camera& c = s_cam[v];
            const float ccx = -(c.R[0] * c.t[0] + c.R[3] * c.t[1] + c.R[6] * c.t[2]);
            const float ccy = -(c.R[1] * c.t[0] + c.R[4] * c.t[1] + c.R[7] * c.t[2]);
            const float ccz = -(c.R[2] * c.t[0] + c.R[5] * c.t[1] + c.R[8] * c.t[2]);
            float ddx = me.x - ccx, ddy = me.y - ccy, ddz = me.z - ccz;
            const float il = rsqrtf(ddx * ddx + ddy * ddy + ddz * ddz);
            ddx *= il; ddy *= il; ddz *= il;
            float Y[16];
            sh_eval_basis(SHD, ddx, ddy, ddz, Y);
#pragma unroll
            for (int kk = 0; kk < NC; kk++)
#pragma unroll
                for (int ch = 0; ch < 3; ch++) ash[3 * kk + ch] += gc[ch] * Y[kk];
        }
    }
    float4 om = make_float4(am[0], am[1], am[2], alogit);
    float4 os = make_float4(0.f, 0.f, 0.f, 0.f), oq = os;  // zeros for a Gaussian no view lists
    if (vis) {
        const float4 qe = quat[g], se = scale[g];
        const float qi = rsqrtf(qe.x * qe.x + qe.y * qe.y + qe.z * qe.z + qe.w * qe.w);
        const float qw = qe.x * qi, qx = qe.y * qi, qy = qe.z * qi, qz = qe.w * qi;
        float Rq[9];
        quat_rotation(qw, qx, qy, qz, Rq);
        // d/d log s'_k = s'_k sum_r H[r][k] Rq[r][k], then back from the filtered scales s' to the
        // log-scales (the opacity factor f3 too): d log s' / d log s = s^2 / s'^2, d log f3 / d log s =
        // v / s'^2
        const float s0[3] = {expf(se.x), expf(se.y), expf(se.z)};
        const float fv = filter3d ? filter3d[g] : 0.f;
        const float l3 = a3 * f3 * opa;  // dL / d log f3
        float ls[3];
#pragma unroll
        for (int kk = 0; kk < 3; kk++) {
            const float sp = filter3d ? sqrtf(s0[kk] * s0[kk] + fv) : s0[kk];
            const float dsq = filter3d ? s0[kk] * s0[kk] / (sp * sp) : 1.f;
            const float gl = (aH[kk] * Rq[kk] + aH[3 + kk] * Rq[3 + kk] + aH[6 + kk] * Rq[6 + kk]) * sp;
            ls[kk] = gl * dsq + l3 * fv / (sp * sp);
        }
        os = make_float4(ls[0], ls[1], ls[2], 0.f);
        // dL/dRq = H diag(s'), then rotation matrix -> normalised quaternion -> raw quaternion
        float gRq[9];
#pragma unroll
        for (int k = 0; k < 9; k++) gRq[k] = aH[k] * (filter3d ? sqrtf(s0[k % 3] * s0[k % 3] + fv) : s0[k % 3]);
        float gq[4];
        gq[0] = 2.f * (-qz * gRq[1] + qy * gRq[2] + qz * gRq[3] - qx * gRq[5] - qy * gRq[6] + qx * gRq[7]);
        gq[1] = 2.f * (qy * gRq[1] + qz * gRq[2] + qy * gRq[3] - 2.f * qx * gRq[4] - qw * gRq[5] + qz * gRq[6] +
                       qw * gRq[7] - 2.f * qx * gRq[8]);
        gq[2] = 2.f * (-2.f * qy * gRq[0] + qx * gRq[1] + qw * gRq[2] + qx * gRq[3] + qz * gRq[5] - qw * gRq[6] +
                       qz * gRq[7] - 2.f * qy * gRq[8]);
        gq[3] = 2.f * (-2.f * qz * gRq[0] - qw * gRq[1] + qx * gRq[2] + qw * gRq[3] - 2.f * qz * gRq[4] +
                       qy * gRq[5] + qx * gRq[6] + qy * gRq[7]);
        const float qd = gq[0] * qw + gq[1] * qx + gq[2] * qy + gq[3] * qz;
        oq = make_float4((gq[0] - qw * qd) * qi, (gq[1] - qx * qd) * qi, (gq[2] - qy * qd) * qi, (gq[3] - qz * qd) * qi);
    }
    if (cfg.accumulate) {
        const float4 a = g_mean_opa[g], b = g_scale[g], q = g_quat[g];
        om.x += a.x; om.y += a.y; om.z += a.z; om.w += a.w;
        os.x += b.x; os.y += b.y; os.z += b.z; os.w += b.w;
        oq.x += q.x; oq.y += q.y; oq.z += q.z; oq.w += q.w;
    }
    g_mean_opa[g] = om;
    g_scale[g] = os;
    g_quat[g] = oq;
#pragma unroll
    for (int r = 0; r < 12; r++) {
        float4 val = make_float4(4 * r < 3 * NC ? ash[4 * r] : 0.f, 4 * r + 1 < 3 * NC ? ash[4 * r + 1] : 0.f,
                                 4 * r + 2 < 3 * NC ? ash[4 * r + 2] : 0.f, 4 * r + 3 < 3 * NC ? ash[4 * r + 3] : 0.f);
        if (cfg.accumulate) {
            const float4 old = g_sh[12 * g + r];
            val.x += old.x; val.y += old.y; val.z += old.z; val.w += old.w;
        }
        g_sh[12 * g + r] = val;
    }
    uint8_t* vd = visible + g;
    *vd = (vis || (cfg.accumulate && *vd)) ? 1 : 0;
}

// dL/dxi of view v = sum over CTAs of pose_part[v][b][6], fixed tree order.
__global__ void __launch_bounds__(256) k_pose_reduce(const float* __restrict__ pose_part, int64_t nb,
                                                     float* __restrict__ dL_dpose) {
    __shared__ float s[256][6];
    const int v = blockIdx.x;
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
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
    float4* rec;
    uint32_t* counter;
};

static BwdWs carve_bwd(char* base, size_t cap, int64_t n, int n_views, int64_t capacity, size_t* used) {
    Carve c{base, 0, cap};
    BwdWs w;
    w.part0 = c.take<float4>(capacity);
    w.part1 = c.take<float4>(capacity);
    w.part2 = c.take<float>(capacity);
    w.pose_part = c.take<float>((size_t)n_views * ceil_div(n, kPBThreads) * 6);
    w.counter = c.take<uint32_t>(4);
    w.rec = c.take<float4>((size_t)n_views * n * 3);  // per-item sums of the pair partials
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
    if (g->n > 0 && (!pairs->offset || !pairs->status)) return GS_ERR_INVALID_ARG;
    size_t need = 0;
    BwdWs w = carve_bwd((char*)ws, ws_bytes, g->n, f->n_views, pairs->capacity, &need);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (g->n == 0) {
        cudaMemsetAsync(dL_dpose, 0, sizeof(float) * 6 * f->n_views, s);
        GS_CUDA_CHECK_LAUNCH();
        return GS_OK;
    }
    const int64_t nb = ceil_div(g->n, kPBThreads);  // CTAs of k_project_bwd (pose partials per view)
    const int64_t n_items = (int64_t)f->n_views * g->n;
    k_item_partials<<<(unsigned)ceil_div(n_items, 32 * kGatherWarps), 32 * kGatherWarps, 0, s>>>(
        n_items, p->n_tiles, pairs->offset, w.part0, w.part1, w.part2, pairs->capacity, pairs->status, w.rec, d_proj);
    count_launch();
    const unsigned grid = (unsigned)ceil_div(g->n, kPBThreads);
#define GS_PB(D)                                                                                                \
    if (f->n_views <= kPBDeferViews) { GS_PB2(D, kPBDeferViews); } else { GS_PB2(D, 0); }
#define GS_PB2(D, DV)                                                                                           \
    k_project_bwd<D, DV><<<grid, kPBThreads, 0, s>>>((const float4*)g->mean_opa, (const float4*)g->scale,          \
                                                 (const float4*)g->quat, (const float4*)g->sh, g->n,           \
                                                 g->filter3d, cams, *f,                                         \
                                                 *cfg, p->n_tiles, w.rec, (float4*)grads->mean_opa,               \
                                                 (float4*)grads->scale, (float4*)grads->quat,                     \
                                                 (float4*)grads->sh, grads->visible, w.pose_part)
    switch (cfg->sh_degree) {
        case 0: GS_PB(0); break;
        case 1: GS_PB(1); break;
        case 2: GS_PB(2); break;
        default: GS_PB(3); break;
    }
#undef GS_PB
#undef GS_PB2
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
