// EWA projection + SH colour (K1). One thread per (view, Gaussian); every CTA
// reads one camera. The view is the fastest-varying CTA index, so the CTAs of
// one block of 256 Gaussians in all views run side by side and the attribute
// rows read from DRAM by the first are L2 hits for the others. Attributes are
// read as 128-bit rows; SH coefficients are read only for Gaussians that
// survive the cull.
#include <atomic>
#include <cstring>

#include "common.cuh"
#include "sh.cuh"

namespace gs {

__global__ void __launch_bounds__(256, 4) k_project(const float4* __restrict__ mean_opa, const float4* __restrict__ scale,
                                                    const float4* __restrict__ quat, const float4* __restrict__ sh,
                                                    int64_t n, const float* __restrict__ filter3d,
                                                    const gs_camera* __restrict__ cams, gs_frame f,
                                                    gs_config cfg, float2* __restrict__ mean2d,
                                                    float4* __restrict__ conic_opa, float4* __restrict__ rgb_depth,
                                                    ushort4* __restrict__ rect, int32_t* __restrict__ n_tiles) {
    __shared__ gs_camera cam_s;
    const int v = (int)(blockIdx.x % (unsigned)f.n_views);
    const int64_t gblock = blockIdx.x / (unsigned)f.n_views;
    if (threadIdx.x < sizeof(gs_camera) / 4)
        reinterpret_cast<float*>(&cam_s)[threadIdx.x] = reinterpret_cast<const float*>(cams + v)[threadIdx.x];
    __syncthreads();
    const int64_t g = gblock * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const int64_t item = (int64_t)v * n + g;
    const gs_camera& c = cam_s;

    const float4 mo = mean_opa[g];
    const float x = c.R[0] * mo.x + c.R[1] * mo.y + c.R[2] * mo.z + c.t[0];
    const float y = c.R[3] * mo.x + c.R[4] * mo.y + c.R[5] * mo.z + c.t[1];
    const float z = c.R[6] * mo.x + c.R[7] * mo.y + c.R[8] * mo.z + c.t[2];
    bool keep = z > cfg.near_z;  // false for NaN

    float a = 0.f, b = 0.f, cc = 0.f, det = 0.f, u = 0.f, vv = 0.f, fmip = 1.f, f3 = 1.f;
    int x0 = 0, y0 = 0, x1 = 0, y1 = 0;
    if (keep) {
        const float4 q4 = quat[g];
        const float4 s4 = scale[g];
        const float qi = rsqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
        const float qw = q4.x * qi, qx = q4.y * qi, qy = q4.z * qi, qz = q4.w * qi;
        float Rq[9];
        Rq[0] = 1.f - 2.f * (qy * qy + qz * qz); Rq[1] = 2.f * (qx * qy - qw * qz); Rq[2] = 2.f * (qx * qz + qw * qy);
        Rq[3] = 2.f * (qx * qy + qw * qz); Rq[4] = 1.f - 2.f * (qx * qx + qz * qz); Rq[5] = 2.f * (qy * qz - qw * qx);
        Rq[6] = 2.f * (qx * qz - qw * qy); Rq[7] = 2.f * (qy * qz + qw * qx); Rq[8] = 1.f - 2.f * (qx * qx + qy * qy);
        float sx = expf(s4.x), sy = expf(s4.y), sz = expf(s4.z);
        if (filter3d) {  // 3-D filter: Sigma + v I has scales sqrt(s^2 + v); opacity x prod s / sqrt(s^2 + v)
            const float fv = filter3d[g];
            const float px = sqrtf(sx * sx + fv), py = sqrtf(sy * sy + fv), pz = sqrtf(sz * sz + fv);
            f3 = (sx / px) * (sy / py) * (sz / pz);
            sx = px; sy = py; sz = pz;
        }
        // T = R_cam * Rq * diag(s): camera-space principal axes; Sc = T T^T
        float T[9];
#pragma unroll
        for (int r = 0; r < 3; r++) {
            const float m0 = c.R[3 * r] * Rq[0] + c.R[3 * r + 1] * Rq[3] + c.R[3 * r + 2] * Rq[6];
            const float m1 = c.R[3 * r] * Rq[1] + c.R[3 * r + 1] * Rq[4] + c.R[3 * r + 2] * Rq[7];
            const float m2 = c.R[3 * r] * Rq[2] + c.R[3 * r + 1] * Rq[5] + c.R[3 * r + 2] * Rq[8];
            T[3 * r] = m0 * sx; T[3 * r + 1] = m1 * sy; T[3 * r + 2] = m2 * sz;
        }
        const float limx = 1.3f * 0.5f * (float)c.width / c.fx;
        const float limy = 1.3f * 0.5f * (float)c.height / c.fy;
        const float iz = 1.f / z;
        const float txz = fminf(limx, fmaxf(-limx, x * iz));
        const float tyz = fminf(limy, fmaxf(-limy, y * iz));
        // rows of J T (2x3): J = [[fx/z, 0, -fx txz/z], [0, fy/z, -fy tyz/z]]
        float A0[3], A1[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            A0[k] = c.fx * iz * (T[k] - txz * T[6 + k]);
            A1[k] = c.fy * iz * (T[3 + k] - tyz * T[6 + k]);
        }
        const float a0 = A0[0] * A0[0] + A0[1] * A0[1] + A0[2] * A0[2];
        b = A0[0] * A1[0] + A0[1] * A1[1] + A0[2] * A1[2];
        const float c0 = A1[0] * A1[0] + A1[1] * A1[1] + A1[2] * A1[2];
        a = a0 + cfg.dilation;
        cc = c0 + cfg.dilation;
        det = a * cc - b * b;
        if (cfg.mip_filter) {  // filter factor sqrt(det Sigma2D / det(Sigma2D + dil I)), rho floored at 1e-6
            // det Sigma2D = |A0|^2 |A1|^2 - (A0.A1)^2 = |A0 x A1|^2: no cancellation for thin splats
            const float k0 = A0[1] * A1[2] - A0[2] * A1[1], k1 = A0[2] * A1[0] - A0[0] * A1[2];
            const float k2 = A0[0] * A1[1] - A0[1] * A1[0];
            const float rho = (k0 * k0 + k1 * k1 + k2 * k2) / det;
            fmip = sqrtf(rho > 1e-6f ? rho : 1e-6f);
        }
        u = c.fx * x * iz + c.cx;
        vv = c.fy * y * iz + c.cy;
        keep = det > 0.f && isfinite(u) && isfinite(vv);
        if (keep) {
            const float mid = 0.5f * (a + cc);
            const float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - det));
            const float r = ceilf(3.f * sqrtf(lam));
            const int T_ = f.tile;
            // the tile size is 8, 16 or 32: multiplying by its reciprocal is exactly the division
            const float iT = 1.f / (float)T_;
            const int tx = f.tiles_x[v], ty = f.tiles_y[v];
            x0 = (int)fminf((float)tx, fmaxf(0.f, floorf((u - r) * iT)));
            y0 = (int)fminf((float)ty, fmaxf(0.f, floorf((vv - r) * iT)));
            x1 = (int)fminf((float)tx, fmaxf(0.f, floorf((u + r + T_ - 1) * iT)));
            y1 = (int)fminf((float)ty, fmaxf(0.f, floorf((vv + r + T_ - 1) * iT)));
            if (cfg.alpha_rect) {
                // only the tiles the box of the ellipse where alpha can reach alpha_min overlaps
                const float oe = f3 * fmip / (1.f + expf(-mo.w));
                if (!(oe >= cfg.alpha_min)) {
                    x1 = x0;  // the opacity never reaches alpha_min: listed nowhere
                } else {
                    const float ta = 2.f * logf(oe / cfg.alpha_min);
                    const float hx = sqrtf(ta * a), hy = sqrtf(ta * cc);
                    x0 = max(x0, (int)fminf((float)tx, fmaxf(0.f, floorf((u - hx) * iT))));
                    y0 = max(y0, (int)fminf((float)ty, fmaxf(0.f, floorf((vv - hy) * iT))));
                    x1 = min(x1, (int)fminf((float)tx, fmaxf(0.f, floorf((u + hx) * iT) + 1.f)));
                    y1 = min(y1, (int)fminf((float)ty, fmaxf(0.f, floorf((vv + hy) * iT) + 1.f)));
                    x1 = max(x1, x0);
                    y1 = max(y1, y0);
                }
            }
            keep = (x1 - x0) * (y1 - y0) > 0;
        }
    }
    float3 rgb = make_float3(0.f, 0.f, 0.f);
    float opa = 0.f;
    if (keep) {
        // view direction: mean - camera centre, centre = -R^T t
        const float cx_ = -(c.R[0] * c.t[0] + c.R[3] * c.t[1] + c.R[6] * c.t[2]);
        const float cy_ = -(c.R[1] * c.t[0] + c.R[4] * c.t[1] + c.R[7] * c.t[2]);
        const float cz_ = -(c.R[2] * c.t[0] + c.R[5] * c.t[1] + c.R[8] * c.t[2]);
        float dx = mo.x - cx_, dy = mo.y - cy_, dz = mo.z - cz_;
        const float il = rsqrtf(dx * dx + dy * dy + dz * dz);
        dx *= il; dy *= il; dz *= il;
        float Y[16];
        sh_eval_basis(cfg.sh_degree, dx, dy, dz, Y);
        rgb = sh_color(sh + 12 * g, cfg.sh_degree, Y);
        opa = f3 * fmip / (1.f + expf(-mo.w));
        keep = isfinite(rgb.x) && isfinite(rgb.y) && isfinite(rgb.z) && isfinite(opa);
        rgb.x = fmaxf(rgb.x, 0.f); rgb.y = fmaxf(rgb.y, 0.f); rgb.z = fmaxf(rgb.z, 0.f);
    }
    if (!keep) {
        n_tiles[item] = 0;
        rect[item] = make_ushort4(0, 0, 0, 0);
        return;
    }
    const float idet = 1.f / det;
    mean2d[item] = make_float2(u, vv);
    conic_opa[item] = make_float4(cc * idet, -b * idet, a * idet, opa);
    rgb_depth[item] = make_float4(rgb.x, rgb.y, rgb.z, z);
    rect[item] = make_ushort4((unsigned short)x0, (unsigned short)y0, (unsigned short)x1, (unsigned short)y1);
    n_tiles[item] = (x1 - x0) * (y1 - y0);
}

// 3-D filter variance (Mip-Splatting's 3-D smoothing filter): nu = the largest
// sampling rate fx / z over the views in which the mean lies in front of the
// near plane and projects inside the image enlarged by 15% on each side;
// v = s2 / nu^2. Gaussians no view samples get -1 here and the largest v of the
// sampled ones (the coarsest filter) in k_filter3d_unseen; vmax_bits collects
// that largest v as float bits (positive floats order like their bits).
__global__ void k_filter3d(const float4* __restrict__ mean_opa, int64_t n, const gs_camera* __restrict__ cams,
                           int n_views, float near_z, float s2, float* __restrict__ out, unsigned* vmax_bits) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const float4 mo = mean_opa[g];
    float nu = 0.f;
    for (int v = 0; v < n_views; v++) {
        const gs_camera& c = cams[v];
        const float x = c.R[0] * mo.x + c.R[1] * mo.y + c.R[2] * mo.z + c.t[0];
        const float y = c.R[3] * mo.x + c.R[4] * mo.y + c.R[5] * mo.z + c.t[1];
        const float z = c.R[6] * mo.x + c.R[7] * mo.y + c.R[8] * mo.z + c.t[2];
        if (!(z > near_z)) continue;
        const float u = c.fx * x / z + c.cx, w = c.fy * y / z + c.cy;
        const float W = (float)c.width, H = (float)c.height;
        if (!(u >= -0.15f * W && u <= 1.15f * W && w >= -0.15f * H && w <= 1.15f * H)) continue;
        nu = fmaxf(nu, c.fx / z);
    }
    if (nu > 0.f) {
        const float fv = s2 / (nu * nu);
        out[g] = fv;
        atomicMax(vmax_bits, __float_as_uint(fv));
    } else {
        out[g] = -1.f;
    }
}

__global__ void k_filter3d_unseen(float* __restrict__ out, int64_t n, const unsigned* vmax_bits) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < n && out[g] < 0.f) out[g] = __uint_as_float(*vmax_bits);
}

}  // namespace gs

namespace gs {
static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
}  // namespace gs

using namespace gs;

extern "C" int64_t gs_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

extern "C" void gs_config_default(gs_config* cfg) {
    cfg->tile = 16;
    cfg->sh_degree = 3;
    cfg->near_z = 0.2f;
    cfg->dilation = 0.3f;
    cfg->alpha_min = 1.f / 255.f;
    cfg->alpha_max = 0.99f;
    cfg->t_min = 1e-4f;
    cfg->mip_filter = 0;
    cfg->alpha_rect = 1;
    cfg->bg[0] = cfg->bg[1] = cfg->bg[2] = 0.f;
    cfg->pose_grad_through_sh = 0;
    cfg->schedule = 0;
    cfg->accumulate = 0;
    cfg->fwd_batch = 0;
    cfg->bwd_batch = 0;
}

extern "C" int gs_frame_init(gs_frame* f, int32_t n_views, const int32_t* width, const int32_t* height,
                             int32_t tile) {
    if (!f || !width || !height || n_views < 1 || n_views > GS_MAX_VIEWS || (tile != 8 && tile != 16 && tile != 32))
        return GS_ERR_INVALID_ARG;
    memset(f, 0, sizeof(*f));
    f->n_views = n_views;
    f->tile = tile;
    int64_t tb = 0, pb = 0;
    for (int v = 0; v < n_views; v++) {
        if (width[v] <= 0 || height[v] <= 0 || width[v] > 65535 * tile || height[v] > 65535 * tile)
            return GS_ERR_INVALID_ARG;
        f->width[v] = width[v];
        f->height[v] = height[v];
        f->tiles_x[v] = (width[v] + tile - 1) / tile;
        f->tiles_y[v] = (height[v] + tile - 1) / tile;
        f->tile_base[v] = (int32_t)tb;
        f->pix_base[v] = pb;
        tb += (int64_t)f->tiles_x[v] * f->tiles_y[v];
        pb += (int64_t)width[v] * height[v];
        if (tb > INT32_MAX || pb > INT32_MAX) return GS_ERR_INVALID_ARG;
    }
    f->tile_base[n_views] = (int32_t)tb;
    f->pix_base[n_views] = pb;
    return GS_OK;
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

extern "C" int gs_project(const gs_gaussians* g, const gs_camera* cams, const gs_frame* f, const gs_config* cfg,
                          const gs_projected* out, void* stream) {
    if (!g || !cams || !f || !cfg || !out) return GS_ERR_INVALID_ARG;
    if (g->n < 0 || g->n > INT32_MAX / 2 || f->n_views < 1 || f->n_views > GS_MAX_VIEWS) return GS_ERR_INVALID_ARG;
    if ((int64_t)f->n_views * g->n > (int64_t)UINT32_MAX) return GS_ERR_INVALID_ARG;
    if (cfg->sh_degree < 0 || cfg->sh_degree > 3 || cfg->tile != f->tile) return GS_ERR_INVALID_ARG;
    if (g->n == 0) return GS_OK;
    if (!aligned16(g->mean_opa) || !aligned16(g->scale) || !aligned16(g->quat) || !aligned16(g->sh) ||
        !aligned16(out->conic_opa) || !aligned16(out->rgb_depth) || !out->mean2d || !out->rect || !out->n_tiles)
        return GS_ERR_INVALID_ARG;
    const int64_t blocks = ceil_div(g->n, 256) * f->n_views;  // <= 2^22 * GS_MAX_VIEWS
    k_project<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(
        (const float4*)g->mean_opa, (const float4*)g->scale, (const float4*)g->quat, (const float4*)g->sh, g->n,
        g->filter3d, cams, *f, *cfg, (float2*)out->mean2d, (float4*)out->conic_opa, (float4*)out->rgb_depth,
        (ushort4*)out->rect, out->n_tiles);
    count_launch();
    GS_CUDA_CHECK_LAUNCH();
    return GS_OK;
}

extern "C" int gs_filter3d(const gs_gaussians* g, const gs_camera* cams, int32_t n_views, float near_z, float s2,
                           float* filter3d, void* ws, size_t ws_bytes, void* stream) {
    if (!g || g->n < 0 || !cams || n_views < 1 || n_views > 4096 || !(s2 > 0.f) || !filter3d) return GS_ERR_INVALID_ARG;
    if (!ws || ws_bytes < 256 || ((uintptr_t)ws & 255)) return GS_ERR_INVALID_ARG;
    if (g->n == 0) return GS_OK;
    if (!aligned16(g->mean_opa)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned* vmax = (unsigned*)ws;
    cudaMemsetAsync(vmax, 0, sizeof(unsigned), s);
    const unsigned grid = (unsigned)ceil_div(g->n, 256);
    k_filter3d<<<grid, 256, 0, s>>>((const float4*)g->mean_opa, g->n, cams, n_views, near_z, s2, filter3d, vmax);
    count_launch();
    k_filter3d_unseen<<<grid, 256, 0, s>>>(filter3d, g->n, vmax);
    count_launch();
    GS_CUDA_CHECK_LAUNCH();
    return GS_OK;
}
