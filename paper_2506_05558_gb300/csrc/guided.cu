// Guided-matching depth refinement (Sec. 4.2, App. A.2). Per pixel of the
// reference frame: n candidates uniform in inverse depth over
// [max(1/Z* - w, 0), 1/Z* + w] around the monocular depth Z*; one neighbour
// per pixel, the usable one (whole candidate segment in front of it and
// inside its map) whose segment is longest in pixels; correlation
// C_k = <F_i(pixel), bilinear F_j(reprojection of candidate k)>; the first
// maximum and a parabola through it and its two neighbours give the inverse
// depth.
//
// Layout and mapping: feature maps [H][W][C] bfloat16 (one pixel's channels
// contiguous, 2C bytes). Four lanes (a quad) own one pixel, each a quarter of
// the channels, so a warp reads eight pixels' features as contiguous
// 2C-byte runs per corner; the quad's partial dot products meet in two
// shuffles. The quad's lanes project four candidates at once and broadcast
// each one's cell and weights, so the scalar work is not repeated per lane.
// Persistent CTAs walk 16 x 4 pixel tiles; the relative poses are composed
// once per CTA in FP64.
#include "common.cuh"

namespace gs {

constexpr int kGmMaxNb = 8;
constexpr int kGmTileX = 16, kGmTileY = 4;  // 64 pixels (256 threads) per CTA

struct GmRel {  // a candidate r / d of the reference is (R r + d b) / d in the neighbour
    float R[9];
    float b[3];
    float fx, fy, cx, cy;
};

template <int C>
__device__ __forceinline__ void gm_load(const uint16_t* p, uint32_t (&w)[C / 8]) {
    if constexpr (C == 8) {
        w[0] = __ldg(reinterpret_cast<const uint32_t*>(p));
    } else if constexpr (C == 16) {
        const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
        w[0] = v.x; w[1] = v.y;
    } else {
#pragma unroll
        for (int i = 0; i < C / 32; i++) {
            const uint4 v = __ldg(reinterpret_cast<const uint4*>(p) + i);
            w[4 * i] = v.x; w[4 * i + 1] = v.y; w[4 * i + 2] = v.z; w[4 * i + 3] = v.w;
        }
    }
}

// c + a.lo b.lo + a.hi b.hi for two packed bfloat16 pairs, by the mixed-precision
// FMA (bf16 multiplicands, FP32 addend and result): the product of two bf16
// values is exact in FP32, so each step rounds once, exactly as an FP32 FMA of
// the widened values would, without spending an integer op per channel on the
// widening.
__device__ __forceinline__ float fma2_bf16(uint32_t a, uint32_t b, float c) {
    float d;
    asm("{\n\t.reg .b16 al, ah, bl, bh;\n\t"
        "mov.b32 {al, ah}, %1;\n\t"
        "mov.b32 {bl, bh}, %2;\n\t"
        "fma.rn.f32.bf16 %0, al, bl, %3;\n\t"
        "fma.rn.f32.bf16 %0, ah, bh, %0;\n\t}"
        : "=&f"(d)
        : "r"(a), "r"(b), "f"(c));
    return d;
}

template <int C>
__device__ __forceinline__ float gm_dot(const uint32_t (&f)[C / 8], const uint32_t (&w)[C / 8]) {
    float a = 0.f;
#pragma unroll
    for (int i = 0; i < C / 8; i++) a = fma2_bf16(f[i], w[i], a);
    return a;
}

template <int C>
__global__ void __launch_bounds__(256) k_guided_depth(const uint16_t* __restrict__ feats,
                                                      const gs_camera* __restrict__ cams, int n_nb, int W, int H,
                                                      const float* __restrict__ z_mono, int n_cand, float window,
                                                      float* __restrict__ depth, int32_t* __restrict__ nb_out,
                                                      float* __restrict__ corr_out) {
    __shared__ GmRel s_rel[kGmMaxNb];
    __shared__ float s_ref[4];
    const int tid = threadIdx.x;
    if (tid < n_nb) {  // once per persistent CTA
        const gs_camera& ci = cams[0];
        const gs_camera& cj = cams[1 + tid];
        double R[9];
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++) {
                double a = 0.0;
                for (int k = 0; k < 3; k++) a += (double)cj.R[3 * r + k] * (double)ci.R[3 * c + k];  // R_j R_i^T
                R[3 * r + c] = a;
            }
        GmRel& g = s_rel[tid];
        for (int r = 0; r < 3; r++) {
            const double Rt = R[3 * r] * ci.t[0] + R[3 * r + 1] * ci.t[1] + R[3 * r + 2] * ci.t[2];
            g.b[r] = (float)((double)cj.t[r] - Rt);
        }
        for (int e = 0; e < 9; e++) g.R[e] = (float)R[e];
        g.fx = cj.fx; g.fy = cj.fy; g.cx = cj.cx; g.cy = cj.cy;
    }
    if (tid == 0) {
        s_ref[0] = cams[0].fx; s_ref[1] = cams[0].fy; s_ref[2] = cams[0].cx; s_ref[3] = cams[0].cy;
    }
    __syncthreads();
    const int q = tid & 3, pix = tid >> 2;
    const int tiles_x = (W + kGmTileX - 1) / kGmTileX;
    const int n_tiles = tiles_x * ((H + kGmTileY - 1) / kGmTileY);
    const float xmax = (float)(W - 1), ymax = (float)(H - 1);
    const float inv = 1.f / (float)(n_cand - 1);
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        // every lane runs the same number of candidate steps (full-warp shuffles); a quad without a pixel
        // or without a usable neighbour samples a fixed in-bounds cell and discards the result
        const int u = (t % tiles_x) * kGmTileX + (pix & (kGmTileX - 1));
        const int v = (t / tiles_x) * kGmTileY + pix / kGmTileX;
        const bool inside = u < W && v < H;
        const int64_t p = inside ? (int64_t)v * W + u : 0;
        const float zm = inside ? z_mono[p] : 0.f;
        const bool ok = isfinite(zm) && zm > 0.f;
        const float rx = (u + 0.5f - s_ref[2]) / s_ref[0], ry = (v + 0.5f - s_ref[3]) / s_ref[1];
        const float dc = ok ? 1.f / zm : 1.f;
        const float lo = fmaxf(dc - window, 0.f), hi = dc + window;
        float best = -1.f;
        int jb = -1;
        float a0 = 0.f, a1 = 0.f, a2 = 1.f, b0 = 0.f, b1 = 0.f, b2 = 0.f;
        float fxj = 0.f, fyj = 0.f, cxj = 0.f, cyj = 0.f;
        if (ok) {
            for (int j = 0; j < n_nb; j++) {  // adaptive neighbour: the longest usable segment
                const GmRel& g = s_rel[j];
                const float e0 = fmaf(g.R[0], rx, fmaf(g.R[1], ry, g.R[2]));
                const float e1 = fmaf(g.R[3], rx, fmaf(g.R[4], ry, g.R[5]));
                const float e2 = fmaf(g.R[6], rx, fmaf(g.R[7], ry, g.R[8]));
                const float z0 = fmaf(lo, g.b[2], e2), z1 = fmaf(hi, g.b[2], e2);
                if (!(z0 > 0.f && z1 > 0.f)) continue;
                const float x0 = g.fx * fmaf(lo, g.b[0], e0) / z0 + g.cx - 0.5f;
                const float y0 = g.fy * fmaf(lo, g.b[1], e1) / z0 + g.cy - 0.5f;
                const float x1 = g.fx * fmaf(hi, g.b[0], e0) / z1 + g.cx - 0.5f;
                const float y1 = g.fy * fmaf(hi, g.b[1], e1) / z1 + g.cy - 0.5f;
                if (!(x0 >= 0.f && x0 <= xmax && y0 >= 0.f && y0 <= ymax && x1 >= 0.f && x1 <= xmax &&
                      y1 >= 0.f && y1 <= ymax))
                    continue;
                const float sl = sqrtf((x1 - x0) * (x1 - x0) + (y1 - y0) * (y1 - y0));
                if (sl > best) {
                    best = sl; jb = j;
                    a0 = e0; a1 = e1; a2 = e2; b0 = g.b[0]; b1 = g.b[1]; b2 = g.b[2];
                    fxj = g.fx; fyj = g.fy; cxj = g.cx - 0.5f; cyj = g.cy - 0.5f;
                }
            }
        }
        const bool act = jb >= 0;
        uint32_t fi[C / 8];
        gm_load<C>(feats + p * C + q * (C / 4), fi);
        const uint16_t* Fj = feats + ((int64_t)(1 + (act ? jb : 0)) * H * W) * C + q * (C / 4);
        const float span = hi - lo;
        const int64_t row = (int64_t)W * C;
        float cbest = -INFINITY, cm = 0.f, cp = 0.f, prev = 0.f;
        int kb = 0;
        bool want_next = false;
        const int qbase = (tid & 31) & ~3;
        for (int k0 = 0; k0 < n_cand; k0 += 4) {
            // lane q projects candidate k0 + q (the last group may run past n_cand: those are never used)
            const float d = fmaf(span, (float)(k0 + q) * inv, lo);
            const float iz = fast_rcp(fmaf(d, b2, a2));
            const float sx = fmaf(fxj * fmaf(d, b0, a0), iz, cxj);
            const float sy = fmaf(fyj * fmaf(d, b1, a1), iz, cyj);
            // cell of the sample, clamped so that every read stays in the map (the segment's ends are
            // inside; rounding may put an interior sample a hair outside)
            const int x0 = min(max(__float2int_rd(sx), 0), W - 2);
            const int y0 = min(max(__float2int_rd(sy), 0), H - 2);
            const float wxo = sx - (float)x0, wyo = sy - (float)y0;
            const int offo = (y0 * W + x0) * C;
            const int nk = min(4, n_cand - k0);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                if (j >= nk) break;  // uniform across the warp
                const int off = __shfl_sync(0xffffffffu, offo, qbase + j);
                const float wx = __shfl_sync(0xffffffffu, wxo, qbase + j);
                const float wy = __shfl_sync(0xffffffffu, wyo, qbase + j);
                const uint16_t* r0 = Fj + off;
                const uint16_t* r1 = r0 + row;
                uint32_t w00[C / 8], w01[C / 8], w10[C / 8], w11[C / 8];
                gm_load<C>(r0, w00);
                gm_load<C>(r0 + C, w01);
                gm_load<C>(r1, w10);
                gm_load<C>(r1 + C, w11);
                const float c00 = gm_dot<C>(fi, w00), c01 = gm_dot<C>(fi, w01);
                const float c10 = gm_dot<C>(fi, w10), c11 = gm_dot<C>(fi, w11);
                float c = (1.f - wx) * (1.f - wy) * c00 + wx * (1.f - wy) * c01 + (1.f - wx) * wy * c10 +
                          wx * wy * c11;
                c += __shfl_xor_sync(0xffffffffu, c, 1);
                c += __shfl_xor_sync(0xffffffffu, c, 2);
                const int k = k0 + j;
                if (want_next) { cp = c; want_next = false; }
                if (c > cbest) { cbest = c; kb = k; cm = prev; want_next = true; }
                prev = c;
            }
        }
        float out_d = zm, out_c = 0.f;
        int out_j = -1;
        if (act) {
            float delta = 0.f;
            if (kb > 0 && kb < n_cand - 1) {
                const float den = cm - 2.f * cbest + cp;
                if (den < 0.f) delta = (cm - cp) / (2.f * den);
            }
            const float ds = fmaf(span, (float)kb * inv, lo) + delta * span * inv;
            if (ds > 0.f) { out_d = 1.f / ds; out_j = jb; out_c = cbest; }
        }
        if (inside && q == 0) {
            depth[p] = out_d;
            if (nb_out) nb_out[p] = out_j;
            if (corr_out) corr_out[p] = out_c;
        }
    }
}

}  // namespace gs

using namespace gs;

extern "C" int gs_guided_depth(const uint16_t* feats, const gs_camera* cams, int32_t n_nb, int32_t width,
                               int32_t height, int32_t channels, const float* z_mono, int32_t n_cand, float window,
                               float* depth, int32_t* nb, float* corr, void* stream) {
    if (!feats || !cams || !z_mono || !depth || n_nb < 1 || n_nb > kGmMaxNb || width < 2 || height < 2 ||
        n_cand < 3 || n_cand > 1024 || !(window > 0.f) || !(window < 1e30f) || ((uintptr_t)feats & 15) ||
        (int64_t)width * height * channels > INT32_MAX)
        return GS_ERR_INVALID_ARG;
    const void* fn = channels == 8    ? (const void*)k_guided_depth<8>
                     : channels == 16 ? (const void*)k_guided_depth<16>
                     : channels == 32 ? (const void*)k_guided_depth<32>
                     : channels == 64 ? (const void*)k_guided_depth<64>
                                      : nullptr;
    if (!fn) return GS_ERR_INVALID_ARG;
    const int64_t n_tiles = ceil_div(width, kGmTileX) * ceil_div(height, kGmTileY);
    const int grid = (int)(n_tiles < persistent_grid(fn, 256) ? n_tiles : persistent_grid(fn, 256));
    void* args[] = {(void*)&feats, (void*)&cams, (void*)&n_nb, (void*)&width, (void*)&height, (void*)&z_mono,
                    (void*)&n_cand, (void*)&window, (void*)&depth, (void*)&nb, (void*)&corr};
    if (cudaLaunchKernel(fn, dim3(grid), dim3(256), args, 0, (cudaStream_t)stream) != cudaSuccess) {
        (void)cudaGetLastError();
        return GS_ERR_CUDA;
    }
    count_launch();
    GS_CUDA_CHECK_LAUNCH();
    return GS_OK;
}
