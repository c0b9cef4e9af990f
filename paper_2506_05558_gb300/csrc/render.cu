// Front-to-back alpha compositing (K5) and its adjoint (K6).
//
// One CTA of TILE x TILE threads per tile (TILE = 8, 16 or 32), one pixel per
// thread; each warp owns an 8x4 block of pixels so a small splat touches few
// warps. Each tile's depth-ordered list is walked in batches staged in shared
// memory (128-bit loads of the projected rows). While staging, each Gaussian
// gets the bounding box of the region where its alpha can reach alpha_min; a
// warp tests 32 staged boxes against its 8x4 block with one ballot and
// evaluates only the hits, so Gaussians that cannot touch any of its pixels
// cost nothing. The forward stops a CTA when every pixel's transmittance has
// terminated. The adjoint recomputes the blending state back to front from
// T_final and n_contrib, records per pixel and Gaussian two scalars in a
// per-warp table, forms each Gaussian's 9 partial derivatives from the table
// (sums over the warp's pixels in a fixed order), sums the warps in a fixed
// order and writes ONE partial per (tile, Gaussian) pair to the pair's
// emission slot. No atomics touch gradients: bit-reproducible.
//
// Scheduling: either one CTA per tile (grid order), or persistent CTAs (as
// many as fit on the SMs) that pull tiles from a global counter in the order
// gs_sort produced (largest pair list first), which evens out the tail when
// views of very different sizes and densities share one launch. The counter
// only hands out work; every loop is bounded by the tile count.
#include "common.cuh"

namespace gs {

template <int TILE>
struct Geom {
    static constexpr int kThreads = TILE * TILE;
    static constexpr int kWarps = kThreads / 32;
    static constexpr int kWX = TILE / 8;  // 8x4 warp blocks per tile row
};

struct TileInfo {
    int view, px, py, W, H;
    bool inside;
    int64_t pix;         // pixel index within all views
    int64_t plane;       // H*W of the view
    int64_t color_base;  // index of this pixel's red value in the colour buffer
};

template <int TILE>
__device__ __forceinline__ TileInfo tile_info(const gs_frame& f, int tile) {
    TileInfo t;
    t.view = view_of_tile(f, tile);
    const int local = tile - f.tile_base[t.view];
    const int tx = local % f.tiles_x[t.view], ty = local / f.tiles_x[t.view];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int lx = (w % Geom<TILE>::kWX) * 8 + (lane & 7);
    const int ly = (w / Geom<TILE>::kWX) * 4 + (lane >> 3);
    t.px = tx * TILE + lx;
    t.py = ty * TILE + ly;
    t.W = f.width[t.view];
    t.H = f.height[t.view];
    t.inside = t.px < t.W && t.py < t.H;
    t.plane = (int64_t)t.W * t.H;
    t.pix = f.pix_base[t.view] + (int64_t)t.py * t.W + t.px;
    t.color_base = 3 * f.pix_base[t.view] + (int64_t)t.py * t.W + t.px;
    return t;
}

// Staged form of a projected Gaussian: exponent coefficients in base 2,
// e = A dx^2 + B dx dy + C dy^2 = -(a dx^2 + 2 b dx dy + c dy^2)/2 * log2(e),
// and the bounding box (x0, y0, x1, y1) of the ellipse where o exp(-q/2) can
// reach alpha_min (q = d^T conic d <= 2 ln(o / alpha_min)); the box is widened
// by 0.1% + 0.01 px so that FP32 evaluation never finds a hit outside it.
__device__ __forceinline__ void stage(const float2* __restrict__ mean2d, const float4* __restrict__ conic_opa,
                                      const float4* __restrict__ rgb_depth, uint32_t idx, float alpha_min, float2& xy,
                                      float4& abco, float4& rgb, float4& box) {
    xy = mean2d[idx];
    const float4 co = conic_opa[idx];
    abco = make_float4(-0.5f * kLog2e * co.x, -kLog2e * co.y, -0.5f * kLog2e * co.z, co.w);
    rgb = rgb_depth[idx];
    const float det = co.x * co.z - co.y * co.y;
    if (!(co.w >= alpha_min)) {
        box = make_float4(1e30f, 1e30f, -1e30f, -1e30f);  // can never reach alpha_min
    } else if (!(det > 0.f)) {
        box = make_float4(-1e30f, -1e30f, 1e30f, 1e30f);  // degenerate conic: never skip
    } else {
        const float t = 2.f * logf(co.w / alpha_min);
        const float hx = sqrtf(fmaxf(t * co.z / det, 0.f)) * 1.001f + 0.01f;
        const float hy = sqrtf(fmaxf(t * co.x / det, 0.f)) * 1.001f + 0.01f;
        box = make_float4(xy.x - hx, xy.y - hy, xy.x + hx, xy.y + hy);
    }
}

struct WarpBlock {
    float x0, y0, x1, y1;  // pixel-centre extent of this warp's 8x4 block
    __device__ __forceinline__ bool hits(const float4& b) const {
        return b.x <= x1 && b.z >= x0 && b.y <= y1 && b.w >= y0;
    }
};

__device__ __forceinline__ WarpBlock warp_block(const TileInfo& ti) {
    const int lane = threadIdx.x & 31;
    WarpBlock wb;
    wb.x0 = (float)(ti.px - (lane & 7)) + 0.5f;
    wb.y0 = (float)(ti.py - (lane >> 3)) + 0.5f;
    wb.x1 = wb.x0 + 7.f;
    wb.y1 = wb.y0 + 3.f;
    return wb;
}

// Exponent (base 2) of the Gaussian at offset (dx, dy). The same rounding
// sequence is used forward and backward so both take identical decisions.
__device__ __forceinline__ float exponent2(const float4& abco, float dx, float dy) {
    return __fmaf_rn(__fmul_rn(abco.x, dx), dx,
                     __fmaf_rn(__fmul_rn(abco.z, dy), dy, __fmul_rn(__fmul_rn(abco.y, dx), dy)));
}

// Next tile for this CTA: its own (grid schedule, first call only: tile
// blockIdx.x, or entry blockIdx.x of the work order in the ordered-grid
// schedule) or the next entry of the work order (persistent schedule, with
// the counter). Returns -1 when done.
__device__ __forceinline__ int next_tile(const uint32_t* __restrict__ order, uint32_t* counter, int n_tiles,
                                         bool first, int* s_item) {
    if (!counter) return first ? (order ? (int)order[blockIdx.x] : (int)blockIdx.x) : -1;
    if (threadIdx.x == 0) {
        const uint32_t it = atomicAdd(counter, 1u);
        *s_item = it < (uint32_t)n_tiles ? (int)order[it] : -1;
    }
    __syncthreads();
    const int t = *s_item;
    __syncthreads();
    return t;
}

// DEPTH: also accumulate the depth integral sum_i alpha_i T_i z_i per pixel.
// COUNT (measurement only, never the timed instantiation): also count, into
// counts[0..2], the warp hits the ballot passes (each one runs the compositing
// step on all 32 lanes), the lane evaluations of pixels not yet terminated at
// those hits, and the evaluations that composite (alpha >= alpha_min, before
// termination) - the work the definition requires.
template <int TILE, int FB, bool DEPTH, bool COUNT = false>
__global__ void __launch_bounds__(TILE * TILE) k_render_fwd(gs_frame f, gs_config cfg,
                                                            const uint32_t* __restrict__ range,
                                                            const uint32_t* __restrict__ src,
                                                            const float2* __restrict__ mean2d,
                                                            const float4* __restrict__ conic_opa,
                                                            const float4* __restrict__ rgb_depth,
                                                            float* __restrict__ color, float* __restrict__ t_final,
                                                            int32_t* __restrict__ n_contrib,
                                                            float* __restrict__ depth_out,
                                                            const uint32_t* __restrict__ order, uint32_t* counter,
                                                            int n_tiles, unsigned long long* counts) {
    constexpr int NT = Geom<TILE>::kThreads;
    unsigned long long n_hit = 0, n_eval = 0, n_comp = 0;
    __shared__ float2 s_xy[FB];
    __shared__ float4 s_abco[FB];
    __shared__ float4 s_rgb[FB];
    __shared__ float4 s_box[FB];
    __shared__ int s_item;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    for (int tile = next_tile(order, counter, n_tiles, true, &s_item); tile >= 0;
         tile = next_tile(order, counter, n_tiles, false, &s_item)) {
        const TileInfo ti = tile_info<TILE>(f, tile);
        const WarpBlock wb = warp_block(ti);
        const float px = ti.px + 0.5f, py = ti.py + 0.5f;
        const uint32_t start = range[2 * tile], end = range[2 * tile + 1];
        float T = 1.f, cr = 0.f, cg = 0.f, cb = 0.f, cz = 0.f;
        int last = 0;
        bool done = !ti.inside;
        for (uint32_t b0 = start; b0 < end; b0 += FB) {
            if (__syncthreads_count(done) == NT) break;
            for (int j = threadIdx.x; j < FB; j += NT)
                if (b0 + j < end)
                    stage(mean2d, conic_opa, rgb_depth, src[b0 + j], cfg.alpha_min, s_xy[j], s_abco[j], s_rgb[j],
                          s_box[j]);
            __syncthreads();
            const int cnt = min((uint32_t)FB, end - b0);
            int lastk = -1;  // staged index of this batch's last composited Gaussian
            for (int k0 = 0; k0 < cnt; k0 += 32) {
                if (__all_sync(FULL, done)) break;
                const int kk = k0 + lane;
                unsigned m = __ballot_sync(FULL, kk < cnt && wb.hits(s_box[kk < cnt ? kk : 0]));
                // predicated: every lane runs the same instructions, the
                // pixel's state changes only where the Gaussian composites
                auto composite = [&](int k, const float2 xy, const float4 abco, const float4 c) {
                    const float e = exponent2(abco, px - xy.x, py - xy.y);
                    const float og = __fmul_rn(abco.w, fast_exp2(e));
                    const float alpha = fminf(cfg.alpha_max, og);
                    const bool ok = !done && !(e > 0.f) && alpha >= cfg.alpha_min;
                    const float aT = __fmul_rn(alpha, T);  // the blending weight
                    const float nT = __fsub_rn(T, aT);     // T (1 - alpha)
                    const bool term = ok && nT < cfg.t_min;
                    const bool acc = ok && !term;
                    if (COUNT) {
                        n_hit += 1;
                        n_eval += !done;
                        n_comp += acc;
                    }
                    done = done || term;
                    const float w = acc ? aT : 0.f;
                    cr += w * c.x; cg += w * c.y; cb += w * c.z;
                    if (DEPTH) cz += w * c.w;
                    T = acc ? nT : T;
                    lastk = acc ? k : lastk;
                };
                // two hits per round (warp-uniform): both Gaussians' shared
                // loads are issued before the first composites, in order
                while (m) {
                    const int ka = k0 + __ffs(m) - 1;
                    m &= m - 1;
                    const bool two = m != 0;
                    const int kb = two ? k0 + __ffs(m) - 1 : ka;
                    m &= m - 1;
                    const float2 xya = s_xy[ka], xyb = s_xy[kb];
                    const float4 aba = s_abco[ka], abb = s_abco[kb];
                    const float4 ca = s_rgb[ka], cb2 = s_rgb[kb];
                    composite(ka, xya, aba, ca);
                    if (two) composite(kb, xyb, abb, cb2);
                }
            }
            if (lastk >= 0) last = (int)(b0 - start) + lastk + 1;
        }
        if (ti.inside) {
            color[ti.color_base] = cr + T * cfg.bg[0];
            color[ti.color_base + ti.plane] = cg + T * cfg.bg[1];
            color[ti.color_base + 2 * ti.plane] = cb + T * cfg.bg[2];
            t_final[ti.pix] = T;
            n_contrib[ti.pix] = last;
            if (DEPTH) depth_out[ti.pix] = cz;
        }
        __syncthreads();  // shared buffers are reused by the next tile
    }
    if (COUNT) {
        for (int o = 16; o > 0; o >>= 1) {
            n_eval += __shfl_xor_sync(FULL, n_eval, o);
            n_comp += __shfl_xor_sync(FULL, n_comp, o);
        }
        if (lane == 0) {
            atomicAdd(&counts[0], n_hit);  // every lane counted the warp's hits; lane 0 reports them once
            atomicAdd(&counts[1], n_eval);
            atomicAdd(&counts[2], n_comp);
        }
    }
}

// Compositing adjoint. Per pixel (one lane) and Gaussian, back to front: the
// transmittance in front of it, dL/dalpha and from it the two scalars that all
// nine gradient terms of the (tile, Gaussian) pair are built from - dpow =
// dL/d(exponent) and the blending weight. Rather than a 9-value warp reduction
// per Gaussian, each warp keeps the scalars of its last kBwdHits Gaussians in a
// shared table (row = Gaussian, column = pixel) and, when full, four lanes per
// Gaussian form sum(dpow), sum(dpow dx), ..., sum(w dL/dc) over eight pixels
// each and combine in a fixed order: about a third fewer instructions per hit.
constexpr int kBwdHits = 8;  // hits per table flush (4 lanes per hit, 8 pixels each)

template <int TILE, int BB>
__global__ void __launch_bounds__(TILE * TILE) k_render_bwd(gs_frame f, gs_config cfg,
                                                            const uint32_t* __restrict__ range,
                                                            const uint32_t* __restrict__ src,
                                                            const uint32_t* __restrict__ emit,
                                                            const float2* __restrict__ mean2d,
                                                            const float4* __restrict__ conic_opa,
                                                            const float4* __restrict__ rgb_depth,
                                                            const float* __restrict__ t_final,
                                                            const int32_t* __restrict__ n_contrib,
                                                            const float* __restrict__ dL_dcolor,
                                                            float4* __restrict__ part0, float4* __restrict__ part1,
                                                            float* __restrict__ part2, int64_t capacity,
                                                            const uint32_t* __restrict__ order, uint32_t* counter,
                                                            int n_tiles) {
    constexpr int NT = Geom<TILE>::kThreads;
    constexpr int NW = Geom<TILE>::kWarps;
    __shared__ float2 s_xy[BB];
    __shared__ float4 s_abco[BB];
    __shared__ float4 s_rgb[BB];
    __shared__ float4 s_box[BB];
    __shared__ uint32_t s_emit[BB];
    __shared__ float s_part[NW][BB][9];
    __shared__ uint32_t s_hit[NW][BB / 32];  // which Gaussians each warp wrote
    // per warp: the last HB hits' per-pixel adjoint scalars (row = hit, column =
    // pixel) and each pixel's colour gradient
    __shared__ float2 s_tdw[NW][kBwdHits][33];  // (dpow, weight)
    __shared__ float4 s_pix[NW][32];
    __shared__ int s_max;
    __shared__ int s_item;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const float inv_log2e = 1.f / kLog2e;
    for (int tile = next_tile(order, counter, n_tiles, true, &s_item); tile >= 0;
         tile = next_tile(order, counter, n_tiles, false, &s_item)) {
        const TileInfo ti = tile_info<TILE>(f, tile);
        const WarpBlock wb = warp_block(ti);
        const float px = ti.px + 0.5f, py = ti.py + 0.5f;
        const uint32_t start = range[2 * tile];
        float Tf = 1.f, gr = 0.f, gg = 0.f, gb = 0.f;
        int nc = 0;
        if (ti.inside) {
            Tf = t_final[ti.pix];
            nc = n_contrib[ti.pix];
            gr = dL_dcolor[ti.color_base];
            gg = dL_dcolor[ti.color_base + ti.plane];
            gb = dL_dcolor[ti.color_base + 2 * ti.plane];
        }
        if (threadIdx.x == 0) s_max = 0;
        __syncthreads();
        const int warp_nc = __reduce_max_sync(FULL, (unsigned)nc);
        if (lane == 0) atomicMax(&s_max, warp_nc);
        __syncthreads();
        const int n_list = s_max;
        // pairs past every pixel's last contributor get a zero partial (their
        // emission slots are summed per Gaussian like all others)
        const uint32_t len = range[2 * tile + 1] - start;
        for (uint32_t j = (uint32_t)n_list + threadIdx.x; j < len; j += NT) {
            const uint32_t e = emit[start + j];
            if ((int64_t)e < capacity) {
                part0[e] = make_float4(0.f, 0.f, 0.f, 0.f);
                part1[e] = make_float4(0.f, 0.f, 0.f, 0.f);
                part2[e] = 0.f;
            }
        }
        // gS = sum over channels of dL/dC_ch times the colour composited behind the
        // current Gaussian plus the background seen through T_final: dL/dalpha needs
        // only this dot product, so one scalar replaces three running colours
        float T = Tf, gS = Tf * (gr * cfg.bg[0] + gg * cfg.bg[1] + gb * cfg.bg[2]);
        s_pix[w][lane] = make_float4(gr, gg, gb, 0.f);
        int nh = 0;    // hits recorded in this warp's table (warp-uniform)
        int myk = 0;   // the staged index of hit (lane % HB) of the table
        // Sums over the warp's 32 pixels of the 9 gradient terms of each recorded
        // hit: lanes r, r + HB, ... share hit r, each summing 32 / L pixels from the
        // table, then combine in a fixed order; the first writes the CTA partial.
        auto flush = [&]() {
            __syncwarp();
            const int r = lane % kBwdHits, part = lane / kBwdHits;
            const bool act = r < nh;
            float S[9];
#pragma unroll
            for (int c = 0; c < 9; c++) S[c] = 0.f;
            float4 abco = make_float4(0.f, 0.f, 0.f, 1.f);
            if (act) {
                const float2 xy = s_xy[myk];
                abco = s_abco[myk];
                // pixel p = 8 part + i sits at (x0 + i, y0 + part): the same floats as the
                // compositing pass's pixel centres, so dx is identical; dy is constant over
                // this lane's row, so the dy terms follow from sum(d) and sum(d dx)
                static_assert(kBwdHits == 8, "one pixel row per lane");
                const float dy = (wb.y0 + (float)part) - xy.y;
#pragma unroll
                for (int i = 0; i < kBwdHits; i++) {
                    const int pp = part * kBwdHits + i;
                    const float dx = (wb.x0 + (float)i) - xy.x;
                    const float2 dw = s_tdw[w][r][pp];
                    const float d = dw.x, wv = dw.y;
                    const float4 pc = s_pix[w][pp];
                    const float t1 = d * dx;
                    S[0] += d; S[1] += t1; S[3] += t1 * dx;
                    S[6] += wv * pc.x; S[7] += wv * pc.y; S[8] += wv * pc.z;
                }
                S[2] = dy * S[0];
                S[4] = dy * S[1];
                S[5] = dy * S[2];
            }
#pragma unroll
            for (int off = kBwdHits; off < 32; off <<= 1)
#pragma unroll
                for (int c = 0; c < 9; c++) S[c] += __shfl_xor_sync(FULL, S[c], off);
            if (act && part == 0) {
                float* o = s_part[w][myk];
                o[0] = -inv_log2e * (2.f * abco.x * S[1] + abco.y * S[2]);
                o[1] = -inv_log2e * (abco.y * S[1] + 2.f * abco.z * S[2]);
                o[2] = -0.5f * S[3];
                o[3] = -S[4];
                o[4] = -0.5f * S[5];
                o[5] = abco.w > 0.f ? S[0] / abco.w : 0.f;  // sum of dalpha G = sum of dalpha (o G) / o
                o[6] = S[6]; o[7] = S[7]; o[8] = S[8];
            }
            nh = 0;
            __syncwarp();
        };
        for (int bend = n_list; bend > 0; bend -= BB) {
            const int b0 = max(0, bend - BB);
            const int cnt = bend - b0;
            __syncthreads();
            for (int j = threadIdx.x; j < cnt; j += NT) {
                const uint32_t p = start + b0 + j;
                stage(mean2d, conic_opa, rgb_depth, src[p], cfg.alpha_min, s_xy[j], s_abco[j], s_rgb[j], s_box[j]);
                s_emit[j] = emit[p];
            }
            __syncthreads();
            for (int ch = (cnt - 1) >> 5; ch >= 0; ch--) {
                const int k0 = ch * 32;
                const int kk = k0 + lane;
                const bool cand = kk < cnt && b0 + kk < warp_nc;
                unsigned m = __ballot_sync(FULL, cand && wb.hits(s_box[cand ? kk : 0]));
                const unsigned hits = m;
                unsigned skipped = 0;  // hits where no pixel of the warp composites (rare)
                const int ncb = nc - b0 - k0;  // this lane's contributors past the chunk start
                while (m) {  // back to front inside the chunk
                    const int jb = 31 - __clz(m);
                    m &= ~(1u << jb);
                    const int k = k0 + jb;
                    const float2 xy = s_xy[k];
                    const float4 abco = s_abco[k];
                    const float dx = px - xy.x, dy = py - xy.y;
                    const float e = exponent2(abco, dx, dy);
                    const float G = fast_exp2(e);
                    const float og = __fmul_rn(abco.w, G);
                    const float alpha = fminf(cfg.alpha_max, og);
                    // same decisions as the forward pass: listed before this pixel's
                    // last contributor, exponent <= 0, alpha >= alpha_min
                    const bool contrib = jb < ncb && !(e > 0.f) && alpha >= cfg.alpha_min;
                    if (__any_sync(FULL, contrib)) {
                        // predicated adjoint: non-contributing lanes keep their
                        // state and add zeros
                        const float inv = fast_rcp(1.f - alpha);
                        T = contrib ? T * inv : T;  // transmittance in front of this Gaussian
                        const float4 c = s_rgb[k];
                        const float wgt = contrib ? alpha * T : 0.f;
                        // dL/dalpha = sum_ch dL/dC_ch (T c_ch - S_ch / (1 - alpha))
                        const float gc = gr * c.x + gg * c.y + gb * c.z;
                        const float dalpha = T * gc - gS * inv;
                        gS += wgt * gc;
                        // alpha clamped at alpha_max passes no gradient to the exponent or
                        // opacity; selects (not products with 0) keep a non-finite og or G
                        // of a lane outside the Gaussian out of the sums
                        const bool pass = contrib && og < cfg.alpha_max;
                        const float dpow = pass ? dalpha * og : 0.f;  // d alpha / d(natural exponent)
                        // record this pixel's two scalars; the 9 gradient terms are summed
                        // over the warp's pixels when the table is full
                        s_tdw[w][nh][lane] = make_float2(dpow, wgt);
                        if (lane % kBwdHits == nh) myk = k;
                        if (++nh == kBwdHits) flush();
                    } else {
                        skipped |= 1u << jb;
                    }
                }
                if (lane == 0) s_hit[w][ch] = hits & ~skipped;
            }
            if (nh > 0) flush();
            __syncthreads();
            for (int j = threadIdx.x; j < cnt; j += NT) {
                const int ch = j >> 5;
                const uint32_t bit = 1u << (j & 31);
                float a[9];
#pragma unroll
                for (int c = 0; c < 9; c++) a[c] = 0.f;
                for (int ww = 0; ww < NW; ww++)
                    if (s_hit[ww][ch] & bit)
#pragma unroll
                        for (int c = 0; c < 9; c++) a[c] += s_part[ww][j][c];
                const uint32_t e = s_emit[j];
                if ((int64_t)e < capacity) {
                    part0[e] = make_float4(a[0], a[1], a[2], a[3]);
                    part1[e] = make_float4(a[4], a[5], a[6], a[7]);
                    part2[e] = a[8];
                }
            }
        }
        __syncthreads();  // shared buffers are reused by the next tile
    }
}

// ---------------------------------------------------------------------------
// Launch configurations (the autotuner picks among these)
// ---------------------------------------------------------------------------
struct RenderLaunch {
    const void* fn;
    int threads;
};

static RenderLaunch pick_fwd(int tile, int batch, bool depth = false, bool count = false) {
#define GS_FWD(T, B)                                                                     \
    if (tile == T && batch == B)                                                         \
        return {count   ? (const void*)k_render_fwd<T, B, false, true>                   \
                : depth ? (const void*)k_render_fwd<T, B, true>                          \
                        : (const void*)k_render_fwd<T, B, false>,                        \
                T * T};
    GS_FWD(8, 64) GS_FWD(8, 128) GS_FWD(8, 256)
    GS_FWD(16, 64) GS_FWD(16, 128) GS_FWD(16, 256)
    GS_FWD(32, 128) GS_FWD(32, 256)
#undef GS_FWD
    return {nullptr, 0};
}

static RenderLaunch pick_bwd(int tile, int batch) {
#define GS_BWD(T, B) if (tile == T && batch == B) return {(const void*)k_render_bwd<T, B>, T * T};
    GS_BWD(8, 64) GS_BWD(8, 128) GS_BWD(8, 256)
    GS_BWD(16, 32) GS_BWD(16, 64) GS_BWD(16, 128)
    GS_BWD(32, 32)
#undef GS_BWD
    return {nullptr, 0};
}

static int default_fwd_batch(int tile) { return tile == 8 ? 128 : 256; }
static int default_bwd_batch(int tile) { return tile == 32 ? 32 : tile == 16 ? 64 : 128; }

static int launch(const RenderLaunch& L, int n_tiles, bool persistent, void** args, cudaStream_t s) {
    int grid = n_tiles;
    if (persistent) {
        const int pg = persistent_grid(L.fn, L.threads);
        grid = n_tiles < pg ? n_tiles : pg;
    }
    if (cudaLaunchKernel(L.fn, dim3(grid), dim3(L.threads), args, 0, s) != cudaSuccess) {
        (void)cudaGetLastError();
        return GS_ERR_CUDA;
    }
    count_launch();
    return GS_OK;
}

bool render_batch_supported(int tile, int fwd_batch, int bwd_batch) {
    return pick_fwd(tile, fwd_batch ? fwd_batch : default_fwd_batch(tile)).fn != nullptr &&
           pick_bwd(tile, bwd_batch ? bwd_batch : default_bwd_batch(tile)).fn != nullptr;
}

}  // namespace gs

using namespace gs;

extern "C" size_t gs_render_workspace_size(const gs_frame* f) {
    (void)f;
    return 256;  // the persistent schedule's work counter
}

static bool render_args_ok(const gs_frame* f, const gs_config* cfg) {
    return f && cfg && f->n_views >= 1 && f->n_views <= GS_MAX_VIEWS && cfg->tile == f->tile &&
           render_batch_supported(cfg->tile, cfg->fwd_batch, cfg->bwd_batch);
}

static int render_fwd_impl(const gs_projected* p, const gs_pairs* pairs, const gs_frame* f, const gs_config* cfg,
                           const gs_image* out, void* ws, size_t ws_bytes, void* stream, unsigned long long* counts) {
    if (!p || !pairs || !out || !out->color || !out->t_final || !out->n_contrib || !render_args_ok(f, cfg))
        return GS_ERR_INVALID_ARG;
    const bool persistent = cfg->schedule == 1, ordered = cfg->schedule == 2;
    if (persistent && (!pairs->order || !ws || ws_bytes < 256)) return GS_ERR_INVALID_ARG;
    if (ordered && !pairs->order) return GS_ERR_INVALID_ARG;
    int n_tiles = f->tile_base[f->n_views];
    cudaStream_t s = (cudaStream_t)stream;
    if (counts && cudaMemsetAsync(counts, 0, 3 * sizeof(unsigned long long), s) != cudaSuccess) {
        (void)cudaGetLastError();
        return GS_ERR_CUDA;
    }
    if (n_tiles == 0) return GS_OK;
    uint32_t* counter = persistent ? (uint32_t*)ws : nullptr;
    const uint32_t* order = persistent || ordered ? pairs->order : nullptr;
    if (persistent) cudaMemsetAsync(counter, 0, sizeof(uint32_t), s);
    const RenderLaunch L = pick_fwd(cfg->tile, cfg->fwd_batch ? cfg->fwd_batch : default_fwd_batch(cfg->tile),
                                    out->depth != nullptr && !counts, counts != nullptr);
    gs_frame fv = *f;
    gs_config cv = *cfg;
    const uint32_t* range = pairs->range;
    const uint32_t* src = pairs->src;
    const float2* m2 = (const float2*)p->mean2d;
    const float4* co = (const float4*)p->conic_opa;
    const float4* rd = (const float4*)p->rgb_depth;
    float* color = out->color;
    float* tf = out->t_final;
    int32_t* nc = out->n_contrib;
    float* dz = out->depth;
    void* args[] = {&fv, &cv, (void*)&range, (void*)&src, (void*)&m2, (void*)&co, (void*)&rd,
                    (void*)&color, (void*)&tf, (void*)&nc, (void*)&dz, (void*)&order, (void*)&counter, &n_tiles,
                    (void*)&counts};
    return launch(L, n_tiles, persistent, args, s);
}

extern "C" int gs_render_fwd(const gs_projected* p, const gs_pairs* pairs, const gs_frame* f, const gs_config* cfg,
                             const gs_image* out, void* ws, size_t ws_bytes, void* stream) {
    return render_fwd_impl(p, pairs, f, cfg, out, ws, ws_bytes, stream, nullptr);
}

extern "C" int gs_render_fwd_count(const gs_projected* p, const gs_pairs* pairs, const gs_frame* f,
                                   const gs_config* cfg, const gs_image* out, void* ws, size_t ws_bytes,
                                   unsigned long long* counts, void* stream) {
    if (!counts) return GS_ERR_INVALID_ARG;
    return render_fwd_impl(p, pairs, f, cfg, out, ws, ws_bytes, stream, counts);
}

namespace gs {
int launch_render_bwd(const gs_projected* p, const gs_pairs* pairs, const gs_frame* f, const gs_config* cfg,
                      const gs_image* fwd, const float* dL_dcolor, float4* part0, float4* part1, float* part2,
                      uint32_t* counter, cudaStream_t s) {
    if (!render_args_ok(f, cfg)) return GS_ERR_INVALID_ARG;
    int n_tiles = f->tile_base[f->n_views];
    if (n_tiles == 0) return GS_OK;
    const bool persistent = cfg->schedule == 1, ordered = cfg->schedule == 2;
    if ((persistent || ordered) && !pairs->order) return GS_ERR_INVALID_ARG;
    const uint32_t* order = persistent || ordered ? pairs->order : nullptr;
    if (!persistent) counter = nullptr;
    if (persistent) cudaMemsetAsync(counter, 0, sizeof(uint32_t), s);
    const RenderLaunch L = pick_bwd(cfg->tile, cfg->bwd_batch ? cfg->bwd_batch : default_bwd_batch(cfg->tile));
    gs_frame fv = *f;
    gs_config cv = *cfg;
    const uint32_t* range = pairs->range;
    const uint32_t* src = pairs->src;
    const uint32_t* emit = pairs->emit;
    const float2* m2 = (const float2*)p->mean2d;
    const float4* co = (const float4*)p->conic_opa;
    const float4* rd = (const float4*)p->rgb_depth;
    const float* tf = fwd->t_final;
    const int32_t* nc = fwd->n_contrib;
    int64_t cap = pairs->capacity;
    void* args[] = {&fv, &cv, (void*)&range, (void*)&src, (void*)&emit, (void*)&m2, (void*)&co, (void*)&rd,
                    (void*)&tf, (void*)&nc, (void*)&dL_dcolor, (void*)&part0, (void*)&part1, (void*)&part2,
                    &cap, (void*)&order, (void*)&counter, &n_tiles};
    return launch(L, n_tiles, persistent, args, s);
}
}  // namespace gs
