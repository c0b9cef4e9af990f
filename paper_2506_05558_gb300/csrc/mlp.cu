// Learned spawn proposal: a per-8x8-patch MLP (194 -> 128 -> 128 -> 128 -> 3,
// GELU) with bfloat16 weights/activations and FP32 accumulation, its loss
// against the spawns kept by direct sampling, backward pass and Adam.
//
// Every matrix product is one "TN" GEMM: C[m][n] = sum_k A[m][k] B[n][k], both
// operands bfloat16 and K-major, FP32 accumulation, optional split-K (the
// weight gradients contract over all patches). The producers write each
// activation both row-major and transposed so every product has K-major
// operands: forward Z = H W^T (A = H, B = W), input gradient dH = dZ W (A = dZ,
// B = W^T), weight gradient dW = dZ^T H (A = dZ^T, B = H^T). Elementwise work
// (bias, GELU, its derivative, the loss, the casts) sits in small kernels
// around the GEMMs; partial sums over patches are reduced in a fixed order.
#include <cuda_bf16.h>

#include "common.cuh"
#include "mlp_gemm.cuh"

namespace gs {

constexpr int kIn = 194, kInPad = 208, kHid = 128, kOut = 3, kOutPad = 16;
constexpr int kPatch = 8;
constexpr int kRowAlign = 128;  // patch rows are padded to a multiple of this
constexpr int kSplitK = 256;    // patches per split of a weight-gradient GEMM

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// Kernels that write an activation both row-major [Mp][N] and transposed
// [N][Mp] work on 32 x 32 tiles (blockDim 32 x 8): the row-major value is
// written directly and the tile is turned in shared memory so the transposed
// store is coalesced too.
struct TileT {
    __nv_bfloat16 v[32][33];
};

__device__ __forceinline__ void store_transposed(TileT& t, __nv_bfloat16* __restrict__ dst_t, int64_t Mp, int N,
                                                 int64_t m0, int n0) {
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {  // r: column n of the source tile
        const int n = n0 + r;
        const int64_t m = m0 + threadIdx.x;
        if (n < N && m < Mp) dst_t[(int64_t)n * Mp + m] = t.v[threadIdx.x][r];
    }
}

// X [Mp][208] and X^T [208][Mp] (bf16) from image [3][H][W]; rows >= M and
// columns >= 194 are zero. Row (py, px) in row-major patch order.
__global__ void __launch_bounds__(256) k_mlp_features(const float* __restrict__ image, int W, int H, int64_t M,
                                                      int64_t Mp, __nv_bfloat16* __restrict__ X,
                                                      __nv_bfloat16* __restrict__ Xt) {
    __shared__ TileT t;
    const int64_t m0 = (int64_t)blockIdx.y * 32;
    const int n0 = blockIdx.x * 32;
    const int c = n0 + threadIdx.x;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int64_t m = m0 + r;
        float v = 0.f;
        if (m < M && c < kInPad) {
            const int nx = W / kPatch, ny = H / kPatch;
            const int px = (int)(m % nx), py = (int)(m / nx);
            if (c < 192) {
                const int ch = c / 64, dy = (c % 64) / 8, dx = c % 8;
                v = image[(int64_t)ch * W * H + (int64_t)(py * kPatch + dy) * W + px * kPatch + dx];
            } else if (c == 192) {
                v = (px + 0.5f) / nx * 2.f - 1.f;
            } else if (c == 193) {
                v = (py + 0.5f) / ny * 2.f - 1.f;
            }
        }
        const __nv_bfloat16 b = __float2bfloat16_rn(v);
        if (m < Mp && c < kInPad) X[m * kInPad + c] = b;
        t.v[r][threadIdx.x] = b;
    }
    store_transposed(t, Xt, Mp, kInPad, m0, n0);
}

// Z += b; H = bf16(GELU(Z)) row-major and transposed. Z [Mp][N], b [N].
__global__ void __launch_bounds__(256) k_mlp_bias_gelu(float* __restrict__ Z, const float* __restrict__ b,
                                                       int64_t Mp, int N, __nv_bfloat16* __restrict__ Hm,
                                                       __nv_bfloat16* __restrict__ Ht) {
    __shared__ TileT t;
    const int64_t m0 = (int64_t)blockIdx.y * 32;
    const int n0 = blockIdx.x * 32;
    const int n = n0 + threadIdx.x;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int64_t m = m0 + r;
        __nv_bfloat16 h = __float2bfloat16_rn(0.f);
        if (m < Mp && n < N) {
            const float z = Z[m * N + n] + b[n];
            Z[m * N + n] = z;
            h = __float2bfloat16_rn(gelu_f(z));
            Hm[m * N + n] = h;
        }
        t.v[r][threadIdx.x] = h;
    }
    store_transposed(t, Ht, Mp, N, m0, n0);
}

// Output layer: Y = Z4 + b4 (first 3 columns). Loss terms and dY; rows >= M
// give dY = 0. targets [M][4] = (spawn fraction, depth, log-scale, mask).
// Writes dZ4 (bf16, [Mp][16] and [16][Mp]), dY (fp32 [Mp][16], for db4) and
// one loss partial per block.
__global__ void __launch_bounds__(256) k_mlp_loss(const float* __restrict__ Z4, const float* __restrict__ b4,
                                                  const float* __restrict__ targets, int64_t M, int64_t Mp,
                                                  float w_depth, float w_scale, float* __restrict__ Y,
                                                  float* __restrict__ dY, __nv_bfloat16* __restrict__ dZ,
                                                  __nv_bfloat16* __restrict__ dZt, float* __restrict__ loss_part) {
    __shared__ float s_red[8];
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (m < Mp) {
        float g[kOutPad];
#pragma unroll
        for (int c = 0; c < kOutPad; c++) g[c] = 0.f;
        if (m < M) {
            const float logit = Z4[m * kOutPad + 0] + b4[0];
            const float depth = Z4[m * kOutPad + 1] + b4[1];
            const float ls = Z4[m * kOutPad + 2] + b4[2];
            if (Y) {
                Y[m * 3 + 0] = logit;
                Y[m * 3 + 1] = depth;
                Y[m * 3 + 2] = ls;
            }
            if (targets) {
                const float t = targets[m * 4 + 0], zt = targets[m * 4 + 1], st = targets[m * 4 + 2];
                const float mask = targets[m * 4 + 3];
                const float inv = 1.f / (float)M;
                // softplus(x) - t x, computed stably
                l = fmaxf(logit, 0.f) + log1pf(expf(-fabsf(logit))) - t * logit;
                l += w_depth * mask * fabsf(depth - zt) + w_scale * mask * fabsf(ls - st);
                l *= inv;
                auto sg = [](float x) { return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f); };
                g[0] = (1.f / (1.f + expf(-logit)) - t) * inv;
                g[1] = w_depth * mask * sg(depth - zt) * inv;
                g[2] = w_scale * mask * sg(ls - st) * inv;
            }
        }
        if (dY) {
#pragma unroll
            for (int c = 0; c < kOutPad; c++) {
                dY[m * kOutPad + c] = g[c];
                const __nv_bfloat16 b = __float2bfloat16_rn(g[c]);
                dZ[m * kOutPad + c] = b;
                dZt[(int64_t)c * Mp + m] = b;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0 && loss_part) {
        float s = 0.f;
        for (int k = 0; k < 8; k++) s += s_red[k];
        loss_part[blockIdx.x] = s;
    }
}

// dZ = dH * GELU'(Z): fp32 [Mp][N] for the bias gradient, bf16 row-major and
// transposed for the next products.
__global__ void __launch_bounds__(256) k_mlp_gelu_bwd(const float* __restrict__ dH, const float* __restrict__ Z,
                                                      int64_t Mp, int N, float* __restrict__ dZf,
                                                      __nv_bfloat16* __restrict__ dZ, __nv_bfloat16* __restrict__ dZt) {
    __shared__ TileT t;
    const int64_t m0 = (int64_t)blockIdx.y * 32;
    const int n0 = blockIdx.x * 32;
    const int n = n0 + threadIdx.x;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int64_t m = m0 + r;
        __nv_bfloat16 h = __float2bfloat16_rn(0.f);
        if (m < Mp && n < N) {
            const float d = dH[m * N + n] * gelu_grad_f(Z[m * N + n]);
            dZf[m * N + n] = d;
            h = __float2bfloat16_rn(d);
            dZ[m * N + n] = h;
        }
        t.v[r][threadIdx.x] = h;
    }
    store_transposed(t, dZt, Mp, N, m0, n0);
}

// Column sums of an fp32 [Mp][N] matrix, first pass: block b sums rows
// [256 b, 256 b + 256) of each column (thread = column); the partials are then
// summed in block order by k_split_sum.
constexpr int kColRows = 256;
__global__ void k_col_sum_part(const float* __restrict__ A, int64_t Mp, int N, float* __restrict__ part) {
    const int n = threadIdx.x;
    if (n >= N) return;
    const int64_t r0 = (int64_t)blockIdx.x * kColRows;
    float s = 0.f;
    const int64_t m1 = min(r0 + kColRows, Mp);
#pragma unroll 8
    for (int64_t m = r0; m < m1; m++) s += A[m * N + n];  // loads batched, sum in row order
    part[(int64_t)blockIdx.x * N + n] = s;
}

// Sum of S split-K partials [S][R][C] into [R][Cv] (the first Cv columns).
__global__ void k_split_sum(const float* __restrict__ part, int S, int R, int C, int Cv, int Rv,
                            float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Rv * Cv) return;
    const int r = i / Cv, c = i % Cv;
    float s = 0.f;
#pragma unroll 8
    for (int z = 0; z < S; z++) s += part[((int64_t)z * R + r) * C + c];  // loads batched, sum in split order
    out[i] = s;
}

__global__ void k_sum_partials(const float* __restrict__ p, int n, float* __restrict__ out) {
    __shared__ float s[256];
    float a = 0.f;
    for (int i = threadIdx.x; i < n; i += 256) a += p[i];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

// The four layers' casts in one launch: thread i of the concatenated padded
// matrices finds its layer from the running sizes.
struct CastAll {
    const float* Wm[4];
    __nv_bfloat16 *Wb[4], *Wt[4];
    int rv[4], cv[4], Ro[4], Ci[4];
    int64_t end[4];  // exclusive running sums of Ro * Ci
};
__global__ void k_weight_cast_all(CastAll a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int l = 0;
    while (l < 4 && i >= a.end[l]) l++;
    if (l == 4) return;
    const int64_t j = i - (l > 0 ? a.end[l - 1] : 0);
    const int r = (int)(j / a.Ci[l]), c = (int)(j % a.Ci[l]);
    const float v = (r < a.rv[l] && c < a.cv[l]) ? a.Wm[l][r * a.cv[l] + c] : 0.f;
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    a.Wb[l][j] = b;
    a.Wt[l][(int64_t)c * a.Ro[l] + r] = b;
}

// Adam over all eight parameter tensors in one launch; the gradients are flat
// in the order w1, b1, ..., w4, b4 (seg_end: exclusive running sizes).
struct AdamAll {
    float *p[8], *m[8], *v[8];
    int64_t seg_end[8];
};
__global__ void k_mlp_adam_all(AdamAll a, const float* __restrict__ g, float lr, float b1, float b2, float eps,
                               int32_t step, const int32_t* __restrict__ step_dev) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int k = 0;
    while (k < 8 && i >= a.seg_end[k]) k++;
    if (k == 8) return;
    const int64_t j = i - (k > 0 ? a.seg_end[k - 1] : 0);
    const float t = step_dev ? (float)*step_dev : (float)step;
    const float bc1 = 1.f - powf(b1, t), bc2 = 1.f - powf(b2, t);
    const float gi = g[i];
    const float mi = b1 * a.m[k][j] + (1.f - b1) * gi;
    const float vi = b2 * a.v[k][j] + (1.f - b2) * gi * gi;
    a.m[k][j] = mi;
    a.v[k][j] = vi;
    a.p[k][j] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

// ---------------------------------------------------------------------------
// Workspace
// ---------------------------------------------------------------------------
struct MlpWs {
    __nv_bfloat16 *Wb[4], *Wt[4];
    __nv_bfloat16 *X, *Xt, *H[3], *Ht[3], *dZ, *dZt, *dZ4, *dZ4t;
    float *Z[4], *dH, *dZf, *dY, *part, *loss_part, *grad;
    int64_t M, Mp, nb_loss, splits;
};

static const int kRo[4] = {kHid, kHid, kHid, kOutPad};   // padded out dims
static const int kCi[4] = {kInPad, kHid, kHid, kHid};    // padded in dims
static const int kRv[4] = {kHid, kHid, kHid, kOut};      // true out dims
static const int kCv[4] = {kIn, kHid, kHid, kHid};       // true in dims

static int64_t n_params_layer(int l) { return (int64_t)kRv[l] * kCv[l] + kRv[l]; }
static int64_t n_params_total() {
    int64_t s = 0;
    for (int l = 0; l < 4; l++) s += n_params_layer(l);
    return s;
}

static MlpWs carve_mlp(char* base, size_t cap, int64_t M, size_t* used) {
    Carve c{base, 0, cap};
    MlpWs w;
    w.M = M;
    w.Mp = ceil_div(M, kRowAlign) * kRowAlign;
    const int64_t Mp = w.Mp;
    for (int l = 0; l < 4; l++) {
        w.Wb[l] = c.take<__nv_bfloat16>((size_t)kRo[l] * kCi[l]);
        w.Wt[l] = c.take<__nv_bfloat16>((size_t)kRo[l] * kCi[l]);
    }
    w.X = c.take<__nv_bfloat16>(Mp * kInPad);
    w.Xt = c.take<__nv_bfloat16>(Mp * kInPad);
    for (int l = 0; l < 3; l++) {
        w.H[l] = c.take<__nv_bfloat16>(Mp * kHid);
        w.Ht[l] = c.take<__nv_bfloat16>(Mp * kHid);
        w.Z[l] = c.take<float>(Mp * kHid);
    }
    w.Z[3] = c.take<float>(Mp * kOutPad);
    w.dZ = c.take<__nv_bfloat16>(Mp * kHid);
    w.dZt = c.take<__nv_bfloat16>(Mp * kHid);
    w.dZ4 = c.take<__nv_bfloat16>(Mp * kOutPad);
    w.dZ4t = c.take<__nv_bfloat16>(Mp * kOutPad);
    w.dH = c.take<float>(Mp * kHid);
    w.dZf = c.take<float>(Mp * kHid);
    w.dY = c.take<float>(Mp * kOutPad);
    w.splits = ceil_div(Mp, kSplitK);
    w.part = c.take<float>((size_t)w.splits * kHid * kInPad);
    w.nb_loss = ceil_div(Mp, 256);
    w.loss_part = c.take<float>(w.nb_loss);
    w.grad = c.take<float>(n_params_total());
    *used = c.used;
    return w;
}

int mlp_forward_fused(const float* const* w, const float* const* b, const float* image, int W, int H, float* out,
                      cudaStream_t s);
int mlp_train_forward_fused(const float* const* w, const float* const* b, const float* image, int W, int H,
                            __nv_bfloat16* Xt, float* const* Z, __nv_bfloat16* const* Ht, float* Z3, int64_t Mp,
                            cudaStream_t s);

struct MlpPtrs {
    float* w[4];
    float* b[4];
};

static MlpPtrs ptrs(const gs_mlp_params* p) {
    MlpPtrs r;
    r.w[0] = p->w1; r.b[0] = p->b1; r.w[1] = p->w2; r.b[1] = p->b2;
    r.w[2] = p->w3; r.b[2] = p->b3; r.w[3] = p->w4; r.b[3] = p->b4;
    return r;
}

static bool params_ok(const gs_mlp_params* p) {
    return p && p->w1 && p->b1 && p->w2 && p->b2 && p->w3 && p->b3 && p->w4 && p->b4;
}

#define GS_LAUNCH1(kernel, n, ...)                                                          \
    do {                                                                                    \
        kernel<<<(unsigned)ceil_div((int64_t)(n), 256), 256, 0, s>>>(__VA_ARGS__);          \
        count_launch();                                                                     \
    } while (0)

// Forward: features, 4 GEMMs with their epilogues; Y and dY written by the loss
// kernel when targets are given.
static void cast_weights(const MlpPtrs& P, const MlpWs& w, cudaStream_t s) {
    CastAll a;
    int64_t acc = 0;
    for (int l = 0; l < 4; l++) {
        a.Wm[l] = P.w[l];
        a.Wb[l] = w.Wb[l];
        a.Wt[l] = w.Wt[l];
        a.rv[l] = kRv[l]; a.cv[l] = kCv[l]; a.Ro[l] = kRo[l]; a.Ci[l] = kCi[l];
        acc += (int64_t)kRo[l] * kCi[l];
        a.end[l] = acc;
    }
    k_weight_cast_all<<<(unsigned)ceil_div(acc, 256), 256, 0, s>>>(a);
    count_launch();
}

static int mlp_forward(const MlpPtrs& P, const float* image, int W, int H, const MlpWs& w, int path,
                       const float* targets, float w_depth, float w_scale, float* out, cudaStream_t s) {
    const int64_t M = w.M, Mp = w.Mp;
    cast_weights(P, w, s);
    if (path == 1 && targets && ((uintptr_t)image & 15) == 0) {
        // training forward on the tensor cores in one persistent kernel (weights resident in shared
        // memory), writing the tensors the backward reads; then the loss as below
        int rc = mlp_train_forward_fused(P.w, P.b, image, W, H, w.Xt, w.Z, w.Ht, w.Z[3], Mp, s);
        if (rc != GS_OK) return rc;
        k_mlp_loss<<<(unsigned)w.nb_loss, 256, 0, s>>>(w.Z[3], P.b[3], targets, M, Mp, w_depth, w_scale, out, w.dY,
                                                        w.dZ4, w.dZ4t, w.loss_part);
        count_launch();
        return GS_OK;
    }
    k_mlp_features<<<dim3((unsigned)ceil_div(kInPad, 32), (unsigned)ceil_div(Mp, 32)), dim3(32, 8), 0, s>>>(
        image, W, H, M, Mp, w.X, w.Xt);
    count_launch();
    const __nv_bfloat16* Hin = w.X;
    int K = kInPad;
    for (int l = 0; l < 3; l++) {
        int rc = gemm_tn(path, Hin, K, w.Wb[l], K, w.Z[l], kHid, Mp, kHid, K, K, 0, s);
        if (rc != GS_OK) return rc;
        k_mlp_bias_gelu<<<dim3((unsigned)ceil_div(kHid, 32), (unsigned)ceil_div(Mp, 32)), dim3(32, 8), 0, s>>>(
            w.Z[l], P.b[l], Mp, kHid, w.H[l], w.Ht[l]);
        count_launch();
        Hin = w.H[l];
        K = kHid;
    }
    int rc = gemm_tn(path, Hin, kHid, w.Wb[3], kHid, w.Z[3], kOutPad, Mp, kOutPad, kHid, kHid, 0, s);
    if (rc != GS_OK) return rc;
    k_mlp_loss<<<(unsigned)w.nb_loss, 256, 0, s>>>(w.Z[3], P.b[3], targets, M, Mp, w_depth, w_scale, out,
                                                    targets ? w.dY : nullptr, w.dZ4, w.dZ4t,
                                                    targets ? w.loss_part : nullptr);
    count_launch();
    return GS_OK;
}

// Backward from dY (written by mlp_forward with targets) to the fp32 gradients
// in w.grad, laid out as [w1, b1, w2, b2, w3, b3, w4, b4] (unpadded).
static int mlp_backward(const MlpWs& w, int path, cudaStream_t s) {
    const int64_t Mp = w.Mp;
    int64_t off[4], acc = 0;
    for (int l = 0; l < 4; l++) {
        off[l] = acc;
        acc += n_params_layer(l);
    }
    const __nv_bfloat16* dZ = w.dZ4;
    const __nv_bfloat16* dZt = w.dZ4t;
    const float* dZf = w.dY;
    for (int l = 3; l >= 0; l--) {
        const int out = kRo[l], in = kCi[l];
        const __nv_bfloat16* Hin_t = l > 0 ? w.Ht[l - 1] : w.Xt;
        // dW_l = dZ^T H_{l-1} over all patches (split-K), then a fixed-order sum
        int rc = gemm_tn(path, dZt, Mp, Hin_t, Mp, w.part, in, out, in, Mp, kSplitK, (int64_t)out * in, s);
        if (rc != GS_OK) return rc;
        GS_LAUNCH1(k_split_sum, kRv[l] * kCv[l], w.part, (int)w.splits, out, in, kCv[l], kRv[l], w.grad + off[l]);
        const int ncb = (int)ceil_div(Mp, kColRows);
        k_col_sum_part<<<ncb, 128, 0, s>>>(dZf, Mp, out, w.part);
        count_launch();
        GS_LAUNCH1(k_split_sum, kRv[l], w.part, ncb, 1, out, kRv[l], 1, w.grad + off[l] + (int64_t)kRv[l] * kCv[l]);
        if (l == 0) break;
        // dH_{l-1} = dZ_l W_l, then dZ_{l-1} = dH * GELU'(Z_{l-1})
        rc = gemm_tn(path, dZ, out, w.Wt[l], out, w.dH, kHid, Mp, kHid, out, out, 0, s);
        if (rc != GS_OK) return rc;
        k_mlp_gelu_bwd<<<dim3((unsigned)ceil_div(kHid, 32), (unsigned)ceil_div(Mp, 32)), dim3(32, 8), 0, s>>>(
            w.dH, w.Z[l - 1], Mp, kHid, w.dZf, w.dZ, w.dZt);
        count_launch();
        dZ = w.dZ;
        dZt = w.dZt;
        dZf = w.dZf;
    }
    return GS_OK;
}

}  // namespace gs

using namespace gs;

extern "C" int64_t gs_mlp_patches(int32_t width, int32_t height) {
    if (width <= 0 || height <= 0 || width % kPatch || height % kPatch) return -1;
    return (int64_t)(width / kPatch) * (height / kPatch);
}

extern "C" int64_t gs_mlp_param_count(void) { return n_params_total(); }

extern "C" size_t gs_mlp_workspace_size(int64_t n_patches) {
    if (n_patches <= 0) return 0;
    size_t used = 0;
    carve_mlp(nullptr, 0, n_patches, &used);
    return used;
}

static int mlp_setup(const gs_mlp_params* p, int32_t width, int32_t height, void* ws, size_t ws_bytes,
                     const gs_mlp_config* cfg, MlpWs* w) {
    if (!params_ok(p) || !cfg || (cfg->tensor_path != 0 && cfg->tensor_path != 1)) return GS_ERR_INVALID_ARG;
    const int64_t M = gs_mlp_patches(width, height);
    if (M <= 0) return GS_ERR_INVALID_ARG;
    size_t need = 0;
    *w = carve_mlp((char*)ws, ws_bytes, M, &need);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255)) return GS_ERR_INVALID_ARG;
    return GS_OK;
}

extern "C" int gs_mlp_forward(const gs_mlp_params* p, const float* image, int32_t width, int32_t height,
                              float* out, const gs_mlp_config* cfg, void* ws, size_t ws_bytes, void* stream) {
    MlpWs w;
    int rc = mlp_setup(p, width, height, ws, ws_bytes, cfg, &w);
    if (rc != GS_OK || !image || !out) return rc != GS_OK ? rc : GS_ERR_INVALID_ARG;
    const MlpPtrs P = ptrs(p);
    if (cfg->tensor_path == 1 && ((uintptr_t)image & 15) == 0) {
        // the whole network in one persistent tcgen05 kernel (weights resident in shared memory)
        rc = mlp_forward_fused(P.w, P.b, image, width, height, out, (cudaStream_t)stream);
    } else {
        rc = mlp_forward(P, image, width, height, w, cfg->tensor_path, nullptr, 0.f, 0.f, out, (cudaStream_t)stream);
    }
    if (rc != GS_OK) return rc;
    GS_CUDA_CHECK_LAUNCH();
    return GS_OK;
}

extern "C" int gs_mlp_train_step(const gs_mlp_params* p, const gs_mlp_params* m, const gs_mlp_params* v,
                                 const float* image, int32_t width, int32_t height, const float* targets,
                                 const gs_mlp_config* cfg, int32_t step, const int32_t* step_dev, float* loss,
                                 float* out, float* grads, void* ws, size_t ws_bytes, void* stream) {
    MlpWs w;
    int rc = mlp_setup(p, width, height, ws, ws_bytes, cfg, &w);
    if (rc != GS_OK) return rc;
    if (!image || !targets || !loss || (m && !params_ok(m)) || (v && !params_ok(v)) || (!m != !v) ||
        (m && step < 1 && !step_dev))
        return GS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const MlpPtrs P = ptrs(p);
    rc = mlp_forward(P, image, width, height, w, cfg->tensor_path, targets, cfg->w_depth, cfg->w_scale, out, s);
    if (rc != GS_OK) return rc;
    k_sum_partials<<<1, 256, 0, s>>>(w.loss_part, (int)w.nb_loss, loss);
    count_launch();
    rc = mlp_backward(w, cfg->tensor_path, s);
    if (rc != GS_OK) return rc;
    if (grads) {
        cudaMemcpyAsync(grads, w.grad, sizeof(float) * n_params_total(), cudaMemcpyDeviceToDevice, s);
    }
    if (m) {
        const MlpPtrs Pm = ptrs(m), Pv = ptrs(v);
        AdamAll a;
        int64_t off = 0;
        for (int l = 0; l < 4; l++) {
            const int64_t nw = (int64_t)kRv[l] * kCv[l], nbias = kRv[l];
            a.p[2 * l] = P.w[l]; a.m[2 * l] = Pm.w[l]; a.v[2 * l] = Pv.w[l];
            a.p[2 * l + 1] = P.b[l]; a.m[2 * l + 1] = Pm.b[l]; a.v[2 * l + 1] = Pv.b[l];
            off += nw;
            a.seg_end[2 * l] = off;
            off += nbias;
            a.seg_end[2 * l + 1] = off;
        }
        k_mlp_adam_all<<<(unsigned)ceil_div(off, 256), 256, 0, s>>>(a, w.grad, cfg->lr, cfg->beta1, cfg->beta2,
                                                                     cfg->eps, step, step_dev);
        count_launch();
    }
    GS_CUDA_CHECK_LAUNCH();
    return GS_OK;
}

extern "C" int gs_mlp_gemm_bf16(const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb, float* C, int64_t ldc,
                                int32_t M, int32_t N, int32_t K, int32_t tensor_path, void* stream) {
    if (!A || !B || !C || M <= 0 || N <= 0 || K <= 0 || (tensor_path != 0 && tensor_path != 1)) return GS_ERR_INVALID_ARG;
    if (lda < K || ldb < K || ldc < N || (lda % 8) || (ldb % 8) || (K % 16) || (N % 16) || (ldc % 4) ||
        ((uintptr_t)C & 15))
        return GS_ERR_INVALID_ARG;
    const int rc = gemm_tn(tensor_path, (const __nv_bfloat16*)A, lda, (const __nv_bfloat16*)B, ldb, C, ldc, M, N, K,
                           K, 0, (cudaStream_t)stream);
    if (rc != GS_OK) return rc;
    GS_CUDA_CHECK_LAUNCH();
    return GS_OK;
}
