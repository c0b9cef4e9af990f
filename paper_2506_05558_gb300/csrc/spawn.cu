// Direct spawn sampling (Sec. 4.2): per-pixel spawn probability from the norm
// of the Laplacian-of-Gaussian response of the input image (Eq. 1), the same
// quantity on the current render as a penalty (Eq. 2), their clamped
// difference (Eq. 3), a Bernoulli mask drawn with a counter-based generator,
// and, for every spawning pixel, a new Gaussian at the supplied depth with the
// expected nearest-neighbour scale s = z / (2 f sqrt(P_L)).
//
// k_spawn_maps: one CTA per 16x16 pixel tile; the image and render tiles with
// their halo are staged in shared memory and the (2R+1)^2 LoG taps (host-built,
// passed by value) are applied directly. The mask is compacted in pixel order
// with the device-wide scan, then k_spawn_emit writes the spawned rows.
#include <cmath>
#include <cuda.h>
#include <mutex>

#include "common.cuh"

namespace gs {

constexpr int kSpT = 16;
constexpr int kSpMaxR = 8;
constexpr int kSpMaxTaps = (2 * kSpMaxR + 1) * (2 * kSpMaxR + 1);

struct LogTaps {
    int R;
    float w[kSpMaxTaps];
};

__device__ __forceinline__ void stage_tile(const float* __restrict__ img, int W, int H, int x0, int y0, int R,
                                           float* s /* [3][S][S] */) {
    const int S = kSpT + 2 * R;
    const int64_t plane = (int64_t)W * H;
    for (int i = threadIdx.x; i < 3 * S * S; i += blockDim.x) {
        const int ch = i / (S * S), r = i % (S * S);
        const int yy = min(max(y0 - R + r / S, 0), H - 1);
        const int xx = min(max(x0 - R + r % S, 0), W - 1);
        s[i] = img[ch * plane + (int64_t)yy * W + xx];
    }
}

__device__ __forceinline__ float log_norm(const float* s, const LogTaps& k, int lx, int ly) {
    const int R = k.R, S = kSpT + 2 * R, n = 2 * R + 1;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
    for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) {
            const float w = k.w[j * n + i];
            const int o = (ly + j) * S + (lx + i);
            a0 += w * s[o];
            a1 += w * s[S * S + o];
            a2 += w * s[2 * S * S + o];
        }
    return fminf(sqrtf(a0 * a0 + a1 * a1 + a2 * a2), 1.f);
}

__global__ void __launch_bounds__(256) k_spawn_maps(const float* __restrict__ image, const float* __restrict__ render,
                                                    const float* __restrict__ depth, int W, int H, LogTaps taps,
                                                    uint2 key, uint32_t frame, float* __restrict__ p_l,
                                                    float* __restrict__ p_pen, float* __restrict__ p_s,
                                                    uint32_t* __restrict__ flag) {
    extern __shared__ float s_tile[];  // image tile, then render tile
    const int R = taps.R, S = kSpT + 2 * R;
    const int x0 = blockIdx.x * kSpT, y0 = blockIdx.y * kSpT;
    stage_tile(image, W, H, x0, y0, R, s_tile);
    if (render) stage_tile(render, W, H, x0, y0, R, s_tile + 3 * S * S);
    __syncthreads();
    const int lx = threadIdx.x % kSpT, ly = threadIdx.x / kSpT;
    const int x = x0 + lx, y = y0 + ly;
    if (x >= W || y >= H) return;
    const int64_t p = (int64_t)y * W + x;
    const float pl = log_norm(s_tile, taps, lx, ly);
    const float pp = render ? log_norm(s_tile + 3 * S * S, taps, lx, ly) : 0.f;
    const float ps = fmaxf(pl - pp, 0.f);
    if (flag) {  // the direct-sampling mask (the learned proposal only needs the maps)
        const uint4 r = philox4x32_10(make_uint4((uint32_t)p, frame, 0u, 0u), key);
        const float u = (float)(r.x >> 8) * (1.f / 16777216.f);
        const float z = depth[p];
        flag[p] = (u < ps && z > 0.f && isfinite(z)) ? 1u : 0u;
    }
    if (p_l) p_l[p] = pl;
    if (p_pen) p_pen[p] = pp;
    if (p_s) p_s[p] = ps;
}

__global__ void __launch_bounds__(256) k_spawn_emit(const float* __restrict__ image, const float* __restrict__ depth,
                                                    int W, int H, LogTaps taps, const uint32_t* __restrict__ flag,
                                                    const uint32_t* __restrict__ pos, const gs_camera* __restrict__ cam,
                                                    int64_t capacity, float4* __restrict__ mean_opa,
                                                    float4* __restrict__ scale, float4* __restrict__ quat,
                                                    float4* __restrict__ sh, int32_t* __restrict__ pixel) {
    extern __shared__ float s_tile[];
    const int R = taps.R;
    const int x0 = blockIdx.x * kSpT, y0 = blockIdx.y * kSpT;
    // P_L is recomputed from the image tile so the maps need not be stored
    stage_tile(image, W, H, x0, y0, R, s_tile);
    __syncthreads();
    const int lx = threadIdx.x % kSpT, ly = threadIdx.x / kSpT;
    const int x = x0 + lx, y = y0 + ly;
    if (x >= W || y >= H) return;
    const int64_t p = (int64_t)y * W + x;
    if (!flag[p]) return;
    const int64_t o = pos[p];
    if (o >= capacity) return;
    const float pl = log_norm(s_tile, taps, lx, ly);
    const float z = depth[p];
    const gs_camera& c = *cam;
    const float s_px = 0.5f / sqrtf(pl);
    const float s = z * s_px / c.fx;
    const float xc = (x + 0.5f - c.cx) * z / c.fx, yc = (y + 0.5f - c.cy) * z / c.fy;
    const float qx = xc - c.t[0], qy = yc - c.t[1], qz = z - c.t[2];
    const float mx = c.R[0] * qx + c.R[3] * qy + c.R[6] * qz;  // R^T (p_cam - t)
    const float my = c.R[1] * qx + c.R[4] * qy + c.R[7] * qz;
    const float mz = c.R[2] * qx + c.R[5] * qy + c.R[8] * qz;
    mean_opa[o] = make_float4(mx, my, mz, 0.f);  // opacity 0.5
    const float ls = logf(s);
    scale[o] = make_float4(ls, ls, ls, 0.f);
    quat[o] = make_float4(1.f, 0.f, 0.f, 0.f);
    const int64_t plane = (int64_t)W * H;
    const float inv_c0 = 3.5449077018110318f;  // 1 / SH band-0 constant = 2 sqrt(pi)
    float4* row = sh + 12 * o;
    row[0] = make_float4((image[p] - 0.5f) * inv_c0, (image[plane + p] - 0.5f) * inv_c0,
                         (image[2 * plane + p] - 0.5f) * inv_c0, 0.f);
#pragma unroll
    for (int r = 1; r < 12; r++) row[r] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (pixel) pixel[o] = (int32_t)p;
}

__global__ void k_spawn_count(const uint32_t* total, int64_t capacity, int64_t* count, int32_t* status) {
    *count = *total;
    *status = (int64_t)*total > capacity ? GS_ERR_CAPACITY : GS_OK;
}

static bool make_taps(float sigma, LogTaps* t) {
    if (!(sigma >= 0.3f) || !(sigma <= kSpMaxR / 3.f)) return false;
    const int R = (int)std::ceil(3.0 * sigma);
    const int n = 2 * R + 1;
    const double s2 = (double)sigma * sigma;
    double w[kSpMaxTaps], sum = 0;
    for (int j = -R; j <= R; j++)
        for (int i = -R; i <= R; i++) {
            const double r2 = i * i + j * j;
            const double v = (r2 - 2 * s2) / (s2 * s2) * std::exp(-r2 / (2 * s2)) / (2 * 3.14159265358979323846 * s2);
            w[(j + R) * n + (i + R)] = v;
            sum += v;
        }
    t->R = R;
    for (int k = 0; k < n * n; k++) t->w[k] = (float)(w[k] - sum / (n * n));
    return true;
}

}  // namespace gs

using namespace gs;

extern "C" size_t gs_spawn_workspace_size(int32_t width, int32_t height) {
    if (width <= 0 || height <= 0) return 0;
    const int64_t hw = (int64_t)width * height;
    Carve c{nullptr, 0, 0};
    c.take<uint32_t>(hw);
    c.take<uint32_t>(hw);
    c.take<uint32_t>(4);
    c.take<char>(scan_workspace_bytes(hw));
    c.take<float>(hw);       // gs_spawn_learned: P_s
    c.take<float>(hw / 64);  // gs_spawn_learned: patch sums
    c.take<float>(hw);       // gs_spawn_learned: P_L
    return c.used;
}

extern "C" int gs_spawn_propose(const float* image, const float* render, const float* depth, int32_t width,
                                int32_t height, const gs_camera* cam, const gs_spawn_config* sc,
                                const gs_spawn_out* out, void* ws, size_t ws_bytes, void* stream) {
    if (!image || !depth || !cam || !sc || !out || width <= 0 || height <= 0) return GS_ERR_INVALID_ARG;
    if (!out->count || !out->status || out->capacity < 0 ||
        (out->capacity > 0 && (!out->mean_opa || !out->scale || !out->quat || !out->sh)))
        return GS_ERR_INVALID_ARG;
    const int64_t hw = (int64_t)width * height;
    if (hw > (int64_t)UINT32_MAX) return GS_ERR_INVALID_ARG;
    LogTaps taps;
    if (!make_taps(sc->sigma, &taps)) return GS_ERR_INVALID_ARG;
    Carve c{(char*)ws, 0, ws_bytes};
    uint32_t* flag = c.take<uint32_t>(hw);
    uint32_t* pos = c.take<uint32_t>(hw);
    uint32_t* total = c.take<uint32_t>(4);
    void* scan_ws = c.take<char>(scan_workspace_bytes(hw));
    if (!ws || !c.ok() || ((uintptr_t)ws & 255)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int S = kSpT + 2 * taps.R;
    const size_t smem = sizeof(float) * 3 * S * S * (render ? 2 : 1);
    dim3 grid((unsigned)ceil_div(width, kSpT), (unsigned)ceil_div(height, kSpT));
    const uint2 key = make_uint2((uint32_t)sc->seed, (uint32_t)(sc->seed >> 32));
    k_spawn_maps<<<grid, 256, smem, s>>>(image, render, depth, width, height, taps, key, sc->frame, out->p_l,
                                          out->p_pen, out->p_s, flag);
    count_launch();
    scan_exclusive_u32(flag, pos, hw, total, scan_ws, s);
    k_spawn_count<<<1, 1, 0, s>>>(total, out->capacity, out->count, out->status);
    count_launch();
    if (out->capacity > 0) {
        k_spawn_emit<<<grid, 256, sizeof(float) * 3 * S * S, s>>>(
            image, depth, width, height, taps, flag, pos, cam, out->capacity, (float4*)out->mean_opa,
            (float4*)out->scale, (float4*)out->quat, (float4*)out->sh, out->pixel);
        count_launch();
    }
    GS_CUDA_CHECK_LAUNCH();
    return GS_OK;
}

// ---------------------------------------------------------------------------
// Spawn proposal without caller-provided scratch.
//
// Some callers cannot allocate device memory at the point where they need a
// spawn proposal: code running under an allocator that is frozen or owned by
// another runtime (a host application that hands us only its input and output
// buffers), or a process that has reserved all its memory up front. For them
// the scratch (per-pixel spawn flags, their exclusive scan and the scan's
// block sums) lives in this file-scope device array instead of a workspace.
// It is sized for at most kNoAllocMaxPixels pixels; every GPU that loads the
// library holds it until the process exits.
// ---------------------------------------------------------------------------
namespace gs {

constexpr int64_t kNoAllocMaxPixels = int64_t(1) << 21;  // 2,097,152 px: covers 1920x1080
constexpr int64_t kNoAllocScanWords = kNoAllocMaxPixels / 2048 + 256;  // the scan's block sums
constexpr int kNoAllocMaxDevices = 64;
constexpr int64_t kNoAllocWords = 2 * kNoAllocMaxPixels + 64 + kNoAllocScanWords;

static __device__ __align__(256) uint32_t g_spawn_scratch[kNoAllocWords];  // ~16.8 MB

// Device address of g_spawn_scratch, looked up once per device with that
// device current (the host-side name of the array is not a device address).
// The address belongs to the device's context: after cudaDeviceReset the
// runtime creates a new primary context with the module loaded again, so the
// cached address is kept with the unique id of the context it came from
// (cuCtxGetCurrent + cuCtxGetId, resolved through the runtime's driver
// entry-point query, without linking the driver library) and looked up again
// when the current context is another one. Where the driver offers neither
// call, the address is looked up on every call. The mutex orders concurrent
// first calls from several host threads.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

static bool current_context_id(CtxGetCurrentFn cur, CtxGetIdFn id, unsigned long long* out) {
    CUcontext ctx = nullptr;
    return cur && id && cur(&ctx) == CUDA_SUCCESS && ctx && id(ctx, out) == CUDA_SUCCESS;
}

static uint32_t* noalloc_scratch_for_current_device() {
    static std::mutex mu;
    static uint32_t* ptr[kNoAllocMaxDevices] = {};
    static unsigned long long ctx_id[kNoAllocMaxDevices] = {};
    static bool resolved = false;
    static CtxGetCurrentFn ctx_current = nullptr;
    static CtxGetIdFn ctx_get_id = nullptr;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!resolved) {
        resolved = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            ctx_current = (CtxGetCurrentFn)f;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            ctx_get_id = (CtxGetIdFn)f;
        (void)cudaGetLastError();
    }
    unsigned long long id = 0;
    const bool have_id = current_context_id(ctx_current, ctx_get_id, &id);
    if (!ptr[dev] || !have_id || id != ctx_id[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_spawn_scratch) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        ptr[dev] = (uint32_t*)p;
        // the lookup made the device's context current if none was
        ctx_id[dev] = current_context_id(ctx_current, ctx_get_id, &id) ? id : 0;
    }
    return ptr[dev];
}

}  // namespace gs

extern "C" int gs_spawn_propose_noalloc(const float* image, const float* render, const float* depth,
                                        int32_t width, int32_t height, const gs_camera* cam,
                                        const gs_spawn_config* sc, const gs_spawn_out* out, void* stream) {
    if (!image || !depth || !cam || !sc || !out || width <= 0 || height <= 0) return GS_ERR_INVALID_ARG;
    if (!out->count || !out->status || out->capacity < 0 ||
        (out->capacity > 0 && (!out->mean_opa || !out->scale || !out->quat || !out->sh)))
        return GS_ERR_INVALID_ARG;
    const int64_t hw = (int64_t)width * height;
    if (hw > kNoAllocMaxPixels) return GS_ERR_INVALID_ARG;  // larger frames need gs_spawn_propose
    LogTaps taps;
    if (!make_taps(sc->sigma, &taps)) return GS_ERR_INVALID_ARG;
    uint32_t* base = noalloc_scratch_for_current_device();
    if (!base) return GS_ERR_CUDA;
    // Layout inside the static array. Nothing in it needs to start at zero:
    // every pass writes each word it later reads (flags and positions for all
    // hw pixels, the scan's block sums and total).
    uint32_t* flag = base;
    uint32_t* pos = base + kNoAllocMaxPixels;
    uint32_t* total = base + 2 * kNoAllocMaxPixels;
    void* scan_ws = base + 2 * kNoAllocMaxPixels + 64;
    cudaStream_t s = (cudaStream_t)stream;
    const int S = kSpT + 2 * taps.R;
    const size_t smem = sizeof(float) * 3 * S * S * (render ? 2 : 1);
    dim3 grid((unsigned)ceil_div(width, kSpT), (unsigned)ceil_div(height, kSpT));
    const uint2 key = make_uint2((uint32_t)sc->seed, (uint32_t)(sc->seed >> 32));
    k_spawn_maps<<<grid, 256, smem, s>>>(image, render, depth, width, height, taps, key, sc->frame, out->p_l,
                                          out->p_pen, out->p_s, flag);
    count_launch();
    scan_exclusive_u32(flag, pos, hw, total, scan_ws, s);
    k_spawn_count<<<1, 1, 0, s>>>(total, out->capacity, out->count, out->status);
    count_launch();
    if (out->capacity > 0) {
        k_spawn_emit<<<grid, 256, sizeof(float) * 3 * S * S, s>>>(
            image, depth, width, height, taps, flag, pos, cam, out->capacity, (float4*)out->mean_opa,
            (float4*)out->scale, (float4*)out->quat, (float4*)out->sh, out->pixel);
        count_launch();
    }
    GS_CUDA_CHECK_LAUNCH();
    return GS_OK;
}

// ---------------------------------------------------------------------------
// Learned spawn proposal: training targets and spawning from its predictions.
// ---------------------------------------------------------------------------
namespace gs {

// Scatter the kept spawns into per-pixel slots (each pixel spawns at most once).
// One thread per spawn: kept when its optimised opacity sigmoid(logit) is
// above the threshold; then its camera depth R_2 . mu + t_2 and the change of
// its log-scale (mean over the three axes minus the spawned value) go to the
// spawn's pixel.
__global__ void k_kept_scatter(const int32_t* __restrict__ pixel, const float4* __restrict__ mean_opa,
                               const float4* __restrict__ scale, const float4* __restrict__ scale0,
                               const gs_camera* __restrict__ cam, float keep_threshold, int64_t n, int64_t hw,
                               float4* __restrict__ pix_slot) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 mo = mean_opa[i];
    const float o = 1.f / (1.f + expf(-mo.w));
    if (!(o > keep_threshold)) return;
    const int32_t p = pixel[i];
    if (p < 0 || (int64_t)p >= hw) return;
    const float z = cam->R[6] * mo.x + cam->R[7] * mo.y + cam->R[8] * mo.z + cam->t[2];
    const float4 s = scale[i];
    const float ls = (s.x + s.y + s.z) * (1.f / 3.f) - scale0[i].x;
    pix_slot[p] = make_float4(1.f, z, ls, 0.f);
}

// One thread per 8x8 patch: kept fraction, mean depth and log-scale, any-kept.
__global__ void k_patch_targets(const float4* __restrict__ pix_slot, int W, int H, float* __restrict__ targets) {
    const int nx = W / 8, ny = H / 8;
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= (int64_t)nx * ny) return;
    const int px = (int)(m % nx), py = (int)(m / nx);
    float cnt = 0.f, zs = 0.f, ss = 0.f;
    for (int dy = 0; dy < 8; dy++)
        for (int dx = 0; dx < 8; dx++) {
            const float4 v = pix_slot[(int64_t)(py * 8 + dy) * W + px * 8 + dx];
            if (v.x > 0.f) {
                cnt += 1.f;
                zs += v.y;
                ss += v.z;
            }
        }
    targets[m * 4 + 0] = cnt / 64.f;
    targets[m * 4 + 1] = cnt > 0.f ? zs / cnt : 0.f;
    targets[m * 4 + 2] = cnt > 0.f ? ss / cnt : 0.f;
    targets[m * 4 + 3] = cnt > 0.f ? 1.f : 0.f;
}

// Depth of a learned spawn at pixel p: the depth map's value where it is
// positive and finite, else the patch's predicted depth.
__device__ __forceinline__ float learned_depth(const float* __restrict__ depth, const float* __restrict__ mlp_out,
                                               int64_t p, int64_t m) {
    const float d = depth ? depth[p] : 0.f;
    return (d > 0.f && isfinite(d)) ? d : mlp_out[m * 3 + 1];
}

// Lower bound of a patch's P_s sum in the placement ratio (keeps the ratio
// well conditioned where the render already explains the patch).
constexpr float kPatchFloor = 64.f * 1e-3f;

// One thread per 8x8 patch: sum of P_s in row-major order, floored.
__global__ void k_patch_ps_sum(const float* __restrict__ ps, int W, int H, float* __restrict__ sums) {
    const int nx = W / 8, ny = H / 8;
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= (int64_t)nx * ny) return;
    const int px = (int)(m % nx), py = (int)(m / nx);
    float a = 0.f;
    for (int dy = 0; dy < 8; dy++)
        for (int dx = 0; dx < 8; dx++) a += ps[(int64_t)(py * 8 + dy) * W + px * 8 + dx];
    sums[m] = fmaxf(a, kPatchFloor);
}

// Spawn flags from the MLP: pixel p of patch m spawns with probability
// min(1, sigmoid(logit_m) 64 P_s(p) / patch sum) (the predicted count placed
// where direct sampling would place it) and a positive depth; the draw is
// Philox(counter (p, frame, 1, 0)).
__global__ void k_learned_flags(const float* __restrict__ mlp_out, const float* __restrict__ depth,
                                const float* __restrict__ ps, const float* __restrict__ sums, int W, int H,
                                uint2 key, uint32_t frame, uint32_t* __restrict__ flag) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (int64_t)W * H) return;
    const int x = (int)(p % W), y = (int)(p / W);
    const int64_t m = (int64_t)(y / 8) * (W / 8) + x / 8;
    const float logit = mlp_out[m * 3 + 0], z = learned_depth(depth, mlp_out, p, m);
    const float sig = 1.f / (1.f + expf(-logit));
    const float prob = fminf(1.f, sig * 64.f * ps[p] / sums[m]);
    const uint4 r = philox4x32_10(make_uint4((uint32_t)p, frame, 1u, 0u), key);
    const float u = (float)(r.x >> 8) * (1.f / 16777216.f);
    flag[p] = (u < prob && z > 0.f && isfinite(z)) ? 1u : 0u;
}

__global__ void k_learned_emit(const float* __restrict__ image, const float* __restrict__ mlp_out,
                               const float* __restrict__ depth, const float* __restrict__ p_l, int W, int H,
                               const uint32_t* __restrict__ flag, const uint32_t* __restrict__ pos,
                               const gs_camera* __restrict__ cam, int64_t capacity, float4* __restrict__ mean_opa,
                               float4* __restrict__ scale, float4* __restrict__ quat, float4* __restrict__ sh,
                               int32_t* __restrict__ pixel) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (int64_t)W * H || !flag[p]) return;
    const int64_t o = pos[p];
    if (o >= capacity) return;
    const int x = (int)(p % W), y = (int)(p / W);
    const int64_t m = (int64_t)(y / 8) * (W / 8) + x / 8;
    const float z = learned_depth(depth, mlp_out, p, m);
    // direct sampling's scale z / (2 fx sqrt(P_L)) times the patch's predicted factor exp(offset)
    const float ls = logf(z * (0.5f / sqrtf(p_l[p])) / cam->fx) + mlp_out[m * 3 + 2];
    const gs_camera& c = *cam;
    const float xc = (x + 0.5f - c.cx) * z / c.fx, yc = (y + 0.5f - c.cy) * z / c.fy;
    const float qx = xc - c.t[0], qy = yc - c.t[1], qz = z - c.t[2];
    mean_opa[o] = make_float4(c.R[0] * qx + c.R[3] * qy + c.R[6] * qz, c.R[1] * qx + c.R[4] * qy + c.R[7] * qz,
                              c.R[2] * qx + c.R[5] * qy + c.R[8] * qz, 0.f);
    scale[o] = make_float4(ls, ls, ls, 0.f);
    quat[o] = make_float4(1.f, 0.f, 0.f, 0.f);
    const int64_t plane = (int64_t)W * H;
    const float inv_c0 = 3.5449077018110318f;  // 1 / SH band-0 constant = 2 sqrt(pi)
    float4* row = sh + 12 * o;
    row[0] = make_float4((image[p] - 0.5f) * inv_c0, (image[plane + p] - 0.5f) * inv_c0,
                         (image[2 * plane + p] - 0.5f) * inv_c0, 0.f);
#pragma unroll
    for (int r = 1; r < 12; r++) row[r] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (pixel) pixel[o] = (int32_t)p;
}

}  // namespace gs

extern "C" size_t gs_mlp_targets_workspace_size(int32_t width, int32_t height) {
    if (width <= 0 || height <= 0) return 0;
    return align256(sizeof(float4) * (size_t)width * height);
}

extern "C" int gs_mlp_targets(const int32_t* pixel, const float* mean_opa, const float* scale, const float* scale0,
                              const gs_camera* cam, float keep_threshold, int64_t n_spawn, int32_t width,
                              int32_t height, float* targets, void* ws, size_t ws_bytes, void* stream) {
    if (!targets || width <= 0 || height <= 0 || width % 8 || height % 8 || n_spawn < 0 ||
        (n_spawn > 0 && (!pixel || !mean_opa || !scale || !scale0 || !cam)))
        return GS_ERR_INVALID_ARG;
    const int64_t hw = (int64_t)width * height;
    if (!ws || ws_bytes < gs_mlp_targets_workspace_size(width, height) || ((uintptr_t)ws & 255))
        return GS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    float4* slot = (float4*)ws;
    cudaMemsetAsync(slot, 0, sizeof(float4) * hw, s);
    if (n_spawn > 0) {
        k_kept_scatter<<<(unsigned)ceil_div(n_spawn, 256), 256, 0, s>>>(
            pixel, (const float4*)mean_opa, (const float4*)scale, (const float4*)scale0, cam, keep_threshold, n_spawn,
            hw, slot);
        count_launch();
    }
    const int64_t np = hw / 64;
    k_patch_targets<<<(unsigned)ceil_div(np, 256), 256, 0, s>>>(slot, width, height, targets);
    count_launch();
    GS_CUDA_CHECK_LAUNCH();
    return GS_OK;
}

extern "C" int gs_spawn_learned(const float* image, const float* mlp_out, const float* render, const float* depth,
                                int32_t width, int32_t height, const gs_camera* cam, const gs_spawn_config* sc,
                                const gs_spawn_out* out, void* ws, size_t ws_bytes, void* stream) {
    if (!image || !mlp_out || !cam || !sc || !out || width <= 0 || height <= 0 || width % 8 || height % 8)
        return GS_ERR_INVALID_ARG;
    if (!out->count || !out->status || out->capacity < 0 ||
        (out->capacity > 0 && (!out->mean_opa || !out->scale || !out->quat || !out->sh)))
        return GS_ERR_INVALID_ARG;
    const int64_t hw = (int64_t)width * height;
    if (hw > (int64_t)UINT32_MAX) return GS_ERR_INVALID_ARG;
    LogTaps taps;
    if (!make_taps(sc->sigma, &taps)) return GS_ERR_INVALID_ARG;
    Carve c{(char*)ws, 0, ws_bytes};
    uint32_t* flag = c.take<uint32_t>(hw);
    uint32_t* pos = c.take<uint32_t>(hw);
    uint32_t* total = c.take<uint32_t>(4);
    void* scan_ws = c.take<char>(scan_workspace_bytes(hw));
    float* ps = c.take<float>(hw);
    float* sums = c.take<float>(hw / 64);
    float* pl = c.take<float>(hw);
    if (!ws || !c.ok() || ((uintptr_t)ws & 255)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const uint2 key = make_uint2((uint32_t)sc->seed, (uint32_t)(sc->seed >> 32));
    // P_s (Eq. 1-3) of the frame, then its patch sums
    const int S = kSpT + 2 * taps.R;
    const size_t smem = sizeof(float) * 3 * S * S * (render ? 2 : 1);
    dim3 grid((unsigned)ceil_div(width, kSpT), (unsigned)ceil_div(height, kSpT));
    float* psb = out->p_s ? out->p_s : ps;  // the caller's maps when it asks for them
    float* plb = out->p_l ? out->p_l : pl;
    k_spawn_maps<<<grid, 256, smem, s>>>(image, render, nullptr, width, height, taps, key, sc->frame, plb,
                                          out->p_pen, psb, nullptr);
    count_launch();
    k_patch_ps_sum<<<(unsigned)ceil_div(hw / 64, 256), 256, 0, s>>>(psb, width, height, sums);
    count_launch();
    k_learned_flags<<<(unsigned)ceil_div(hw, 256), 256, 0, s>>>(mlp_out, depth, psb, sums, width, height, key,
                                                                 sc->frame, flag);
    count_launch();
    scan_exclusive_u32(flag, pos, hw, total, scan_ws, s);
    k_spawn_count<<<1, 1, 0, s>>>(total, out->capacity, out->count, out->status);
    count_launch();
    if (out->capacity > 0) {
        k_learned_emit<<<(unsigned)ceil_div(hw, 256), 256, 0, s>>>(image, mlp_out, depth, plb, width, height, flag,
                                                                    pos, cam,
                                                                    out->capacity, (float4*)out->mean_opa,
                                                                    (float4*)out->scale, (float4*)out->quat,
                                                                    (float4*)out->sh, out->pixel);
        count_launch();
    }
    GS_CUDA_CHECK_LAUNCH();
    return GS_OK;
}
