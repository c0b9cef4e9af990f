/*
 * gs.h - C ABI of the GB300 (sm_103a) differentiable Gaussian splatting
 * rasterizer: the hot path of the joint pose and primitive optimisation of
 * "On-the-fly Reconstruction for Large-Scale Novel View Synthesis from Unposed
 * Images" (Sec. 4.3), its direct spawn sampling (Sec. 4.2, Eq. 1-3) and the
 * optimiser step that closes each iteration.
 *
 * The paper gives the problem (render the current Gaussians from the current
 * poses, compare with the images, update poses and primitives; Sec. 4.3) and
 * builds its rasterizer on the 3DGS image-formation model (Sec. 5). The entry
 * points follow the stages of that model:
 *   gs_project     EWA projection, screen bounds, SH colour      (per view x Gaussian)
 *   gs_sort        per-tile duplication and depth ordering       (integer work)
 *   gs_render_fwd  front-to-back alpha compositing               (per pixel)
 *   gs_render_bwd  adjoint of the three stages above, including the camera
 *                  pose gradient as an SE(3) tangent (Sec. 4.3: poses get
 *                  gradients from Gaussian positions and rotations, not SH)
 *   gs_adam_step / gs_pose_step   sparse Adam over visible Gaussians and the
 *                  pose update (Sec. 4.3)
 *   gs_l1_loss     L1 photometric loss and its gradient
 *   gs_spawn_propose  direct spawn sampling (Sec. 4.2)
 *
 * Conventions shared by every call
 *  - All tensor arguments are DEVICE pointers owned by the caller unless a
 *    comment says "host". The library never allocates, frees or synchronises;
 *    every call only enqueues kernels on `stream` (a cudaStream_t passed as
 *    void*, NULL = legacy default stream), so a sequence of calls can be
 *    captured into a CUDA graph.
 *  - float32 throughout. Layouts are structure-of-arrays with 16-byte rows.
 *  - A view's camera looks down +z; pixel (i, j) is sampled at (i+0.5, j+0.5);
 *    u = fx x/z + cx, v = fy y/z + cy.
 *  - Return value: GS_OK, or GS_ERR_INVALID_ARG when a host-side check of
 *    sizes/pointers fails (nothing is enqueued), or GS_ERR_CUDA when a launch
 *    fails. Data-dependent failures (a pair buffer that is too small) are
 *    reported through a device status word the caller reads after it syncs.
 *  - Non-finite Gaussians are culled, never trapped.
 */
#ifndef GS_H
#define GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GS_OK 0
#define GS_ERR_INVALID_ARG (-1)
#define GS_ERR_CAPACITY (-2)
#define GS_ERR_CUDA (-3)
#define GS_ERR_TIMEOUT (-4)

#define GS_MAX_VIEWS 64

/* Pinhole camera, world -> camera: p = R mu + t (R row-major). 72 bytes. */
typedef struct gs_camera {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    int32_t width, height;
} gs_camera;

/* Rasterizer settings (the paper states none of these; the values in the
 * comments are the defaults of gs_config_default). */
typedef struct gs_config {
    int32_t tile;                 /* tile edge in pixels, 8, 16 or 32 (must equal the frame's): 16 */
    int32_t sh_degree;            /* 0..3 */
    float near_z;                 /* cull if z <= near_z: 0.2 */
    float dilation;               /* screen-space low-pass added to Sigma2D: 0.3 px^2 */
    float alpha_min;              /* skip a Gaussian below this alpha: 1/255 */
    float alpha_max;              /* alpha clamp: 0.99 */
    float t_min;                  /* stop before T would fall below this: 1e-4 */
    float bg[3];                  /* background colour: 0 */
    int32_t pose_grad_through_sh; /* 1: pose gradient also through the SH view direction: 0 */
    int32_t schedule;             /* render scheduling: 0 = one CTA per tile, 1 = persistent CTAs
                                     pulling tiles, largest first, from a work queue, 2 = one CTA
                                     per tile, CTA i taking the i-th tile of the largest-first
                                     order (no queue); 1 and 2 need gs_pairs.order */
    int32_t accumulate;           /* gs_render_bwd / gs_project_bwd: 0 overwrite the gradient
                                     buffers, 1 add to them (per-view launches of one step): 0 */
    int32_t fwd_batch;            /* Gaussians staged per round in gs_render_fwd: 0 = default;
                                     tile 8: 64/128/256, tile 16: 64/128/256, tile 32: 128/256 */
    int32_t bwd_batch;            /* the same for the adjoint: 0 = default; tile 8: 64/128/256,
                                     tile 16: 32/64/128, tile 32: 32 */
    int32_t mip_filter;           /* 1: the dilation is a 2-D low-pass filter that keeps the splat's
                                     integral (multi-scale training, Sec. 4.3): opacity times
                                     sqrt(rho), rho = det(Sigma2D) / det(Sigma2D + dilation I)
                                     floored at 1e-6; use dilation 0.1 with it: 0 */
    int32_t alpha_rect;           /* 1: each tile rect is also bounded by the tiles that the box of
                                     the ellipse where o exp(-q/2) reaches alpha_min overlaps (x in
                                     u +- sqrt(2 ln(o / alpha_min) Sigma2D_xx), tiles
                                     [floor((u - hx)/T), floor((u + hx)/T) + 1), y likewise), and an
                                     opacity below alpha_min lists the item nowhere: only list
                                     entries that no pixel composites are dropped; 0: the 3-sigma
                                     rect alone: 1 */
} gs_config;

void gs_config_default(gs_config* cfg);

/* Geometry of a batch of views rendered together (host struct, passed by
 * pointer and copied by value into kernel parameters). Item index of
 * (view v, Gaussian g) is v * n + g. Tiles of all views share one global tile
 * index: tile_base[v] + ty * tiles_x[v] + tx. Pixels of view v start at
 * pix_base[v] in every per-pixel buffer; colour buffers hold 3 planes per view
 * ([3][height][width] starting at 3 * pix_base[v]). */
typedef struct gs_frame {
    int32_t n_views;
    int32_t tile;
    int32_t width[GS_MAX_VIEWS];
    int32_t height[GS_MAX_VIEWS];
    int32_t tiles_x[GS_MAX_VIEWS];
    int32_t tiles_y[GS_MAX_VIEWS];
    int32_t tile_base[GS_MAX_VIEWS + 1];
    int64_t pix_base[GS_MAX_VIEWS + 1];
} gs_frame;

/* Fills f from host arrays width[n_views], height[n_views]. tile: 8, 16 or 32.
 * Returns GS_ERR_INVALID_ARG for n_views outside 1..GS_MAX_VIEWS, a
 * non-positive size or more than 2^31 tiles or pixels in total. */
int gs_frame_init(gs_frame* f, int32_t n_views, const int32_t* width, const int32_t* height, int32_t tile);

/* Gaussian parameters, structure of arrays, n Gaussians (paper Sec. 3: position,
 * scale, rotation, opacity, SH):
 *   mean_opa [n][4]  x, y, z, opacity logit (opacity = sigmoid)
 *   scale    [n][4]  log-scales sx, sy, sz, unused
 *   quat     [n][4]  w, x, y, z (normalised inside)
 *   sh       [n][48] SH coefficient k (k = l^2 + l + m) of channel c at sh[48 g + 3 k + c]
 *   filter3d [n]     optional (NULL: off): variance v of the 3-D smoothing filter of
 *                    each Gaussian (Mip-Splatting's 3-D filter, the "proper filtering"
 *                    of Sec. 4.3; see gs_filter3d). With it, gs_project renders the
 *                    covariance Sigma + v I (scales sqrt(s^2 + v), same rotation) with
 *                    the opacity multiplied by sqrt(det Sigma / det(Sigma + v I)) =
 *                    prod_i s_i / sqrt(s_i^2 + v), and gs_project_bwd differentiates
 *                    through both (v is a constant of the step)
 * Each row must be 16-byte aligned. */
typedef struct gs_gaussians {
    float* mean_opa;
    float* scale;
    float* quat;
    float* sh;
    int64_t n;
    const float* filter3d;
} gs_gaussians;

/* Variance of the 3-D smoothing filter of every Gaussian (Mip-Splatting's 3-D
 * filter, the "proper filtering" of Sec. 4.3) from the training cameras cams
 * [n_views] (device): nu = the largest sampling rate fx / z over the views in
 * which the mean lies in front of near_z and projects inside the image
 * enlarged by 15% on each side, filter3d[g] = s2 / nu^2 (s2 = 0.2 in
 * Mip-Splatting); a Gaussian no view samples gets the largest variance of the
 * sampled ones (0 if none is sampled). Recompute when the cameras or the set
 * change. ws: 256 bytes of device scratch. Only mean_opa of g is read. */
int gs_filter3d(const gs_gaussians* g, const gs_camera* cams, int32_t n_views, float near_z, float s2,
                float* filter3d, void* ws, size_t ws_bytes, void* stream);

/* Per (view, Gaussian) projection outputs, n_views * n items:
 *   mean2d    [items][2]  u, v in pixels
 *   conic_opa [items][4]  inverse 2D covariance (a, b, c) of [[a,b],[b,c]], opacity
 *   rgb_depth [items][4]  colour (clamped at 0), camera-space depth z
 *   rect      [items][4]  uint16 tile bounds x0, y0, x1, y1 (half-open)
 *   n_tiles   [items]     (x1-x0)*(y1-y0); 0 marks a culled item */
typedef struct gs_projected {
    float* mean2d;
    float* conic_opa;
    float* rgb_depth;
    uint16_t* rect;
    int32_t* n_tiles;
} gs_projected;

/* EWA projection + SH colour for every (view, Gaussian) (3DGS model the paper
 * builds on, Sec. 5; cull, dilation, guard band, radius and rect readings as
 * documented in DESIGN). cams: device array of f->n_views cameras. */
int gs_project(const gs_gaussians* g, const gs_camera* cams, const gs_frame* f, const gs_config* cfg,
               const gs_projected* out, void* stream);

/* Sorted (tile, Gaussian) pairs.
 *   src     [capacity]  sorted pair -> item index (view * n + g)
 *   emit    [capacity]  sorted pair -> emission slot; the pairs of one item
 *                       occupy slots offset[item] .. offset[item]+n_tiles-1
 *   offset  [n_views*n] first emission slot of each item: the slots are
 *           assigned in item order (an exclusive sum of n_tiles over items),
 *           so the runs of consecutive items are adjacent
 *   range   [2 * total tiles]  [start, end) of each tile's pairs in src/emit
 *   count   device int64[1]: number of pairs (written by gs_sort)
 *   status  device int32[1]: GS_OK, or GS_ERR_CAPACITY if count > capacity (then
 *           only the first `capacity` pairs, by depth, exist: renders are
 *           incomplete and gs_project_bwd returns zero gradients), or
 *           GS_ERR_TIMEOUT if a scan or radix pass gave up waiting for an
 *           earlier CTA's count (bounded polls; the lists are then invalid)
 *   order   [total tiles] optional (NULL to skip): tile indices by decreasing
 *           pair count (stable), the work order of schedules 1 and 2 */
typedef struct gs_pairs {
    uint32_t* src;
    uint32_t* emit;
    uint32_t* offset;
    uint32_t* range;
    int64_t capacity;
    int64_t* count;
    int32_t* status;
    uint32_t* order;
} gs_pairs;

/* Scratch bytes gs_sort needs for n Gaussians, the frame's views and a pair
 * capacity. */
size_t gs_sort_workspace_size(int64_t n, const gs_frame* f, int64_t capacity);

/* Per-tile duplication and ordering. Visible items are first ordered by fp32
 * depth (stable LSD radix sort, ties by item index), their pairs are emitted
 * in that order, then a stable radix sort on the global tile index yields, per
 * tile, the Gaussians in (depth bits, Gaussian id) order. Scans and radix
 * passes are single-pass (decoupled look-back between CTAs). ws: device
 * scratch of at least gs_sort_workspace_size bytes, 256-byte aligned; calls
 * that share one ws must not overlap on the GPU. */
int gs_sort(const gs_projected* p, int64_t n, const gs_frame* f, const gs_pairs* out, void* ws, size_t ws_bytes,
            void* stream);

/* Forward image and the per-pixel state the adjoint needs.
 *   color     [sum_v 3 * H_v * W_v]  planar RGB per view
 *   t_final   [sum_v H_v * W_v]      final transmittance (alpha = 1 - t_final)
 *   n_contrib [sum_v H_v * W_v]      1 + list position of the last composited
 *                                     Gaussian (0 if none)
 *   depth     [sum_v H_v * W_v]      optional (NULL: not written): depth
 *                                     integral sum_i alpha_i T_i z_i, i.e. the
 *                                     expected camera depth times 1 - t_final
 *                                     (Sec. 4.4 anchors; no gradient) */
typedef struct gs_image {
    float* color;
    float* t_final;
    int32_t* n_contrib;
    float* depth;
} gs_image;

/* Scratch bytes gs_render_fwd / gs_render_bwd need (work queue of the
 * persistent schedule); 0 is valid when cfg->schedule == 0. */
size_t gs_render_workspace_size(const gs_frame* f);

/* Front-to-back alpha compositing (3DGS model): per pixel, over the tile's
 * depth-ordered list, alpha = min(alpha_max, o exp(-d^T conic d / 2)), skipped
 * below alpha_min, stopping before T would fall below t_min; colour =
 * sum alpha T rgb + T_final bg. */
int gs_render_fwd(const gs_projected* p, const gs_pairs* pairs, const gs_frame* f, const gs_config* cfg,
                  const gs_image* out, void* ws, size_t ws_bytes, void* stream);

/* Measurement (not a step of the method): gs_render_fwd with the same
 * arguments and outputs, run by a counting instantiation of its kernel that
 * also writes counts [3] (device, uint64, overwritten): [0] the warp hits its
 * box test passes (each runs the compositing step on 32 lanes), [1] the lane
 * evaluations of pixels not yet terminated at those hits, [2] the evaluations
 * that composite (alpha >= alpha_min, before termination) - the (pixel,
 * Gaussian) work the compositing definition requires (Sec. 4.3; the 3DGS
 * image-formation model). Slower than gs_render_fwd: never timed. */
int gs_render_fwd_count(const gs_projected* p, const gs_pairs* pairs, const gs_frame* f, const gs_config* cfg,
                        const gs_image* out, void* ws, size_t ws_bytes, unsigned long long* counts, void* stream);

/* Measurement (not a step of the method): throughput probes of the FP32 FMA
 * and MUFU pipes, timed by the caller. `blocks` CTAs of 256 threads; each
 * thread performs 128 * iters fused multiply-adds (gs_probe_fma; 2 flops each)
 * or 64 * iters MUFU operations, half 2^x and half 1/x (gs_probe_mufu), and
 * writes one float to out [blocks * 256] (device). */
int gs_probe_fma(float* out, int32_t blocks, int32_t iters, void* stream);
int gs_probe_mufu(float* out, int32_t blocks, int32_t iters, void* stream);

/* Gradients w.r.t. the Gaussian parameters, same layout as gs_gaussians.
 * visible [n] = 1 if the Gaussian has at least one pair in any view. */
typedef struct gs_grads {
    float* mean_opa;
    float* scale;
    float* quat;
    float* sh;
    uint8_t* visible;
} gs_grads;

/* Scratch bytes gs_render_bwd needs for the pair capacity and n Gaussians. */
size_t gs_backward_workspace_size(int64_t n, const gs_frame* f, int64_t capacity);

/* Adjoint of project + sort + render_fwd for all views at once.
 *   dL_dcolor  same layout as gs_image.color
 *   grads      OVERWRITTEN with dL/d(parameters) summed over views
 *   dL_dpose   [n_views][6] OVERWRITTEN: dL/dxi for the left perturbation
 *              T_cw <- exp(xi^) T_cw, xi = (rho, phi) (translation first)
 *   d_proj     optional [n_views*n][9], NULL to skip: dL/d(u, v, conic a, b,
 *              c, opacity, r, g, b) per item (the 2D adjoint, for testing)
 * Per tile the blending state is recomputed back to front from t_final and
 * n_contrib; each (tile, Gaussian) pair gets one partial written to its
 * emission slot and partials are summed per Gaussian in a fixed order: no
 * atomics, bit-reproducible. */
int gs_render_bwd(const gs_gaussians* g, const gs_camera* cams, const gs_projected* p, const gs_pairs* pairs,
                  const gs_frame* f, const gs_config* cfg, const gs_image* fwd, const float* dL_dcolor,
                  const gs_grads* grads, float* dL_dpose, float* d_proj, void* ws, size_t ws_bytes, void* stream);

/* The two halves of gs_render_bwd, for callers that schedule or time them
 * separately; they share the workspace (which must persist between them).
 * gs_composite_bwd: per-tile adjoint of the compositing, one partial per
 *   (tile, Gaussian) pair into the workspace.
 * gs_project_bwd: per-Gaussian sum of those partials over all views and the
 *   adjoint of the projection, pose gradient reduction.
 * Arguments as for gs_render_bwd. */
int gs_composite_bwd(const gs_projected* p, const gs_pairs* pairs, const gs_frame* f, const gs_config* cfg,
                     const gs_image* fwd, const float* dL_dcolor, int64_t n, void* ws, size_t ws_bytes,
                     void* stream);
int gs_project_bwd(const gs_gaussians* g, const gs_camera* cams, const gs_projected* p, const gs_pairs* pairs,
                   const gs_frame* f, const gs_config* cfg, const gs_grads* grads, float* dL_dpose, float* d_proj,
                   void* ws, size_t ws_bytes, void* stream);

/* Number of kernels this library has launched since it was loaded (host-side
 * counter; diagnostics for benchmarks). */
int64_t gs_launch_count(void);

/* Direct spawn sampling settings (Sec. 4.2). sigma: standard deviation in
 * pixels of the Gaussian n_sigma of the LoG operator (the paper leaves it
 * unspecified; 1.0 here), 0.3 <= sigma <= 8/3. The mask draws
 * u = Philox4x32-10(counter = (pixel index, frame, 0, 0), key = seed) and a
 * pixel spawns iff u < P_s and its depth is positive and finite. */
typedef struct gs_spawn_config {
    float sigma;
    uint32_t frame;
    uint64_t seed;
} gs_spawn_config;

/* Spawned Gaussians, compacted in pixel order, in the gs_gaussians row layout
 * (mean + opacity logit 0, log-scale x3, identity quaternion, SH DC from the
 * pixel colour with the higher bands 0), plus the source pixel index (optional,
 * may be NULL). count / status are device words as in gs_pairs. p_l, p_pen, p_s:
 * optional [H*W] maps of Eq. 1, 2, 3 (NULL to skip). */
typedef struct gs_spawn_out {
    float* mean_opa;
    float* scale;
    float* quat;
    float* sh;
    int32_t* pixel;
    int64_t capacity;
    int64_t* count;
    int32_t* status;
    float* p_l;
    float* p_pen;
    float* p_s;
} gs_spawn_out;

/* Workspace bytes gs_spawn_propose needs for a width x height frame (0 for
 * a non-positive size); the workspace is caller-owned, 256-byte aligned. */
size_t gs_spawn_workspace_size(int32_t width, int32_t height);

/* Spawn proposal for a new frame (Sec. 4.2, Eq. 1-3 and the scale from the
 * expected nearest-neighbour distance of a 2-D Poisson process of intensity
 * P_L: s' = 1/(2 sqrt(P_L)) px, s = z s' / fx).
 *   image   [3][height][width] in [0, 1], the new frame
 *   render  [3][height][width] the current Gaussians rendered from the frame's
 *           pose, or NULL when nothing has been reconstructed yet (P~ = 0)
 *   depth   [height][width] depth per pixel (camera z) used for the new means
 *   cam     device camera of the frame (world -> camera)
 * The LoG kernel is the Laplacian of n_sigma sampled at integer offsets up to
 * radius ceil(3 sigma), shifted to zero sum; borders replicate; the norm is
 * over the three colour responses. */
int gs_spawn_propose(const float* image, const float* render, const float* depth, int32_t width, int32_t height,
                     const gs_camera* cam, const gs_spawn_config* sc, const gs_spawn_out* out, void* ws,
                     size_t ws_bytes, void* stream);

/* Anchor trigger (Sec. 4.4): the size of a Gaussian seen from a camera is
 * S / D, S its largest scale, D the distance of its mean to the camera centre;
 * in pixels fx S / D. too_fine [n] (device) = 1 where that is below tau_px
 * (the paper's tau_min = 1 px, measured from the previous camera); count
 * (device int64) = the number of such Gaussians (exact). An anchor is due when
 * count > 0.4 n. */
int gs_anchor_check(const gs_gaussians* g, const gs_camera* cam, float tau_px, uint8_t* too_fine, int64_t* count,
                    void* stream);

/* Anchor offload / reload (Sec. 4.4: the active set and its optimisation state
 * are stored at the anchor in host memory and loaded back when required).
 * gs_anchor_offload copies params (and m, v when both are non-NULL) from the
 * device to caller-owned host arrays (pinned memory gives asynchronous copies);
 * gs_anchor_load copies them back. One cudaMemcpyAsync per array on `stream`;
 * the n of each pair of sets must match. */
int gs_anchor_offload(const gs_gaussians* params, const gs_gaussians* m, const gs_gaussians* v,
                      const gs_gaussians* host_params, const gs_gaussians* host_m, const gs_gaussians* host_v,
                      void* stream);
int gs_anchor_load(const gs_gaussians* host_params, const gs_gaussians* host_m, const gs_gaussians* host_v,
                   const gs_gaussians* params, const gs_gaussians* m, const gs_gaussians* v, void* stream);

/* Merging at an anchor (Sec. 4.4): a random 1/(k+1) of the too-fine
 * Gaussians each absorb up to k nearest too-fine neighbours, giving a coarser
 * active set.
 *  - Gaussian i is selected iff too_fine[i] and u_i < 1/(k+1), u_i the top 24
 *    bits of Philox4x32-10(counter (i, 0, 2, 0), key seed) / 2^24.
 *  - A selected Gaussian proposes the k nearest (Euclidean distance of the
 *    means, ties by index) Gaussians that are too fine and not selected, at
 *    most `radius` away; a Gaussian proposed by several selected ones is
 *    claimed by the lowest index.
 *  - Each selected Gaussian and the ones it claimed are replaced by their
 *    moment-matching merge: weights w_i = o_i a_i (opacity times the product
 *    of the two largest scales), mean and covariance the w-weighted mean and
 *    second moment about it (scales and rotation from its eigen-decomposition),
 *    SH the w-weighted mean, opacity min(0.99, sum_i w_i / a) with a the merged
 *    product of the two largest scales.
 *  - Claimed Gaussians leave the set; all others are copied unchanged. The
 *    output keeps index order; *n_out (device int64) = its size (<= in->n).
 * out (and m_out, v_out) need in->n rows. m_in, v_in, m_out, v_out: the Adam
 * moments (all four or none); merged rows get zero moments. lr_in, lr_out:
 * the per-Gaussian rate multipliers of gs_adam_step (both or none); merged
 * rows restart at 1. radius > 0, 1 <= k <= 8. ws:
 * gs_anchor_merge_workspace_size(in->n, k) bytes. */
size_t gs_anchor_merge_workspace_size(int64_t n, int32_t k);
int gs_anchor_merge(const gs_gaussians* in, const gs_gaussians* m_in, const gs_gaussians* v_in, const float* lr_in,
                    const uint8_t* too_fine, float radius, int32_t k, uint64_t seed, const gs_gaussians* out,
                    const gs_gaussians* m_out, const gs_gaussians* v_out, float* lr_out, int64_t* n_out, void* ws,
                    size_t ws_bytes, void* stream);

/* Opacity culling (Sec. 4.3, as in 3DGS): keeps the Gaussians with
 * sigmoid(logit) >= min_opacity, in index order, with their Adam moments and
 * rate multipliers when given (m/v: all four or none; lr: both or none);
 * *n_out (device int64) = the kept count. out needs in->n rows. ws:
 * gs_cull_opacity_workspace_size(in->n) bytes. */
size_t gs_cull_opacity_workspace_size(int64_t n);
int gs_cull_opacity(const gs_gaussians* in, const gs_gaussians* m_in, const gs_gaussians* v_in, const float* lr_in,
                    float min_opacity, const gs_gaussians* out, const gs_gaussians* m_out, const gs_gaussians* v_out,
                    float* lr_out, int64_t* n_out, void* ws, size_t ws_bytes, void* stream);

/* Anchor blending for novel views (Sec. 4.4, Eq. of w(r)): with d1 <= d2 the
 * distances of the camera to the two closest anchors, r = d1 / d2 and overlap
 * o in (0, 0.5): weight of the closest anchor = 1 for r < 1 - o, else
 * 1 - (r - (1 - o)) 0.5 / o. Host function; returns NaN for invalid input. */
float gs_anchor_blend_weight(float d1, float d2, float overlap);

/* Scales the opacities of n Gaussians by w in [0, 1] in place (opacity logit
 * l -> logit(w sigmoid(l))): the two anchors' sets are blended by rendering
 * their union with weights w and 1 - w. */
int gs_scale_opacity(float* mean_opa, int64_t n, float w, void* stream);

/* gs_spawn_propose for callers that cannot allocate device memory: the paper
 * has no counterpart; this is a deployment convenience. Callers such as a host
 * application that owns the allocator, or a process that reserved its memory
 * up front, can pass only their inputs and outputs: the scratch gs_spawn_propose
 * takes as `ws` is instead a file-scope device array inside the library, sized
 * for frames of at most 2,097,152 pixels (1920x1080 fits); about 16.8 MB that
 * every GPU which loads the library holds until the process exits. Arguments
 * and outputs are those of gs_spawn_propose; no workspace argument.
 *  - Returns GS_ERR_INVALID_ARG for width * height > 2,097,152 (use
 *    gs_spawn_propose for larger frames) and for the checks gs_spawn_propose
 *    makes; GS_ERR_CUDA if the array's device address cannot be obtained.
 *  - Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 *  - The first call on each device looks up the array's device address with
 *    that device current (cudaGetSymbolAddress); make that first call before
 *    any stream capture. The address belongs to the device's context: after
 *    cudaDeviceReset (a new primary context) the next call looks it up again,
 *    so that call too belongs outside a capture. Concurrent first calls from
 *    several host threads are serialised by a lock.
 *  - Every call shares the one array, which keeps the previous call's
 *    contents; nothing in it needs to start at zero (each pass writes what it
 *    reads). Calls whose kernels overlap on a GPU race on the array: issue them
 *    on one stream or otherwise order them. */
int gs_spawn_propose_noalloc(const float* image, const float* render, const float* depth, int32_t width,
                             int32_t height, const gs_camera* cam, const gs_spawn_config* sc, const gs_spawn_out* out,
                             void* stream);

/* Learned spawn proposal (not in the paper; the workload's per-patch MLP):
 * for each 8x8 patch of a frame, x = (its 192 pixel values, channel-major then
 * row-major, and the patch centre in [-1, 1]^2) -> 3 x (Linear 128 + GELU) ->
 * Linear 3 = (spawn logit, depth, log-scale). Weights and activations are
 * bfloat16 in the matrix products, accumulation and everything else FP32.
 * The log-scale output is an offset to direct sampling's scale (see
 * gs_spawn_learned).
 * Parameters (device, FP32 masters, nn.Linear layout): w1 [128][194], b1 [128],
 * w2 [128][128], b2, w3 [128][128], b3, w4 [3][128], b4 [3]. */
typedef struct gs_mlp_params {
    float *w1, *b1, *w2, *b2, *w3, *b3, *w4, *b4;
} gs_mlp_params;

typedef struct gs_mlp_config {
    int32_t tensor_path; /* 0: mma.sync bf16 tiles; 1: tcgen05.mma with the accumulator in tensor memory */
    float w_depth;       /* weight of the L1 depth term */
    float w_scale;       /* weight of the L1 log-scale term */
    float lr, beta1, beta2, eps; /* Adam */
} gs_mlp_config;

/* Patches of a width x height frame (both multiples of 8), -1 otherwise. */
int64_t gs_mlp_patches(int32_t width, int32_t height);
/* Number of parameters (58,243): the layout of `grads` below. */
int64_t gs_mlp_param_count(void);
size_t gs_mlp_workspace_size(int64_t n_patches);

/* Inference: out [n_patches][3] = (spawn logit, depth, log-scale) per patch in
 * row-major patch order. image [3][height][width]. */
int gs_mlp_forward(const gs_mlp_params* p, const float* image, int32_t width, int32_t height, float* out,
                   const gs_mlp_config* cfg, void* ws, size_t ws_bytes, void* stream);

/* One training step on a frame. targets [n_patches][4] = (fraction of the
 * patch's pixels whose direct-sampling spawn was kept, their mean depth, mean
 * log-scale, 1 if any was kept else 0). Loss (device float) = mean over
 * patches of BCE(sigmoid(logit), fraction) + w_depth |depth - target| mask +
 * w_scale |log-scale - target| mask. grads (optional, device [param_count])
 * receives dL/d(w1, b1, w2, b2, w3, b3, w4, b4) flattened in that order; when
 * m and v are given (Adam moments, same layout as p) p is updated by Adam with
 * step `step` (>= 1) or *step_dev. out (optional) as in gs_mlp_forward. */
int gs_mlp_train_step(const gs_mlp_params* p, const gs_mlp_params* m, const gs_mlp_params* v, const float* image,
                      int32_t width, int32_t height, const float* targets, const gs_mlp_config* cfg, int32_t step,
                      const int32_t* step_dev, float* loss, float* out, float* grads, void* ws, size_t ws_bytes,
                      void* stream);

/* The MLP's matrix product on its own, for testing the two tensor-core paths:
 * C [M][N] (ldc) = A [M][K] (lda) . B [N][K]^T (ldb); A, B bfloat16 (uint16
 * bit patterns), K-major; K, N multiples of 16, lda, ldb multiples of 8, ldc a
 * multiple of 4 and C 16-byte aligned. */
int gs_mlp_gemm_bf16(const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb, float* C, int64_t ldc,
                     int32_t M, int32_t N, int32_t K, int32_t tensor_path, void* stream);

/* Training targets of the learned proposal from one frame's spawns after the
 * frame's optimisation (the primitives direct sampling produces and keeps,
 * Sec. 4.2). Spawn i: pixel[i], where it was spawned; its Gaussian row after
 * the optimisation, mean_opa [n_spawn][4] (mean, opacity logit) and scale
 * [n_spawn][4] (log-scales); scale0 [n_spawn][4], its log-scale when spawned
 * (x used); cam, the frame's camera (device). Spawn i is kept when
 * sigmoid(logit) > keep_threshold (still present with some opacity; 0.05 in
 * the streaming loop). targets [n_patches][4] per 8x8 patch = (kept count /
 * 64, mean camera depth R_2 . mu + t_2 of the kept, mean over the kept of
 * (mean of the three log-scales - scale0.x), 1 if any kept else 0): the
 * change the optimisation made to the log-scale is what the network's third
 * output learns. Device buffers; ws: gs_mlp_targets_workspace_size bytes. */
size_t gs_mlp_targets_workspace_size(int32_t width, int32_t height);
int gs_mlp_targets(const int32_t* pixel, const float* mean_opa, const float* scale, const float* scale0,
                   const gs_camera* cam, float keep_threshold, int64_t n_spawn, int32_t width, int32_t height,
                   float* targets, void* ws, size_t ws_bytes, void* stream);

/* Spawning from the learned proposal's outputs mlp_out [n_patches][3]: the
 * network gives each 8x8 patch m its expected number of kept spawns
 * 64 sigmoid(logit_m); they are placed where direct sampling would place them.
 * Pixel p spawns iff u < min(1, sigmoid(logit_m) 64 P_s(p) / S_m) and its
 * depth is positive, with P_s the spawn probability of Eq. 1-3 (render
 * penalty included; render may be NULL), S_m = max(sum of P_s over the patch,
 * 0.064) and u = Philox4x32-10 of counter (p, frame, 1, 0) and key seed
 * (LoG sigma from sc). The depth is depth[p] (the per-pixel map
 * gs_spawn_propose takes; may be NULL) where that is positive and finite,
 * else the patch's predicted depth. The new Gaussian sits at the pixel
 * centre at that depth z with, on all axes, direct sampling's log-scale
 * log(z / (2 fx sqrt(P_L(p)))) plus the patch's predicted log-scale offset
 * (other attributes as gs_spawn_propose). Output (p_l, p_pen, p_s maps
 * optional), workspace size and status as for gs_spawn_propose. */
int gs_spawn_learned(const float* image, const float* mlp_out, const float* render, const float* depth,
                     int32_t width, int32_t height, const gs_camera* cam, const gs_spawn_config* sc,
                     const gs_spawn_out* out, void* ws, size_t ws_bytes, void* stream);

/* Error code recorded by a tensor-memory GEMM whose completion wait timed out
 * (0 = none). Synchronous; for tests. */
int gs_mlp_tc_error(int32_t* out);

/* Learning rates of the parameter groups and the Adam constants. */
typedef struct gs_adam_config {
    float lr_mean, lr_opacity, lr_scale, lr_rot, lr_sh_dc, lr_sh_rest;
    float beta1, beta2, eps;
    float decay; /* per-Gaussian rate decay (App. A.3): with lr_scale, each processed Gaussian's multiplier
                    is multiplied by decay after its update (1 = none) */
} gs_adam_config;

/* Sparse Adam over Gaussians with visible[g] != 0 (others untouched); params,
 * m, v in the gs_gaussians layout. lr_scale (optional, device float [n]):
 * per-Gaussian multiplier of every group rate, set to 1 when a Gaussian is
 * introduced and multiplied by cfg->decay after each step that processes it
 * (App. A.3). The step number (>= 1, for the bias
 * correction) is `step`, or, when step_dev is non-NULL, the device int32 it
 * points to (so a captured CUDA graph sees the current step; advance it with
 * gs_counter_add). */
int gs_adam_step(const gs_gaussians* params, const gs_grads* grads, const gs_gaussians* m, const gs_gaussians* v,
                 const gs_adam_config* cfg, int32_t step, const int32_t* step_dev, float* lr_scale, void* stream);

/* Pose update: Adam on the tangent gradient dL_dpose [n_views][6] with moments
 * m, v [n_views][6], then T_cw <- exp(delta^) T_cw with delta the Adam step;
 * cams updated in place. lr_t for rho, lr_r for phi. step / step_dev as for
 * gs_adam_step. */
int gs_pose_step(gs_camera* cams, int32_t n_views, const float* dL_dpose, float* m, float* v, float lr_t,
                 float lr_r, float beta1, float beta2, float eps, int32_t step, const int32_t* step_dev,
                 void* stream);

/* Pose of a differentiable render (Sec. 4.3 poses optimised jointly with the
 * Gaussians, written on the SE(3) tangent): cams_out[i] = exp(xi_i^) cams_ref[i]
 * for xi [n_views][6] = (rho, phi) on the device. The exponential is evaluated
 * in FP64 and rounded once into the FP32 camera. cams_out may equal cams_ref.
 * Intrinsics and sizes are copied. */
int gs_pose_apply(const gs_camera* cams_ref, const float* xi, int32_t n_views, gs_camera* cams_out, void* stream);

/* Gradient with respect to xi of a loss of exp(xi^) T_ref, from the tangent
 * gradient dL_ddelta that gs_render_bwd returns at T = exp(xi^) T_ref:
 * dL_dxi = J_l(xi)^T dL_ddelta, J_l the left Jacobian of SE(3) (closed form,
 * FP64). All arrays [n_views][6] on the device; dL_dxi may equal dL_ddelta. */
int gs_pose_tangent_grad(const float* xi, const float* dL_ddelta, int32_t n_views, float* dL_dxi, void* stream);

/* Coarse-to-fine training (Sec. 4.3: a new image is first used with 2^l
 * downsampling, l decremented every five iterations): out
 * [3][ceil(height/factor)][ceil(width/factor)] = the mean of each factor x
 * factor block of image [3][height][width] (partial blocks at ragged edges
 * average the pixels they have). The matching camera divides fx, fy, cx, cy
 * by the factor; pixel centres stay at I + 0.5. */
int gs_downsample(const float* image, int32_t width, int32_t height, int32_t factor, float* out, void* stream);

/* Mini bundle adjustment of the initial pose estimation (Sec. 4.1 bootstrapping,
 * App. A.1): `iterations` Levenberg-Marquardt iterations over the shared focal
 * length, the poses of frames 1..F-1 (frame 0 fixed) and P points, each point
 * observed in all F frames (2 <= F <= 8).
 *   obs     device float [P][F][2]: observed pixel of point p in frame f
 *   fl      device float [1], in/out: focal length (fx = fy; principal point cx, cy)
 *   poses   device float [F][12], in/out: world->camera R (row-major) | t
 *   points  device float [P][4], in/out: x, y, z, unused (16-byte aligned)
 *   lam     device float [1], in/out: damping (App. A.1 starts at 1e-5)
 * Residual r = (fl x/z + cx, fl y/z + cy) - obs for (x, y, z) = R X + t. Each
 * iteration discards observations whose |r| exceeds median + 4 MAD (lower
 * medians, selected by one CTA; P F <= 2^26), weights the rest by Huber
 * (threshold huber_delta px), solves
 * (H + lam diag(H) + 1e-9 I) d = -J^T W r by the Schur complement on the points
 * (reduced camera system in FP64), applies d (poses: T <- exp(d^) T) and keeps
 * it iff the robust cost on the same observations decreases (lam /= nu), else
 * lam *= nu; lam is kept within [1e-12, 1e10]. history (optional, device float [iterations][3]) receives (cost,
 * trial cost, accepted) per iteration; *failed (device int32) = 1 if a reduced
 * system was not positive definite (its step is then zero). Everything stays
 * on the device: the call can be captured into a CUDA graph. ws:
 * gs_ba_workspace_size(F, P) bytes. */
size_t gs_ba_workspace_size(int32_t n_frames, int64_t n_points);
/* The mini bundle adjustment's camera model: obs [P][F][2] = (fl x/z + cx,
 * fl y/z + cy) of every point in every frame (same layouts as gs_ba_lm). */
int gs_ba_project(const float* fl, const float* poses, const float* points, int32_t n_frames, int64_t n_points,
                  float cx, float cy, float* obs, void* stream);
int gs_ba_lm(const float* obs, int32_t n_frames, int64_t n_points, float cx, float cy, float* fl, float* poses,
             float* points, float* lam, int32_t iterations, float huber_delta, float nu, float* history,
             int32_t* failed, void* ws, size_t ws_bytes, void* stream);

/* Pose refinement of a new frame (Sec. 4.1, subsequent frames: 20 iterations
 * with all inliers after RANSAC): the iteration of gs_ba_lm over one camera
 * pose only, the M 3-D points and the focal length held fixed. Each
 * iteration: residual norms, median + 4 MAD rejection (lower medians), Huber
 * weights (threshold huber_delta px), (H + lam diag(H) + 1e-9 I) d = -J^T W r
 * for the left perturbation d = (rho, phi) of the pose (6 x 6, FP64), the
 * retracted trial pose T <- exp(d^) T kept iff the robust cost on the same
 * observations decreases (lam /= nu), else lam *= nu; lam in [1e-12, 1e10].
 *   points  device float [M][4]: x, y, z, unused (16-byte aligned)
 *   obs     device float [M][2]: observed pixel of each point
 *   fl      device float [1]: focal length (fx = fy; principal point cx, cy)
 *   pose    device float [12], in/out: world->camera R (row-major) | t
 *   lam     device float [1], in/out: damping
 *   history optional device float [iterations][3]: cost, trial cost, accepted
 *   failed  device int32 [1]: 1 if a damped system was not positive definite
 * ws: gs_ba_pose_workspace_size(M) bytes (0 for M outside 1..2^26). Nothing
 * leaves the device: the call can be captured into a CUDA graph. */
size_t gs_ba_pose_workspace_size(int64_t n_obs);
int gs_ba_pose_lm(const float* points, const float* obs, int64_t n_obs, const float* fl, float cx, float cy,
                  float* pose, float* lam, int32_t iterations, float huber_delta, float nu, float* history,
                  int32_t* failed, void* ws, size_t ws_bytes, void* stream);

/* Guided-matching depth refinement (Sec. 4.2 depth for new primitives,
 * App. A.2). For every pixel of the reference frame: n_cand inverse depths
 * d_k = d_lo + k (d_hi - d_lo) / (n_cand - 1), d_lo = max(1/Z* - window, 0),
 * d_hi = 1/Z* + window (the appendix uses window 0.1) around the monocular
 * depth Z*; among the n_nb neighbours, those for which the whole candidate
 * segment lies in front of the camera and inside the bilinear domain of its
 * map (sample coordinates x - 0.5 in [0, W-1] x [0, H-1]) are usable, and the
 * one whose segment is longest in pixels is chosen (adaptive matching; ties:
 * lower index); C_k = <F_ref(pixel), bilinear F_j(reprojected candidate k)>
 * in FP32; k* = the first maximum; when 0 < k* < n_cand - 1 the parabola
 * through C_{k*-1}, C_{k*}, C_{k*+1} moves d by its vertex offset times the
 * candidate step; depth = 1 / d.
 *   feats    device bfloat16 bit patterns [1 + n_nb][H][W][C]: the reference
 *            frame's map, then the neighbours'; C = channels in {8, 16, 32, 64};
 *            16-byte aligned
 *   cams     device gs_camera [1 + n_nb], reference first; intrinsics refer to
 *            the W x H maps (their width/height fields are not read)
 *   z_mono   device float [H][W]: monocular depth (z in the reference camera)
 *   depth    device float [H][W] out: refined depth; pixels with no usable
 *            neighbour, a monocular depth that is not a positive finite
 *            number, or a refined inverse depth <= 0 keep z_mono
 *   nb       device int32 [H][W] out, optional: chosen neighbour (0-based), -1
 *            where depth kept z_mono
 *   corr     device float [H][W] out, optional: C_{k*} (0 where nb = -1)
 * 1 <= n_nb <= 8, W, H >= 2, W H C < 2^31, 3 <= n_cand <= 1024, window > 0. */
int gs_guided_depth(const uint16_t* feats, const gs_camera* cams, int32_t n_nb, int32_t width, int32_t height,
                    int32_t channels, const float* z_mono, int32_t n_cand, float window, float* depth, int32_t* nb,
                    float* corr, void* stream);

/* counter[0] += delta on the device (advances a graph-visible step counter). */
int gs_counter_add(int32_t* counter, int32_t delta, void* stream);

/* L1 loss: loss[0] = sum |color - target| / count (deterministic reduction),
 * dL_dcolor = sign(color - target) / count. ws: 4 * 4096 bytes. */
int gs_l1_loss(const float* color, const float* target, int64_t count, float* dL_dcolor, float* loss, void* ws,
               size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GS_H */
