/*
 * gsr.h -- C ABI of the GB300-native differentiable RGB-D Gaussian splatting
 * renderer (GS-SLAM, arXiv 2311.11700: the hot path of mapping and tracking).
 *
 * What the library computes (paper passages):
 *   - the scene: N Gaussians (X, Sigma, Lambda, Y) with Sigma = R S S^T R^T,
 *     R from a quaternion (Sec. 3.1, Eq. scene-rep, Eq. covariance, supp. Eq. q2R);
 *   - the projected 2D covariance Sigma' = J W Sigma W^T J^T (Eq. covariance2d);
 *   - front-to-back alpha blending of colour (Eq. color_render), depth (Eq. depth)
 *     and accumulated opacity (Sec. 3.2, adding step) over depth-sorted Gaussians;
 *   - the L1 colour/depth loss (Eq. map_loss, Eq. track_loss) and its adjoint;
 *   - gradients w.r.t. every Gaussian parameter and the 6-DoF camera twist
 *     (Eq. pose_grad, supp. Sec. A);
 *   - the adaptive expansion step (Eq. add_method, Eq. delete_method, Eq. init-rep)
 *     and the reliable-Gaussian selection (Eq. coarse2fine).
 *
 * Definition constants (the paper is silent; the inherited rasteriser's
 * conventions): alpha = min(0.99, sigmoid(Lambda) exp(-q/2)) with
 * q = d^T Sigma'^-1 d; a Gaussian is skipped where q > 9 or alpha < 1/255; the
 * Gaussian whose blend would take the transmittance T below 1e-4 is not blended
 * and ends the pixel; 0.3 px^2 is added to the diagonal of Sigma'; the x/z, y/z
 * entering J are clamped to 1.3 tan(fov/2); Gaussians with camera z <= z_near are
 * dropped; colour = max(0, SH(dir) + 0.5) (real SH, Condon-Shortley phase kept,
 * degree 0..3); scale = exp(log_scale); pixel (u, v) has its centre at
 * (u + 0.5, v + 0.5).  The per-pixel 3-sigma test makes every result independent
 * of the tile size.  Equal depths are ordered by Gaussian index.
 *
 * Memory: every pointer in these structs is a DEVICE pointer unless stated.
 * The caller owns every parameter, image, gradient and workspace buffer; the
 * library allocates no device memory.  All entry points are asynchronous on the
 * given stream (a cudaStream_t passed as void*; NULL = legacy default stream)
 * and return after enqueueing.  The kernels of a call are launched with
 * programmatic stream serialisation and each waits for the grids before it at
 * entry, so stream order is kept; the calls can be captured in a CUDA graph
 * (the forward forks its short segment sorts onto a second stream of the
 * context and joins them with events).  Host-side argument errors return a status and
 * enqueue nothing.  Conditions only the device can see (pair-list capacity
 * exceeded, a bounded wait that ran out) set a sticky flag in the workspace;
 * later kernels of the call then do no work, and gs_workspace_status() reports
 * the flag.
 */
#ifndef GSR_H
#define GSR_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GS_API __attribute__((visibility("default")))
#else
#define GS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gs_status {
  GS_OK = 0,
  GS_ERR_INVALID_ARG = 1,   /* bad pointer, size, count or degree (host check)   */
  GS_ERR_CAPACITY = 2,      /* the (Gaussian, tile) pair list exceeded max_pairs  */
  GS_ERR_TIMEOUT = 3,       /* a bounded device-side wait ran out                 */
  GS_ERR_CUDA = 4,          /* a CUDA runtime call failed (see gs_last_error)     */
  GS_ERR_UNSUPPORTED = 5,   /* device or configuration not supported              */
  GS_ERR_STATE = 6          /* workspace does not hold a matching forward pass    */
} gs_status;

#define GS_MAX_VIEWS 32     /* views per call   */
#define GS_MAX_SCENES 32    /* scenes per call  */

/* One Gaussian parameter set, component-major planes of n floats each
 * (Eq. scene-rep, Eq. covariance):
 *   mean          [3][n]  world position X
 *   log_scale     [3][n]  log of the scale vector S
 *   quat          [4][n]  rotation quaternion (q_r, q_i, q_j, q_k), normalised inside
 *   opacity_logit [n]     Lambda before the sigmoid
 *   sh            [3K][n] SH coefficients, plane k*3 + c, K = (sh_degree+1)^2
 *   mask          [n]     optional (NULL = all): only Gaussians with mask != 0 render
 * All planes 4-byte aligned; n < 2^31. */
typedef struct gs_scene {
  int64_t n;
  int32_t sh_degree;        /* 0..3 */
  int32_t reserved;
  const float* mean;
  const float* log_scale;
  const float* quat;
  const float* opacity_logit;
  const float* sh;
  const uint8_t* mask;
} gs_scene;

/* Gradients of one parameter set: same layout as gs_scene.  By default every entry
 * point ACCUMULATES (+=) into these buffers and the caller zeroes them
 * (gs_ctx_set_grad_mode selects writing instead).  A NULL plane is not written.
 * Optional density statistics (both NULL = off), always accumulated (+=) over
 * calls: vs_grad_norm[i] += ||dL/dmu_ndc|| of Gaussian i in every view that renders
 * it (the gradient w.r.t. its projected centre in normalised device coordinates,
 * i.e. the pixel gradient scaled by (W/2, H/2)), vs_count[i] += 1 per such view;
 * gs_densify consumes them. */
typedef struct gs_grads {
  float* mean;
  float* log_scale;
  float* quat;
  float* opacity_logit;
  float* sh;
  float* vs_grad_norm;
  float* vs_count;
} gs_grads;

/* One camera view.  Pinhole intrinsics in pixels, world->camera pose W = [R | t]
 * (row-major 3x4, camera looks along +z, y down).  T_cw holds the pose by value;
 * T_cw_dev, when not NULL, points at 12 device floats that replace it (a pose
 * that kernels update, e.g. tracking inside a captured graph).  pixel_mask
 * (device [height][width], optional) restricts rendering and loss to pixels with
 * mask != 0; other pixels output 0. */
typedef struct gs_view {
  int32_t width, height;    /* 1 .. 16384 */
  int32_t scene;            /* index into the scenes array of the call */
  int32_t reserved;
  float fx, fy, cx, cy;
  float z_near;             /* Gaussians with camera z <= z_near are dropped */
  float bg[3];              /* background colour added with weight T_final   */
  float T_cw[12];
  const float* T_cw_dev;
  const uint8_t* pixel_mask;
} gs_view;

/* Images of all views of a call, packed view after view: view v starts at
 * pixel offset off_v = sum_{u<v} W_u H_u; colour holds planes [3][H][W] at
 * 3*off_v, depth and acc hold [H][W] at off_v.  A NULL plane is not written
 * (forward) or read as zero (backward). */
typedef struct gs_images {
  float* color;
  float* depth;
  float* acc;
} gs_images;

typedef struct gs_ctx gs_ctx;

/* Context: host-side only (device properties, tile size, last error text).
 * It owns no device memory.  One context may serve many workspaces.
 * device = -1 creates a host-only context that answers queries
 * (gs_workspace_query, gs_workspace_layout) but launches nothing. */
GS_API gs_status gs_ctx_create(gs_ctx** out, int device);
GS_API void gs_ctx_destroy(gs_ctx* ctx);
GS_API const char* gs_last_error(const gs_ctx* ctx);

/* Tile shape used by the forward and the backward (results do not depend on
 * it): tile_w x tile_h in {8x8, 16x8, 16x16, 32x8}.  Default 16x16. */
GS_API gs_status gs_ctx_set_tiling(gs_ctx* ctx, int tile_w, int tile_h);

/* Warp strip shapes of the compositing kernels (results do not depend on them):
 * each warp renders a strip of its tile and tests every Gaussian of the tile's
 * list against that strip.  0 = the tile's width x 4 rows, two pixels per lane
 * (any tile); for 16x16 tiles also 1 = 8x4 (one pixel per lane), 2 = 8x8 (two),
 * 3 = 16x2 (one), 4 = 16x8 (four), 5 = 8x16 (four).  The forward and the backward may use different shapes: the
 * strip test only skips Gaussians that cannot blend at any pixel of the strip.
 * Default: 2 for both (other tiles always use 0). */
GS_API gs_status gs_ctx_set_strip(gs_ctx* ctx, int strip_fwd, int strip_bwd);

/* How the per-tile depth-ordered lists of "sorting and alpha-blending" (Sec. 3.1)
 * are built; both give the same lists: within a tile, ascending float bits of the
 * camera depth, ties to the lower splat index.
 *   0 (default) per-tile counting sort: the projection counts the pairs of every
 *     tile, a scan turns the counts into the tile ranges, the pairs are appended to
 *     their tile's segment, and every segment is sorted by (depth bits, index);
 *   1 global stable LSD radix sort of the 64-bit (tile << 32 | depth bits) keys:
 *     the depth digits on the visible splats, then the tile digits on the pairs.
 * The mode changes the workspace size (query after setting it).  Any other mode:
 * GS_ERR_INVALID_ARG. */
GS_API gs_status gs_ctx_set_binning(gs_ctx* ctx, int mode);

/* Launch form of gs_render_step_l1's compositing kernel (results do not depend on
 * it).  0 (default): one CTA per (view, tile), CTAs in the longest-list-first order
 * (the grid form).  1: the persistent form: a grid of the kernel's resident CTAs on
 * every SM, whose warps take (tile, strip) work items -- one tile each in the
 * compacted-pixel form -- in the same order from a per-call ticket in the
 * workspace header until none is left.  Any other mode: GS_ERR_INVALID_ARG. */
GS_API gs_status gs_ctx_set_persistent(gs_ctx* ctx, int mode);

/* Bound of the device-side waits of the context's calls: the decoupled look-backs
 * of binning mode 1, gs_expand and gs_densify give up after `window_reads` reads of
 * their predecessors' status words (16 words a read) that have not completed their
 * prefix, set GS_ERR_TIMEOUT in the workspace header (gs_workspace_status reports
 * it) and let the later kernels of the call do nothing.  0 makes every such wait
 * give up before its first read (every work tile but the first reports the
 * timeout): a way to exercise that path without a hung GPU.  Default 2^20 (about a
 * second).  No wait in device code is unbounded.
 *
 * Failure injection for tests (no GPU fault involved): the environment variable
 * GSR_FAULT, read when a context is created, holds a comma-separated subset of
 *   alloc     the context's stream / event creation fails: render calls return
 *             GS_ERR_CUDA before they enqueue anything;
 *   capacity  the kernels see a pair capacity of 0: a forward that emits a pair
 *             reports GS_ERR_CAPACITY (with the real pairs_needed);
 *   timeout   the waits above get a bound of 0 reads. */
GS_API gs_status gs_ctx_set_spin_limit(gs_ctx* ctx, uint32_t window_reads);

/* How gs_render_backward / gs_pose_grad deliver gradients.
 *   0 (default) add: the parameter and twist gradients are added (+=) to the
 *     caller's buffers, which the caller zeroes;
 *   1 write: the buffers receive this call's gradients (=).  A scene rendered by
 *     exactly one view of the call is written directly by the projection adjoint
 *     (zeros for Gaussians that did not render); any other scene's buffers and the
 *     twist buffer are zeroed on the stream first and then accumulated.
 * Any other mode: GS_ERR_INVALID_ARG. */
GS_API gs_status gs_ctx_set_grad_mode(gs_ctx* ctx, int mode);

/* Which form of the compositing kernels ("sorting and alpha-blending", Sec. 3.1,
 * and its adjoint) serves a call.  The strip form gives every warp a fixed strip of
 * the tile (gs_ctx_set_strip); the compacted-pixel form gives one warp per tile,
 * which gathers the tile's pixels inside the call's pixel masks (the backward: the
 * pixels with a non-empty run) and walks the tile's list once per 32 of them.  For a
 * sparse pixel subset, such as the coarse stage of pose tracking (Sec. 3.3), that
 * skips the list walks of pixels that are masked out.  Both forms give identical
 * images, T_final and runs; gradients agree to float32 summation order.
 *   0 strip form always;
 *   1 (default) compacted form when every view of the call has a pixel_mask;
 *   2 compacted form always.
 * Any other mode: GS_ERR_INVALID_ARG. */
GS_API gs_status gs_ctx_set_compact(gs_ctx* ctx, int mode);

/* Bytes of workspace a call with these scenes/views and pair capacity needs.
 * max_pairs bounds the number of (Gaussian, tile) overlaps of all views. */
GS_API gs_status gs_workspace_query(gs_ctx* ctx, const gs_scene* scenes, int n_scenes,
                             const gs_view* views, int n_views, int64_t max_pairs,
                             size_t* bytes);

/* Forward render of n_views views (Eq. covariance2d, Eq. color_render, Eq. depth,
 * accumulated opacity).  Writes out->color/depth/acc and keeps in the workspace
 * what the backward needs (projected Gaussians, the per-tile depth-sorted
 * lists, per-pixel final transmittance and run length).  The workspace must be
 * at least gs_workspace_query(...) bytes, 256-byte aligned. */
GS_API gs_status gs_render_forward(gs_ctx* ctx, const gs_scene* scenes, int n_scenes,
                            const gs_view* views, int n_views, void* workspace,
                            size_t workspace_bytes, int64_t max_pairs,
                            const gs_images* out, void* stream);

/* L1 loss and its adjoint (Eq. map_loss, Eq. track_loss):
 *   L_v = w_c sum_{m in mask} sum_ch |C_hat - C_obs| + w_d sum_{m in mask, D_obs>0} |D_hat - D_obs|
 * loss[v] (device, n_views floats) is OVERWRITTEN; dL_dout->color/depth are
 * overwritten with w_c sign(C_hat - C_obs) and w_d sign(D_hat - D_obs)
 * (sign(0) = 0), dL_dout->acc (if not NULL) with 0.  target_rgb / target_depth
 * use the packed image layout. */
GS_API gs_status gs_loss_l1(gs_ctx* ctx, const gs_view* views, int n_views,
                     const gs_images* rendered, const float* target_rgb,
                     const float* target_depth, float w_c, float w_d, float* loss,
                     const gs_images* dL_dout, void* stream);

/* gs_render_forward and gs_loss_l1 in one pass: the compositing kernel computes
 * each pixel's L1 loss terms and writes the adjoint images in its epilogue
 * (Eq. map_loss, Eq. track_loss; same definitions as gs_loss_l1), so the rendered
 * images are not read back.  loss[v] is overwritten; out planes may be NULL. */
GS_API gs_status gs_render_forward_l1(gs_ctx* ctx, const gs_scene* scenes, int n_scenes,
                               const gs_view* views, int n_views, void* workspace,
                               size_t workspace_bytes, int64_t max_pairs, const gs_images* out,
                               const float* target_rgb, const float* target_depth, float w_c,
                               float w_d, float* loss, const gs_images* dL_dout, void* stream);

/* Backward of the preceding gs_render_forward on the same workspace with the
 * same scenes/views (Eq. pose_grad, supp. Sec. A).  dL_dout holds dL/dcolor,
 * dL/ddepth, dL/dacc (packed; NULL planes read as 0).  Accumulates parameter
 * gradients into grads[s] (one gs_grads per scene; grads may be NULL) and the
 * twist gradient into dL_dtwist (device [n_views][6], (rho, phi), left
 * perturbation exp(eps^) W; may be NULL).  pose_mode 0 = exact; 1 = the paper's
 * approximation (drops dSigma'/dP and the colour term of the twist gradient).
 * The forward's saved state is consumed: each forward allows one backward. */
GS_API gs_status gs_render_backward(gs_ctx* ctx, const gs_scene* scenes, int n_scenes,
                             const gs_view* views, int n_views, void* workspace,
                             size_t workspace_bytes, int64_t max_pairs,
                             const gs_images* dL_dout, const gs_grads* grads,
                             float* dL_dtwist, int pose_mode, void* stream);

/* As gs_render_backward, but only the twist gradient is produced (tracking,
 * Alg. 1): no parameter gradient is written. */
GS_API gs_status gs_pose_grad(gs_ctx* ctx, const gs_scene* scenes, int n_scenes,
                       const gs_view* views, int n_views, void* workspace,
                       size_t workspace_bytes, int64_t max_pairs,
                       const gs_images* dL_dout, float* dL_dtwist, int pose_mode,
                       void* stream);

/* One optimisation step of the L1 loss (Eq. map_loss, Eq. track_loss) in one
 * call: gs_render_forward_l1 followed by gs_render_backward (grads != NULL) or
 * gs_pose_grad (grads == NULL), with the compositing forward, the loss and the
 * compositing adjoint fused into one kernel.  The adjoint of the L1 loss at a
 * pixel depends on that pixel only, so every warp composites its pixels front to
 * back, forms the loss and its adjoint in registers and walks the same list back
 * to front; the per-pixel state never goes through memory.
 *   out        images to write (NULL, or members NULL: not written)
 *   loss       float[n_views]: per-view loss, written (zeroed by the call)
 *   grads      as in gs_render_backward (gs_ctx_set_grad_mode applies), or NULL
 *              for the pose gradient alone
 *   dL_dtwist  float[n_views][6] or NULL (at least one of grads, dL_dtwist)
 * The compositing uses the backward's strip shape (gs_ctx_set_strip) and the
 * compacted-pixel form under the same rule as the other calls.  Images equal
 * gs_render_forward_l1's bit for bit; gradients equal the separate calls' up to
 * the order of float atomics.  The workspace keeps no state for a later backward. */
GS_API gs_status gs_render_step_l1(gs_ctx* ctx, const gs_scene* scenes, int n_scenes,
                            const gs_view* views, int n_views, void* workspace,
                            size_t workspace_bytes, int64_t max_pairs, const gs_images* out,
                            const float* target_rgb, const float* target_depth, float w_c,
                            float w_d, float* loss, const gs_grads* grads, float* dL_dtwist,
                            int pose_mode, void* stream);

/* Byte offsets of the forward's saved state inside a workspace of this call,
 * for inspection and tests (all arrays indexed by splat s = splat_off[v] + i
 * for Gaussian i of view v, splat_off[v] = sum_{u<v} roundup(n_scene(u), 256)):
 *   rec      float[S][16]: (mu_x hi, mu_y hi, A, B, C, opacity, depth, mu_x lo,
 *                           red, green, blue, mu_y lo, ext_x, ext_y, lo, qth),
 *                           conic = [[A,B],[B,C]]; ext = footprint half-extents;
 *                           lo = log2(opacity), qth = max(-4.5 log2(e) + lo, -log2(255))
 *   rect     uint32[S][4]: (tx0 | tx1 << 16, ty0 | ty1 << 16, ext_x bits, ext_y bits)
 *   ntiles   uint32[S]   : tiles touched (0 = not rendered)
 *   dkey     uint32[S]   : float bits of the camera depth (the sort key)
 *   ranges   uint32[T][2]: [start, end) of global tile t in the sorted pair list
 *   pair_val uint32[P]   : splat of each sorted pair
 *   header   uint32[5]   : (error bits, visible splats, pairs, pairs needed,
 *                           segments longer than 2048 entries)
 *   order    uint32[T]   : the compositing kernels' launch order, a permutation of
 *                           the tiles by non-increasing length bucket: for list
 *                           length n, 8 floor(log2(n + 1)) plus the three bits of
 *                           n + 1 after its leading one (8 buckets per octave)
 * Valid after the forward has run (stream-ordered). */
typedef struct gs_layout {
  int64_t rec, rect, ntiles, dkey, ranges, pair_val, header;
  int64_t n_splats;     /* S (padded) */
  int64_t n_tiles;      /* T (all views) */
  int64_t splat_off[GS_MAX_VIEWS];
  int64_t tile_off[GS_MAX_VIEWS];
  int64_t order;
} gs_layout;

GS_API gs_status gs_workspace_layout(gs_ctx* ctx, const gs_scene* scenes, int n_scenes,
                              const gs_view* views, int n_views, int64_t max_pairs,
                              gs_layout* layout);

/* Stage timing (tracing).  on = 0: off.  on = 1: every call records a CUDA
 * event pair around each stage on its stream, and the compositing kernels count
 * the Gaussian-pixel evaluations they perform (workspace counters; the counting
 * costs the compositing kernels a few percent).  on = 2: the event pairs only,
 * with the compositing kernels of the untimed path.  Other values return
 * GS_ERR_INVALID_ARG.  Stages:
 *   0 setup (control memset, call tables)
 *   1 projection, with the per-tile pair counts and their scan (binning mode 0)
 *     or the visible-splat compaction (mode 1)
 *   2 pair emission (mode 1: after the four depth radix passes)
 *   3 tile sort (mode 0: the per-segment sorts; mode 1: the tile-digit radix
 *     passes and the tile ranges)
 *   4 composite fwd   5 L1 loss   6 composite bwd   7 projection bwd
 *   8 composite step (gs_render_step_l1: forward, L1 loss and backward in one kernel)
 * and, inside those (binning mode 0): 9 the tile scan (part of 1), 10 the short
 * segment sorts on the context's second stream and 11 the long ones on the call's
 * stream (both part of 3; 3 is their joint wall time).
 * gs_ctx_read_timing waits for the recorded events, adds their durations to
 * out (ms and launches per stage, calls) and, with reset, clears the totals.
 * Do not enable timing while a stream is being captured into a graph. */
#define GS_N_STAGES 12
typedef struct gs_timing {
  double ms[16];
  int64_t launches[16];
  int64_t calls;
} gs_timing;

GS_API gs_status gs_ctx_set_timing(gs_ctx* ctx, int on);
GS_API gs_status gs_ctx_read_timing(gs_ctx* ctx, gs_timing* out, int reset);

/* Counters of the workspace's last forward/backward (synchronises `stream`):
 * out[0] visible splats, out[1] pairs, out[2] blended (pixel, Gaussian) pairs of
 * the forward, out[3] of the backward (equal to out[2]), out[4..6] backward
 * warp-Gaussian iterations visited / with a blend / reduced across the warp,
 * out[7] tile segments longer than 512 entries (the medium and large segment
 * sorts' work in binning mode 0; 0 in mode 1).  out[2..6] are counted in timing
 * mode 1 only, 0 otherwise. */
GS_API gs_status gs_workspace_counters(gs_ctx* ctx, const void* workspace, void* stream,
                                int64_t out[8]);

/* Tracking (Sec. 3.3, Alg. 1).  One Adam step per view on its pose:
 * g = dL_dtwist[v] (the left-perturbation twist gradient, (rho, phi)),
 * m <- b1 m + (1-b1) g, s <- b2 s + (1-b2) g^2, delta = -lr * mhat / (sqrt(shat) + eps)
 * with bias-corrected mhat, shat, then T_cw_dev[v] <- exp(delta^) T_cw_dev[v] and
 * dL_dtwist[v] <- 0.  T_cw_dev: device [n_views][12] row-major world->camera poses;
 * state: device [n_views][16] = (m[6], s[6], step, unused[3]), zero before the first
 * step; lr: host [6] per-component learning rates. */
GS_API gs_status gs_pose_adam(gs_ctx* ctx, int n_views, float* T_cw_dev, float* dL_dtwist,
                       float* state, const float lr[6], float beta1, float beta2, float eps,
                       void* stream);

/* Pose apply (the camera model's twist, Sec. 3.3, supp. Sec. A): for every view v,
 * T_out[v] = exp(twist[v]^) T_in[v] with twist = (rho, phi) the left perturbation of
 * the world->camera pose (the same float32 exponential as gs_pose_adam).  twist:
 * device [n_views][6]; T_in, T_out: device [n_views][12] row-major [R | t] (may be the
 * same buffer).  One launch. */
GS_API gs_status gs_pose_apply(gs_ctx* ctx, int n_views, const float* twist, const float* T_in, float* T_out,
                               void* stream);

/* Gradient of a loss L(exp(xi^) T) w.r.t. the twist xi from dL_deps, the left-
 * perturbation gradient at the applied pose exp(xi^) T (what gs_render_backward
 * returns for a view rendered at that pose): dL_dtwist[v] = J(xi_v)^T dL_deps[v], with
 * J the left Jacobian of SE(3) (exp((xi + d)^) = exp((J d)^) exp(xi^) to first order),
 * summed as its power series in the adjoint of xi; exact to float32 rounding for
 * |phi| <= 2 pi.  At xi = 0, J = I.  twist, dL_deps, dL_dtwist: device [n_views][6]
 * (dL_dtwist is written, and may alias dL_deps).  One launch. */
GS_API gs_status gs_twist_chain(gs_ctx* ctx, int n_views, const float* twist, const float* dL_deps,
                                float* dL_dtwist, void* stream);

/* Reliable-Gaussian selection (Eq. coarse2fine): mask_out[i] = 1 when Gaussian i
 * projects (camera z > z_near) onto a pixel (floor of its centre) of `view` whose
 * observed depth D (obs_depth, device [H][W]) is > 0 with |D - z_i| <= eps, else 0.
 * The view's pose may be device-resident (T_cw_dev).  mask_out: device [n]. */
GS_API gs_status gs_select_reliable(gs_ctx* ctx, const gs_scene* scene, const gs_view* view,
                             const float* obs_depth, float eps, uint8_t* mask_out, void* stream);

/* Opacity selection: mask_out[i] = 1 when sigmoid(opacity_logit[i]) > thr and (keep
 * is NULL or keep[i] != 0). */
GS_API gs_status gs_select_opacity(gs_ctx* ctx, const gs_scene* scene, float thr, const uint8_t* keep,
                            uint8_t* mask_out, void* stream);

/* Adaptive expansion of the map at a keyframe (Sec. 3.2), out of place.
 *   delete (Eq. delete_method): a Gaussian whose centre projects (camera z > z_near)
 *     onto a pixel (floor of its centre) with observed depth D > 0 and D - z > gamma
 *     (it floats in front of the observed surface) gets opacity eta * opacity;
 *   prune: Gaussians with opacity < prune_opacity are dropped;
 *   add (Eq. add_method): each pixel with D > 0 and rendered accumulated opacity
 *     A < tau_T or |D - D_hat| > tau_D (optionally only the (u + v) even half, the
 *     first-frame sampling) becomes a Gaussian initialised as in Eq. init-rep: at the
 *     back-projection of the pixel centre at depth D, isotropic scale
 *     D / (sqrt(fx fy) sqrt(density)), identity rotation, opacity init_opacity, SH-0
 *     colour = the observed pixel colour, higher SH coefficients 0.
 * out receives the kept Gaussians (input order) then the new ones (raster order),
 * planes of `capacity` floats per component (mean [3][capacity], ...).  count_out
 * (device int64[4]): kept, added, written (min(total, capacity)), total.  A total
 * above capacity sets GS_ERR_CAPACITY in the expansion workspace (its first word);
 * rendered_acc / rendered_depth / obs_depth: device [H][W]; obs_rgb: [3][H][W]. */
#define GS_EXPAND_ADD 1
#define GS_EXPAND_DELETE 2
#define GS_EXPAND_PRUNE 4
#define GS_EXPAND_CHECKERBOARD 8
typedef struct gs_expand_params {
  float tau_T, tau_D;       /* Eq. add_method thresholds                 */
  float eta, gamma;         /* Eq. delete_method decay and distance (m)  */
  float init_opacity;       /* Eq. init-rep opacity, in (0, 1)           */
  float density;            /* fraction of pixels sampled, in (0, 1]     */
  float prune_opacity;      /* drop Gaussians below this opacity          */
  int32_t flags;            /* GS_EXPAND_* */
} gs_expand_params;

/* Adaptive density control (supp. implementation details: densify every 10
 * iterations in the first 70 of 100, gradient threshold 0.002, scale threshold
 * 0.02 m; the clone / split mechanics follow the inherited 3DGS method).
 * Gaussian i densifies when vs_grad_norm[i] / vs_count[i] >= grad_thr (never when
 * vs_count[i] = 0): with max(exp(log_scale)) <= scale_thr it is cloned (an identical
 * copy is added), otherwise split into two children at mean + R(q/|q|) (s * z_c),
 * s = exp(log_scale), z_c = (noise[3c][i], noise[3c+1][i], noise[3c+2][i]) for child
 * c = 0, 1 (noise: [6][n] standard normal samples drawn by the caller), with scale
 * s / split_scale and the parent's rotation, opacity and SH.  Decisions in float32.
 * Output (out of place, `capacity` floats per component): the Gaussians that are
 * not split (index order), then the clones (index order), then the children (two per
 * split Gaussian, index order).  count_out (device, int64[4]) receives (kept,
 * cloned, split, needed); entries beyond capacity are not written and the
 * workspace header flags GS_ERR_CAPACITY (read count_out[3]).  The workspace holds
 * gs_densify_workspace_query bytes, 256-byte aligned.  Stream-ordered. */
typedef struct gs_densify_params {
  float grad_thr;     /* 0.002 */
  float scale_thr;    /* 0.02 m */
  float split_scale;  /* 1.6: the children's scale divisor */
  int32_t reserved;
} gs_densify_params;

/* Output planes of gs_expand (device, `capacity` floats per component). */
typedef struct gs_scene_out {
  float* mean;
  float* log_scale;
  float* quat;
  float* opacity_logit;
  float* sh;
} gs_scene_out;

GS_API gs_status gs_densify_workspace_query(gs_ctx* ctx, int64_t n, size_t* bytes);
GS_API gs_status gs_densify(gs_ctx* ctx, const gs_scene* in, const float* vs_grad_norm,
                            const float* vs_count, const float* noise, const gs_densify_params* params,
                            const gs_scene_out* out, int64_t capacity, int64_t* count_out,
                            void* workspace, size_t workspace_bytes, void* stream);

GS_API gs_status gs_expand_workspace_query(gs_ctx* ctx, int64_t n, const gs_view* view, size_t* bytes);
GS_API gs_status gs_expand(gs_ctx* ctx, const gs_scene* in, const gs_view* view,
                    const float* rendered_acc, const float* rendered_depth, const float* obs_rgb,
                    const float* obs_depth, const gs_expand_params* params,
                    const gs_scene_out* out, int64_t capacity, int64_t* count_out,
                    void* workspace, size_t workspace_bytes, void* stream);

/* Autotuner of the launch configuration (results do not depend on it: the
 * footprint gate is per pixel, both binning modes build the same lists, and a warp
 * strip only skips Gaussians that cannot blend in it).  gs_autotune times this
 * call's forward and backward under every configuration of the search space --
 * tile {16x16, 16x8, 8x8, 32x8} x binning mode {0, 1}, and for 16x16 tiles the
 * forward and the backward warp strip 0..5 (each timed on its own) -- with CUDA
 * events on `stream`, best of `reps` calls after one warm-up, and makes the
 * fastest (forward + backward) the context's configuration.  It is cached in the
 * context under the batch's shape key (each view's size and scene, each scene's
 * Gaussian count rounded up to a power of two and its SH degree): a later call
 * with the same key only applies the cached choice (result->timed = 0) unless
 * force != 0.  The workspace must hold gs_autotune_workspace_query bytes (the
 * largest configuration); configurations whose pairs overflow max_pairs are
 * skipped.  out, dL_dout and grads are written by the timing calls (gradients
 * accumulate; their contents afterwards are unspecified).  Synchronises
 * `stream`; not to be called while the stream is being captured.
 * gs_autotune_save / gs_autotune_load write / read the context's cache as text,
 * one line per key. */
typedef struct gs_tune_result {
  int tile_w, tile_h, strip_fwd, strip_bwd, binning;
  float ms_fwd, ms_bwd;  /* best forward / backward time of the chosen configuration */
  int timed;             /* configurations timed (0: taken from the cache) */
} gs_tune_result;

GS_API gs_status gs_autotune_workspace_query(gs_ctx* ctx, const gs_scene* scenes, int n_scenes,
                                             const gs_view* views, int n_views, int64_t max_pairs,
                                             size_t* bytes);
GS_API gs_status gs_autotune(gs_ctx* ctx, const gs_scene* scenes, int n_scenes, const gs_view* views,
                             int n_views, void* workspace, size_t workspace_bytes, int64_t max_pairs,
                             const gs_images* out, const gs_images* dL_dout, const gs_grads* grads,
                             int reps, int force, gs_tune_result* result, void* stream);
/* The autotuner of gs_render_step_l1: same search space, cache and rules as
 * gs_autotune, but every configuration times the fused step itself (the arguments
 * are gs_render_step_l1's, then reps, force, result and stream).  The fused kernel
 * walks both ways in the backward's strip shape, so each strip shape s of 16x16
 * tiles is timed as (s, s), and the separate forward and backward timings of
 * gs_autotune need not rank it the same.  result->ms_fwd is the step's time,
 * ms_bwd 0.  The choice is cached under its own key (parameter and pose-only
 * steps apart).  out, loss, grads and dL_dtwist are written by the timing calls
 * (gradients accumulate in gradient write mode 0; contents afterwards
 * unspecified). */
GS_API gs_status gs_autotune_step_l1(gs_ctx* ctx, const gs_scene* scenes, int n_scenes,
                                     const gs_view* views, int n_views, void* workspace,
                                     size_t workspace_bytes, int64_t max_pairs, const gs_images* out,
                                     const float* target_rgb, const float* target_depth, float w_c,
                                     float w_d, float* loss, const gs_grads* grads, float* dL_dtwist,
                                     int pose_mode, int reps, int force, gs_tune_result* result,
                                     void* stream);
GS_API gs_status gs_autotune_save(gs_ctx* ctx, const char* path);
GS_API gs_status gs_autotune_load(gs_ctx* ctx, const char* path);

/* Pixel outlier rejection of the tracking loss (supp. tracking hyper-parameters:
 * a pixel whose loss exceeds ten times the median loss is ignored).  For every view
 * v: the per-pixel loss l = w_c ((|dR| + |dG|) + |dB|) + (D_obs > 0 ? w_d |dD| : 0),
 * evaluated in float32 in that order without fused multiply-adds, over the pixels of
 * views[v].pixel_mask (NULL: all); its lower median m (the masked loss of rank
 * (n - 1) / 2, found exactly); and mask_out[p] = 1 for the masked pixels with
 * l <= fl(factor x m), 0 elsewhere (all 0 for a view with no masked pixel).
 * rendered / targets are packed per view like gs_render_forward's images; with
 * w_d = 0 no depth is read (rendered->depth and target_depth may be NULL).  Weights
 * >= 0, factor > 0.  Workspace of gs_outlier_mask_workspace_query bytes, 256-byte
 * aligned.  Stream-ordered, 7 launches. */
GS_API gs_status gs_outlier_mask_workspace_query(gs_ctx* ctx, const gs_view* views, int n_views,
                                                 size_t* bytes);
GS_API gs_status gs_outlier_mask(gs_ctx* ctx, const gs_view* views, int n_views,
                                 const gs_images* rendered, const float* target_rgb,
                                 const float* target_depth, float w_c, float w_d, float factor,
                                 uint8_t* mask_out, void* workspace, size_t workspace_bytes,
                                 void* stream);

/* Reads the workspace's device-side status after the stream's work so far
 * (synchronises `stream`).  *pairs_needed (optional) receives the pair count the
 * last forward needed (compare with max_pairs after GS_ERR_CAPACITY). */
GS_API gs_status gs_workspace_status(gs_ctx* ctx, const void* workspace, void* stream,
                              int64_t* pairs_needed);

/* Forward render without a workspace: for callers that cannot allocate device
 * memory when they render, such as a plug-in whose host application owns the
 * GPU memory budget and offers no allocator, or a per-frame callback on a
 * latency-critical thread where cudaMalloc may block on a device-wide lock.
 * The paper has no counterpart; this is a deployment convenience.
 *
 * Same arguments and results as gs_render_forward minus the workspace: the
 * scratch lives in one static device array of 32 MiB per GPU, reserved by every
 * GPU that loads the library until the process exits.  A call whose
 * gs_workspace_query size exceeds 32 MiB returns GS_ERR_INVALID_ARG with the
 * sizes in gs_last_error (a 640x480 view of ~100k Gaussians fits).  It calls no
 * allocator.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture.  All calls share the array and it keeps the last call's
 * contents (each call clears what must start at zero), so calls that overlap on
 * the GPU, e.g. on two streams, race and corrupt each other: serialise them.
 * The saved state is overwritten by the next call, so keep a workspace and
 * gs_render_forward for renders that need a backward (a gs_render_backward given
 * the static array returns GS_ERR_STATE).  Device-side conditions (the pair list
 * exceeding max_pairs) are read with gs_render_forward_static_status. */
GS_API gs_status gs_render_forward_static(gs_ctx* ctx, const gs_scene* scenes, int n_scenes,
                                   const gs_view* views, int n_views, int64_t max_pairs,
                                   const gs_images* out, void* stream);

/* gs_workspace_status for the static array of gs_render_forward_static: the
 * device-side status of the last such call on the context's device (after a
 * GS_ERR_CAPACITY, *pairs_needed tells how many pairs that call needed; its images
 * are then not written).  Synchronises `stream`.  GS_ERR_STATE if no static
 * forward has run on the device.  The paper has no counterpart. */
GS_API gs_status gs_render_forward_static_status(gs_ctx* ctx, void* stream, int64_t* pairs_needed);

#ifdef __cplusplus
}
#endif
#endif /* GSR_H */
