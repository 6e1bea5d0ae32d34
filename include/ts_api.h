/*
 * ts_api.h -- C ABI of libts, the GB300 (sm_103a) differentiable triangle-splatting rasterizer.
 *
 * The library renders a triangle soup (or indexed mesh) with per-vertex colour and opacity into
 * colour, depth and opacity images, and back-propagates image-space loss gradients to vertex
 * positions, colours, opacities and the SE(3) camera pose.  It implements Triangle Splatting SLAM:
 *   Eq. 1  projection v_I = pi(T_CW v_W);
 *   Eq. 2  SDF phi(p) = max_i L_i(p) of the projected triangle, L_i the outward edge functions;
 *   Eq. 3  window I(p) = ReLU(phi(p) / phi(s))^sigma, s the incentre;
 *   Sec. 3.1 barycentric vertex-colour interpolation, face opacity o_F = (o_i + o_j + o_k) / 3;
 *   Eq. 4  front-to-back alpha compositing over faces sorted in depth order;
 *   Eq. 5-7 the analytic pose Jacobian, D v_C / D T_CW = [I_3, -[v_C]x], tau = (rho, theta).
 *
 * Conventions (all calls):
 *   - Every pointer named "device" is CUDA device memory owned by the caller; libts never
 *     allocates device memory.  Host pointers are read during the call only.
 *   - All calls except ts_plan_init, ts_workspace_size, ts_status_string and ts_sync_status
 *     are asynchronous on the given stream, perform no host synchronisation and no allocation,
 *     and may be captured into a CUDA graph.
 *   - Argument errors are returned synchronously (TS_ERR_INVALID_ARG, nothing launched).
 *     Errors detected on the device (pair-capacity overflow, a bounded wait that timed out) are
 *     latched in the workspace and reported by ts_sync_status; outputs are then unspecified.
 *   - Calls on one workspace must run in the order ts_project -> ts_bin -> ts_render_fwd ->
 *     ts_render_bwd -> ts_pose_grad on one stream (a later call may be repeated or omitted).
 *     The workspace keeps the per-face records, the sorted tile lists and, per pixel, the final
 *     transmittance and the list position of the last contribution, so that the backward pass
 *     recomputes blending state instead of storing it.
 *   - Images of the views are packed back to back: view v's colour starts at 3 * pix_off[v]
 *     and is planar [3][H][W]; depth, alpha and the other per-pixel arrays start at pix_off[v]
 *     and are [H][W]; pix_off[v] = sum over u < v of W_u * H_u.
 *   - Pixel (x, y) samples the image point (x + 0.5, y + 0.5).
 */
#ifndef TS_API_H
#define TS_API_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* ts_stream; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
  TS_OK = 0,
  TS_ERR_INVALID_ARG = 1, /* bad pointer, size, or parameter; nothing was launched */
  TS_ERR_CUDA = 2,        /* a CUDA launch or runtime call failed */
  TS_ERR_CAPACITY = 3,    /* more (tile, face) pairs than the plan's pair capacity */
  TS_ERR_TIMEOUT = 4,     /* a bounded device wait expired; outputs unspecified */
  TS_ERR_UNSUPPORTED = 5  /* a parameter combination the library does not implement */
} ts_status;

#define TS_MAX_VIEWS 256

/* Pinhole camera of one view (Eq. 1): u = fx * x_c / z_c + cx, v = fy * y_c / z_c + cy. */
typedef struct {
  float fx, fy, cx, cy;
  int32_t width, height;
} ts_camera;

/* World-to-camera pose T_CW (Eq. 1): v_C = R v_W + t, R row-major. */
typedef struct {
  float R[9];
  float t[3];
} ts_pose;

/* Rasterization parameters.  The paper fixes sigma (Table S5: 0.5); the rest are readings where
 * the paper is silent: alpha = min(alpha_max, o_F * I); a contribution with alpha < alpha_min is
 * skipped; a pixel stops before the face that would take its transmittance below T_min; faces
 * with a vertex at z <= z_near, an inradius below r_min pixels, o_F < alpha_min or an empty
 * pixel box are culled; bg is the background colour (weight T_final). */
typedef struct {
  float sigma, alpha_min, alpha_max, T_min, z_near, r_min;
  float bg[3];
  int32_t tile_w, tile_h;   /* tile shape: tile_w in {8, 16, 32}, tile_h in {4, 8, 16, 32}, <= 512 px */
  int32_t tris_per_stage;   /* faces staged in shared memory per step: 32, 64 or 128 */
  int32_t flags;            /* TS_FLAG_* bits; other bits must be 0 */
} ts_raster_params;

/* ts_raster_params.flags: run the raster kernels as persistent CTAs (as many as are resident on
 * the GPU) that take (view, tile) work items from a device counter, instead of one CTA per tile.
 * Results are identical; it helps when tiles of very uneven cost (mixed resolutions) are batched. */
#define TS_FLAG_PERSISTENT 1

/* ts_raster_params.flags: also render the normal map of Eq. 12 (ts_render_fwd_n) and take its
 * gradient (ts_render_bwd_n).  The projection then stores each visible face's unit normal in
 * camera space, turned towards the camera (triangles are two-sided), 16 bytes per (view, face),
 * and the raster kernels stage it beside the face's record. */
#define TS_FLAG_NORMALS 2

/* ts_raster_params.flags: the forward also counts, per (view, face), the pixels at which it
 * blended the face (4 bytes per (view, face) in the workspace), for ts_face_stats. */
#define TS_FLAG_STATS 4

/* ts_raster_params.flags: the Mesh Splatting face opacity o_F = min(o_i, o_j, o_k) instead of the
 * paper's mean (Sec. 3.1); dL/do_F then goes to the first vertex, in face order, that attains the
 * minimum. */
#define TS_FLAG_MIN_OPACITY 8

/* ts_raster_params.flags: each face has its own window exponent sigma_F (ts_map.sigma) in
 * I = ReLU(phi / phi(s))^sigma_F, as in Triangle Splatting, and ts_render_bwd returns dL/dsigma_F
 * (ts_map_grad.gsigma); the global sigma is then unused. */
#define TS_FLAG_FACE_SIGMA 16

/* ts_raster_params.flags: a forward-only plan, for callers that render without differentiating
 * (the render requests of a serving loop).  Its workspace holds no gradient slots and no per-pair
 * lane masks, the projection clears no gradient slots and the forward records no lane masks.
 * ts_render_bwd, ts_render_bwd_n, ts_render_step_l1 and ts_pose_grad on such a plan return
 * TS_ERR_INVALID_ARG. */
#define TS_FLAG_FORWARD_ONLY 32

/* The map (Sec. 3.1): N vertices with position, colour, opacity as structure-of-arrays float32
 * device buffers, and M faces.  faces = NULL selects triangle-soup mode (face m uses vertices
 * 3m, 3m+1, 3m+2; N = 3M); otherwise faces is device int32 [M][3].  The buffers must stay valid
 * and unchanged from ts_project until the ts_render_bwd of the same workspace has completed. */
typedef struct {
  const float *px, *py, *pz;
  const float *cr, *cg, *cb;
  const float *op;
  const int32_t* faces;
  int64_t n_vertices, n_faces;
  const float* sigma;  /* [n_faces] window exponents, read with TS_FLAG_FACE_SIGMA (else may be NULL) */
} ts_map;

/* Gradient buffers (device float32, same layout as ts_map).  ts_render_bwd ADDS into them, so
 * the caller zeroes them once and multi-view sums need no extra pass.  Any pointer may be NULL
 * to skip that gradient. */
typedef struct {
  float *gpx, *gpy, *gpz;
  float *gcr, *gcg, *gcb;
  float *gop;
  float *gsigma;  /* [n_faces] dL/dsigma_F with TS_FLAG_FACE_SIGMA (may be NULL) */
} ts_map_grad;

/* Host-side plan: the views, the map size, the parameters and the workspace layout.  Filled by
 * ts_plan_init; treat as opaque.  The caller owns it (stack or heap); it holds no pointers. */
#define TS_PLAN_BYTES 24576
typedef struct {
  uint64_t opaque[TS_PLAN_BYTES / 8];
} ts_plan;

/* Device-side counters, copied to the host by ts_sync_status. */
typedef struct {
  uint64_t n_pairs;          /* (tile, face) pairs emitted by ts_bin (may exceed capacity) */
  uint64_t pair_capacity;    /* the plan's capacity */
  uint64_t n_visible;        /* (view, face) records that survived culling */
  uint64_t fwd_contrib;      /* (pixel, face) contributions blended by ts_render_fwd */
  uint64_t bwd_contrib;      /* (pixel, face) contributions differentiated by ts_render_bwd */
  uint32_t error_bits;       /* bit 0 capacity overflow, bit 1 wait timeout, bit 2 an internal index
                                failed its bounds check and the access was skipped (TS_ERR_CUDA) */
  uint32_t reserved;
} ts_counters;

/* Default parameters: sigma 0.5 (Table S5), alpha_min 1/255, alpha_max 0.99, T_min 1e-4,
 * z_near 0.01, r_min 0.01 px, bg 0, tile 16 x 8, 64 faces per stage. */
void ts_default_params(ts_raster_params* out);

/* Validate the views and parameters and lay out the workspace.
 *   cams: host array [n_views]; 1 <= n_views <= TS_MAX_VIEWS; 1 <= width, height <= 16384.
 *   n_faces >= 0 (0 renders background only).
 *   pair_capacity: (tile, face) pairs the workspace can hold; 0 picks 4 * n_views * n_faces
 *   (at least 1024).  Returns TS_ERR_INVALID_ARG on any bad value. */
ts_status ts_plan_init(ts_plan* plan, const ts_camera* cams, int32_t n_views, int64_t n_faces,
                       const ts_raster_params* params, int64_t pair_capacity);

/* Bytes of device workspace the plan needs (256-byte aligned base required). */
size_t ts_workspace_size(const ts_plan* plan);

/* Zero the workspace's persistent state (counters, error word, per-pixel backward state).  Call
 * once after allocating the workspace and again after any device-side error; a workspace may then
 * be reused by plans of any layout that fits it.  Asynchronous. */
ts_status ts_workspace_init(const ts_plan* plan, void* ws, size_t ws_bytes, ts_stream stream);

/* Eq. 1-3 per (view, face): rigid transform, projection, culling, the face's screen-space
 * record (edge functions, barycentric interpolants, opacity) and its tile box and depth key.
 *   map:   device buffers (see ts_map); map->n_faces must equal the plan's n_faces.
 *   poses: device array [n_views] of ts_pose.
 *   ws:    device workspace of at least ts_workspace_size(plan) bytes, 256-byte aligned. */
ts_status ts_project(const ts_plan* plan, const ts_map* map, const ts_pose* poses, void* ws,
                     size_t ws_bytes, ts_stream stream);

/* Depth ordering per tile (Eq. 4, "sorted in depth order"): per-tile pair counts and their
 * exclusive scan (the per-tile [start, end) ranges), placement of each (tile, face) pair in its
 * tile's segment, and a sort of every segment by (depth bits, face id).  The result is the pair
 * list of 64-bit keys (global tile id << 32 | depth bits) with face-id values, ascending by key,
 * ties in ascending face id.  Pairs beyond the plan's capacity are dropped and latch
 * TS_ERR_CAPACITY (ts_sync_status). */
ts_status ts_bin(const ts_plan* plan, void* ws, ts_stream stream);

/* Eq. 3-4 forward: per pixel, front-to-back compositing of its tile's list with early
 * termination.  Writes (device, packed per view) color [3][H][W], depth [H][W] (sum of
 * z(p) alpha T, unnormalised) and alpha [H][W] (= 1 - T_final).  color must not alias the
 * others.  Any output may be NULL except that the workspace always records T_final and the
 * last-contribution position needed by ts_render_bwd. */
ts_status ts_render_fwd(const ts_plan* plan, void* ws, float* color, float* depth, float* alpha,
                        ts_stream stream);

/* ts_render_fwd that also writes the rendered normal map of Eq. 12: normal [3][H][W] packed per
 * view like color, N = sum alpha_n T_n n_F with n_F the face's camera-space unit normal turned
 * towards the camera, no background term.  normal != NULL needs a plan with TS_FLAG_NORMALS
 * (else TS_ERR_INVALID_ARG) and must not alias the other outputs. */
ts_status ts_render_fwd_n(const ts_plan* plan, void* ws, float* color, float* depth, float* alpha, float* normal,
                          ts_stream stream);

/* Adjoint of Eq. 1-4: back-to-front re-traversal from each pixel's last contribution, recovering
 * transmittance by division, warp-level reduction of per-face gradients before global atomics,
 * then the chain rule through the projection into the map gradients (added, see ts_map_grad)
 * and the per-view pose gradient partials consumed by ts_pose_grad.
 *   dC [3][H][W], dD, dA [H][W] packed per view (device); dD or dA may be NULL (zero).
 *   grad may be NULL or have NULL members to skip map gradients.
 * The per-face sums it accumulates start from the slots ts_project cleared, so each backward (this
 * call, ts_render_bwd_n or ts_render_step_l1) needs a ts_project of its own: a second backward
 * after one projection adds into the first one's sums. */
ts_status ts_render_bwd(const ts_plan* plan, void* ws, const float* dC, const float* dD,
                        const float* dA, const ts_map_grad* grad, ts_stream stream);

/* ts_render_bwd with the gradient dN [3][H][W] of the loss w.r.t. the normal map (device, packed
 * per view; NULL = zero), which reaches the vertex positions and the pose through each face's
 * normal and through alpha and T.  dN != NULL needs a plan with TS_FLAG_NORMALS. */
ts_status ts_render_bwd_n(const ts_plan* plan, void* ws, const float* dC, const float* dD, const float* dA,
                          const float* dN, const ts_map_grad* grad, ts_stream stream);

/* Map statistics of the last ts_project / ts_render_fwd (Sec. 3.4: densification by pixel
 * coverage above theta_blur * H * W, pruning by projected area above epsilon_a, keyframing by
 * triangle co-visibility), per (view, face) in view-major order [n_views][n_faces]:
 *   coverage:  device uint32, pixels at which the forward blended the face (alpha >= alpha_min,
 *              before termination); needs TS_FLAG_STATS;
 *   area:      device float, projected area |D2| / 2 in pixels^2 of a face that passed culling,
 *              else 0 (D2 formed from the record's vertices in the projection's operation order);
 *   visible:   device uint32 [n_views][ceil(n_faces / 32)], bit m of view v set when the face's
 *              coverage is > 0; needs TS_FLAG_STATS;
 *   n_visible: device uint32 [n_views], the number of visible faces; needs TS_FLAG_STATS.
 * Any output may be NULL.  Asking for a TS_FLAG_STATS output without the flag returns
 * TS_ERR_INVALID_ARG.  Integer outputs are exact; all are deterministic. */
ts_status ts_face_stats(const ts_plan* plan, void* ws, uint32_t* coverage, float* area, uint32_t* visible,
                        uint32_t* n_visible, ts_stream stream);

/* Triangle co-visibility between views (Sec. 3.4 keyframing): iou[i][j] = |S_i and S_j| /
 * |S_i or S_j| of the visible-face sets written by ts_face_stats (device uint32
 * [n_views][ceil(n_faces / 32)]); 0 when both are empty.  iou: device float [n_views][n_views]. */
ts_status ts_covisibility(const ts_plan* plan, const uint32_t* visible, float* iou, ts_stream stream);

/* Normal loss of Eq. 12 per view: loss_v = sum over pixels with a sensor normal (tgt_normal not
 * the zero vector) of (1 - N . Nbar) / (HW), N as rendered (not renormalised); dN = weight *
 * dloss_v/dN (written; weight is lambda_norm of Eq. 15, 0.05 in Table S5).  normal, tgt_normal
 * and dN: device [3][H][W] packed per view; loss: device float [n_views], overwritten.
 * Deterministic.  Needs no earlier call on the workspace. */
ts_status ts_normal_loss(const ts_plan* plan, void* ws, const float* normal, const float* tgt_normal, float weight,
                         float* loss, float* dN, ts_stream stream);

/* One training step's raster work in one pass per tile: the Eq. 3-4 forward, the mean-L1 loss of
 * ts_l1_loss (the L1 part of Eq. 8 with the depth term of Eq. 9) and the backward of ts_render_bwd
 * driven by that loss's dC and dD (no dA), with the same results as those three calls.  The L1
 * gradient of a pixel depends on that pixel alone, so each tile runs its backward right after its
 * forward while its staged records and its pixels' state are still on the chip: no image gradient
 * is written and read back, and most records are not staged twice.
 *   tgt_color [3][H][W], tgt_depth [H][W]: targets packed per view (device), as in ts_l1_loss;
 *   color [3][H][W], depth, alpha [H][W]: outputs as in ts_render_fwd (depth, alpha may be NULL);
 *   loss: device float [n_views], overwritten (fixed-order sums of per-tile partials);
 *   dC, dD: NULL, or device images that also receive the loss gradients;
 *   grad: as in ts_render_bwd (map gradients added; pose partials for ts_pose_grad).
 * Calls on the workspace: ts_project -> ts_bin -> ts_render_step_l1 [-> ts_pose_grad].  The fused
 * step does not record the per-pixel T_final and last-contribution position (its backward keeps
 * them on the chip), so ts_render_bwd cannot follow it without a new ts_render_fwd; as for every
 * backward, a second one needs a new ts_project.  A plan with
 * TS_FLAG_NORMALS or TS_FLAG_FACE_SIGMA, a NULL required pointer, or a negative or non-finite
 * lambda_dep returns TS_ERR_INVALID_ARG. */
ts_status ts_render_step_l1(const ts_plan* plan, void* ws, const float* tgt_color, const float* tgt_depth,
                           float lambda_dep, float* color, float* depth, float* alpha, float* loss, float* dC,
                           float* dD, const ts_map_grad* grad, ts_stream stream);

/* Eq. 5-7: dL/dtau per view for the left perturbation Exp(tau) o T_CW, tau = (rho, theta), as
 * sum over the view's visible face vertices of [g_C ; v_C x g_C], reduced deterministically.
 *   dtau: device float [n_views][6], overwritten. */
ts_status ts_pose_grad(const ts_plan* plan, void* ws, float* dtau, ts_stream stream);

/* Mean-L1 colour + depth loss used by tracking and mapping (Eq. 8 L1 part, Eq. 9): per view,
 *   loss_v = sum |C - Cbar| / (3HW) + lambda_dep * sum_{Dbar > 0} |D - Dbar| / (HW),
 * with dC = dloss/dC and dD = dloss/dD (overwritten; sign(0) = 0).  All pointers device, packed
 * per view; loss: float [n_views], overwritten.  Deterministic.  Uses only the workspace's
 * partial-sum region: no earlier call on the workspace is needed.  A negative or non-finite
 * lambda_dep returns TS_ERR_INVALID_ARG. */
ts_status ts_l1_loss(const ts_plan* plan, void* ws, const float* color, const float* depth,
                     const float* tgt_color, const float* tgt_depth, float lambda_dep, float* loss,
                     float* dC, float* dD, ts_stream stream);

/* Tracking / mapping photometric loss of Eq. 8 with the depth term of Eq. 9-10, per view:
 *   loss_v = (1 - lambda_ssim) sum |C - Cbar| / (3HW) + lambda_ssim (1 - sum SSIM / (3HW))
 *            + lambda_dep sum_{Dbar > 0} |D - Dbar| / (HW),
 * SSIM the per-pixel, per-channel structural similarity (Wang et al. 2004) under an 11 x 11
 * Gaussian window (sigma 1.5, normalised, zeros outside the image), C1 = 0.01^2, C2 = 0.03^2;
 * the paper weights D-SSIM by lambda_ssim = 0.2 (Table S5).  Writes dC = dloss/dC and
 * dD = dloss/dD (overwritten; sign(0) = 0).  Pointers and packing as in ts_l1_loss; loss: device
 * float [n_views], overwritten.  lambda_ssim = 0 gives the ts_l1_loss value.  lambda_ssim outside
 * [0, 1] or a negative or non-finite lambda_dep returns TS_ERR_INVALID_ARG.  Deterministic: the
 * partial sums per 32 x 32 tile are reduced in a fixed order.  Like ts_l1_loss it needs no earlier
 * call on the workspace. */
ts_status ts_pho_loss(const ts_plan* plan, void* ws, const float* color, const float* depth,
                      const float* tgt_color, const float* tgt_depth, float lambda_ssim, float lambda_dep,
                      float* loss, float* dC, float* dD, ts_stream stream);

/* The same loss as ts_l1_loss for callers that cannot give the library any device memory of its
 * own: an application that owns the whole device budget and lends out only the image buffers,
 * or a loop in which a cudaMalloc would synchronise the device or exceed a fixed memory pool.
 * The paper has no counterpart; this is a deployment variant of the loss above.
 *   cams: host array [n_views] describing the packed images (only width and height are used);
 *   color, depth, tgt_color, tgt_depth, loss, dC, dD: device, as in ts_l1_loss.
 * Needs no plan and no workspace and allocates nothing: the per-block partial sums live in one
 * static device array of 512 KiB (65536 (view, 2048-pixel block) slots), held by every GPU that
 * loads the library until the process exits.  n_views * ceil(max W*H / 2048) above 65536 returns
 * TS_ERR_INVALID_ARG, as do null pointers, bad sizes and a negative or non-finite lambda_dep.
 * The buffers and the stream must belong to the current device, whose copy of the array the call
 * uses; the cameras alone fix how far the kernels read and write, so each buffer must hold what
 * they describe.  The first call on a device looks up the array's address (make it before any
 * stream capture); the address stays valid while the device's context lives, so after a
 * cudaDeviceReset the call must not be used on that device again.  Each call rewrites every slot
 * it reads, so nothing carries over between calls; calls that overlap on the GPU share the array
 * and race. */
ts_status ts_l1_loss_noalloc(const ts_camera* cams, int32_t n_views, const float* color, const float* depth,
                             const float* tgt_color, const float* tgt_depth, float lambda_dep, float* loss,
                             float* dC, float* dD, ts_stream stream);

/* Equilateral regulariser of the mapping loss (Eq. 14), over the plan's n_faces faces of map:
 *   E = (1/M) sum_faces (1/3) sum_n (cos theta_n - 0.5)^2,
 * theta_n the internal angle at vertex n, its cosine from the normalised edge vectors leaving
 * vertex n.  A face with a zero-length edge adds 0 and no gradient (it still counts in M).
 *   map:    device buffers as for ts_project (only positions and faces are read).
 *   ws:     the plan's workspace (only its partial-sum region is written; no earlier call needed).
 *   loss:   device float [1], overwritten with E (unweighted).
 *   grad:   NULL, or device buffers whose gpx, gpy, gpz (each may be NULL) receive
 *           += weight * dE/dpos; the paper weights E by lambda_equi = 1.2 (Table S5).
 * Deterministic for soup maps; indexed meshes add shared-vertex terms with atomics.  A face
 * index outside [0, n_vertices) latches the bounds bit (TS_ERR_CUDA at ts_sync_status) and the
 * face is skipped. */
ts_status ts_equilateral(const ts_plan* plan, const ts_map* map, void* ws, size_t ws_bytes, float weight,
                         float* loss, const ts_map_grad* grad, ts_stream stream);

/* Pose update for tracking: poses[v] <- Exp(-step[v]) o poses[v] (left perturbation, closed-form
 * SE(3) exponential), step = (rho, theta) device float [n_views][6]; poses device [n_views]. */
ts_status ts_pose_apply(const ts_plan* plan, ts_pose* poses, const float* step, ts_stream stream);

/* Gradient-descent tracking step (Sec. 3.3: the pose is optimised by gradient descent on
 * dL/dtau; rotation and translation learning rates of Table S5): Adam on dtau per view, then
 * poses[v] <- Exp(-step) o poses[v].  state: device float [n_views][13] (first moments, second
 * moments, step count), zeroed by the caller before the first step and updated in place, so the
 * step can be captured in a CUDA graph and replayed.  lr_rho scales the translation part. */
ts_status ts_pose_adam(const ts_plan* plan, ts_pose* poses, const float* dtau, float* state, float lr_rho,
                       float lr_theta, float beta1, float beta2, float eps, ts_stream stream);

/* Synchronise the stream, copy the device counters into *out (may be NULL) and return
 * TS_ERR_CAPACITY / TS_ERR_TIMEOUT if the device latched an error since ts_workspace_init,
 * else TS_OK. */
ts_status ts_sync_status(const ts_plan* plan, void* ws, ts_stream stream, ts_counters* out);

/* Views, tiles and pixel offsets of the plan (host, for packing images).
 *   pix_off, tile_off: host int64 [n_views + 1] (may be NULL). */
ts_status ts_plan_layout(const ts_plan* plan, int64_t* pix_off, int64_t* tile_off,
                         int32_t* tiles_x, int32_t* tiles_y);

/* Debug access to intermediate arrays (asynchronous device-to-device copy of up to bytes).
 *   what: 0 sorted keys (uint64 [capacity]), 1 sorted face ids (uint32 [capacity]),
 *         2 tile ranges (uint32 [n_tiles][2]), 3 tile boxes (int16 [V*M][4]),
 *         4 depth keys (uint32 [V*M]), 5 tiles touched (uint32 [V*M]),
 *         6 T_final (float [total px]), 7 last-contribution positions (int32 [total px]),
 *         8 face records (float [V*M][32]). */
ts_status ts_debug_copy(const ts_plan* plan, void* ws, int32_t what, void* dst, size_t bytes,
                        ts_stream stream);

/* Failure-detection probe: launches one thread that waits, with the library's bounded wait, for
 * an mbarrier phase that nothing completes; after limit_us microseconds
 * (1..5,000,000) it latches the timeout bit, which ts_sync_status then reports as TS_ERR_TIMEOUT.
 * Nothing is copied and nothing faults; ts_workspace_init clears the bit. */
ts_status ts_debug_timeout_probe(const ts_plan* plan, void* ws, uint32_t limit_us, ts_stream stream);

/* Per-stage CUDA-event timing: when events != NULL, later calls record events[2k] before and
 * events[2k+1] after stage k (see TS_STAGE_*) on the launching stream.  events: host array of
 * 2 * TS_N_STAGES cudaEvent_t created by the caller; NULL disables timing. */
enum { TS_STAGE_PROJECT = 0, TS_STAGE_BIN = 1, TS_STAGE_FWD = 2, TS_STAGE_BWD_RASTER = 3,
       TS_STAGE_BWD_PROJECT = 4, TS_STAGE_POSE = 5, TS_STAGE_LOSS = 6, TS_N_STAGES = 7 };
ts_status ts_set_stage_events(ts_plan* plan, void* const* events);

const char* ts_status_string(ts_status s);

#ifdef __cplusplus
}
#endif

#endif /* TS_API_H */
