/*
 * dags.h -- C ABI of the GB300 (sm_103a) MP-aware differentiable Gaussian
 * splatting library (libdags.so): the data-parallel hot path of DAGS-SLAM
 * (arXiv 2602.21644).
 *
 * Conventions for every entry point
 *   - extern "C", plain pointers and sizes; no C++ or framework types.
 *   - "device" pointers are CUDA global-memory pointers on the current device;
 *     "host" pointers are ordinary CPU memory, read before the call returns.
 *   - Work is enqueued asynchronously on the given cudaStream_t (passed as
 *     void*; NULL = legacy default stream). No call synchronises the device
 *     except dags_sync_status and the e2e helpers that say so.
 *   - The caller owns every input and output buffer; a dags_ctx owns only
 *     its workspace. A ctx must not be used from two streams at once.
 *   - Return value: DAGS_OK (0) or a negative DAGS_E_* code. Argument errors
 *     are found on the host before anything is launched. Errors that only the
 *     device can see (pair-capacity overflow, a bounded wait that gave up)
 *     are recorded in the ctx's device status word, which dags_sync_status
 *     reads (and clears); the outputs of the call that raised them are
 *     undefined. Enqueuing never waits for the device.
 *   - Nothing traps, asserts or spins without a bound on the device.
 *
 * Data layouts
 *   Gaussian record: 16 x 32-bit words (64 bytes), n records contiguous:
 *     0-2 mean (world, m) | 3 opacity logit | 4-7 rotation quaternion
 *     (w, x, y, z; any non-zero norm) | 8-10 natural-log scale per axis |
 *     11 motion probability M in [0, 1] | 12 = bf16(r) | bf16(g) << 16 |
 *     13 = bf16(b) | 14-15 ignored.  (Sec. IV-A: a Gaussian is a mean,
 *     opacity, scale and rotation, augmented with its MP state; colour is
 *     view-independent RGB stored in BF16.)
 *   Pose: 12 doubles, row-major 3x4 [R | t], world -> camera (T_CW).
 *   Targets: per view H*W float4 (r, g, b, depth) in row-major pixel order;
 *     depth <= 0 marks a pixel without valid depth (no depth term), r < 0 a
 *     pixel without valid colour (left out of the loss altogether).
 *   Image (forward output): per view DAGS_IMG_CHANNELS planes of H*W float:
 *     0-2 colour C, 3 depth D, 4 opacity O = 1 - T_final, 5 rendered MP
 *     R_MP = sum_k omega_k M_k, 6 final transmittance, 7 static weight w(u)
 *     of Eq. (20) (0 when no targets are given).
 *   Gaussian gradient: 16 floats per Gaussian, same slots as the record
 *     (mean, opacity logit, quaternion, log-scale, 0, colour r g b, 0, 0).
 *   Pose gradient / twist: 6 doubles (rho_x, rho_y, rho_z, phi_x, phi_y,
 *     phi_z) of the left perturbation T <- exp(xi^) T.
 *   Pixel (i, j) is the point (u, v) = (i, j); u = fx x / z + cx.
 */
#ifndef DAGS_H
#define DAGS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DAGS_ABI_VERSION 1
#define DAGS_IMG_CHANNELS 8
#define DAGS_GRAD_WORDS 16
#define DAGS_RECORD_WORDS 16

enum {
  DAGS_OK = 0,
  DAGS_E_INVAL = -1,     /* bad argument (host check)                         */
  DAGS_E_CUDA = -2,      /* a CUDA runtime call failed                        */
  DAGS_E_CAPACITY = -3,  /* tile/Gaussian pairs exceeded the ctx's max_pairs  */
  DAGS_E_TIMEOUT = -4,   /* a bounded device wait gave up                     */
  DAGS_E_NOMEM = -5,     /* workspace allocation failed                       */
  DAGS_E_ORDER = -6,     /* splat_backward without its matching splat_forward */
  DAGS_E_BOUNDS = -7     /* an index out of range: a DAGS_CHECK build's check, or an
                            epipolar_verify match id; the access was skipped */
};

typedef struct dags_ctx dags_ctx;

/* Pinhole camera shared by all views of a call. */
typedef struct {
  float fx, fy, cx, cy;
  int32_t width, height;
} dags_camera;

/* Rasteriser constants. The paper inherits the 3DGS rasteriser without
 * printing it (Sec. IV-D, "during rasterization"); these are the readings
 * the oracle uses. tile must be 16. */
typedef struct {
  int32_t tile;       /* 16 */
  float alpha_min;    /* skip a Gaussian whose alpha is below this (1/255)    */
  float alpha_max;    /* clamp alpha to this (0.99)                           */
  float t_min;        /* stop before transmittance would fall below (1e-4)    */
  float dilation;     /* added to the 2D covariance diagonal, px^2 (0.3)      */
  float z_near;       /* cull means with camera z <= z_near, m (0.2)          */
  float guard;        /* Jacobian evaluated with |x/z| clamped to guard * W/(2 fx) (1.3) */
} dags_raster_cfg;

/* MP-weighted loss of Eqs. (20)-(22): L = sum_u w(u) (lambda_pho ||C - C_gt||_1
 * + lambda_depth [D_gt > 0] |D - D_gt|). weight_mode 0: w = (O - R_MP) / O
 * (compositing weights normalised to sum to 1, as Eq. (20) states; w = 0
 * where O <= o_eps); 1: w = O - R_MP. weight_grad 0: w is a constant of the
 * adjoint (stop-gradient); 1: it is differentiated. lambda_pho = 0.9,
 * lambda_depth = 0.1 are the paper's (Sec. V-A(c)). */
typedef struct {
  float lambda_pho, lambda_depth;
  int32_t weight_mode, weight_grad;
  float o_eps;
} dags_loss_cfg;

/* Adam on the pose twist (Eq. (27)'s pose part; first-order reading of the
 * paper's pose refinement). lr per twist component. */
typedef struct {
  double lr[6];
  double beta1, beta2, eps;
} dags_pose_cfg;

void dags_default_raster_cfg(dags_raster_cfg *cfg);
void dags_default_loss_cfg(dags_loss_cfg *cfg);
void dags_default_pose_cfg(dags_pose_cfg *cfg);

/* Create a context on the current CUDA device with workspace for up to
 * max_gaussians Gaussians, images up to max_width x max_height, max_views
 * views per call and max_pairs (tile, Gaussian) pairs per call (0 picks the
 * larger of 16 * max_gaussians * max_views and min(max_gaussians, 4096) *
 * tiles * max_views, so that splat_track's fixed-capacity tile buckets hold
 * at least min(max_gaussians, 4096) entries each). Allocates device memory
 * (cudaMalloc).
 * Returns DAGS_E_INVAL / DAGS_E_NOMEM / DAGS_E_CUDA on failure (*out = NULL). */
int dags_create(dags_ctx **out, int64_t max_gaussians, int32_t max_width, int32_t max_height,
                int32_t max_views, int64_t max_pairs);
void dags_destroy(dags_ctx *ctx);
const char *dags_status_string(int code);
int dags_abi_version(void);

/* Synchronise the ctx's last stream, read and clear the device status word.
 * Returns the pending status (DAGS_OK if none); *required_pairs (may be
 * NULL) receives the pair count the last forward needed. */
int dags_sync_status(dags_ctx *ctx, int64_t *required_pairs);

/* Introspection (tests): after a splat_forward on this ctx, copy its tile
 * offsets (n_start = n_views * tiles + 1 uint32, tiles = ceil(W/16) *
 * ceil(H/16), view-major then row-major tiles) and the depth-ordered Gaussian
 * ids of all tiles (up to cap uint32) to host memory. Synchronises the ctx's
 * last stream. *n_pairs (may be NULL) receives the pair count. Returns
 * DAGS_E_CAPACITY if that forward overflowed, DAGS_E_INVAL if n_start does
 * not match it. The sort key is (tile, FP32 camera depth of the mean
 * computed as ((r20 mx + r21 my) + r22 mz) + tz without FMA, Gaussian id). */
int dags_copy_bins(dags_ctx *ctx, uint32_t *tile_start, int64_t n_start, uint32_t *ids, int64_t cap,
                   int64_t *n_pairs);

/* Forward: project, bin, depth-sort and alpha-composite n Gaussians into
 * n_views views (one camera, per-view poses), and with targets the loss.
 *
 * gauss     device, n records (see layout). n may be 0.
 * cam       host, one camera; width/height <= the ctx maxima.
 * poses     device, n_views x 12 doubles.
 * targets   device, n_views x H*W float4, or NULL (no loss, w = 0).
 * image     device out, n_views x DAGS_IMG_CHANNELS x H*W floats.
 * last      device out, n_views x H*W int32: per pixel, how many entries of
 *           its tile's depth-sorted list the compositing walked up to and
 *           including its last contributor (forward state for the backward).
 * loss      device out (1 double) or NULL; the sum over views of Eq. (21),
 *           (22) weighted by lambda_pho, lambda_depth; needs targets.
 * The ctx keeps the depth-sorted tile lists and the projected Gaussians of
 * this call for splat_backward.
 * Sec. IV-D (MP-guided rendering), Eqs. (20)-(22). */
int splat_forward(dags_ctx *ctx, const float *gauss, int64_t n, const dags_camera *cam,
                  const double *poses, int32_t n_views, const float *targets,
                  const dags_raster_cfg *rcfg, const dags_loss_cfg *lcfg, float *image,
                  int32_t *last, double *loss, void *stream);

#define DAGS_GRAD_GAUSS 1u
#define DAGS_GRAD_POSE 2u

/* Backward of the loss of the preceding splat_forward on this ctx (same
 * gauss, n, cam, poses, n_views, targets, configs, image and last; the ctx
 * checks that image and last are the buffers of its latest forward and
 * returns DAGS_E_ORDER otherwise). targets must be non-NULL.
 * grad_flags   DAGS_GRAD_GAUSS and/or DAGS_GRAD_POSE.
 * grad_gauss   device out n x 16 floats (overwritten), needed with
 *              DAGS_GRAD_GAUSS, else may be NULL.
 * grad_pose    device out n_views x 6 doubles (overwritten), needed with
 *              DAGS_GRAD_POSE, else may be NULL.
 * The adjoint re-derives each pixel's transmittance backwards from its
 * final value and walks only its recorded contributors; per-Gaussian 2D
 * gradients are summed over each warp before one atomic add per Gaussian;
 * the pose gradient is reduced in a fixed order in FP64.
 * Eq. (27): joint optimisation of Gaussian parameters and camera poses. */
int splat_backward(dags_ctx *ctx, const float *gauss, int64_t n, const dags_camera *cam,
                   const double *poses, int32_t n_views, const float *targets,
                   const dags_raster_cfg *rcfg, const dags_loss_cfg *lcfg, const float *image,
                   const int32_t *last, uint32_t grad_flags, float *grad_gauss,
                   double *grad_pose, void *stream);

/* Backward of a caller's own function F of the rendered channels through
 * the preceding splat_forward on this ctx (same gauss, n, cam, poses,
 * n_views, raster config, image and last; DAGS_E_ORDER otherwise): the
 * adjoint of the compositing of Eq. (20) and of the projection, with the
 * upstream gradients given per pixel instead of formed from the loss of
 * Eqs. (21), (22). Lets a caller put its own loss on C, D, O and R_MP.
 * grad_image   device, n_views x 6 x H*W floats: dF/dC_r, dF/dC_g, dF/dC_b,
 *              dF/dD, dF/dO, dF/dR_MP planes (image planes 0-5).
 * grad_flags, grad_gauss, grad_pose   as for splat_backward (overwritten).
 * The forward's targets and loss are not used. */
int splat_backward_upstream(dags_ctx *ctx, const float *gauss, int64_t n, const dags_camera *cam,
                            const double *poses, int32_t n_views, const dags_raster_cfg *rcfg,
                            const float *image, const int32_t *last, const float *grad_image,
                            uint32_t grad_flags, float *grad_gauss, double *grad_pose, void *stream);

/* FP64 pose step for n_views poses: Adam on the twist (state per view: 13
 * doubles m[6], v[6], step, device, in/out), then pose <- exp(xi^) pose.
 * poses device in/out n_views x 12; grad device n_views x 6; cfg host.
 * Sec. V-A(c) (pose refinement) and Eq. (27). */
int pose_step(dags_ctx *ctx, double *poses, const double *grad, double *adam_state,
              int32_t n_views, const dags_pose_cfg *cfg, void *stream);

/* Allocation-free forward: splat_forward for one view with no dags_ctx. No
 * paper counterpart. It is for callers that must not allocate device memory
 * once they run (a real-time pipeline that forbids allocation after
 * start-up, a plugin whose host owns all device memory): it calls no
 * cudaMalloc, cudaFree or allocating library routine. Its workspace is one
 * file-scope device array of about 4.4 MB, shared by every call in the
 * process; every GPU that loads the library holds it until the process
 * exits. Limits: n <= 16384 Gaussians, width and height <= 256, at most
 * 131072 (tile, Gaussian) pairs; larger n, width or height return
 * DAGS_E_INVAL before any launch. The first call on a device resolves the
 * array's device address (cudaGetSymbolAddress) for that device, and so does
 * the first call after the device's primary context was reset and created
 * again (the address is cached with the context it belongs to); make those
 * calls before any stream capture. Each device that loads the library has
 * its own copy of the array. Each call clears the array's counters and
 * leaves its other contents in place; two calls on the same device whose
 * work overlaps on the GPU (different streams, or the same stream with no
 * ordering between them) race on that device's copy and must be ordered by
 * the caller; calls on different devices do not share it.
 * Arguments are those of splat_forward with n_views = 1 (pose: device, 12
 * doubles); status: device, 2 int64 or NULL. status[0] receives DAGS_OK,
 * DAGS_E_CAPACITY (more pairs than the limit; image, last and loss are then
 * undefined) or, from a DAGS_CHECK build, DAGS_E_BOUNDS (an index check
 * failed and the access was skipped); status[1] the number of pairs the call
 * needed. */
int splat_forward_static(const float *gauss, int64_t n, const dags_camera *cam, const double *pose,
                         const float *targets, const dags_raster_cfg *rcfg, const dags_loss_cfg *lcfg,
                         float *image, int32_t *last, double *loss, int64_t *status, void *stream);

/* Mapping optimiser on the Gaussian parameters (the map side of the joint
 * optimisation of Eq. (27); the paper names no optimiser): Adam (Kingma and
 * Ba) per parameter with one learning rate per group. Defaults from
 * dags_default_gauss_adam_cfg: the published 3D Gaussian splatting rates
 * (opacity 0.05, quaternion 1e-3, log-scale 5e-3, colour 2.5e-3) and 1e-3 m
 * for the means; beta 0.9 / 0.999, eps 1e-8. */
typedef struct {
  float lr_mean, lr_opacity, lr_quat, lr_scale, lr_colour;
  float beta1, beta2, eps;
} dags_gauss_adam_cfg;

void dags_default_gauss_adam_cfg(dags_gauss_adam_cfg *cfg);

/* Optimiser state of n Gaussians: colour (device, n x 4 floats) receives the
 * FP32 master colour decoded from the records' BF16 colours, and adam_m,
 * adam_v (device, n x 16 floats each, in the gradient's slot order) are
 * zeroed. Call once before the first gauss_adam_step. */
int gauss_adam_init(dags_ctx *ctx, const float *gauss, int64_t n, float *colour, float *adam_m, float *adam_v,
                    void *stream);

/* One Adam step, step number `step` >= 1 (bias corrections 1 - beta^step),
 * on the records' mean (words 0-2), opacity logit (3), quaternion (4-7) and
 * log-scale (8-10), in place in FP32, and on the FP32 master colour, which
 * is then written into the record's BF16 colour words (round to nearest,
 * ties to even). The MP word (11) is left to mp_update. grad: device, n x 16
 * floats as splat_backward writes them (colour in slots 12-14); the moments
 * are updated in place. All buffers 16-byte aligned; DAGS_E_INVAL on a
 * bad argument, a non-finite rate or beta outside [0, 1). */
int gauss_adam_step(dags_ctx *ctx, float *gauss, int64_t n, float *colour, float *adam_m, float *adam_v,
                    const float *grad, int64_t step, const dags_gauss_adam_cfg *cfg, void *stream);

/* Tracking loop: iters x { the forward with loss of splat_forward, the
 * pose-only backward of splat_backward (DAGS_GRAD_POSE), pose_step } on one
 * view, enqueued by the library -- the pose refinement of the tracking thread
 * (Sec. III) with the pose part of Eq. (27). The map is culled once at the
 * starting pose (the Gaussians that can be visible within 0.01 rad and
 * 0.01 m of it); when a pose step leaves those bounds, the next iteration
 * takes every Gaussian and culls again at its pose. Results do not depend
 * on the culling. Each iteration is four kernels:
 * projection and binning straight into per-tile buckets of max_pairs /
 * tiles slots each (no scan or emit pass), the forward with loss, which also
 * records per warp the list entries its pixels took, the pose adjoint, which
 * visits only those, and the chain to the pose twist with the FP64 pose
 * step. pose (device, 12 doubles) and adam_state (device, 13
 * doubles) are updated in place; image, last, loss and grad_pose hold the
 * last iteration's values. With use_graph != 0 (and timing off) one
 * iteration and a chunk of ten are captured once into CUDA graphs on a
 * private stream, cached in the ctx for exactly these arguments (pointers,
 * sizes, camera, configs), and replayed on `stream` (chunks, then single
 * iterations); (re)capturing synchronises `stream` first. A tile whose list
 * exceeds its bucket is reported by dags_sync_status as DAGS_E_CAPACITY with
 * the max_pairs that would hold every bucket (the longest list times the
 * tiles); the iteration's outputs are then undefined. A splat_backward or
 * dags_copy_bins after splat_track returns DAGS_E_ORDER (no forward of its
 * own precedes it). */
int splat_track(dags_ctx *ctx, const float *gauss, int64_t n, const dags_camera *cam, double *pose,
                const float *targets, const dags_raster_cfg *rcfg, const dags_loss_cfg *lcfg,
                const dags_pose_cfg *pcfg, int32_t iters, double *adam_state, float *image, int32_t *last,
                double *loss, double *grad_pose, int32_t use_graph, void *stream);

/* Spatiotemporal MP update constants (Sec. IV-A, Eq. (17)). The paper gives
 * none of their values ("unified configuration", Sec. V-A(c)); defaults
 * from dags_default_mp_cfg. */
typedef struct {
  float kappa_c;     /* m of residual per unit of L1 colour residual in e(p) (0.05)       */
  float lam;         /* lambda of e_ub = mu_e + lambda sigma_e, Eq. (4) (2)                */
  float sigma_min;   /* instance with sigma_e below this uses its mean error, m (0.005)    */
  float e_floor;     /* floor on e_ub, m (0.05)                                            */
  float sigma_g;     /* Gamma_geo = exp(-sigma / sigma_g), after Eq. (7), m (0.05)         */
  float sigma_c;     /* C = exp(-sigma_e,G / sigma_c), Eq. (11), m (0.05)                  */
  float lam_u;       /* lambda_u, Eq. (10) (1)                                             */
  float eps;         /* epsilon, Eq. (10) (1e-6)                                           */
  float alpha_min, alpha_max;  /* Eq. (11) (0.05, 0.6)                                     */
  float rho;         /* stale-prior rate factor, Eq. (17) (0.5)                            */
  float r_s;         /* association radius, Eq. (1), px (2)                                */
  float sigma_w;     /* association kernel width, px (1)                                   */
  float vis_tol;     /* observed iff z <= max rendered depth over N(G) + vis_tol, m (0.1) */
  float z_near;      /* m (0.2)                                                            */
  float tau_floor;   /* Eq. (12) (0.5)                                                     */
  int32_t fusion_mode;  /* 0 fused, 1 K = 0 (MP_ins only), 2 K = 1 (MP_geo only)           */
  int32_t scales;       /* pyramid levels S of the association, Eq. (1), 1..DAGS_MP_MAX_SCALES (1) */
} dags_mp_cfg;

void dags_default_mp_cfg(dags_mp_cfg *cfg);

#define DAGS_MP_MAX_REGIONS 256
#define DAGS_MP_MAX_SCALES 3
#define DAGS_MP_STATS_HEAD 6

/* Spatiotemporal MP update of one view (Sec. IV-A, Eqs. (1)-(12); Eq. (17)).
 * Per pixel p (the hot path's "features"): residual e(p) = |D_obs - D_rend|
 * (where D_obs > 0) + kappa_c ||C_obs - C_rend||_1; region k = inst[p]
 * (0 = background, its own region); region mean/std of e, Eq. (4) (e_ub
 * floored at e_floor; an instance with sigma_e < sigma_min uses its mean);
 * MP_geo, Eq. (5), with the region's e_ub (background pixels: the
 * background region's); MP_ins and Gamma_ins from the region table, Eq. (2);
 * Gamma_geo = exp(-sigma / sigma_g) with sigma the region's sigma_e inside an
 * instance and, for a background pixel, the population std of e over the
 * pixel's own disk {di^2 + dj^2 <= r_s^2} clipped to the image (its
 * associated neighbourhood, the sentence after Eq. (7)); fusion, Eqs. (6),(7),
 * stored per pixel in the ctx. Per Gaussian (in FP32): N(G), Eq. (1), the
 * union over pyramid levels s = 0 .. scales-1 of the level-s pixels within
 * r_s of its projected mean / 2^s, weighted 2^-s exp(-d^2 / (2 sigma_w^2))
 * (level s + 1: 2x2 box means of level s for M_p and e, 2x2 maxima for the
 * rendered depth, an odd last row or column dropped; scales = 1 is the
 * single-scale disk); observed iff z > z_near, N(G) is non-empty and
 * z <= max rendered depth over N(G) + vis_tol; M_hat, Eq. (8); U, Eq. (10), min-max normalised over the
 * observed Gaussians; alpha, Eq. (11), times rho unless seg_refreshed,
 * Eq. (17); M^t, Eq. (9), written into word 11 of each observed record.
 * Per frame: tau = max(lower median of M^t over observed, tau_floor), Eq. (12);
 * labels[i] = M^t > tau for observed Gaussians (others keep theirs);
 * U_bar = lower median of U_tilde over observed, Eq. (13).
 *
 * gauss     device in/out, n records (the MP word is updated)
 * pose      device, 12 doubles (world -> camera)
 * targets   device, H*W float4: observed r, g, b, depth (depth <= 0 invalid)
 * image     device, DAGS_IMG_CHANNELS x H*W: a splat_forward image of this
 *           view (rendered colour planes 0-2 and depth plane 3 are read)
 * inst      device, H*W uint8 region labels, each < n_regions
 * table     device, n_regions x 2 floats: (mu, c) of the region's class;
 *           row 0 = background (mu(bg), c_bg)
 * labels    device in/out, n uint8 (1 = dynamic)
 * stats     device out, DAGS_MP_STATS_HEAD + 4 * n_regions doubles: tau,
 *           U_bar, median M^t, U_min, U_max, number observed; then per region
 *           count, mean e, std e, e_ub.
 * mp_map    device, H*W floats, or NULL: an external per-pixel MP (the
 *           learned proposal between semantic invocations, not in the paper)
 *           used in place of the fused M_p in Eqs. (8) and (10); the
 *           residual terms and region statistics are the frame's own.
 * mp_pixel  device out, H*W floats, or NULL: the fused M_p of Eq. (7) per
 *           pixel (the method's own map, e.g. a training target).
 * Needs a ctx created with max_views >= 1 and images at least H x W. */
int mp_update(dags_ctx *ctx, float *gauss, int64_t n, const dags_camera *cam, const double *pose,
              const float *targets, const float *image, const uint8_t *inst, const float *table,
              int32_t n_regions, const dags_mp_cfg *cfg, int32_t seg_refreshed, uint8_t *labels,
              double *stats, const float *mp_map, float *mp_pixel, void *stream);

/* Levenberg-Marquardt pose refinement (Sec. V-A(c), which names the method
 * and gives no constants; defaults from dags_default_lm_cfg). The objective
 * is the MP-weighted L1 loss of Eqs. (20)-(22) with the static weight w(u)
 * held constant in the linearisation. Each channel residual r (r, g, b with
 * c = lambda_pho w; depth with c = lambda_depth w where the observed depth
 * is > 0) enters by iterative reweighting, W = c / max(|r|, delta):
 *   H = sum W J J^T,  g = sum W r J,  J = d(rendered channel) / d xi
 * for the left-perturbation twist xi = (rho, phi), T <- exp(xi^) T, taken at
 * the render's discrete decisions. One iteration linearises at T_try; the
 * point is accepted if its loss is below the best so far (mu <- max(mu down,
 * mu_min)), else rejected (mu <- min(mu up, mu_max)); then
 * (H_best + mu diag(H_best) + floor tr(H_best)/6 I) Delta = -g_best is solved
 * in FP64 (Delta = 0 if tr H_best <= 0 or the factorisation fails) and
 * T_try = exp(Delta^) T_best. */
typedef struct {
  double mu0;             /* initial damping (1e-2)                               */
  double mu_min, mu_max;  /* damping bounds (1e-9, 1e9)                           */
  double down, up;        /* damping factors after accept / reject (0.1, 10)      */
  double delta;           /* IRLS floor on |r|, colour units and metres (0.01)    */
  double floor;           /* ridge relative to tr(H) / 6 (1e-9)                   */
} dags_lm_cfg;

void dags_default_lm_cfg(dags_lm_cfg *cfg);

#define DAGS_LM_NORMAL 28 /* L, upper triangle of H row-major (21), g (6) */
#define DAGS_LM_STATE 48  /* T_best[12], L_best, mu, H_best[21], g_best[6], accepted, iterations,
                             last L, last accepted (0/1), unused */

/* The normal equations of one view at pose (device, 12 doubles): the
 * preprocess and binning of splat_forward, the twist tangents of every
 * visible Gaussian, and the forward-mode compositing of colour and depth.
 * normal  device out, DAGS_LM_NORMAL doubles, summed in FP64 in a fixed
 *         order (deterministic); L is NaN after a pair-capacity overflow
 * jac     device out, H*W*24 floats (per pixel: r, g, b, depth, each the 6
 *         twist components), 16-byte aligned, or NULL
 * image   device out, DAGS_IMG_CHANNELS x H*W as splat_forward, or NULL
 * last    device out, H*W int32 as splat_forward, or NULL
 * targets required (H*W float4, 16-byte aligned); delta > 0. The first LM
 * call on a ctx allocates its buffers (before any stream capture).
 * splat_backward does not follow this call (DAGS_E_ORDER). */
int splat_normal_equations(dags_ctx *ctx, const float *gauss, int64_t n, const dags_camera *cam,
                           const double *pose, const float *targets, const dags_raster_cfg *rcfg,
                           const dags_loss_cfg *lcfg, double delta, double *normal, float *jac, float *image,
                           int32_t *last, void *stream);

/* Starts an LM refinement: state (device, DAGS_LM_STATE doubles) takes
 * T_best = pose, L_best = +inf, mu = mu0; pose_try (device, 12) = pose. */
int lm_init(dags_ctx *ctx, const double *pose, const dags_lm_cfg *cfg, double *state, double *pose_try,
            void *stream);

/* One LM decision and step from the normal equations at pose_try (one FP64
 * thread): accept or reject, adapt mu, solve, write the next pose_try and
 * T_best into pose_best (device, 12 doubles). */
int lm_pose_step(dags_ctx *ctx, const double *normal, const dags_lm_cfg *cfg, double *state, double *pose_try,
                 double *pose_best, void *stream);

/* iters LM iterations of one view starting from pose (device in/out, 12
 * doubles; out: T_best): lm_init, then per iteration the normal equations
 * at the ctx's pose_try (as splat_normal_equations computes them) and the
 * step of lm_pose_step. state: device, DAGS_LM_STATE doubles. As in
 * splat_track, the map is culled once at the starting pose and the
 * iterations bin into fixed-capacity tile buckets (an iteration whose pose
 * leaves the culling bounds takes every Gaussian); a tile whose list
 * exceeds its bucket makes the iteration's loss NaN, so its point is
 * rejected, and dags_sync_status reports DAGS_E_CAPACITY with the max_pairs
 * that would hold every bucket. A splat_backward or dags_copy_bins after it
 * returns DAGS_E_ORDER. With use_graph one iteration and a chunk of ten are
 * captured once per argument set into CUDA graphs and replayed (chunks,
 * then single iterations). */
int splat_track_lm(dags_ctx *ctx, const float *gauss, int64_t n, const dags_camera *cam, double *pose,
                   const float *targets, const dags_raster_cfg *rcfg, const dags_loss_cfg *lcfg,
                   const dags_lm_cfg *lmcfg, int32_t iters, double *state, int32_t use_graph, void *stream);

/* MP-based motion-consistency regulariser (Sec. IV-D, Eqs. (23), (24)):
 *   mu_hat_k = T_rel mu_k^{t-1},  lambda L_MP = lambda sum_k (1 - M_k) |mu_k - mu_hat_k|^2
 * over all n Gaussians, M_k = the record's MP (word 11, held constant).
 * gauss      device, n records (the current means, words 0-2)
 * prev       device, n records: the snapshot after the previous mapping
 *            update (only words 0-2 are read), 16-byte aligned
 * rel_pose   device, 12 doubles [R | t] mapping the previous frame's
 *            coordinates to the current ones, or NULL: identity (a map in
 *            world coordinates, as this library keeps it)
 * lambda     the weight (the paper's lambda_3 = 500)
 * grad_gauss device, n x 16 floats, or NULL: d(lambda L_MP)/d mu is ADDED to
 *            words 0-2 (the splat_backward layout), other words untouched
 * loss       device, 1 double, or NULL: lambda L_MP, summed in a fixed
 *            order (FP32 within a warp, FP64 across warps and CTAs;
 *            deterministic)
 * The first call on a ctx allocates a small buffer (before any stream
 * capture). */
int splat_mp_consistency(dags_ctx *ctx, const float *gauss, int64_t n, const float *prev, const double *rel_pose,
                         float lambda, float *grad_gauss, double *loss, void *stream);

/* MP-guided edge-warp regulariser constants (Sec. IV-D; defaults from
 * dags_default_edge_cfg). */
typedef struct {
  float edge_rel;   /* depth step that makes an edge pixel, relative to D_i(u) (0.05) */
  float huber;      /* Huber threshold of rho, m (0.05)                           */
  float z_near;     /* warped points at or before this depth are skipped (0.2)   */
  int32_t literal;  /* 0: compare D_j(u') with the warped depth Y_z; 1: with D_i(u),
                       as Eq. (26) prints it (0)                                  */
} dags_edge_cfg;

void dags_default_edge_cfg(dags_edge_cfg *cfg);

/* Edge-warp regulariser from frame i to frame j (Sec. IV-D, Eqs. (25), (26)):
 * every pixel u of frame i with D_i(u) > 0 and a valid 4-neighbour more than
 * edge_rel D_i(u) away is back-projected with D_i(u), moved by T_ji = T_jW T_iW^-1,
 * projected to u' (Eq. (25)); D_j and w^j are sampled bilinearly over the four
 * pixels around u' (all inside the image with D_j > 0, else u is skipped) and
 *   lambda L_edge = lambda sum_u rho(w^j(u') (D_j(u') - z_ref)),
 * rho the Huber kernel, z_ref per cfg->literal (Eq. (26)). Pixel centres are
 * the integer coordinates.
 * depth_i, depth_j   device, H*W floats (observed depth, <= 0 invalid)
 * weight_j           device, H*W floats: the static weight w^j of Eq. (20),
 *                    e.g. channel 7 of frame j's splat_forward image
 * pose_i, pose_j     device, 12 doubles each (world -> camera)
 * out                device, 13 doubles: lambda L_edge, then its gradient
 *                    with respect to the left twist of pose_i (6) and of
 *                    pose_j (6); sums in a fixed order (FP32 within a
 *                    CTA, FP64 across CTAs; deterministic)
 * The first call on a ctx allocates a small buffer (before any stream
 * capture). */
int splat_edge_warp(dags_ctx *ctx, const dags_camera *cam, const float *depth_i, const float *depth_j,
                    const float *weight_j, const double *pose_i, const double *pose_j, const dags_edge_cfg *cfg,
                    float lambda, double *out, void *stream);

/* Epipolar verification and static recovery (Sec. IV-C, Eqs. (18), (19)).
 * F = K^-T [t]x R K^-1 from the camera and the relative pose (R, t) =
 * T_21 = T_2W T_1W^-1; for every match k, in FP64,
 *   d_k = |p2^T F p1| / sqrt(a^2 + b^2),  (a, b, c) = F p1       Eq. (18)
 * per Gaussian G the lower median dbar(G) of d over its matches (Eq. (19));
 * G with dbar < eps that is labelled dynamic (1) is restored: label 0 and
 * M <- min(M, m_static) (word 11 of its record). Gaussians without matches
 * are unchanged. Densification is not part of this call.
 * pose_1, pose_2  device, 12 doubles each (world -> camera)
 * p1, p2          device, m x 2 floats: pixel coordinates in frames 1, 2
 *                 (pixel i samples u = i), 8-byte aligned
 * gid             device, m int32: the Gaussian of each match; an id outside
 *                 [0, n) is skipped and reported as DAGS_E_BOUNDS at the next
 *                 dags_sync_status
 * gauss, labels   device in/out, n records and n uint8
 * eps             the paper's 1 px (> 0); m_static in [0, 1] (0.1)
 * d_out           device out, m floats, or NULL
 * dbar_out        device out, n floats (NaN where G has no match), or NULL
 * Buffers grow with m and n (allocations then, so not during a stream
 * capture). */
int epipolar_verify(dags_ctx *ctx, const dags_camera *cam, const double *pose_1, const double *pose_2,
                    const float *p1, const float *p2, const int32_t *gid, int64_t m, float *gauss, int64_t n,
                    uint8_t *labels, float eps, float m_static, float *d_out, float *dbar_out, void *stream);

/* Semantic-on-demand trigger constants (Sec. IV-B). The paper gives none of
 * their values; defaults from dags_default_sched_cfg. */
typedef struct {
  double w_u, w_r;   /* weights of U_bar and R, Eq. (15) (0.5, 0.5): >= 0, summing to 1 */
  double theta;      /* trigger threshold, Eq. (16) (0.35)                               */
  double e_ref;      /* reference residual of Eq. (14), m (0.05)                         */
  int32_t n_max;     /* maximum skip interval of Eq. (16), frames (10)                   */
} dags_sched_cfg;

void dags_default_sched_cfg(dags_sched_cfg *cfg);

/* Uncertainty-aware semantic-on-demand trigger of one frame (Sec. IV-B,
 * Eqs. (13)-(16)), enqueued after the frame's mp_update; one thread, FP64.
 *   e_bar = the frame's mean residual e(p) over the background region (label
 *           0, the pixels no instance mask claims; 0 if it is empty): the hot
 *           path's stand-in for the mean reprojection error over verified
 *           correspondences
 *   R     = clip(e_bar / e_ref, 0, 1), Eq. (14)
 *   S     = w_u U_bar + w_r R, Eq. (15), U_bar from Eq. (13)
 *   since = 0 if seg_refreshed else since + 1
 *   next  = S > theta or since + 1 >= n_max, Eq. (16): whether the NEXT frame
 *           should invoke segmentation (the score of frame t serves frame t+1)
 * stats     device, the frame's mp_update stats (U_bar at [1], region 0's
 *           count and mean residual at [DAGS_MP_STATS_HEAD] and [+1])
 * seg_refreshed  nonzero if this frame's prior was fresh
 * state     device in/out, 2 int32: [0] since (frames since the last refresh
 *           as of the previous frame; any value before a refreshed first
 *           frame), [1] out: next (0 or 1)
 * score     device out, 3 doubles (e_bar, R, S), or NULL
 * Returns DAGS_E_INVAL for a NULL ctx/stats/state, negative weights, weights
 * not summing to 1 (within 1e-6), e_ref <= 0 or n_max < 1. */
int semantic_trigger(dags_ctx *ctx, const double *stats, const dags_sched_cfg *cfg, int32_t seg_refreshed,
                     int32_t *state, double *score, void *stream);

/* Learned per-pixel MP proposal network (not in the paper: the task's
 * learned stand-in for the stale instance prior between scheduled semantic
 * invocations, Sec. IV-B). Per pixel, NHWC:
 *   z1 = W1 x + b1 (1x1, 8 -> 32), a1 = bf16(relu(z1))
 *   z2 = conv3x3(a1) + b2 (32 -> 32, zero padding), a2 = bf16(relu(z2))
 *   z3 = W3 a2 + b3 (1x1), a3 = bf16(relu(z3))
 *   y  = sigmoid(w4 . a3 + b4)
 * BF16 operands on the tensor cores (tcgen05) with FP32 accumulation.
 * Input channels: rendered MP, |dR|, |dG|, |dB|, |dDepth|, depth, rendered
 * opacity, prior mask.
 * Weight blob (device, DAGS_MPNET_WEIGHT_BYTES, 16-byte aligned), byte
 * offsets: W1 bf16 [32][16] at 0 (input channels 8-15 zero), W2 bf16
 * [32][288] at 1024 (column (ky * 3 + kx) * 32 + in), W3 bf16 [32][32] at
 * 19456, w4 bf16 [32] at 21504, b1 f32 [32] at 21568, b2 at 21696, b3 at
 * 21824, b4 f32 at 21952. */
#define DAGS_MPNET_WEIGHT_BYTES 22016
#define DAGS_MPNET_ACT_WORDS 96

/* Network input of one view (height x width pixels): per pixel 8 BF16
 * (rendered MP R_MP, |C_obs - C_rend| r g b, |D_obs - D_rend| where D_obs >
 * 0 else 0, D_obs where > 0 else 0, rendered opacity O, table[inst].mu, the
 * MP_ins of the pixel's region, Eq. (2)). image, targets, inst, table as for
 * mp_update; feats device out, 16-byte aligned, H*W*8 bf16. */
int mpnet_features(dags_ctx *ctx, const float *image, const float *targets, const uint8_t *inst,
                   const float *table, int32_t n_regions, int32_t width, int32_t height, uint16_t *feats,
                   void *stream);

/* Inference: feats device, batch x height x width x 8 bf16 (16-byte
 * aligned); mp_out device, batch x height x width float; acts device or NULL:
 * per pixel 96 bf16 (a1, a2, a3) for training. A wait that gives up records
 * DAGS_E_TIMEOUT in the status word. */
int mpnet_infer(dags_ctx *ctx, const void *weights, const uint16_t *feats, int32_t batch, int32_t width,
                int32_t height, float *mp_out, uint16_t *acts, void *stream);

/* Training step (mean binary cross-entropy over pixels whose target is
 * >= 0, then one Adam step, beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected
 * with `step` >= 1). Gradients flow through the BF16 activations as if their
 * rounding were the identity; the pixel reductions of the weight gradients
 * run on the tensor cores in BF16 with FP32 accumulation.
 * Parameter vector (FP32, DAGS_MPNET_PARAMS floats, layout of master, adam_m,
 * adam_v and grad_out): W1 [32][16] at 0, W2 [32][288] at 512, W3 [32][32]
 * at 9728, w4 [32] at 10752, b1 [32] at 10784, b2 at 10816, b3 at 10848, b4
 * at 10880 (same row/column order as the blob). master holds the FP32
 * weights; the step updates master, adam_m and adam_v in place and rewrites
 * the blob from master (weights rounded to BF16). W1's padded input
 * channels 8-15 stay zero.
 * feats as for mpnet_infer; target device float [batch][height][width],
 * negative = pixel excluded; loss device double (written: the loss at the
 * weights before the step); grad_out device float [DAGS_MPNET_PARAMS] or
 * NULL. Scratch of 2 + 2 * 96 + 2 * 32 bytes per pixel is owned by the ctx
 * and grows on demand (synchronising the stream); the call is not
 * capturable when it grows. lr >= 0. Errors: DAGS_E_INVAL for NULL or
 * unaligned buffers or bad sizes, DAGS_E_NOMEM, DAGS_E_CUDA. */
#define DAGS_MPNET_PARAMS 10881
int mpnet_train_step(dags_ctx *ctx, void *weights, float *master, float *adam_m, float *adam_v, int32_t step,
                     const uint16_t *feats, const float *target, int32_t batch, int32_t width, int32_t height,
                     float lr, double *loss, float *grad_out, void *stream);

/* Failure-path self-test (no paper counterpart): one device thread waits,
 * for `spins` bounded iterations, on an mbarrier phase that nothing
 * completes - the same bounded wait the tensor-core kernels use - and records
 * DAGS_E_TIMEOUT in the ctx's status word, which the next dags_sync_status
 * returns and clears. Nothing hangs or faults; the ctx stays usable.
 * 0 <= spins <= 2^24, else DAGS_E_INVAL. */
int dags_selftest_timeout(dags_ctx *ctx, int64_t spins, void *stream);

/* Per-kernel device timing (tracing). When enabled, every kernel the
 * library launches on a stream that is not being captured into a CUDA graph
 * is bracketed by a pair of CUDA events on that stream. dags_timing_read
 * waits for them, writes the accumulated milliseconds and launch counts per
 * kernel id (DAGS_K_*) into ms[count] and launches[count], and resets them.
 * Disabling collects and keeps the pending totals. Not for use from two
 * host threads at once. */
enum {
  DAGS_K_PREPROCESS = 0,   /* projection + tile counts + offsets           */
  DAGS_K_EMIT,             /* (depth, id) keys into per-tile buckets       */
  DAGS_K_TILE_SORT,        /* per-tile depth sort (both sort kernels)      */
  DAGS_K_RENDER_FWD,       /* forward compositing + loss                   */
  DAGS_K_RENDER_BWD,       /* adjoint compositing                          */
  DAGS_K_PREPROCESS_BWD,   /* adjoint projection + pose reduction          */
  DAGS_K_POSE_STEP,        /* FP64 pose step                               */
  DAGS_K_MP_PIXEL,         /* MP update: per-pixel observation             */
  DAGS_K_MP_GAUSS,         /* MP update: per-Gaussian update and medians   */
  DAGS_K_MPNET,            /* learned MP network, inference                */
  DAGS_K_MPNET_TRAIN,      /* learned MP network, training step            */
  DAGS_K_POSE_TANGENT,     /* LM: twist tangents of the visible Gaussians  */
  DAGS_K_RENDER_JAC,       /* LM: forward-mode compositing + normal eqs.   */
  DAGS_K_LM_STEP,          /* LM: FP64 decision, solve and pose step       */
  DAGS_K_REGULARISER,      /* L_MP and L_edge regularisers                 */
  DAGS_K_EPIPOLAR,         /* epipolar verification and static recovery    */
  DAGS_K_GAUSS_ADAM,       /* mapping: Adam step on the Gaussians          */
  DAGS_KERNEL_COUNT
};
int dags_timing_enable(dags_ctx *ctx, int enable);
int dags_timing_read(dags_ctx *ctx, double *ms, int64_t *launches, int32_t count);

/* Evaluation counts of the compositing kernels (measurement; no paper
 * counterpart). While enabled, splat_forward and splat_backward add, per
 * launch, the pixel-Gaussian exponents they evaluate (the list entries a
 * pixel's warp keeps after its box test and the pixel reaches before it
 * saturates or passes its last contributor) and the contributions among them
 * (alpha >= alpha_min). dags_eval_read waits for the ctx's last stream, writes
 * counts[4] = {forward evaluations, forward contributions, backward
 * evaluations, backward contributions} accumulated since the last read, and
 * resets them. Counting costs one warp reduction and atomic per warp and
 * launch. DAGS_E_INVAL on a NULL ctx or counts. */
int dags_eval_counting(dags_ctx *ctx, int32_t enable);
int dags_eval_read(dags_ctx *ctx, int64_t *counts);

/* Throughput probe of the current device's FP32 pipe (kind 0: fused
 * multiply-adds) or special-function pipe (kind 1: ex2.approx), for the
 * roofline peaks of the ALU-bound kernels (measurement; no paper
 * counterpart). Launches one warm-up and one timed grid of (SMs x resident
 * CTAs) x 256 threads, each running 8 independent chains of `iters` dependent
 * operations, on a private stream, and waits for it. ops_per_s (host out):
 * lane operations per second; ms (host out, or NULL): the timed launch.
 * 1 <= iters <= 2^24, kind 0 or 1, else DAGS_E_INVAL. */
int dags_measure_alu(int32_t kind, int64_t iters, double *ops_per_s, double *ms);

/* Rate probe of the current device's tensor core (measurement; no paper
 * counterpart): one CTA of `groups` warpgroups (1, 2 or 4), thread 0 of each
 * issuing `reps` back-to-back accumulating tcgen05.mma kind::f16 with M =
 * m_rows (64 or 128), N = n_cols, K = 16, BF16 operands in shared memory and FP32
 * accumulators in tensor memory, then a commit and a bounded wait; on a
 * private launch, synchronised. mac_per_cycle (host out): multiply-adds per
 * SM cycle of the slowest-to-complete average warpgroup; cycles_per_mma
 * (host out, or NULL): the mean issue cycles per MMA of one issuing thread.
 * m_rows 64 or 128, n_cols a multiple of 16 in [16, 256] with n_cols <= 512 /
 * groups and n_cols <= 128 for 4 groups, 1 <= reps <= 4096, else DAGS_E_INVAL;
 * DAGS_E_TIMEOUT if a wait ran out. */
int dags_measure_mma(int32_t m_rows, int32_t n_cols, int32_t groups, int32_t reps, double *mac_per_cycle,
                     double *cycles_per_mma);

#ifdef __cplusplus
}
#endif

#endif /* DAGS_H */
