/*
 * vt.h - pyramidal Lucas-Kanade (KLT) feature tracking on one GB300 GPU.
 *
 * The operation: the LK optical-flow front-end of DL-VINS-Factory tracks
 * keypoints from the previous frame to the current one and, in stereo, from
 * the left to the right image, keeping only features that pass a
 * cross-camera optical-flow check (Sec. IV: Shi-Tomasi corners with LK
 * optical flow as the classical front-end; Sec. III-A: LK tracking needs
 * keypoints only, so any extractor's keypoints P in R^{N x 2} of Eq. 1 can
 * feed it; Table I: the KLT tracker inherited from VINS-Fusion; Sec. V-A:
 * stereo features enter the temporal pool only after the cross-camera flow
 * check).  The paper fixes none of the tracker's constants; the readings this
 * library implements are stated beside each call.
 *
 * Conventions for every call:
 *   - Plain C ABI: pointers and sizes only.  "device" pointers are CUDA
 *     global-memory addresses valid on the current device; "host" pointers
 *     are ordinary (preferably pinned) host memory.
 *   - cuda_stream is a cudaStream_t (NULL = legacy default stream).  Every
 *     call is asynchronous on that stream unless stated otherwise; results
 *     are visible after the stream is synchronised.
 *   - Images are 8-bit grey, row-major, `pitch` bytes between rows.
 *   - Points are float2 (x, y) in level-0 pixels; pixel centres sit at
 *     integer coordinates.
 *   - Errors are returned, never thrown: VT_ERR_ARG for a bad argument
 *     (nothing is launched), VT_ERR_OOM when device memory runs out,
 *     VT_ERR_CUDA when a CUDA call or launch fails (the stream may hold
 *     partial work).  Per-point failures are reported in `status`.
 *   - Ownership: the caller owns every point / status / error buffer; the
 *     library owns pyramids (vt_pyramid_free releases them).
 */
#ifndef VT_H
#define VT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define VT_API __attribute__((visibility("default")))
#else
#define VT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum vt_status {
    VT_OK = 0,
    VT_ERR_ARG = 1,
    VT_ERR_OOM = 2,
    VT_ERR_CUDA = 3,
    VT_ERR_TIMEOUT = 4,
    VT_ERR_UNSUPPORTED = 5
} vt_status;

/* Gradient storage of a pyramid. */
typedef enum vt_grad_type {
    VT_GRAD_NONE = 0,
    VT_GRAD_S16 = 1, /* raw Scharr as int16 pairs (dx, dy), range [-4080, 4080] */
    VT_GRAD_F16 = 2  /* raw / 32 as half pairs, round to nearest even */
} vt_grad_type;

/* Per-point reason codes (optional diagnostics). */
enum {
    VT_TRACKED = 0,
    VT_LOST_EIG = 1,   /* lambda_min(G) below threshold, or det(G) <= 0 */
    VT_LOST_OOB = 2,   /* estimate left the image (see vt_klt_track) */
    VT_LOST_FB = 3,    /* forward-backward distance above threshold */
    VT_LOST_INPUT = 4, /* input point outside [0, W-1] x [0, H-1] or NaN; for
                          vt_stereo_gate: pair not tracked or not finite */
    VT_LOST_DISP = 5,  /* stereo gate: negligible disparity */
    VT_LOST_DEPTH = 6, /* stereo gate: depth outside the valid range (or behind a camera) */
    VT_LOST_REPROJ = 7 /* stereo gate: reprojection error above the bound in a view */
};

enum { VT_MAX_LEVELS = 8 };      /* levels per pyramid */
#define VT_DEFAULT_MIN_EIG 1e-4f /* threshold on lambda_min(G) / (win^2 * 255^2) */

/* Window sides the tracking kernels are built for. */
#define VT_SUPPORTED_WINDOWS {9, 15, 21, 31}

typedef struct vt_pyramid vt_pyramid; /* opaque, device-resident, owned by the library */

/*
 * vt_pyramid_build - Gaussian image pyramid (the coarse-to-fine pyramid of
 * the LK tracker, Sec. IV; its filter is unstated in the paper).
 *
 * Level 0 is a copy of `img` (w x h, `pitch` bytes per row; a host pointer
 * when img_on_device == 0, else a device pointer).  Level l+1 has size
 * ceil(w_l / 2) x ceil(h_l / 2) and is the 5x5 separable [1 4 6 4 1]^2 / 256
 * sum centred at (2x, 2y) of level l, reflect-101 borders (clamp on a 1-px
 * side), rounded as (s + 128) >> 8: bit-exact integer arithmetic.
 *
 * levels: 1..VT_MAX_LEVELS (ceil-halving keeps every level >= 1x1; 1-px levels
 * repeat).  VT_ERR_ARG for w, h <= 0, pitch < w or levels out of range.
 * *out == NULL: a new pyramid is allocated (one cudaMalloc) and returned.
 * *out != NULL: it must have been built with the same w, h and levels; it is
 *   rebuilt in place without allocating (VT_ERR_ARG on a mismatch).
 * Gradients of a rebuilt pyramid are stale until vt_gradients is called.
 */
VT_API vt_status vt_pyramid_build(const uint8_t *img, int w, int h, int pitch, int levels, int img_on_device,
                           void *cuda_stream, vt_pyramid **out);

/*
 * vt_gradients - Scharr derivatives of every level of `p`:
 *   dx = [-3 0 3; -10 0 10; -3 0 3] * I,  dy = its transpose,
 * reflect-101 borders, stored as (dx, dy) pairs per pixel: raw int16
 * (VT_GRAD_S16, bit-exact) or raw / 32 rounded to half (VT_GRAD_F16).
 * raw / 32 is the derivative in grey levels per pixel.
 */
VT_API vt_status vt_gradients(vt_pyramid *p, vt_grad_type t, void *cuda_stream);

/*
 * vt_pyramid_build_grad - vt_pyramid_build followed by vt_gradients in one
 * pass over each level (level l's gradients are computed from the same
 * staged tile that produces level l+1).  Same arguments and results.
 */
VT_API vt_status vt_pyramid_build_grad(const uint8_t *img, int w, int h, int pitch, int levels, int img_on_device,
                                vt_grad_type t, void *cuda_stream, vt_pyramid **out);

/*
 * vt_pyramid_create - allocate (one cudaMalloc) an empty pyramid for w x h
 * images with `levels` levels, for use as a vt_batch build target.  Same
 * argument rules as vt_pyramid_build.  Synchronous.
 */
VT_API vt_status vt_pyramid_create(int w, int h, int levels, vt_pyramid **out);

/*
 * vt_pyramid_create_on - like vt_pyramid_create, but level 0 of the pyramid
 * is the caller's device buffer `level0` (h rows of `pitch` bytes, row y at
 * level0 + y * pitch) instead of library memory: a frame that lands there
 * (a camera or host upload, one slot of an input ring) is level 0 as it is,
 * and a build or batched run that names `level0` as its image builds the
 * upper levels and the Scharr planes from it without copying it
 * (Sec. IV: the pyramids are built from the incoming frames).
 *
 * Ownership: the buffer stays the caller's; the library never frees it
 * (vt_pyramid_free releases only the levels above 0 and the planes).  The
 * caller keeps it allocated, and leaves it unchanged while queued builds or
 * tracking calls read it.  A build from another image, or vt_pyramid_upload,
 * writes that image into the caller's buffer.
 *
 * Layout rules (VT_ERR_ARG otherwise): level0 16-byte aligned, pitch a
 * multiple of 16 and >= w, and level0_bytes >= pitch * h + 32: the tracking
 * kernels stage windows in whole aligned 16-byte chunks, which may read up
 * to 31 bytes past a row's last pixel (contents unused).  Other arguments as
 * vt_pyramid_create.  Synchronous.
 */
VT_API vt_status vt_pyramid_create_on(const uint8_t *level0, int pitch, size_t level0_bytes, int w, int h,
                                      int levels, vt_pyramid **out);

/*
 * vt_pyramid_upload - copy a w x h frame (`pitch` bytes per row; host memory,
 * pinned for an asynchronous copy, or device memory with img_on_device = 1)
 * into level 0 of `p` on `cuda_stream` (one 2-D memory copy, no kernel), so
 * that a later build names level 0 itself as its image and copies nothing.
 * The caller must not upload into a pyramid that queued work still reads.
 * VT_ERR_ARG for a null pointer or pitch < w; VT_ERR_CUDA if the copy fails
 * to start.
 */
VT_API vt_status vt_pyramid_upload(vt_pyramid *p, const uint8_t *img, int pitch, int img_on_device,
                                   void *cuda_stream);

/* Level `lvl` of `p`: device image pointer, size and pitch (bytes). */
VT_API vt_status vt_pyramid_level(const vt_pyramid *p, int lvl, const uint8_t **ptr, int *w, int *h, int *pitch);

/* Gradient plane of level `lvl`: device pointer to (dx, dy) pairs, pitch in
 * pairs, storage type (VT_GRAD_NONE before vt_gradients). */
VT_API vt_status vt_pyramid_grad(const vt_pyramid *p, int lvl, const void **ptr, int *pitch_pairs, vt_grad_type *t);

/* Shape of `p`. */
VT_API vt_status vt_pyramid_info(const vt_pyramid *p, int *w, int *h, int *levels, size_t *device_bytes);

/* Frees `p` (synchronises the device first; NULL is ignored). */
VT_API void vt_pyramid_free(vt_pyramid *p);

/*
 * vt_klt_track - pyramidal Lucas-Kanade from `prev` to `cur` (the
 * prev->cur temporal tracking of the LK front-end; with prev = left and
 * cur = right it is the cross-camera flow of Sec. V-A).
 *
 * Both pyramids need gradients (vt_gradients).  For each point u (float2,
 * device, n entries), levels l = levels-1 .. 0, u_l = u / 2^l, window
 * offsets x in [-h, h]^2 with h = win / 2:
 *   T(x) = I_l(u_l + x) and grad T(x) bilinearly sampled (replicate-clamped
 *   neighbours) from prev's level l image and gradient planes;
 *   G = sum grad T grad T^T; the point is lost if lambda_min(G) / (win^2 255^2)
 *   < min_eig (VT_DEFAULT_MIN_EIG here) or det(G) <= 0;
 *   nu = 0; up to max_iters times: q = u_l + g_l + nu must lie in
 *   [-h, w_l - 1 + h] x [-h, h_l - 1 + h] (else lost), r(x) = T(x) - J_l(q + x),
 *   b = sum r grad T, eta = G^-1 b, nu += eta, stop when |eta|^2 < eps^2;
 *   g_{l-1} = 2 (g_l + nu); g_{levels-1} = 0, or (guess - u) / 2^(levels-1)
 *   when pts_guess (device, nullable) is given.
 * The result v = u + g_0 + nu must lie in [0, W-1] x [0, H-1] (else lost).
 * Outputs (device, caller-owned, n entries): pts_out = v (for a lost point:
 * its last estimate, scaled to level 0), status = 1 tracked / 0 lost,
 * err = mean |T(x) - J_0(v + x)| over the window (0 when lost; nullable).
 * G, b and the residual are accumulated in FP32; det(G) and the adjugate
 * products of the 2x2 solve are evaluated in FP32 with Kahan's FMA scheme
 * (relative error <= 2 ulp, sign exact), so no FP64 is used.
 * win: one of VT_SUPPORTED_WINDOWS.  levels: 1..min(prev, cur levels).
 * max_iters >= 1, eps >= 0.  n == 0 launches nothing.
 */
VT_API vt_status vt_klt_track(const vt_pyramid *prev, const vt_pyramid *cur, const float *pts_in, int n,
                       const float *pts_guess, int win, int levels, int max_iters, float eps, float *pts_out,
                       uint8_t *status, float *err, void *cuda_stream);

/* Tracking parameters for the _ex / _fb / batched calls. */
typedef struct vt_klt_params {
    int win;       /* one of VT_SUPPORTED_WINDOWS */
    int levels;    /* levels used */
    int max_iters; /* Newton iterations per level, >= 1 */
    float eps;     /* stop when |eta| < eps (level pixels) */
    float min_eig; /* threshold on lambda_min(G) / (win^2 255^2) */
    float fb_thr;  /* forward-backward threshold in level-0 pixels (fused calls) */
} vt_klt_params;

/* Optional per-point diagnostics (device arrays of n entries, each nullable). */
typedef struct vt_klt_diag {
    uint8_t *reason; /* VT_TRACKED / VT_LOST_* */
    int32_t *iters;  /* Newton iterations summed over levels (and over both
                        passes in the fused forward-backward calls) */
    float *lmin;     /* normalised lambda_min of G at the last level examined
                        (forward pass) */
    int32_t *flops;  /* algorithmic FLOPs spent on the point: win^2 x (27 per
                        template sweep + 12 per Newton iteration + 9 per error
                        sweep), both passes in the fused calls */
    int32_t *sweeps; /* footprint sweeps the Newton iterations executed (an
                        iteration whose integer cell is unchanged reuses the
                        previous sweep's moments) */
} vt_klt_diag;

/* vt_klt_track with an explicit parameter block and diagnostics (diag nullable). */
VT_API vt_status vt_klt_track_ex(const vt_pyramid *prev, const vt_pyramid *cur, const float *pts_in, int n,
                          const float *pts_guess, const vt_klt_params *prm, float *pts_out, uint8_t *status,
                          float *err, const vt_klt_diag *diag, void *cuda_stream);

/*
 * vt_fb_check - forward-backward consistency (the cross-camera / temporal
 * flow check of Sec. V-A): status_out[i] = st_f[i] && st_b[i] &&
 * |p0[i] - p0_back[i]|_2 <= thr (inclusive).  All arrays device, n entries.
 */
VT_API vt_status vt_fb_check(const float *p0, const float *p0_back, const uint8_t *st_f, const uint8_t *st_b, int n,
                      float thr, uint8_t *status_out, void *cuda_stream);

/*
 * vt_klt_track_fb - forward track prev->cur, backward track cur->prev from
 * the forward result, and vt_fb_check with prm->fb_thr, fused in one launch
 * (one warp carries a point through both passes).  pts_out / err are the
 * forward results; status is the forward-backward status; diag->reason
 * gives the first failure (forward, then backward, then VT_LOST_FB).
 * Identical to vt_klt_track_ex + vt_klt_track_ex + vt_fb_check.
 */
VT_API vt_status vt_klt_track_fb(const vt_pyramid *prev, const vt_pyramid *cur, const float *pts_in, int n,
                          const vt_klt_params *prm, float *pts_out, uint8_t *status, float *err,
                          const vt_klt_diag *diag, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Shi-Tomasi (GFTT) corner detection on a pyramid level: the classical
 * detector the paper pairs with LK tracking (Sec. IV; CPU-based in the paper,
 * Sec. V-F).  It reuses the level's int16 Scharr gradients (VT_GRAD_S16).
 *   score(x)  lambda_min of [a b; b c], a, b, c the (2 block_radius + 1)^2 box
 *             sums of gx^2, gx gy, gy^2 (raw Scharr, reflect-101 borders),
 *             evaluated in single precision as
 *             ((a + c) - sqrt((a - c)^2 + 4 b^2)) / 2, clamped at 0;
 *   candidate score >= quality * (maximum score of the level) and > 0, at
 *             least `border` px from every edge, the maximum of its
 *             (2 nms_radius + 1)^2 neighbourhood (a tie goes to the smaller
 *             row-major index), squared distance >= min_dist^2 to every mask
 *             point (e.g. points already tracked);
 *   selection in order of score (descending, then index ascending), keep a
 *             candidate when no kept corner is closer than min_dist; at most
 *             max_corners.
 * Corners (float2, integer coordinates of the level) and scores come out in
 * that order; *count_out (a device int) receives how many.
 * ---------------------------------------------------------------------- */
typedef struct vt_gftt_params {
    int max_corners;  /* 0 .. 8192 (vt_gftt_detect; per job in vt_gftt_detect_many) */
    float quality;    /* relative threshold, e.g. 0.01 */
    int min_dist;     /* >= 1 px */
    int nms_radius;   /* 0 .. 8 */
    int block_radius; /* 0 .. 3 (1 = 3x3 block) */
    int border;       /* >= 0 px */
} vt_gftt_params;

typedef struct vt_gftt vt_gftt; /* opaque: workspace for levels up to max_w x max_h */

/* Allocates the workspace (score map, candidate keys) for one level of at
 * most max_w x max_h pixels. */
VT_API vt_status vt_gftt_create(int max_w, int max_h, vt_gftt **out);

/* Workspace for vt_gftt_detect_many: the levels of one call may hold up to
 * max_pixels pixels together (about 50 bytes of device memory per pixel). */
VT_API vt_status vt_gftt_create_pixels(long long max_pixels, vt_gftt **out);

/* Detect corners on level `level` of `p`.  mask_pts: device float2[n_mask]
 * (nullable when n_mask == 0).  corners_out: device float2[max_corners];
 * scores_out: device float[max_corners] (nullable); count_out: device int.
 * Calls on one vt_gftt must be serialised (they share its workspace). */
VT_API vt_status vt_gftt_detect(vt_gftt *g, const vt_pyramid *p, int level, const vt_gftt_params *prm,
                                const float *mask_pts, int n_mask, float *corners_out, float *scores_out,
                                int *count_out, void *cuda_stream);

/* Many frames in one sequence of launches (every kernel covers every
 * frame): one job per level, each with its own mask and outputs, the
 * detector parameters of `prm` (its max_corners is ignored: per job).
 * At most 64 jobs; VT_ERR_ARG when the levels' pixels exceed the workspace. */
typedef struct vt_gftt_job {
    const vt_pyramid *pyr; /* VT_GRAD_S16 gradients */
    int level;
    const float *mask_pts; /* device float2[n_mask], nullable when n_mask == 0 */
    int n_mask;
    float *corners_out; /* device float2[max_corners] */
    float *scores_out;  /* device float[max_corners], nullable */
    int *count_out;     /* device int */
    int max_corners;    /* 0 .. 8192 */
} vt_gftt_job;

VT_API vt_status vt_gftt_detect_many(vt_gftt *g, const vt_gftt_job *jobs, int njobs, const vt_gftt_params *prm,
                                     void *cuda_stream);

/* Frees the workspace (synchronises the device first; NULL is ignored). */
VT_API void vt_gftt_free(vt_gftt *g);

/* ------------------------------------------------------------------------
 * Stereo triangulation gate: the geometric check of stereo correspondences
 * (Sec. III-C: matches with negligible disparity are dropped; the others are
 * triangulated with the rig's extrinsics and kept only when the point has a
 * positive depth inside a valid range and reprojects to within 1.5 px of the
 * observation in both views).  Applied here to the left->right LK
 * correspondences, one per point, after the cross-camera flow check.
 * Reading (the paper fixes only the 1.5 px), evaluated in FP64:
 *   disparity |p_R - pi_R(R K_L^-1 (p_L, 1))|: distance in the right image
 *             from the image of the left ray's point at infinity (infinite
 *             when that point is behind the right camera); kept when
 *             > min_disp, else VT_LOST_DISP;
 *   point     linear (DLT) two-view triangulation on normalised coordinates
 *             with P_L = [I | 0], P_R = [R | t]: the unit X minimising
 *             |A X|, A's rows x P^3 - P^1 and y P^3 - P^2 of each view;
 *   depth     X_4 != 0, Z_R > 0 and z_min <= Z_L <= z_max, else
 *             VT_LOST_DEPTH;
 *   reprojection  |pi_L(X) - p_L| <= max_reproj and |pi_R(R X + t) - p_R| <=
 *             max_reproj (pixels, each view), else VT_LOST_REPROJ.
 * An untracked (status_in == 0) or non-finite pair is VT_LOST_INPUT.
 * ---------------------------------------------------------------------- */
typedef struct vt_stereo_rig {
    double kl[4]; /* left pinhole fx, fy, cx, cy (px); observations undistorted */
    double kr[4]; /* right pinhole fx, fy, cx, cy (px) */
    double R[9];  /* row-major rotation, left-camera to right-camera coordinates */
    double t[3];  /* translation in metres: X_R = R X_L + t */
} vt_stereo_rig;

typedef struct vt_gate_params {
    double min_disp;   /* px, >= 0: kept when disparity > min_disp */
    double z_min;      /* m: kept when z_min <= Z_L ... */
    double z_max;      /* ... <= z_max (z_min <= z_max; z_max may be +inf) */
    double max_reproj; /* px, >= 0: 1.5 in the paper */
} vt_gate_params;

/* pts_l, pts_r: device float2[n] (left observation, right observation);
 * status_in: device uint8[n], nullable (all tracked); xyz_out: device
 * float[3 n], nullable: the triangulated point in the left-camera frame when
 * triangulation ran (0 for VT_LOST_INPUT / VT_LOST_DISP or X_4 == 0);
 * status_out: device uint8[n], 1 kept / 0 rejected (may alias status_in);
 * reason_out: device uint8[n], nullable.  rig and prm are host pointers read
 * during the call.  VT_ERR_ARG for n < 0, a missing array, non-finite rig
 * values, a zero focal length or out-of-range parameters. */
VT_API vt_status vt_stereo_gate(const float *pts_l, const float *pts_r, const uint8_t *status_in, int n,
                                const vt_stereo_rig *rig, const vt_gate_params *prm, float *xyz_out,
                                uint8_t *status_out, uint8_t *reason_out, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Track bookkeeping on the device: identity carry-over, thinning and
 * spawning of new tracks for many camera streams at once (one CTA per
 * stream; counts stay on the device, so a step needs no host round trip).
 * The paper describes the identity rules for its matching front-end
 * (Sec. III-C: first-frame detections all start tracks; associated features
 * keep their identities, unassociated detections start new ones) and the
 * LK front-end's pool (Sec. V-A: in stereo only features passing the
 * cross-camera flow check enter it; in mono it carries itself over), with a
 * feature cap (Sec. IV: 256).  Reading implemented (VINS-Fusion's tracker):
 *   carry  features whose temporal track succeeded keep identity, take the
 *          tracked position and age + 1; in order of age (descending, ties:
 *          smaller previous index first) a survivor is kept when no kept
 *          survivor lies at squared distance < min_dist^2 (FP32,
 *          dx*dx + dy*dy); kept survivors rewrite the pool in that order;
 *   spawn  accepted detections, in their (detector priority) order, fill
 *          the pool up to `cap` with identities next_id, next_id + 1, ...
 *          and age 1.
 * ---------------------------------------------------------------------- */
enum { VT_POOL_MAX = 4096 }; /* features per pool */

typedef struct vt_track_pool {
    float *pts;    /* device float2[cap] */
    int32_t *ids;  /* device int32[cap] */
    int32_t *ages; /* device int32[cap]: frames the feature has been tracked in */
    int *count;    /* device int: live features (first *count entries) */
    int *next_id;  /* device int: the stream's next unused identity */
    int cap;       /* 1 .. VT_POOL_MAX */
} vt_track_pool;

typedef struct vt_carry_job {
    vt_track_pool pool;     /* rewritten in place */
    const float *tracked;   /* device float2[>= *count]: temporal result for the pool's points */
    const uint8_t *status;  /* device uint8[>= *count]: 1 = tracked (forward-backward checked) */
    float *mask;            /* device float2[cap], nullable: kept positions, padded with NaN to cap
                               (a vt_gftt_detect mask with n_mask = cap) */
} vt_carry_job;

/* At most 192 jobs per call, one per pool; min_dist > 0 px.  VT_ERR_ARG for
 * a missing array or a cap outside 1..VT_POOL_MAX. */
VT_API vt_status vt_tracks_carry(const vt_carry_job *jobs, int njobs, float min_dist, void *cuda_stream);

typedef struct vt_spawn_job {
    vt_track_pool pool;
    const float *corners;   /* device float2[*n_corners], in priority order */
    const int *n_corners;   /* device int */
    const uint8_t *accept;  /* device uint8[*n_corners], nullable (all accepted) */
} vt_spawn_job;

/* At most 192 jobs per call; the pool grows by min(accepted, cap - count). */
VT_API vt_status vt_tracks_spawn(const vt_spawn_job *jobs, int njobs, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Batched tracking: the frames and tracking tasks of many independent camera
 * streams in one fixed sequence of persistent launches (one per pyramid
 * level, one for the last levels' gradients, one for every tracking task),
 * replayable as a CUDA graph.  Results equal those of the single-pair calls
 * (vt_pyramid_build_grad, vt_klt_track_ex / vt_klt_track_fb) on the same
 * inputs; a point's result does not depend on the rest of the batch.
 * ---------------------------------------------------------------------- */

/* Build pyramid `pyr` (levels and gradients) from the device image `img`
 * (the pyramid's w x h, `pitch` bytes per row, any alignment; pinned host
 * memory also works -- the kernels then read it over the host link, which is
 * slower than copying it first).  `img` may be the pyramid's own level 0
 * (vt_pyramid_level(pyr, 0, ...), with that level's pitch; VT_ERR_ARG with
 * another pitch), for instance after vt_pyramid_upload: the frame is then
 * built in place and level 0 is not copied. */
typedef struct vt_frame_job {
    const uint8_t *img;
    int pitch;
    vt_pyramid *pyr;
} vt_frame_job;

/* Track n points (device float2) from `prev` to `cur`; fb = 1 runs the
 * forward-backward variant (vt_klt_track_fb semantics).  Outputs are device
 * arrays of n entries; err, reason and flops are nullable.  A pyramid built
 * in the same run may serve as prev or cur.  levels: pyramid levels used by
 * this task (0 = the run's vt_klt_params.levels). */
typedef struct vt_track_task {
    const vt_pyramid *prev;
    const vt_pyramid *cur;
    const float *pts_in;
    int n;
    int fb;
    float *pts_out;
    uint8_t *status;
    float *err;
    uint8_t *reason;
    int32_t *flops;
    int levels;
    const int *n_dev; /* device int, nullable: only the first min(n, *n_dev) points are
                         tracked (the rest of the outputs is left untouched), so a count
                         that lives on the device (a vt_track_pool's) needs no host copy */
} vt_track_task;

typedef struct vt_batch vt_batch; /* opaque: pinned + device job tables, work counter, graphs */

/* Capacity: at most max_frames pyramid builds and max_tasks tasks per run.
 * Allocates two pinned and two device table buffers (a few tens of KB). */
VT_API vt_status vt_batch_create(int max_frames, int max_tasks, vt_batch **out);

/* Frees the batch (synchronises the device first; NULL is ignored). */
VT_API void vt_batch_free(vt_batch *b);

/*
 * Launch shape of the persistent KLT kernel: warps per CTA (4 or 8) and CTAs
 * per SM (0 = as many as fit); CTAs of the pyramid launches (0 = SMs x
 * resident CTAs).  Takes effect at the next vt_batch_set.
 */
VT_API vt_status vt_batch_config(vt_batch *b, int klt_warps_per_cta, int klt_ctas_per_sm, int pyr_ctas);

/*
 * Stage the next run: `nframes` pyramid builds with gradient type `gtype`
 * (S16 or F16) and `ntasks` tracking tasks with parameters `prm` (the window
 * and gradient type are per run).  Host-only: copies the descriptors into a
 * pinned staging buffer (two alternate, so a run may still execute while
 * the next is staged; staging waits for the run that last used the buffer).
 * Tasks of one run see the pyramids as they are after this run's builds.
 */
VT_API vt_status vt_batch_set(vt_batch *b, const vt_frame_job *frames, int nframes, vt_grad_type gtype,
                              const vt_track_task *tasks, int ntasks, const vt_klt_params *prm);

/* One stereo-gate task of a batched run (vt_stereo_gate semantics): pairs
 * (pts_l[i], pts_r[i]) of one rig.  The arrays may be outputs of the same
 * run's tracking tasks (e.g. pts_r = a left->right task's pts_out and
 * status_in its status): the gate runs after the tracking launch. */
typedef struct vt_gate_task {
    const float *pts_l;       /* device float2[n] */
    const float *pts_r;       /* device float2[n] */
    const uint8_t *status_in; /* device uint8[n], nullable */
    int n;
    vt_stereo_rig rig;   /* copied into the staged tables */
    float *xyz;          /* device float[3 n], nullable */
    uint8_t *status_out; /* device uint8[n] (may alias status_in) */
    uint8_t *reason;     /* device uint8[n], nullable */
} vt_gate_task;

/*
 * Add stereo-gate tasks to the run staged by the last vt_batch_set (before it
 * is run; VT_ERR_ARG otherwise).  They run as one more launch after the
 * tracking launch, one thread per pair, with parameters `prm` (host pointer,
 * copied).  At most max_tasks gate tasks.  A vt_batch_set without this call
 * stages a run without gates.
 */
VT_API vt_status vt_batch_set_gates(vt_batch *b, const vt_gate_task *gates, int ngates, const vt_gate_params *prm);

/* Run the staged batch with direct launches on `cuda_stream`.  Runs of one
 * batch must be issued on one stream (or otherwise serialised). */
VT_API vt_status vt_batch_run(vt_batch *b, void *cuda_stream);

/* Same as vt_batch_run through a CUDA graph: captured (on an internal stream)
 * the first time a staging buffer is run with a given topology (deepest
 * pyramid, gradient type, window, launch shape, stereo gate, FP64 pass), then
 * replayed; each staging buffer keeps the graphs of up to 8 topologies. */
VT_API vt_status vt_batch_run_graph(vt_batch *b, void *cuda_stream);

/* vt_batch_run that also records the (nullable) CUDA events `ev_pyr0` /
 * `ev_pyr1` around the pyramid launches and `ev_klt0` / `ev_klt1` around the
 * tracking launch, for live per-kernel timing. */
VT_API vt_status vt_batch_run_timed(vt_batch *b, void *cuda_stream, void *ev_pyr0, void *ev_pyr1, void *ev_klt0,
                                    void *ev_klt1);

/* vt_batch_run_timed that also records one event after each pyramid launch:
 * events[0..3] as ev_pyr0, ev_pyr1, ev_klt0, ev_klt1 of vt_batch_run_timed,
 * events[4 + i] after pyramid launch i (the tiled launches of levels 0, 1,
 * .., then the tail launch).  `nevents` must be at least 4 + the staged
 * run's pyramid launches (launches_per_run of vt_batch_info minus the
 * tracking and gate launches); VT_ERR_ARG otherwise.  Null entries are
 * skipped. */
VT_API vt_status vt_batch_run_levels_timed(vt_batch *b, void *cuda_stream, void **events, int nevents);

/* Launch shape of the staged run and the number of kernel launches per run. */
VT_API vt_status vt_batch_info(const vt_batch *b, int *klt_grid_ctas, int *klt_warps_per_cta, int *pyr_grid_ctas,
                               int *launches_per_run);

/*
 * vt_klt_track_tasks_noalloc - the batched tracking launch for callers that
 * cannot allocate device memory when they call: real-time loops that must
 * not wait on the allocator or on the device-wide synchronisation cudaFree
 * may cause, and hosts (frameworks, plug-in hosts) that hand out all device
 * memory from their own pools and forbid allocation by the code they call.
 * The paper has no counterpart; it is an addition of this library.
 *
 * Tracks `ntasks` tasks (vt_track_task, pyramids already built, one gradient
 * type, `prm` as for vt_batch_set) in one persistent launch, like the
 * tracking launch of vt_batch_run, with the same results.  Nothing is
 * allocated: the job table and the work counter live in a fixed array of
 * 24,064 bytes in device memory that every device loading the library keeps
 * until the process exits.  The table is handed to a small fill kernel as
 * its launch parameter (a snapshot taken by the launch; no host buffer has
 * to outlive the call), which writes it into the array and zeroes the
 * counter; the tracking launch follows on the same stream.  Limit: at most
 * 256 tasks per call (VT_ERR_ARG beyond; any number of points per task up
 * to 2^31 in total).
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it.  Every call shares the array and
 * overwrites it, so calls that overlap on the GPU - on different streams
 * without ordering, or from different threads - race; serialise them.
 */
VT_API vt_status vt_klt_track_tasks_noalloc(const vt_track_task *tasks, int ntasks, const vt_klt_params *prm,
                                            void *cuda_stream);

/*
 * vt_fp32_fma_probe - measurement helper, not part of the method: one launch
 * of (SMs x 8) CTAs of 256 threads, each thread running 8 independent FP32
 * FMA chains of 8 x `iters` FMAs, on `cuda_stream`.  Timing it with CUDA
 * events gives this device's FP32 FMA throughput at its current clocks, the
 * denominator of the tracking kernel's roofline.  `out`: device float array
 * of at least SMs x 2048 entries (`out_floats` entries), overwritten with one
 * value per thread; `*flops` (host) receives the launch's FLOP count
 * (2 per FMA).  VT_ERR_ARG for iters < 1, null pointers or a short array.
 */
VT_API vt_status vt_fp32_fma_probe(int iters, float *out, long long out_floats, long long *flops,
                                   void *cuda_stream);

/*
 * vt_copy_async - issue `n` memory copies on `cuda_stream`, in order, one
 * cudaMemcpyAsync each (kind inferred from the addresses: device memory and
 * pinned host memory); a request loop's per-request uploads and downloads
 * in one call instead of one host-language call per copy.  Part of the
 * serving runtime, not of the method.  Entries with bytes == 0 are skipped.
 * VT_ERR_ARG for a null table or pointer, VT_ERR_CUDA if a copy fails to
 * start (the copies before it stay queued).
 */
typedef struct vt_copy {
    void *dst;
    const void *src;
    size_t bytes;
} vt_copy;

VT_API vt_status vt_copy_async(const vt_copy *copies, int n, void *cuda_stream);

/* Human-readable name of a status code. */
VT_API const char *vt_status_str(vt_status s);

/* Library version string and the device architecture it was built for. */
VT_API const char *vt_version(void);

#ifdef __cplusplus
}
#endif

#endif /* VT_H */
