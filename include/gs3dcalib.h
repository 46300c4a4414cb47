/*
 * gs3dcalib.h -- C ABI of libgs3dcalib.so: differentiable tile-based 3D
 * Gaussian splatting for LiDAR-camera spatiotemporal calibration
 * (3DGS-Calib, arXiv 2403.11577), hand-written CUDA for sm_103a (GB300).
 *
 * The path, in the paper's terms:
 *   pose     Eq. 1      T^n = T_L(t^n + delta_i) * L_T^i       gs_pose_compose
 *   project  Eq. 2-3    X^n = (T^n)^-1 X,  r^n = (R^n)^-1 r,
 *                       EWA projection of each Gaussian           gs_project
 *   bin/sort Eq. 5 (Phi) tile binning + depth order               gs_bin_sort
 *   render   Eq. 5 (Phi) front-to-back alpha compositing          gs_render_fwd
 *   loss     Eq. 4      L1 term of L_photo                        gs_loss_l1
 *                       L_photo = (1 - lambda1) L1 + lambda1 D-SSIM gs_loss_photo
 *   backward Sec. III-B "gradients are backpropagated to both the Gaussian
 *                       parameters, and the calibration parameters through
 *                       the input pose"                           gs_render_bwd,
 *                                                                 gs_pose_grad
 *
 * Conventions (all entry points):
 *   - Pointers named *_dev, and every tensor argument unless stated, are
 *     DEVICE pointers owned by the caller.  The library never allocates or
 *     frees device memory; scratch lives in one caller-allocated workspace
 *     of gs_workspace_size() bytes (256-byte aligned).
 *   - Every call enqueues work on `stream` (a cudaStream_t; NULL = legacy
 *     default stream) and returns without synchronising, except
 *     gs_batch_init and gs_read_stats, which are synchronous.  The hot-path
 *     calls (gs_pose_compose through gs_pose_grad) can be captured into a
 *     CUDA graph.
 *   - Layouts are row-major and contiguous; float is IEEE binary32, double
 *     binary64.  Quaternions are Hamilton (w, x, y, z).  An extrinsic is the
 *     camera-to-LiDAR transform L_T^i = [Exp(omega) | t] stored as
 *     (omega_x, omega_y, omega_z, t_x, t_y, t_z), omega a rotation vector.
 *   - Return value: GS_OK, or a host-detected error (nothing was enqueued
 *     for GS_ERR_INVALID_ARG; GS_ERR_CUDA means a launch failed).  Errors
 *     found on the device (pair-buffer overflow, non-finite values) set
 *     bits of a status word in the workspace; read it with gs_read_stats.
 *   - Per-(frame, Gaussian) "records": frame f owns records
 *     [record_offset, record_offset + gauss_count); record r of frame f is
 *     Gaussian gauss_offset + (r - record_offset).
 */
#ifndef GS3DCALIB_H
#define GS3DCALIB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t gs_status;
enum {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = 1,
    GS_ERR_CAPACITY = 2,
    GS_ERR_CUDA = 3,
    GS_ERR_UNSUPPORTED = 4
};

/* bits of the device status word */
enum {
    GS_DEV_PAIR_OVERFLOW = 1u,  /* more tile-Gaussian pairs than pair_capacity:
                                   the batch was rendered with no Gaussians */
    GS_DEV_NONFINITE = 2u       /* a Gaussian with non-finite parameters or
                                   projection was culled */
};

/* One camera frame n_i (Sec. III-A notation table). */
typedef struct {
    int32_t width, height;      /* image size in pixels */
    float fx, fy, cx, cy;       /* pinhole intrinsics; pixel (u,v) is the
                                   image point (u,v) of fx*x/z + cx */
    int32_t camera_id;          /* camera i: index into ext[] and delta[] */
    int32_t traj_id;            /* LiDAR trajectory (scene) of the frame */
    int32_t gauss_offset;       /* first Gaussian of the frame's scene */
    int32_t gauss_count;        /* Gaussians in the scene (G) */
    double timestamp;           /* t^{n_i}, seconds, camera clock */
    /* written by gs_batch_init: */
    int64_t record_offset;      /* first per-(frame, Gaussian) record */
    int64_t pixel_offset;       /* first pixel in the image outputs */
    int32_t tile_offset;        /* first global tile id */
    int32_t tiles_x, tiles_y;   /* tiles covering rows [row0, height) */
    /* input: */
    int32_t row0;               /* first image row rendered: the frame's output
                                   is rows [row0, height) of the full camera
                                   image (0 = whole image; height / 2 = the
                                   bottom half the paper's losses use,
                                   Sec. III-D).  The camera, and so every
                                   pixel's value, is unchanged by the crop. */
} gs_frame;

/* Renderer settings.  The paper defers the renderer to 3DGS
 * [kerbl20233d] and EWA [zwicker2001ewa]; these are that renderer's
 * choices, exposed as parameters. */
typedef struct {
    float near_z;     /* cull centres with camera depth <= near_z, metres
                         ("remove the points behind the camera", Sec. III-C) */
    float lowpass;    /* EWA screen-space filter variance added to the 2D
                         covariance diagonal, px^2 (0.3) */
    float alpha_min;  /* skip a Gaussian whose alpha is below this (1/255) */
    float alpha_max;  /* clamp alpha to at most this (0.99) */
    float t_min;      /* stop before transmittance would drop below (1e-4) */
    float scale_max;  /* clamp each axis scale to at most this, metres;
                         +inf = off (voxel-size bound, Sec. III-D1) */
    float bg[3];      /* background colour */
    int32_t tile;     /* tile edge in pixels: 8, 16 or 32 */
    int32_t batch;    /* Gaussians staged in shared memory per round:
                         64, 128 or 256 */
    float frustum_margin; /* the EWA Jacobian is evaluated with x/z, y/z
                         clamped to the field of view widened by this
                         fraction of the image size per side (0.15, 3DGS's
                         1.3x half field of view); negative = no clamp */
    int32_t exact_tiles; /* 1: gs_bin_sort lists a record only for the tiles
                         of its rectangle that its alpha >= alpha_min
                         ellipse can meet (row by row, with a margin), read
                         from the projection's splat records; the image is
                         the same as with whole rectangles, with fewer pairs.
                         0: whole rectangles (needs only rect and depth) */
} gs_opts;

/* A batch of frames planned by gs_batch_init. */
typedef struct {
    const gs_frame *frames_dev; /* device copy of the frame table */
    int32_t num_frames;         /* F */
    int32_t num_cameras;        /* entries of ext[] / delta[] */
    int32_t num_trajs;          /* entries of traj_offset[] minus one */
    int32_t num_gaussians;      /* rows of the Gaussian parameter arrays */
    int32_t tile;               /* tile edge the plan was made for */
    int32_t num_tiles;          /* total tiles over all frames */
    int64_t num_records;        /* total per-(frame, Gaussian) records */
    int64_t num_pixels;         /* total pixels over all frames */
    int64_t pair_capacity;      /* tile-Gaussian pairs the workspace holds */
} gs_batch;

/* Counters kept in the workspace (gs_read_stats). */
typedef struct {
    uint32_t status;            /* GS_DEV_* bits, sticky until gs_reset_status */
    uint32_t reserved;
    uint64_t num_pairs;         /* tile-Gaussian pairs of the last gs_bin_sort */
    uint64_t eval_fwd;          /* composited (pixel, Gaussian) pairs, last gs_render_fwd */
    uint64_t eval_bwd;          /* composited (pixel, Gaussian) pairs, last gs_render_bwd */
} gs_stats;

/* ------------------------------------------------------------ planning -- */

/* Version string of the library. */
const char *gs_version(void);

/* sizeof(gs_frame), sizeof(gs_opts), sizeof(gs_batch), sizeof(gs_stats)
 * written to out[0..n) so that bindings can check their struct mirrors.
 * Returns the number of sizes written. */
int32_t gs_struct_sizes(size_t *out, int32_t n);

/* Plan a batch (host, synchronous).  frames_host[F] is read and its
 * gs_batch_init-written fields are filled; the completed table is copied
 * to frames_dev (caller-allocated device memory of F * sizeof(gs_frame)
 * bytes) with cudaMemcpy.  tile must be 8, 16 or 32.  Frames are checked:
 * positive sizes, 0 <= row0 < height, camera_id < num_cameras, traj_id <
 * num_trajs, Gaussian range inside [0, num_gaussians), tiles_x and tiles_y
 * < 65536.  A frame contributes width * (height - row0) pixels.
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA (copy failed). */
gs_status gs_batch_init(gs_frame *frames_host, int32_t num_frames, int32_t num_gaussians,
                        int32_t num_cameras, int32_t num_trajs, int32_t tile,
                        int64_t pair_capacity, gs_frame *frames_dev, gs_batch *out);

/* Workspace bytes needed by a batch (host).  0 on invalid input. */
size_t gs_workspace_size(const gs_batch *batch);

/* Byte offsets of the workspace regions (host), for tests and tools that
 * read intermediate buffers:  [0] stats, [1] pose32 (float[F][32]: R_cw
 * row-major 9 (high parts), camera centre hi 3, camera centre lo 3, pad,
 * R_cw row-major 9 (low parts: R_cw - high part, rounded), pad 7), [2] pose64
 * (double[F][32]), [3] rect (uint32[R][2]: x0 | y0 << 16, x1 | y1 << 16,
 * inclusive tile coordinates, empty as x0 > x1), [4] depth (float[R];
 * +inf for a record with an empty rectangle),
 * [5] splat (float4[R][2]: (mean_x, mean_y, A, B), (C, F, rx, ry), the
 * base-2 exponent log2 alpha = A dx^2 + B dx dy + C dy^2 + F and the
 * half-widths of the box outside which alpha < alpha_min), [6] grad2d
 * (float4[R][3]: d/d(mean_x, mean_y, A, B), d/d(C, F, r, g), d/d(b)), [7] keys
 * (uint32[pair_capacity]: the global tile of each sorted pair), [8] vals
 * (uint32[pair_capacity]: Gaussian index within its scene), [9] ranges
 * (uint32[T][2]: [start, end) of each tile in keys/vals).  Returns the
 * number of offsets written (<= max_entries). */
int32_t gs_workspace_offsets(const gs_batch *batch, size_t *offsets, int32_t max_entries);

/* Read the counters (synchronises `stream`). */
gs_status gs_read_stats(const gs_batch *batch, const void *ws_dev, void *stream, gs_stats *out);

/* Clear the device status bits (async). */
gs_status gs_reset_status(const gs_batch *batch, void *ws_dev, void *stream);

/* kernels selectable by gs_profile_events */
enum {
    GS_PROF_NONE = 0,
    GS_PROF_PROJECT = 1,
    GS_PROF_BIN_SORT = 2,
    GS_PROF_RENDER_FWD = 3,
    GS_PROF_RENDER_BWD = 4,
    GS_PROF_PROJECT_BWD = 5,
    GS_PROF_LOSS = 6
};
/* Kernel timing hook.  After this call, every launch of the selected
 * kernel is bracketed by records of the start/stop events on the kernel's
 * own stream; while the stream is being captured into a CUDA graph they are
 * recorded with cudaEventRecordExternal, so they become event-record nodes
 * that fire on every replay.
 * kernel: GS_PROF_NONE (0) disables the hook; GS_PROF_PROJECT,
 * GS_PROF_BIN_SORT (the whole binning and sorting sequence),
 * GS_PROF_RENDER_FWD, GS_PROF_RENDER_BWD (the compositing backward only),
 * GS_PROF_PROJECT_BWD, GS_PROF_LOSS (gs_loss_l1 or gs_loss_photo).  The
 * events are cudaEvent_t handles owned by the
 * caller (created with timing enabled).  Process-wide setting; not thread
 * safe.  Errors: GS_ERR_INVALID_ARG for an unknown kernel or NULL events. */
gs_status gs_profile_events(int32_t kernel, void *start_event, void *stop_event);

/* ----------------------------------------------------------- hot path -- */

/* Eq. 1 (Sec. III-A): camera pose of every frame.  The LiDAR trajectory
 * T_L(t) interpolates keyframes linearly in position and by SLERP in
 * orientation; the segment [t_k, t_{k+1}) holding tau = t^{n_i} + delta_i is
 * used (the end segments extend linearly beyond the keyframes).
 *   traj_t[K]        keyframe times (double), increasing within a trajectory
 *   traj_pose[K][7]  keyframe LiDAR-to-world pose (p_x,p_y,p_z, q_w,q_x,q_y,q_z)
 *   traj_offset[num_trajs+1]  trajectory j owns keyframes
 *                    [traj_offset[j], traj_offset[j+1]) (int32, >= 1 each)
 *   ext[C][6]        camera-to-LiDAR extrinsic per camera (double)
 *   delta[C]         time offset per camera, seconds (double)
 * Writes the world-to-camera pose of each frame (and the camera-frame
 * velocity twist used by the time-offset gradient) to the workspace. */
gs_status gs_pose_compose(const gs_batch *batch, const double *traj_t, const double *traj_pose,
                          const int32_t *traj_offset, const double *ext, const double *delta,
                          void *ws_dev, void *stream);

/* Eq. 2-3 and the EWA projection of Phi (Eq. 5): for every (frame,
 * Gaussian) record, the camera-frame centre X^n = (T^n)^-1 X, the
 * camera-frame covariance R^n^-1 Sigma R^n^-T, the 2D mean, the conic
 * (inverse of J Sigma_c J^T + lowpass I), the opacity, and the rectangle of
 * tiles where alpha can reach alpha_min.  The camera-frame centre is formed
 * in float-float arithmetic, and the depth and the 2D mean are rounded once:
 * the depth is the float nearest to the exact depth, the depth order's key.
 * Gaussians with that depth <= near_z or opacity < alpha_min are culled
 * (empty rectangle, and depth +inf, so that gs_bin_sort drops the record).
 *   X[N][3]        centres, world frame (float; fixed LiDAR points, Sec. III-B)
 *   quat[N][4]     rotation r, any non-zero norm (normalised inside)
 *   log_scale[N][3] s = exp(log_scale), clamped to scale_max
 *   logit_opacity[N] alpha = sigmoid(logit_opacity)
 * Reads the poses written by gs_pose_compose. */
gs_status gs_project(const gs_batch *batch, const float *X, const float *quat,
                     const float *log_scale, const float *logit_opacity, const gs_opts *opts,
                     void *ws_dev, void *stream);

/* Tile binning and depth ordering for Phi (Eq. 5).  Each record emits one
 * pair per tile it can reach, value = Gaussian index within its scene:
 *   opts->exact_tiles != 0 (the default): only the tiles of its rectangle
 *     that its alpha >= alpha_min ellipse can meet (in each tile row, a run
 *     between the ellipse's x-extremes, tested with a margin above float32
 *     rounding, so the rendered image is the same as with whole rectangles);
 *   opts->exact_tiles == 0: every tile of its rectangle.
 * The pairs end up in the order of the key (global tile << 32) | float bits
 * of the depth, equal keys in record order (a stable sort), and each tile's
 * [start, end) range is found, plus a heavy-first order of the tiles for
 * the render.  The workspace keys region holds each sorted pair's global
 * tile (the high half of that key).  It reads the rect, depth and splat
 * regions that gs_project wrote; a record of depth +inf is dropped before
 * the sort (gs_project writes +inf for every culled record), and a record
 * with an empty rectangle emits no pair.  If the pairs exceed pair_capacity,
 * GS_DEV_PAIR_OVERFLOW is set and the batch is treated as having no pairs. */
gs_status gs_bin_sort(const gs_batch *batch, const gs_opts *opts, void *ws_dev, void *stream);

/* Phi (Eq. 5): front-to-back alpha compositing per pixel over its tile's
 * depth-ordered Gaussians: alpha = min(alpha_max, opacity * exp(power)),
 * power = -1/2 d^T conic d, skip alpha < alpha_min, stop before T would fall
 * below t_min; C = sum c alpha T + T_final bg.
 *   colors[N][3]      view-independent colour c (float, used as is)
 *   out_rgb[P][3]     rendered colour, P = num_pixels, frame f at
 *                     pixel_offset, row-major (float)
 *   out_T[P]          final transmittance (float)
 *   out_last[P]       one past the position, within the tile's sorted
 *                     range, of the last composited Gaussian; 0 if none
 *                     (int32) -- the backward's starting point
 * It also leaves in the workspace, per band of pixels and per 32 entries of
 * the tile's list, a mask of the entries some pixel of the band composited,
 * which gs_render_bwd walks. */
gs_status gs_render_fwd(const gs_batch *batch, const float *colors, const gs_opts *opts,
                        void *ws_dev, float *out_rgb, float *out_T, int32_t *out_last,
                        void *stream);

/* L1 term of L_photo (Eq. 4): loss = mean |rgb - target| over n values and
 * grad = sign(rgb - target) / n (0 where equal) * scale.
 *   out_loss[1] (double) is overwritten; grad may alias nothing.
 *   ws_dev: a workspace of this batch (uses its reduction scratch). */
gs_status gs_loss_l1(const gs_batch *batch, const float *rgb, const float *target, int64_t n,
                     float scale, double *out_loss, float *out_grad, void *ws_dev, void *stream);

/* The photometric loss of Eq. 4 over the batch's images:
 *   L_photo = (1 - lambda1) L1 + lambda1 D-SSIM    (lambda1 = 0.2 in the paper)
 * L1 = mean |rgb - target| and D-SSIM = 1 - mean SSIM, both over all
 * 3 * num_pixels values.  SSIM per channel and pixel with the 11x11
 * Gaussian window of sigma 1.5, zero padding at each frame's image border
 * (a cropped frame's image is its rows [row0, height): the paper's losses
 * use the bottom half, Sec. III-D) and C1 = 0.01^2, C2 = 0.03^2, as in
 * [kerbl20233d].
 *   rgb, target[num_pixels][3]  frame f at pixel_offset, row-major
 *   lambda1 in [0, 1]
 *   out_loss[3] (device double, overwritten): L_photo, L1, D-SSIM
 *   out_grad[num_pixels][3] (optional): scale * dL_photo/drgb, overwritten
 *   ws_dev: the batch's workspace (its SSIM maps and partial sums).
 * The loss is reduced in a fixed order (deterministic).
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
gs_status gs_loss_photo(const gs_batch *batch, const float *rgb, const float *target, float lambda1,
                        float scale, double *out_loss, float *out_grad, void *ws_dev, void *stream);

/* Backward of Phi and of the projection (Sec. III-B): walks each pixel's
 * composited Gaussians in reverse order, recovering transmittance by
 * division instead of storing it, reduces per-pixel gradients warp-first,
 * accumulates per-record 2D gradients, then carries them through the EWA
 * projection and Eq. 2-3 to the Gaussian parameters and to a per-frame
 * camera twist (kept in the workspace for gs_pose_grad).
 *   dL_drgb[P][3]  gradient of the loss w.r.t. out_rgb
 *   out_T, out_last: as written by gs_render_fwd for the same inputs (the
 *                  masks that call left in the workspace are read too: the
 *                  pair list must still be the one it rendered)
 *   d_quat[N][4], d_log_scale[N][3], d_logit_opacity[N], d_colors[N][3]:
 *                  gradients of all N Gaussians; added to the arrays if
 *                  accumulate != 0, written over them if accumulate == 0.
 * gs_project zeroes the per-record accumulators this call consumes, so each
 * gs_render_bwd needs its own preceding gs_project. */
gs_status gs_render_bwd(const gs_batch *batch, const float *X, const float *quat,
                        const float *log_scale, const float *logit_opacity, const float *colors,
                        const gs_opts *opts, void *ws_dev, const float *out_T,
                        const int32_t *out_last, const float *dL_drgb, float *d_quat,
                        float *d_log_scale, float *d_logit_opacity, float *d_colors,
                        int32_t accumulate, void *stream);

/* Gradient w.r.t. the calibration parameters "through the input pose"
 * (Sec. III-B, Eq. 1): sums the per-frame camera twists of gs_render_bwd
 * per camera and maps them to
 *   d_ext[C][6]   dL/d(omega, t) of the extrinsic (double)
 *   d_delta[C]    dL/d delta (double)
 *   d_xi[C][6]    optional (NULL to skip): dL/dxi for the right
 *                 perturbation L_T^i <- L_T^i Exp(xi), xi = (rho, phi)
 *   ext[C][6]     the extrinsic used by gs_pose_compose
 *   accumulate    0: outputs are written; otherwise added to. */
gs_status gs_pose_grad(const gs_batch *batch, const double *ext, void *ws_dev, double *d_ext,
                       double *d_delta, double *d_xi, int32_t accumulate, void *stream);

/* ------------------------------------------- hash-grid attribute model -- */

/* The attribute model F(X | Theta) of Sec. III-C: the Instant-NGP
 * multiresolution hash encoding of a Gaussian's centre, then an MLP
 * 2L -> 64 -> 64 -> 11 (ReLU after the hidden layers) whose four heads give
 * the renderer's inputs: rgb = sigmoid(o0..2), logit_opacity = o3,
 * log_scale = o4..6, quat = o7..10.
 * Encoding: 2 features per level; a point maps to p in [0, 1]^3 (clamped)
 * through the box; at level l, q = p * res[l], cell c = min(floor(q),
 * res[l] - 1), trilinear interpolation of the cell's 8 vertices.  A vertex
 * v indexes the level's table densely (x + y (res+1) + z (res+1)^2) when the
 * (res+1)^3 vertices fit in T = 2^log2_table entries, otherwise by the
 * spatial hash (x * 1 ^ y * 2654435761 ^ z * 805459861) mod 2^32 mod T.
 * theta (float, device): the tables [levels][T][2], then W1 [64][2 levels],
 * b1 [64], W2 [64][64], b2 [64], W3 [11][64], b3 [11]; 8-byte aligned. */
typedef struct {
    float aabb_min[3], aabb_max[3];  /* box mapped to [0, 1]^3 */
    int32_t levels;                  /* L, 1..16 */
    int32_t log2_table;              /* 4..26 */
    int32_t res[16];                 /* per-level grid resolution, 1..2^20 */
} gs_ngp;

/* Number of floats of theta; -1 for an invalid configuration (host). */
int64_t gs_ngp_param_count(const gs_ngp *cfg);

/* Attributes of n points X[n][3]: rgb[n][3], logit_opacity[n],
 * log_scale[n][3], quat[n][4] (device float, overwritten).
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
gs_status gs_ngp_forward(const gs_ngp *cfg, const float *theta, const float *X, int64_t n, float *rgb,
                         float *logit_opacity, float *log_scale, float *quat, void *stream);

/* Backward of sum(d_attr . F(X | theta)): adds the gradient with respect to
 * theta into d_theta (the caller zeroes it first; table entries are summed
 * with atomics, so their float rounding order varies between runs).
 * theta must be 8-byte and d_theta 16-byte aligned (the table gradient is
 * added with float2 and float4 atomics).
 * Errors: GS_ERR_INVALID_ARG (also for misaligned pointers), GS_ERR_CUDA. */
gs_status gs_ngp_backward(const gs_ngp *cfg, const float *theta, const float *X, int64_t n, const float *d_rgb,
                          const float *d_logit_opacity, const float *d_log_scale, const float *d_quat,
                          float *d_theta, void *stream);

/* Reads and clears the fault word of the hash-grid kernels on the current
 * device (host; waits for the device).  Bit 0: a tensor-core wait of
 * gs_ngp_forward or gs_ngp_backward ran out of time (one second), so that
 * call's outputs are incomplete; the backward then also adds NaN to
 * d_theta[0].  Errors: GS_ERR_INVALID_ARG (NULL out), GS_ERR_CUDA. */
gs_status gs_ngp_fault(uint32_t *out);

/* Sets the bound on the hash-grid kernels' waits for their tensor-core MMAs,
 * in ns, for every later call on the current device (host; default one
 * second, the value to restore).  0 makes a wait give up as soon as one
 * non-blocking test finds the MMAs unfinished, which lets a test drive the
 * timeout path (gs_ngp_fault then reports bit 0).  After a timeout the
 * kernels still wait, for at most one second whatever this bound, for the
 * MMAs in flight before they release tensor memory.  The paper has no
 * counterpart: it bounds the waits of this implementation.
 * Errors: GS_ERR_CUDA. */
gs_status gs_ngp_set_wait_limit(uint64_t ns);

/* Accumulated-LiDAR downsampling (Sec. III-D): keep one point per occupied
 * voxel of edge `voxel`, the point of smallest index.  A point's voxel is
 * (floor(x / voxel), floor(y / voxel), floor(z / voxel)) with the quotients
 * in float32 (IEEE division).  Points with a non-finite coordinate or a voxel
 * coordinate outside (-2^20, 2^20) are dropped.  With one point per voxel,
 * the paper also bounds the Gaussians' scales by the voxel size
 * (gs_opts.scale_max).
 *   X[n][3] (device float)     points
 *   out_index[n] (device int32) receives the kept indices in ascending
 *                              order (the first out_count[0] entries)
 *   out_count[1] (device uint64) number of kept points
 *   scratch_dev: gs_voxel_scratch_size(n) bytes of device memory, 256-byte
 *                aligned, owned by the caller (no state kept between calls)
 * Errors: GS_ERR_INVALID_ARG (n < 0 or n >= 2^31, voxel not finite or <= 0,
 * NULL or misaligned pointers), GS_ERR_CUDA. */
size_t gs_voxel_scratch_size(int64_t n);
gs_status gs_voxel_downsample(const float *X, int64_t n, float voxel, int32_t *out_index, uint64_t *out_count,
                              void *scratch_dev, void *stream);

/* ------------------------------------------------- no allocation at all -- */

/* The tile binning and depth sort of gs_bin_sort for callers that cannot
 * allocate device memory: for instance a host framework that owns every
 * device buffer and hands a plugin only its inputs and outputs, or a
 * real-time loop where an allocation's latency or failure is not
 * acceptable.  Such a caller cannot provide the workspace gs_bin_sort needs.
 * The paper has no counterpart; it is a deployment convenience.
 *
 * It bins whole rectangles (the caller passes rect and depth, not the
 * splat records): opts->exact_tiles must be 0, else GS_ERR_UNSUPPORTED.
 * vals and ranges are the same as gs_bin_sort's, bit for bit, and keys are
 * the full 64-bit keys (global tile << 32 | float bits of the depth) whose
 * high halves are gs_bin_sort's workspace keys; the inputs and outputs are
 * the caller's buffers instead of workspace regions:
 *   rect[R][2]   uint32 rectangles (x0 | y0 << 16, x1 | y1 << 16, inclusive
 *                tiles; empty when x0 > x1), R = batch->num_records,
 *                8-byte aligned.  A non-empty rectangle must lie within its
 *                frame: x1 < tiles_x and y1 < tiles_y (tile rows counted
 *                from the frame's row0).  If any does not, nothing is
 *                written: out_pairs = {0, UINT64_MAX} and ranges are zero.
 *   depth[R]     float camera depths (the key's low 32 bits), 4-byte aligned
 *   keys[pair_capacity] (8-byte aligned), vals[pair_capacity] (4-byte
 *                aligned)  sorted pairs (output)
 *   ranges[num_tiles][2]  [start, end) of each tile (output), 8-byte aligned
 *   out_pairs[2] (device, uint64, 8-byte aligned): pairs written and pairs
 *                requested; if the request exceeds batch->pair_capacity
 *                nothing is written, out_pairs[0] = 0 and ranges are zero.
 * A misaligned pointer returns GS_ERR_INVALID_ARG without enqueuing anything.
 * Scratch: one fixed array of 12,878,912 bytes (12.9 MB, 12.3 MiB) compiled
 * into the library (every GPU that loads the library holds it until the
 * process exits), sized for at most 2^20 pairs (batch->pair_capacity) and
 * 2^22 records; larger batches return GS_ERR_CAPACITY without enqueuing
 * anything.  No cudaMalloc,
 * cudaFree or allocating library routine is called.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one array and it keeps
 * the last call's contents: calls that overlap on the GPU (different
 * streams, or different host threads) race and corrupt each other.
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_UNSUPPORTED, GS_ERR_CAPACITY, GS_ERR_CUDA. */
gs_status gs_bin_sort_noalloc(const gs_batch *batch, const gs_opts *opts, const uint32_t *rect,
                              const float *depth, uint64_t *keys, uint32_t *vals, uint32_t *ranges,
                              uint64_t *out_pairs, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GS3DCALIB_H */
