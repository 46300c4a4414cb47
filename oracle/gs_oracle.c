/*
 * gs_oracle.c -- plain, slow FP64 CPU oracle for the 3DGS-Calib splatting
 * path (arXiv 2403.11577).  TEST INFRASTRUCTURE ONLY: it exists to check the
 * CUDA path and must never be called by the product path.  It shares no
 * code, header or constant table with the CUDA library.
 *
 * What it computes, in the paper's order:
 *   Sec. III-A, Eq. 1  camera pose  T^n = T_L(t^n + delta) * L_T_i, with the
 *                      LiDAR trajectory interpolated linearly in position and
 *                      by SLERP in orientation between keyframes.
 *   Sec. III-B, Eq. 2  X^n = (T^n)^-1 X   (Gaussian centres, camera frame)
 *   Sec. III-B, Eq. 3  r^n = (R^n)^-1 r   (Gaussian orientation, camera frame)
 *   Sec. III-B, Eq. 5  Phi: EWA splatting [zwicker2001ewa] -- each 3D
 *                      Gaussian becomes a 2D Gaussian through the Jacobian of
 *                      the pinhole map plus a screen-space low-pass filter,
 *                      and the 2D Gaussians are alpha-composited front to
 *                      back in depth order.
 *   Sec. III-B         backpropagation to the Gaussian parameters and, through
 *                      the input pose, to the extrinsic and the time offset.
 *   Sec. III-B, Eq. 4  the photometric loss: its L1 part, and the D-SSIM
 *                      part with the structural similarity of [kerbl20233d]
 *                      (11x11 Gaussian window, sigma 1.5, zero padding).
 *
 * There is no tiling: every requested pixel is composited over every visible
 * Gaussian in one global (depth, index) order.  The renderer details the
 * paper leaves open (activations, low-pass, thresholds, pixel centres,
 * tie-breaking) are parameters; see or_opts.
 *
 * Everything is double precision; float32 inputs are widened exactly by the
 * Python wrapper before the call.
 * Build: gcc -O2 -shared -fPIC -ffp-contract=off (see oracle/build.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- types -- */

typedef struct {
    double near_z;     /* cull centres with camera depth <= near_z (Sec. III-C) */
    double lowpass;    /* EWA screen-space filter variance, px^2 */
    double alpha_min;  /* a Gaussian with alpha below this is skipped */
    double alpha_max;  /* alpha is clamped to at most this */
    double t_min;      /* compositing stops before T would drop below this */
    double scale_max;  /* axis scales are clamped to at most this */
    double bg[3];      /* background colour */
    double frustum_margin; /* the EWA Jacobian is evaluated with x/z, y/z clamped to
                              the image's field of view widened by this fraction of
                              the image size on each side (3DGS uses 1.3x the half
                              field of view, i.e. 0.15); negative = no clamp */
} or_opts;

typedef struct {
    int width, height;
    double fx, fy, cx, cy;
} or_cam;

/* Per-pixel flags.  The renderer takes its discrete decisions (skip,
 * stop, clamp, order) on float32 values; the oracle decides in FP64 and
 * bounds how far the float32 evaluation can lie from the exact value (see
 * "float32 decision bounds" below).  A decision whose exact value lies
 * within that bound of its threshold is ambiguous: both outcomes are
 * correct results of the method in float32.
 *   OR_FLAG_BRANCH       an ambiguous skip (alpha_min, exponent > 0) or stop
 *                        (t_min) decision: every outcome is rendered as an
 *                        alternative result (or_render's out_alt); the
 *                        pixel's gradient depends on the outcome.
 *   OR_FLAG_CLAMP_EDGE   a composited Gaussian's alpha lies within the bound
 *                        of alpha_max: the colour is continuous there, its
 *                        gradient is not.
 *   OR_FLAG_DEPTH_TIE    two consecutive contributors whose order is not
 *                        decided: one of them has an exact depth within the
 *                        bound of a float32 rounding boundary, and its other
 *                        candidate key would put the pair out of (key,
 *                        index) order.
 *   OR_FLAG_NEAR_EDGE    a Gaussian whose float32 depth key is not decided
 *                        at the near plane would contribute.
 *   OR_FLAG_BRANCH_LIMIT more than OR_MAX_BRANCHES outcomes. */
enum {
    OR_FLAG_BRANCH = 1,
    OR_FLAG_CLAMP_EDGE = 2,
    OR_FLAG_DEPTH_TIE = 4,
    OR_FLAG_NEAR_EDGE = 16,
    OR_FLAG_BRANCH_LIMIT = 32,
};

#define OR_MAX_BRANCHES 16  /* outcomes per pixel: the FP64 one and up to 15 alternatives */
#define OR_MAX_DECISIONS 48 /* ambiguous decisions per pass that can be enumerated */

/* ------------------------------------------------------ 3x3 linear algebra */

static void m3_mul(const double *A, const double *B, double *C) {
    double T[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++) s += A[3 * i + k] * B[3 * k + j];
            T[3 * i + j] = s;
        }
    memcpy(C, T, sizeof T);
}

static void m3_transpose(const double *A, double *B) {
    double T[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) T[3 * i + j] = A[3 * j + i];
    memcpy(B, T, sizeof T);
}

static void m3_vec(const double *A, const double *v, double *o) {
    double t[3];
    for (int i = 0; i < 3; i++) t[i] = A[3 * i] * v[0] + A[3 * i + 1] * v[1] + A[3 * i + 2] * v[2];
    memcpy(o, t, sizeof t);
}

static void m3_tvec(const double *A, const double *v, double *o) { /* A^T v */
    double t[3];
    for (int i = 0; i < 3; i++) t[i] = A[i] * v[0] + A[3 + i] * v[1] + A[6 + i] * v[2];
    memcpy(o, t, sizeof t);
}

static double m3_dot(const double *A, const double *B) { /* sum_ij A_ij B_ij */
    double s = 0.0;
    for (int i = 0; i < 9; i++) s += A[i] * B[i];
    return s;
}

static void skew(const double *w, double *K) {
    K[0] = 0; K[1] = -w[2]; K[2] = w[1];
    K[3] = w[2]; K[4] = 0; K[5] = -w[0];
    K[6] = -w[1]; K[7] = w[0]; K[8] = 0;
}

static void cross(const double *a, const double *b, double *c) {
    double t[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
    memcpy(c, t, sizeof t);
}

/* ----------------------------------------------------------- rotations -- */

/* Rotation matrix of a unit Hamilton quaternion (w, x, y, z). */
static void quat_to_rot(const double *q, double *R) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Directional derivative of quat_to_rot at q along dq. */
static void quat_to_rot_dir(const double *q, const double *dq, double *dR) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double dw = dq[0], dx = dq[1], dy = dq[2], dz = dq[3];
    dR[0] = -4 * (y * dy + z * dz);
    dR[1] = 2 * (x * dy + y * dx - w * dz - z * dw);
    dR[2] = 2 * (x * dz + z * dx + w * dy + y * dw);
    dR[3] = 2 * (x * dy + y * dx + w * dz + z * dw);
    dR[4] = -4 * (x * dx + z * dz);
    dR[5] = 2 * (y * dz + z * dy - w * dx - x * dw);
    dR[6] = 2 * (x * dz + z * dx - w * dy - y * dw);
    dR[7] = 2 * (y * dz + z * dy + w * dx + x * dw);
    dR[8] = -4 * (x * dx + y * dy);
}

/* Rodrigues' formula R = exp([w]x). */
static void rodrigues(const double *w, double *R) {
    double th = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    double K[9], K2[9];
    if (th < 1e-12) {
        skew(w, K);
        for (int i = 0; i < 9; i++) R[i] = (i % 4 == 0 ? 1.0 : 0.0) + K[i];
        return;
    }
    double u[3] = {w[0] / th, w[1] / th, w[2] / th};
    skew(u, K);
    m3_mul(K, K, K2);
    for (int i = 0; i < 9; i++) R[i] = (i % 4 == 0 ? 1.0 : 0.0) + sin(th) * K[i] + (1 - cos(th)) * K2[i];
}

/* dR/dw_k for R = exp([w]x), by the compact formula of Gallego and Yezzi
 * (J. Math. Imaging Vis. 2015):  dR/dw_k = (w_k [w]x + [w x ((I-R) e_k)]x) R / |w|^2,
 * which tends to [e_k]x as w -> 0. */
static void rodrigues_grad(const double *w, const double *R, double dR[3][9]) {
    double n2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    for (int k = 0; k < 3; k++) {
        double e[3] = {0, 0, 0}, A[9];
        e[k] = 1.0;
        if (n2 < 1e-16) {
            skew(e, A);
            memcpy(dR[k], A, sizeof A);
            continue;
        }
        double ImRe[3] = {e[0] - R[k], e[1] - R[3 + k], e[2] - R[6 + k]}; /* (I - R) e_k */
        double c[3], W[9], C[9];
        cross(w, ImRe, c);
        skew(w, W);
        skew(c, C);
        for (int i = 0; i < 9; i++) A[i] = (w[k] * W[i] + C[i]) / n2;
        m3_mul(A, R, dR[k]);
    }
}

/* SLERP between unit quaternions q0 and q1 at s in [0,1] (shortest arc),
 * with its derivative d q / d s [shoemake1985animating]. */
static void slerp(const double *q0, const double *q1in, double s, double *q, double *dq) {
    double q1[4];
    double d = q0[0] * q1in[0] + q0[1] * q1in[1] + q0[2] * q1in[2] + q0[3] * q1in[3];
    double sg = d < 0 ? -1.0 : 1.0;
    for (int i = 0; i < 4; i++) q1[i] = sg * q1in[i];
    d = fabs(d);
    if (d > 1.0) d = 1.0;
    double th = acos(d);
    if (th < 1e-9) {
        for (int i = 0; i < 4; i++) {
            q[i] = (1 - s) * q0[i] + s * q1[i];
            dq[i] = q1[i] - q0[i];
        }
        return;
    }
    double st = sin(th);
    for (int i = 0; i < 4; i++) {
        q[i] = (sin((1 - s) * th) * q0[i] + sin(s * th) * q1[i]) / st;
        dq[i] = th * (-cos((1 - s) * th) * q0[i] + cos(s * th) * q1[i]) / st;
    }
}

/* ------------------------------------------------------ trajectory (Eq.1) */

/* LiDAR-to-world pose T_L(tau): the segment [t_k, t_{k+1}) holding tau
 * (right-continuous; the end segments are extended linearly outside the
 * keyframes), lerp for the position and SLERP for the orientation (Sec.
 * III-A).  Also returns d/dtau of both. */
void or_lidar_pose(const double *traj_t, const double *traj_p, const double *traj_q, int K,
                   double tau, double *R_wL, double *p_wL, double *dR_dtau, double *dp_dtau) {
    if (K == 1) {
        double qn[4], n = 0;
        for (int i = 0; i < 4; i++) n += traj_q[i] * traj_q[i];
        n = sqrt(n);
        for (int i = 0; i < 4; i++) qn[i] = traj_q[i] / n;
        quat_to_rot(qn, R_wL);
        for (int i = 0; i < 3; i++) { p_wL[i] = traj_p[i]; dp_dtau[i] = 0; }
        for (int i = 0; i < 9; i++) dR_dtau[i] = 0;
        return;
    }
    int k = 0;
    while (k + 1 < K - 1 && traj_t[k + 1] <= tau) k++;
    double dt = traj_t[k + 1] - traj_t[k];
    double s = (tau - traj_t[k]) / dt;
    const double *p0 = traj_p + 3 * k, *p1 = traj_p + 3 * (k + 1);
    for (int i = 0; i < 3; i++) {
        p_wL[i] = (1 - s) * p0[i] + s * p1[i];
        dp_dtau[i] = (p1[i] - p0[i]) / dt;
    }
    double qa[4], qb[4], na = 0, nb = 0;
    for (int i = 0; i < 4; i++) { na += traj_q[4 * k + i] * traj_q[4 * k + i]; nb += traj_q[4 * k + 4 + i] * traj_q[4 * k + 4 + i]; }
    for (int i = 0; i < 4; i++) { qa[i] = traj_q[4 * k + i] / sqrt(na); qb[i] = traj_q[4 * k + 4 + i] / sqrt(nb); }
    double q[4], dq[4];
    slerp(qa, qb, s, q, dq);
    quat_to_rot(q, R_wL);
    quat_to_rot_dir(q, dq, dR_dtau);
    for (int i = 0; i < 9; i++) dR_dtau[i] /= dt;
}

/* World-to-camera transform of frame n (inverse of Eq. 1):
 * T^n = T_L(t + delta) * [R_e | t_e], R_e = exp([omega]x);  X^n = (T^n)^-1 X (Eq. 2). */
void or_frame_pose(const double *traj_t, const double *traj_p, const double *traj_q, int K,
                   const double *ext, double delta, double t_frame, double *R_cw, double *t_cw) {
    double R_wL[9], p_wL[3], dR[9], dp[3], R_e[9], R_wc[9], t_wc[3];
    or_lidar_pose(traj_t, traj_p, traj_q, K, t_frame + delta, R_wL, p_wL, dR, dp);
    rodrigues(ext, R_e);
    m3_mul(R_wL, R_e, R_wc);
    m3_vec(R_wL, ext + 3, t_wc);
    for (int i = 0; i < 3; i++) t_wc[i] += p_wL[i];
    m3_transpose(R_wc, R_cw);
    m3_vec(R_cw, t_wc, t_cw);
    for (int i = 0; i < 3; i++) t_cw[i] = -t_cw[i];
}

/* ------------------------------------------------------------ projection */

typedef struct {
    int valid;          /* in front of the near plane and opacity >= alpha_min */
    int near_edge;      /* the near-plane culling is not decided in float32 */
    float zkey;         /* depth rounded to float32: the depth order's key */
    int zamb;           /* the exact depth lies within the bound of a float32 rounding boundary */
    float zalt;         /* the other candidate key where zamb (the float across that boundary), else zkey */
    double dm[2];       /* bound on the float32 2D mean's error, px */
    double kq;          /* bound on the conic's share of the float32 exponent error, per unit of |e2| */
    double dF;          /* bound on the float32 log2 opacity's error */
    double X[3], pc[3];
    double q[4], qn, Rg[9], s[3];
    int s_clamped[3];
    double Sig[9], Sigc[9];
    double J[6];
    double jx, jy;      /* x/z and y/z used in J (clamped to the widened field of view) */
    int jclamp_x, jclamp_y;
    double cov[3];      /* 2D covariance (xx, xy, yy), including the low-pass */
    double conic[3];    /* inverse 2D covariance (a, b, c) */
    double mean[2];
    double opacity;
    double extent[2];   /* half-widths of the alpha >= alpha_min ellipse's box */
} or_proj;

/* ------------------------------------------- float32 decision bounds --
 *
 * The renderer evaluates, per pixel and Gaussian, the base-2 exponent
 *   e2 = A dx^2 + B dx dy + C dy^2,  e = e2 + F   (A = -a/2 log2 e,
 *   B = -b log2 e, C = -c/2 log2 e, (a, b, c) the conic, F = log2 opacity,
 *   dx = u - mean_x, dy = v - mean_y)
 * in float32 from float32 projections, and decides: skip if e2 > 0, skip if
 * e < log2 alpha_min, clamp alpha = 2^e at alpha_max, stop if T (1 - alpha)
 * < t_min.  These bounds follow the rounding of that evaluation (u = 2^-24
 * per operation, first order):
 *   mean: rounded once from fx x/z + cx (float-float before the rounding),
 *     so off by half a float32 spacing at the mean, plus the rounding of the
 *     intrinsics to float32 and a far smaller float-float term;
 *   conic: about twenty roundings, each relative to the terms of the 2D
 *     covariance J Sigma_c J^T, whose size is |J|^2 lambda_max(Sigma); a
 *     covariance error d(cov) moves the exponent by (Q d)^T d(cov) (Q d)
 *     <= |d(cov)| |e2| / lambda_min(cov) (Q the conic), so that share is
 *     16 u (1 + |J|^2 lambda_max(Sigma) / lambda_min(cov)) |e2|, plus 4 u
 *     times the size of e2's terms for the rounding of A, B, C themselves;
 *   F: log2 of a float32 sigmoid, within 2^-20 (1 + |F|);
 *   the exponent itself: six roundings relative to its terms, plus the
 *     offset dx when u - mean_x is not exact;
 *   2^e: the hardware approximation, relative error below 2^-20;
 *   thresholds: log2 of float32 alpha_min within 2^-19; alpha_max and t_min
 *     rounded to float32. */
#define OR_U32 0x1p-24

static double f32_spacing(double x) { /* spacing of float32 values just above |x| */
    float f = (float)fabs(x);
    return (double)nextafterf(f, INFINITY) - (double)f;
}

static void decision_bounds(or_proj *P, const or_cam *cam, const or_opts *o) {
    (void)o;
    double z = P->pc[2];
    double dn = sqrt(P->pc[0] * P->pc[0] + P->pc[1] * P->pc[1] + z * z) / z;
    double f[2] = {cam->fx, cam->fy}, c[2] = {cam->cx, cam->cy};
    for (int i = 0; i < 2; i++) {
        double r = P->pc[i] / z;
        P->dm[i] = 0.5 * f32_spacing(P->mean[i]) + fabs(f[i] - (double)(float)f[i]) * fabs(r)
                 + fabs(c[i] - (double)(float)c[i])
                 + 0x1p-36 * (fabs(P->mean[i]) + fabs(f[i]) * (1.0 + fabs(r)) * dn + 1.0);
    }
    double smax = P->s[0] > P->s[1] ? P->s[0] : P->s[1];
    if (P->s[2] > smax) smax = P->s[2];
    double J2 = P->J[0] * P->J[0] + P->J[2] * P->J[2] + P->J[4] * P->J[4] + P->J[5] * P->J[5];
    double h = 0.5 * (P->cov[0] + P->cov[2]);
    double r = sqrt(0.25 * (P->cov[0] - P->cov[2]) * (P->cov[0] - P->cov[2]) + P->cov[1] * P->cov[1]);
    double lmin = h - r;
    P->kq = 16.0 * OR_U32 * (1.0 + J2 * smax * smax / lmin);
    P->dF = 0x1p-20 * (1.0 + fabs(log2(P->opacity)));
}

static void project_one(const double *X, const double *q, const double *log_s, double logit_o,
                        const or_cam *cam, const double *R_cw, const double *t_cw,
                        const or_opts *o, or_proj *P) {
    memset(P, 0, sizeof *P);
    for (int i = 0; i < 3; i++) P->X[i] = X[i];
    m3_vec(R_cw, P->X, P->pc);
    for (int i = 0; i < 3; i++) P->pc[i] += t_cw[i];
    double z = P->pc[2];
    /* The depth order and the near-plane culling are decided on the depth
     * rounded to float32 (the renderer's precision for its sort key).  The
     * kernel forms the depth in float-float arithmetic and rounds it once;
     * its value and this one differ by far less than 2^-40 (|X| + 2|t| + |z|),
     * so the two roundings can differ only within that distance of a
     * rounding boundary. */
    P->zkey = (float)z;
    {
        double eps = 0x1p-40 * (fabs(X[0]) + fabs(X[1]) + fabs(X[2]) + 2.0 * (fabs(t_cw[0]) + fabs(t_cw[1]) + fabs(t_cw[2])) + fabs(z));
        float k = P->zkey;
        double below = 0.5 * ((double)k + (double)nextafterf(k, -INFINITY));
        double above = 0.5 * ((double)k + (double)nextafterf(k, INFINITY));
        P->zamb = (z - below < eps) || (above - z < eps);
        float near = (float)o->near_z;
        float other = z - below < eps ? nextafterf(k, -INFINITY) : nextafterf(k, INFINITY);
        P->zalt = P->zamb ? other : k;
        P->near_edge = P->zamb && ((k > near) != (other > near));
    }
    int in_front = P->zkey > (float)o->near_z;
    /* Gaussian covariance Sigma = R S S^T R^T in the world frame */
    double n2 = 0;
    for (int i = 0; i < 4; i++) { P->q[i] = q[i]; n2 += P->q[i] * P->q[i]; }
    P->qn = sqrt(n2);
    double qu[4];
    for (int i = 0; i < 4; i++) qu[i] = P->q[i] / P->qn;
    quat_to_rot(qu, P->Rg);
    for (int i = 0; i < 3; i++) {
        double s = exp(log_s[i]);
        P->s_clamped[i] = s > o->scale_max;
        P->s[i] = P->s_clamped[i] ? o->scale_max : s;
    }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double v = 0;
            for (int k = 0; k < 3; k++) v += P->Rg[3 * i + k] * P->s[k] * P->s[k] * P->Rg[3 * j + k];
            P->Sig[3 * i + j] = v;
        }
    /* Eq. 3: rotate into the camera frame, Sigma_c = R_cw Sigma R_cw^T */
    double T1[9], Rt[9];
    m3_mul(R_cw, P->Sig, T1);
    m3_transpose(R_cw, Rt);
    m3_mul(T1, Rt, P->Sigc);
    P->opacity = 1.0 / (1.0 + exp(-logit_o));
    if (!in_front && !P->near_edge) return;
    if (z <= 1e-9) return;
    /* EWA: Jacobian of (x,y,z) -> (fx x/z + cx, fy y/z + cy), evaluated at
     * x/z and y/z limited to the widened field of view (3DGS's EWA), which
     * bounds the footprint of centres far outside the image */
    double x = P->pc[0], y = P->pc[1];
    P->jx = x / z;
    P->jy = y / z;
    if (o->frustum_margin >= 0) {
        double mx = o->frustum_margin * cam->width, my = o->frustum_margin * cam->height;
        double xlo = -(cam->cx + mx) / cam->fx, xhi = (cam->width - cam->cx + mx) / cam->fx;
        double ylo = -(cam->cy + my) / cam->fy, yhi = (cam->height - cam->cy + my) / cam->fy;
        if (P->jx < xlo) { P->jx = xlo; P->jclamp_x = 1; }
        if (P->jx > xhi) { P->jx = xhi; P->jclamp_x = 1; }
        if (P->jy < ylo) { P->jy = ylo; P->jclamp_y = 1; }
        if (P->jy > yhi) { P->jy = yhi; P->jclamp_y = 1; }
    }
    P->J[0] = cam->fx / z; P->J[1] = 0;             P->J[2] = -cam->fx * P->jx / z;
    P->J[3] = 0;           P->J[4] = cam->fy / z;   P->J[5] = -cam->fy * P->jy / z;
    double JS[6];
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 3; c++) {
            double v = 0;
            for (int k = 0; k < 3; k++) v += P->J[3 * r + k] * P->Sigc[3 * k + c];
            JS[3 * r + c] = v;
        }
    double C2[4];
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 2; c++) {
            double v = 0;
            for (int k = 0; k < 3; k++) v += JS[3 * r + k] * P->J[3 * c + k];
            C2[2 * r + c] = v;
        }
    P->cov[0] = C2[0] + o->lowpass;
    P->cov[1] = 0.5 * (C2[1] + C2[2]);
    P->cov[2] = C2[3] + o->lowpass;
    double det = P->cov[0] * P->cov[2] - P->cov[1] * P->cov[1];
    if (!(det > 0)) return;
    P->conic[0] = P->cov[2] / det;
    P->conic[1] = -P->cov[1] / det;
    P->conic[2] = P->cov[0] / det;
    P->mean[0] = cam->fx * x / z + cam->cx;
    P->mean[1] = cam->fy * y / z + cam->cy;
    decision_bounds(P, cam, o);
    if (P->opacity < o->alpha_min) return;
    /* alpha >= alpha_min  <=>  d^T conic d <= 2 ln(opacity / alpha_min); the
     * box of that ellipse has half-widths sqrt(k cov_xx), sqrt(k cov_yy). */
    double kk = o->alpha_min > 0 ? 2.0 * log(P->opacity / o->alpha_min) : INFINITY;
    P->extent[0] = sqrt(kk * P->cov[0]);
    P->extent[1] = sqrt(kk * P->cov[2]);
    P->valid = in_front;
}

/* Exported: projection of all Gaussians of a scene for one camera pose.
 * out_* arrays have N rows; rect is [N][4] = (x0,y0,x1,y1) in tiles of
 * size `tile`, inclusive, clamped to the image, empty as x0 > x1.
 * out_bounds (optional) is [N][7]: the float32 depth key, whether its
 * rounding is undecided (1/0), whether the near-plane culling is undecided
 * (1/0), the float32 mean's error bounds (x, y, px), the conic's share of
 * the exponent error per unit of |e2|, the log2 opacity's error bound
 * (see "float32 decision bounds"). */
void or_project(int N, const double *X, const double *q, const double *log_s, const double *logit_o,
                const or_cam *cam, const double *R_cw, const double *t_cw, const or_opts *o,
                int tile, int32_t *out_valid, double *out_depth, double *out_mean,
                double *out_conic, double *out_opacity, double *out_extent, double *out_cov,
                int32_t *out_rect, double *out_bounds) {
    int tx = (cam->width + tile - 1) / tile, ty = (cam->height + tile - 1) / tile;
    for (int g = 0; g < N; g++) {
        or_proj P;
        project_one(X + 3 * g, q + 4 * g, log_s + 3 * g, logit_o[g], cam, R_cw, t_cw, o, &P);
        out_valid[g] = P.valid;
        out_depth[g] = P.pc[2];
        out_mean[2 * g] = P.mean[0]; out_mean[2 * g + 1] = P.mean[1];
        for (int i = 0; i < 3; i++) { out_conic[3 * g + i] = P.conic[i]; out_cov[3 * g + i] = P.cov[i]; }
        out_opacity[g] = P.opacity;
        out_extent[2 * g] = P.extent[0]; out_extent[2 * g + 1] = P.extent[1];
        if (out_bounds) {
            double *b = out_bounds + 7 * (size_t)g;
            b[0] = P.zkey; b[1] = P.zamb; b[2] = P.near_edge;
            b[3] = P.dm[0]; b[4] = P.dm[1]; b[5] = P.kq; b[6] = P.dF;
        }
        int x0 = 1, y0 = 1, x1 = 0, y1 = 0;
        if (P.valid && !(isfinite(P.extent[0]) && isfinite(P.extent[1]))) {
            x0 = 0; y0 = 0; x1 = tx - 1; y1 = ty - 1;
        } else if (P.valid) {
            x0 = (int)floor((P.mean[0] - P.extent[0]) / tile);
            x1 = (int)floor((P.mean[0] + P.extent[0]) / tile);
            y0 = (int)floor((P.mean[1] - P.extent[1]) / tile);
            y1 = (int)floor((P.mean[1] + P.extent[1]) / tile);
            if (x0 < 0) x0 = 0;
            if (y0 < 0) y0 = 0;
            if (x1 > tx - 1) x1 = tx - 1;
            if (y1 > ty - 1) y1 = ty - 1;
            if (x0 > x1 || y0 > y1) { x0 = 1; x1 = 0; y0 = 1; y1 = 0; }
        }
        int32_t *r = out_rect + 4 * g;
        r[0] = x0; r[1] = y0; r[2] = x1; r[3] = y1;
    }
}

/* ---------------------------------------------------------- compositing */

/* Depth order (Eq. 5 composites in depth order): by the float32 depth key,
 * equal keys by Gaussian index. */
typedef struct { float z; int g; } zkey;

static int cmp_zkey(const void *a, const void *b) {
    const zkey *x = a, *y = b;
    if (x->z < y->z) return -1;
    if (x->z > y->z) return 1;
    return (x->g > y->g) - (x->g < y->g);
}

typedef struct {
    int N, M;           /* Gaussians, visible Gaussians in depth order */
    or_proj *P;
    int *order;         /* visible Gaussian ids by (depth, id) */
    int *edge_ids;      /* Gaussians straddling the near plane */
    int n_edge;
} or_frame_state;

static void frame_state(or_frame_state *S, int N, const double *X, const double *q, const double *log_s,
                        const double *logit_o, const or_cam *cam, const double *R_cw,
                        const double *t_cw, const or_opts *o) {
    S->N = N;
    S->P = (or_proj *)malloc(sizeof(or_proj) * (N > 0 ? N : 1));
    zkey *keys = (zkey *)malloc(sizeof(zkey) * (N > 0 ? N : 1));
    S->edge_ids = (int *)malloc(sizeof(int) * (N > 0 ? N : 1));
    S->M = 0;
    S->n_edge = 0;
    for (int g = 0; g < N; g++) {
        project_one(X + 3 * g, q + 4 * g, log_s + 3 * g, logit_o[g], cam, R_cw, t_cw, o, &S->P[g]);
        if (S->P[g].valid) { keys[S->M].z = S->P[g].zkey; keys[S->M].g = g; S->M++; }
        if (S->P[g].near_edge) S->edge_ids[S->n_edge++] = g;
    }
    qsort(keys, S->M, sizeof(zkey), cmp_zkey);
    S->order = (int *)malloc(sizeof(int) * (S->M > 0 ? S->M : 1));
    for (int i = 0; i < S->M; i++) S->order[i] = keys[i].g;
    free(keys);
}

static void frame_state_free(or_frame_state *S) {
    free(S->P); free(S->order); free(S->edge_ids);
}

/* power and alpha of Gaussian P at pixel (u, v): the 2D Gaussian's exponent
 * and alpha = min(alpha_max, opacity * exp(power)). */
static void eval_alpha(const or_proj *P, double u, double v, const or_opts *o,
                       double *dx, double *dy, double *power, double *G, double *alpha, int *clamped) {
    *dx = u - P->mean[0];
    *dy = v - P->mean[1];
    *power = -0.5 * (P->conic[0] * (*dx) * (*dx) + P->conic[2] * (*dy) * (*dy)) - P->conic[1] * (*dx) * (*dy);
    *G = exp(*power);
    double a = P->opacity * (*G);
    *clamped = a > o->alpha_max;
    *alpha = *clamped ? o->alpha_max : a;
}

/* Blend list of one pixel: the Gaussians that are composited, in order, with
 * their alpha and the transmittance in front of each. */
typedef struct {
    int n;
    int *g;
    double *alpha, *T, *G, *dx, *dy;
    int *clamped;
    double T_final;
    int flags;
    int ndec;                         /* ambiguous decisions met by this pass */
} or_blend;

/* The outcome of each ambiguous decision of a pass, in the order met: the
 * first n are given (1 = the outcome opposite to FP64's), the rest take the
 * FP64 outcome. */
typedef struct {
    int n;
    unsigned char flip[OR_MAX_DECISIONS];
} or_path;

/* Take an ambiguous decision: the FP64 outcome, or its opposite where the
 * path says so. */
static int decide(or_blend *B, const or_path *path, int fp64_outcome) {
    int j = B->ndec;
    if (j >= OR_MAX_DECISIONS) { B->flags |= OR_FLAG_BRANCH_LIMIT; return fp64_outcome; }
    B->ndec++;
    B->flags |= OR_FLAG_BRANCH;
    return (j < path->n && path->flip[j]) ? !fp64_outcome : fp64_outcome;
}

/* One front-to-back pass over the pixel's depth-ordered Gaussians (Eq. 5,
 * with the skip/stop rules of the readings in or_opts), taking every
 * ambiguous decision as `path` says. */
static void blend_pixel_path(const or_frame_state *S, double u, double v, const or_opts *o, const or_path *path,
                             or_blend *B) {
    B->n = 0;
    B->flags = 0;
    B->ndec = 0;
    double T = 1.0;
    double eT = 0.0;                  /* bound on the float32 transmittance's relative error */
    float kprev_max = 0.f;  /* the previous contributor's largest candidate key, and its index */
    int gprev = -1;
    const double log2e = 1.0 / log(2.0);
    const double lmin = o->alpha_min > 0 ? log2(o->alpha_min) : -INFINITY;
    const double lmax = log2(o->alpha_max);
    const double amax32 = (double)(float)o->alpha_max, tmin32 = (double)(float)o->t_min;
    for (int i = 0; i < S->M; i++) {
        const or_proj *P = &S->P[S->order[i]];
        double dx, dy, power, G, alpha;
        int clamped;
        eval_alpha(P, u, v, o, &dx, &dy, &power, &G, &alpha, &clamped);
        /* the exponent in base 2 and the bound on its float32 evaluation */
        double A = -0.5 * log2e * P->conic[0], Bc = -log2e * P->conic[1], C = -0.5 * log2e * P->conic[2];
        double e2 = power * log2e, F = log2(P->opacity), e = e2 + F;
        double mag = fabs(A) * dx * dx + fabs(Bc * dx * dy) + fabs(C) * dy * dy;
        double gx = fabs(2.0 * A * dx + Bc * dy), gy = fabs(Bc * dx + 2.0 * C * dy);
        double eps2 = gx * (P->dm[0] + OR_U32 * fabs(dx)) + gy * (P->dm[1] + OR_U32 * fabs(dy))
                    + P->kq * fabs(e2) + 10.0 * OR_U32 * mag;
        double eps = eps2 + OR_U32 * (fabs(e2) + fabs(F)) + P->dF;
        /* skip where the exponent is positive (only by rounding: the form is
         * negative definite) */
        int skip = power > 0;
        if (e2 + eps2 > 0) skip = decide(B, path, skip);
        if (skip) continue;
        /* skip alpha < alpha_min */
        skip = alpha < o->alpha_min;
        if (o->alpha_min > 0 && fabs(e - lmin) <= eps + 0x1p-19) skip = decide(B, path, skip);
        if (skip) continue;
        /* the clamp at alpha_max is continuous in colour, not in gradient */
        int near_clamp = o->alpha_max < 1.0 && fabs(e - lmax) <= eps + 0x1p-22;
        /* float32 alpha's relative error, then (1 - alpha)'s */
        double ea = clamped && !near_clamp ? fabs(amax32 - o->alpha_max) / o->alpha_max
                                           : log(2.0) * eps + 0x1p-20;
        double e1 = alpha * ea / (1.0 - alpha) + OR_U32;
        double testT = T * (1.0 - alpha);
        int stop = testT < o->t_min;
        if (o->t_min > 0 && fabs(testT - o->t_min) <= testT * (eT + e1 + 2.0 * OR_U32) + fabs(tmin32 - o->t_min))
            stop = decide(B, path, stop);
        if (stop) break;
        if (near_clamp) B->flags |= OR_FLAG_CLAMP_EDGE;
        /* consecutive contributors whose float32 order is not decided: some
         * choice of their candidate keys puts them out of (key, index) order */
        {
            const int gcur = S->order[i];
            const float kmin = P->zalt < P->zkey ? P->zalt : P->zkey;
            if (gprev >= 0 && (kmin < kprev_max || (kmin == kprev_max && gcur < gprev)))
                B->flags |= OR_FLAG_DEPTH_TIE;
            kprev_max = P->zalt > P->zkey ? P->zalt : P->zkey;
            gprev = gcur;
        }
        int k = B->n++;
        B->g[k] = S->order[i];
        B->alpha[k] = alpha;
        B->T[k] = T;
        B->G[k] = G;
        B->dx[k] = dx;
        B->dy[k] = dy;
        B->clamped[k] = clamped;
        T = testT;
        eT += e1 + 2.0 * OR_U32;
    }
    B->T_final = T;
    for (int e = 0; e < S->n_edge; e++) {
        const or_proj *P = &S->P[S->edge_ids[e]];
        if (!(P->conic[0] > 0)) continue;
        double dx, dy, power, G, alpha;
        int clamped;
        eval_alpha(P, u, v, o, &dx, &dy, &power, &G, &alpha, &clamped);
        if (power <= 0 && alpha >= o->alpha_min) B->flags |= OR_FLAG_NEAR_EDGE;
    }
}

/* The FP64 pass (every ambiguous decision takes its FP64 outcome). */
static void blend_pixel(const or_frame_state *S, double u, double v, const or_opts *o, or_blend *B) {
    or_path none;
    none.n = 0;
    blend_pixel_path(S, u, v, o, &none, B);
}

static void blend_alloc(or_blend *B, int M) {
    int m = M > 0 ? M : 1;
    B->g = (int *)malloc(sizeof(int) * m);
    B->clamped = (int *)malloc(sizeof(int) * m);
    B->alpha = (double *)malloc(sizeof(double) * m);
    B->T = (double *)malloc(sizeof(double) * m);
    B->G = (double *)malloc(sizeof(double) * m);
    B->dx = (double *)malloc(sizeof(double) * m);
    B->dy = (double *)malloc(sizeof(double) * m);
}

static void blend_free(or_blend *B) {
    free(B->g); free(B->clamped); free(B->alpha); free(B->T); free(B->G); free(B->dx); free(B->dy);
}

/* The outcome of a pass: rgb = sum_i c_i alpha_i T_i + T_final bg, T_final,
 * last composited Gaussian (-1 if none). */
static void blend_result(const or_blend *B, const double *rgb, const or_opts *o, double *out5) {
    double C[3] = {0, 0, 0};
    for (int k = 0; k < B->n; k++)
        for (int ch = 0; ch < 3; ch++) C[ch] += rgb[3 * B->g[k] + ch] * B->alpha[k] * B->T[k];
    for (int ch = 0; ch < 3; ch++) out5[ch] = C[ch] + B->T_final * o->bg[ch];
    out5[3] = B->T_final;
    out5[4] = B->n > 0 ? B->g[B->n - 1] : -1;
}

typedef struct {
    const or_frame_state *S;
    const double *rgb;
    const or_opts *o;
    double u, v;
    or_blend *B;
    int count;                 /* outcomes found */
    double out[OR_MAX_BRANCHES][5];
    int flags;
} or_branches;

/* Every outcome of the pixel's ambiguous decisions, depth first: run the
 * pass for `path` (its later decisions at their FP64 outcome), keep its
 * result, then for each later decision it met, the path that flips it. */
static void explore(or_branches *X, const or_path *path) {
    if (X->count >= OR_MAX_BRANCHES) { X->flags |= OR_FLAG_BRANCH_LIMIT; return; }
    blend_pixel_path(X->S, X->u, X->v, X->o, path, X->B);
    blend_result(X->B, X->rgb, X->o, X->out[X->count++]);
    X->flags |= X->B->flags;
    int ndec = X->B->ndec;
    for (int j = path->n; j < ndec && j < OR_MAX_DECISIONS; j++) {
        or_path child = *path;
        for (int k = path->n; k < j; k++) child.flip[k] = 0;
        child.flip[j] = 1;
        child.n = j + 1;
        explore(X, &child);
    }
}

/* Exported: render the requested pixels of one frame.
 * pix: [npix][2] integer pixel coordinates (u, v), or NULL for all pixels in
 * row-major order.  Pixel (u, v) is the image point (u, v) in the same
 * coordinates as fx x/z + cx (pinhole, OpenCV convention).
 * Outputs per requested pixel: rgb[3] = sum_i c_i alpha_i T_i + T_final bg,
 * T_final, last = id of the last composited Gaussian (-1 if none), flags
 * (OR_FLAG_*), all for the FP64 outcome of every decision.  If out_alt is
 * given, out_nalt[p] is the number of other outcomes of the pixel's
 * ambiguous decisions (0..OR_MAX_BRANCHES-1) and out_alt[p][k] = (rgb[3],
 * T_final, last) of outcome k. */
void or_render(int N, const double *X, const double *q, const double *log_s, const double *logit_o,
               const double *rgb, const or_cam *cam, const double *R_cw, const double *t_cw,
               const or_opts *o, int npix, const int32_t *pix,
               double *out_rgb, double *out_T, int32_t *out_last, int32_t *out_flags,
               int32_t *out_nalt, double *out_alt) {
    or_frame_state S;
    frame_state(&S, N, X, q, log_s, logit_o, cam, R_cw, t_cw, o);
    or_blend B;
    blend_alloc(&B, S.M);
    or_branches *Xb = (or_branches *)malloc(sizeof(or_branches));
    int total = pix ? npix : cam->width * cam->height;
    for (int p = 0; p < total; p++) {
        double u = pix ? pix[2 * p] : (double)(p % cam->width);
        double v = pix ? pix[2 * p + 1] : (double)(p / cam->width);
        Xb->S = &S; Xb->rgb = rgb; Xb->o = o; Xb->u = u; Xb->v = v; Xb->B = &B;
        Xb->count = 0;
        Xb->flags = 0;
        or_path none;
        none.n = 0;
        if (out_alt) {
            explore(Xb, &none);
        } else {
            blend_pixel_path(&S, u, v, o, &none, &B);
            blend_result(&B, rgb, o, Xb->out[0]);
            Xb->count = 1;
            Xb->flags = B.flags;
        }
        for (int ch = 0; ch < 3; ch++) out_rgb[3 * p + ch] = Xb->out[0][ch];
        out_T[p] = Xb->out[0][3];
        out_last[p] = (int32_t)Xb->out[0][4];
        out_flags[p] = Xb->flags;
        if (out_alt) {
            out_nalt[p] = Xb->count - 1;
            for (int k = 1; k < Xb->count; k++)
                for (int j = 0; j < 5; j++) out_alt[((size_t)p * (OR_MAX_BRANCHES - 1) + k - 1) * 5 + j] = Xb->out[k][j];
        }
    }
    free(Xb);
    blend_free(&B);
    frame_state_free(&S);
}

/* ----------------------------------------------------------- backward -- */

/* Exported: gradients of L = sum_p dL_dC[p] . C(p) over the requested pixels
 * of one frame, for the Gaussian parameters (accumulated into d_q, d_log_s,
 * d_logit_o, d_rgb) and, through the camera pose of Eq. 1, for the extrinsic
 * (omega, t_e) and the time offset delta (accumulated into d_ext[6],
 * d_delta[0]).
 *
 * Chain, all by plain matrix calculus:
 *   C(p) = sum_i c_i alpha_i T_i + T_final bg, so
 *     dC/dc_i = alpha_i T_i,
 *     dC/dalpha_i = c_i T_i - (sum_{j>i} c_j alpha_j T_j + T_final bg) / (1 - alpha_i);
 *   alpha = opacity * exp(power) (zero derivative where clamped);
 *   power = -1/2 d^T Q d, d = pixel - mean, Q = conic = cov^-1;
 *   cov = J Sigma_c J^T + lowpass I;  Sigma_c = R_cw Sigma R_cw^T;
 *   Sigma = R_g diag(s)^2 R_g^T; p_c = R_cw X + t_cw; mean = pinhole(p_c);
 *   [R_cw | t_cw] = inverse of T_L(t + delta) [R_e | t_e], R_e = exp([omega]x).
 */
void or_backward(int N, const double *X, const double *q, const double *log_s, const double *logit_o,
                 const double *rgb, const or_cam *cam,
                 const double *traj_t, const double *traj_p, const double *traj_q, int K,
                 const double *ext, double delta, double t_frame, const or_opts *o,
                 int npix, const int32_t *pix, const double *dL_dC,
                 double *d_q, double *d_log_s, double *d_logit_o, double *d_rgb,
                 double *d_ext, double *d_delta, double *out_g_mean, double *out_g_conic,
                 double *out_g_opacity) {
    double R_cw[9], t_cw[3];
    or_frame_pose(traj_t, traj_p, traj_q, K, ext, delta, t_frame, R_cw, t_cw);
    or_frame_state S;
    frame_state(&S, N, X, q, log_s, logit_o, cam, R_cw, t_cw, o);
    or_blend B;
    blend_alloc(&B, S.M);
    /* per-Gaussian 2D gradients */
    double *g_mean = (double *)calloc(2 * (size_t)(N > 0 ? N : 1), sizeof(double));
    double *g_conic = (double *)calloc(3 * (size_t)(N > 0 ? N : 1), sizeof(double));
    double *g_opac = (double *)calloc((size_t)(N > 0 ? N : 1), sizeof(double));
    double *suffix = (double *)malloc(sizeof(double) * 3 * (S.M + 1));
    int total = pix ? npix : cam->width * cam->height;
    for (int p = 0; p < total; p++) {
        const double *gC = dL_dC + 3 * p;
        if (gC[0] == 0 && gC[1] == 0 && gC[2] == 0) continue;
        double u = pix ? pix[2 * p] : (double)(p % cam->width);
        double v = pix ? pix[2 * p + 1] : (double)(p / cam->width);
        blend_pixel(&S, u, v, o, &B);
        /* suffix[k] = sum_{j >= k} c_j alpha_j T_j */
        for (int ch = 0; ch < 3; ch++) suffix[3 * B.n + ch] = 0;
        for (int k = B.n - 1; k >= 0; k--)
            for (int ch = 0; ch < 3; ch++)
                suffix[3 * k + ch] = suffix[3 * (k + 1) + ch] + rgb[3 * B.g[k] + ch] * B.alpha[k] * B.T[k];
        for (int k = 0; k < B.n; k++) {
            int g = B.g[k];
            const or_proj *P = &S.P[g];
            double dalpha = 0;
            for (int ch = 0; ch < 3; ch++) {
                d_rgb[3 * g + ch] += gC[ch] * B.alpha[k] * B.T[k];
                double dCda = rgb[3 * g + ch] * B.T[k]
                            - (suffix[3 * (k + 1) + ch] + B.T_final * o->bg[ch]) / (1.0 - B.alpha[k]);
                dalpha += gC[ch] * dCda;
            }
            if (B.clamped[k]) continue;
            g_opac[g] += dalpha * B.G[k];
            double dpower = dalpha * B.alpha[k];
            double dx = B.dx[k], dy = B.dy[k];
            /* power = -1/2 (a dx^2 + 2 b dx dy + c dy^2), dx = u - mean_x */
            g_mean[2 * g] += dpower * (P->conic[0] * dx + P->conic[1] * dy);
            g_mean[2 * g + 1] += dpower * (P->conic[1] * dx + P->conic[2] * dy);
            g_conic[3 * g] += dpower * (-0.5 * dx * dx);
            g_conic[3 * g + 1] += dpower * (-dx * dy);
            g_conic[3 * g + 2] += dpower * (-0.5 * dy * dy);
        }
    }
    /* optional: the per-Gaussian 2D gradients (mean, conic (a,b,c), opacity) */
    for (int g = 0; g < N; g++) {
        if (out_g_mean) { out_g_mean[2 * g] += g_mean[2 * g]; out_g_mean[2 * g + 1] += g_mean[2 * g + 1]; }
        if (out_g_conic) for (int i = 0; i < 3; i++) out_g_conic[3 * g + i] += g_conic[3 * g + i];
        if (out_g_opacity) out_g_opacity[g] += g_opac[g];
    }
    /* 3D chain per Gaussian; pose gradient as dL/dR_cw and dL/dt_cw */
    double gR_cw[9] = {0}, gt_cw[3] = {0};
    for (int g = 0; g < N; g++) {
        const or_proj *P = &S.P[g];
        if (!P->valid) continue;
        double gm0 = g_mean[2 * g], gm1 = g_mean[2 * g + 1];
        double ga = g_conic[3 * g], gb = g_conic[3 * g + 1], gc = g_conic[3 * g + 2];
        if (gm0 == 0 && gm1 == 0 && ga == 0 && gb == 0 && gc == 0 && g_opac[g] == 0) continue;
        d_logit_o[g] += g_opac[g] * P->opacity * (1.0 - P->opacity);
        /* Q = cov^-1 with Q = [[a,b],[b,c]]; b sits in two entries, so the
         * matrix gradient is Gq = [[ga, gb/2],[gb/2, gc]];  dL/dcov = -Q Gq Q */
        double Q[4] = {P->conic[0], P->conic[1], P->conic[1], P->conic[2]};
        double Gq[4] = {ga, 0.5 * gb, 0.5 * gb, gc};
        double T1[4], Gc[4];
        for (int r = 0; r < 2; r++)
            for (int c = 0; c < 2; c++) T1[2 * r + c] = Q[2 * r] * Gq[c] + Q[2 * r + 1] * Gq[2 + c];
        for (int r = 0; r < 2; r++)
            for (int c = 0; c < 2; c++) Gc[2 * r + c] = -(T1[2 * r] * Q[c] + T1[2 * r + 1] * Q[2 + c]);
        /* cov = J Sigma_c J^T + lp I:  dL/dSigma_c = J^T Gc J,  dL/dJ = 2 Gc J Sigma_c */
        double GS[9];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double s = 0;
                for (int r = 0; r < 2; r++)
                    for (int c = 0; c < 2; c++) s += P->J[3 * r + i] * Gc[2 * r + c] * P->J[3 * c + j];
                GS[3 * i + j] = s;
            }
        double GJ[6];
        for (int r = 0; r < 2; r++)
            for (int j = 0; j < 3; j++) {
                double s = 0;
                for (int c = 0; c < 2; c++)
                    for (int k = 0; k < 3; k++) s += Gc[2 * r + c] * P->J[3 * c + k] * P->Sigc[3 * k + j];
                GJ[3 * r + j] = 2.0 * s;
            }
        /* J and mean as functions of p_c: J02 = -fx jx / z with jx = x/z, or
         * a constant where clamped (then jx carries no gradient) */
        double x = P->pc[0], y = P->pc[1], z = P->pc[2];
        double fx = cam->fx, fy = cam->fy;
        double djx_dx = P->jclamp_x ? 0.0 : 1.0 / z, djx_dz = P->jclamp_x ? 0.0 : -x / (z * z);
        double djy_dy = P->jclamp_y ? 0.0 : 1.0 / z, djy_dz = P->jclamp_y ? 0.0 : -y / (z * z);
        double gp[3];
        gp[0] = GJ[2] * (-fx / z) * djx_dx + gm0 * fx / z;
        gp[1] = GJ[5] * (-fy / z) * djy_dy + gm1 * fy / z;
        gp[2] = GJ[0] * (-fx / (z * z)) + GJ[2] * (fx * P->jx / (z * z) - fx / z * djx_dz)
              + GJ[4] * (-fy / (z * z)) + GJ[5] * (fy * P->jy / (z * z) - fy / z * djy_dz)
              + gm0 * (-fx * x / (z * z)) + gm1 * (-fy * y / (z * z));
        /* Sigma_c = R_cw Sigma R_cw^T */
        double Rt[9], T2[9], GSig[9];
        m3_transpose(R_cw, Rt);
        m3_mul(Rt, GS, T2);
        m3_mul(T2, R_cw, GSig);
        double T3[9], T4[9];
        m3_mul(GS, R_cw, T3);
        m3_mul(T3, P->Sig, T4);
        for (int i = 0; i < 9; i++) gR_cw[i] += 2.0 * T4[i];
        /* p_c = R_cw X + t_cw */
        for (int i = 0; i < 3; i++) {
            for (int j = 0; j < 3; j++) gR_cw[3 * i + j] += gp[i] * P->X[j];
            gt_cw[i] += gp[i];
        }
        /* Sigma = R_g S^2 R_g^T */
        double S2[3] = {P->s[0] * P->s[0], P->s[1] * P->s[1], P->s[2] * P->s[2]};
        double gRg[9];
        for (int i = 0; i < 3; i++)
            for (int k = 0; k < 3; k++) {
                double s = 0;
                for (int j = 0; j < 3; j++) s += GSig[3 * i + j] * P->Rg[3 * j + k];
                gRg[3 * i + k] = 2.0 * s * S2[k];
            }
        for (int k = 0; k < 3; k++) {
            double s = 0;
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) s += P->Rg[3 * i + k] * GSig[3 * i + j] * P->Rg[3 * j + k];
            double gs = 2.0 * P->s[k] * s;
            if (!P->s_clamped[k]) d_log_s[3 * g + k] += gs * P->s[k];
        }
        /* R_g = R(q / |q|) */
        double qu[4], gqu[4];
        for (int i = 0; i < 4; i++) qu[i] = P->q[i] / P->qn;
        for (int i = 0; i < 4; i++) {
            double e[4] = {0, 0, 0, 0}, dR[9];
            e[i] = 1.0;
            quat_to_rot_dir(qu, e, dR);
            gqu[i] = m3_dot(gRg, dR);
        }
        double dotq = 0;
        for (int i = 0; i < 4; i++) dotq += qu[i] * gqu[i];
        for (int i = 0; i < 4; i++) d_q[4 * g + i] += (gqu[i] - qu[i] * dotq) / P->qn;
    }
    /* pose chain: [R_cw | t_cw] = inv([R_wc | t_wc]), R_wc = R_wL R_e,
     * t_wc = R_wL t_e + p_wL, (R_wL, p_wL) = T_L(t + delta) */
    double R_wL[9], p_wL[3], dR_dtau[9], dp_dtau[3], R_e[9], R_wc[9], t_wc[3];
    or_lidar_pose(traj_t, traj_p, traj_q, K, t_frame + delta, R_wL, p_wL, dR_dtau, dp_dtau);
    rodrigues(ext, R_e);
    m3_mul(R_wL, R_e, R_wc);
    m3_vec(R_wL, ext + 3, t_wc);
    for (int i = 0; i < 3; i++) t_wc[i] += p_wL[i];
    double gR_wc[9], gt_wc[3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) gR_wc[3 * i + j] = gR_cw[3 * j + i] - t_wc[i] * gt_cw[j];
    m3_vec(R_wc, gt_cw, gt_wc);
    for (int i = 0; i < 3; i++) gt_wc[i] = -gt_wc[i];
    double Ret[9], gR_wL[9], gR_e[9], RwLt[9];
    m3_transpose(R_e, Ret);
    m3_mul(gR_wc, Ret, gR_wL);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) gR_wL[3 * i + j] += gt_wc[i] * ext[3 + j];
    m3_transpose(R_wL, RwLt);
    m3_mul(RwLt, gR_wc, gR_e);
    double gt_e[3];
    m3_tvec(R_wL, gt_wc, gt_e);
    double dRe[3][9];
    rodrigues_grad(ext, R_e, dRe);
    for (int k = 0; k < 3; k++) d_ext[k] += m3_dot(gR_e, dRe[k]);
    for (int k = 0; k < 3; k++) d_ext[3 + k] += gt_e[k];
    d_delta[0] += m3_dot(gR_wL, dR_dtau) + gt_wc[0] * dp_dtau[0] + gt_wc[1] * dp_dtau[1] + gt_wc[2] * dp_dtau[2];
    free(g_mean); free(g_conic); free(g_opac); free(suffix);
    blend_free(&B);
    frame_state_free(&S);
}

/* --------------------------------------------------------------- loss -- */

/* Exported: L1 term of the photometric loss (Eq. 4), mean over n values,
 * and its gradient sign(C - C_gt) / n (zero where equal). */
double or_l1(int64_t n, const double *C, const double *Cgt, double *grad) {
    double s = 0;
    for (int64_t i = 0; i < n; i++) {
        double d = C[i] - Cgt[i];
        s += fabs(d);
        if (grad) grad[i] = (d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0)) / (double)n;
    }
    return s / (double)n;
}

/* Exported: the D-SSIM part of the photometric loss (Eq. 4) over a batch of
 * F images and its gradient with respect to the rendered images.
 *
 * Image f is rows x cols x 3 (row-major, channels interleaved) at value
 * offset off[f] in img/tgt/grad.  Per channel and pixel q, with the
 * normalised 11x11 Gaussian window G (sigma 1.5) and zero padding outside
 * the image (Wang et al.'s SSIM as used by 3DGS):
 *   mu_a = sum_p G(p - q) a(p),   mu_b likewise,
 *   s_aa = sum_p G a(p)^2 - mu_a^2,  s_bb likewise,  s_ab = sum_p G a b - mu_a mu_b,
 *   SSIM(q) = (2 mu_a mu_b + C1)(2 s_ab + C2) / ((mu_a^2 + mu_b^2 + C1)(s_aa + s_bb + C2)),
 * C1 = 0.01^2, C2 = 0.03^2.  D-SSIM = 1 - mean of SSIM over all pixels and
 * channels of the batch (n values).  Its gradient follows the chain rule
 * through mu_a, s_aa and s_ab:
 *   d(mean SSIM)/da(p) = (1/n) sum_q G(p - q) [ S_mu(q) + S_aa(q) (2 a(p) - 2 mu_a(q))
 *                                              + S_ab(q) (b(p) - mu_b(q)) ]
 * with S_mu, S_aa, S_ab the partial derivatives of SSIM(q) in mu_a, s_aa,
 * s_ab.  grad (optional) receives d(D-SSIM)/d img; ssim_map (optional)
 * receives SSIM(q) per value.  Returns D-SSIM. */
static void ssim_window(double g[11]) {
    double s = 0;
    for (int i = 0; i < 11; i++) {
        g[i] = exp(-(double)((i - 5) * (i - 5)) / (2.0 * 1.5 * 1.5));
        s += g[i];
    }
    for (int i = 0; i < 11; i++) g[i] /= s;
}

double or_dssim(int F, const int32_t *rows, const int32_t *cols, const int64_t *off, const double *img,
                const double *tgt, double *grad, double *ssim_map) {
    const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
    double g[11];
    ssim_window(g);
    int64_t n = 0;
    for (int f = 0; f < F; f++) n += (int64_t)rows[f] * cols[f] * 3;
    double sum = 0;
    for (int f = 0; f < F; f++) {
        const int H = rows[f], W = cols[f];
        const double *a = img + off[f], *b = tgt + off[f];
        const int64_t m = (int64_t)H * W;
        /* per pixel and channel: S_mu, S_aa, S_ab and mu_a, mu_b */
        double *Smu = malloc(sizeof(double) * m * 3), *Saa = malloc(sizeof(double) * m * 3);
        double *Sab = malloc(sizeof(double) * m * 3), *mua = malloc(sizeof(double) * m * 3);
        double *mub = malloc(sizeof(double) * m * 3);
        for (int y = 0; y < H; y++)
            for (int x = 0; x < W; x++)
                for (int c = 0; c < 3; c++) {
                    double ma = 0, mb = 0, eaa = 0, ebb = 0, eab = 0;
                    for (int dy = -5; dy <= 5; dy++) {
                        const int yy = y + dy;
                        if (yy < 0 || yy >= H) continue;
                        for (int dx = -5; dx <= 5; dx++) {
                            const int xx = x + dx;
                            if (xx < 0 || xx >= W) continue;
                            const double w = g[dy + 5] * g[dx + 5];
                            const double va = a[((int64_t)yy * W + xx) * 3 + c];
                            const double vb = b[((int64_t)yy * W + xx) * 3 + c];
                            ma += w * va;
                            mb += w * vb;
                            eaa += w * va * va;
                            ebb += w * vb * vb;
                            eab += w * va * vb;
                        }
                    }
                    const double saa = eaa - ma * ma, sbb = ebb - mb * mb, sab = eab - ma * mb;
                    const double A = 2 * ma * mb + C1, B = 2 * sab + C2;
                    const double Cc = ma * ma + mb * mb + C1, D = saa + sbb + C2;
                    const double S = (A * B) / (Cc * D);
                    const int64_t i = ((int64_t)y * W + x) * 3 + c;
                    sum += S;
                    if (ssim_map) ssim_map[off[f] + i] = S;
                    Smu[i] = 2 * mb * B / (Cc * D) - 2 * ma * S / Cc;
                    Saa[i] = -S / D;
                    Sab[i] = 2 * A / (Cc * D);
                    mua[i] = ma;
                    mub[i] = mb;
                }
        if (grad) {
            for (int y = 0; y < H; y++)
                for (int x = 0; x < W; x++)
                    for (int c = 0; c < 3; c++) {
                        const int64_t ip = ((int64_t)y * W + x) * 3 + c;
                        double d = 0;
                        for (int dy = -5; dy <= 5; dy++) {
                            const int yy = y + dy;
                            if (yy < 0 || yy >= H) continue;
                            for (int dx = -5; dx <= 5; dx++) {
                                const int xx = x + dx;
                                if (xx < 0 || xx >= W) continue;
                                const int64_t iq = ((int64_t)yy * W + xx) * 3 + c;
                                d += g[dy + 5] * g[dx + 5] *
                                     (Smu[iq] + Saa[iq] * (2 * a[ip] - 2 * mua[iq]) + Sab[iq] * (b[ip] - mub[iq]));
                            }
                        }
                        grad[off[f] + ip] = -d / (double)n;
                    }
        }
        free(Smu);
        free(Saa);
        free(Sab);
        free(mua);
        free(mub);
    }
    return 1.0 - sum / (double)n;
}

/* --------------------------------------------------------- tile binning -- */

typedef struct { uint64_t key; uint32_t val; } or_pair;

static int cmp_pair(const void *a, const void *b) {
    const or_pair *x = a, *y = b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->val > y->val) - (x->val < y->val);
}

/* Exported: tile binning and depth ordering of the per-(frame, Gaussian)
 * records.  Frame f owns records [rec_off[f], rec_off[f+1]) and global
 * tiles [tile_off[f], tile_off[f] + tiles_x[f] * tiles_y[f]).  Each record r
 * with a non-empty rect emits one pair per covered tile:
 *   key = (global tile id << 32) | bit pattern of the float32 depth,
 *   val = r - rec_off[f]   (the Gaussian's index within its scene).
 * Pairs are ordered by key; pairs with equal keys keep their emission order,
 * which is ascending val within a frame, so ordering by (key, val) is the
 * stable order.  ranges[2t], ranges[2t+1] = [start, end) of tile t.
 * Returns the number of pairs, or -1 if it exceeds cap. */
int64_t or_bin_sort(int F, const int64_t *rec_off, const int32_t *tile_off, const int32_t *tiles_x,
                    const int32_t *rect, const float *depth, int64_t cap, int32_t num_tiles,
                    uint64_t *out_keys, uint32_t *out_vals, int64_t *out_ranges) {
    int64_t P = 0;
    for (int f = 0; f < F; f++)
        for (int64_t r = rec_off[f]; r < rec_off[f + 1]; r++) {
            const int32_t *b = rect + 4 * r;
            if (b[0] > b[2] || b[1] > b[3]) continue;
            P += (int64_t)(b[2] - b[0] + 1) * (b[3] - b[1] + 1);
        }
    if (P > cap) return -1;
    or_pair *pairs = (or_pair *)malloc(sizeof(or_pair) * (P > 0 ? P : 1));
    int64_t n = 0;
    for (int f = 0; f < F; f++)
        for (int64_t r = rec_off[f]; r < rec_off[f + 1]; r++) {
            const int32_t *b = rect + 4 * r;
            if (b[0] > b[2] || b[1] > b[3]) continue;
            uint32_t bits;
            memcpy(&bits, &depth[r], 4);
            for (int ty = b[1]; ty <= b[3]; ty++)
                for (int tx = b[0]; tx <= b[2]; tx++) {
                    uint64_t tile = (uint64_t)(tile_off[f] + ty * tiles_x[f] + tx);
                    pairs[n].key = (tile << 32) | bits;
                    pairs[n].val = (uint32_t)(r - rec_off[f]);
                    n++;
                }
        }
    qsort(pairs, P, sizeof(or_pair), cmp_pair);
    for (int64_t t = 0; t < 2 * (int64_t)num_tiles; t++) out_ranges[t] = 0;
    for (int64_t i = 0; i < P; i++) {
        out_keys[i] = pairs[i].key;
        out_vals[i] = pairs[i].val;
        int64_t t = (int64_t)(pairs[i].key >> 32);
        if (i == 0 || (pairs[i - 1].key >> 32) != (uint64_t)t) out_ranges[2 * t] = i;
        if (i == P - 1 || (pairs[i + 1].key >> 32) != (uint64_t)t) out_ranges[2 * t + 1] = i + 1;
    }
    free(pairs);
    return P;
}
