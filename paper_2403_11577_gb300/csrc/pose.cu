// Camera poses of Eq. 1 and the calibration gradient through them.
//
// gs_pose_compose: one thread per frame, double precision.
//   tau = t + delta_i; T_L(tau) from the keyframe segment holding tau:
//   p(tau) = p_k + s (p_{k+1} - p_k);  R(tau) = R_k Exp(s w_k) where
//   w_k = Log(R_k^T R_{k+1}) (the rotation-matrix form of SLERP).
//   Camera-to-world T^n = T_L(tau) [R_e | t_e];  world-to-camera R_cw =
//   (R_L R_e)^T, camera centre c = R_L t_e + p.  Stored in float with R_cw
//   and c each split into hi + lo floats, so that the projection can form
//   R_cw (X - c) in float-float arithmetic and round the depth and the 2D
//   mean once.
//   The time-offset gradient needs the camera-frame velocity twist
//   nu = Ad(T_e^-1) eta, eta = (R_L^T p_dot, w_k / dt) the LiDAR body twist:
//   nu = (R_e^T (v + w x t_e), R_e^T w).
//
// gs_pose_grad: sums, per camera, the per-frame twist gradients g_eps (left
// perturbation T_cw <- Exp(eps) T_cw, eps = (rho, phi)) and maps them:
//   right perturbation of the extrinsic xi:   dL/dxi = -g_eps
//   parameters (omega, t_e):  dL/dt_e = -R_e g_rho,  dL/domega = -J_r(omega)^T g_phi
//   time offset:              dL/ddelta = -nu . g_eps
#include "common.cuh"

namespace gs {

namespace {

__device__ void m3mul(const double *A, const double *B, double *C) {
    double T[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            T[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
    for (int i = 0; i < 9; i++) C[i] = T[i];
}

// R = Exp([w]x) with the series form near zero.
__device__ void so3_exp(const double *w, double *R) {
    double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double th = sqrt(th2);
    double A, B;
    if (th < 1e-6) {
        A = 1.0 - th2 / 6.0;
        B = 0.5 - th2 / 24.0;
    } else {
        A = sin(th) / th;
        B = (1.0 - cos(th)) / th2;
    }
    double x = w[0], y = w[1], z = w[2];
    R[0] = 1 - B * (y * y + z * z); R[1] = -A * z + B * x * y;     R[2] = A * y + B * x * z;
    R[3] = A * z + B * x * y;       R[4] = 1 - B * (x * x + z * z); R[5] = -A * x + B * y * z;
    R[6] = -A * y + B * x * z;      R[7] = A * x + B * y * z;       R[8] = 1 - B * (x * x + y * y);
}

// Right Jacobian of SO(3): J_r(w) = I - (1-cos)/th^2 [w]x + (th-sin)/th^3 [w]x^2.
__device__ void so3_right_jacobian(const double *w, double *J) {
    double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double th = sqrt(th2);
    double a, b;
    if (th < 1e-6) {
        a = 0.5 - th2 / 24.0;
        b = 1.0 / 6.0 - th2 / 120.0;
    } else {
        a = (1.0 - cos(th)) / th2;
        b = (th - sin(th)) / (th2 * th);
    }
    double K[9] = {0, -w[2], w[1], w[2], 0, -w[0], -w[1], w[0], 0};
    double K2[9];
    m3mul(K, K, K2);
    for (int i = 0; i < 9; i++) J[i] = (i % 4 == 0 ? 1.0 : 0.0) - a * K[i] + b * K2[i];
}

// Rotation matrix of a quaternion (normalised here).
__device__ void quat_rot(const double *q, double *R) {
    double n = rsqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double w = q[0] * n, x = q[1] * n, y = q[2] * n, z = q[3] * n;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

// Rotation vector of the relative rotation q_a^-1 q_b (shortest arc).
__device__ void quat_rel_log(const double *qa, const double *qb, double *w) {
    double na = rsqrt(qa[0] * qa[0] + qa[1] * qa[1] + qa[2] * qa[2] + qa[3] * qa[3]);
    double nb = rsqrt(qb[0] * qb[0] + qb[1] * qb[1] + qb[2] * qb[2] + qb[3] * qb[3]);
    double aw = qa[0] * na, ax = -qa[1] * na, ay = -qa[2] * na, az = -qa[3] * na;  // conj(qa)
    double bw = qb[0] * nb, bx = qb[1] * nb, by = qb[2] * nb, bz = qb[3] * nb;
    double rw = aw * bw - ax * bx - ay * by - az * bz;
    double rx = aw * bx + ax * bw + ay * bz - az * by;
    double ry = aw * by - ax * bz + ay * bw + az * bx;
    double rz = aw * bz + ax * by - ay * bx + az * bw;
    if (rw < 0) { rw = -rw; rx = -rx; ry = -ry; rz = -rz; }
    double vn = sqrt(rx * rx + ry * ry + rz * rz);
    double f = vn < 1e-12 ? 2.0 / rw : 2.0 * atan2(vn, rw) / vn;
    w[0] = f * rx; w[1] = f * ry; w[2] = f * rz;
}

__global__ void k_pose_compose(const gs_frame *__restrict__ frames, int F, const double *__restrict__ traj_t,
                               const double *__restrict__ traj_pose, const int32_t *__restrict__ traj_off,
                               const double *__restrict__ ext, const double *__restrict__ delta,
                               float *__restrict__ pose32, double *__restrict__ pose64) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    const gs_frame fr = frames[f];
    const int cam = fr.camera_id;
    const int k0 = traj_off[fr.traj_id], K = traj_off[fr.traj_id + 1] - k0;
    const double tau = fr.timestamp + delta[cam];
    double R_L[9], p[3], v_world[3] = {0, 0, 0}, w_body[3] = {0, 0, 0};
    if (K < 1) {  // no keyframes: identity LiDAR pose
        for (int i = 0; i < 9; i++) R_L[i] = (i % 4 == 0) ? 1.0 : 0.0;
        for (int i = 0; i < 3; i++) p[i] = 0.0;
    } else if (K == 1) {
        quat_rot(traj_pose + 7 * k0 + 3, R_L);
        for (int i = 0; i < 3; i++) p[i] = traj_pose[7 * k0 + i];
    } else {
        int lo = 0, hi = K - 2;  // last segment start <= tau, clamped to [0, K-2]
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (traj_t[k0 + mid] <= tau) lo = mid; else hi = mid - 1;
        }
        const int k = k0 + lo;
        const double dt = traj_t[k + 1] - traj_t[k];
        const double s = (tau - traj_t[k]) / dt;
        const double *P0 = traj_pose + 7 * k, *P1 = traj_pose + 7 * (k + 1);
        for (int i = 0; i < 3; i++) {
            p[i] = P0[i] + s * (P1[i] - P0[i]);
            v_world[i] = (P1[i] - P0[i]) / dt;
        }
        double wk[3], sw[3], Rk[9], Es[9];
        quat_rel_log(P0 + 3, P1 + 3, wk);
        for (int i = 0; i < 3; i++) { sw[i] = s * wk[i]; w_body[i] = wk[i] / dt; }
        quat_rot(P0 + 3, Rk);
        so3_exp(sw, Es);
        m3mul(Rk, Es, R_L);
    }
    const double *e = ext + 6 * cam;
    double R_e[9], R_wc[9];
    so3_exp(e, R_e);
    m3mul(R_L, R_e, R_wc);
    double c[3];
    for (int i = 0; i < 3; i++)
        c[i] = R_L[3 * i] * e[3] + R_L[3 * i + 1] * e[4] + R_L[3 * i + 2] * e[5] + p[i];
    // nu = (R_e^T (v + w x t_e), R_e^T w), v = R_L^T v_world
    double v[3], wxt[3], a[3];
    for (int i = 0; i < 3; i++) v[i] = R_L[i] * v_world[0] + R_L[3 + i] * v_world[1] + R_L[6 + i] * v_world[2];
    wxt[0] = w_body[1] * e[5] - w_body[2] * e[4];
    wxt[1] = w_body[2] * e[3] - w_body[0] * e[5];
    wxt[2] = w_body[0] * e[4] - w_body[1] * e[3];
    for (int i = 0; i < 3; i++) a[i] = v[i] + wxt[i];
    float *o32 = pose32 + kPose32Stride * f;
    double *o64 = pose64 + kPose64Stride * f;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double r = R_wc[3 * j + i];  // R_cw = R_wc^T
            const float hi = (float)r;
            o32[3 * i + j] = hi;
            o32[kPoseRlo + 3 * i + j] = (float)(r - (double)hi);
            o64[3 * i + j] = r;
        }
    for (int i = 0; i < 3; i++) {
        float hi = (float)c[i];
        o32[9 + i] = hi;
        o32[12 + i] = (float)(c[i] - (double)hi);
        o64[9 + i] = c[i];
        o64[12 + i] = R_e[i] * a[0] + R_e[3 + i] * a[1] + R_e[6 + i] * a[2];                  // nu_rho
        o64[15 + i] = R_e[i] * w_body[0] + R_e[3 + i] * w_body[1] + R_e[6 + i] * w_body[2];   // nu_phi
    }
    o32[15] = 0.f;
    for (int i = kPoseRlo + 9; i < kPose32Stride; i++) o32[i] = 0.f;
    for (int i = 0; i < 9; i++) o64[18 + i] = R_e[i];
    for (int i = 27; i < kPose64Stride; i++) o64[i] = 0.0;
}

// The frame's twist from its per-warp partials, in FP64 and a fixed order
// (deterministic): block (f, s) sums slice s of the partials into mid, then
// one thread per (frame, component) sums the slices.
constexpr int kTwistSlices = 32;

__global__ void __launch_bounds__(256)
k_twist_reduce(int nparts, const double *__restrict__ twist_part, double *__restrict__ mid) {
    __shared__ double red[256 / 32][6];
    const int f = blockIdx.x, sl = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int per = (nparts + kTwistSlices - 1) / kTwistSlices;
    const int lo = min(sl * per, nparts), hi = min(lo + per, nparts);
    double g[6] = {0, 0, 0, 0, 0, 0};
    for (int b = lo + threadIdx.x; b < hi; b += blockDim.x) {
        const double *src = twist_part + ((size_t)f * nparts + b) * 6;
        for (int i = 0; i < 6; i++) g[i] += src[i];
    }
    for (int i = 0; i < 6; i++)
        for (int s = 16; s > 0; s >>= 1) g[i] += __shfl_xor_sync(0xffffffffu, g[i], s);
    if (lane == 0)
        for (int i = 0; i < 6; i++) red[warp][i] = g[i];
    __syncthreads();
    if (threadIdx.x < 6) {
        double s = 0;
        for (int w = 0; w < 256 / 32; w++) s += red[w][threadIdx.x];
        mid[((size_t)f * kTwistSlices + sl) * 6 + threadIdx.x] = s;
    }
}

__global__ void k_twist_final(int F, const double *__restrict__ mid, double *__restrict__ g_eps) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 6 * F) return;
    const int f = k / 6, i = k % 6;
    double s = 0;
    for (int sl = 0; sl < kTwistSlices; sl++) s += mid[((size_t)f * kTwistSlices + sl) * 6 + i];
    g_eps[k] = s;
}

// One thread per camera: sum the twists of the camera's frames and map them
// to the parameter gradients.
__global__ void k_pose_grad(const gs_frame *__restrict__ frames, int F, int C, const double *__restrict__ g_eps,
                            const double *__restrict__ pose64, const double *__restrict__ ext,
                            double *__restrict__ d_ext, double *__restrict__ d_delta, double *__restrict__ d_xi,
                            bool acc) {
    const int cam = blockIdx.x * blockDim.x + threadIdx.x;
    if (cam >= C) return;
    double g[7] = {0, 0, 0, 0, 0, 0, 0};  // g_eps (6) and -nu . g_eps
    for (int f = 0; f < F; f++) {
        if (frames[f].camera_id != cam) continue;
        const double *ge = g_eps + 6 * f;
        const double *nu = pose64 + kPose64Stride * f + 12;
        for (int i = 0; i < 6; i++) {
            g[i] += ge[i];
            g[6] -= nu[i] * ge[i];
        }
    }
    const double *e = ext + 6 * cam;
    double R_e[9], Jr[9];
    so3_exp(e, R_e);
    so3_right_jacobian(e, Jr);
    auto put = [acc](double *dst, double v) { *dst = acc ? *dst + v : v; };
    for (int i = 0; i < 3; i++) {
        // dL/dt_e = -R_e g_rho ; dL/domega = -J_r^T g_phi
        put(d_ext + 6 * cam + 3 + i, -(R_e[3 * i] * g[0] + R_e[3 * i + 1] * g[1] + R_e[3 * i + 2] * g[2]));
        put(d_ext + 6 * cam + i, -(Jr[i] * g[3] + Jr[3 + i] * g[4] + Jr[6 + i] * g[5]));
    }
    put(d_delta + cam, g[6]);
    if (d_xi)
        for (int i = 0; i < 6; i++) put(d_xi + 6 * cam + i, -g[i]);
}

}  // namespace

cudaError_t launch_pose_compose(const gs_batch *b, const double *traj_t, const double *traj_pose,
                                const int32_t *traj_off, const double *ext, const double *delta,
                                float *pose32, double *pose64, cudaStream_t s) {
    int F = b->num_frames;
    k_pose_compose<<<(F + 63) / 64, 64, 0, s>>>(b->frames_dev, F, traj_t, traj_pose, traj_off, ext,
                                                 delta, pose32, pose64);
    return cudaGetLastError();
}

cudaError_t launch_pose_grad(const gs_batch *b, int nparts, const double *twist_part, double *twist_mid,
                             double *g_eps,
                             const double *pose64, const double *ext, double *d_ext, double *d_delta,
                             double *d_xi, bool acc, cudaStream_t s) {
    k_twist_reduce<<<dim3(b->num_frames, kTwistSlices), 256, 0, s>>>(nparts, twist_part, twist_mid);
    k_twist_final<<<(6 * b->num_frames + 255) / 256, 256, 0, s>>>(b->num_frames, twist_mid, g_eps);
    const int C = b->num_cameras;
    k_pose_grad<<<(C + 31) / 32, 32, 0, s>>>(b->frames_dev, b->num_frames, C, g_eps, pose64, ext, d_ext, d_delta,
                                             d_xi, acc);
    return cudaGetLastError();
}

}  // namespace gs
