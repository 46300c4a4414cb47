// EWA projection of the Gaussians (Eq. 2-3 and the projection step of Phi,
// Eq. 5) and its backward.
//
// Layout: one thread per Gaussian of the whole batch; the thread reads the
// Gaussian's parameters once (44 bytes) and loops over the frames of its
// scene, writing one record per frame.  Frame-dependent work uses
//   p = R_cw (X - c)        (Eq. 2: X^n = (T^n)^-1 X), formed in float-float
//                           arithmetic from R_cw and c given as hi + lo
//                           floats; the depth p.z and the 2D mean are each
//                           rounded once, so they are the floats nearest to
//                           their exact values (the depth key and the culling
//                           at the near plane are decided on that float),
//   T = J R_cw              (J: Jacobian of the pinhole map at p, with x/z
//                            and y/z limited to the widened field of view),
//   cov = T Sigma T^T + lowpass I   (= J Sigma_c J^T, Sigma_c of Eq. 3),
// with Sigma = R_g diag(s)^2 R_g^T built once per Gaussian.
//
// Record outputs (frame f, Gaussian g -> record r):
//   rect[r]   tiles [x0,x1]x[y0,y1] where alpha >= alpha_min is possible
//             (tile rows counted from the frame's first rendered row, row0):
//             the box of the ellipse d^T conic d <= 2 ln(opacity/alpha_min),
//             half-widths sqrt(k cov_xx), sqrt(k cov_yy), widened by a
//             relative 1e-4 and 0.01 px against float32 rounding;
//   depth[r]  camera depth p.z, the float nearest to its exact value;
//   splat[r]  (mean_x, mean_y, A, B), (C, F, rx, ry) with the exponent in
//             base 2: log2 alpha = A dx^2 + B dx dy + C dy^2 + F,
//             A = -a/2 log2 e, B = -b log2 e, C = -c/2 log2 e, F = log2 opacity,
//             (a, b, c) the conic, and (rx, ry) the guarded half-widths of the
//             box outside which alpha < alpha_min (the rect's extents, in px);
//   grad2d[r] zeroed for visible records (the render backward accumulates
//             into it).
#include "common.cuh"

namespace gs {

namespace {

struct GaussParams {
    float X[3];
    float q[4];       // normalised
    float qn;         // norm of the input quaternion
    float Rg[9];
    float s[3];
    bool s_clamped[3];
    float Sig[6];     // xx, xy, xz, yy, yz, zz
    float o, F, kext; // opacity, log2 opacity, 2 ln(opacity / alpha_min)
};

__device__ __forceinline__ void load_gauss(int g, const float *__restrict__ X, const float *__restrict__ quat,
                                           const float *__restrict__ log_s, const float *__restrict__ logit_o,
                                           const gs_opts &o, GaussParams &G) {
    G.X[0] = X[3 * g]; G.X[1] = X[3 * g + 1]; G.X[2] = X[3 * g + 2];
    float qw = quat[4 * g], qx = quat[4 * g + 1], qy = quat[4 * g + 2], qz = quat[4 * g + 3];
    float n2 = qw * qw + qx * qx + qy * qy + qz * qz;
    float inv = rsqrtf(n2);
    G.qn = n2 * inv;
    qw *= inv; qx *= inv; qy *= inv; qz *= inv;
    G.q[0] = qw; G.q[1] = qx; G.q[2] = qy; G.q[3] = qz;
    float *R = G.Rg;
    R[0] = 1.f - 2.f * (qy * qy + qz * qz); R[1] = 2.f * (qx * qy - qw * qz); R[2] = 2.f * (qx * qz + qw * qy);
    R[3] = 2.f * (qx * qy + qw * qz); R[4] = 1.f - 2.f * (qx * qx + qz * qz); R[5] = 2.f * (qy * qz - qw * qx);
    R[6] = 2.f * (qx * qz - qw * qy); R[7] = 2.f * (qy * qz + qw * qx); R[8] = 1.f - 2.f * (qx * qx + qy * qy);
    for (int i = 0; i < 3; i++) {
        float s = expf(log_s[3 * g + i]);
        G.s_clamped[i] = s > o.scale_max;
        G.s[i] = G.s_clamped[i] ? o.scale_max : s;
    }
    // Sigma = M M^T with M = R_g diag(s)
    float M[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) M[3 * i + j] = R[3 * i + j] * G.s[j];
    G.Sig[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    G.Sig[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    G.Sig[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    G.Sig[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    G.Sig[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    G.Sig[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
    float lo = logit_o[g];
    G.o = 1.f / (1.f + expf(-lo));
    G.F = log2f(G.o);
    G.kext = 2.f * kLn2 * (G.F - log2f(o.alpha_min));
}

// Frame-dependent projection.  Returns false if culled.
struct Proj {
    float p[3], iz, xz, yz;   // camera-frame centre, 1/z, x/z, y/z
    float jx, jy;             // x/z, y/z as used in J (clamped to the widened view)
    bool clx, cly;            // whether they were clamped
    float T[6];               // J R_cw
    float U[6];               // T Sigma
    float cov[3];             // xx, xy, yy (with low-pass)
    float conic[3];           // a, b, c
    float mean[2];
};

// Camera-frame centre p = R_cw (X - c) (Eq. 2) in float-float arithmetic.
// R_cw and c come as hi + lo floats; X - c_hi is split exactly (two_sum),
// each product R_ij d_j is kept exactly to first order (two_prod plus the
// cross terms) and the sums are carried with their rounding errors, so that
// p_i = ph_i + pl_i is within a few 2^-48 sum_j |R_ij| |d_j| of the exact
// value for the float inputs X and the double pose.  ph_i is that sum
// rounded once, so the depth ph_2 is the float nearest to the exact depth
// (unless the exact depth lies within that error of a rounding boundary).
__device__ __forceinline__ void camera_point(const float (&X)[3], const float *__restrict__ P, float (&ph)[3],
                                             float (&pl)[3]) {
    float dh[3], dl[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        float e;
        two_sum(X[k], -P[9 + k], dh[k], e);
        dl[k] = __fsub_rn(e, P[12 + k]);
    }
#pragma unroll
    for (int i = 0; i < 3; i++) {
        float sh = 0.f, sl = 0.f;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const float rh = P[3 * i + k], rl = P[kPoseRlo + 3 * i + k];
            float pr, pe, te;
            two_prod(rh, dh[k], pr, pe);
            pe = __fadd_rn(pe, __fmaf_rn(rh, dl[k], __fmul_rn(rl, dh[k])));
            two_sum(sh, pr, sh, te);
            sl = __fadd_rn(sl, __fadd_rn(te, pe));
        }
        two_sum(sh, sl, ph[i], pl[i]);
    }
}

// (xh + xl) / (zh + zl) as q + ql, to a few 2^-48 relative, from an
// approximate reciprocal iz of zh: q = xh iz is off by a few 2^-24; its
// residual xh - q zh (one fma), plus the low parts, times iz is the
// correction, whose own error is of second order.
__device__ __forceinline__ void ff_div(float xh, float xl, float zh, float zl, float iz, float &q, float &ql) {
    q = __fmul_rn(xh, iz);
    float r = __fmaf_rn(-q, zh, xh);
    r = __fadd_rn(r, __fmaf_rn(-q, zl, xl));
    ql = __fmul_rn(r, iz);
}

// f (q + ql) + c rounded once (two_prod and two_sum keep the parts exact).
__device__ __forceinline__ float ff_affine(float f, float q, float ql, float c) {
    float a, ae, sh, se;
    two_prod(f, q, a, ae);
    ae = __fmaf_rn(f, ql, ae);
    two_sum(a, c, sh, se);
    return __fadd_rn(sh, __fadd_rn(se, ae));
}

// kExact (the forward): p in float-float, the depth key and the 2D mean
// rounded once, culling at the near plane on the key.  Otherwise (the
// backward, whose records were kept by the forward's rectangles): p in plain
// float arithmetic, no near-plane test and no mean; every quantity the
// gradient needs (J, the covariance, the conic) to float accuracy.
template <bool kExact>
__device__ __forceinline__ bool project_frame(const GaussParams &G, const float *__restrict__ P,
                                              const gs_frame &fr, const gs_opts &o, Proj &Q) {
    float pl[3] = {0.f, 0.f, 0.f};
    if (kExact) {
        camera_point(G.X, P, Q.p, pl);
    } else {
        const float d0 = (G.X[0] - P[9]) - P[12], d1 = (G.X[1] - P[10]) - P[13], d2 = (G.X[2] - P[11]) - P[14];
        for (int i = 0; i < 3; i++) Q.p[i] = P[3 * i] * d0 + P[3 * i + 1] * d1 + P[3 * i + 2] * d2;
    }
    // the depth key is the float nearest to the exact depth: the culling
    // at the near plane and the depth order are decided on it
    const float z = Q.p[2];
    if (kExact ? !(z > o.near_z) : !(z > 0.f)) return false;
    Q.iz = rcp_approx(z);
    float xl = 0.f, yl = 0.f;
    if (kExact) {
        ff_div(Q.p[0], pl[0], z, pl[2], Q.iz, Q.xz, xl);
        ff_div(Q.p[1], pl[1], z, pl[2], Q.iz, Q.yz, yl);
    } else {
        Q.xz = Q.p[0] * Q.iz;
        Q.yz = Q.p[1] * Q.iz;
    }
    // J at x/z, y/z limited to the field of view widened by frustum_margin
    // of the image size per side (bounds the footprint of far off-image centres)
    Q.jx = Q.xz;
    Q.jy = Q.yz;
    Q.clx = Q.cly = false;
    if (o.frustum_margin >= 0.f) {
        const float mx = o.frustum_margin * (float)fr.width, my = o.frustum_margin * (float)fr.height;
        const float xlo = -(fr.cx + mx) / fr.fx, xhi = ((float)fr.width - fr.cx + mx) / fr.fx;
        const float ylo = -(fr.cy + my) / fr.fy, yhi = ((float)fr.height - fr.cy + my) / fr.fy;
        Q.jx = fminf(fmaxf(Q.xz, xlo), xhi);
        Q.jy = fminf(fmaxf(Q.yz, ylo), yhi);
        Q.clx = Q.jx != Q.xz;
        Q.cly = Q.jy != Q.yz;
    }
    float fxz = fr.fx * Q.iz, fyz = fr.fy * Q.iz;
    for (int j = 0; j < 3; j++) {
        Q.T[j] = fxz * (P[j] - Q.jx * P[6 + j]);
        Q.T[3 + j] = fyz * (P[3 + j] - Q.jy * P[6 + j]);
    }
    const float *S = G.Sig;
    for (int r = 0; r < 2; r++) {
        const float *t = Q.T + 3 * r;
        Q.U[3 * r + 0] = t[0] * S[0] + t[1] * S[1] + t[2] * S[2];
        Q.U[3 * r + 1] = t[0] * S[1] + t[1] * S[3] + t[2] * S[4];
        Q.U[3 * r + 2] = t[0] * S[2] + t[1] * S[4] + t[2] * S[5];
    }
    Q.cov[0] = Q.U[0] * Q.T[0] + Q.U[1] * Q.T[1] + Q.U[2] * Q.T[2] + o.lowpass;
    Q.cov[1] = Q.U[0] * Q.T[3] + Q.U[1] * Q.T[4] + Q.U[2] * Q.T[5];
    Q.cov[2] = Q.U[3] * Q.T[3] + Q.U[4] * Q.T[4] + Q.U[5] * Q.T[5] + o.lowpass;
    float det = Q.cov[0] * Q.cov[2] - Q.cov[1] * Q.cov[1];
    if (!(det > 0.f) || !isfinite(det)) return false;
    float idet = 1.f / det;
    Q.conic[0] = Q.cov[2] * idet;
    Q.conic[1] = -Q.cov[1] * idet;
    Q.conic[2] = Q.cov[0] * idet;
    if (!kExact) return true;
    // the 2D mean, rounded once from fx x/z + cx, fy y/z + cy
    Q.mean[0] = ff_affine(fr.fx, Q.xz, xl, fr.cx);
    Q.mean[1] = ff_affine(fr.fy, Q.yz, yl, fr.cy);
    return isfinite(Q.mean[0]) && isfinite(Q.mean[1]);
}

constexpr uint32_t kEmptyLo = 1u | (1u << 16);  // x0 = y0 = 1
constexpr uint32_t kEmptyHi = 0u;               // x1 = y1 = 0

__device__ __forceinline__ int clamp_tile(float v, int n) {
    // floor(v) clamped to [-1, n] before the integer conversion
    v = fminf(fmaxf(v, -1.f), (float)n);
    return (int)floorf(v);
}

__global__ void __launch_bounds__(kProjThreads)
k_project(const gs_frame *__restrict__ frames, int F, int N, const float *__restrict__ pose32,
          const float *__restrict__ X, const float *__restrict__ quat, const float *__restrict__ log_s,
          const float *__restrict__ logit_o, gs_opts o, uint2 *__restrict__ rect, float *__restrict__ depth,
          float4 *__restrict__ splat, float4 *__restrict__ grad2d, Stats *__restrict__ stats) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= N) return;
    GaussParams G;
    load_gauss(g, X, quat, log_s, logit_o, o, G);
    // non-finite parameters: cull the Gaussian and report it
    bool nonfinite = !(isfinite(G.X[0]) && isfinite(G.X[1]) && isfinite(G.X[2]) && isfinite(G.Sig[0]) &&
                       isfinite(G.Sig[3]) && isfinite(G.Sig[5]) && isfinite(G.F));
    const bool opaque_enough = !nonfinite && G.o >= o.alpha_min;
    const float tile = (float)o.tile, itile = 1.f / tile;
    for (int f = 0; f < F; f++) {
        const gs_frame &fr = frames[f];
        if (g < fr.gauss_offset || g >= fr.gauss_offset + fr.gauss_count) continue;
        const long long r = fr.record_offset + (g - fr.gauss_offset);
        Proj Q;
        bool vis = opaque_enough && project_frame<true>(G, pose32 + kPose32Stride * f, fr, o, Q);
        uint2 rc = make_uint2(kEmptyLo, kEmptyHi);
        if (vis) {
            float rx = sqrtf(G.kext * Q.cov[0]) * 1.0001f + 0.01f;
            float ry = sqrtf(G.kext * Q.cov[2]) * 1.0001f + 0.01f;
            if (!isfinite(rx) || !isfinite(ry)) { nonfinite = true; vis = false; }
            if (vis) {
                int x0 = max(clamp_tile((Q.mean[0] - rx) * itile, fr.tiles_x), 0);
                int x1 = min(clamp_tile((Q.mean[0] + rx) * itile, fr.tiles_x), fr.tiles_x - 1);
                const float my = Q.mean[1] - (float)fr.row0;  // tile rows start at the crop's first row
                int y0 = max(clamp_tile((my - ry) * itile, fr.tiles_y), 0);
                int y1 = min(clamp_tile((my + ry) * itile, fr.tiles_y), fr.tiles_y - 1);
                if (x0 <= x1 && y0 <= y1) {
                    rc = make_uint2((uint32_t)x0 | ((uint32_t)y0 << 16), (uint32_t)x1 | ((uint32_t)y1 << 16));
                    const float s2 = -0.5f * kLog2e;
                    splat[2 * r] = make_float4(Q.mean[0], Q.mean[1], s2 * Q.conic[0], -kLog2e * Q.conic[1]);
                    splat[2 * r + 1] = make_float4(s2 * Q.conic[2], G.F, rx, ry);
                    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
                    grad2d[3 * r] = z4;
                    grad2d[3 * r + 1] = z4;
                    grad2d[3 * r + 2] = z4;
                }
            }
        }
        rect[r] = rc;
        depth[r] = rect_count(rc) ? Q.p[2] : INFINITY;  // +inf: culled (the sort drops it)
    }
    if (nonfinite) atomicOr(&stats->status, (unsigned)GS_DEV_NONFINITE);
}

// ---------------------------------------------------------------- backward

// Sum of six per-lane values over the warp, transposed: the first three
// butterfly steps halve the values each lane carries (8 slots, the last two
// zero), the last two finish the sum.  Lane L returns the total of value
// L / 4 (0..7).
__device__ __forceinline__ float warp_sum6(const float (&v)[6], int lane) {
    const float z[8] = {v[0], v[1], v[2], v[3], v[4], v[5], 0.f, 0.f};
    const bool b16 = lane & 16, b8 = lane & 8, b4 = lane & 4;
    float a[4];
#pragma unroll
    for (int i = 0; i < 4; i++) a[i] = (b16 ? z[i + 4] : z[i]) + __shfl_xor_sync(0xffffffffu, b16 ? z[i] : z[i + 4], 16);
    float c[2];
#pragma unroll
    for (int i = 0; i < 2; i++) c[i] = (b8 ? a[i + 2] : a[i]) + __shfl_xor_sync(0xffffffffu, b8 ? a[i] : a[i + 2], 8);
    float y = (b4 ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, b4 ? c[0] : c[1], 4);
    y += __shfl_xor_sync(0xffffffffu, y, 2);
    y += __shfl_xor_sync(0xffffffffu, y, 1);
    return y;
}

// Chain the per-record 2D gradients back to the Gaussian parameters (summed
// over frames) and to the per-frame camera twist g_eps = (rho, phi) of the
// left perturbation T_cw <- Exp(eps) T_cw:
//   g_rho = sum dL/dp,  g_phi = sum p x dL/dp + axial(R_cw (dL/dT)^T J),
// where axial(M) = (M12 - M21, M20 - M02, M01 - M10) is the vector with
// tr(M [phi]x) = phi . axial(M).
template <int NT>
__global__ void __launch_bounds__(NT)
k_project_bwd(const gs_frame *__restrict__ frames, int F, int N, const float *__restrict__ pose32,
              const float *__restrict__ X, const float *__restrict__ quat, const float *__restrict__ log_s,
              const float *__restrict__ logit_o, gs_opts o, const uint2 *__restrict__ rect,
              const float4 *__restrict__ grad2d, float *__restrict__ d_quat, float *__restrict__ d_log_s,
              float *__restrict__ d_logit, float *__restrict__ d_col, double *__restrict__ twist_part,
              int nparts, bool acc) {
    const int g = blockIdx.x * NT + threadIdx.x;
    const bool active = g < N;
    GaussParams G;
    if (active) load_gauss(g, X, quat, log_s, logit_o, o, G);
    float dSig[6] = {0, 0, 0, 0, 0, 0};
    float dF = 0.f, dc0 = 0.f, dc1 = 0.f, dc2 = 0.f;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int f = 0; f < F; f++) {
        const gs_frame &fr = frames[f];
        float tw[6] = {0, 0, 0, 0, 0, 0};
        bool mine = active && g >= fr.gauss_offset && g < fr.gauss_offset + fr.gauss_count;
        if (mine) {
            const long long r = fr.record_offset + (g - fr.gauss_offset);
            uint2 rc = rect[r];
            bool vis = (rc.x & 0xffffu) <= (rc.y & 0xffffu);
            Proj Q;
            const float *P = pose32 + kPose32Stride * f;
            if (vis && project_frame<false>(G, P, fr, o, Q)) {
                float4 g0 = grad2d[3 * r], g1 = grad2d[3 * r + 1], g2 = grad2d[3 * r + 2];
                dc0 += g1.z; dc1 += g1.w; dc2 += g2.x;
                dF += g1.y;
                // stored exponent coefficients -> conic (a, b, c)
                const float ga = g0.z * (-0.5f * kLog2e), gb = g0.w * (-kLog2e), gc = g1.x * (-0.5f * kLog2e);
                const float a = Q.conic[0], b = Q.conic[1], c = Q.conic[2];
                // conic = cov^-1 -> cov (xx, xy, yy); xy appears once in cov
                const float gxx = -(a * a * ga + a * b * gb + b * b * gc);
                const float gxy = -(2.f * a * b * ga + (a * c + b * b) * gb + 2.f * b * c * gc);
                const float gyy = -(b * b * ga + b * c * gb + c * c * gc);
                // H = dL/dcov as a symmetric 2x2
                const float h00 = gxx, h01 = 0.5f * gxy, h11 = gyy;
                float HT[6];
                for (int j = 0; j < 3; j++) {
                    HT[j] = h00 * Q.T[j] + h01 * Q.T[3 + j];
                    HT[3 + j] = h01 * Q.T[j] + h11 * Q.T[3 + j];
                }
                // G = dL/dSigma = T^T H T, a full symmetric matrix (six entries kept)
                dSig[0] += Q.T[0] * HT[0] + Q.T[3] * HT[3];
                dSig[1] += Q.T[0] * HT[1] + Q.T[3] * HT[4];
                dSig[2] += Q.T[0] * HT[2] + Q.T[3] * HT[5];
                dSig[3] += Q.T[1] * HT[1] + Q.T[4] * HT[4];
                dSig[4] += Q.T[1] * HT[2] + Q.T[4] * HT[5];
                dSig[5] += Q.T[2] * HT[2] + Q.T[5] * HT[5];
                // dL/dT = 2 H U (U = T Sigma)
                float dT[6];
                for (int j = 0; j < 3; j++) {
                    dT[j] = 2.f * (h00 * Q.U[j] + h01 * Q.U[3 + j]);
                    dT[3 + j] = 2.f * (h01 * Q.U[j] + h11 * Q.U[3 + j]);
                }
                // dL/dJ = dL/dT R_cw^T (only the non-zero entries of J)
                float dJ00 = dT[0] * P[0] + dT[1] * P[1] + dT[2] * P[2];
                float dJ02 = dT[0] * P[6] + dT[1] * P[7] + dT[2] * P[8];
                float dJ11 = dT[3] * P[3] + dT[4] * P[4] + dT[5] * P[5];
                float dJ12 = dT[3] * P[6] + dT[4] * P[7] + dT[5] * P[8];
                const float iz = Q.iz, iz2 = iz * iz;
                const float fx = fr.fx, fy = fr.fy;
                const float gmx = g0.x, gmy = g0.y;
                // J00 = fx/z, J02 = -fx jx/z, J11 = fy/z, J12 = -fy jy/z, with
                // jx = x/z (jy = y/z) unless clamped, where it is a constant
                const float dJ02_dx = Q.clx ? 0.f : -fx * iz2, dJ12_dy = Q.cly ? 0.f : -fy * iz2;
                const float dJ02_dz = Q.clx ? fx * Q.jx * iz2 : 2.f * fx * Q.xz * iz2;
                const float dJ12_dz = Q.cly ? fy * Q.jy * iz2 : 2.f * fy * Q.yz * iz2;
                float dp[3];
                dp[0] = dJ02_dx * dJ02 + fx * iz * gmx;
                dp[1] = dJ12_dy * dJ12 + fy * iz * gmy;
                dp[2] = -fx * iz2 * dJ00 + dJ02_dz * dJ02 - fy * iz2 * dJ11 + dJ12_dz * dJ12 -
                        fx * Q.xz * iz * gmx - fy * Q.yz * iz * gmy;
                // twist: rotation part through T = J R_cw: M = R_cw N, N = dT^T J
                float J00 = fx * iz, J02 = -fx * Q.jx * iz, J11 = fy * iz, J12 = -fy * Q.jy * iz;
                float Nm[9];
                for (int i = 0; i < 3; i++) {
                    Nm[3 * i + 0] = dT[i] * J00;
                    Nm[3 * i + 1] = dT[3 + i] * J11;
                    Nm[3 * i + 2] = dT[i] * J02 + dT[3 + i] * J12;
                }
                float Mm[9];
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++)
                        Mm[3 * i + j] = P[3 * i] * Nm[j] + P[3 * i + 1] * Nm[3 + j] + P[3 * i + 2] * Nm[6 + j];
                const float *p = Q.p;
                tw[0] = dp[0];
                tw[1] = dp[1];
                tw[2] = dp[2];
                tw[3] = (p[1] * dp[2] - p[2] * dp[1]) + (Mm[5] - Mm[7]);
                tw[4] = (p[2] * dp[0] - p[0] * dp[2]) + (Mm[6] - Mm[2]);
                tw[5] = (p[0] * dp[1] - p[1] * dp[0]) + (Mm[1] - Mm[3]);
            }
        }
        // the frame's twist summed over the warp in float (32 terms, a fixed
        // order), one FP64 partial per (frame, warp): no block barrier, so
        // the next frame's loads overlap this one's reduction (GB300's FP64
        // rate is low, so only the per-warp partials are widened)
        const float tot = warp_sum6(tw, lane);
        if ((lane & 3) == 0 && (lane >> 2) < 6)
            twist_part[((size_t)f * nparts + (size_t)blockIdx.x * (NT / 32) + warp) * 6 + (lane >> 2)] =
                (double)tot;
    }
    if (!active) return;
    // colour and opacity
    auto put = [acc](float *dst, float v) { *dst = acc ? *dst + v : v; };
    put(d_col + 3 * g, dc0);
    put(d_col + 3 * g + 1, dc1);
    put(d_col + 3 * g + 2, dc2);
    // F = log2(sigmoid(l)):  dF/dl = (1 - o) / ln 2
    put(d_logit + g, dF * (1.f - G.o) * (1.f / kLn2));
    // Sigma = M M^T, M = R_g diag(s): dL/dM = 2 G M, G = dL/dSigma as the
    // full symmetric matrix T^T H T (dSig holds its six distinct entries)
    const float S00 = dSig[0], S01 = dSig[1], S02 = dSig[2];
    const float S11 = dSig[3], S12 = dSig[4], S22 = dSig[5];
    const float Sg[9] = {S00, S01, S02, S01, S11, S12, S02, S12, S22};
    const float *R = G.Rg;
    float dR[9];
    for (int j = 0; j < 3; j++) {
        float sj = G.s[j];
        float ds = 0.f;
        for (int i = 0; i < 3; i++) {
            float dM = 2.f * (Sg[3 * i] * R[j] + Sg[3 * i + 1] * R[3 + j] + Sg[3 * i + 2] * R[6 + j]) * sj;
            ds += dM * R[3 * i + j];
            dR[3 * i + j] = dM * sj;
        }
        put(d_log_s + 3 * g + j, G.s_clamped[j] ? 0.f : ds * sj);
    }
    // R(q) for the unit quaternion (w, x, y, z) -> dL/dq_unit
    const float w = G.q[0], x = G.q[1], y = G.q[2], z = G.q[3];
    float gw = 2.f * (z * (dR[3] - dR[1]) + y * (dR[2] - dR[6]) + x * (dR[7] - dR[5]));
    float gx = 2.f * (y * (dR[1] + dR[3]) + z * (dR[2] + dR[6]) + w * (dR[7] - dR[5])) - 4.f * x * (dR[4] + dR[8]);
    float gy = 2.f * (x * (dR[1] + dR[3]) + w * (dR[2] - dR[6]) + z * (dR[5] + dR[7])) - 4.f * y * (dR[0] + dR[8]);
    float gz = 2.f * (w * (dR[3] - dR[1]) + x * (dR[2] + dR[6]) + y * (dR[5] + dR[7])) - 4.f * z * (dR[0] + dR[4]);
    // normalisation q_unit = q / |q|
    float dot = w * gw + x * gx + y * gy + z * gz;
    float iq = 1.f / G.qn;
    put(d_quat + 4 * g, (gw - w * dot) * iq);
    put(d_quat + 4 * g + 1, (gx - x * dot) * iq);
    put(d_quat + 4 * g + 2, (gy - y * dot) * iq);
    put(d_quat + 4 * g + 3, (gz - z * dot) * iq);
}

}  // namespace

cudaError_t launch_project(const gs_batch *b, const float *pose32, const float *X, const float *quat,
                           const float *log_s, const float *logit_o, const gs_opts *o, uint2 *rect,
                           float *depth, float4 *splat, float4 *grad2d, Stats *stats, cudaStream_t s) {
    int N = b->num_gaussians;
    if (N == 0) return cudaSuccess;
    k_project<<<(N + kProjThreads - 1) / kProjThreads, kProjThreads, 0, s>>>(
        b->frames_dev, b->num_frames, N, pose32, X, quat, log_s, logit_o, *o, rect, depth, splat, grad2d, stats);
    return cudaGetLastError();
}

int project_bwd_blocks(const gs_batch *b) { return (b->num_gaussians + kProjThreads - 1) / kProjThreads; }

// Twist partials per frame: one per warp of the projection backward.
int project_bwd_parts(const gs_batch *b) { return project_bwd_blocks(b) * (kProjThreads / 32); }

cudaError_t launch_project_bwd(const gs_batch *b, const float *pose32, const float *X, const float *quat,
                               const float *log_s, const float *logit_o, const gs_opts *o, const uint2 *rect,
                               const float4 *grad2d, float *d_quat, float *d_log_s, float *d_logit,
                               float *d_col, double *twist_part, bool acc, cudaStream_t s) {
    int nb = project_bwd_blocks(b);
    if (nb == 0) return cudaSuccess;
    k_project_bwd<kProjThreads><<<nb, kProjThreads, 0, s>>>(b->frames_dev, b->num_frames, b->num_gaussians,
                                                           pose32, X, quat, log_s, logit_o, *o, rect, grad2d,
                                                           d_quat, d_log_s, d_logit, d_col, twist_part,
                                                           nb * (kProjThreads / 32), acc);
    return cudaGetLastError();
}

}  // namespace gs
