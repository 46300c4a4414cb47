// L_photo (Eq. 4): (1 - lambda1) L1 + lambda1 D-SSIM over the batch's
// images, with lambda1 = 0.2 in the paper, and its gradient with respect to
// the rendered colours.
//
// SSIM of a channel at pixel q [kerbl20233d]: with the normalised 11x11
// Gaussian window G (sigma 1.5) and zero padding at the image border (a
// cropped frame's image is its rows [row0, height)),
//   mu_a = G*a, mu_b = G*b, s_aa = G*a^2 - mu_a^2, s_bb = G*b^2 - mu_b^2,
//   s_ab = G*(ab) - mu_a mu_b,
//   SSIM = (2 mu_a mu_b + C1)(2 s_ab + C2) / ((mu_a^2 + mu_b^2 + C1)(s_aa + s_bb + C2)),
// C1 = 0.01^2, C2 = 0.03^2; D-SSIM = 1 - mean SSIM over all n values.  Its
// gradient is a second filtering: with S_mu, S_aa, S_ab the partial
// derivatives of SSIM(q) in mu_a, s_aa, s_ab,
//   d(mean SSIM)/da(p) = (1/n) [ G*(S_mu - 2 mu_a S_aa - mu_b S_ab) + 2 a(p) G*S_aa
//                                + b(p) G*S_ab ](p).
//
// k_ssim_fwd: one block per render tile (its TR x TR pixels); the rendered
// and target values of the tile and a 5-pixel halo are staged in shared
// memory, the five moments of each channel are filtered separably (11 taps
// along rows, then along columns), and the three maps A1 = S_mu - 2 mu_a S_aa -
// mu_b S_ab, A2 = S_aa, A3 = S_ab are written to the workspace (planar:
// map (3 ch + k) holds A_{k+1} of channel ch for every pixel) with FP64
// per-block partial sums of SSIM and |a - b| (float within a warp).  k_ssim_bwd filters the maps
// the same way and writes the gradient of L_photo; k_photo_final reduces the
// partials in a fixed order (deterministic).
#include <cmath>

#include "common.cuh"

namespace gs {

namespace {

constexpr int kWin = 5;  // window radius: 11 taps
constexpr int kPhotoThreads = 256;

struct SsimWindow {
    float w[2 * kWin + 1];
};

template <int TR>
struct FwdSmem {
    static constexpr int E = TR + 2 * kWin;
    float in[6][E][E];    // rendered r, g, b, target r, g, b
    float h[15][E][TR];   // row-filtered a, b, a^2, b^2, ab per channel
    double red[2][kPhotoThreads / 32];
};

template <int TR>
struct BwdSmem {
    static constexpr int E = TR + 2 * kWin;
    float in[9][E][E];    // A1, A2, A3 per channel
    float h[9][E][TR];
};

// Frame f, image rows R = height - row0 and the tile's first (row, column).
struct TileGeom {
    const gs_frame *fr;
    int R, W, r0, c0;
};

template <int TR>
__device__ __forceinline__ TileGeom tile_geom(const gs_frame *__restrict__ frames, int F, int t) {
    TileGeom g;
    const int f = frame_of_tile(frames, F, t);
    g.fr = frames + f;
    g.R = g.fr->height - g.fr->row0;
    g.W = g.fr->width;
    const int lt = t - g.fr->tile_offset;
    g.r0 = (lt / g.fr->tiles_x) * TR;
    g.c0 = (lt % g.fr->tiles_x) * TR;
    return g;
}

// The three channels are filtered together: one staging round, one
// row-filter round and one column-filter round per block.
template <int TR>
__global__ void __launch_bounds__(kPhotoThreads)
k_ssim_fwd(const gs_frame *__restrict__ frames, int F, long long P, const float *__restrict__ x,
           const float *__restrict__ y, SsimWindow G, float *__restrict__ maps, double *__restrict__ part) {
    constexpr int E = FwdSmem<TR>::E;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FwdSmem<TR> &S = *reinterpret_cast<FwdSmem<TR> *>(smem_raw);
    const TileGeom g = tile_geom<TR>(frames, F, blockIdx.x);
    const long long pix0 = g.fr->pixel_offset;
    const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
    float ssim_acc = 0.f, l1_acc = 0.f;  // at most 3 values per thread
    for (int i = threadIdx.x; i < E * E; i += kPhotoThreads) {
        const int rr = g.r0 - kWin + i / E, cc = g.c0 - kWin + i % E;
        const bool in = rr >= 0 && rr < g.R && cc >= 0 && cc < g.W;
        const long long v = 3 * (pix0 + (long long)rr * g.W + cc);
#pragma unroll
        for (int ch = 0; ch < 3; ch++) {
            S.in[ch][i / E][i % E] = in ? x[v + ch] : 0.f;
            S.in[3 + ch][i / E][i % E] = in ? y[v + ch] : 0.f;
        }
    }
    __syncthreads();
    // row filter: each thread two adjacent columns of one channel row, from
    // the 12 staged values of a and of b they share (float2 loads; E, TR even)
    for (int i = threadIdx.x; i < 3 * E * (TR / 2); i += kPhotoThreads) {
        const int ch = i / (E * (TR / 2)), j = i % (E * (TR / 2));
        const int r = j / (TR / 2), c = 2 * (j % (TR / 2));
        float va[2 * kWin + 2], vb[2 * kWin + 2];
        const float2 *ra = reinterpret_cast<const float2 *>(&S.in[ch][r][c]);
        const float2 *rb = reinterpret_cast<const float2 *>(&S.in[3 + ch][r][c]);
#pragma unroll
        for (int q = 0; q < kWin + 1; q++) {
            const float2 ta = ra[q], tb = rb[q];
            va[2 * q] = ta.x;
            va[2 * q + 1] = ta.y;
            vb[2 * q] = tb.x;
            vb[2 * q + 1] = tb.y;
        }
#pragma unroll
        for (int o = 0; o < 2; o++) {
            float sa = 0.f, sb = 0.f, saa = 0.f, sbb = 0.f, sab = 0.f;
#pragma unroll
            for (int k = 0; k < 2 * kWin + 1; k++) {
                const float a = va[k + o], b = vb[k + o], w = G.w[k];
                sa = fmaf(w, a, sa);
                sb = fmaf(w, b, sb);
                saa = fmaf(w * a, a, saa);
                sbb = fmaf(w * b, b, sbb);
                sab = fmaf(w * a, b, sab);
            }
            S.h[5 * ch][r][c + o] = sa;
            S.h[5 * ch + 1][r][c + o] = sb;
            S.h[5 * ch + 2][r][c + o] = saa;
            S.h[5 * ch + 3][r][c + o] = sbb;
            S.h[5 * ch + 4][r][c + o] = sab;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * TR * TR; i += kPhotoThreads) {
        const int ch = i / (TR * TR), j = i % (TR * TR);
        const int r = j / TR, c = j % TR;
        const int rr = g.r0 + r, cc = g.c0 + c;
        if (rr >= g.R || cc >= g.W) continue;
        float ma = 0.f, mb = 0.f, eaa = 0.f, ebb = 0.f, eab = 0.f;
#pragma unroll
        for (int k = 0; k < 2 * kWin + 1; k++) {
            const float w = G.w[k];
            ma = fmaf(w, S.h[5 * ch][r + k][c], ma);
            mb = fmaf(w, S.h[5 * ch + 1][r + k][c], mb);
            eaa = fmaf(w, S.h[5 * ch + 2][r + k][c], eaa);
            ebb = fmaf(w, S.h[5 * ch + 3][r + k][c], ebb);
            eab = fmaf(w, S.h[5 * ch + 4][r + k][c], eab);
        }
        const float s_aa = eaa - ma * ma, s_bb = ebb - mb * mb, s_ab = eab - ma * mb;
        const float A = 2.f * ma * mb + C1, B = 2.f * s_ab + C2;
        const float Cc = ma * ma + mb * mb + C1, D = s_aa + s_bb + C2;
        const float inv = 1.f / (Cc * D);
        const float ssim = A * B * inv;
        const float S_mu = 2.f * mb * B * inv - 2.f * ma * ssim / Cc;
        const float S_aa = -ssim / D;
        const float S_ab = 2.f * A * inv;
        const long long p = pix0 + (long long)rr * g.W + cc;
        maps[(3 * ch) * P + p] = S_mu - 2.f * ma * S_aa - mb * S_ab;
        maps[(3 * ch + 1) * P + p] = S_aa;
        maps[(3 * ch + 2) * P + p] = S_ab;
        ssim_acc += ssim;
        l1_acc += fabsf(S.in[ch][r + kWin][c + kWin] - S.in[3 + ch][r + kWin][c + kWin]);
    }
    // summed over the warp in float (96 terms), widened per warp: GB300's
    // FP64 rate is low, and per-pixel FP64 adds kept its FP64 pipe busy
    for (int s = 16; s > 0; s >>= 1) {
        ssim_acc += __shfl_xor_sync(0xffffffffu, ssim_acc, s);
        l1_acc += __shfl_xor_sync(0xffffffffu, l1_acc, s);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        S.red[0][warp] = (double)ssim_acc;
        S.red[1][warp] = (double)l1_acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < kPhotoThreads / 32; w++) {
            a += S.red[0][w];
            b += S.red[1][w];
        }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

template <int TR>
__global__ void __launch_bounds__(kPhotoThreads)
k_ssim_bwd(const gs_frame *__restrict__ frames, int F, long long P, const float *__restrict__ x,
           const float *__restrict__ y, SsimWindow G, const float *__restrict__ maps, float inv_n, float lambda1,
           float scale, float *__restrict__ grad) {
    constexpr int E = BwdSmem<TR>::E;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BwdSmem<TR> &S = *reinterpret_cast<BwdSmem<TR> *>(smem_raw);
    const TileGeom g = tile_geom<TR>(frames, F, blockIdx.x);
    const long long pix0 = g.fr->pixel_offset;
    for (int i = threadIdx.x; i < E * E; i += kPhotoThreads) {
        const int rr = g.r0 - kWin + i / E, cc = g.c0 - kWin + i % E;
        const bool in = rr >= 0 && rr < g.R && cc >= 0 && cc < g.W;
        const long long p = pix0 + (long long)rr * g.W + cc;
#pragma unroll
        for (int m = 0; m < 9; m++) S.in[m][i / E][i % E] = in ? maps[m * P + p] : 0.f;
    }
    __syncthreads();
    // row filter: each thread two adjacent columns of one map row, from the
    // 12 staged values they share (float2 loads; E and TR are even)
    for (int i = threadIdx.x; i < 9 * E * (TR / 2); i += kPhotoThreads) {
        const int m = i / (E * (TR / 2)), j = i % (E * (TR / 2));
        const int r = j / (TR / 2), c = 2 * (j % (TR / 2));
        float v[2 * kWin + 2];
        const float2 *row = reinterpret_cast<const float2 *>(&S.in[m][r][c]);
#pragma unroll
        for (int q = 0; q < kWin + 1; q++) {
            const float2 t = row[q];
            v[2 * q] = t.x;
            v[2 * q + 1] = t.y;
        }
        float s0 = 0.f, s1 = 0.f;
#pragma unroll
        for (int k = 0; k < 2 * kWin + 1; k++) {
            s0 = fmaf(G.w[k], v[k], s0);
            s1 = fmaf(G.w[k], v[k + 1], s1);
        }
        *reinterpret_cast<float2 *>(&S.h[m][r][c]) = make_float2(s0, s1);
    }
    __syncthreads();
    // column filter: each thread two adjacent rows of one pixel column and
    // channel, from the 12 row-filtered values they share
    for (int i = threadIdx.x; i < 3 * (TR / 2) * TR; i += kPhotoThreads) {
        const int ch = i / ((TR / 2) * TR), j = i % ((TR / 2) * TR);
        const int r = 2 * (j / TR), c = j % TR;
        float gg[3][2];
#pragma unroll
        for (int m = 0; m < 3; m++) {
            float s0 = 0.f, s1 = 0.f, prev = S.h[3 * ch + m][r][c];
#pragma unroll
            for (int k = 0; k < 2 * kWin + 1; k++) {
                const float nxt = S.h[3 * ch + m][r + k + 1][c];
                s0 = fmaf(G.w[k], prev, s0);
                s1 = fmaf(G.w[k], nxt, s1);
                prev = nxt;
            }
            gg[m][0] = s0;
            gg[m][1] = s1;
        }
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const int rr = g.r0 + r + q, cc = g.c0 + c;
            if (rr >= g.R || cc >= g.W) continue;
            const long long v = 3 * (pix0 + (long long)rr * g.W + cc) + ch;
            const float a = x[v], b = y[v];
            const float d_ssim = (gg[0][q] + 2.f * a * gg[1][q] + b * gg[2][q]) * inv_n;  // d(mean SSIM)/da
            const float d_l1 = (a > b ? inv_n : (a < b ? -inv_n : 0.f));
            grad[v] = scale * ((1.f - lambda1) * d_l1 - lambda1 * d_ssim);
        }
    }
}

__global__ void k_photo_final(const double *__restrict__ part, int nb, double n, double lambda1,
                              double *__restrict__ out) {
    __shared__ double sh[2][256];
    double s = 0.0, l = 0.0;
    for (int i = threadIdx.x; i < nb; i += 256) {
        s += part[2 * i];
        l += part[2 * i + 1];
    }
    sh[0][threadIdx.x] = s;
    sh[1][threadIdx.x] = l;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + k];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + k];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double dssim = n > 0 ? 1.0 - sh[0][0] / n : 0.0;
        const double l1 = n > 0 ? sh[1][0] / n : 0.0;
        out[0] = (1.0 - lambda1) * l1 + lambda1 * dssim;
        out[1] = l1;
        out[2] = dssim;
    }
}

SsimWindow make_window() {
    SsimWindow G;
    double w[2 * kWin + 1], s = 0.0;
    for (int i = 0; i <= 2 * kWin; i++) {
        w[i] = std::exp(-(double)((i - kWin) * (i - kWin)) / (2.0 * 1.5 * 1.5));
        s += w[i];
    }
    for (int i = 0; i <= 2 * kWin; i++) G.w[i] = (float)(w[i] / s);
    return G;
}

template <int TR>
cudaError_t run_photo(const gs_batch *b, const float *x, const float *y, float lambda1, float scale, double *out,
                      float *grad, float *maps, double *part, cudaStream_t s) {
    const SsimWindow G = make_window();
    const int T = b->num_tiles;
    const double n = 3.0 * (double)b->num_pixels;
    constexpr int fs = (int)sizeof(FwdSmem<TR>), bs = (int)sizeof(BwdSmem<TR>);
    cudaError_t e = cudaFuncSetAttribute(k_ssim_fwd<TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, fs);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_ssim_bwd<TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, bs);
    if (e != cudaSuccess) return e;
    k_ssim_fwd<TR><<<T, kPhotoThreads, fs, s>>>(b->frames_dev, b->num_frames, b->num_pixels, x, y, G, maps, part);
    k_photo_final<<<1, 256, 0, s>>>(part, T, n, (double)lambda1, out);
    if (grad)
        k_ssim_bwd<TR><<<T, kPhotoThreads, bs, s>>>(b->frames_dev, b->num_frames, b->num_pixels, x, y, G, maps,
                                                    n > 0 ? (float)(1.0 / n) : 0.f, lambda1, scale, grad);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_photo(const gs_batch *b, const float *x, const float *y, float lambda1, float scale,
                         double *out, float *grad, float *maps, double *part, cudaStream_t s) {
    if (b->num_tiles <= 0) return cudaSuccess;
    switch (b->tile) {
    case 8: return run_photo<8>(b, x, y, lambda1, scale, out, grad, maps, part, s);
    case 16: return run_photo<16>(b, x, y, lambda1, scale, out, grad, maps, part, s);
    case 32: return run_photo<32>(b, x, y, lambda1, scale, out, grad, maps, part, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace gs
