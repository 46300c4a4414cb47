// F(X | Theta) (Sec. III-C): the Instant-NGP multiresolution hash encoding of
// a Gaussian's centre followed by an MLP whose four heads give the Gaussian's
// colour, opacity, scale and rotation; forward and backward.
//
// Encoding: L <= 16 levels of 2 features, T = 2^log2_table entries per level.
// A point maps to p in [0, 1]^3 (clamped) through the bounding box; at level
// l its coordinates are q = p N_l, its cell c = min(floor(q), N_l - 1), and
// its two features are the trilinear interpolation of the cell's 8 vertices
// (weights from q - c).  A vertex v indexes the level's table densely,
// x + y (N_l + 1) + z (N_l + 1)^2, when the (N_l + 1)^3 vertices fit,
// otherwise by the spatial hash (x * 1 ^ y * 2654435761 ^ z * 805459861)
// mod 2^32 mod T.
// MLP: 2L -> 64 -> 64 -> 11 with ReLU after the hidden layers; heads
// rgb = sigmoid(o0..2), logit opacity o3, log scale o4..6, quaternion o7..10
// (the renderer's raw inputs).
// Parameters (theta, float): the L tables [L][T][2], then W1 [64][2L],
// b1 [64], W2 [64][64], b2 [64], W3 [11][64], b3 [11].
//
// Both kernels take chunks of 32 points per iteration of a block (grid
// stride, weights staged once per block in shared memory with padded rows):
// the encoding is computed per (point, level) by the block's threads, and
// each layer is a small matrix product over the chunk in shared memory.  The
// backward recomputes the forward, carries the attribute gradients back
// through the heads and the layers, accumulates the weight gradients of its
// chunks in shared memory (each thread owns fixed entries, so there are no
// atomics inside the block), adds them to d_theta once per block, and
// scatters the encoding gradient into the tables with one float2 atomic per
// (point, level, vertex).
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace gs {

namespace {

constexpr int kH = 64, kO = 11, kMaxLevels = 16;
constexpr int kNgpThreads = 128, kChunk = 32;
constexpr int kHP = kH + 1;  // padded row of a 64-wide matrix

struct NgpArgs {
    float lo[3], inv_ext[3];
    int L, D;            // levels, encoding width 2L
    uint32_t T, tmask;   // table entries (a power of two) and T - 1
    int res[kMaxLevels];
    int dense[kMaxLevels];
    long long w1;        // offset of W1 in theta; b1, W2, b2, W3, b3 follow
};

// Offsets, within the MLP block, of b1, W2, b2, W3, b3 and the block size.
__host__ __device__ constexpr int off_b1(int D) { return kH * D; }
__host__ __device__ constexpr int off_w2(int D) { return kH * D + kH; }
__host__ __device__ constexpr int off_b2(int D) { return kH * D + kH + kH * kH; }
__host__ __device__ constexpr int off_w3(int D) { return kH * D + 2 * kH + kH * kH; }
__host__ __device__ constexpr int off_b3(int D) { return kH * D + 2 * kH + kH * kH + kO * kH; }
__host__ __device__ constexpr int mlp_size(int D) { return kH * D + 2 * kH + kH * kH + kO * kH + kO; }

// The 8 vertices of a point's cell at level l: table slots and weights.
__device__ __forceinline__ void cell_taps(const NgpArgs &a, int l, float px, float py, float pz, uint32_t (&slot)[8],
                                          float (&w)[8]) {
    const float r = (float)a.res[l];
    const float qx = px * r, qy = py * r, qz = pz * r;
    const float cx = fminf(floorf(qx), r - 1.f), cy = fminf(floorf(qy), r - 1.f), cz = fminf(floorf(qz), r - 1.f);
    const float fx = qx - cx, fy = qy - cy, fz = qz - cz;
    const uint32_t ix = (uint32_t)cx, iy = (uint32_t)cy, iz = (uint32_t)cz;
    const uint32_t n1 = (uint32_t)a.res[l] + 1u;
#pragma unroll
    for (int c = 0; c < 8; c++) {
        const uint32_t dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
        const uint32_t vx = ix + dx, vy = iy + dy, vz = iz + dz;
        w[c] = ((dx ? fx : 1.f - fx) * (dy ? fy : 1.f - fy)) * (dz ? fz : 1.f - fz);
        slot[c] = a.dense[l] ? vx + vy * n1 + vz * n1 * n1
                             : ((vx * 1u) ^ (vy * 2654435761u) ^ (vz * 805459861u)) & a.tmask;
    }
}

__device__ __forceinline__ void unit_point(const NgpArgs &a, const float *__restrict__ X, long long i, float &px,
                                           float &py, float &pz) {
    px = fminf(fmaxf((X[3 * i] - a.lo[0]) * a.inv_ext[0], 0.f), 1.f);
    py = fminf(fmaxf((X[3 * i + 1] - a.lo[1]) * a.inv_ext[1], 0.f), 1.f);
    pz = fminf(fmaxf((X[3 * i + 2] - a.lo[2]) * a.inv_ext[2], 0.f), 1.f);
}

// Shared memory of a block: the weights with padded rows, then chunk buffers.
struct Weights {
    float *W1, *b1, *W2, *b2, *W3, *b3;  // W1 [64][D+1], W2 [64][65], W3 [11][65]
};

__device__ __forceinline__ float *stage_weights(const NgpArgs &a, const float *__restrict__ theta, float *sm,
                                                Weights &W) {
    const int D = a.D, DP = D + 1;
    W.W1 = sm;
    W.b1 = W.W1 + kH * DP;
    W.W2 = W.b1 + kH;
    W.b2 = W.W2 + kH * kHP;
    W.W3 = W.b2 + kH;
    W.b3 = W.W3 + kO * kHP;
    const float *m = theta + a.w1;
    for (int e = threadIdx.x; e < kH * D; e += kNgpThreads) W.W1[(e / D) * DP + e % D] = m[e];
    for (int e = threadIdx.x; e < kH; e += kNgpThreads) W.b1[e] = m[off_b1(D) + e];
    for (int e = threadIdx.x; e < kH * kH; e += kNgpThreads) W.W2[(e / kH) * kHP + e % kH] = m[off_w2(D) + e];
    for (int e = threadIdx.x; e < kH; e += kNgpThreads) W.b2[e] = m[off_b2(D) + e];
    for (int e = threadIdx.x; e < kO * kH; e += kNgpThreads) W.W3[(e / kH) * kHP + e % kH] = m[off_w3(D) + e];
    for (int e = threadIdx.x; e < kO; e += kNgpThreads) W.b3[e] = m[off_b3(D) + e];
    return W.b3 + kO + 1;
}

// Encoding of the chunk: ENC [32][D+1].
__device__ __forceinline__ void encode_chunk(const NgpArgs &a, const float *__restrict__ theta,
                                             const float *__restrict__ X, long long n, long long base, float *ENC) {
    const int DP = a.D + 1;
    for (int t = threadIdx.x; t < kChunk * a.L; t += kNgpThreads) {
        const int p = t & (kChunk - 1), l = t / kChunk;
        const long long i = base + p;
        float e0 = 0.f, e1 = 0.f;
        if (i < n) {
            float px, py, pz;
            unit_point(a, X, i, px, py, pz);
            uint32_t slot[8];
            float w[8];
            cell_taps(a, l, px, py, pz, slot, w);
            const float2 *tab = reinterpret_cast<const float2 *>(theta) + (size_t)l * a.T;
#pragma unroll
            for (int c = 0; c < 8; c++) {
                const float2 v = tab[slot[c]];
                e0 = fmaf(w[c], v.x, e0);
                e1 = fmaf(w[c], v.y, e1);
            }
        }
        ENC[p * DP + 2 * l] = e0;
        ENC[p * DP + 2 * l + 1] = e1;
    }
}

// Hidden layers of the chunk: H1 = relu(W1 ENC + b1), H2 = relu(W2 H1 + b2), [32][65] each.
__device__ __forceinline__ void hidden_chunk(const NgpArgs &a, const Weights &W, const float *ENC, float *H1,
                                             float *H2) {
    const int D = a.D, DP = D + 1;
    for (int o = threadIdx.x; o < kChunk * kH; o += kNgpThreads) {
        const int p = o / kH, j = o % kH;
        float acc = W.b1[j];
        for (int i = 0; i < D; i++) acc = fmaf(ENC[p * DP + i], W.W1[j * DP + i], acc);
        H1[p * kHP + j] = fmaxf(acc, 0.f);
    }
    __syncthreads();
    for (int o = threadIdx.x; o < kChunk * kH; o += kNgpThreads) {
        const int p = o / kH, j = o % kH;
        float acc = W.b2[j];
#pragma unroll 8
        for (int i = 0; i < kH; i++) acc = fmaf(H1[p * kHP + i], W.W2[j * kHP + i], acc);
        H2[p * kHP + j] = fmaxf(acc, 0.f);
    }
    __syncthreads();
}

__device__ __forceinline__ float out_unit(const Weights &W, const float *H2, int p, int k) {
    float acc = W.b3[k];
#pragma unroll 8
    for (int j = 0; j < kH; j++) acc = fmaf(H2[p * kHP + j], W.W3[k * kHP + j], acc);
    return acc;
}

__device__ __forceinline__ float sigmoidf(float x) { return 1.f / (1.f + expf(-x)); }

__global__ void __launch_bounds__(kNgpThreads)
k_ngp_fwd(NgpArgs a, const float *__restrict__ theta, const float *__restrict__ X, long long n,
          float *__restrict__ rgb, float *__restrict__ logit_o, float *__restrict__ log_s, float *__restrict__ quat) {
    extern __shared__ __align__(16) float sm[];
    Weights W;
    float *ENC = stage_weights(a, theta, sm, W);
    float *H1 = ENC + kChunk * (a.D + 1);
    float *H2 = H1 + kChunk * kHP;
    __syncthreads();
    for (long long base = (long long)blockIdx.x * kChunk; base < n; base += (long long)gridDim.x * kChunk) {
        encode_chunk(a, theta, X, n, base, ENC);
        __syncthreads();
        hidden_chunk(a, W, ENC, H1, H2);
        for (int o = threadIdx.x; o < kChunk * kO; o += kNgpThreads) {
            const int p = o / kO, k = o % kO;
            const long long i = base + p;
            if (i >= n) continue;
            const float v = out_unit(W, H2, p, k);
            if (k < 3) rgb[3 * i + k] = sigmoidf(v);
            else if (k == 3) logit_o[i] = v;
            else if (k < 7) log_s[3 * i + (k - 4)] = v;
            else quat[4 * i + (k - 7)] = v;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kNgpThreads)
k_ngp_bwd(NgpArgs a, const float *__restrict__ theta, const float *__restrict__ X, long long n,
          const float *__restrict__ d_rgb, const float *__restrict__ d_logit_o, const float *__restrict__ d_log_s,
          const float *__restrict__ d_quat, float *__restrict__ d_theta) {
    extern __shared__ __align__(16) float sm[];
    const int D = a.D, DP = D + 1, G = mlp_size(D);
    Weights W;
    float *ENC = stage_weights(a, theta, sm, W);
    float *H1 = ENC + kChunk * DP;
    float *H2 = H1 + kChunk * kHP;
    float *dO = H2 + kChunk * kHP;       // [32][12]
    float *dA2 = dO + kChunk * 12;       // [32][65]
    float *dA1 = dA2 + kChunk * kHP;     // [32][65]
    float *dENC = dA1 + kChunk * kHP;    // [32][D+1]
    float *acc = dENC + kChunk * DP;     // [G] weight gradients of this block
    for (int e = threadIdx.x; e < G; e += kNgpThreads) acc[e] = 0.f;
    __syncthreads();
    for (long long base = (long long)blockIdx.x * kChunk; base < n; base += (long long)gridDim.x * kChunk) {
        encode_chunk(a, theta, X, n, base, ENC);
        __syncthreads();
        hidden_chunk(a, W, ENC, H1, H2);
        // heads: dL/do (zero for the chunk's points beyond n)
        for (int o = threadIdx.x; o < kChunk * kO; o += kNgpThreads) {
            const int p = o / kO, k = o % kO;
            const long long i = base + p;
            float g = 0.f;
            if (i < n) {
                if (k < 3) {
                    const float s = sigmoidf(out_unit(W, H2, p, k));
                    g = d_rgb[3 * i + k] * s * (1.f - s);
                } else if (k == 3) {
                    g = d_logit_o[i];
                } else if (k < 7) {
                    g = d_log_s[3 * i + (k - 4)];
                } else {
                    g = d_quat[4 * i + (k - 7)];
                }
            }
            dO[p * 12 + k] = g;
        }
        __syncthreads();
        for (int o = threadIdx.x; o < kChunk * kH; o += kNgpThreads) {
            const int p = o / kH, j = o % kH;
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < kO; k++) s = fmaf(dO[p * 12 + k], W.W3[k * kHP + j], s);
            dA2[p * kHP + j] = H2[p * kHP + j] > 0.f ? s : 0.f;
        }
        __syncthreads();
        for (int o = threadIdx.x; o < kChunk * kH; o += kNgpThreads) {
            const int p = o / kH, j = o % kH;
            float s = 0.f;
#pragma unroll 8
            for (int m = 0; m < kH; m++) s = fmaf(dA2[p * kHP + m], W.W2[m * kHP + j], s);
            dA1[p * kHP + j] = H1[p * kHP + j] > 0.f ? s : 0.f;
        }
        __syncthreads();
        for (int o = threadIdx.x; o < kChunk * D; o += kNgpThreads) {
            const int p = o / D, i = o % D;
            float s = 0.f;
#pragma unroll 8
            for (int j = 0; j < kH; j++) s = fmaf(dA1[p * kHP + j], W.W1[j * DP + i], s);
            dENC[p * DP + i] = s;
        }
        // weight gradients summed over the chunk's points (entries owned per thread)
        for (int e = threadIdx.x; e < G; e += kNgpThreads) {
            float s = 0.f;
            if (e < off_b1(D)) {
                const int j = e / D, i = e % D;
                for (int p = 0; p < kChunk; p++) s = fmaf(dA1[p * kHP + j], ENC[p * DP + i], s);
            } else if (e < off_w2(D)) {
                const int j = e - off_b1(D);
                for (int p = 0; p < kChunk; p++) s += dA1[p * kHP + j];
            } else if (e < off_b2(D)) {
                const int j = (e - off_w2(D)) / kH, m = (e - off_w2(D)) % kH;
                for (int p = 0; p < kChunk; p++) s = fmaf(dA2[p * kHP + j], H1[p * kHP + m], s);
            } else if (e < off_w3(D)) {
                const int j = e - off_b2(D);
                for (int p = 0; p < kChunk; p++) s += dA2[p * kHP + j];
            } else if (e < off_b3(D)) {
                const int k = (e - off_w3(D)) / kH, j = (e - off_w3(D)) % kH;
                for (int p = 0; p < kChunk; p++) s = fmaf(dO[p * 12 + k], H2[p * kHP + j], s);
            } else {
                const int k = e - off_b3(D);
                for (int p = 0; p < kChunk; p++) s += dO[p * 12 + k];
            }
            acc[e] += s;
        }
        __syncthreads();
        // encoding gradient into the tables
        for (int t = threadIdx.x; t < kChunk * a.L; t += kNgpThreads) {
            const int p = t & (kChunk - 1), l = t / kChunk;
            const long long i = base + p;
            if (i >= n) continue;
            float px, py, pz;
            unit_point(a, X, i, px, py, pz);
            uint32_t slot[8];
            float w[8];
            cell_taps(a, l, px, py, pz, slot, w);
            const float g0 = dENC[p * DP + 2 * l], g1 = dENC[p * DP + 2 * l + 1];
            float2 *tab = reinterpret_cast<float2 *>(d_theta) + (size_t)l * a.T;
#pragma unroll
            for (int c = 0; c < 8; c++) atomicAdd(tab + slot[c], make_float2(w[c] * g0, w[c] * g1));
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < G; e += kNgpThreads)
        if (acc[e] != 0.f) atomicAdd(d_theta + a.w1 + e, acc[e]);
}

size_t fwd_smem(int D) {
    return sizeof(float) * ((size_t)kH * (D + 1) + kH + kH * kHP + kH + kO * kHP + kO + 1 + kChunk * (D + 1) +
                            2 * kChunk * kHP);
}

size_t bwd_smem(int D) {
    return fwd_smem(D) + sizeof(float) * ((size_t)kChunk * 12 + 2 * kChunk * kHP + kChunk * (D + 1) + mlp_size(D));
}

}  // namespace

static bool ngp_args(const gs_ngp *c, NgpArgs *a) {
    if (!c || c->levels < 1 || c->levels > kMaxLevels || c->log2_table < 4 || c->log2_table > 26) return false;
    a->L = c->levels;
    a->D = 2 * c->levels;
    a->T = 1u << c->log2_table;
    a->tmask = a->T - 1u;
    for (int d = 0; d < 3; d++) {
        const float ext = c->aabb_max[d] - c->aabb_min[d];
        if (!(ext > 0.f) || !std::isfinite(ext)) return false;
        a->lo[d] = c->aabb_min[d];
        a->inv_ext[d] = 1.f / ext;
    }
    for (int l = 0; l < kMaxLevels; l++) {
        a->res[l] = l < c->levels ? c->res[l] : 1;
        if (l < c->levels && (c->res[l] < 1 || c->res[l] > (1 << 20))) return false;
        const double n1 = (double)a->res[l] + 1.0;
        a->dense[l] = n1 * n1 * n1 <= (double)a->T;
    }
    a->w1 = (long long)c->levels * a->T * 2;
    return true;
}

long long ngp_param_count(const gs_ngp *c) {
    NgpArgs a;
    return ngp_args(c, &a) ? a.w1 + mlp_size(a.D) : -1;
}

cudaError_t launch_ngp_fwd(const gs_ngp *c, const float *theta, const float *X, long long n, float *rgb,
                           float *logit_o, float *log_s, float *quat, cudaStream_t s) {
    NgpArgs a;
    if (!ngp_args(c, &a)) return cudaErrorInvalidValue;
    if (n == 0) return cudaSuccess;
    const size_t smem = fwd_smem(a.D);
    cudaError_t e = cudaFuncSetAttribute(k_ngp_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const long long chunks = (n + kChunk - 1) / kChunk;
    const int grid = (int)std::min<long long>(chunks, 4ll * sms);
    k_ngp_fwd<<<grid, kNgpThreads, smem, s>>>(a, theta, X, n, rgb, logit_o, log_s, quat);
    return cudaGetLastError();
}

cudaError_t launch_ngp_bwd(const gs_ngp *c, const float *theta, const float *X, long long n, const float *d_rgb,
                           const float *d_logit_o, const float *d_log_s, const float *d_quat, float *d_theta,
                           cudaStream_t s) {
    NgpArgs a;
    if (!ngp_args(c, &a)) return cudaErrorInvalidValue;
    if (n == 0) return cudaSuccess;
    const size_t smem = bwd_smem(a.D);
    cudaError_t e = cudaFuncSetAttribute(k_ngp_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const long long chunks = (n + kChunk - 1) / kChunk;
    const int grid = (int)std::min<long long>(chunks, 2ll * sms);
    k_ngp_bwd<<<grid, kNgpThreads, smem, s>>>(a, theta, X, n, d_rgb, d_logit_o, d_log_s, d_quat, d_theta);
    return cudaGetLastError();
}

}  // namespace gs
