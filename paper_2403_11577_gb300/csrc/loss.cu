// L1 term of the photometric loss (Eq. 4): mean absolute error and its
// gradient sign(rgb - target) / n * scale, in one pass (16-byte accesses
// when the buffers allow); the loss is reduced deterministically (fixed
// grid, per-block partials, ordered final sum).
#include "common.cuh"

namespace gs {

namespace {

__device__ __forceinline__ float l1_sign(float d, float g) { return d > 0.f ? g : (d < 0.f ? -g : 0.f); }

// VEC: x, y and grad are 16-byte aligned; elements are taken four at a time
// (16-byte loads and stores), the n % 4 tail by block 0.
template <bool VEC>
__global__ void __launch_bounds__(kLossThreads)
k_l1(const float *__restrict__ x, const float *__restrict__ y, long long n, float gscale,
     float *__restrict__ grad, double *__restrict__ part) {
    __shared__ double sh[kLossThreads / 32];
    float acc = 0.f;
    double dacc = 0.0;
    int cnt = 0;
    const long long stride = (long long)gridDim.x * kLossThreads;
    if (VEC) {
        const long long n4 = n / 4;
        const float4 *x4 = reinterpret_cast<const float4 *>(x), *y4 = reinterpret_cast<const float4 *>(y);
        float4 *g4 = reinterpret_cast<float4 *>(grad);
        for (long long i = (long long)blockIdx.x * kLossThreads + threadIdx.x; i < n4; i += stride) {
            const float4 a = x4[i], b = y4[i];
            const float d0 = a.x - b.x, d1 = a.y - b.y, d2 = a.z - b.z, d3 = a.w - b.w;
            acc += fabsf(d0) + fabsf(d1) + (fabsf(d2) + fabsf(d3));
            if (grad) g4[i] = make_float4(l1_sign(d0, gscale), l1_sign(d1, gscale), l1_sign(d2, gscale),
                                          l1_sign(d3, gscale));
            if (++cnt == 16) {  // bound the float partial sums (64 terms)
                dacc += acc;
                acc = 0.f;
                cnt = 0;
            }
        }
        if (blockIdx.x == 0 && threadIdx.x < (n & 3)) {
            const long long i = 4 * n4 + threadIdx.x;
            const float d = x[i] - y[i];
            acc += fabsf(d);
            if (grad) grad[i] = l1_sign(d, gscale);
        }
    } else {
        for (long long i = (long long)blockIdx.x * kLossThreads + threadIdx.x; i < n; i += stride) {
            const float d = x[i] - y[i];
            acc += fabsf(d);
            if (grad) grad[i] = l1_sign(d, gscale);
            if (++cnt == 64) {  // bound the float partial sums
                dacc += acc;
                acc = 0.f;
                cnt = 0;
            }
        }
    }
    double v = dacc + acc;
    for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int w = 0; w < kLossThreads / 32; w++) t += sh[w];
        part[blockIdx.x] = t;
    }
}

__global__ void k_l1_final(const double *__restrict__ part, int nb, long long n, double *__restrict__ out) {
    __shared__ double sh[256];
    double s = 0;
    for (int i = threadIdx.x; i < nb; i += 256) s += part[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = n > 0 ? sh[0] / (double)n : 0.0;
}

}  // namespace

cudaError_t launch_l1(const float *x, const float *y, long long n, float scale, double *out_loss, float *grad,
                      double *part, cudaStream_t s) {
    const float gscale = n > 0 ? (float)((double)scale / (double)n) : 0.f;
    auto a16 = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    if (a16(x) && a16(y) && (!grad || a16(grad)))
        k_l1<true><<<kLossBlocks, kLossThreads, 0, s>>>(x, y, n, gscale, grad, part);
    else
        k_l1<false><<<kLossBlocks, kLossThreads, 0, s>>>(x, y, n, gscale, grad, part);
    k_l1_final<<<1, 256, 0, s>>>(part, kLossBlocks, n, out_loss);
    return cudaGetLastError();
}

}  // namespace gs
