// L1 term of the photometric loss (Eq. 4): mean absolute error and its
// gradient sign(rgb - target) / n * scale, in one pass; the loss is reduced
// deterministically (fixed grid, per-block partials, ordered final sum).
#include "common.cuh"

namespace gs {

namespace {

__global__ void __launch_bounds__(kLossThreads)
k_l1(const float *__restrict__ x, const float *__restrict__ y, long long n, float gscale,
     float *__restrict__ grad, double *__restrict__ part) {
    __shared__ double sh[kLossThreads / 32];
    float acc = 0.f;
    double dacc = 0.0;
    int cnt = 0;
    for (long long i = (long long)blockIdx.x * kLossThreads + threadIdx.x; i < n;
         i += (long long)gridDim.x * kLossThreads) {
        const float d = x[i] - y[i];
        acc += fabsf(d);
        if (grad) grad[i] = d > 0.f ? gscale : (d < 0.f ? -gscale : 0.f);
        if (++cnt == 64) {  // bound the float partial sums
            dacc += acc;
            acc = 0.f;
            cnt = 0;
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
    k_l1<<<kLossBlocks, kLossThreads, 0, s>>>(x, y, n, gscale, grad, part);
    k_l1_final<<<1, 256, 0, s>>>(part, kLossBlocks, n, out_loss);
    return cudaGetLastError();
}

}  // namespace gs
