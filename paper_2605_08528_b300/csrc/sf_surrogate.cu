// sf_surrogate.cu -- training-side kernels of the dynamics surrogate:
// column statistics of the collected transitions and normalised minibatches.
#include <cuda_runtime.h>

#include <cstdint>

#include "sf_internal.cuh"

namespace {

// compensated (Kahan) float sum of the block's per-thread partials: FP32 only
__device__ float block_sum(float v, float* red) {
    red[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const float r = red[0];
    __syncthreads();
    return r;
}

// mean and standard deviation of every column of x [n][k] (two passes, each
// thread a Kahan-compensated float sum); one block per column; std floored at
// 1e-6 of the column's scale
__global__ void col_stats_kernel(const float* __restrict__ x, unsigned long long n, int k, float* __restrict__ stats) {
    const int c = blockIdx.x;
    __shared__ float red[256];
    float s = 0.f, comp = 0.f;
    for (unsigned long long i = threadIdx.x; i < n; i += blockDim.x) {
        const float yv = x[i * k + c] - comp;
        const float t = s + yv;
        comp = (t - s) - yv;
        s = t;
    }
    const float inv_n = 1.f / (float)(n ? n : 1);
    const float mean = block_sum(s, red) * inv_n;
    float q = 0.f;
    comp = 0.f;
    for (unsigned long long i = threadIdx.x; i < n; i += blockDim.x) {
        const float d = x[i * k + c] - mean;
        const float yv = d * d - comp;
        const float t = q + yv;
        comp = (t - q) - yv;
        q = t;
    }
    const float var = block_sum(q, red) * inv_n;
    if (threadIdx.x == 0) {
        float sd = sqrtf(var);
        const float floor_ = 1e-6f * (fabsf(mean) + 1e-3f);
        if (!(sd > floor_)) sd = floor_ > 1e-12f ? floor_ : 1.f;
        stats[c] = mean;
        stats[k + c] = sd;
    }
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// minibatch row b of step t: row index from a counter hash; normalised copies
__global__ void gather_kernel(const float* __restrict__ x, const float* __restrict__ y, unsigned long long n,
                              const float* __restrict__ xs, const float* __restrict__ ys, int batch,
                              unsigned long long seed, unsigned long long t, float* __restrict__ bx,
                              float* __restrict__ by) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    const unsigned long long r = mix64(mix64(seed ^ t) ^ (unsigned long long)b) % n;
#pragma unroll
    for (int k = 0; k < kSurrIn; ++k) bx[(size_t)b * kSurrIn + k] = (x[r * kSurrIn + k] - xs[k]) / xs[kSurrIn + k];
#pragma unroll
    for (int k = 0; k < kSurrOut; ++k)
        by[(size_t)b * kSurrOut + k] = (y[r * kSurrOut + k] - ys[k]) / ys[kSurrOut + k];
}

}  // namespace

cudaError_t sf_launch_col_stats(const float* x, unsigned long long n, int k, float* stats, cudaStream_t s) {
    col_stats_kernel<<<k, 256, 0, s>>>(x, n, k, stats);
    return cudaGetLastError();
}

cudaError_t sf_launch_gather(const float* x, const float* y, unsigned long long n, const float* xs, const float* ys,
                             int batch, unsigned long long seed, unsigned long long t, float* bx, float* by,
                             cudaStream_t s) {
    gather_kernel<<<(batch + 255) / 256, 256, 0, s>>>(x, y, n, xs, ys, batch, seed, t, bx, by);
    return cudaGetLastError();
}
