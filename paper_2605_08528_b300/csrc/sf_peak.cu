// sf_peak.cu -- the FP32 fused multiply-add throughput of the device, measured:
// the denominator of the step's ALU roofline (the step kernels are not
// tensor-core work, and their FP32 share is reported against this figure).
#include <cuda_runtime.h>

#include "../../include/sf.h"

namespace {

constexpr int kChains = 8;      // independent FMA chains per thread (hide the FMA latency)
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) fma_kernel(float* __restrict__ out, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = __fmaf_rn(x[c], a, b);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678f) out[blockIdx.x] = s;   // keeps the chains live; never true for the inputs used
}

}  // namespace

extern "C" sf_status sf_fp32_fma_peak(void* stream, int iters, double* out_tflops) {
    if (!out_tflops || iters < 1) return SF_ERR_INVALID_ARG;
    *out_tflops = 0.0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess)
        return SF_ERR_CUDA;
    float* out = nullptr;
    if (cudaMalloc(&out, sizeof(float) * 8 * sms) != cudaSuccess) return SF_ERR_OOM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = 8 * sms;   // 8 blocks of 8 warps: every SM full
    fma_kernel<<<blocks, kThreads, 0, st>>>(out, iters, 0.9999999f, 1e-7f);   // warm-up
    cudaEventRecord(e0, st);
    fma_kernel<<<blocks, kThreads, 0, st>>>(out, iters, 0.9999999f, 1e-7f);
    cudaEventRecord(e1, st);
    const cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess || !(ms > 0.f)) return SF_ERR_CUDA;
    const double flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
    *out_tflops = flops / (ms * 1e-3) / 1e12;
    return SF_OK;
}
