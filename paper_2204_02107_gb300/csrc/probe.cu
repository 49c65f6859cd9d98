// Measurement helper (no counterpart in the paper): the FP64 fused multiply-add rate of the current device, the
// denominator of the FP64 step's roofline (on GB300 the FP64 form of the step is bound by FP64 arithmetic, not
// by HBM).  Eight independent FMA chains per thread, enough CTAs for every SM, timed with CUDA events.
#include <cuda_runtime.h>

#include "vf_internal.h"

namespace vf {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_fp64_fma(double* out, int iters, double a, double b)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3 + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678) out[0] = s;     // keeps the chains alive; never true for the inputs used
}

}  // namespace
}  // namespace vf

extern "C" int vf_measure_fp64_rate(double* gflops)
{
    if (!gflops) return VF_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess)
        return VF_ECUDA;
    double* out = nullptr;
    if (cudaMalloc(&out, sizeof(double)) != cudaSuccess) return VF_ENOMEM;
    const int blocks = sms * 8, threads = 256, iters = 4096;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    vf::k_fp64_fma<<<blocks, threads>>>(out, 64, 0.999999, 1e-7);   // warm-up
    cudaEventRecord(e0);
    vf::k_fp64_fma<<<blocks, threads>>>(out, iters, 0.999999, 1e-7);
    cudaEventRecord(e1);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess || ms <= 0.f) return VF_ECUDA;
    const double flops = 2.0 * (double)blocks * threads * iters * vf::kChains;
    *gflops = flops / (ms * 1e-3) / 1e9;
    return VF_OK;
}
