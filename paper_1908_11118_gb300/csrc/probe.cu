// probe.cu -- FP32 FFMA-loop microbenchmark (sm_103a).
//
// The sweep kernel's roofline fraction is quoted against the FP32 pipe's
// peak.  This kernel measures that peak on the GPU at hand: every thread runs
// eight independent chains of fused multiply-adds (enough independent work to
// hide the FMA latency at full occupancy), on 8 CTAs of 256 threads per SM.
#include "launch.h"
#include "../../include/regc_probe.h"

namespace regc {
namespace {

constexpr int kChains = 8, kUnroll = 16;

__global__ void __launch_bounds__(256) ffma_kernel(float* sink, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 1e-3f * (float)threadIdx.x + (float)k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == -1.0f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;   // never true: keeps the chains live
}

}  // namespace
}  // namespace regc

extern "C" REGC_API regc_status regc_probe_fp32_peak(int iters, void* cuda_stream, double* tflops) {
    if (iters < 1 || !tflops) return REGC_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8, threads = 256;
    float* sink = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess) e = cudaMallocAsync(&sink, (size_t)blocks * threads * sizeof(float), s);
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    float ms = 0.f;
    if (e == cudaSuccess) {
        regc::ffma_kernel<<<blocks, threads, 0, s>>>(sink, iters / 4 + 1, 0.999f, 1e-3f);   // warm-up
        cudaEventRecord(t0, s);
        regc::ffma_kernel<<<blocks, threads, 0, s>>>(sink, iters, 0.999f, 1e-3f);
        cudaEventRecord(t1, s);
        e = cudaEventSynchronize(t1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (sink) cudaFreeAsync(sink, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess || !(ms > 0.f)) return REGC_ECUDA;
    const double flops = 2.0 * regc::kChains * regc::kUnroll * (double)iters * blocks * threads;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return REGC_OK;
}
