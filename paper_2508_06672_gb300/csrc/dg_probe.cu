// dg_probe.cu -- measured FP32 FMA throughput of the device.
//
// The CUDA-core kernels (the direct correlation, the chunked-DFT combine, the
// convolution layers) are stated against the FP32 peak of the chip. That peak
// is measured here rather than computed from a unit count and a clock: every
// thread of a grid that fills each SM with resident warps runs independent
// chains of fused multiply-adds, and the rate is 2 flops per FMA over the
// CUDA-event time of the launch.
#include <cuda_runtime.h>

#include "dg.h"

namespace dg {
namespace {

constexpr int kChains = 8;      // independent FMA chains per thread (latency 4 cycles)
constexpr int kUnroll = 16;     // FMAs per chain per loop iteration
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8; // 2048 resident threads per SM

__global__ void __launch_bounds__(kThreads) k_ffma_probe(float *sink, int iters, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = 1e-3f * (float)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) x[i] = fmaf(x[i], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    // never true for the arguments the host passes (the chains converge to
    // b / (1 - a) = 0.1): keeps the chains live without a store per thread
    if (s == -1.0f) sink[blockIdx.x] = s;
}

}  // namespace
}  // namespace dg

extern "C" dg_status dg_fp32_peak(void *cuda_stream, int32_t iters, double *tflops, double *ms, int32_t *sm_count)
{
    using namespace dg;
    if (iters <= 0 || !tflops) return DG_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return DG_ECUDA;
    float *sink = nullptr;
    if (cudaMallocAsync((void **)&sink, sizeof(float) * (size_t)sms * kBlocksPerSm, st) != cudaSuccess)
        return DG_ENOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    dg_status rc = DG_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = DG_ECUDA;
    const dim3 grid(sms * kBlocksPerSm);
    float t = 0.f;
    if (rc == DG_OK) {
        k_ffma_probe<<<grid, kThreads, 0, st>>>(sink, iters / 8 + 1, 0.5f, 0.05f);  // warm-up
        cudaEventRecord(e0, st);
        k_ffma_probe<<<grid, kThreads, 0, st>>>(sink, iters, 0.5f, 0.05f);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess ||
            cudaGetLastError() != cudaSuccess)
            rc = DG_ECUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(sink, st);
    if (rc != DG_OK) return rc;
    const double fmas = (double)grid.x * kThreads * kChains * kUnroll * (double)iters;
    *tflops = 2.0 * fmas / (t * 1e-3) / 1e12;
    if (ms) *ms = t;
    if (sm_count) *sm_count = sms;
    return DG_OK;
}
