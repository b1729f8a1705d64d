// ma_probe.cu -- ma_probe_fp64_rate(): the FP64 fused-multiply-add issue rate
// of the current device, measured, the peak the FP64 kernels are held to.
//
// Every FP64 kernel of this library is bound by GB300's FP64 pipe (it issues
// FP64 at a small fraction of the FP32 rate), so their roofline is an FP64
// operation rate, not bandwidth.  The probe runs independent chains of
// dependent DFMAs (eight per thread, enough to cover the pipe's latency) on
// every SM and times them with CUDA events.
#include <cuda_runtime.h>

#include "ma.h"
#include "ma_internal.h"

namespace {

constexpr int kChains = 8, kIters = 2048, kThreads = 256, kBlocksPerSm = 8;

// keeps the chains' results live; written only when a value is impossible
__device__ double g_probe_sink;

__global__ void __launch_bounds__(kThreads) k_dfma_probe(double x, double y)
{
    double a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = (double)(threadIdx.x + c);
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], x, y);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == -1.2345e300) g_probe_sink = s;
}

}  // namespace

extern "C" ma_status ma_probe_fp64_rate(double* ops_per_s, ma_stream_t stream)
{
    if (!ops_per_s) {
        ma::set_last_error("ma_probe_fp64_rate: null argument");
        return MA_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    const int blocks = sms * kBlocksPerSm;
    // x slightly below 1 keeps the chains finite and away from denormals
    const double x = 0.999999, y = 1e-6;
    float ms = 0.0f;
    if (e == cudaSuccess) {
        ma::count_launches(2);
        k_dfma_probe<<<blocks, kThreads, 0, s>>>(x, y);   // warm-up
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(t0, s);
    if (e == cudaSuccess) {
        k_dfma_probe<<<blocks, kThreads, 0, s>>>(x, y);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(t1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (e != cudaSuccess || !(ms > 0.0f)) {
        ma::set_last_error(e != cudaSuccess ? cudaGetErrorString(e) : "ma_probe_fp64_rate: zero time");
        return MA_ERR_CUDA;
    }
    *ops_per_s = (double)blocks * kThreads * kIters * kChains / (ms * 1e-3);
    return MA_OK;
}
