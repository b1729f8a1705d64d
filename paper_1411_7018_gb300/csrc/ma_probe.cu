// ma_probe.cu -- device probes behind the library's design choices.
//
// ma_probe_fp64_rate(): the FP64 fused-multiply-add issue rate of the current
// device, measured, the peak the FP64 kernels are held to.
//
// ma_probe_phase_chain(): what one dependent phase of a chain costs as a
// launch in a CUDA graph and as a grid-wide barrier in one cooperative
// (persistent) kernel.  A multigrid cycle is a chain of such phases (colour
// sweeps, residual, transfers on every level); the hierarchies and the shared
// batch replay them as CUDA graphs, and this probe measures the persistent
// alternative on the same device.
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

// ---- phase chains -----------------------------------------------------------

constexpr int kPhaseThreads = 128;
constexpr long long kBarrierPolls = 1ll << 22;   // ~0.1-1 s, then the barrier gives up

// One phase: b = a * (1 + 1e-4) + 1 over n elements, blocks striding over the
// n / 128 tiles from tile0.
__device__ __forceinline__ void phase_body(const float* __restrict__ a, float* __restrict__ b, long long n,
                                           long long tile0, long long tstride)
{
    const long long tiles = (n + kPhaseThreads - 1) / kPhaseThreads;
    for (long long t = tile0; t < tiles; t += tstride) {
        const long long i = t * kPhaseThreads + threadIdx.x;
        if (i < n) b[i] = fmaf(a[i], 1.0001f, 1.0f);
    }
}

__global__ void __launch_bounds__(kPhaseThreads) k_phase(const float* a, float* b, long long n)
{
    phase_body(a, b, n, blockIdx.x, gridDim.x);
}

// Grid-wide barrier of a cooperative launch.  sync[0] counts arrivals,
// sync[1] is the generation, sync[2] the error flag.  Thread 0 of each block
// arrives (after a fence that publishes the block's writes) and polls the
// generation with acquire loads; the last to arrive resets the count and
// releases the others.  The poll is bounded: past kBarrierPolls it sets the
// error flag and the block leaves, so a grid that was not co-resident ends
// with an error instead of waiting forever.  Returns false once the flag is
// set (by this block or another).
__device__ __forceinline__ bool grid_barrier(unsigned* sync)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        const unsigned gen = *(volatile unsigned*)(sync + 1);
        __threadfence();
        if (atomicAdd(sync, 1u) == gridDim.x - 1) {
            atomicExch(sync, 0u);
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(sync + 1) : "memory");
        } else {
            for (long long it = 0;; ++it) {
                unsigned v;
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(sync + 1) : "memory");
                if (v != gen) break;
                if (it > kBarrierPolls) {
                    atomicExch(sync + 2, 1u);
                    break;
                }
            }
        }
        __threadfence();
        if (*(volatile unsigned*)(sync + 2)) ok = 0;
    }
    __syncthreads();
    return ok != 0;
}

// The whole chain in one launch: phase p reads the array phase p - 1 wrote,
// with a grid barrier between consecutive phases.
__global__ void __launch_bounds__(kPhaseThreads) k_phase_chain(float* a, float* b, long long n, int phases,
                                                               unsigned* sync)
{
    for (int p = 0; p < phases; ++p) {
        phase_body((p & 1) ? b : a, (p & 1) ? a : b, n, blockIdx.x, gridDim.x);
        if (p + 1 < phases && !grid_barrier(sync)) return;
    }
}

// Best of 5 timed runs (after 2 untimed) of fn on stream s, in ms.
template <typename F>
cudaError_t best_ms(cudaStream_t s, cudaEvent_t t0, cudaEvent_t t1, F fn, float* best)
{
    *best = 3.4e38f;
    for (int r = 0; r < 7; ++r) {
        cudaError_t e = cudaEventRecord(t0, s);
        if (e == cudaSuccess) e = fn();
        if (e == cudaSuccess) e = cudaEventRecord(t1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (e != cudaSuccess) return e;
        if (r >= 2 && ms < *best) *best = ms;
    }
    return cudaSuccess;
}

// A CUDA graph of `phases` dependent launches of k_phase on `grid` blocks.
cudaError_t chain_graph(cudaStream_t s, float* a, float* b, long long n, int phases, int grid, cudaGraphExec_t* out)
{
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    for (int p = 0; p < phases; ++p) k_phase<<<grid, kPhaseThreads, 0, s>>>((p & 1) ? b : a, (p & 1) ? a : b, n);
    const cudaError_t le = cudaGetLastError();
    e = cudaStreamEndCapture(s, &g);
    if (e == cudaSuccess) e = le;
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    return e;
}

}  // namespace

extern "C" ma_status ma_probe_phase_chain(float* a_dev, float* b_dev, size_t n, int phases, int blocks_per_sm,
                                          unsigned* sync_dev, double* out_us, ma_stream_t stream)
{
    if (!a_dev || !b_dev || !sync_dev || !out_us || n < 1 || n > ((size_t)1 << 40) || phases < 2 ||
        phases > 4096 || blocks_per_sm < 1) {
        ma::set_last_error("ma_probe_phase_chain: null pointer, n outside [1, 2^40], phases outside [2, 4096] "
                           "or blocks_per_sm < 1");
        return MA_ERR_INVALID_ARG;
    }
    int dev = 0, sms = 0, occ = 0, coop = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_phase_chain, kPhaseThreads, 0);
    if (e != cudaSuccess) {
        ma::set_last_error(cudaGetErrorString(e));
        return MA_ERR_CUDA;
    }
    if (!coop || blocks_per_sm > occ) {
        ma::set_last_error("ma_probe_phase_chain: no cooperative launch on this device, or blocks_per_sm above the "
                           "resident limit");
        return MA_ERR_INVALID_ARG;
    }
    // a private stream that can be captured, ordered after the caller's
    cudaStream_t s = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaGraphExec_t g_one = nullptr, g_stride = nullptr;
    const long long nn = (long long)n;
    const long long tiles = (nn + kPhaseThreads - 1) / kPhaseThreads;
    const int grid_one = (int)(tiles < (1ll << 30) ? tiles : (1ll << 30));
    const long long cap = (long long)blocks_per_sm * sms;
    const int grid_p = (int)(tiles < cap ? tiles : cap);
    float ms[3] = {0.0f, 0.0f, 0.0f};
    unsigned flag = 0;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    if (e == cudaSuccess) e = cudaEventRecord(t0, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, t0, 0);
    if (e == cudaSuccess) e = chain_graph(s, a_dev, b_dev, nn, phases, grid_one, &g_one);
    if (e == cudaSuccess) e = chain_graph(s, a_dev, b_dev, nn, phases, grid_p, &g_stride);
    if (e == cudaSuccess) e = cudaMemsetAsync(sync_dev, 0, 3 * sizeof(unsigned), s);
    if (e == cudaSuccess) {
        ma::count_launches(7ull * (2 * phases + 1));
        e = best_ms(s, t0, t1, [&] { return cudaGraphLaunch(g_one, s); }, &ms[0]);
    }
    if (e == cudaSuccess) e = best_ms(s, t0, t1, [&] { return cudaGraphLaunch(g_stride, s); }, &ms[1]);
    if (e == cudaSuccess) {
        void* args[] = {(void*)&a_dev, (void*)&b_dev, (void*)&nn, (void*)&phases, (void*)&sync_dev};
        e = best_ms(s, t0, t1,
                    [&] {
                        return cudaLaunchCooperativeKernel((const void*)k_phase_chain, dim3(grid_p),
                                                           dim3(kPhaseThreads), args, 0, s);
                    },
                    &ms[2]);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, sync_dev + 2, sizeof flag, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (g_one) cudaGraphExecDestroy(g_one);
    if (g_stride) cudaGraphExecDestroy(g_stride);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (s) cudaStreamDestroy(s);
    if (e != cudaSuccess) {
        ma::set_last_error(cudaGetErrorString(e));
        return MA_ERR_CUDA;
    }
    if (flag) {
        ma::set_last_error("ma_probe_phase_chain: a grid barrier gave up waiting (grid not co-resident)");
        return MA_ERR_CUDA;
    }
    for (int q = 0; q < 3; ++q) out_us[q] = 1e3 * ms[q] / phases;
    return MA_OK;
}

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
