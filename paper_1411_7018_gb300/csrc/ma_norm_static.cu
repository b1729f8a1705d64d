// ma_norm_static.cu -- ma_norm_static(): the grid norms of ma_norm() without
// any caller-provided or allocated scratch.
//
// Who needs it: callers that cannot allocate device memory at the point where
// they want a norm -- for example code whose device memory is entirely owned
// and already reserved by another allocator, or a loop where the implicit
// device synchronisation of cudaMalloc/cudaFree is not acceptable -- and that
// have no spare buffer to lend.  The reduction partials live instead in a
// fixed array in this library's device memory, reserved once when the library
// is loaded on a device and held until the process exits.
//
// The kernels are the same ones ma_norm() runs (norm partials, then a
// fixed-order final fold); only the source of the scratch differs.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "ma.h"
#include "ma_internal.h"

namespace {

// Largest grid the fixed scratch serves: n = MA_NORM_STATIC_MAX_N points per
// side.  The norm kernels use one (max, sum of squares) pair per block of a
// ceil(n/32) x ceil(n/4) x min(n,16) grid, plus two doubles for the result.
constexpr int kMaxN = MA_NORM_STATIC_MAX_N;
constexpr int kMaxPartials = ((kMaxN + 31) / 32) * ((kMaxN + 3) / 4) * (kMaxN < 16 ? kMaxN : 16);
constexpr size_t kScratchDoubles = 2 * (size_t)kMaxPartials + 2;

// File-scope device scratch shared by every call on a device (about 550 KB).
// Its contents persist between calls; every call overwrites all partials it
// reads, so nothing has to be cleared first.
static __device__ __align__(256) double g_norm_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_norm_scratch on the current device.  In host code the
// symbol name is only a host-side stand-in, so the address is looked up once
// per device (with that device current) and cached.
cudaError_t scratch_for_current_device(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_norm_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = (double*)p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" ma_status ma_norm_static(const double* v_dev, int n, double h, double* out_host, ma_stream_t stream)
{
    char msg[200];
    if (!v_dev || !out_host || !(h > 0.0) || n < 3 || (n % 2) == 0) {
        ma::set_last_error("ma_norm_static: bad arguments");
        return MA_ERR_INVALID_ARG;
    }
    if (n > kMaxN) {
        snprintf(msg, sizeof msg, "ma_norm_static: n = %d exceeds the fixed scratch limit n <= %d", n, kMaxN);
        ma::set_last_error(msg);
        return MA_ERR_INVALID_ARG;
    }
    const int count = ma::norm_partial_count(n);
    if (count > kMaxPartials) {
        snprintf(msg, sizeof msg, "ma_norm_static: %d partials exceed the fixed scratch", count);
        ma::set_last_error(msg);
        return MA_ERR_INVALID_ARG;
    }
    double* scratch = nullptr;
    cudaError_t e = scratch_for_current_device(&scratch);
    cudaStream_t s = (cudaStream_t)stream;
    double* out2 = (e == cudaSuccess) ? scratch + 2 * (size_t)count : nullptr;
    if (e == cudaSuccess) e = ma::launch_norm_partials(v_dev, n, scratch, s);
    if (e == cudaSuccess) e = ma::launch_norm_final(scratch, count, h, out2, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, out2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "ma_norm_static: %s", cudaGetErrorString(e));
        ma::set_last_error(msg);
        return MA_ERR_CUDA;
    }
    return MA_OK;
}
