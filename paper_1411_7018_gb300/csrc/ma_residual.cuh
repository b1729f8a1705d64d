// ma_residual.cuh -- the FP64 fine-grid residual r = rhs - det(D^2_h u)
// (Algorithm 1 step 3; the operator of Eq. MA_discrete) with the partials of
// its max and discrete-L2 norms (stopping rule of Section 4).
//
// FP64 throughput bounds this kernel on GB300, so each thread walks one (i, j)
// column through a contiguous run of k and reuses the x- and y-differences
// Dx = u(i+1) - u(i-1), Dy = u(j+1) - u(j-1) of the planes above and below:
// the xz and yz cross sums are Dx(k+1) - Dx(k-1) and Dy(k+1) - Dy(k-1), two
// FP64 operations per point instead of six.  The norm partials are taken on
// the FP32 value of r (the stopping rule needs ~7 digits of a norm, not 16),
// which keeps them off the FP64 pipe.  Grid: (ceil(n/32), ceil(n/4), kz)
// blocks of 32 x 4 threads, k runs of ceil(n/kz) planes; one partial pair per
// block.
#pragma once

#include "ma_point.cuh"

namespace ma {
namespace resid {

constexpr int RX = 32, RY = 4;

// Writes the residual value of interior point (i, j, k), linear index p
// (H4 = 4 h^2 D^2_h u at the point, for outputs that also store it).
struct NaturalF64Out {
    double* r;
    __device__ __forceinline__ void put(long long p, int, int, int, int, double v, float, const HessS&) const
    {
        r[p] = v;
    }
    __device__ __forceinline__ void zero(long long p) const { r[p] = 0.0; }
};

// Block body with the block index and the grid's dimensions as arguments (a
// batched launch over several grids runs the same code).
template <typename Out>
__device__ __forceinline__ void residual_col_block(const double* __restrict__ u, const double* __restrict__ rhs,
                                                   const Out& out, int n, double inv_h6, double* partials, int kchunk,
                                                   uint3 bid, uint3 gdim)
{
    const int i = bid.x * RX + threadIdx.x;
    const int j = bid.y * RY + threadIdx.y;
    const int k0 = bid.z * kchunk;
    const int k1 = min(n, k0 + kchunk);
    const long long sy = n, sz = (long long)n * n;
    float mx = 0.0f, ss = 0.0f;
    if (i < n && j < n && k0 < k1) {
        const bool col_interior = i > 0 && j > 0 && i < n - 1 && j < n - 1;
        if (!col_interior) {
            for (int k = k0; k < k1; ++k) out.zero(((long long)k * n + j) * n + i);
        } else {
            auto DX = [&](int k) -> double {
                const double* q = u + ((long long)k * n + j) * n + i;
                return __ldg(q + 1) - __ldg(q - 1);
            };
            auto DY = [&](int k) -> double {
                const double* q = u + ((long long)k * n + j) * n + i;
                return __ldg(q + sy) - __ldg(q - sy);
            };
            double dxa = k0 >= 1 ? DX(k0 - 1) : 0.0, dya = k0 >= 1 ? DY(k0 - 1) : 0.0;
            double dxb = DX(k0), dyb = DY(k0);
            for (int k = k0; k < k1; ++k) {
                const long long p = ((long long)k * n + j) * n + i;
                if (k == 0 || k == n - 1) {
                    out.zero(p);
                } else {
                    const double dxc = DX(k + 1), dyc = DY(k + 1);
                    const double* q = u + p;
                    const double v0 = q[0];
                    const double a = __ldg(q + 1) + __ldg(q - 1);
                    const double b = __ldg(q + sy) + __ldg(q - sy);
                    const double c = __ldg(q + sz) + __ldg(q - sz);
                    const double r4 = (__ldg(q + sy + 1) - __ldg(q + sy - 1)) - (__ldg(q - sy + 1) - __ldg(q - sy - 1));
                    HessS H;
                    const double m8v = -8.0 * v0;
                    H.A = fma(4.0, a, m8v);
                    H.B = fma(4.0, b, m8v);
                    H.C = fma(4.0, c, m8v);
                    H.R = r4;
                    H.S = dxc - dxa;
                    H.T = dyc - dya;
                    const double val = fma(-det0(H), inv_h6, rhs[p]);   // inv_h6 = 1 / (64 h^6)
                    const float v32 = d2f_trunc(val);
                    mx = fmaxf(mx, fabsf(v32));
                    ss = fmaf(v32, v32, ss);
                    out.put(p, i, j, k, n, val, v32, H);
                    dxa = dxb; dya = dyb;
                    dxb = dxc; dyb = dyc;
                    continue;
                }
                // boundary plane: advance the difference window
                if (k + 1 <= n - 1) {
                    const double dxc = DX(k + 1), dyc = DY(k + 1);
                    dxa = dxb; dya = dyb;
                    dxb = dxc; dyb = dyc;
                }
            }
        }
    }
    if (partials) {
        __shared__ float smx[RX * RY / 32], sss[RX * RY / 32];
        for (int o = 16; o > 0; o >>= 1) {
            mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
            ss += __shfl_down_sync(0xffffffffu, ss, o);
        }
        const int t = threadIdx.y * RX + threadIdx.x;
        if ((t & 31) == 0) { smx[t >> 5] = mx; sss[t >> 5] = ss; }
        __syncthreads();
        if (t == 0) {
            double m = f2d(smx[0]), q = f2d(sss[0]);
            for (int w = 1; w < RX * RY / 32; ++w) { m = fmax(m, f2d(smx[w])); q += f2d(sss[w]); }
            const int slot = (bid.z * gdim.y + bid.y) * gdim.x + bid.x;
            partials[2 * slot] = m;
            partials[2 * slot + 1] = q;
        }
    }
}

template <typename Out>
__global__ void __launch_bounds__(RX * RY) k_residual_col(const double* __restrict__ u, const double* __restrict__ rhs,
                                                          Out out, int n, double inv_h6, double* partials, int kchunk)
{
    residual_col_block<Out>(u, rhs, out, n, inv_h6, partials, kchunk, blockIdx, gridDim);
}

// One block of NF = 256 threads folds the (max, sum of squares) partials in
// a fixed order: out2 = (max, sqrt(h^3 sum)), the max and discrete L2 norms
// of the stopping rule (Section 4).
constexpr int NF = 256;

__device__ __forceinline__ void norm_final_block(const double* __restrict__ partials, int count, double h3,
                                                 double* out2)
{
    __shared__ double smx[NF], sss[NF];
    double mx = 0.0, ss = 0.0;
    for (int q = threadIdx.x; q < count; q += NF) {
        mx = fmax(mx, partials[2 * q]);
        ss += partials[2 * q + 1];
    }
    smx[threadIdx.x] = mx;
    sss[threadIdx.x] = ss;
    __syncthreads();
    for (int w = NF / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            smx[threadIdx.x] = fmax(smx[threadIdx.x], smx[threadIdx.x + w]);
            sss[threadIdx.x] += sss[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out2[0] = smx[0];
        out2[1] = sqrt(h3 * sss[0]);
    }
}

inline dim3 grid_for(int n, int kz) { return dim3((n + RX - 1) / RX, (n + RY - 1) / RY, kz); }

}  // namespace resid
}  // namespace ma
