// ma_transfer.cuh -- grid transfers of the FAS V-cycle (Section 3 of Liu,
// Froese, Oberman, Xiao), templated on the element type so the FP64 cycle and
// the FP32 correction cycle run the same code.  Grids are n^3 values in
// [k][j][i] order, boundary shell included; coarse point (I, J, K) sits on fine
// point (2I, 2J, 2K), nf = 2 nc - 1.
#pragma once

#include <cuda_runtime.h>

namespace ma {
namespace xfer {

constexpr int BX = 32, BY = 4;

__device__ __forceinline__ long long lin(int i, int j, int k, int n)
{
    return ((long long)k * n + j) * n + i;
}

// Restriction I_h^H at a fine point p with strides sy, sz.  kind 0: the
// printed 7-point half weighting (6 centre + 6 faces) / 12; kind 1: 27-point
// full weighting, separable (1 2 1)/4 along each axis.
template <typename T>
__device__ __forceinline__ T weighted_restrict(const T* __restrict__ v, long long p, long long sy, long long sz,
                                               int kind)
{
    if (kind == 0) {
        const T faces = (v[p + 1] + v[p - 1]) + (v[p + sy] + v[p - sy]) + (v[p + sz] + v[p - sz]);
        return (T(6) * v[p] + faces) * (T(1) / T(12));
    }
    T acc = T(0);
    #pragma unroll
    for (int dk = -1; dk <= 1; ++dk) {
        T plane = T(0);
        #pragma unroll
        for (int dj = -1; dj <= 1; ++dj) {
            const long long q = p + dk * sz + dj * sy;
            const T row = v[q - 1] + T(2) * v[q] + v[q + 1];
            plane += (dj == 0 ? T(2) : T(1)) * row;
        }
        acc += (dk == 0 ? T(2) : T(1)) * plane;
    }
    return acc * (T(1) / T(64));
}

// Coarse-grid outputs, any may be null: rc = I r (0 on the shell);
// wc = approximation restriction of uf (approx 0: injection everywhere;
// 1: the kind weighting inside, injection on the shell); uc = copy of wc.
template <typename T>
__global__ void __launch_bounds__(BX * BY) k_restrict(const T* __restrict__ uf, const T* __restrict__ rf, int nf,
                                                      T* __restrict__ wc, T* __restrict__ uc, T* __restrict__ rc,
                                                      int nc, int kind, int approx)
{
    const int I = blockIdx.x * BX + threadIdx.x;
    const int J = blockIdx.y * BY + threadIdx.y;
    const int K = blockIdx.z;
    if (I >= nc || J >= nc) return;
    const long long pc = lin(I, J, K, nc);
    const long long pf = lin(2 * I, 2 * J, 2 * K, nf);
    const long long sy = nf, sz = (long long)nf * nf;
    const bool interior = I > 0 && J > 0 && K > 0 && I < nc - 1 && J < nc - 1 && K < nc - 1;
    if (rc) rc[pc] = interior ? weighted_restrict(rf, pf, sy, sz, kind) : T(0);
    if (uf) {
        const T w = (interior && approx == 1) ? weighted_restrict(uf, pf, sy, sz, kind) : uf[pf];
        if (wc) wc[pc] = w;
        if (uc) uc[pc] = w;
    }
}

// Trilinear interpolation at fine interior points: along each axis an even
// index sits on a coarse point, an odd one halfway between two.  Thread
// (I, j, k) writes fine points i = 2I + 1 and 2I + 2 of row (j, k): with
// L(I) the coarse values d = uc - wc (add != 0) or d = uc (add == 0) summed
// over the one, two or four coarse rows around (j, k) and scaled by their
// weight, fine 2I + 2 gets L(I + 1) and fine 2I + 1 gets (L(I) + L(I + 1)) / 2.
// A lane computes L(I + 1) and takes L(I) from the lane before it.
// add != 0: uf += I(uc - wc) (coarse-grid correction); add == 0: uf = I(uc).
// Grid: prolong_grid(nf), blocks of BX x BY.
template <typename T>
__global__ void __launch_bounds__(BX * BY) k_prolong(const T* __restrict__ uc, const T* __restrict__ wc, int nc,
                                                     T* __restrict__ uf, int nf, int add)
{
    const int I = blockIdx.x * BX + threadIdx.x;
    const int j = 1 + blockIdx.y * BY + threadIdx.y;
    const int k = 1 + blockIdx.z;
    const bool row = j <= nf - 2;   // uniform over the warp (BX = 32)
    const int J0 = j >> 1, K0 = k >> 1, oj = j & 1, ok = k & 1;
    const T w = T(1) / T(1 << (oj + ok));
    auto line = [&](int Ic) -> T {
        T s = T(0);
        for (int dk = 0; dk <= ok; ++dk)
            for (int dj = 0; dj <= oj; ++dj) {
                const long long q = lin(Ic, J0 + dj, K0 + dk, nc);
                s += add ? (uc[q] - wc[q]) : uc[q];
            }
        return s * w;
    };
    const bool act = row && I <= nc - 2;
    const T b = act ? line(I + 1) : T(0);
    T a = __shfl_up_sync(0xffffffffu, b, 1);
    if (!act) return;
    if (threadIdx.x == 0) a = line(I);
    const long long p = lin(2 * I + 1, j, k, nf);
    const T mid = (a + b) * T(0.5);
    uf[p] = add ? uf[p] + mid : mid;
    if (2 * I + 2 <= nf - 2) uf[p + 1] = add ? uf[p + 1] + b : b;
}

inline dim3 prolong_grid(int nf)
{
    const int nc = (nf + 1) / 2;
    return dim3((nc - 1 + BX - 1) / BX, (nf - 2 + BY - 1) / BY, nf - 2);
}

template <typename T>
__global__ void k_inject(const T* __restrict__ vf, int nf, T* __restrict__ vc, int nc)
{
    const int I = blockIdx.x * BX + threadIdx.x;
    const int J = blockIdx.y * BY + threadIdx.y;
    const int K = blockIdx.z;
    if (I >= nc || J >= nc) return;
    vc[lin(I, J, K, nc)] = vf[lin(2 * I, 2 * J, 2 * K, nf)];
}

template <typename T>
__global__ void k_zero_interior(T* u, int n)
{
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = blockIdx.z;
    if (i < 1 || j < 1 || k < 1 || i > n - 2 || j > n - 2 || k > n - 2) return;
    u[lin(i, j, k, n)] = T(0);
}

inline dim3 grid_of(int n) { return dim3((n + BX - 1) / BX, (n + BY - 1) / BY, n); }

}  // namespace xfer
}  // namespace ma
