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

__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

// Restriction I_h^H at a fine point p with strides sy, sz.  kind 0: the
// printed 7-point half weighting (6 centre + 6 faces) / 12; kind 1: 27-point
// full weighting, separable (1 2 1)/4 along each axis.  Written with explicit
// fused multiply-adds in a fixed order so that every kernel that inlines it
// rounds identically.
template <typename T>
__device__ __forceinline__ T weighted_restrict(const T* __restrict__ v, long long p, long long sy, long long sz,
                                               int kind)
{
    if (kind == 0) {
        const T faces = (v[p + 1] + v[p - 1]) + (v[p + sy] + v[p - sy]) + (v[p + sz] + v[p - sz]);
        return fma_t(T(6), v[p], faces) * (T(1) / T(12));
    }
    T acc = T(0);
#pragma unroll
    for (int dk = -1; dk <= 1; ++dk) {
        T plane = T(0);
#pragma unroll
        for (int dj = -1; dj <= 1; ++dj) {
            const long long q = p + dk * sz + dj * sy;
            const T row = fma_t(T(2), v[q], v[q - 1] + v[q + 1]);
            plane = fma_t(dj == 0 ? T(2) : T(1), row, plane);
        }
        acc = fma_t(dk == 0 ? T(2) : T(1), plane, acc);
    }
    return acc * (T(1) / T(64));
}

// Coarse-grid outputs, any may be null: rc = I r (0 on the shell);
// wc = approximation restriction of uf (approx 0: injection everywhere;
// 1: the kind weighting inside, injection on the shell); uc = copy of wc.
// The block body takes its block index as an argument, so that a batched
// launch over the grids of several hierarchies runs the same code.
template <typename T>
__device__ __forceinline__ void restrict_block(const T* __restrict__ uf, const T* __restrict__ rf, int nf,
                                               T* __restrict__ wc, T* __restrict__ uc, T* __restrict__ rc, int nc,
                                               int kind, int approx, uint3 bid)
{
    const int I = bid.x * BX + threadIdx.x;
    const int J = bid.y * BY + threadIdx.y;
    const int K = bid.z;
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

template <typename T>
__global__ void __launch_bounds__(BX * BY) k_restrict(const T* __restrict__ uf, const T* __restrict__ rf, int nf,
                                                      T* __restrict__ wc, T* __restrict__ uc, T* __restrict__ rc,
                                                      int nc, int kind, int approx)
{
    restrict_block<T>(uf, rf, nf, wc, uc, rc, nc, kind, approx, blockIdx);
}

// Trilinear interpolation at fine interior points: along each axis an even
// index sits on a coarse point, an odd one halfway between two.  With L(I) the
// coarse values d = uc - wc (add != 0) or d = uc (add == 0) summed over the
// one, two or four coarse rows around fine row (j, k) and scaled by their
// weight, fine point 2I gets L(I) and fine point 2I + 1 gets
// (L(I) + L(I + 1)) / 2.
// add != 0: uf += I(uc - wc) (coarse-grid correction); add == 0: uf = I(uc).
//
// Thread (I, J, K) owns the coarse cell between coarse points I..I+1,
// J..J+1, K..K+1: the four fine rows j in {2J, 2J + 1}, k in {2K, 2K + 1}
// (rows on the shell skipped) and two fine points of each.  It loads the four
// coarse rows' values at column I + 1 once for all four fine rows and takes
// those at column I from the lane before it (lane 0 loads them).  nf is odd,
// so in fine row (j, k) the point pair that starts at an even linear index is
// (2I, 2I + 1) when j + k is even and (2I + 1, 2I + 2) when it is odd: each
// lane moves that pair as one aligned 2-element access (scalar accesses
// where the pair would reach the shell, or where uf is not aligned to two
// elements).  With add != 0 the fine pairs are loaded first, so their HBM
// latency overlaps the coarse loads.  Every fine value is the same
// expression, summed in the same order (dk outer, dj inner), as one thread
// per fine point would form it.
// Grid: prolong_grid(nf), blocks of BX x BY.
template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
    using type = float2;
};
template <>
struct Vec2<double> {
    using type = double2;
};

template <typename T>
__device__ __forceinline__ void prolong_block(const T* __restrict__ uc, const T* __restrict__ wc, int nc,
                                              T* __restrict__ uf, int nf, int add, uint3 bid)
{
    using V = typename Vec2<T>::type;
    const int I = bid.x * BX + threadIdx.x;
    const int J = bid.y * BY + threadIdx.y;
    const int K = bid.z;
    const bool act = I <= nc - 2 && J <= nc - 2;   // J uniform over the warp (BX = 32)
    const bool vec = ((unsigned long long)uf & (2 * sizeof(T) - 1)) == 0;
    // the fine pair of row (j, k): its first point p0 and whether both points
    // are interior (else only the second, 2I + 1, for even rows at I = 0, or
    // only the first, 2I + 1, for odd rows at the far end)
    auto pair_at = [&](int j, int k, long long* p0, bool* full) {
        const bool even = ((j + k) & 1) == 0;
        *p0 = lin(even ? 2 * I : 2 * I + 1, j, k, nf);
        *full = even ? I >= 1 : 2 * I + 2 <= nf - 2;
        return even;
    };
    T f[2][2][2];
#pragma unroll
    for (int ok = 0; ok < 2; ++ok)
#pragma unroll
        for (int oj = 0; oj < 2; ++oj) {
            f[ok][oj][0] = f[ok][oj][1] = T(0);
            const int j = 2 * J + oj, k = 2 * K + ok;
            if (!add || !act || j < 1 || k < 1) continue;
            long long p0;
            bool full;
            const bool even = pair_at(j, k, &p0, &full);
            if (full && vec) {
                const V v = *reinterpret_cast<const V*>(uf + p0);
                f[ok][oj][0] = v.x;
                f[ok][oj][1] = v.y;
            } else {
                if (full || !even) f[ok][oj][0] = uf[p0];
                if (full || even) f[ok][oj][1] = uf[p0 + 1];
            }
        }
    T db[2][2], da[2][2];   // [dk][dj]: coarse d at columns I + 1 and I
#pragma unroll
    for (int dk = 0; dk < 2; ++dk)
#pragma unroll
        for (int dj = 0; dj < 2; ++dj) {
            T v = T(0);
            if (act) {
                const long long q = lin(I + 1, J + dj, K + dk, nc);
                v = add ? uc[q] - wc[q] : uc[q];
            }
            db[dk][dj] = v;
        }
#pragma unroll
    for (int dk = 0; dk < 2; ++dk)
#pragma unroll
        for (int dj = 0; dj < 2; ++dj) {
            T v = __shfl_up_sync(0xffffffffu, db[dk][dj], 1);
            if (threadIdx.x == 0 && act) {
                const long long q = lin(I, J + dj, K + dk, nc);
                v = add ? uc[q] - wc[q] : uc[q];
            }
            da[dk][dj] = v;
        }
    if (!act) return;
#pragma unroll
    for (int ok = 0; ok < 2; ++ok)
#pragma unroll
        for (int oj = 0; oj < 2; ++oj) {
            const int j = 2 * J + oj, k = 2 * K + ok;
            if (j < 1 || k < 1) continue;
            const T w = T(1) / T(1 << (oj + ok));
            T sa = T(0), sb = T(0);
#pragma unroll
            for (int dk = 0; dk <= ok; ++dk)
#pragma unroll
                for (int dj = 0; dj <= oj; ++dj) {
                    sa += da[dk][dj];
                    sb += db[dk][dj];
                }
            const T a = sa * w, b = sb * w;
            const T mid = (a + b) * T(0.5);
            long long p0;
            bool full;
            const bool even = pair_at(j, k, &p0, &full);
            const T v0 = even ? a : mid, v1 = even ? mid : b;   // values at p0, p0 + 1
            const T r0 = add ? f[ok][oj][0] + v0 : v0, r1 = add ? f[ok][oj][1] + v1 : v1;
            if (full && vec) {
                V v;
                v.x = r0;
                v.y = r1;
                *reinterpret_cast<V*>(uf + p0) = v;
            } else {
                if (full || !even) uf[p0] = r0;
                if (full || even) uf[p0 + 1] = r1;
            }
        }
}

template <typename T>
__global__ void __launch_bounds__(BX * BY) k_prolong(const T* __restrict__ uc, const T* __restrict__ wc, int nc,
                                                     T* __restrict__ uf, int nf, int add)
{
    prolong_block<T>(uc, wc, nc, uf, nf, add, blockIdx);
}

// One thread per coarse cell (I, J, K), I, J, K in [0, nc - 2].
inline dim3 prolong_grid(int nf)
{
    const int nc = (nf + 1) / 2;
    return dim3((nc - 1 + BX - 1) / BX, (nc - 1 + BY - 1) / BY, nc - 1);
}

// Cubic interpolation (Algorithm 2 step 4) as three 1-D passes, x then y
// then z.  Along an axis, fine index i on a coarse grid of nc points: even i
// is coarse point i/2; odd i, halfway between coarse I0 = (i-1)/2 and I0 + 1,
// takes the cubic through four coarse neighbours -- I0-1 .. I0+2 with weights
// (-1, 9, 9, -1)/16, or the four nearest ones next to either end ((5, 15, -5,
// 1)/16 from the left end, mirrored at the right) -- a 3-point grid the
// quadratic (3, 6, -1)/8 (mirrored for the second interval), a 2-point grid
// the midpoint.  Returns the first coarse index and fills up to 4 weights.
__device__ __forceinline__ int cubic_axis(int i, int nc, double w[4], int* cnt)
{
    if ((i & 1) == 0) {
        w[0] = 1.0;
        *cnt = 1;
        return i >> 1;
    }
    const int I0 = i >> 1;
    if (nc == 2) {
        w[0] = w[1] = 0.5;
        *cnt = 2;
        return 0;
    }
    if (nc == 3) {
        *cnt = 3;
        if (I0 == 0) { w[0] = 0.375; w[1] = 0.75; w[2] = -0.125; }
        else { w[0] = -0.125; w[1] = 0.75; w[2] = 0.375; }
        return 0;
    }
    *cnt = 4;
    if (I0 == 0) {
        w[0] = 0.3125; w[1] = 0.9375; w[2] = -0.3125; w[3] = 0.0625;
        return 0;
    }
    if (I0 == nc - 2) {
        w[0] = 0.0625; w[1] = -0.3125; w[2] = 0.9375; w[3] = 0.3125;
        return nc - 4;
    }
    w[0] = -0.0625; w[1] = 0.5625; w[2] = 0.5625; w[3] = -0.0625;
    return I0 - 1;
}

// One pass along axis AX (0 = x, 1 = y, 2 = z): out has dims ox x oy x oz
// ([z][y][x], x fastest), in has the same dims except nc along AX.  A thread
// per output point (threads run along x); interior_only writes only points
// with every index in 1 .. dim-2 (the last pass, which keeps the Dirichlet
// shell of the target).
template <int AX>
__device__ __forceinline__ void cubic_pass_block(const double* __restrict__ in, double* __restrict__ out, int nc,
                                                 int ox, int oy, int oz, int interior_only, uint3 bid)
{
    const int x = bid.x * BX + threadIdx.x;
    const int y = bid.y * BY + threadIdx.y;
    const int z = bid.z;
    if (x >= ox || y >= oy) return;
    if (interior_only && (x < 1 || x > ox - 2 || y < 1 || y > oy - 2 || z < 1 || z > oz - 2)) return;
    const int ix = AX == 0 ? nc : ox, iy = AX == 1 ? nc : oy;
    const int a = AX == 0 ? x : (AX == 1 ? y : z);
    double w[4];
    int cnt;
    const int I = cubic_axis(a, nc, w, &cnt);
    const long long step = AX == 0 ? 1 : (AX == 1 ? (long long)ix : (long long)ix * iy);
    const int xi = AX == 0 ? I : x, yi = AX == 1 ? I : y, zi = AX == 2 ? I : z;
    const double* src = in + ((long long)zi * iy + yi) * ix + xi;
    double s = w[0] * src[0];
    for (int q = 1; q < cnt; ++q) s = fma(w[q], src[q * step], s);
    out[((long long)z * oy + y) * ox + x] = s;
}

template <int AX>
__global__ void __launch_bounds__(BX * BY) k_cubic_pass(const double* __restrict__ in, double* __restrict__ out,
                                                        int nc, int ox, int oy, int oz, int interior_only)
{
    cubic_pass_block<AX>(in, out, nc, ox, oy, oz, interior_only, blockIdx);
}

template <typename T>
__device__ __forceinline__ void inject_block(const T* __restrict__ vf, int nf, T* __restrict__ vc, int nc, uint3 bid)
{
    const int I = bid.x * BX + threadIdx.x;
    const int J = bid.y * BY + threadIdx.y;
    const int K = bid.z;
    if (I >= nc || J >= nc) return;
    vc[lin(I, J, K, nc)] = vf[lin(2 * I, 2 * J, 2 * K, nf)];
}

template <typename T>
__global__ void k_inject(const T* __restrict__ vf, int nf, T* __restrict__ vc, int nc)
{
    inject_block<T>(vf, nf, vc, nc, blockIdx);
}

template <typename T>
__device__ __forceinline__ void zero_interior_block(T* u, int n, uint3 bid)
{
    const int i = bid.x * BX + threadIdx.x;
    const int j = bid.y * BY + threadIdx.y;
    const int k = bid.z;
    if (i < 1 || j < 1 || k < 1 || i > n - 2 || j > n - 2 || k > n - 2) return;
    u[lin(i, j, k, n)] = T(0);
}

template <typename T>
__global__ void k_zero_interior(T* u, int n)
{
    zero_interior_block<T>(u, n, blockIdx);
}

inline dim3 grid_of(int n) { return dim3((n + BX - 1) / BX, (n + BY - 1) / BY, n); }

}  // namespace xfer
}  // namespace ma
