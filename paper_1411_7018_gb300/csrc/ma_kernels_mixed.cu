// ma_kernels_mixed.cu -- kernels of the mixed-precision solve: FP32 FAS
// V-cycles on a correction e under an FP64 fine-grid residual and update
// (defect correction).  The paper computes in FP64 throughout and notes that
// round-off limits its finest grid (round-off remark of Example 4, Section 4);
// here FP64 is kept exactly where that round-off bites -- the fine residual
// f - det(D^2_h u) and the update u += e -- and everything that only has to
// produce a correction runs in FP32.
//
// Correction operator.  With u fixed, the correction problem is
//     N(e) = det(B + K(e)) - det(B) = r,    B = D^2_h u,  K(e) = D^2_h e,
// which is exactly det(D^2_h (u + e)) = f when r = f - det(D^2_h u).  For 3x3
// matrices det(B + K) - det(B) = tr(cof(B) K) + tr(B cof(K)) + det(K), so N(e)
// is evaluated without subtracting two O(f) numbers: its FP32 round-off scales
// with the correction, not with f.  B comes from an FP32 hi/lo split of u
// (u = hi + lo to ~2^-48 relative) with differences to the centre taken first,
// which keeps ~1e-5 relative accuracy where FP32 u alone would give percent
// errors at 513^3.  The point update solves N = r for the centre value with
// the same smallest-root rule as the FP64 smoother (Section 2, Eq. realroots):
// det(G - z I) = det(B) + r with G = B + K, the root below the smallest
// eigenvalue of G; FP32 Newton from z = 0 when G is positive definite, else
// the FP64 routines of ma_point.cuh on the same data.
#include <atomic>

#include "ma_internal.h"
#include "ma_point.cuh"
#include "ma_transfer.cuh"
#include "ma_residual.cuh"

namespace ma {

namespace {

using xfer::BX;
using xfer::BY;
using xfer::grid_of;
using xfer::lin;

struct S3f {
    float xx, yy, zz, xy, xz, yz;
};

// Scaled Hessian (divided by h^2) from a difference functor d(di, dj, dk) =
// value at the offset minus the centre value; every user builds B and K
// through this one routine, in the same order of operations.
template <typename D>
__device__ __forceinline__ S3f hess_from_diff(D d, float inv_h2)
{
    S3f B;
    const float q = 0.25f * inv_h2;
    B.xx = (d(1, 0, 0) + d(-1, 0, 0)) * inv_h2;
    B.yy = (d(0, 1, 0) + d(0, -1, 0)) * inv_h2;
    B.zz = (d(0, 0, 1) + d(0, 0, -1)) * inv_h2;
    B.xy = ((d(1, 1, 0) + d(-1, -1, 0)) - (d(-1, 1, 0) + d(1, -1, 0))) * q;
    B.xz = ((d(1, 0, 1) + d(-1, 0, -1)) - (d(-1, 0, 1) + d(1, 0, -1))) * q;
    B.yz = ((d(0, 1, 1) + d(0, -1, -1)) - (d(0, 1, -1) + d(0, -1, 1))) * q;
    return B;
}

// B = D^2_h u from the hi/lo split of u in global memory.
__device__ __forceinline__ S3f base_hess(const float* __restrict__ hi, const float* __restrict__ lo, long long p,
                                         long long sy, long long sz, float inv_h2)
{
    const float vh = hi[p], vl = lo[p];
    return hess_from_diff(
        [&](int di, int dj, int dk) -> float {
            const long long o = p + di + dj * sy + dk * sz;
            return (__ldg(hi + o) - vh) + (__ldg(lo + o) - vl);
        },
        inv_h2);
}

// K = D^2_h e at the current centre value e0, e in global memory.
__device__ __forceinline__ S3f corr_hess(const float* __restrict__ e, long long p, long long sy, long long sz,
                                         float e0, float inv_h2)
{
    return hess_from_diff(
        [&](int di, int dj, int dk) -> float { return __ldg(e + p + di + dj * sy + dk * sz) - e0; }, inv_h2);
}

__device__ __forceinline__ float det3(const S3f& A)
{
    return A.xx * (A.yy * A.zz - A.yz * A.yz) - A.xy * (A.xy * A.zz - A.xz * A.yz) +
           A.xz * (A.xy * A.yz - A.yy * A.xz);
}

// tr(cof(A) X) for symmetric A, X.
__device__ __forceinline__ float cof_dot(const S3f& A, const S3f& X)
{
    const float cxx = A.yy * A.zz - A.yz * A.yz;
    const float cyy = A.xx * A.zz - A.xz * A.xz;
    const float czz = A.xx * A.yy - A.xy * A.xy;
    const float cxy = A.xz * A.yz - A.xy * A.zz;
    const float cxz = A.xy * A.yz - A.xz * A.yy;
    const float cyz = A.xy * A.xz - A.xx * A.yz;
    return cxx * X.xx + cyy * X.yy + czz * X.zz + 2.0f * (cxy * X.xy + cxz * X.xz + cyz * X.yz);
}

// N = det(B + K) - det(B) by the 3x3 expansion.
__device__ __forceinline__ float delta_det(const S3f& B, const S3f& K)
{
    return cof_dot(B, K) + cof_dot(K, B) + det3(K);
}

// Smallest-root update of the correction problem at one point; returns z with
// e_new = e0 + h^2 z / 2.
__device__ __forceinline__ float corr_root(const S3f& B, const S3f& K, float r, bool* nonconvex)
{
    S3f G;
    G.xx = B.xx + K.xx; G.yy = B.yy + K.yy; G.zz = B.zz + K.zz;
    G.xy = B.xy + K.xy; G.xz = B.xz + K.xz; G.yz = B.yz + K.yz;
    const float c = delta_det(B, K) - r;   // F(0)
    const float T = G.xx + G.yy + G.zz;
    const float M = (G.xx * G.yy - G.xy * G.xy) + (G.xx * G.zz - G.xz * G.xz) + (G.yy * G.zz - G.yz * G.yz);
    const float dG = det3(G);
    const bool pd = G.xx > 0.0f && G.xx * G.yy - G.xy * G.xy > 0.0f && dG > 0.0f;
    const float scale = fabsf(G.xx) + fabsf(G.yy) + fabsf(G.zz) + fabsf(G.xy) + fabsf(G.xz) + fabsf(G.yz);
    if (pd && M > 0.05f * scale * scale) {
        // F(z) = c - z M + z^2 T - z^3 = det(G - zI) - det(B) - r
        float z = 0.0f;
        for (int it = 0; it < 30; ++it) {
            const float F = c - z * (M - z * (T - z));
            const float Mz = M - z * (2.0f * T - 3.0f * z);
            const float dz = __fdividef(F, Mz);
            z += dz;
            if (!isfinite(z)) break;
            if (fabsf(dz) <= 1e-6f * fabsf(z) + 1e-12f * scale) return z;
        }
    }
    // FP64 on the same data: the target is det(G - zI) = det(B) + r.
    HessS H;
    H.A = G.xx; H.B = G.yy; H.C = G.zz; H.R = G.xy; H.S = G.xz; H.T = G.yz;
    const double tot = (double)det3(B) + (double)r;
    if (tot > 0.0) return (float)root_f64_monotone(H, tot);
    *nonconvex = true;
    return (float)root_f64_all_real_min(H, tot);
}

__host__ __device__ __forceinline__ int colour_count(int n, int parity) { return parity ? (n - 1) / 2 : (n - 3) / 2; }

// ---------------------------------------------------------------------------
// Colour-major stores.  Colour c = (i&1)|(j&1)<<1|(k&1)<<2; its interior
// points form a dense ni x nj x nk box (ni = interior indices of parity i&1
// along an axis), and the boxes of colours 0..7 follow each other.  A warp of
// one colour phase then reads contiguous memory.  Two per-level arrays use
// this layout: the base Hessian B = D^2_h u (six FP32 components per point,
// component-major inside each colour box, refreshed once per outer
// iteration) and the correction right-hand side rhs.  (A BF16 B halves the
// bytes a sweep streams, but its 2^-9 error cost an extra FP64 outer
// iteration per solve, more than the sweeps saved.)
// ---------------------------------------------------------------------------

// Points of colours 0..c-1.
__host__ __device__ __forceinline__ long long cm_offset(int n, int c)
{
    long long off = 0;
    for (int q = 0; q < c; ++q)
        off += (long long)colour_count(n, q & 1) * colour_count(n, (q >> 1) & 1) * colour_count(n, (q >> 2) & 1);
    return off;
}

struct CmPos {
    long long off;   // points of lower colours
    long long cnt;   // points of this colour
    long long idx;   // position inside this colour's box
};

// Colour-major position of interior point (i, j, k).
__device__ __forceinline__ CmPos cm_pos(int i, int j, int k, int n)
{
    const int pi = i & 1, pj = j & 1, pk = k & 1;
    const int ni = colour_count(n, pi), nj = colour_count(n, pj), nk = colour_count(n, pk);
    const int ii = (i - (pi ? 1 : 2)) >> 1, jj = (j - (pj ? 1 : 2)) >> 1, kk = (k - (pk ? 1 : 2)) >> 1;
    CmPos r;
    r.off = cm_offset(n, pi | (pj << 1) | (pk << 2));
    r.cnt = (long long)ni * nj * nk;
    r.idx = ((long long)kk * nj + jj) * ni + ii;
    return r;
}

// B is read once per colour phase: streaming loads (evict-first) keep it from
// pushing e, which every phase re-reads through its stencil, out of L2.
__device__ __forceinline__ S3f load_b(const float* __restrict__ b, long long cnt)
{
    S3f B;
    B.xx = __ldcs(b);
    B.yy = __ldcs(b + cnt);
    B.zz = __ldcs(b + 2 * cnt);
    B.xy = __ldcs(b + 3 * cnt);
    B.xz = __ldcs(b + 4 * cnt);
    B.yz = __ldcs(b + 5 * cnt);
    return B;
}

// B from the hi/lo split, stored at the point's colour-major slot.
__global__ void __launch_bounds__(BX * BY) k_base_colour(const float* __restrict__ hi, const float* __restrict__ lo,
                                                         float* __restrict__ bstore, int n, float inv_h2)
{
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = blockIdx.z;
    if (i < 1 || j < 1 || k < 1 || i > n - 2 || j > n - 2 || k > n - 2) return;
    const long long sy = n, sz = (long long)n * n;
    const S3f B = base_hess(hi, lo, lin(i, j, k, n), sy, sz, inv_h2);
    const CmPos c = cm_pos(i, j, k, n);
    float* b = bstore + 6 * c.off + c.idx;
    b[0] = B.xx;
    b[c.cnt] = B.yy;
    b[2 * c.cnt] = B.zz;
    b[3 * c.cnt] = B.xy;
    b[4 * c.cnt] = B.xz;
    b[5 * c.cnt] = B.yz;
}

// Natural-layout interior values -> colour-major order.
__global__ void __launch_bounds__(BX * BY) k_to_cm(const float* __restrict__ nat, float* __restrict__ cm, int n)
{
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = blockIdx.z;
    if (i < 1 || j < 1 || k < 1 || i > n - 2 || j > n - 2 || k > n - 2) return;
    const CmPos c = cm_pos(i, j, k, n);
    cm[c.off + c.idx] = nat[lin(i, j, k, n)];
}

// Correction smoother, one colour per launch: bc / rc point at this colour's
// B and rhs boxes; e is in the natural layout (19-point stencil).
template <int PI, int PJ, int PK>
__global__ void __launch_bounds__(BX * BY) k_smooth_corr(float* e, const float* __restrict__ bc,
                                                          const float* __restrict__ rc, int n, float inv_h2,
                                                          float h2half, unsigned long long* events)
{
    const int ii = blockIdx.x * BX + threadIdx.x;
    const int jj = blockIdx.y * BY + threadIdx.y;
    const int kk = blockIdx.z;
    const int ni = colour_count(n, PI), nj = colour_count(n, PJ);
    if (ii >= ni || jj >= nj) return;
    const int i = (PI ? 1 : 2) + 2 * ii, j = (PJ ? 1 : 2) + 2 * jj, k = (PK ? 1 : 2) + 2 * kk;
    const long long cnt = (long long)ni * nj * colour_count(n, PK);
    const long long idx = ((long long)kk * nj + jj) * ni + ii;
    const S3f B = load_b(bc + idx, cnt);
    const long long sy = n, sz = (long long)n * n;
    const long long p = lin(i, j, k, n);
    const float e0 = e[p];
    const S3f K = corr_hess(e, p, sy, sz, e0, inv_h2);
    bool nonconvex = false;
    const float z = corr_root(B, K, __ldcs(rc + idx), &nonconvex);
    e[p] = fmaf(h2half, z, e0);
    if (nonconvex && events) atomicAdd(events, 1ull);
}

template <int C>
cudaError_t launch_colour_corr(float* e, const float* bstore, const float* rhs_cm, int n, float inv_h2,
                               float h2half, unsigned long long* ev, cudaStream_t s)
{
    constexpr int PI = C & 1, PJ = (C >> 1) & 1, PK = (C >> 2) & 1;
    const int ni = colour_count(n, PI), nj = colour_count(n, PJ), nk = colour_count(n, PK);
    if (ni <= 0 || nj <= 0 || nk <= 0) return cudaSuccess;
    dim3 grid((ni + BX - 1) / BX, (nj + BY - 1) / BY, nk);
    const long long off = cm_offset(n, C);
    count_launches(1);
    k_smooth_corr<PI, PJ, PK><<<grid, dim3(BX, BY), 0, s>>>(e, bstore + 6 * off, rhs_cm + off, n, inv_h2, h2half,
                                                             ev);
    return cudaGetLastError();
}

// res = rhs - N(e) on the interior (natural layout), 0 on the shell.
__global__ void __launch_bounds__(BX * BY) k_residual_corr(const float* __restrict__ e,
                                                           const float* __restrict__ bstore,
                                                           const float* __restrict__ rhs_cm,
                                                           float* __restrict__ res, int n, float inv_h2)
{
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= n || j >= n) return;
    const long long p = lin(i, j, k, n);
    float v = 0.0f;
    if (i > 0 && j > 0 && k > 0 && i < n - 1 && j < n - 1 && k < n - 1) {
        const long long sy = n, sz = (long long)n * n;
        const CmPos c = cm_pos(i, j, k, n);
        const S3f B = load_b(bstore + 6 * c.off + c.idx, c.cnt);
        const S3f K = corr_hess(e, p, sy, sz, e[p], inv_h2);
        v = rhs_cm[c.off + c.idx] - delta_det(B, K);
    }
    res[p] = v;
}

// rhs_H = N_H(w_H) + res_H on the coarse interior, written colour-major.
__global__ void __launch_bounds__(BX * BY) k_coarse_rhs_corr(const float* __restrict__ w,
                                                             const float* __restrict__ bstore,
                                                             const float* __restrict__ resc,
                                                             float* __restrict__ rhs_cm, int n, float inv_h2)
{
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = blockIdx.z;
    if (i < 1 || j < 1 || k < 1 || i > n - 2 || j > n - 2 || k > n - 2) return;
    const long long p = lin(i, j, k, n);
    const long long sy = n, sz = (long long)n * n;
    const CmPos c = cm_pos(i, j, k, n);
    const S3f B = load_b(bstore + 6 * c.off + c.idx, c.cnt);
    const S3f K = corr_hess(w, p, sy, sz, w[p], inv_h2);
    rhs_cm[c.off + c.idx] = delta_det(B, K) + resc[p];
}

// Coarsest correction grid: one block, shared memory, FP32 sweeps until
// max|de| <= 2e-6 max|e| (FP32 resolution of the correction; at most 40
// sweeps), or a fixed count.
constexpr int CT = 256;

__device__ __forceinline__ S3f corr_hess_sm(const float* e, int p, int sy, int sz, float e0, float inv_h2)
{
    return hess_from_diff([&](int di, int dj, int dk) -> float { return e[p + di + dj * sy + dk * sz] - e0; },
                          inv_h2);
}

// smem: e (n^3, natural), B (6 floats per interior point, colour-major),
// rhs (colour-major).
__global__ void __launch_bounds__(CT) k_coarsest_corr(float* e, const float* __restrict__ bstore,
                                                      const float* __restrict__ rhs_cm, int n, float inv_h2,
                                                      float h2half, int sweeps, unsigned long long* events)
{
    extern __shared__ float smf[];
    const int m = n * n * n;
    const int mi = (n - 2) * (n - 2) * (n - 2);
    float* se = smf;
    float* sb = smf + m;
    float* sr = smf + m + 6 * mi;
    __shared__ float red[CT / 32][2];
    __shared__ int stop;
    for (int q = threadIdx.x; q < m; q += CT) se[q] = e[q];
    for (int q = threadIdx.x; q < 6 * mi; q += CT) sb[q] = bstore[q];
    for (int q = threadIdx.x; q < mi; q += CT) sr[q] = rhs_cm[q];
    __syncthreads();
    const int max_sweeps = sweeps > 0 ? sweeps : 40;
    unsigned long long ev = 0;
    for (int s = 0; s < max_sweeps; ++s) {
        float du = 0.0f, um = 0.0f;
        long long off = 0;
        for (int c = 0; c < 8; ++c) {
            const int pi = c & 1, pj = (c >> 1) & 1, pk = (c >> 2) & 1;
            const int ni = colour_count(n, pi), nj = colour_count(n, pj), nk = colour_count(n, pk);
            const int cnt = (ni > 0 && nj > 0 && nk > 0) ? ni * nj * nk : 0;
            for (int t = threadIdx.x; t < cnt; t += CT) {
                const int i = (pi ? 1 : 2) + 2 * (t % ni);
                const int j = (pj ? 1 : 2) + 2 * ((t / ni) % nj);
                const int k = (pk ? 1 : 2) + 2 * (t / (ni * nj));
                const int p = (k * n + j) * n + i;
                const float e0 = se[p];
                const float* b = sb + 6 * off + t;
                S3f B;
                B.xx = b[0]; B.yy = b[cnt]; B.zz = b[2 * cnt]; B.xy = b[3 * cnt]; B.xz = b[4 * cnt]; B.yz = b[5 * cnt];
                const S3f K = corr_hess_sm(se, p, n, n * n, e0, inv_h2);
                bool nonconvex = false;
                const float z = corr_root(B, K, sr[off + t], &nonconvex);
                const float v = fmaf(h2half, z, e0);
                se[p] = v;
                du = fmaxf(du, fabsf(v - e0));
                um = fmaxf(um, fabsf(v));
                ev += nonconvex ? 1ull : 0ull;
            }
            off += cnt;
            __syncthreads();
        }
        if (sweeps > 0) continue;
        for (int o = 16; o > 0; o >>= 1) {
            du = fmaxf(du, __shfl_down_sync(0xffffffffu, du, o));
            um = fmaxf(um, __shfl_down_sync(0xffffffffu, um, o));
        }
        if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5][0] = du; red[threadIdx.x >> 5][1] = um; }
        __syncthreads();
        if (threadIdx.x == 0) {
            float a = 0.0f, b = 0.0f;
            for (int w = 0; w < CT / 32; ++w) { a = fmaxf(a, red[w][0]); b = fmaxf(b, red[w][1]); }
            stop = (a <= 2e-6f * b) ? 1 : 0;
        }
        __syncthreads();
        if (stop) break;
    }
    for (int q = threadIdx.x; q < m; q += CT) e[q] = se[q];
    if (events && ev) atomicAdd(events, ev);
}

// u += e (optional), then u = hi + lo (FP32 split) and e = 0, over the whole grid.
__global__ void k_split_update(double* __restrict__ u, float* __restrict__ e, float* __restrict__ hi,
                               float* __restrict__ lo, long long m, int apply)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= m) return;
    double v = u[p];
    if (apply) {
        v += f2d(e[p]);
        u[p] = v;
    }
    // hi = v truncated to FP32; v - hi is exact in FP64 and below one FP32
    // ulp of hi, so lo = its FP32 truncation keeps v = hi + lo to ~2^-47.
    const float h = d2f_trunc(v);
    hi[p] = h;
    lo[p] = d2f_trunc(v - f2d(h));
    e[p] = 0.0f;
}

// FP64 fine residual, written as FP32 in colour-major order (the correction
// problem's right-hand side); the shell is not stored.
struct CmF32Out {
    float* r;
    __device__ __forceinline__ void put(long long, int i, int j, int k, int n, double, float v32) const
    {
        const CmPos c = cm_pos(i, j, k, n);
        r[c.off + c.idx] = v32;
    }
    __device__ __forceinline__ void zero(long long) const {}
};

}  // namespace

size_t base_store_bytes(int n)
{
    return n >= 3 ? 6 * sizeof(float) * (size_t)(n - 2) * (n - 2) * (n - 2) : 0;
}

size_t cm_points(int n) { return n >= 3 ? (size_t)(n - 2) * (n - 2) * (n - 2) : 0; }

cudaError_t launch_base_colour(const float* hi, const float* lo, void* bstore, int n, double h, cudaStream_t s)
{
    count_launches(1);
    k_base_colour<<<grid_of(n), dim3(BX, BY), 0, s>>>(hi, lo, (float*)bstore, n, (float)(1.0 / (h * h)));
    return cudaGetLastError();
}

cudaError_t launch_to_cm(const float* nat, float* cm, int n, cudaStream_t s)
{
    count_launches(1);
    k_to_cm<<<grid_of(n), dim3(BX, BY), 0, s>>>(nat, cm, n);
    return cudaGetLastError();
}

cudaError_t launch_smooth_corr(float* e, const void* bstore, const float* rhs_cm, int n, double h, int nsweeps,
                               unsigned long long* events, cudaStream_t s)
{
    const float inv_h2 = (float)(1.0 / (h * h));
    const float h2half = (float)(0.5 * h * h);
    const float* b = (const float*)bstore;
    for (int sw = 0; sw < nsweeps; ++sw) {
        cudaError_t e_;
        if ((e_ = launch_colour_corr<0>(e, b, rhs_cm, n, inv_h2, h2half, events, s)) != cudaSuccess) return e_;
        if ((e_ = launch_colour_corr<1>(e, b, rhs_cm, n, inv_h2, h2half, events, s)) != cudaSuccess) return e_;
        if ((e_ = launch_colour_corr<2>(e, b, rhs_cm, n, inv_h2, h2half, events, s)) != cudaSuccess) return e_;
        if ((e_ = launch_colour_corr<3>(e, b, rhs_cm, n, inv_h2, h2half, events, s)) != cudaSuccess) return e_;
        if ((e_ = launch_colour_corr<4>(e, b, rhs_cm, n, inv_h2, h2half, events, s)) != cudaSuccess) return e_;
        if ((e_ = launch_colour_corr<5>(e, b, rhs_cm, n, inv_h2, h2half, events, s)) != cudaSuccess) return e_;
        if ((e_ = launch_colour_corr<6>(e, b, rhs_cm, n, inv_h2, h2half, events, s)) != cudaSuccess) return e_;
        if ((e_ = launch_colour_corr<7>(e, b, rhs_cm, n, inv_h2, h2half, events, s)) != cudaSuccess) return e_;
    }
    return cudaSuccess;
}

cudaError_t launch_residual_corr(const float* e, const void* bstore, const float* rhs_cm, float* res, int n,
                                 double h, cudaStream_t s)
{
    count_launches(1);
    k_residual_corr<<<grid_of(n), dim3(BX, BY), 0, s>>>(e, (const float*)bstore, rhs_cm, res, n,
                                                        (float)(1.0 / (h * h)));
    return cudaGetLastError();
}

cudaError_t launch_coarse_rhs_corr(const float* w, const void* bstore, const float* resc, float* rhs_cm, int nc,
                                   double H, cudaStream_t s)
{
    count_launches(1);
    k_coarse_rhs_corr<<<grid_of(nc), dim3(BX, BY), 0, s>>>(w, (const float*)bstore, resc, rhs_cm, nc,
                                                           (float)(1.0 / (H * H)));
    return cudaGetLastError();
}

cudaError_t launch_restrict_level_f32(const float* ef, const float* rf, int nf, float* wc, float* ec, float* rc,
                                      int kind, int approx, cudaStream_t s)
{
    const int nc = (nf + 1) / 2;
    count_launches(1);
    xfer::k_restrict<float><<<grid_of(nc), dim3(BX, BY), 0, s>>>(ef, rf, nf, wc, ec, rc, nc, kind, approx);
    return cudaGetLastError();
}

cudaError_t launch_prolong_add_f32(const float* ec, const float* wc, int nc, float* ef, cudaStream_t s)
{
    const int nf = 2 * nc - 1;
    count_launches(1);
    xfer::k_prolong<float><<<grid_of(nf), dim3(BX, BY), 0, s>>>(ec, wc, nc, ef, nf, 1);
    return cudaGetLastError();
}

cudaError_t launch_inject_f32(const float* vf, int nf, float* vc, cudaStream_t s)
{
    const int nc = (nf + 1) / 2;
    count_launches(1);
    xfer::k_inject<float><<<grid_of(nc), dim3(BX, BY), 0, s>>>(vf, nf, vc, nc);
    return cudaGetLastError();
}

static size_t coarsest_corr_smem(int n)
{
    return sizeof(float) * ((size_t)n * n * n + 7 * cm_points(n));
}

cudaError_t launch_coarsest_corr(float* e, const void* bstore, const float* rhs_cm, int n, double h, int sweeps,
                                 unsigned long long* events, cudaStream_t s)
{
    count_launches(1);
    k_coarsest_corr<<<1, CT, coarsest_corr_smem(n), s>>>(e, (const float*)bstore, rhs_cm, n,
                                                         (float)(1.0 / (h * h)), (float)(0.5 * h * h), sweeps,
                                                         events);
    return cudaGetLastError();
}

cudaError_t prepare_coarsest_f64();

cudaError_t prepare_coarsest_kernels()
{
    cudaError_t e = prepare_coarsest_f64();
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_coarsest_corr, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)coarsest_corr_smem(17));
}

cudaError_t launch_split_update(double* u, float* e, float* hi, float* lo, int n, int apply, cudaStream_t s)
{
    const long long m = (long long)n * n * n;
    count_launches(1);
    k_split_update<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(u, e, hi, lo, m, apply);
    return cudaGetLastError();
}

cudaError_t launch_residual64_to32(const double* u, const double* rhs, float* r_cm, int n, double h,
                                   double* partials, cudaStream_t s)
{
    const double h2 = h * h;
    count_launches(1);
    const int kz = n < 16 ? n : 16;
    const int kchunk = (n + kz - 1) / kz;
    resid::k_residual_col<CmF32Out><<<resid::grid_for(n, kz), dim3(resid::RX, resid::RY), 0, s>>>(
        u, rhs, CmF32Out{r_cm}, n, 1.0 / (64.0 * h2 * h2 * h2), partials, kchunk);
    return cudaGetLastError();
}

}  // namespace ma
