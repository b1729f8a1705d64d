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
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "ma_internal.h"
#include "ma_batched.cuh"
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

// The FP32 products below are written as explicit fused multiply-adds in a
// fixed order, so that every kernel that inlines them (by-colour and plane
// sweeps, residuals, the fused tail) rounds identically: the compiler may
// otherwise contract a*b + c*d either way depending on the surrounding code.
__device__ __forceinline__ float mdiff(float a, float b, float c, float d) { return fmaf(a, b, -(c * d)); }   // ab - cd

__device__ __forceinline__ float det3(const S3f& A)
{
    const float c1 = mdiff(A.yy, A.zz, A.yz, A.yz);
    const float c2 = mdiff(A.xy, A.zz, A.xz, A.yz);
    const float c3 = mdiff(A.xy, A.yz, A.yy, A.xz);
    return fmaf(A.xz, c3, fmaf(A.xx, c1, -(A.xy * c2)));
}

// tr(cof(A) X) for symmetric A, X.
__device__ __forceinline__ float cof_dot(const S3f& A, const S3f& X)
{
    const float cxx = mdiff(A.yy, A.zz, A.yz, A.yz);
    const float cyy = mdiff(A.xx, A.zz, A.xz, A.xz);
    const float czz = mdiff(A.xx, A.yy, A.xy, A.xy);
    const float cxy = mdiff(A.xz, A.yz, A.xy, A.zz);
    const float cxz = mdiff(A.xy, A.yz, A.xz, A.yy);
    const float cyz = mdiff(A.xy, A.xz, A.xx, A.yz);
    const float diag = fmaf(czz, X.zz, fmaf(cyy, X.yy, cxx * X.xx));
    const float off = fmaf(cyz, X.yz, fmaf(cxz, X.xz, cxy * X.xy));
    return fmaf(2.0f, off, diag);
}

// N = det(B + K) - det(B) by the 3x3 expansion.
__device__ __forceinline__ float delta_det(const S3f& B, const S3f& K)
{
    return cof_dot(B, K) + cof_dot(K, B) + det3(K);
}

// Smallest-root update of the correction problem at one point, z with
// e_new = e0 + h^2 z / 2.  Fast path: FP32 Newton on
// F(z) = det(G - zI) - det(B) - r from z = 0 (its first step is z = F(0) / M)
// when G = B + K is positive definite and not near-degenerate, and the
// target det(B) + r = det(G) - F(0) is clearly positive (Theorem 2.2: then F
// is decreasing and convex left of the smallest eigenvalue of G, which lies
// right of z = 0, and has its one root there; with a target <= 0 Eq.
// (realroots) asks for the smallest real root elsewhere, which only the FP64
// path finds and counts).  It stops once a step is at most 1e-4 |z|: Newton
// converges quadratically there, so the step just taken leaves an error of
// order (1e-4)^2 |z|, below FP32 resolution.  Returns false (z unset) when
// the point needs the FP64 path.
__device__ __forceinline__ bool corr_root_fast(const S3f& B, const S3f& K, float r, float* zout)
{
    S3f G;
    G.xx = B.xx + K.xx; G.yy = B.yy + K.yy; G.zz = B.zz + K.zz;
    G.xy = B.xy + K.xy; G.xz = B.xz + K.xz; G.yz = B.yz + K.yz;
    const float c = delta_det(B, K) - r;   // F(0)
    const float T = G.xx + G.yy + G.zz;
    const float m2 = mdiff(G.xx, G.yy, G.xy, G.xy);
    const float M = m2 + mdiff(G.xx, G.zz, G.xz, G.xz) + mdiff(G.yy, G.zz, G.yz, G.yz);
    const float dG = det3(G);
    const bool pd = G.xx > 0.0f && m2 > 0.0f && dG > 0.0f;
    // with a positive diagonal, |G| summed entrywise is T + |off-diagonals|
    const float scale = T + fabsf(G.xy) + fabsf(G.xz) + fabsf(G.yz);
    if (!(pd && M > 0.05f * (scale * scale))) return false;
    // the target det(B) + r, far enough above 0 that FP32 rounding of the
    // two determinants cannot flip its sign (margin 1e-5 scale^3)
    if (!(dG - c > 1e-5f * (scale * scale * scale))) return false;
    // F(z) = c - z M + z^2 T - z^3 = c - z (M - z (T - z));  M(z) = -F'(z)
    float z = __fdividef(c, M);
    const float T2 = 2.0f * T;
    for (int it = 0; it < 30; ++it) {
        const float F = fmaf(-z, fmaf(-z, T - z, M), c);
        const float Mz = fmaf(-z, fmaf(-3.0f, z, T2), M);
        const float dz = __fdividef(F, Mz);
        z += dz;
        if (fabsf(dz) <= fmaf(1e-4f, fabsf(z), 1e-12f * scale)) {
            *zout = z;
            return isfinite(z);
        }
    }
    return false;
}

// The correction cubic in FP64 from the FP32 data: with G = B + K,
//     F(z) = det(G - zI) - det(B) - r = c - M z + T z^2 - z^3,
// c = tr(cof(B) K) + tr(B cof(K)) + det(K) - r, evaluated without the
// subtraction of two O(f) numbers (det(B) in FP32 would put an error of
// ~1e-7 f into the target and stall defect correction there).
struct CorrCubic {
    double c, M, T, tot;   // tot = det(B) + r = det(G) - c: the sign decides the branch
    double g[6];           // G: xx, yy, zz, xy, xz, yz
};

__device__ __forceinline__ double cof_dot_d(const double* A, const double* X)
{
    const double cxx = A[1] * A[2] - A[5] * A[5];
    const double cyy = A[0] * A[2] - A[4] * A[4];
    const double czz = A[0] * A[1] - A[3] * A[3];
    const double cxy = A[4] * A[5] - A[3] * A[2];
    const double cxz = A[3] * A[5] - A[4] * A[1];
    const double cyz = A[3] * A[4] - A[0] * A[5];
    return cxx * X[0] + cyy * X[1] + czz * X[2] + 2.0 * (cxy * X[3] + cxz * X[4] + cyz * X[5]);
}

__device__ __forceinline__ double det3_d(const double* A)
{
    return A[0] * (A[1] * A[2] - A[5] * A[5]) - A[3] * (A[3] * A[2] - A[4] * A[5]) +
           A[4] * (A[3] * A[5] - A[1] * A[4]);
}

__device__ __forceinline__ CorrCubic corr_cubic(const S3f& B, const S3f& K, float r)
{
    const double b[6] = {B.xx, B.yy, B.zz, B.xy, B.xz, B.yz};
    const double k[6] = {K.xx, K.yy, K.zz, K.xy, K.xz, K.yz};
    CorrCubic C;
    for (int q = 0; q < 6; ++q) C.g[q] = b[q] + k[q];
    C.c = cof_dot_d(b, k) + cof_dot_d(k, b) + det3_d(k) - (double)r;
    C.T = C.g[0] + C.g[1] + C.g[2];
    C.M = (C.g[0] * C.g[1] - C.g[3] * C.g[3]) + (C.g[0] * C.g[2] - C.g[4] * C.g[4]) +
          (C.g[1] * C.g[2] - C.g[5] * C.g[5]);
    C.tot = det3_d(C.g) - C.c;
    return C;
}

__device__ __forceinline__ double corr_F(const CorrCubic& C, double z) { return C.c - z * (C.M - z * (C.T - z)); }
__device__ __forceinline__ double corr_Mz(const CorrCubic& C, double z) { return C.M - z * (2.0 * C.T - 3.0 * z); }

// FP64 path (near-degenerate or indefinite G, or no FP32 convergence).
// tot > 0: F is decreasing and convex left of the smallest eigenvalue of G
// and has its unique root there; monotone Newton from the Gershgorin bound
// minus tot^(1/3), where F >= 0.  tot <= 0: Eq. (realroots) taken
// literally, the smallest real root of the cubic, bracketed between the
// Gershgorin bounds and the stationary points of det(G - zI) and found by
// bisection (smallest_root_nonpositive), counted in *nonconvex.
__device__ __noinline__ float corr_root_slow(S3f B, S3f K, float r, bool* nonconvex)
{
    const CorrCubic C = corr_cubic(B, K, r);
    if (C.tot > 0.0) {
        const double g0 = C.g[0] - fabs(C.g[3]) - fabs(C.g[4]);
        const double g1 = C.g[1] - fabs(C.g[3]) - fabs(C.g[5]);
        const double g2 = C.g[2] - fabs(C.g[4]) - fabs(C.g[5]);
        double z = fmin(g0, fmin(g1, g2)) - cbrt(C.tot);
        for (int it = 0; it < 200; ++it) {
            const double F = corr_F(C, z);
            const double m = corr_Mz(C, z);
            if (!(F > 0.0) || !(m > 0.0)) break;
            const double zn = z + F / m;
            if (!(zn > z)) break;
            z = zn;
        }
        return (float)z;
    }
    *nonconvex = true;
    const double glo = fmin(C.g[0] - fabs(C.g[3]) - fabs(C.g[4]),
                            fmin(C.g[1] - fabs(C.g[3]) - fabs(C.g[5]), C.g[2] - fabs(C.g[4]) - fabs(C.g[5])));
    const double ghi = fmax(C.g[0] + fabs(C.g[3]) + fabs(C.g[4]),
                            fmax(C.g[1] + fabs(C.g[3]) + fabs(C.g[5]), C.g[2] + fabs(C.g[4]) + fabs(C.g[5])));
    double scale = 0.0;
    for (int q = 0; q < 6; ++q) scale += fabs(C.g[q]);
    return (float)smallest_root_nonpositive([&](double z) { return corr_F(C, z); }, C.T, C.M, glo, ghi, C.tot, scale);
}

__device__ __forceinline__ float corr_root(const S3f& B, const S3f& K, float r, bool* nonconvex)
{
    float z;
    if (corr_root_fast(B, K, r, &z)) return z;
    return corr_root_slow(B, K, r, nonconvex);
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

// Points of colours 0..c-1.  With a, b the interior counts of even and odd
// indices along an axis and S(p) = p ? b : a, colour q = (pi, pj, pk) holds
// S(pi) S(pj) S(pk) points, and the colours before c = (pi, pj, pk) are those
// with a smaller pk, then those with pk and a smaller pj, then (0, pj, pk)
// when pi = 1:
//     offset = pk (a + b)^2 a + pj (a + b) a S(pk) + pi a S(pj) S(pk),
// the same integer as the sum over the boxes, without a loop.
__host__ __device__ __forceinline__ long long cm_offset(int n, int c)
{
    const long long a = colour_count(n, 0), b = colour_count(n, 1);
    const long long sj = (c & 2) ? b : a, sk = (c & 4) ? b : a;
    return ((c & 4) ? (a + b) * (a + b) * a : 0) + ((c & 2) ? (a + b) * a * sk : 0) + ((c & 1) ? a * sj * sk : 0);
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
__device__ __forceinline__ void base_colour_block(const float* __restrict__ hi, const float* __restrict__ lo,
                                                  float* __restrict__ bstore, int n, float inv_h2, uint3 bid)
{
    const int i = bid.x * BX + threadIdx.x;
    const int j = bid.y * BY + threadIdx.y;
    const int k = bid.z;
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

__global__ void __launch_bounds__(BX * BY) k_base_colour(const float* __restrict__ hi, const float* __restrict__ lo,
                                                         float* __restrict__ bstore, int n, float inv_h2)
{
    base_colour_block(hi, lo, bstore, n, inv_h2, blockIdx);
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
// B and rhs boxes; e is in the natural layout (19-point stencil).  Idx is int
// for grids up to 1289^3 (32-bit index arithmetic), long long above.  The
// point solve is latency-bound, so the launch bounds ask for 12 resident
// blocks per SM (40 registers, no spills; 14 would spill).  NN > 0 fixes the
// grid size at compile time (n = NN): the 18 neighbour offsets and the box
// strides become constants, so each load is one instruction with an
// immediate offset instead of an address computed per load; the arithmetic
// of a point is the same, and so are the bits.
template <int PI, int PJ, int PK, typename Idx, int NN = 0>
__device__ __forceinline__ void smooth_corr_block(float* e, const float* __restrict__ bc, const float* __restrict__ rc,
                                                  int n_rt, float inv_h2, float h2half, unsigned long long* events,
                                                  uint3 bid)
{
    const int n = NN > 0 ? NN : n_rt;
    const int ii = bid.x * BX + threadIdx.x;
    const int jj = bid.y * BY + threadIdx.y;
    const int kk = bid.z;
    const int ni = colour_count(n, PI), nj = colour_count(n, PJ);
    if (ii >= ni || jj >= nj) return;
    const int i = (PI ? 1 : 2) + 2 * ii, j = (PJ ? 1 : 2) + 2 * jj, k = (PK ? 1 : 2) + 2 * kk;
    const Idx cnt = (Idx)ni * nj * colour_count(n, PK);
    const Idx idx = ((Idx)kk * nj + jj) * ni + ii;
    const float* bp = bc + idx;
    S3f B;
    B.xx = __ldcs(bp);
    B.yy = __ldcs(bp + cnt);
    B.zz = __ldcs(bp + 2 * cnt);
    B.xy = __ldcs(bp + 3 * cnt);
    B.xz = __ldcs(bp + 4 * cnt);
    B.yz = __ldcs(bp + 5 * cnt);
    const Idx sy = n, sz = (Idx)n * n;
    float* q = e + (((Idx)k * n + j) * n + i);
    float e0;
    S3f K;
    if constexpr (NN > 0) {
        // e is 8-byte aligned and n is odd, so element (i, j, k) is 8-byte
        // aligned exactly when i + j + k is even, a constant of the colour.
        // In the point's own row and in the four rows at one face step the
        // aligned pair holds two of the three values the stencil needs (i-1,
        // i or i, i+1), so those rows take one 8-byte and one 4-byte load:
        // 14 loads for the 19 values, the same bytes, fewer L1 requests.
        constexpr int P = (PI + PJ + PK) & 1;
        float v[3][3][3];   // [dk + 1][dj + 1][di + 1]
        auto pair_row = [&](int dj, int dk, int par) {
            const float* r = q + (dj * sy + dk * sz);
            if (par == 0) {   // (i, i + 1) aligned
                const float2 a = __ldg(reinterpret_cast<const float2*>(r));
                v[dk + 1][dj + 1][1] = a.x;
                v[dk + 1][dj + 1][2] = a.y;
                v[dk + 1][dj + 1][0] = __ldg(r - 1);
            } else {          // (i - 1, i) aligned
                const float2 a = __ldg(reinterpret_cast<const float2*>(r - 1));
                v[dk + 1][dj + 1][0] = a.x;
                v[dk + 1][dj + 1][1] = a.y;
                v[dk + 1][dj + 1][2] = __ldg(r + 1);
            }
        };
        pair_row(0, 0, P);
        pair_row(1, 0, P ^ 1);
        pair_row(-1, 0, P ^ 1);
        pair_row(0, 1, P ^ 1);
        pair_row(0, -1, P ^ 1);
        v[2][2][1] = __ldg(q + (sy + sz));
        v[0][0][1] = __ldg(q - (sy + sz));
        v[0][2][1] = __ldg(q + (sy - sz));
        v[2][0][1] = __ldg(q + (sz - sy));
        e0 = v[1][1][1];
        K = hess_from_diff([&](int di, int dj, int dk) -> float { return v[dk + 1][dj + 1][di + 1] - e0; }, inv_h2);
    } else {
        e0 = q[0];
        K = hess_from_diff([&](int di, int dj, int dk) -> float { return __ldg(q + (di + dj * sy + dk * sz)) - e0; },
                           inv_h2);
    }
    bool nonconvex = false;
    const float z = corr_root(B, K, __ldcs(rc + idx), &nonconvex);
    q[0] = fmaf(h2half, z, e0);
    if (nonconvex && events) atomicAdd(events, 1ull);
}

template <int PI, int PJ, int PK, typename Idx>
__global__ void __launch_bounds__(BX * BY, 12) k_smooth_corr(float* e, const float* __restrict__ bc,
                                                              const float* __restrict__ rc, int n, float inv_h2,
                                                              float h2half, unsigned long long* events)
{
    smooth_corr_block<PI, PJ, PK, Idx>(e, bc, rc, n, inv_h2, h2half, events, blockIdx);
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
    if (n <= 1289)
        k_smooth_corr<PI, PJ, PK, int><<<grid, dim3(BX, BY), 0, s>>>(e, bstore + 6 * off, rhs_cm + off, n, inv_h2,
                                                                      h2half, ev);
    else
        k_smooth_corr<PI, PJ, PK, long long><<<grid, dim3(BX, BY), 0, s>>>(e, bstore + 6 * off, rhs_cm + off, n,
                                                                            inv_h2, h2half, ev);
    return cudaGetLastError();
}

// Colours C and C^7 in one launch.  The 19-point stencil of a colour-C
// point holds every colour but C^7 (the corners are not in it), so the
// updates of the two colours are independent, and one launch performs the
// sequential sweep of colour C followed by colour C^7.  Blocks with z below
// nk0 sweep colour C, the rest colour C^7; x and y cover the larger of the
// two colour boxes.
template <int C, typename Idx, int NN = 0>
__global__ void __launch_bounds__(BX * BY, 12) k_smooth_corr_pair(float* e, const float* __restrict__ b0,
                                                                   const float* __restrict__ r0,
                                                                   const float* __restrict__ b1,
                                                                   const float* __restrict__ r1, int n, float inv_h2,
                                                                   float h2half, unsigned long long* events, int nk0)
{
    constexpr int D = C ^ 7;
    uint3 bid = blockIdx;
    if ((int)bid.z < nk0) {
        smooth_corr_block<C & 1, (C >> 1) & 1, (C >> 2) & 1, Idx, NN>(e, b0, r0, n, inv_h2, h2half, events, bid);
    } else {
        bid.z -= nk0;
        smooth_corr_block<D & 1, (D >> 1) & 1, (D >> 2) & 1, Idx, NN>(e, b1, r1, n, inv_h2, h2half, events, bid);
    }
}

// The pair launch with the grid size fixed at compile time for the sizes
// where the sweep streams from HBM (see smooth_corr_block).
template <int C, int NN>
void launch_pair_fixed(dim3 grid, cudaStream_t s, float* e, const float* b0, const float* r0, const float* b1,
                       const float* r1, float inv_h2, float h2half, unsigned long long* ev, int nk0)
{
    k_smooth_corr_pair<C, int, NN><<<grid, dim3(BX, BY), 0, s>>>(e, b0, r0, b1, r1, NN, inv_h2, h2half, ev, nk0);
}

template <int C>
cudaError_t launch_colour_corr_pair(float* e, const float* bstore, const float* rhs_cm, int n, float inv_h2,
                                    float h2half, unsigned long long* ev, cudaStream_t s)
{
    constexpr int D = C ^ 7;
    const int nk0 = colour_count(n, (C >> 2) & 1), nk1 = colour_count(n, (D >> 2) & 1);
    const int ni = colour_count(n, 1), nj = colour_count(n, 1);   // the larger box edge
    if (ni <= 0 || nk0 + nk1 <= 0) return cudaSuccess;
    if (colour_count(n, 0) <= 0)   // n = 3: colour 7 alone
        return C == 0 ? launch_colour_corr<7>(e, bstore, rhs_cm, n, inv_h2, h2half, ev, s) : cudaSuccess;
    dim3 grid((ni + BX - 1) / BX, (nj + BY - 1) / BY, nk0 + nk1);
    const long long o0 = cm_offset(n, C), o1 = cm_offset(n, D);
    count_launches(1);
    const float *b0 = bstore + 6 * o0, *r0 = rhs_cm + o0, *b1 = bstore + 6 * o1, *r1 = rhs_cm + o1;
    if (((uintptr_t)e & 7) == 0) switch (n) {   // the fixed-size kernels read 8-byte pairs of e
    case 129: launch_pair_fixed<C, 129>(grid, s, e, b0, r0, b1, r1, inv_h2, h2half, ev, nk0); return cudaGetLastError();
    case 257: launch_pair_fixed<C, 257>(grid, s, e, b0, r0, b1, r1, inv_h2, h2half, ev, nk0); return cudaGetLastError();
    case 513: launch_pair_fixed<C, 513>(grid, s, e, b0, r0, b1, r1, inv_h2, h2half, ev, nk0); return cudaGetLastError();
    case 1025: launch_pair_fixed<C, 1025>(grid, s, e, b0, r0, b1, r1, inv_h2, h2half, ev, nk0); return cudaGetLastError();
    default: break;
    }
    if (n <= 1289)
        k_smooth_corr_pair<C, int><<<grid, dim3(BX, BY), 0, s>>>(e, bstore + 6 * o0, rhs_cm + o0, bstore + 6 * o1,
                                                                  rhs_cm + o1, n, inv_h2, h2half, ev, nk0);
    else
        k_smooth_corr_pair<C, long long><<<grid, dim3(BX, BY), 0, s>>>(e, bstore + 6 * o0, rhs_cm + o0,
                                                                        bstore + 6 * o1, rhs_cm + o1, n, inv_h2,
                                                                        h2half, ev, nk0);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Plane-phase correction sweep.  Colours 0-3 lie on even planes k and colours
// 4-7 on odd planes, and every neighbour of a point in planes k +- 1 has the
// other k parity.  So during colours 0-3 of a sweep the even planes see only
// old values of the odd planes and do not interact with each other; during
// colours 4-7 the odd planes see only the (now final) even planes.  One sweep
// is therefore two launches, one per k parity, each running the four in-plane
// colour phases (i, j parities (0,0), (1,0), (0,1), (1,1)) of one PT x PT tile
// of one plane per block, with __syncthreads between the phases.  In-plane
// colour q needs the new values of colours < q at in-plane distance 1, so a
// block also updates colour q on a halo of 3 - q points around its tile; it
// does so from the same inputs and with the same arithmetic as the block that
// owns those points, so the values agree bit for bit and the result is the
// sequential 8-colour sweep.  Blocks read the old plane from `own` and write
// their tile to `dst`, a second buffer, so that no block reads a neighbour's
// new values in place of the old ones.  Phase k-even: own = nbr = src;
// phase k-odd: own = src, nbr = dst (the new even planes).
// ---------------------------------------------------------------------------
// Tiles: PT x PT points (PT even), an e halo of PH = 4 in shared memory.  A
// shared-memory row of PW = PT + 8 values keeps the even and the odd x = i - x0
// in two halves, so the 32 lanes of a warp, which update points two apart in
// i, read 32 consecutive words (no bank conflicts).
constexpr int PH = 4;

template <int PT>
struct Tile {
    static constexpr int PW = PT + 2 * PH;
    static constexpr int PWH = PW / 2;
    static constexpr int SMEM = 3 * PW * PW * (int)sizeof(float);
};

// Blocks per SM the launch bounds ask for: shared memory limits the 64-point
// tile to 3; the smaller tiles allow 80 registers per thread.
__host__ __device__ constexpr int plane_min_blocks(int pt, int nt) { return pt >= 64 ? 3 : 65536 / (80 * nt); }

// 4-byte asynchronous global -> shared copy (cp.async); src_bytes 0 writes a
// zero and reads nothing.
__device__ __forceinline__ void cp_async_f32(float* dst_smem, const float* src, int src_bytes)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Loads planes k-1, k, k+1 of e over the tile and its halo into sp
// ([3][PW][PW], parity-split rows) with asynchronous copies, one warp per
// row.  Points outside the grid read as 0 and are never used.  Ends with the
// copies complete and visible to the block.
template <int PT, int NT>
__device__ __forceinline__ void load_plane_tile(float* sp, const float* own, const float* nbr, int n, int k, int x0,
                                                int y0)
{
    constexpr int PW = Tile<PT>::PW, PWH = Tile<PT>::PWH, NCH = (PW + 31) / 32;
    const int lane = threadIdx.x & 31;
    bool xok[NCH];
    int xs[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        const int x = lane + 32 * c;
        xok[c] = x < PW && x0 + x >= 0 && x0 + x < n;
        xs[c] = (x & 1) * PWH + (x >> 1);
    }
    for (int r = threadIdx.x >> 5; r < 3 * PW; r += NT / 32) {
        const int pl = r / PW, y = r - pl * PW;
        const int gj = y0 + y;
        const bool row_ok = gj >= 0 && gj < n;
        const float* base = pl == 1 ? own : nbr;
        const long long row = ((long long)(k - 1 + pl) * n + (row_ok ? gj : 0)) * n;
        float* drow = sp + r * PW;
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            const int x = lane + 32 * c;
            if (x < PW) {
                const bool ok = row_ok && xok[c];
                cp_async_f32(drow + xs[c], ok ? base + row + (x0 + x) : base, ok ? 4 : 0);
            }
        }
    }
    cp_async_wait_all();
    __syncthreads();
}

// Points of in-plane colour Q (i parity Q & 1, j parity Q >> 1) of plane k
// with i in [ia - hq, ia + PT - 1 + hq] and j likewise, inside the interior:
// (a, b) -> i = ilo + 2a, j = jlo + 2b.
struct ColourRegion {
    int ilo, jlo, ci, cj;
};

__device__ __forceinline__ ColourRegion colour_region(int n, int ia, int ja, int pt, int hq, int pi, int pj)
{
    ColourRegion R;
    R.ilo = max(1, ia - hq);
    R.jlo = max(1, ja - hq);
    const int ihi = min(n - 2, ia + pt - 1 + hq), jhi = min(n - 2, ja + pt - 1 + hq);
    R.ilo += (R.ilo & 1) != pi;
    R.jlo += (R.jlo & 1) != pj;
    R.ci = ihi >= R.ilo ? (ihi - R.ilo) / 2 + 1 : 0;
    R.cj = jhi >= R.jlo ? (jhi - R.jlo) / 2 + 1 : 0;
    return R;
}

// One in-plane colour phase over a region of plane k (in shared memory), the
// points spread over the block's NT threads.  SMOOTH: update each point by
// the smallest-root rule; else write res = rhs - N(e) to global memory.
// Returns the rhs <= 0 root events of this thread.
template <int Q, int PT, int NT, bool SMOOTH>
__device__ __forceinline__ unsigned colour_phase(float* sp, const float* __restrict__ bstore,
                                                 const float* __restrict__ rhs_cm, float* __restrict__ res, int n,
                                                 int pk, int kk, int k, int ia, int ja, int x0, int y0, int hq,
                                                 float inv_h2, float h2half)
{
    constexpr int PW = Tile<PT>::PW, PWH = Tile<PT>::PWH;
    constexpr int pi = Q & 1, pj = Q >> 1;
    constexpr int XP = pi ^ 1;                       // parity of x = i - x0 (x0 = ia - 4 is odd)
    static_assert(((PT + 6) / 2 + 1) * ((PT + 6) / 2 + 1) <= 32 * NT, "a thread's points of a colour must fit 32 bits");
    constexpr int DXP = XP ? 1 - PWH : PWH;          // shared-memory offset of i + 1
    constexpr int DXM = XP ? -PWH : PWH - 1;         // of i - 1
    const ColourRegion R = colour_region(n, ia, ja, PT, hq, pi, pj);
    const int total = R.ci * R.cj;
    if (total == 0) return 0;
    const int ni = colour_count(n, pi), nj = colour_count(n, pj);
    const long long cnt = (long long)ni * nj * colour_count(n, pk);
    const long long off = cm_offset(n, Q | (pk << 2));
    const long long base = ((long long)kk * nj + ((R.jlo - (pj ? 1 : 2)) >> 1)) * ni + ((R.ilo - (pi ? 1 : 2)) >> 1);
    const float* bq = bstore + 6 * off + base;
    const float* rq = rhs_cm + off + base;
    const int s0 = (PW + (R.jlo - y0)) * PW + XP * PWH + ((R.ilo - x0) >> 1);
    int a = threadIdx.x % R.ci, b = threadIdx.x / R.ci;
    const int da = NT % R.ci, db = NT / R.ci;
    unsigned slow = 0;   // SMOOTH: iterations whose point needs the FP64 root (at most 32 per thread)
    int it = 0;
    for (int t = threadIdx.x; t < total; t += NT, ++it) {
        const int rel = b * ni + a;
        const S3f B = load_b(bq + rel, cnt);
        const float rr = __ldcs(rq + rel);
        const int sc = s0 + 2 * b * PW + a;
        const float e0 = sp[sc];
        const S3f K = hess_from_diff(
            [&](int di, int dj, int dk) -> float {
                return sp[sc + dk * PW * PW + dj * PW + (di > 0 ? DXP : (di < 0 ? DXM : 0))] - e0;
            },
            inv_h2);
        if (SMOOTH) {
            float z;
            if (corr_root_fast(B, K, rr, &z)) sp[sc] = fmaf(h2half, z, e0);
            else slow |= 1u << it;
        } else {
            res[((long long)k * n + (R.jlo + 2 * b)) * n + (R.ilo + 2 * a)] = rr - delta_det(B, K);
        }
        a += da;
        b += db;
        if (a >= R.ci) {
            a -= R.ci;
            ++b;
        }
    }
    // points of this colour are independent, so the rare FP64 roots can
    // follow the others (their neighbours have other colours)
    unsigned ev = 0;
    while (SMOOTH && slow) {
        const int q = __ffs(slow) - 1;
        slow &= slow - 1;
        const int t = threadIdx.x + q * NT;
        const int a2 = t % R.ci, b2 = t / R.ci;
        const int rel = b2 * ni + a2;
        const S3f B = load_b(bq + rel, cnt);
        const int sc = s0 + 2 * b2 * PW + a2;
        const float e0 = sp[sc];
        const S3f K = hess_from_diff(
            [&](int di, int dj, int dk) -> float {
                return sp[sc + dk * PW * PW + dj * PW + (di > 0 ? DXP : (di < 0 ? DXM : 0))] - e0;
            },
            inv_h2);
        bool nonconvex = false;
        const float z = corr_root_slow(B, K, __ldcs(rq + rel), &nonconvex);
        sp[sc] = fmaf(h2half, z, e0);
        // count each point once: halo points are the neighbouring block's
        const int i2 = R.ilo + 2 * a2, j2 = R.jlo + 2 * b2;
        const bool owned = i2 >= ia && i2 < ia + PT && j2 >= ja && j2 < ja + PT;
        ev += (nonconvex && owned) ? 1u : 0u;
    }
    return ev;
}

template <int PK, int PT, int NT>
__device__ __forceinline__ void smooth_corr_plane_block(const float* __restrict__ own, const float* __restrict__ nbr,
                                                        float* __restrict__ dst, const float* __restrict__ bstore,
                                                        const float* __restrict__ rhs_cm, int n, float inv_h2,
                                                        float h2half, unsigned long long* events, uint3 bid)
{
    extern __shared__ float sp[];
    constexpr int PW = Tile<PT>::PW, PWH = Tile<PT>::PWH;
    const int ia = 1 + PT * (int)bid.x, ja = 1 + PT * (int)bid.y;
    const int kk = bid.z;
    const int k = (PK ? 1 : 2) + 2 * kk;
    const int x0 = ia - PH, y0 = ja - PH;
    load_plane_tile<PT, NT>(sp, own, nbr, n, k, x0, y0);
    unsigned ev = colour_phase<0, PT, NT, true>(sp, bstore, rhs_cm, nullptr, n, PK, kk, k, ia, ja, x0, y0, 3, inv_h2,
                                                h2half);
    __syncthreads();
    ev += colour_phase<1, PT, NT, true>(sp, bstore, rhs_cm, nullptr, n, PK, kk, k, ia, ja, x0, y0, 2, inv_h2,
                                        h2half);
    __syncthreads();
    ev += colour_phase<2, PT, NT, true>(sp, bstore, rhs_cm, nullptr, n, PK, kk, k, ia, ja, x0, y0, 1, inv_h2,
                                        h2half);
    __syncthreads();
    ev += colour_phase<3, PT, NT, true>(sp, bstore, rhs_cm, nullptr, n, PK, kk, k, ia, ja, x0, y0, 0, inv_h2,
                                        h2half);
    __syncthreads();
    const int ihi = min(n - 2, ia + PT - 1), jhi = min(n - 2, ja + PT - 1);
    for (int r = threadIdx.x >> 5; r <= jhi - ja; r += NT / 32) {
        const int j = ja + r;
        float* d = dst + ((long long)k * n + j) * n;
        const float* srow = sp + (PW + (j - y0)) * PW;
        for (int i = ia + (threadIdx.x & 31); i <= ihi; i += 32) {
            const int x = i - x0;
            d[i] = srow[(x & 1) * PWH + (x >> 1)];
        }
    }
    if (events && ev) atomicAdd(events, (unsigned long long)ev);
}

template <int PK, int PT, int NT>
__global__ void __launch_bounds__(NT, plane_min_blocks(PT, NT))
    k_smooth_corr_plane(const float* __restrict__ own, const float* __restrict__ nbr, float* __restrict__ dst,
                        const float* __restrict__ bstore, const float* __restrict__ rhs_cm, int n, float inv_h2,
                        float h2half, unsigned long long* events)
{
    smooth_corr_plane_block<PK, PT, NT>(own, nbr, dst, bstore, rhs_cm, n, inv_h2, h2half, events, blockIdx);
}

// res = rhs - N(e) over one PT x PT tile of one interior plane: e staged in
// shared memory, B and rhs read per in-plane colour (contiguous in the
// colour-major store).
template <int PT, int NT>
__device__ __forceinline__ void residual_corr_plane_block(const float* __restrict__ e, const float* __restrict__ bstore,
                                                          const float* __restrict__ rhs_cm, float* __restrict__ res,
                                                          int n, float inv_h2, uint3 bid)
{
    extern __shared__ float sp[];
    const int ia = 1 + PT * (int)bid.x, ja = 1 + PT * (int)bid.y;
    const int k = 1 + (int)bid.z;
    const int pk = k & 1;
    const int kk = (k - (pk ? 1 : 2)) >> 1;
    const int x0 = ia - PH, y0 = ja - PH;
    load_plane_tile<PT, NT>(sp, e, e, n, k, x0, y0);
    colour_phase<0, PT, NT, false>(sp, bstore, rhs_cm, res, n, pk, kk, k, ia, ja, x0, y0, 0, inv_h2, 0.0f);
    colour_phase<1, PT, NT, false>(sp, bstore, rhs_cm, res, n, pk, kk, k, ia, ja, x0, y0, 0, inv_h2, 0.0f);
    colour_phase<2, PT, NT, false>(sp, bstore, rhs_cm, res, n, pk, kk, k, ia, ja, x0, y0, 0, inv_h2, 0.0f);
    colour_phase<3, PT, NT, false>(sp, bstore, rhs_cm, res, n, pk, kk, k, ia, ja, x0, y0, 0, inv_h2, 0.0f);
}

template <int PT, int NT>
__global__ void __launch_bounds__(NT, plane_min_blocks(PT, NT))
    k_residual_corr_plane(const float* __restrict__ e, const float* __restrict__ bstore,
                          const float* __restrict__ rhs_cm, float* __restrict__ res, int n, float inv_h2)
{
    residual_corr_plane_block<PT, NT>(e, bstore, rhs_cm, res, n, inv_h2, blockIdx);
}

// res = rhs - N(e) by columns.  A warp covers CW = 30 interior points of a
// row (i = i0 .. i0 + 29) with a halo lane on either side and walks a run of
// planes in k, holding the centre, north (j + 1) and south (j - 1) values of
// planes k - 1, k, k + 1 in registers; the x-neighbours come from the
// adjacent lanes by shuffles.  Per point that is three loads and six
// shuffles instead of staging a halo tile, and the colour-major B and rhs of
// a column alternate between two colour boxes, addressed incrementally.
// Every difference to the centre is formed from the same two floats as in
// the tile kernels, so the values are the same bits.  Grid: col_grid(n, kc),
// blocks of 32 x 4 (four rows).
constexpr int CW = 30;

// CRHS = false: the correction residual res = rhs - N(e), rhs colour-major,
// res natural.  CRHS = true: the tau-corrected coarse right-hand side
// out = N(w) + r with e = w, rhs_cm = r (natural layout) and res = out
// (colour-major), the same stencil values and the same delta_det(B, K) + r as
// one thread per point forms them.
template <int NN = 0, bool CRHS = false>
__device__ __forceinline__ void residual_corr_col_block(const float* __restrict__ e, const float* __restrict__ bstore,
                                                        const float* __restrict__ rhs_cm, float* __restrict__ res,
                                                        int n_rt, float inv_h2, int kc, uint3 bid)
{
    // NN > 0: the grid size at compile time (strides and box sizes become
    // constants; the same arithmetic and bits)
    const int n = NN > 0 ? NN : n_rt;
    const int lane = threadIdx.x;
    const int i = (int)bid.x * CW + lane;   // i0 - 1 + lane, i0 = 1 + CW bid.x
    const int j = 1 + (int)bid.y * 4 + (int)threadIdx.y;
    if (j > n - 2) return;                  // the whole warp (one row per warp)
    const int k0 = 1 + (int)bid.z * kc;
    const int k1 = min(n - 2, k0 + kc - 1);
    const bool inrow = i <= n - 1;
    const bool act = lane >= 1 && lane <= CW && i <= n - 2;
    const long long sy = n, sz = (long long)n * n;
    const float* q = e + ((long long)j * n + (inrow ? i : 0));
    auto ld = [&](int k, long long dj) -> float { return inrow ? __ldg(q + k * sz + dj) : 0.0f; };
    constexpr unsigned FULL = 0xffffffffu;
    // colour-major addressing of this column: the two colour boxes (k even, odd)
    const int pi = i & 1, pj = j & 1;
    const int ni = colour_count(n, pi), nj = colour_count(n, pj);
    const int ii = (i - (pi ? 1 : 2)) >> 1, jj = (j - (pj ? 1 : 2)) >> 1;
    const long long off0 = cm_offset(n, pi | (pj << 1)), off1 = cm_offset(n, pi | (pj << 1) | 4);
    const long long cnt0 = (long long)ni * nj * colour_count(n, 0), cnt1 = (long long)ni * nj * colour_count(n, 1);
    const long long plane = (long long)ni * nj, rowoff = (long long)jj * ni + ii;
    // B and rhs of point k (act lanes only): the loads are issued one point ahead
    auto load_bk = [&](int k, S3f* B, float* rr) {
        const int pk = k & 1;
        const long long w = (long long)((k - (pk ? 1 : 2)) >> 1) * plane + rowoff;
        const long long off = pk ? off1 : off0;
        *B = load_b(bstore + 6 * off + w, pk ? cnt1 : cnt0);
        *rr = CRHS ? __ldcs(rhs_cm + (((long long)k * n + j) * n + i)) : __ldcs(rhs_cm + off + w);
    };
    float Cm = ld(k0 - 1, 0), Nm = ld(k0 - 1, sy), Sm = ld(k0 - 1, -sy);
    float Cc = ld(k0, 0), Nc = ld(k0, sy), Sc = ld(k0, -sy);
    float Cp = ld(k0 + 1, 0), Np = ld(k0 + 1, sy), Sp = ld(k0 + 1, -sy);
    float Cm_e = __shfl_down_sync(FULL, Cm, 1), Cm_w = __shfl_up_sync(FULL, Cm, 1);
    float Cc_e = __shfl_down_sync(FULL, Cc, 1), Cc_w = __shfl_up_sync(FULL, Cc, 1);
    S3f Bk = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    float rk = 0.0f;
    if (act) load_bk(k0, &Bk, &rk);
    for (int k = k0; k <= k1; ++k) {
        // plane k + 2 and the B, rhs of point k + 1, in flight while point k is computed
        float Cq = 0.0f, Nq = 0.0f, Sq = 0.0f;
        S3f Bq = Bk;
        float rq = rk;
        if (k < k1) {
            Cq = ld(k + 2, 0);
            Nq = ld(k + 2, sy);
            Sq = ld(k + 2, -sy);
            if (act) load_bk(k + 1, &Bq, &rq);
        }
        const float Cp_e = __shfl_down_sync(FULL, Cp, 1), Cp_w = __shfl_up_sync(FULL, Cp, 1);
        const float Nc_e = __shfl_down_sync(FULL, Nc, 1), Nc_w = __shfl_up_sync(FULL, Nc, 1);
        const float Sc_e = __shfl_down_sync(FULL, Sc, 1), Sc_w = __shfl_up_sync(FULL, Sc, 1);
        if (act) {
            const float e0 = Cc;
            const S3f K = hess_from_diff(
                [&](int di, int dj, int dk) -> float {
                    float v;
                    if (dk == 0) {
                        if (dj == 0) v = di > 0 ? Cc_e : Cc_w;
                        else if (dj > 0) v = di > 0 ? Nc_e : (di < 0 ? Nc_w : Nc);
                        else v = di > 0 ? Sc_e : (di < 0 ? Sc_w : Sc);
                    } else if (dk > 0) {
                        if (dj == 0) v = di > 0 ? Cp_e : (di < 0 ? Cp_w : Cp);
                        else v = dj > 0 ? Np : Sp;
                    } else {
                        if (dj == 0) v = di > 0 ? Cm_e : (di < 0 ? Cm_w : Cm);
                        else v = dj > 0 ? Nm : Sm;
                    }
                    return v - e0;
                },
                inv_h2);
            if constexpr (CRHS) {
                const int pk = k & 1;
                const long long w = (long long)((k - (pk ? 1 : 2)) >> 1) * plane + rowoff;
                res[(pk ? off1 : off0) + w] = delta_det(Bk, K) + rk;
            } else {
                res[((long long)k * n + j) * n + i] = rk - delta_det(Bk, K);
            }
        }
        Cm = Cc; Nm = Nc; Sm = Sc; Cm_e = Cc_e; Cm_w = Cc_w;
        Cc = Cp; Nc = Np; Sc = Sp; Cc_e = Cp_e; Cc_w = Cp_w;
        Cp = Cq; Np = Nq; Sp = Sq;
        Bk = Bq;
        rk = rq;
    }
}

template <int NN = 0>
__global__ void __launch_bounds__(BX * BY, 8) k_residual_corr_col(const float* __restrict__ e,
                                                                  const float* __restrict__ bstore,
                                                                  const float* __restrict__ rhs_cm,
                                                                  float* __restrict__ res, int n, float inv_h2,
                                                                  int kc)
{
    residual_corr_col_block<NN>(e, bstore, rhs_cm, res, n, inv_h2, kc, blockIdx);
}

// Planes per column run, and the grid of the column residual.
// (8 planes up to 129^3, 16 from 257^3: measured, 21.1 against 24.6 us at 129^3 and
// 147.3 against 150.4 us at 257^3 under graph replay)
__host__ __device__ inline int col_chunk(int n) { return n >= 257 ? 16 : 8; }
inline dim3 col_grid(int n, int kc) { return dim3((n - 2 + CW - 1) / CW, (n - 2 + 3) / 4, (n - 2 + kc - 1) / kc); }

// The shell of res (faces of the cube) is 0.
__global__ void k_zero_shell(float* v, int n)
{
    const int a = blockIdx.x * BX + threadIdx.x, b = blockIdx.y * BY + threadIdx.y;
    if (a >= n || b >= n) return;
    const long long sz = (long long)n * n;
    const int face = blockIdx.z;   // 0,1: k = 0, n-1; 2,3: j = 0, n-1; 4,5: i = 0, n-1
    const int m = (face & 1) ? n - 1 : 0;
    long long p;
    if (face < 2) p = (long long)m * sz + (long long)b * n + a;
    else if (face < 4) p = (long long)b * sz + (long long)m * n + a;
    else p = (long long)b * sz + (long long)a * n + m;
    v[p] = 0.0f;
}

// rhs_H = N_H(w_H) + res_H on the coarse interior, written colour-major.
// The tau-corrected coarse right-hand side of the correction problem,
// rhs_H = N_H(w_H) + I r_h (Algorithm 1 step 4; N(w) = det(B + D^2_h w) -
// det(B)), colour-major.  From 129^3 up by columns as the correction residual
// walks them (k_coarse_rhs_corr_col: 3 loads of w a point); below, where the
// level is latency-bound and a column of 8 points a thread would cut the
// parallelism 8-fold, one point a thread (k_coarse_rhs_corr).  The same
// values either way.
constexpr int kCoarseRhsColMin = 129;

template <int NN = 0>
__global__ void __launch_bounds__(BX * BY, 8) k_coarse_rhs_corr_col(const float* __restrict__ w,
                                                                    const float* __restrict__ bstore,
                                                                    const float* __restrict__ resc,
                                                                    float* __restrict__ rhs_cm, int n, float inv_h2,
                                                                    int kc)
{
    residual_corr_col_block<NN, true>(w, bstore, resc, rhs_cm, n, inv_h2, kc, blockIdx);
}

__device__ __forceinline__ void coarse_rhs_corr_block(const float* __restrict__ w, const float* __restrict__ bstore,
                                                      const float* __restrict__ resc, float* __restrict__ rhs_cm,
                                                      int n, float inv_h2, uint3 bid)
{
    const int i = bid.x * BX + threadIdx.x;
    const int j = bid.y * BY + threadIdx.y;
    const int k = bid.z;
    if (i < 1 || j < 1 || k < 1 || i > n - 2 || j > n - 2 || k > n - 2) return;
    const long long p = lin(i, j, k, n);
    const long long sy = n, sz = (long long)n * n;
    const CmPos c = cm_pos(i, j, k, n);
    const S3f B = load_b(bstore + 6 * c.off + c.idx, c.cnt);
    const float e0 = w[p];
    const S3f K = hess_from_diff(
        [&](int di, int dj, int dk) -> float { return __ldg(w + p + di + dj * sy + dk * sz) - e0; }, inv_h2);
    rhs_cm[c.off + c.idx] = delta_det(B, K) + resc[p];
}

__global__ void __launch_bounds__(BX * BY) k_coarse_rhs_corr(const float* __restrict__ w,
                                                             const float* __restrict__ bstore,
                                                             const float* __restrict__ resc,
                                                             float* __restrict__ rhs_cm, int n, float inv_h2)
{
    coarse_rhs_corr_block(w, bstore, resc, rhs_cm, n, inv_h2, blockIdx);
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
__device__ __forceinline__ void coarsest_corr_body(float* e, const float* __restrict__ bstore,
                                                   const float* __restrict__ rhs_cm, int n, float inv_h2, float h2half,
                                                   int sweeps, unsigned long long* events)
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

__global__ void __launch_bounds__(CT) k_coarsest_corr(float* e, const float* __restrict__ bstore,
                                                      const float* __restrict__ rhs_cm, int n, float inv_h2,
                                                      float h2half, int sweeps, unsigned long long* events)
{
    coarsest_corr_body(e, bstore, rhs_cm, n, inv_h2, h2half, sweeps, events);
}

// ---------------------------------------------------------------------------
// The tail of a correction V-cycle in one block: every level with n <= 17
// (or a smaller bound set by set_corr_tail), from the level the cycle enters
// there down to the coarsest grid and back,
// with e, w, the residual, B and rhs of those levels in shared memory.  Each
// step does the per-point arithmetic of its separate kernel -- the sweeps of
// k_smooth_corr, the residual of the plane and column kernels, the restriction of
// xfer::k_restrict, the right-hand side of k_coarse_rhs_corr, the coarsest
// solve of k_coarsest_corr, the prolongation of xfer::k_prolong -- so the
// result is the same bits; it replaces the ~25-40 launches of these latency-
// bound levels by one.
// ---------------------------------------------------------------------------
constexpr int kTailMaxN = 17;
constexpr int TT = 1024;

struct TailLevel {
    int n;
    int pairs;           // sweep order: colour pairs (c, c^7) in the order 0, 7, 1, 6, 2, 5, 3, 4, else ascending
    float inv_h2, h2half;
    float* e;            // global iterate (read on the top level, written back there)
    const float* b;      // global colour-major B store
    const float* rhs;    // global colour-major rhs (read on the top level)
};

struct TailArgs {
    int nlev;
    TailLevel lev[4];
    int nu1, nu2, kind, approx, coarse_sweeps;
    unsigned long long* events;
};

__host__ __device__ inline int tail_level_floats(int n, bool top)
{
    const int m = n * n * n, mi = (n - 2) * (n - 2) * (n - 2);
    return m /* e */ + (top ? 0 : m) /* w */ + m /* res */ + 6 * mi /* B */ + mi /* rhs */;
}

struct TailSmem {
    float *e, *w, *r, *b, *rhs;
};

// nsw sweeps of one tail level in shared memory, in the order the level's
// own sweep uses (its corr_smooth_choice, recorded in TailLevel::pairs), so
// that the tail and the level-by-level cycle give the same bits under any
// tuning.  Pairs: colours c and c^7 in one phase (independent: the stencil
// of a colour-c point holds every colour but c^7), phases (0, 7), (1, 6),
// (2, 5), (3, 4), the colour-pair kernel's sweep; otherwise one colour a
// phase in ascending order.  Each point runs the separate kernels'
// arithmetic; a colour with no points takes no barrier.
__device__ __forceinline__ void tail_smooth(const TailSmem& S, int n, float inv_h2, float h2half, int nsw, bool pairs,
                                            unsigned long long* ev)
{
    int cnts[8], offs[8];
    {
        int off = 0;
        for (int c = 0; c < 8; ++c) {
            const int ni = colour_count(n, c & 1), nj = colour_count(n, (c >> 1) & 1),
                      nk = colour_count(n, (c >> 2) & 1);
            cnts[c] = (ni > 0 && nj > 0 && nk > 0) ? ni * nj * nk : 0;
            offs[c] = off;
            off += cnts[c];
        }
    }
    auto point = [&](int c, int t) {
        const int pi = c & 1, pj = (c >> 1) & 1, pk = (c >> 2) & 1;
        const int ni = colour_count(n, pi), nj = colour_count(n, pj);
        const int cnt = cnts[c], off = offs[c];
        const int i = (pi ? 1 : 2) + 2 * (t % ni);
        const int j = (pj ? 1 : 2) + 2 * ((t / ni) % nj);
        const int k = (pk ? 1 : 2) + 2 * (t / (ni * nj));
        const int p = (k * n + j) * n + i;
        const float* bp = S.b + 6 * off + t;
        S3f B;
        B.xx = bp[0]; B.yy = bp[cnt]; B.zz = bp[2 * cnt]; B.xy = bp[3 * cnt]; B.xz = bp[4 * cnt];
        B.yz = bp[5 * cnt];
        const float e0 = S.e[p];
        const S3f K = corr_hess_sm(S.e, p, n, n * n, e0, inv_h2);
        bool nonconvex = false;
        const float z = corr_root(B, K, S.rhs[off + t], &nonconvex);
        S.e[p] = fmaf(h2half, z, e0);
        *ev += nonconvex ? 1ull : 0ull;
    };
    for (int sw = 0; sw < nsw; ++sw) {
        if (pairs) {
            for (int c = 0; c < 4; ++c) {
                const int d = c ^ 7, nc_ = cnts[c], tot = cnts[c] + cnts[d];
                if (tot == 0) continue;
                for (int t = threadIdx.x; t < tot; t += TT) {
                    if (t < nc_) point(c, t);
                    else point(d, t - nc_);
                }
                __syncthreads();
            }
        } else {
            for (int c = 0; c < 8; ++c) {
                if (cnts[c] == 0) continue;
                for (int t = threadIdx.x; t < cnts[c]; t += TT) point(c, t);
                __syncthreads();
            }
        }
    }
}

// B and rhs of interior point (i, j, k) in the colour-major shared copies.
__device__ __forceinline__ int tail_cm(int i, int j, int k, int n, int* cnt)
{
    const CmPos c = cm_pos(i, j, k, n);
    *cnt = (int)c.cnt;
    return (int)(c.off + c.idx);
}

__device__ __forceinline__ S3f tail_b(const float* b, int i, int j, int k, int n)
{
    const CmPos c = cm_pos(i, j, k, n);
    const float* bp = b + 6 * c.off + c.idx;
    const int cnt = (int)c.cnt;
    S3f B;
    B.xx = bp[0]; B.yy = bp[cnt]; B.zz = bp[2 * cnt]; B.xy = bp[3 * cnt]; B.xz = bp[4 * cnt]; B.yz = bp[5 * cnt];
    return B;
}

__device__ __forceinline__ float tail_line(const float* uc, const float* wc, int nc, int Ic, int J0, int K0, int oj,
                                           int ok, float w)
{
    float s = 0.0f;
    for (int dk = 0; dk <= ok; ++dk)
        for (int dj = 0; dj <= oj; ++dj) {
            const int q = ((K0 + dk) * nc + (J0 + dj)) * nc + Ic;
            s += uc[q] - wc[q];
        }
    return s * w;
}

__device__ __forceinline__ void corr_tail_body(const TailArgs& A)
{
    extern __shared__ float tsm[];
    TailSmem S[4];
    {
        float* q = tsm;
        for (int l = 0; l < A.nlev; ++l) {
            const int n = A.lev[l].n, m = n * n * n, mi = (n - 2) * (n - 2) * (n - 2);
            S[l].e = q; q += m;
            S[l].w = l > 0 ? q : nullptr; q += l > 0 ? m : 0;
            S[l].r = q; q += m;
            S[l].b = q; q += 6 * mi;
            S[l].rhs = q; q += mi;
        }
    }
    // inputs: the top level's iterate and rhs, every level's B; residual
    // shells 0 (restrictions only read the interior, as in the separate path)
    for (int l = 0; l < A.nlev; ++l) {
        const int n = A.lev[l].n, m = n * n * n, mi = (n - 2) * (n - 2) * (n - 2);
        for (int q = threadIdx.x; q < 6 * mi; q += TT) S[l].b[q] = A.lev[l].b[q];
        for (int q = threadIdx.x; q < m; q += TT) S[l].r[q] = 0.0f;
        if (l == 0) {
            for (int q = threadIdx.x; q < m; q += TT) S[0].e[q] = A.lev[0].e[q];
            for (int q = threadIdx.x; q < mi; q += TT) S[0].rhs[q] = A.lev[0].rhs[q];
        }
    }
    __syncthreads();
    unsigned long long ev = 0;
    const int L = A.nlev;
    for (int l = 0; l < L - 1; ++l) {
        const TailSmem& F = S[l];
        const TailSmem& C = S[l + 1];
        const int nf = A.lev[l].n, nc = A.lev[l + 1].n;
        tail_smooth(F, nf, A.lev[l].inv_h2, A.lev[l].h2half, A.nu1, A.lev[l].pairs != 0, &ev);
        // residual on the fine interior
        for (int q = threadIdx.x; q < (nf - 2) * (nf - 2) * (nf - 2); q += TT) {
            const int i = 1 + q % (nf - 2), j = 1 + (q / (nf - 2)) % (nf - 2), k = 1 + q / ((nf - 2) * (nf - 2));
            const int p = (k * nf + j) * nf + i;
            int cnt;
            const int cm = tail_cm(i, j, k, nf, &cnt);
            const S3f B = tail_b(F.b, i, j, k, nf);
            const S3f K = corr_hess_sm(F.e, p, nf, nf * nf, F.e[p], A.lev[l].inv_h2);
            F.r[p] = F.rhs[cm] - delta_det(B, K);
        }
        __syncthreads();
        // restriction: coarse residual, approximation restriction of e
        for (int pc = threadIdx.x; pc < nc * nc * nc; pc += TT) {
            const int I = pc % nc, J = (pc / nc) % nc, K = pc / (nc * nc);
            const int pf = ((2 * K) * nf + 2 * J) * nf + 2 * I;
            const bool inside = I > 0 && J > 0 && K > 0 && I < nc - 1 && J < nc - 1 && K < nc - 1;
            C.r[pc] = inside ? xfer::weighted_restrict(F.r, pf, nf, (long long)nf * nf, A.kind) : 0.0f;
            const float w = (inside && A.approx == 1) ? xfer::weighted_restrict(F.e, pf, nf, (long long)nf * nf, A.kind)
                                                     : F.e[pf];
            C.w[pc] = w;
            C.e[pc] = w;
        }
        __syncthreads();
        // coarse right-hand side N_H(w_H) + res_H, colour-major
        for (int q = threadIdx.x; q < (nc - 2) * (nc - 2) * (nc - 2); q += TT) {
            const int i = 1 + q % (nc - 2), j = 1 + (q / (nc - 2)) % (nc - 2), k = 1 + q / ((nc - 2) * (nc - 2));
            const int p = (k * nc + j) * nc + i;
            int cnt;
            const int cm = tail_cm(i, j, k, nc, &cnt);
            const S3f B = tail_b(C.b, i, j, k, nc);
            const S3f K = corr_hess_sm(C.w, p, nc, nc * nc, C.w[p], A.lev[l + 1].inv_h2);
            C.rhs[cm] = delta_det(B, K) + C.r[p];
        }
        __syncthreads();
    }
    {   // coarsest grid: sweeps until max|de| <= 2e-6 max|e| (at most 40), or a fixed count
        const TailSmem& Bt = S[L - 1];
        const int n = A.lev[L - 1].n;
        __shared__ float red[TT / 32][2];
        __shared__ int stop;
        const int max_sweeps = A.coarse_sweeps > 0 ? A.coarse_sweeps : 40;
        for (int s = 0; s < max_sweeps; ++s) {
            float du = 0.0f, um = 0.0f;
            int off = 0;
            for (int c = 0; c < 8; ++c) {
                const int pi = c & 1, pj = (c >> 1) & 1, pk = (c >> 2) & 1;
                const int ni = colour_count(n, pi), nj = colour_count(n, pj), nk = colour_count(n, pk);
                const int cnt = (ni > 0 && nj > 0 && nk > 0) ? ni * nj * nk : 0;
                for (int t = threadIdx.x; t < cnt; t += TT) {
                    const int i = (pi ? 1 : 2) + 2 * (t % ni);
                    const int j = (pj ? 1 : 2) + 2 * ((t / ni) % nj);
                    const int k = (pk ? 1 : 2) + 2 * (t / (ni * nj));
                    const int p = (k * n + j) * n + i;
                    const float e0 = Bt.e[p];
                    const float* b = Bt.b + 6 * off + t;
                    S3f Bm;
                    Bm.xx = b[0]; Bm.yy = b[cnt]; Bm.zz = b[2 * cnt]; Bm.xy = b[3 * cnt]; Bm.xz = b[4 * cnt];
                    Bm.yz = b[5 * cnt];
                    const S3f K = corr_hess_sm(Bt.e, p, n, n * n, e0, A.lev[L - 1].inv_h2);
                    bool nonconvex = false;
                    const float z = corr_root(Bm, K, Bt.rhs[off + t], &nonconvex);
                    const float v = fmaf(A.lev[L - 1].h2half, z, e0);
                    Bt.e[p] = v;
                    du = fmaxf(du, fabsf(v - e0));
                    um = fmaxf(um, fabsf(v));
                    ev += nonconvex ? 1ull : 0ull;
                }
                off += cnt;
                __syncthreads();
            }
            if (A.coarse_sweeps > 0) continue;
            for (int o = 16; o > 0; o >>= 1) {
                du = fmaxf(du, __shfl_down_sync(0xffffffffu, du, o));
                um = fmaxf(um, __shfl_down_sync(0xffffffffu, um, o));
            }
            if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5][0] = du; red[threadIdx.x >> 5][1] = um; }
            __syncthreads();
            if (threadIdx.x == 0) {
                float a = 0.0f, b = 0.0f;
                for (int w = 0; w < TT / 32; ++w) { a = fmaxf(a, red[w][0]); b = fmaxf(b, red[w][1]); }
                stop = (a <= 2e-6f * b) ? 1 : 0;
            }
            __syncthreads();
            if (stop) break;
        }
    }
    for (int l = L - 2; l >= 0; --l) {
        const TailSmem& F = S[l];
        const TailSmem& C = S[l + 1];
        const int nf = A.lev[l].n, nc = A.lev[l + 1].n;
        // prolongation e_h += I(e_H - w_H) on the fine interior, each value formed as xfer::k_prolong forms it
        for (int q = threadIdx.x; q < (nf - 2) * (nf - 2) * (nf - 2); q += TT) {
            const int i = 1 + q % (nf - 2), j = 1 + (q / (nf - 2)) % (nf - 2), k = 1 + q / ((nf - 2) * (nf - 2));
            const int J0 = j >> 1, K0 = k >> 1, oj = j & 1, ok = k & 1;
            const float w = 1.0f / (float)(1 << (oj + ok));
            float v;
            if (i & 1) {
                const int I = i >> 1;
                const float a = tail_line(C.e, C.w, nc, I, J0, K0, oj, ok, w);
                const float b = tail_line(C.e, C.w, nc, I + 1, J0, K0, oj, ok, w);
                v = (a + b) * 0.5f;
            } else {
                v = tail_line(C.e, C.w, nc, i >> 1, J0, K0, oj, ok, w);
            }
            const int p = (k * nf + j) * nf + i;
            F.e[p] = F.e[p] + v;
        }
        __syncthreads();
        tail_smooth(F, nf, A.lev[l].inv_h2, A.lev[l].h2half, A.nu2, A.lev[l].pairs != 0, &ev);
    }
    const int m0 = A.lev[0].n * A.lev[0].n * A.lev[0].n;
    for (int q = threadIdx.x; q < m0; q += TT) A.lev[0].e[q] = S[0].e[q];
    if (A.events && ev) atomicAdd(A.events, ev);
}

__global__ void __launch_bounds__(TT, 1) k_corr_vcycle_tail(TailArgs A) { corr_tail_body(A); }

// FP64 <-> FP32 copies of whole grids (the FP32 mode's iterate and data).
__global__ void k_f64_to_f32(const double* __restrict__ u, float* __restrict__ e, long long m)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < m) e[p] = __double2float_rn(u[p]);
}

__global__ void k_f32_to_f64(const float* __restrict__ e, double* __restrict__ u, long long m)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < m) u[p] = (double)e[p];
}

// FP64 fine residual, written as FP32 in colour-major order (the correction
// problem's right-hand side), and with it the fine base Hessian B = D^2_h u
// of the correction operator, rounded to FP32 from the FP64 Hessian the
// residual already formed; the shell is not stored.
struct CmF32Out {
    float* r;
    float* b;        // colour-major B store of the level
    float inv_4h2;   // 1 / (4 h^2)
    // the residual without FP64 arithmetic (resid::residual_f2_block)
    __device__ __forceinline__ void put2(long long, int i, int j, int k, int n, const resid::ResF2& v) const
    {
        const CmPos c = cm_pos(i, j, k, n);
        r[c.off + c.idx] = v.val.hi;
        float* q = b + 6 * c.off + c.idx;
        q[0] = v.H[0].hi * inv_4h2;
        q[c.cnt] = v.H[1].hi * inv_4h2;
        q[2 * c.cnt] = v.H[2].hi * inv_4h2;
        q[3 * c.cnt] = v.H[3].hi * inv_4h2;
        q[4 * c.cnt] = v.H[4].hi * inv_4h2;
        q[5 * c.cnt] = v.H[5].hi * inv_4h2;
    }
    __device__ __forceinline__ void zero(long long) const {}
};

// u += e (optional) and e = 0 over the whole grid.
constexpr int UT = 256;   // threads of the k_update blocks

__device__ __forceinline__ void update_block(double* __restrict__ u, float* __restrict__ e, long long m, int apply,
                                             unsigned bx)
{
    const long long p = (long long)bx * UT + threadIdx.x;
    if (p >= m) return;
    if (apply) u[p] += f2d(e[p]);
    e[p] = 0.0f;
}

__global__ void __launch_bounds__(UT) k_update(double* __restrict__ u, float* __restrict__ e, long long m, int apply)
{
    update_block(u, e, m, apply, blockIdx.x);
}

// Coarse-level FP32 split hi + lo of the injected FP64 iterate: coarse point
// (I, J, K) takes fine point (sI, sJ, sK), s = 2^level.
__device__ __forceinline__ void split_inject_block(const double* __restrict__ u0, int n0, int stride,
                                                   float* __restrict__ hi, float* __restrict__ lo, int nc, uint3 bid)
{
    const int I = bid.x * BX + threadIdx.x;
    const int J = bid.y * BY + threadIdx.y;
    const int K = bid.z;
    if (I >= nc || J >= nc) return;
    const double v = u0[lin(stride * I, stride * J, stride * K, n0)];
    const float h = d2f_trunc(v);
    const long long pc = lin(I, J, K, nc);
    hi[pc] = h;
    lo[pc] = d2f_trunc(v - f2d(h));
}

__global__ void __launch_bounds__(BX * BY) k_split_inject(const double* __restrict__ u0, int n0, int stride,
                                                          float* __restrict__ hi, float* __restrict__ lo, int nc)
{
    split_inject_block(u0, n0, stride, hi, lo, nc, blockIdx);
}

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

// One sweep in colour pairs (4 launches): the colour order 0, 7, 1, 6, 2, 5,
// 3, 4.
static cudaError_t colour_sweep_corr_pair(float* e, const float* b, const float* rhs_cm, int n, float inv_h2,
                                          float h2half, unsigned long long* events, cudaStream_t s)
{
    cudaError_t e_;
    if ((e_ = launch_colour_corr_pair<0>(e, b, rhs_cm, n, inv_h2, h2half, events, s)) != cudaSuccess) return e_;
    if ((e_ = launch_colour_corr_pair<1>(e, b, rhs_cm, n, inv_h2, h2half, events, s)) != cudaSuccess) return e_;
    if ((e_ = launch_colour_corr_pair<2>(e, b, rhs_cm, n, inv_h2, h2half, events, s)) != cudaSuccess) return e_;
    return launch_colour_corr_pair<3>(e, b, rhs_cm, n, inv_h2, h2half, events, s);
}

// One sweep of in-place per-colour launches (8 launches).
static cudaError_t colour_sweep_corr(float* e, const float* b, const float* rhs_cm, int n, float inv_h2, float h2half,
                                     unsigned long long* events, cudaStream_t s)
{
    cudaError_t e_;
    if ((e_ = launch_colour_corr<0>(e, b, rhs_cm, n, inv_h2, h2half, events, s)) != cudaSuccess) return e_;
    if ((e_ = launch_colour_corr<1>(e, b, rhs_cm, n, inv_h2, h2half, events, s)) != cudaSuccess) return e_;
    if ((e_ = launch_colour_corr<2>(e, b, rhs_cm, n, inv_h2, h2half, events, s)) != cudaSuccess) return e_;
    if ((e_ = launch_colour_corr<3>(e, b, rhs_cm, n, inv_h2, h2half, events, s)) != cudaSuccess) return e_;
    if ((e_ = launch_colour_corr<4>(e, b, rhs_cm, n, inv_h2, h2half, events, s)) != cudaSuccess) return e_;
    if ((e_ = launch_colour_corr<5>(e, b, rhs_cm, n, inv_h2, h2half, events, s)) != cudaSuccess) return e_;
    if ((e_ = launch_colour_corr<6>(e, b, rhs_cm, n, inv_h2, h2half, events, s)) != cudaSuccess) return e_;
    return launch_colour_corr<7>(e, b, rhs_cm, n, inv_h2, h2half, events, s);
}

namespace {

// ---- choice of smoother and residual kernels per level size ----------------
// Tuning table: per grid size n (odd, 3 .. 4097), the correction-smoother
// variant (CORR_BY_COLOUR or a plane tile) and the residual variant (a plane
// tile or CORR_COLUMN), set by the
// autotuner (ma_tune_corr) or by hand; -1 = the built-in default.
constexpr int kTuneMaxN = 4097;
std::atomic<int> g_smooth_choice[kTuneMaxN + 1];
std::atomic<int> g_resid_choice[kTuneMaxN + 1];
std::atomic<int> g_tune_init{0};

int tune_slot(int n) { return (n >= 3 && n <= kTuneMaxN && (n & 1)) ? n : -1; }

void tune_init()
{
    if (g_tune_init.load(std::memory_order_acquire)) return;
    for (int i = 0; i <= kTuneMaxN; ++i) {
        g_smooth_choice[i].store(-1, std::memory_order_relaxed);
        g_resid_choice[i].store(-1, std::memory_order_relaxed);
    }
    g_tune_init.store(1, std::memory_order_release);
}

// Defaults before tuning: small grids are launch-latency bound, so the
// plane-phase sweep (2 launches per sweep instead of 8) with small tiles.
// The colour-pair sweep at every size: timed inside CUDA graphs, the form in
// which hierarchies run their cycles, it is the fastest variant from 9^3 to
// 513^3 (a dependent launch costs ~1 us there, so its 4 launches a sweep
// beat the plane tiles' 2 longer ones even on small grids).
int default_smooth_choice(int) { return CORR_PAIRS; }
int default_resid_choice(int) { return CORR_COLUMN; }   // the fastest residual at 33^3 .. 513^3 on GB300

template <int PT>
dim3 tile_grid(int n, int planes)
{
    const int t = (n - 2 + PT - 1) / PT;
    return dim3(t, t, planes);
}

// One sweep by k parity (2 launches): src -> dst, both with a zero shell.
template <int PT, int NT>
cudaError_t plane_sweep_t(const float* src, float* dst, const float* b, const float* rhs_cm, int n, float inv_h2,
                          float h2half, unsigned long long* events, cudaStream_t s)
{
    const int ne = colour_count(n, 0), no = colour_count(n, 1);
    if (ne > 0) {
        count_launches(1);
        k_smooth_corr_plane<0, PT, NT><<<tile_grid<PT>(n, ne), NT, Tile<PT>::SMEM, s>>>(src, src, dst, b, rhs_cm, n,
                                                                                         inv_h2, h2half, events);
        cudaError_t e_ = cudaGetLastError();
        if (e_ != cudaSuccess) return e_;
    }
    count_launches(1);
    k_smooth_corr_plane<1, PT, NT><<<tile_grid<PT>(n, no), NT, Tile<PT>::SMEM, s>>>(src, dst, dst, b, rhs_cm, n,
                                                                                     inv_h2, h2half, events);
    return cudaGetLastError();
}

cudaError_t plane_sweep(int choice, const float* src, float* dst, const float* b, const float* rhs_cm, int n,
                        float inv_h2, float h2half, unsigned long long* events, cudaStream_t s)
{
    switch (choice) {
    case CORR_PLANE16: return plane_sweep_t<16, 128>(src, dst, b, rhs_cm, n, inv_h2, h2half, events, s);
    case CORR_PLANE32: return plane_sweep_t<32, 128>(src, dst, b, rhs_cm, n, inv_h2, h2half, events, s);
    default: return plane_sweep_t<64, 256>(src, dst, b, rhs_cm, n, inv_h2, h2half, events, s);
    }
}

template <int PT, int NT>
cudaError_t residual_t(const float* e, const float* b, const float* rhs_cm, float* res, int n, float inv_h2,
                       cudaStream_t s)
{
    count_launches(1);
    k_residual_corr_plane<PT, NT><<<tile_grid<PT>(n, n - 2), NT, Tile<PT>::SMEM, s>>>(e, b, rhs_cm, res, n, inv_h2);
    return cudaGetLastError();
}

}  // namespace

int corr_smooth_choice(int n)
{
    tune_init();
    const int sl = tune_slot(n);
    const int c = sl >= 0 ? g_smooth_choice[sl].load(std::memory_order_relaxed) : -1;
    return c >= 0 ? c : default_smooth_choice(n);
}

int corr_resid_choice(int n)
{
    tune_init();
    const int sl = tune_slot(n);
    const int c = sl >= 0 ? g_resid_choice[sl].load(std::memory_order_relaxed) : -1;
    return c >= 0 ? c : default_resid_choice(n);
}

bool set_corr_tuning(int n, int smooth, int resid)
{
    tune_init();
    const int sl = tune_slot(n);
    if (sl < 0) return false;
    g_smooth_choice[sl].store(smooth, std::memory_order_relaxed);
    g_resid_choice[sl].store(resid, std::memory_order_relaxed);
    return true;
}

cudaError_t launch_smooth_corr_choice(int choice, float* e, float* e2, const void* bstore, const float* rhs_cm, int n,
                                      double h, int nsweeps, unsigned long long* events, cudaStream_t s)
{
    const float inv_h2 = (float)(1.0 / (h * h));
    const float h2half = (float)(0.5 * h * h);
    const float* b = (const float*)bstore;
    int sw = 0;
    cudaError_t e_;
    // pairs of sweeps e -> e2 -> e by k parity; the rest in place by colour
    if (choice == CORR_PAIRS) {
        for (; sw < nsweeps; ++sw)
            if ((e_ = colour_sweep_corr_pair(e, b, rhs_cm, n, inv_h2, h2half, events, s)) != cudaSuccess) return e_;
        return cudaSuccess;
    }
    if (choice != CORR_BY_COLOUR && e2 && n >= 5)
        for (; sw + 2 <= nsweeps; sw += 2) {
            if ((e_ = plane_sweep(choice, e, e2, b, rhs_cm, n, inv_h2, h2half, events, s)) != cudaSuccess) return e_;
            if ((e_ = plane_sweep(choice, e2, e, b, rhs_cm, n, inv_h2, h2half, events, s)) != cudaSuccess) return e_;
        }
    for (; sw < nsweeps; ++sw)
        if ((e_ = colour_sweep_corr(e, b, rhs_cm, n, inv_h2, h2half, events, s)) != cudaSuccess) return e_;
    return cudaSuccess;
}

cudaError_t launch_smooth_corr_colour(int colour, float* e, const void* bstore, const float* rhs_cm, int n, double h,
                                      unsigned long long* events, cudaStream_t s)
{
    const float inv_h2 = (float)(1.0 / (h * h));
    const float h2half = (float)(0.5 * h * h);
    const float* b = (const float*)bstore;
    switch (colour) {
    case 0: return launch_colour_corr<0>(e, b, rhs_cm, n, inv_h2, h2half, events, s);
    case 1: return launch_colour_corr<1>(e, b, rhs_cm, n, inv_h2, h2half, events, s);
    case 2: return launch_colour_corr<2>(e, b, rhs_cm, n, inv_h2, h2half, events, s);
    case 3: return launch_colour_corr<3>(e, b, rhs_cm, n, inv_h2, h2half, events, s);
    case 4: return launch_colour_corr<4>(e, b, rhs_cm, n, inv_h2, h2half, events, s);
    case 5: return launch_colour_corr<5>(e, b, rhs_cm, n, inv_h2, h2half, events, s);
    case 6: return launch_colour_corr<6>(e, b, rhs_cm, n, inv_h2, h2half, events, s);
    case 7: return launch_colour_corr<7>(e, b, rhs_cm, n, inv_h2, h2half, events, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_smooth_corr(float* e, float* e2, const void* bstore, const float* rhs_cm, int n, double h,
                               int nsweeps, unsigned long long* events, cudaStream_t s)
{
    return launch_smooth_corr_choice(corr_smooth_choice(n), e, e2, bstore, rhs_cm, n, h, nsweeps, events, s);
}

cudaError_t launch_residual_corr_choice(int choice, const float* e, const void* bstore, const float* rhs_cm,
                                        float* res, int n, double h, cudaStream_t s)
{
    if (n < 3) return cudaSuccess;
    const float inv_h2 = (float)(1.0 / (h * h));
    const float* b = (const float*)bstore;
    switch (choice) {
    case CORR_PLANE16: return residual_t<16, 128>(e, b, rhs_cm, res, n, inv_h2, s);
    case CORR_PLANE32: return residual_t<32, 128>(e, b, rhs_cm, res, n, inv_h2, s);
    case CORR_COLUMN: {
        const int kc = col_chunk(n);
        count_launches(1);
        const dim3 g = col_grid(n, kc), blk(BX, BY);
        switch (n) {
        case 129: k_residual_corr_col<129><<<g, blk, 0, s>>>(e, b, rhs_cm, res, n, inv_h2, kc); break;
        case 257: k_residual_corr_col<257><<<g, blk, 0, s>>>(e, b, rhs_cm, res, n, inv_h2, kc); break;
        case 513: k_residual_corr_col<513><<<g, blk, 0, s>>>(e, b, rhs_cm, res, n, inv_h2, kc); break;
        default: k_residual_corr_col<0><<<g, blk, 0, s>>>(e, b, rhs_cm, res, n, inv_h2, kc); break;
        }
        return cudaGetLastError();
    }
    default: return residual_t<64, 256>(e, b, rhs_cm, res, n, inv_h2, s);
    }
}

cudaError_t launch_residual_corr(const float* e, const void* bstore, const float* rhs_cm, float* res, int n,
                                 double h, cudaStream_t s)
{
    return launch_residual_corr_choice(corr_resid_choice(n), e, bstore, rhs_cm, res, n, h, s);
}

cudaError_t launch_zero_shell_f32(float* v, int n, cudaStream_t s)
{
    count_launches(1);
    k_zero_shell<<<dim3((n + BX - 1) / BX, (n + BY - 1) / BY, 6), dim3(BX, BY), 0, s>>>(v, n);
    return cudaGetLastError();
}

cudaError_t launch_coarse_rhs_corr(const float* w, const void* bstore, const float* resc, float* rhs_cm, int nc,
                                   double H, cudaStream_t s)
{
    if (nc < 3) return cudaSuccess;
    const float* b = (const float*)bstore;
    const float inv_h2 = (float)(1.0 / (H * H));
    const dim3 blk(BX, BY);
    count_launches(1);
    if (nc < kCoarseRhsColMin) {
        k_coarse_rhs_corr<<<grid_of(nc), blk, 0, s>>>(w, b, resc, rhs_cm, nc, inv_h2);
        return cudaGetLastError();
    }
    const int kc = col_chunk(nc);
    const dim3 g = col_grid(nc, kc);
    switch (nc) {
    case 129: k_coarse_rhs_corr_col<129><<<g, blk, 0, s>>>(w, b, resc, rhs_cm, nc, inv_h2, kc); break;
    case 257: k_coarse_rhs_corr_col<257><<<g, blk, 0, s>>>(w, b, resc, rhs_cm, nc, inv_h2, kc); break;
    case 513: k_coarse_rhs_corr_col<513><<<g, blk, 0, s>>>(w, b, resc, rhs_cm, nc, inv_h2, kc); break;
    default: k_coarse_rhs_corr_col<0><<<g, blk, 0, s>>>(w, b, resc, rhs_cm, nc, inv_h2, kc); break;
    }
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
    xfer::k_prolong<float><<<xfer::prolong_grid(nf), dim3(BX, BY), 0, s>>>(ec, wc, nc, ef, nf, 1);
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

int tail_smem_bytes(const int* ns, int nlev)
{
    int f = 0;
    for (int l = 0; l < nlev; ++l) f += tail_level_floats(ns[l], l == 0);
    return f * (int)sizeof(float);
}

// Default largest level of the fused tail: at 17^3 one SM's serial colour
// phases take longer than the launches they replace, at 9^3 and below the
// launches cost more (measured on whole solves from 33^3 to 257^3).
constexpr int kTailDefault = 9;
std::atomic<int> g_tail_max{kTailDefault};

int corr_tail_max_n() { return g_tail_max.load(std::memory_order_relaxed); }

bool set_corr_tail(int max_n)
{
    if (max_n == 1) max_n = kTailDefault;
    if (!(max_n == 0 || max_n == 3 || max_n == 5 || max_n == 9 || max_n == kTailMaxN)) return false;
    g_tail_max.store(max_n, std::memory_order_relaxed);
    return true;
}

cudaError_t launch_corr_vcycle_tail(const TailSpec* lv, int nlev, int nu1, int nu2, int kind, int approx,
                                    int coarse_sweeps, unsigned long long* events, cudaStream_t s)
{
    if (nlev < 1 || nlev > 4) return cudaErrorInvalidValue;
    TailArgs A;
    A.nlev = nlev;
    int ns[4];
    for (int l = 0; l < nlev; ++l) {
        const double h = lv[l].h;
        A.lev[l].n = ns[l] = lv[l].n;
        A.lev[l].pairs = corr_smooth_choice(lv[l].n) == CORR_PAIRS;
        A.lev[l].inv_h2 = (float)(1.0 / (h * h));
        A.lev[l].h2half = (float)(0.5 * h * h);
        A.lev[l].e = lv[l].e;
        A.lev[l].b = (const float*)lv[l].bstore;
        A.lev[l].rhs = lv[l].rhs_cm;
    }
    A.nu1 = nu1;
    A.nu2 = nu2;
    A.kind = kind;
    A.approx = approx;
    A.coarse_sweeps = coarse_sweeps;
    A.events = events;
    count_launches(1);
    k_corr_vcycle_tail<<<1, TT, tail_smem_bytes(ns, nlev), s>>>(A);
    return cudaGetLastError();
}

cudaError_t prepare_coarsest_f64();
cudaError_t prepare_batched_kernels();

cudaError_t prepare_kernels()
{
    cudaError_t e = prepare_coarsest_f64();
    if (e != cudaSuccess) return e;
    if ((e = prepare_batched_kernels()) != cudaSuccess) return e;
    constexpr int big = Tile<64>::SMEM;
    if ((e = cudaFuncSetAttribute(k_smooth_corr_plane<0, 64, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) !=
        cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_smooth_corr_plane<1, 64, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) !=
        cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_residual_corr_plane<64, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) !=
        cudaSuccess)
        return e;
    const int tail_ns[4] = {17, 9, 5, 3};
    if ((e = cudaFuncSetAttribute(k_corr_vcycle_tail, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  tail_smem_bytes(tail_ns, 4))) != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(k_coarsest_corr, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)coarsest_corr_smem(17));
}

cudaError_t launch_update(double* u, float* e, int n, int apply, cudaStream_t s)
{
    const long long m = (long long)n * n * n;
    count_launches(1);
    k_update<<<(unsigned)((m + UT - 1) / UT), UT, 0, s>>>(u, e, m, apply);
    return cudaGetLastError();
}

cudaError_t launch_f64_to_f32(const double* u, float* e, int n, cudaStream_t s)
{
    const long long m = (long long)n * n * n;
    count_launches(1);
    k_f64_to_f32<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(u, e, m);
    return cudaGetLastError();
}

cudaError_t launch_f32_to_f64(const float* e, double* u, int n, cudaStream_t s)
{
    const long long m = (long long)n * n * n;
    count_launches(1);
    k_f32_to_f64<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(e, u, m);
    return cudaGetLastError();
}

cudaError_t launch_interpolate_f32(const float* ec, int nc, float* ef, cudaStream_t s)
{
    const int nf = 2 * nc - 1;
    count_launches(1);
    xfer::k_prolong<float><<<xfer::prolong_grid(nf), dim3(BX, BY), 0, s>>>(ec, nullptr, nc, ef, nf, 0);
    return cudaGetLastError();
}

cudaError_t launch_zero_interior_f32(float* e, int n, cudaStream_t s)
{
    count_launches(1);
    xfer::k_zero_interior<float><<<grid_of(n), dim3(BX, BY), 0, s>>>(e, n);
    return cudaGetLastError();
}

cudaError_t launch_split_inject(const double* u0, int n0, int stride, float* hi, float* lo, int nc, cudaStream_t s)
{
    count_launches(1);
    k_split_inject<<<grid_of(nc), dim3(BX, BY), 0, s>>>(u0, n0, stride, hi, lo, nc);
    return cudaGetLastError();
}

cudaError_t launch_residual_f2(const double* u, const double* rhs, double* r, int n, double h, cudaStream_t s)
{
    const double h2 = h * h;
    count_launches(1);
    const int kz = n < 16 ? n : 16;
    const int kchunk = (n + kz - 1) / kz;
    resid::launch_k_residual_f2(resid::grid_for(n, kz), s, u, rhs, resid::NaturalF2Out{r}, n,
                                1.0 / (64.0 * h2 * h2 * h2), nullptr, kchunk);
    return cudaGetLastError();
}

cudaError_t launch_residual64_to32(const double* u, const double* rhs, float* r_cm, void* bstore, int n, double h,
                                   double* partials, cudaStream_t s)
{
    const double h2 = h * h;
    count_launches(1);
    const int kz = n < 16 ? n : 16;
    const int kchunk = (n + kz - 1) / kz;
    resid::launch_k_residual_f2(resid::grid_for(n, kz), s, u, rhs, CmF32Out{r_cm, (float*)bstore, (float)(0.25 / h2)},
                                n, 1.0 / (64.0 * h2 * h2 * h2), partials, kchunk);
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Batched launches: the kernels of a mixed-precision outer iteration over the
// levels of several hierarchies at once.  A launch carries a table of jobs
// (one per hierarchy that has work at this step) and the first block of each;
// block b finds its job by binary search, skips it when the hierarchy's
// active flag is 0, and runs the same block body as the single-grid kernel
// with its block index inside that job's grid.  The levels are aligned by
// depth: the descents of all hierarchies run depth by depth, every
// hierarchy's fused tail (or coarsest solve) in one launch, then the ascents.
// ---------------------------------------------------------------------------
namespace {

using batched::split_block;
using batched::BLaunch;
using batched::TableBuilder;

struct SmoothJob {
    int inst, n, gx, gy;
    float inv_h2, h2half;
    float* e;
    const float* bc;
    const float* rc;
    unsigned long long* events;
};

template <int C>
struct OpSmooth {
    static constexpr int NT = BX * BY, MINB = 12;
    using Job = SmoothJob;
    static __device__ __forceinline__ void run(const Job& J, int q)
    {
        smooth_corr_block<C & 1, (C >> 1) & 1, (C >> 2) & 1, int>(J.e, J.bc, J.rc, J.n, J.inv_h2, J.h2half, J.events,
                                                                  split_block(q, J.gx, J.gy));
    }
};

// Colours C and C^7 of one grid (the colour-pair sweep): blocks with z below
// nk0 sweep colour C from the boxes b0 / r0, the rest colour C^7 from b1 / r1.
struct PairSmoothJob {
    int inst, n, gx, gy, nk0;
    float inv_h2, h2half;
    float* e;
    const float* b0;
    const float* r0;
    const float* b1;
    const float* r1;
    unsigned long long* events;
};

template <int C>
struct OpSmoothPair {
    static constexpr int NT = BX * BY, MINB = 12;
    using Job = PairSmoothJob;
    static __device__ __forceinline__ void run(const Job& J, int q)
    {
        constexpr int D = C ^ 7;
        uint3 bid = split_block(q, J.gx, J.gy);
        if ((int)bid.z < J.nk0) {
            smooth_corr_block<C & 1, (C >> 1) & 1, (C >> 2) & 1, int>(J.e, J.b0, J.r0, J.n, J.inv_h2, J.h2half,
                                                                      J.events, bid);
        } else {
            bid.z -= J.nk0;
            smooth_corr_block<D & 1, (D >> 1) & 1, (D >> 2) & 1, int>(J.e, J.b1, J.r1, J.n, J.inv_h2, J.h2half,
                                                                      J.events, bid);
        }
    }
};

struct PlaneSmoothJob {
    int inst, n, gx, gy;
    float inv_h2, h2half;
    const float* own;
    const float* nbr;
    float* dst;
    const float* b;
    const float* rhs;
    unsigned long long* events;
};

template <int PK, int PT, int NTH>
struct OpPlaneSmooth {
    static constexpr int NT = NTH, MINB = plane_min_blocks(PT, NTH);
    using Job = PlaneSmoothJob;
    static __device__ __forceinline__ void run(const Job& J, int q)
    {
        smooth_corr_plane_block<PK, PT, NTH>(J.own, J.nbr, J.dst, J.b, J.rhs, J.n, J.inv_h2, J.h2half, J.events,
                                             split_block(q, J.gx, J.gy));
    }
};

struct OpColResid {
    static constexpr int NT = BX * BY, MINB = 6;   // 8 spills with the job lookup
    struct Job {
        int inst, n, kc, gx, gy;
        float inv_h2;
        const float* e;
        const float* b;
        const float* rhs;
        float* res;
    };
    static __device__ __forceinline__ void run(const Job& J, int q)
    {
        residual_corr_col_block(J.e, J.b, J.rhs, J.res, J.n, J.inv_h2, J.kc, split_block(q, J.gx, J.gy));
    }
};

struct OpRestrict {
    static constexpr int NT = BX * BY, MINB = 1;
    struct Job {
        int inst, nf, nc, kind, approx, gx, gy;
        const float* ef;
        const float* rf;
        float* wc;
        float* ec;
        float* rc;
    };
    static __device__ __forceinline__ void run(const Job& J, int q)
    {
        xfer::restrict_block<float>(J.ef, J.rf, J.nf, J.wc, J.ec, J.rc, J.nc, J.kind, J.approx,
                                    split_block(q, J.gx, J.gy));
    }
};

// kc > 0: by columns (kc planes a thread, col_grid); kc = 0: one point a
// thread (grid_of), the forms and sizes of launch_coarse_rhs_corr.
struct OpCoarseRhs {
    static constexpr int NT = BX * BY, MINB = 6;
    struct Job {
        int inst, n, kc, gx, gy;
        float inv_h2;
        const float* w;
        const float* b;
        const float* resc;
        float* rhs;
    };
    static __device__ __forceinline__ void run(const Job& J, int q)
    {
        if (J.kc > 0)
            residual_corr_col_block<0, true>(J.w, J.b, J.resc, J.rhs, J.n, J.inv_h2, J.kc,
                                             split_block(q, J.gx, J.gy));
        else
            coarse_rhs_corr_block(J.w, J.b, J.resc, J.rhs, J.n, J.inv_h2, split_block(q, J.gx, J.gy));
    }
};

struct OpProlong {
    static constexpr int NT = BX * BY, MINB = 1;
    struct Job {
        int inst, nc, nf, gx, gy;
        const float* ec;
        const float* wc;
        float* ef;
    };
    static __device__ __forceinline__ void run(const Job& J, int q)
    {
        xfer::prolong_block<float>(J.ec, J.wc, J.nc, J.ef, J.nf, 1, split_block(q, J.gx, J.gy));
    }
};

struct OpTail {
    static constexpr int NT = TT, MINB = 1;
    struct Job {
        int inst;
        TailArgs A;
    };
    static __device__ __forceinline__ void run(const Job& J, int) { corr_tail_body(J.A); }
};

struct OpCoarsest {
    static constexpr int NT = CT, MINB = 1;
    struct Job {
        int inst, n, sweeps;
        float inv_h2, h2half;
        float* e;
        const float* b;
        const float* rhs;
        unsigned long long* events;
    };
    static __device__ __forceinline__ void run(const Job& J, int)
    {
        coarsest_corr_body(J.e, J.b, J.rhs, J.n, J.inv_h2, J.h2half, J.sweeps, J.events);
    }
};

struct OpUpdate {
    static constexpr int NT = UT, MINB = 1;
    struct Job {
        int inst, apply;
        long long m;
        double* u;
        float* e;
    };
    static __device__ __forceinline__ void run(const Job& J, int q)
    {
        update_block(J.u, J.e, J.m, J.apply, (unsigned)q);
    }
};

struct OpSplit {
    static constexpr int NT = BX * BY, MINB = 1;
    struct Job {
        int inst, n0, stride, nc, gx, gy;
        const double* u0;
        float* hi;
        float* lo;
    };
    static __device__ __forceinline__ void run(const Job& J, int q)
    {
        split_inject_block(J.u0, J.n0, J.stride, J.hi, J.lo, J.nc, split_block(q, J.gx, J.gy));
    }
};

struct OpBase {
    static constexpr int NT = BX * BY, MINB = 1;
    struct Job {
        int inst, n, gx, gy;
        float inv_h2;
        const float* hi;
        const float* lo;
        float* b;
    };
    static __device__ __forceinline__ void run(const Job& J, int q)
    {
        base_colour_block(J.hi, J.lo, J.b, J.n, J.inv_h2, split_block(q, J.gx, J.gy));
    }
};

struct OpRes64 {
    static constexpr int NT = resid::RX * resid::RY, MINB = 1;
    struct Job {
        int inst, n, kchunk, gx, gy, gz;
        double inv_h6;
        const double* u;
        const double* rhs;
        double* partials;
        CmF32Out out;
    };
    static __device__ __forceinline__ void run(const Job& J, int q)
    {
        resid::residual_f2_block<CmF32Out>(J.u, J.rhs, J.out, J.n, J.inv_h6, J.partials, J.kchunk,
                                           split_block(q, J.gx, J.gy),
                                           make_uint3((unsigned)J.gx, (unsigned)J.gy, (unsigned)J.gz));
    }
};

// The norms (max, L2) into out2 and a copy into pk (2 doubles); with ev_src,
// the root-event counter's bits into ev_dst.
struct OpNorm {
    static constexpr int NT = resid::NF, MINB = 1;
    struct Job {
        int inst, count;
        double h3;
        const double* partials;
        double* out2;
        double* pk;
        const unsigned long long* ev_src;
        double* ev_dst;
    };
    static __device__ __forceinline__ void run(const Job& J, int)
    {
        resid::norm_final_block(J.partials, J.count, J.h3, J.out2);
        if (threadIdx.x == 0) {
            if (J.pk) {
                J.pk[0] = J.out2[0];
                J.pk[1] = J.out2[1];
            }
            if (J.ev_src && J.ev_dst) {
                const unsigned long long ev = *J.ev_src;
                double d;
                memcpy(&d, &ev, sizeof d);
                *J.ev_dst = d;
            }
        }
    }
};

enum BatchOpId {
    B_SMOOTH0 = 0,   // .. B_SMOOTH0 + 7
    B_RESTRICT = 8, B_COARSE_RHS, B_PROLONG, B_TAIL, B_COARSEST, B_UPDATE, B_SPLIT, B_BASE, B_RES64, B_NORM,
    B_PSMOOTH16_0, B_PSMOOTH16_1, B_PSMOOTH32_0, B_PSMOOTH32_1,   // k-parity sweeps, tiles of 16 / 32, parity 0 / 1
    B_CRESID,                                                     // residual by columns
    B_PAIR0                                                       // .. B_PAIR0 + 3: colours c and c^7
};

dim3 batch_grid2(int n) { return dim3((n + BX - 1) / BX, (n + BY - 1) / BY, n); }

}  // namespace

struct BatchPlan {
    std::vector<BLaunch> start;   // FMG and the first outer iteration
    std::vector<BLaunch> seq;     // one outer iteration
    char* dev = nullptr;
    const int* active = nullptr;
};

namespace {

int tail_start(const BatchInstance& I, int tmax)
{
    int lt = I.L - 1;
    while (lt > 0 && I.lev[lt - 1].n <= tmax) --lt;
    return I.lev[lt].n <= tmax ? lt : -1;   // -1: no fused tail (coarsest solve alone)
}

// The launches of one batched outer iteration (start: the whole start, FMG
// included, before it; fmg_step: instead, an FMG level of the mixed solve,
// which ma_capi.cu's mixed_fmg_step runs for one hierarchy: e = 0 and the
// base Hessians below the top, the FP64 residual at the top without norms,
// the correction cycles, u += e at the top).
void build_sequence(TableBuilder& T, const BatchInstance* in, int count, const BatchParams& p, double* packed,
                    bool start, bool fmg_step = false)
{
    const auto inv_h2 = [](double h) { return (float)(1.0 / (h * h)); };
    const auto h2half = [](double h) { return (float)(0.5 * h * h); };
    // first level of each instance's tail (or its coarsest level)
    std::vector<int> lt(count);
    std::vector<int> fused(count);
    int D = 0;
    for (int b = 0; b < count; ++b) {
        const int t = tail_start(in[b], p.tail_max);
        fused[b] = t >= 0;
        lt[b] = t >= 0 ? t : in[b].L - 1;
        D = lt[b] > D ? lt[b] : D;
    }
    // Sweeps at depth d.  A grid whose size takes the colour-pair sweep
    // (corr_smooth_choice) runs it: 4 launches a sweep, colours c and c^7
    // together, the sequential sweep in the colour order 0, 7, 1, 6, 2, 5,
    // 3, 4.  The other grids sweep colours in ascending order: by k parity
    // through e2 (pairs of sweeps, 4 launches a pair) when all of them have
    // n <= 65, where launches cost more than the sweeps' work, by colour
    // otherwise, which are the same sweep bit for bit.  Every grid thus
    // takes the bits of its solo sweep.
    auto pairs_at = [&](int b, int d) { return corr_smooth_choice(in[b].lev[d].n) == CORR_PAIRS; };
    auto max_n_at = [&](int d) {   // over the grids that sweep in ascending order
        int m = 0;
        for (int b = 0; b < count; ++b)
            if (d < lt[b] && !pairs_at(b, d)) m = in[b].lev[d].n > m ? in[b].lev[d].n : m;
        return m;
    };
    auto pair_sweep = [&](int d) {
        for (int c = 0; c < 4; ++c) {
            std::vector<PairSmoothJob> jobs;
            std::vector<int> blocks;
            for (int b = 0; b < count; ++b) {
                if (d >= lt[b] || !pairs_at(b, d)) continue;
                const BatchLevel& F = in[b].lev[d];
                const int n = F.n;
                const int c7 = c ^ 7;
                const int nk0 = colour_count(n, (c >> 2) & 1), nk1 = colour_count(n, (c7 >> 2) & 1);
                const int edge = colour_count(n, 1);   // the larger box edge
                if (edge <= 0 || nk0 + nk1 <= 0) continue;
                const long long o0 = cm_offset(n, c), o1 = cm_offset(n, c7);
                PairSmoothJob J;
                J.inst = in[b].id;
                J.n = n;
                J.gx = (edge + BX - 1) / BX;
                J.gy = (edge + BY - 1) / BY;
                J.nk0 = nk0;
                J.inv_h2 = inv_h2(F.h);
                J.h2half = h2half(F.h);
                J.e = F.e;
                J.b0 = (const float*)F.bstore + 6 * o0;
                J.r0 = F.rhs32 + o0;
                J.b1 = (const float*)F.bstore + 6 * o1;
                J.r1 = F.rhs32 + o1;
                J.events = in[b].events;
                jobs.push_back(J);
                blocks.push_back(J.gx * J.gy * (nk0 + nk1));
            }
            T.emit(B_PAIR0 + c, jobs, blocks, 0);
        }
    };
    auto plane_pair = [&](int d) {
        const int mx = max_n_at(d);
        const int PT = mx <= 33 ? 16 : 32;
        for (int half = 0; half < 2; ++half)          // e -> e2, then e2 -> e
            for (int pk = 0; pk < 2; ++pk) {
                std::vector<PlaneSmoothJob> jobs;
                std::vector<int> blocks;
                for (int b = 0; b < count; ++b) {
                    if (d >= lt[b] || pairs_at(b, d)) continue;
                    const BatchLevel& F = in[b].lev[d];
                    const int n = F.n;
                    const int planes = colour_count(n, pk);
                    if (planes <= 0) continue;
                    float* src = half == 0 ? F.e : F.e2;
                    float* dst = half == 0 ? F.e2 : F.e;
                    PlaneSmoothJob J;
                    J.inst = in[b].id;
                    J.n = n;
                    J.gx = J.gy = (n - 2 + PT - 1) / PT;
                    J.inv_h2 = inv_h2(F.h);
                    J.h2half = h2half(F.h);
                    J.own = src;
                    J.nbr = pk == 0 ? src : dst;
                    J.dst = dst;
                    J.b = (const float*)F.bstore;
                    J.rhs = F.rhs32;
                    J.events = in[b].events;
                    jobs.push_back(J);
                    blocks.push_back(J.gx * J.gy * planes);
                }
                const int op = PT == 16 ? (pk ? B_PSMOOTH16_1 : B_PSMOOTH16_0) : (pk ? B_PSMOOTH32_1 : B_PSMOOTH32_0);
                T.emit(op, jobs, blocks, PT == 16 ? Tile<16>::SMEM : Tile<32>::SMEM);
            }
    };
    auto smooth = [&](int d, int nsweeps) {
        bool any_pairs = false, any_ascending = false;
        for (int b = 0; b < count; ++b)
            if (d < lt[b]) (pairs_at(b, d) ? any_pairs : any_ascending) = true;
        if (any_pairs)
            for (int q = 0; q < nsweeps; ++q) pair_sweep(d);
        if (!any_ascending) return;
        int sw = 0;
        bool plane = max_n_at(d) <= 65;
        for (int b = 0; b < count && plane; ++b)
            if (d < lt[b] && !pairs_at(b, d) && (!in[b].lev[d].e2 || in[b].lev[d].n < 5)) plane = false;
        if (plane)
            for (; sw + 2 <= nsweeps; sw += 2) plane_pair(d);
        for (; sw < nsweeps; ++sw)
            for (int c = 0; c < 8; ++c) {
                std::vector<SmoothJob> jobs;
                std::vector<int> blocks;
                for (int b = 0; b < count; ++b) {
                    if (d >= lt[b] || pairs_at(b, d)) continue;
                    const BatchLevel& F = in[b].lev[d];
                    const int n = F.n;
                    const int ni = colour_count(n, c & 1), nj = colour_count(n, (c >> 1) & 1),
                              nk = colour_count(n, (c >> 2) & 1);
                    if (ni <= 0 || nj <= 0 || nk <= 0) continue;
                    const long long off = cm_offset(n, c);
                    SmoothJob J;
                    J.inst = in[b].id;
                    J.n = n;
                    J.gx = (ni + BX - 1) / BX;
                    J.gy = (nj + BY - 1) / BY;
                    J.inv_h2 = inv_h2(F.h);
                    J.h2half = h2half(F.h);
                    J.e = F.e;
                    J.bc = (const float*)F.bstore + 6 * off;
                    J.rc = F.rhs32 + off;
                    J.events = in[b].events;
                    jobs.push_back(J);
                    blocks.push_back(J.gx * J.gy * nk);
                }
                T.emit(B_SMOOTH0 + c, jobs, blocks, 0);
            }
    };
    auto cycles = [&]() {
    for (int cyc = 0; cyc < p.inner; ++cyc) {
        for (int d = 0; d < D; ++d) {
            smooth(d, p.nu1);
            std::vector<OpColResid::Job> rj;
            std::vector<OpRestrict::Job> sj;
            std::vector<OpCoarseRhs::Job> cj;
            std::vector<int> rb, sb, cb;
            for (int b = 0; b < count; ++b) {
                if (d >= lt[b]) continue;
                const BatchLevel& F = in[b].lev[d];
                const BatchLevel& C = in[b].lev[d + 1];
                const dim3 gc = batch_grid2(C.n);
                const int kc = col_chunk(F.n);
                const dim3 gr = col_grid(F.n, kc);
                rj.push_back(OpColResid::Job{in[b].id, F.n, kc, (int)gr.x, (int)gr.y, inv_h2(F.h), F.e,
                                             (const float*)F.bstore, F.rhs32, F.res32});
                rb.push_back((int)(gr.x * gr.y * gr.z));
                OpRestrict::Job s{in[b].id, F.n, C.n, p.kind, p.approx, (int)gc.x, (int)gc.y, F.e, F.res32, C.w32, C.e,
                                  C.res32};
                sj.push_back(s);
                sb.push_back((int)(gc.x * gc.y * gc.z));
                const int kcc = C.n >= kCoarseRhsColMin ? col_chunk(C.n) : 0;
                const dim3 gq = kcc > 0 ? col_grid(C.n, kcc) : batch_grid2(C.n);
                OpCoarseRhs::Job q{in[b].id, C.n, kcc, (int)gq.x, (int)gq.y, inv_h2(C.h), C.w32,
                                   (const float*)C.bstore, C.res32, C.rhs32};
                cj.push_back(q);
                cb.push_back((int)(gq.x * gq.y * gq.z));
            }
            T.emit(B_CRESID, rj, rb, 0);   // the residual by columns: the fastest form at every size
            T.emit(B_RESTRICT, sj, sb, 0);
            T.emit(B_COARSE_RHS, cj, cb, 0);
        }
        {   // every hierarchy's tail (or coarsest solve), one launch
            std::vector<OpTail::Job> tj;
            std::vector<OpCoarsest::Job> kj;
            std::vector<int> tb, kb;
            int tsmem = 0, ksmem = 0;
            for (int b = 0; b < count; ++b) {
                const BatchInstance& I = in[b];
                if (fused[b]) {
                    OpTail::Job J;
                    std::memset(&J, 0, sizeof J);
                    J.inst = in[b].id;
                    TailArgs& A = J.A;
                    A.nlev = I.L - lt[b];
                    int ns[4] = {0, 0, 0, 0};
                    for (int q = 0; q < A.nlev; ++q) {
                        const BatchLevel& V = I.lev[lt[b] + q];
                        ns[q] = V.n;
                        A.lev[q].n = V.n;
                        A.lev[q].pairs = corr_smooth_choice(V.n) == CORR_PAIRS;
                        A.lev[q].inv_h2 = inv_h2(V.h);
                        A.lev[q].h2half = h2half(V.h);
                        A.lev[q].e = V.e;
                        A.lev[q].b = (const float*)V.bstore;
                        A.lev[q].rhs = V.rhs32;
                    }
                    A.nu1 = p.nu1;
                    A.nu2 = p.nu2;
                    A.kind = p.kind;
                    A.approx = p.approx;
                    A.coarse_sweeps = p.coarse_sweeps;
                    A.events = I.events;
                    const int sm = tail_smem_bytes(ns, A.nlev);
                    tsmem = sm > tsmem ? sm : tsmem;
                    tj.push_back(J);
                    tb.push_back(1);
                } else {
                    const BatchLevel& V = I.lev[I.L - 1];
                    OpCoarsest::Job J{in[b].id, V.n, p.coarse_sweeps, inv_h2(V.h), h2half(V.h), V.e,
                                      (const float*)V.bstore, V.rhs32, I.events};
                    const int sm = (int)coarsest_corr_smem(V.n);
                    ksmem = sm > ksmem ? sm : ksmem;
                    kj.push_back(J);
                    kb.push_back(1);
                }
            }
            T.emit(B_TAIL, tj, tb, tsmem);
            T.emit(B_COARSEST, kj, kb, ksmem);
        }
        for (int d = D - 1; d >= 0; --d) {
            std::vector<OpProlong::Job> pj;
            std::vector<int> pb;
            for (int b = 0; b < count; ++b) {
                if (d >= lt[b]) continue;
                const BatchLevel& F = in[b].lev[d];
                const BatchLevel& C = in[b].lev[d + 1];
                const dim3 g = xfer::prolong_grid(F.n);
                OpProlong::Job J{in[b].id, C.n, F.n, (int)g.x, (int)g.y, C.e, C.w32, F.e};
                pj.push_back(J);
                pb.push_back((int)(g.x * g.y * g.z));
            }
            T.emit(B_PROLONG, pj, pb, 0);
            smooth(d, p.nu2);
        }
    }
    };
    // u += e (apply) and e = 0; the coarse base Hessians of the iterate
    auto update = [&](int apply) {
        std::vector<OpUpdate::Job> uj;
        std::vector<int> ub;
        for (int b = 0; b < count; ++b) {
            const BatchLevel& F = in[b].lev[0];
            const long long m = (long long)F.n * F.n * F.n;
            uj.push_back(OpUpdate::Job{in[b].id, apply, m, F.u, F.e});
            ub.push_back((int)((m + UT - 1) / UT));
        }
        T.emit(B_UPDATE, uj, ub, 0);
    };
    auto refresh = [&](int apply) {
        update(apply);
        int Lmax = 0;
        for (int b = 0; b < count; ++b) Lmax = in[b].L > Lmax ? in[b].L : Lmax;
        for (int l = 1; l < Lmax; ++l) {
            std::vector<OpSplit::Job> sj;
            std::vector<OpBase::Job> bj;
            std::vector<int> sb, bb;
            for (int b = 0; b < count; ++b) {
                if (l >= in[b].L) continue;
                const BatchLevel& F = in[b].lev[0];
                const BatchLevel& A = in[b].lev[l];
                const dim3 g = batch_grid2(A.n);
                sj.push_back(OpSplit::Job{in[b].id, F.n, 1 << l, A.n, (int)g.x, (int)g.y, F.u, A.hi, A.lo});
                sb.push_back((int)(g.x * g.y * g.z));
                bj.push_back(
                    OpBase::Job{in[b].id, A.n, (int)g.x, (int)g.y, inv_h2(A.h), A.hi, A.lo, (float*)A.bstore});
                bb.push_back((int)(g.x * g.y * g.z));
            }
            T.emit(B_SPLIT, sj, sb, 0);
            T.emit(B_BASE, bj, bb, 0);
        }
    };
    // FP64 fine residual (the next correction rhs and the fine B) and its norms
    auto residual_norm = [&](bool norms) {
        std::vector<OpRes64::Job> rj;
        std::vector<OpNorm::Job> nj;
        std::vector<int> rb, nb;
        for (int b = 0; b < count; ++b) {
            const BatchInstance& I = in[b];
            const BatchLevel& F = I.lev[0];
            const int n = F.n;
            const double h2 = F.h * F.h;
            const int kz = n < 16 ? n : 16;
            const dim3 g = resid::grid_for(n, kz);
            OpRes64::Job J;
            std::memset(&J, 0, sizeof J);
            J.inst = in[b].id;
            J.n = n;
            J.kchunk = (n + kz - 1) / kz;
            J.gx = (int)g.x;
            J.gy = (int)g.y;
            J.gz = (int)g.z;
            J.inv_h6 = 1.0 / (64.0 * h2 * h2 * h2);
            J.u = F.u;
            J.rhs = F.rhs;
            J.partials = I.partials;
            J.out = CmF32Out{F.rhs32, (float*)F.bstore, (float)(0.25 / h2)};
            rj.push_back(J);
            rb.push_back((int)(g.x * g.y * g.z));
            OpNorm::Job N{in[b].id, I.npartials, F.h * F.h * F.h, I.partials, I.out2,
                          packed ? packed + 5 * in[b].id : nullptr, I.events,
                          packed ? packed + 5 * in[b].id + 4 : nullptr};
            nj.push_back(N);
            nb.push_back(1);
        }
        T.emit(B_RES64, rj, rb, 0);
        if (norms) T.emit(B_NORM, nj, nb, 0);
    };
    if (fmg_step) {
        refresh(0);
        residual_norm(false);
        cycles();
        update(1);
        return;
    }
    if (start) {
        // Algorithm 2 as ma_solve_begin runs it in mixed precision: the
        // reference norms of f, FMG with a mixed step on each level below
        // the finest, then the finest level's first outer iteration
        emit_rhs_partials_f64(T, in, count);
        std::vector<OpNorm::Job> nj;
        std::vector<int> nb;
        for (int b = 0; b < count; ++b) {
            const BatchInstance& I = in[b];
            const double h = I.lev[0].h;
            nj.push_back(OpNorm::Job{I.id, I.npartials, h * h * h, I.partials, I.ref_out2,
                                     packed ? packed + 5 * I.id + 2 : nullptr, nullptr, nullptr});
            nb.push_back(1);
        }
        T.emit(B_NORM, nj, nb, 0);
        // the FMG levels below the finest as mixed steps on the hierarchies
        // seen from that level down (in an FMG step they all have the same
        // level sizes, so the depth-aligned launches apply)
        emit_fmg_f64(T, in, count, p, [&](const std::vector<std::pair<int, int>>& E) {
            std::vector<BatchInstance> sub;
            for (const std::pair<int, int>& v : E) {
                BatchInstance I = in[v.first];
                I.L = in[v.first].L - v.second;
                for (int k = 0; k < I.L; ++k) I.lev[k] = in[v.first].lev[v.second + k];
                sub.push_back(I);
            }
            BatchParams q = p;
            q.inner = kFmgCorrCycles;
            build_sequence(T, sub.data(), (int)sub.size(), q, packed, false, true);
        });
        refresh(0);
        residual_norm(true);
    }
    cycles();
    refresh(1);
    residual_norm(true);
}

template <typename Op>
cudaError_t launch_batched(const BatchPlan* P, const BLaunch& L, dim3 block, cudaStream_t s)
{
    return batched::launch<Op>(P->dev, L, block, P->active, s);
}

}  // namespace

size_t batch_tables_bytes(const BatchInstance* in, int count, const BatchParams& p)
{
    TableBuilder T;
    build_sequence(T, in, count, p, nullptr, true);
    build_sequence(T, in, count, p, nullptr, false);
    return T.buf.size();
}

BatchPlan* batch_plan_create(const BatchInstance* in, int count, const BatchParams& p, void* tables_dev,
                             const int* active_dev, double* packed_dev, cudaStream_t s, cudaError_t* err)
{
    TableBuilder T;
    build_sequence(T, in, count, p, packed_dev, true);
    const size_t nstart = T.seq.size();
    build_sequence(T, in, count, p, packed_dev, false);
    *err = cudaSuccess;
    if (!T.buf.empty()) {
        *err = cudaMemcpyAsync(tables_dev, T.buf.data(), T.buf.size(), cudaMemcpyHostToDevice, s);
        if (*err == cudaSuccess) *err = cudaStreamSynchronize(s);
    }
    if (*err != cudaSuccess) return nullptr;
    BatchPlan* P = new (std::nothrow) BatchPlan();
    if (!P) {
        *err = cudaErrorMemoryAllocation;
        return nullptr;
    }
    P->start.assign(T.seq.begin(), T.seq.begin() + nstart);
    P->seq.assign(T.seq.begin() + nstart, T.seq.end());
    P->dev = (char*)tables_dev;
    P->active = active_dev;
    return P;
}

static cudaError_t run_sequence(const BatchPlan* P, const std::vector<BLaunch>& seq, cudaStream_t s)
{
    const dim3 b2(BX, BY);
    for (const BLaunch& L : seq) {
        cudaError_t e;
        if (L.op >= batched::kF64Ops) {
            if ((e = batch_launch_f64(P->dev, L, P->active, s)) != cudaSuccess) return e;
            continue;
        }
        switch (L.op) {
        case B_SMOOTH0 + 0: e = launch_batched<OpSmooth<0>>(P, L, b2, s); break;
        case B_SMOOTH0 + 1: e = launch_batched<OpSmooth<1>>(P, L, b2, s); break;
        case B_SMOOTH0 + 2: e = launch_batched<OpSmooth<2>>(P, L, b2, s); break;
        case B_SMOOTH0 + 3: e = launch_batched<OpSmooth<3>>(P, L, b2, s); break;
        case B_SMOOTH0 + 4: e = launch_batched<OpSmooth<4>>(P, L, b2, s); break;
        case B_SMOOTH0 + 5: e = launch_batched<OpSmooth<5>>(P, L, b2, s); break;
        case B_SMOOTH0 + 6: e = launch_batched<OpSmooth<6>>(P, L, b2, s); break;
        case B_SMOOTH0 + 7: e = launch_batched<OpSmooth<7>>(P, L, b2, s); break;
        case B_RESTRICT: e = launch_batched<OpRestrict>(P, L, b2, s); break;
        case B_COARSE_RHS: e = launch_batched<OpCoarseRhs>(P, L, b2, s); break;
        case B_PROLONG: e = launch_batched<OpProlong>(P, L, b2, s); break;
        case B_TAIL: e = launch_batched<OpTail>(P, L, dim3(OpTail::NT), s); break;
        case B_COARSEST: e = launch_batched<OpCoarsest>(P, L, dim3(OpCoarsest::NT), s); break;
        case B_UPDATE: e = launch_batched<OpUpdate>(P, L, dim3(OpUpdate::NT), s); break;
        case B_SPLIT: e = launch_batched<OpSplit>(P, L, b2, s); break;
        case B_BASE: e = launch_batched<OpBase>(P, L, b2, s); break;
        case B_RES64: e = launch_batched<OpRes64>(P, L, dim3(resid::RX, resid::RY), s); break;
        case B_NORM: e = launch_batched<OpNorm>(P, L, dim3(OpNorm::NT), s); break;
        case B_PSMOOTH16_0: e = launch_batched<OpPlaneSmooth<0, 16, 128>>(P, L, dim3(128), s); break;
        case B_PSMOOTH16_1: e = launch_batched<OpPlaneSmooth<1, 16, 128>>(P, L, dim3(128), s); break;
        case B_PSMOOTH32_0: e = launch_batched<OpPlaneSmooth<0, 32, 128>>(P, L, dim3(128), s); break;
        case B_PSMOOTH32_1: e = launch_batched<OpPlaneSmooth<1, 32, 128>>(P, L, dim3(128), s); break;
        case B_CRESID: e = launch_batched<OpColResid>(P, L, b2, s); break;
        case B_PAIR0 + 0: e = launch_batched<OpSmoothPair<0>>(P, L, b2, s); break;
        case B_PAIR0 + 1: e = launch_batched<OpSmoothPair<1>>(P, L, b2, s); break;
        case B_PAIR0 + 2: e = launch_batched<OpSmoothPair<2>>(P, L, b2, s); break;
        case B_PAIR0 + 3: e = launch_batched<OpSmoothPair<3>>(P, L, b2, s); break;
        default: e = cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t batch_plan_start(const BatchPlan* P, cudaStream_t s) { return run_sequence(P, P->start, s); }

cudaError_t batch_plan_iteration(const BatchPlan* P, cudaStream_t s) { return run_sequence(P, P->seq, s); }

void batch_plan_destroy(BatchPlan* P) { delete P; }

cudaError_t prepare_batched_kernels()
{
    const int tail_ns[4] = {17, 9, 5, 3};
    cudaError_t e = cudaFuncSetAttribute(batched::k_batched<OpTail>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         tail_smem_bytes(tail_ns, 4));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(batched::k_batched<OpCoarsest>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)coarsest_corr_smem(17));
}

}  // namespace ma
