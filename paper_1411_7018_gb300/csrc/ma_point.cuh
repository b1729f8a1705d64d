// ma_point.cuh -- per-point arithmetic of the nonlinear Gauss-Seidel smoother
// (Section 2 of Liu, Froese, Oberman, Xiao): the 19-point stencil gather, the
// discrete Hessian, and the smallest-real-root selection of Eq. (realroots).
//
// Working units.  Everything is kept "h^2-scaled": Hs = h^2 D^2(u^h; v0)
// (the gathers return 4 Hs, with the right-hand side scaled to match),
// the discrete Hessian at the current centre value v0 times h^2, whose
// entries are exactly a - 2 v0, b - 2 v0, c - 2 v0, r, s, t with a..t the
// neighbour combinations defined after Eq. (MA3Dcubic).  With the centre
// moved to v = v0 + zeta / 2 the local equation P3(v) = 0 is
//     g(zeta) = det(Hs - zeta I) - h^6 rhs = 0,
// the same cubic as Eq. (MA3Dcubic) in the shifted variable (exact algebra;
// it avoids the cancellation of the monomial coefficients noted in the
// round-off remark of Example 4).  Theorem 2.2: for rhs > 0, g is decreasing
// and convex left of the smallest eigenvalue l1 of Hs, g(l1) < 0, and the
// smallest real root is the unique root below l1.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace ma {

// FP64 <-> FP32 moves done with integer operations on the bit patterns, so
// they do not occupy GB300's narrow FP64 pipe (which also executes the
// conversion instructions).  d2f_trunc truncates (the result is only an FP32
// starting value, never stored as a solution); values below FP32's normal
// range become signed zero, above it infinity.  f2d is exact for normal
// floats and zero.
__device__ __forceinline__ float d2f_trunc(double x)
{
    const int hi = __double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const unsigned sign = (unsigned)hi & 0x80000000u;
    const int ex = ((hi >> 20) & 0x7ff) - 1023 + 127;
    const unsigned mant = (((unsigned)hi & 0xfffffu) << 3) | (lo >> 29);
    unsigned r = sign;
    if (ex >= 255) r |= 0x7f800000u;
    else if (ex > 0) r |= ((unsigned)ex << 23) | mant;
    return __uint_as_float(r);
}

__device__ __forceinline__ double f2d(float f)
{
    const unsigned b = __float_as_uint(f);
    const unsigned sign = b & 0x80000000u;
    const int ex = (b >> 23) & 0xff;
    if (ex == 0) return __hiloint2double((int)sign, 0);
    const unsigned mant = b & 0x7fffffu;
    const unsigned hi = ex == 255 ? (sign | 0x7ff00000u | (mant >> 3))
                                  : (sign | ((unsigned)(ex - 127 + 1023) << 20) | (mant >> 3));
    return __hiloint2double((int)hi, (int)(mant << 29));
}

struct HessS {   // h^2-scaled symmetric Hessian: diagonal A, B, C; off-diagonal R (xy), S (xz), T (yz)
    double A, B, C, R, S, T;
};

struct HessSf {
    float A, B, C, R, S, T;
};

// 19-point gather at linear index p with strides sy (one j step) and sz
// (one k step); v0 is the current centre value.  Returns 4 Hs (the
// h^2-scaled discrete Hessian times 4): 4(a - 2 v0), ..., 4r = the bare cross
// sums, so no 1/4 scalings are spent; callers use det(4 Hs) = 64 det(Hs) and
// v = v0 + zeta4 / 8.  Neighbour loads go through the read-only path: no
// launch writes a point and reads it as a neighbour.
__device__ __forceinline__ HessS gather_hess(const double* __restrict__ u, long long p, long long sy,
                                             long long sz, double v0)
{
    const double* q = u + p;
    const double a = __ldg(q + 1) + __ldg(q - 1);
    const double b = __ldg(q + sy) + __ldg(q - sy);
    const double c = __ldg(q + sz) + __ldg(q - sz);
    const double r4 = (__ldg(q + sy + 1) + __ldg(q - sy - 1)) - (__ldg(q + sy - 1) + __ldg(q - sy + 1));
    const double s4 = (__ldg(q + sz + 1) + __ldg(q - sz - 1)) - (__ldg(q + sz - 1) + __ldg(q - sz + 1));
    const double t4 = (__ldg(q + sz + sy) + __ldg(q - sz - sy)) - (__ldg(q + sy - sz) + __ldg(q - sy + sz));
    HessS H;
    const double m8v = -8.0 * v0;
    H.A = fma(4.0, a, m8v);
    H.B = fma(4.0, b, m8v);
    H.C = fma(4.0, c, m8v);
    H.R = r4;
    H.S = s4;
    H.T = t4;
    return H;
}

// det(Hs - z I) by cofactor expansion along the first row.
__device__ __forceinline__ double det_shift(const HessS& H, double z)
{
    const double a = H.A - z, b = H.B - z, c = H.C - z;
    const double c1 = fma(b, c, -H.T * H.T);
    const double c2 = fma(H.R, c, -H.S * H.T);
    const double c3 = fma(H.R, H.T, -b * H.S);
    return fma(a, c1, fma(-H.R, c2, H.S * c3));
}

__device__ __forceinline__ double det0(const HessS& H)
{
    const double c1 = fma(H.B, H.C, -H.T * H.T);
    const double c2 = fma(H.R, H.C, -H.S * H.T);
    const double c3 = fma(H.R, H.T, -H.B * H.S);
    return fma(H.A, c1, fma(-H.R, c2, H.S * c3));
}

// Sum of the principal 2x2 minors of (Hs - z I); g'(z) = -minors_shift(z).
__device__ __forceinline__ double minors_shift(const HessS& H, double z)
{
    const double a = H.A - z, b = H.B - z, c = H.C - z;
    return fma(a, b, -H.R * H.R) + fma(a, c, -H.S * H.S) + fma(b, c, -H.T * H.T);
}

__device__ __forceinline__ float det_shift_f(const HessSf& H, float z)
{
    const float a = H.A - z, b = H.B - z, c = H.C - z;
    const float c1 = fmaf(b, c, -H.T * H.T);
    const float c2 = fmaf(H.R, c, -H.S * H.T);
    const float c3 = fmaf(H.R, H.T, -b * H.S);
    return fmaf(a, c1, fmaf(-H.R, c2, H.S * c3));
}

__device__ __forceinline__ float minors_shift_f(const HessSf& H, float z)
{
    const float a = H.A - z, b = H.B - z, c = H.C - z;
    return fmaf(a, b, -H.R * H.R) + fmaf(a, c, -H.S * H.S) + fmaf(b, c, -H.T * H.T);
}

// Lower bound of the smallest eigenvalue (Gershgorin discs).
template <typename M, typename F>
__device__ __forceinline__ F gershgorin_low(const M& H)
{
    const F g0 = H.A - fabs(H.R) - fabs(H.S);
    const F g1 = H.B - fabs(H.R) - fabs(H.T);
    const F g2 = H.C - fabs(H.S) - fabs(H.T);
    return fmin(g0, fmin(g1, g2));
}

// Sylvester's criterion: Hs positive definite.
template <typename M, typename F>
__device__ __forceinline__ bool is_pd(const M& H, F det)
{
    return H.A > F(0) && H.A * H.B - H.R * H.R > F(0) && det > F(0);
}

// FP64 monotone Newton from a point left of the root (g >= 0 there): for
// rhs > 0 the iterates increase to the unique root below l1 (convexity).
// Used when the FP32 first pass is not trustworthy (degenerate or far from
// convex); each step costs an FP64 division.
static __device__ __noinline__ double root_f64_monotone(const HessS H, double rhs6)
{
    double z = gershgorin_low<HessS, double>(H) - cbrt(rhs6);
    for (int it = 0; it < 200; ++it) {
        const double g = det_shift(H, z) - rhs6;
        const double m = minors_shift(H, z);
        if (!(g > 0.0) || !(m > 0.0)) break;
        const double zn = z + g / m;
        if (!(zn > z)) break;
        z = zn;
    }
    return z;
}

// Smallest real root of q(z) = c - M z + T z^2 - z^3 = 0 for a symmetric 3x3
// matrix X with trace T, principal-minor sum M and Gershgorin bounds [lo, hi]
// of its eigenvalues, when q(z) = det(X - z I) - t with t <= 0 (Eq.
// (realroots) taken literally: no root lies below the smallest eigenvalue).
// q > 0 below the eigenvalues; det(X - z I) has its local minimum at
// za = (T - sqrt(T^2 - 3M)) / 3, between the two smallest eigenvalues, and its
// local maximum at zb = (T + sqrt(T^2 - 3M)) / 3.  If q(za) <= 0 (within
// rounding: a double root) the smallest root is in [lo, za], else it is the
// root beyond zb, below hi + (-t)^(1/3).  Bisection on the bracket.
template <typename Q>
__device__ __forceinline__ double smallest_root_nonpositive(Q q, double T, double M, double glo, double ghi, double t,
                                                            double scale)
{
    const double sq = sqrt(fmax(T * T - 3.0 * M, 0.0));
    const double za = (T - sq) / 3.0, zb = (T + sq) / 3.0;
    const double tiny = 64.0 * 2.220446049250313e-16 * scale * scale * scale;
    double lo, hi;
    if (q(za) <= tiny) {
        lo = fmin(glo, za);
        hi = za;
    } else {
        lo = zb;
        hi = fmax(ghi, zb) + cbrt(fmax(-t, 0.0)) + tiny;
    }
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        if (q(mid) > 0.0) lo = mid;
        else hi = mid;
    }
    return q(lo) <= 0.0 ? lo : hi;
}

// rhs <= 0 for the FP64 smoother: the smallest real root of
// det(Hs - z I) = rhs6.
static __device__ __noinline__ double root_f64_all_real_min(const HessS H, double rhs6)
{
    const double T = H.A + H.B + H.C;
    const double M = minors_shift(H, 0.0);
    const double glo = gershgorin_low<HessS, double>(H);
    const double ghi = fmax(H.A + fabs(H.R) + fabs(H.S), fmax(H.B + fabs(H.R) + fabs(H.T), H.C + fabs(H.S) + fabs(H.T)));
    const double scale = fabs(H.A) + fabs(H.B) + fabs(H.C) + fabs(H.R) + fabs(H.S) + fabs(H.T);
    return smallest_root_nonpositive([&](double z) { return det_shift(H, z) - rhs6; }, T, M, glo, ghi, rhs6, scale);
}

// Smallest real root zeta of det(Hs - zeta I) = rhs6 (rhs6 = h^6 rhs).
//
// Fast path (rhs6 > 0): Newton in FP32 on the FP32-rounded cubic -- from
// zeta = 0 when Hs is positive definite (0 < l1, so Newton converges to the
// root below l1 with at most one step overshooting to its left), else from
// the Gershgorin bound minus rhs^(1/3) (left of the root) -- then one Newton
// correction whose residual g(zeta) is evaluated in FP64 with the FP32
// derivative.  That correction contracts the FP32 error by the derivative's
// relative error (~1e-7), leaving the root at FP64 accuracy; the fixed point
// of the sweep is therefore the FP64 discrete solution.  Degenerate cases
// (tiny derivative, no convergence, non-finite) take the FP64 path.
// *nonconvex is set when rhs6 <= 0.
__device__ __forceinline__ double smallest_root(const HessS& H, double rhs6, bool* nonconvex)
{
    if (!(rhs6 > 0.0)) {
        *nonconvex = true;
        return root_f64_all_real_min(H, rhs6);
    }
    HessSf F;
    F.A = d2f_trunc(H.A); F.B = d2f_trunc(H.B); F.C = d2f_trunc(H.C);
    F.R = d2f_trunc(H.R); F.S = d2f_trunc(H.S); F.T = d2f_trunc(H.T);
    const float r6 = d2f_trunc(rhs6);
    const float scale = fabsf(F.A) + fabsf(F.B) + fabsf(F.C) + fabsf(F.R) + fabsf(F.S) + fabsf(F.T);
    const float d0 = det_shift_f(F, 0.0f);
    float z = is_pd<HessSf, float>(F, d0) ? 0.0f : gershgorin_low<HessSf, float>(F) - cbrtf(r6);
    bool conv = false;
    float m = 0.0f;
    for (int it = 0; it < 60; ++it) {
        const float g = det_shift_f(F, z) - r6;
        m = minors_shift_f(F, z);
        const float dz = g / m;
        z += dz;
        if (!isfinite(z)) break;
        // FP32 resolves the root to ~1e-7 of the entries' size; stop there.
        if (fabsf(dz) <= 2e-6f * scale) { conv = true; break; }
    }
    m = minors_shift_f(F, z);
    // m = -g'(root); a small m (near-degenerate Hessian at the root) makes
    // the FP32 root and derivative too inaccurate for one FP64 correction.
    if (!conv || !(m > 0.05f * scale * scale) || !(r6 > 0.0f)) {
        return root_f64_monotone(H, rhs6);
    }
    double zd = f2d(z);
    const double g64 = det_shift(H, zd) - rhs6;
    zd = fma(g64, f2d(1.0f / m), zd);
    return zd;
}

// The same root, then one more Newton step with the FP64 derivative: a few
// ulps of the root instead of ~1e-14 of the entries' size.  For the coarsest
// grid, which is swept to a 1e-14 relative change.
__device__ __forceinline__ double smallest_root_precise(const HessS& H, double rhs6, bool* nonconvex)
{
    double z = smallest_root(H, rhs6, nonconvex);
    if (*nonconvex) return z;
    const double g = det_shift(H, z) - rhs6;
    const double m = minors_shift(H, z);
    if (m > 0.0) {
        const double zn = z + g / m;
        if (isfinite(zn)) z = zn;
    }
    return z;
}

}  // namespace ma
