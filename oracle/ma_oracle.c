/*
 * ma_oracle.c -- plain FP64 CPU statement of the FAS multigrid method for the
 * 3D elliptic Monge-Ampere equation  det(D^2 u) = f > 0,  u = g on the
 * boundary, u convex  (Liu, Froese, Oberman, Xiao, "A multigrid scheme for 3D
 * Monge-Ampere equations", arXiv:1411.7018).
 *
 * TEST INFRASTRUCTURE.  This file is the slow, obviously-correct oracle that
 * the CUDA library is checked against.  Only the test suite, the package's
 * smoke check and the benchmark's CPU-baseline leg may load it.  It shares no
 * code, header, table or constant with the CUDA path and the product path
 * never calls it.  Every routine follows the paper's definitions step by step
 * with no blocking, fusion or reordering; a reader should be able to check
 * each one against the cited passage by eye.
 *
 * Parity status: every exported routine is pinned by tests that do not use
 * this file's own formulas (closed forms, brute force, the paper's printed
 * values, library root finders); see tests/test_oracle_pins.py.
 *
 * Grid (Section 2): x_i = x0 + i h, i = 0..N, h = len / N.  A level stores all
 * n = N + 1 points per side, boundary shell included, as n^3 doubles in
 * [k][j][i] order (i fastest).  Shell values are the Dirichlet data g
 * (Eq. DBC) and no routine here changes them, except where stated.
 *
 * Root formulation.  Section 2 writes the local equation as the monomial cubic
 * P3(v) (Eq. MA3Dcubic) in the centre value v.  Its matrix form is
 *     P3(v) = det([[a-2v, r, s], [r, b-2v, t], [s, t, c-2v]]) - h^6 f
 *           = h^6 ( det(D^2(u^h; v)) - f ),
 * with D^2(u^h; v) the discrete Hessian of Eq. (discreteHessian).  Writing
 * v = v0 + h^2 z / 2 around the current value v0 gives D^2(u^h; v) = H - z I
 * with H = D^2(u^h; v0), so the roots in v are the roots in z of
 *     Q(z) = det(H - z I) - f = (l1 - z)(l2 - z)(l3 - z) - f,
 * l1 <= l2 <= l3 the eigenvalues of H (the form used in the proof of
 * Theorem 2.2).  This is exact algebra; it only avoids evaluating the
 * monomial coefficients, whose O(v^3) terms cancel down to O(h^6 f)
 * (the round-off remark at the end of Example 4).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define AT(u, n, i, j, k) ((u)[(((size_t)(k)) * (size_t)(n) + (size_t)(j)) * (size_t)(n) + (size_t)(i)])

enum { ORC_COLOUR8 = 0, ORC_LEXICOGRAPHIC = 1, ORC_COLOUR8_REVERSED = 2, ORC_COLOUR8_PAIRS = 3 };
enum { ORC_HALF_WEIGHTING = 0, ORC_FULL_WEIGHTING = 1 };
enum { ORC_NORM_MAX = 0, ORC_NORM_L2 = 1 };
enum { ORC_APPROX_INJECTION = 0, ORC_APPROX_WEIGHTED = 1 };
enum { ORC_FMG_TRILINEAR = 0, ORC_FMG_CUBIC = 1 };

/* ------------------------------------------------------------------------ */
/* Section 2: the stencil                                                    */
/* ------------------------------------------------------------------------ */

/* The six neighbour combinations a, b, c, r, s, t defined after
 * Eq. (MA3Dcubic), in that order, for interior point (i, j, k). */
static void neighbour_sums(const double *u, int n, int i, int j, int k, double q[6])
{
    q[0] = AT(u, n, i + 1, j, k) + AT(u, n, i - 1, j, k);
    q[1] = AT(u, n, i, j + 1, k) + AT(u, n, i, j - 1, k);
    q[2] = AT(u, n, i, j, k + 1) + AT(u, n, i, j, k - 1);
    q[3] = 0.25 * (AT(u, n, i + 1, j + 1, k) + AT(u, n, i - 1, j - 1, k)
                   - AT(u, n, i - 1, j + 1, k) - AT(u, n, i + 1, j - 1, k));
    q[4] = 0.25 * (AT(u, n, i + 1, j, k + 1) + AT(u, n, i - 1, j, k - 1)
                   - AT(u, n, i - 1, j, k + 1) - AT(u, n, i + 1, j, k - 1));
    q[5] = 0.25 * (AT(u, n, i, j + 1, k + 1) + AT(u, n, i, j - 1, k - 1)
                   - AT(u, n, i, j + 1, k - 1) - AT(u, n, i, j - 1, k + 1));
}

/* Eq. (discreteHessian): the discrete Hessian when the centre value is v and
 * the neighbours are held fixed; with v = u_ijk it is the centred-difference
 * Hessian of Eqs. (2.1)-(2.6). */
static void hessian_with_centre(const double q[6], double v, double h, double H[3][3])
{
    const double ih2 = 1.0 / (h * h);
    H[0][0] = (q[0] - 2.0 * v) * ih2;
    H[1][1] = (q[1] - 2.0 * v) * ih2;
    H[2][2] = (q[2] - 2.0 * v) * ih2;
    H[0][1] = H[1][0] = q[3] * ih2;
    H[0][2] = H[2][0] = q[4] * ih2;
    H[1][2] = H[2][1] = q[5] * ih2;
}

/* Section 1: the explicit form of det(D^2 u) in three dimensions. */
static double det_sym3(const double H[3][3])
{
    const double uxx = H[0][0], uyy = H[1][1], uzz = H[2][2];
    const double uxy = H[0][1], uxz = H[0][2], uyz = H[1][2];
    return uxx * uyy * uzz + 2.0 * uxy * uyz * uxz
         - uxx * uyz * uyz - uyy * uxz * uxz - uzz * uxy * uxy;
}

/* det(D^2_h u) at interior point (i, j, k) (Eq. MA_discrete, left side). */
static double discrete_ma(const double *u, int n, double h, int i, int j, int k)
{
    double q[6], H[3][3];
    neighbour_sums(u, n, i, j, k, q);
    hessian_with_centre(q, AT(u, n, i, j, k), h, H);
    return det_sym3(H);
}

/* ------------------------------------------------------------------------ */
/* Eigenvalues of a real symmetric 3x3 matrix (cyclic Jacobi rotations).     */
/* ------------------------------------------------------------------------ */

static void sym3_eigenvalues(const double M[3][3], double lam[3])
{
    double A[3][3];
    memcpy(A, M, sizeof A);
    static const int P[3] = {0, 0, 1}, Qx[3] = {1, 2, 2};
    for (int sweep = 0; sweep < 64; ++sweep) {
        const double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        const double dia = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
        if (off == 0.0 || off <= 1e-36 * dia) break;
        for (int m = 0; m < 3; ++m) {
            const int p = P[m], q = Qx[m];
            const double apq = A[p][q];
            if (apq == 0.0) continue;
            /* rotation J (J_pp = J_qq = c, J_pq = s, J_qp = -s) with
             * (J^T A J)_pq = 0 */
            const double theta = (A[q][q] - A[p][p]) / (2.0 * apq);
            double t;
            if (fabs(theta) > 1e150) t = 0.5 / theta;
            else t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
            const int r = 3 - p - q;
            const double arp = A[r][p], arq = A[r][q];
            A[r][p] = A[p][r] = c * arp - s * arq;
            A[r][q] = A[q][r] = s * arp + c * arq;
            A[p][p] -= t * apq;
            A[q][q] += t * apq;
            A[p][q] = A[q][p] = 0.0;
        }
    }
    lam[0] = A[0][0]; lam[1] = A[1][1]; lam[2] = A[2][2];
    /* ascending order */
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2 - a; ++b)
            if (lam[b] > lam[b + 1]) { double x = lam[b]; lam[b] = lam[b + 1]; lam[b + 1] = x; }
}

/* Q(z) = (l1 - z)(l2 - z)(l3 - z) - rhs and its derivative. */
static double q_eval(const double lam[3], double rhs, double z, double *dq)
{
    const double p0 = lam[0] - z, p1 = lam[1] - z, p2 = lam[2] - z;
    if (dq) *dq = -(p1 * p2 + p0 * p2 + p0 * p1);
    return p0 * p1 * p2 - rhs;
}


/* Eq. (realroots): the smallest real root z of Q(z) = det(H - z I) - rhs.
 *
 * rhs > 0 (Theorem 2.2): Q is strictly decreasing and convex on (-inf, l1),
 * Q(l1) = -rhs < 0 and Q(l1 - rhs^(1/3)) >= 0, so the smallest real root is
 * the unique root in [l1 - rhs^(1/3), l1).  Newton's method started at the
 * left end of that bracket increases monotonically to it; it stops when the
 * floating-point iterates stop increasing.
 *
 * rhs <= 0 (possible for a coarse-grid right-hand side b_H): no root lies
 * below l1; the literal rule of Eq. (realroots) is applied -- all real roots of
 * the cubic, polished by Newton, and the smallest is kept.  *nonconvex counts
 * these events. */
static double smallest_root(const double H[3][3], double rhs, long *nonconvex)
{
    double lam[3];
    sym3_eigenvalues(H, lam);
    if (rhs > 0.0) {
        double z = lam[0] - cbrt(rhs);
        for (int it = 0; it < 500; ++it) {
            double dq;
            const double qz = q_eval(lam, rhs, z, &dq);
            if (!(qz > 0.0) || !(dq < 0.0)) break;
            const double zn = z - qz / dq;
            if (!(zn > z) || !(zn < lam[0])) break;
            z = zn;
        }
        return z;
    }
    if (nonconvex) *nonconvex += 1;
    /* rhs <= 0: Eq. (realroots) literally, the smallest real root of
     * q(z) = (l1 - z)(l2 - z)(l3 - z) - rhs.  q > 0 below l1 and q(l1) =
     * q(l2) = -rhs >= 0; between l1 and l2 q dips to its minimum at
     * z* = (T - sqrt(S)) / 3 (T = l1 + l2 + l3, S = T^2 - 3 (l1 l2 + l1 l3 +
     * l2 l3) = ((l1-l2)^2 + (l1-l3)^2 + (l2-l3)^2) / 2), and it is positive
     * between l2 and l3 and decreasing beyond l3.  So the smallest root is l1
     * if rhs = 0, else in [l1, z*] if q(z*) <= 0 (a double root when = 0),
     * else the single root in (l3, l3 + (-rhs)^(1/3)].  Found by bisection
     * on the product form, which keeps double and triple roots exact. */
    if (rhs == 0.0) return lam[0];
    const double T = lam[0] + lam[1] + lam[2];
    const double S = 0.5 * ((lam[0] - lam[1]) * (lam[0] - lam[1]) + (lam[0] - lam[2]) * (lam[0] - lam[2]) +
                            (lam[1] - lam[2]) * (lam[1] - lam[2]));
    double zs = (T - sqrt(S)) / 3.0;
    if (zs < lam[0]) zs = lam[0];
    if (zs > lam[1]) zs = lam[1];
    double lo, hi;
    if (q_eval(lam, rhs, zs, NULL) <= 0.0) { lo = lam[0]; hi = zs; }
    else { lo = lam[2]; hi = lam[2] + cbrt(-rhs); }
    /* q(lo) >= 0 >= q(hi), q decreasing on [lo, hi] */
    for (int it = 0; it < 400; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        if (q_eval(lam, rhs, mid, NULL) > 0.0) lo = mid;
        else hi = mid;
    }
    return q_eval(lam, rhs, lo, NULL) <= 0.0 ? lo : hi;
}

/* One nonlinear Gauss-Seidel point update (Section 2, Eq. realroots): the new
 * u_ijk is the smallest real root v of P3(v; u), returned as
 * v = v0 + h^2 z / 2 with z the smallest root of det(D^2(u^h; v0) - z I) - rhs. */
static double point_update(const double q[6], double v0, double h, double rhs, long *nonconvex)
{
    double H[3][3];
    hessian_with_centre(q, v0, h, H);
    const double z = smallest_root(H, rhs, nonconvex);
    return v0 + 0.5 * h * h * z;
}

/* ------------------------------------------------------------------------ */
/* Nonlinear Gauss-Seidel sweeps (Section 2; smoother of Section 3)          */
/* ------------------------------------------------------------------------ */

static int first_interior(int parity) { return parity ? 1 : 2; }

/* One sweep over all interior points.  ORC_COLOUR8: eight colours
 * c = (i&1) | (j&1)<<1 | (k&1)<<2 visited in ascending c; no stencil
 * neighbour of a point has the point's colour (every neighbour differs in at
 * least one index parity), so the points of one colour are independent and
 * may be updated in any order.  ORC_COLOUR8_REVERSED visits each colour's
 * points in the opposite order (same result by that independence).
 * ORC_COLOUR8_PAIRS visits the colours in the order 0, 7, 1, 6, 2, 5, 3, 4
 * (each colour followed by the one that differs in all three parities).
 * ORC_LEXICOGRAPHIC is the paper's own ordering.  rhs is f on the finest
 * level and b_H on coarse levels.  Returns the number of point updates whose
 * right-hand side was <= 0. */
long orc_gs_sweep(double *u, const double *rhs, int n, double h, int ordering)
{
    long events = 0;
    if (ordering == ORC_LEXICOGRAPHIC) {
        for (int k = 1; k <= n - 2; ++k)
            for (int j = 1; j <= n - 2; ++j)
                for (int i = 1; i <= n - 2; ++i) {
                    double q[6];
                    neighbour_sums(u, n, i, j, k, q);
                    AT(u, n, i, j, k) = point_update(q, AT(u, n, i, j, k), h, AT(rhs, n, i, j, k), &events);
                }
        return events;
    }
    static const int pair_order[8] = {0, 7, 1, 6, 2, 5, 3, 4};
    for (int q = 0; q < 8; ++q) {
        const int c = (ordering == ORC_COLOUR8_PAIRS) ? pair_order[q] : q;
        const int pi = c & 1, pj = (c >> 1) & 1, pk = (c >> 2) & 1;
        const int i0 = first_interior(pi), j0 = first_interior(pj), k0 = first_interior(pk);
        const int nk = (n - 2 >= k0) ? (n - 2 - k0) / 2 + 1 : 0;
        long ev = 0;
#pragma omp parallel for reduction(+ : ev) schedule(static)
        for (int kk = 0; kk < nk; ++kk) {
            const int k = (ordering == ORC_COLOUR8_REVERSED) ? k0 + 2 * (nk - 1 - kk) : k0 + 2 * kk;
            for (int j = j0; j <= n - 2; j += 2)
                for (int i = i0; i <= n - 2; i += 2) {
                    int ii = i, jj = j;
                    if (ordering == ORC_COLOUR8_REVERSED) {
                        ii = i0 + (n - 2 - i0) / 2 * 2 - (i - i0);
                        jj = j0 + (n - 2 - j0) / 2 * 2 - (j - j0);
                    }
                    double q[6];
                    neighbour_sums(u, n, ii, jj, k, q);
                    AT(u, n, ii, jj, k) = point_update(q, AT(u, n, ii, jj, k), h, AT(rhs, n, ii, jj, k), &ev);
                }
        }
        events += ev;
    }
    return events;
}

/* ------------------------------------------------------------------------ */
/* Residual and norms (Algorithm 1 step 3; stopping rule of Section 4)       */
/* ------------------------------------------------------------------------ */

/* r = rhs - S_h(u) with S_h(u) = det(D^2_h u) on the interior; r = 0 on the
 * shell. */
void orc_residual(const double *u, const double *rhs, double *r, int n, double h)
{
    memset(r, 0, sizeof(double) * (size_t)n * n * n);
#pragma omp parallel for schedule(static)
    for (int k = 1; k <= n - 2; ++k)
        for (int j = 1; j <= n - 2; ++j)
            for (int i = 1; i <= n - 2; ++i)
                AT(r, n, i, j, k) = AT(rhs, n, i, j, k) - discrete_ma(u, n, h, i, j, k);
}

/* Max norm, or the discrete L2 norm sqrt(h^3 sum v^2), over the interior. */
double orc_norm(const double *v, int n, double h, int kind)
{
    double mx = 0.0, ss = 0.0;
    for (int k = 1; k <= n - 2; ++k)
        for (int j = 1; j <= n - 2; ++j)
            for (int i = 1; i <= n - 2; ++i) {
                const double x = AT(v, n, i, j, k);
                if (fabs(x) > mx) mx = fabs(x);
                ss += x * x;
            }
    return kind == ORC_NORM_MAX ? mx : sqrt(h * h * h * ss);
}

/* ------------------------------------------------------------------------ */
/* Grid transfers (Section 3)                                                */
/* ------------------------------------------------------------------------ */

/* Restriction I_h^H at coarse interior point (I, J, K), i.e. at fine point
 * (2I, 2J, 2K).  Half weighting is the 7-point stencil printed in Section 3:
 * (6 * centre + the six face neighbours) / 12.  Full weighting is the 27-point
 * tensor-product stencil with weights 8 (centre), 4 (face), 2 (edge),
 * 1 (corner), divided by 64. */
static double restrict_point(const double *vf, int nf, int I, int J, int K, int kind)
{
    const int i = 2 * I, j = 2 * J, k = 2 * K;
    if (kind == ORC_HALF_WEIGHTING) {
        return (6.0 * AT(vf, nf, i, j, k)
                + AT(vf, nf, i + 1, j, k) + AT(vf, nf, i - 1, j, k)
                + AT(vf, nf, i, j + 1, k) + AT(vf, nf, i, j - 1, k)
                + AT(vf, nf, i, j, k + 1) + AT(vf, nf, i, j, k - 1)) / 12.0;
    }
    double s = 0.0;
    for (int dk = -1; dk <= 1; ++dk)
        for (int dj = -1; dj <= 1; ++dj)
            for (int di = -1; di <= 1; ++di) {
                const double w = (double)((2 - abs(di)) * (2 - abs(dj)) * (2 - abs(dk)));
                s += w * AT(vf, nf, i + di, j + dj, k + dk);
            }
    return s / 64.0;
}

/* r_H = I_h^H r_h on the coarse interior; 0 on the coarse shell. */
void orc_restrict_residual(const double *rf, int nf, double *rc, int nc, int kind)
{
    memset(rc, 0, sizeof(double) * (size_t)nc * nc * nc);
    for (int K = 1; K <= nc - 2; ++K)
        for (int J = 1; J <= nc - 2; ++J)
            for (int I = 1; I <= nc - 2; ++I)
                AT(rc, nc, I, J, K) = restrict_point(rf, nf, I, J, K, kind);
}

/* Straight injection (the operator written with a tilde in Algorithm 1):
 * v_H(I, J, K) = v_h(2I, 2J, 2K) at every coarse point, shell included. */
void orc_inject(const double *vf, int nf, double *vc, int nc)
{
    for (int K = 0; K < nc; ++K)
        for (int J = 0; J < nc; ++J)
            for (int I = 0; I < nc; ++I)
                AT(vc, nc, I, J, K) = AT(vf, nf, 2 * I, 2 * J, 2 * K);
}

/* u_H = I_h^H w_h (Algorithm 1 step 4): restriction on the coarse interior,
 * injection of the Dirichlet data on the coarse shell. */
void orc_restrict_solution(const double *uf, int nf, double *uc, int nc, int kind)
{
    orc_inject(uf, nf, uc, nc);
    for (int K = 1; K <= nc - 2; ++K)
        for (int J = 1; J <= nc - 2; ++J)
            for (int I = 1; I <= nc - 2; ++I)
                AT(uc, nc, I, J, K) = restrict_point(uf, nf, I, J, K, kind);
}

/* Trilinear interpolation of coarse field d at fine point (i, j, k): along each
 * axis an even fine index sits on a coarse point (weight 1) and an odd one
 * halfway between two (weights 1/2, 1/2). */
static double trilinear_at(const double *d, int nc, int i, int j, int k)
{
    int I[2], J[2], K[2];
    double wi[2], wj[2], wk[2];
    int ni, nj, nk;
    if (i % 2 == 0) { I[0] = i / 2; wi[0] = 1.0; ni = 1; } else { I[0] = (i - 1) / 2; I[1] = (i + 1) / 2; wi[0] = wi[1] = 0.5; ni = 2; }
    if (j % 2 == 0) { J[0] = j / 2; wj[0] = 1.0; nj = 1; } else { J[0] = (j - 1) / 2; J[1] = (j + 1) / 2; wj[0] = wj[1] = 0.5; nj = 2; }
    if (k % 2 == 0) { K[0] = k / 2; wk[0] = 1.0; nk = 1; } else { K[0] = (k - 1) / 2; K[1] = (k + 1) / 2; wk[0] = wk[1] = 0.5; nk = 2; }
    double s = 0.0;
    for (int c = 0; c < nk; ++c)
        for (int b = 0; b < nj; ++b)
            for (int a = 0; a < ni; ++a)
                s += wi[a] * wj[b] * wk[c] * AT(d, nc, I[a], J[b], K[c]);
    return s;
}

/* Algorithm 1 steps 7-8: w_h := w_h + I_H^h (u_H - w_H) on the fine interior
 * (I_H^h trilinear; the correction vanishes on the shell). */
void orc_prolong_add(const double *uc, const double *wc, int nc, double *uf, int nf)
{
    const size_t m = (size_t)nc * nc * nc;
    double *d = (double *)malloc(sizeof(double) * m);
    for (size_t p = 0; p < m; ++p) d[p] = uc[p] - wc[p];
    for (int k = 1; k <= nf - 2; ++k)
        for (int j = 1; j <= nf - 2; ++j)
            for (int i = 1; i <= nf - 2; ++i)
                AT(uf, nf, i, j, k) += trilinear_at(d, nc, i, j, k);
    free(d);
}

/* Algorithm 2 step 4 with trilinear interpolation in place of the cubic one:
 * fine interior values from the coarse solution; the fine shell keeps g. */
void orc_interpolate(const double *uc, int nc, double *uf, int nf)
{
    for (int k = 1; k <= nf - 2; ++k)
        for (int j = 1; j <= nf - 2; ++j)
            for (int i = 1; i <= nf - 2; ++i)
                AT(uf, nf, i, j, k) = trilinear_at(uc, nc, i, j, k);
}

/* Cubic interpolation along one axis (Algorithm 2 step 4, the cubic
 * interpolation the paper recommends for FMG): the coarse points and weights
 * that give fine index i.  An even i sits on coarse point i/2.  An odd i lies
 * halfway between coarse points I0 = (i-1)/2 and I0 + 1 and takes the cubic
 * through four neighbouring coarse points: I0-1 .. I0+2 (weights -1, 9, 9, -1
 * over 16), or, next to the boundary, the four nearest ones (0..3 with 5, 15,
 * -5, 1 over 16, and the mirror image at the far end).  A 3-point coarse grid
 * has only a quadratic (3, 6, -1 over 8), a 2-point one a linear midpoint.
 * Returns the number of points. */
static int cubic_stencil(int i, int nc, int idx[4], double w[4])
{
    if (i % 2 == 0) { idx[0] = i / 2; w[0] = 1.0; return 1; }
    const int I0 = (i - 1) / 2;
    if (nc == 2) { idx[0] = 0; idx[1] = 1; w[0] = w[1] = 0.5; return 2; }
    if (nc == 3) {
        idx[0] = 0; idx[1] = 1; idx[2] = 2;
        if (I0 == 0) { w[0] = 3.0 / 8; w[1] = 6.0 / 8; w[2] = -1.0 / 8; }
        else         { w[0] = -1.0 / 8; w[1] = 6.0 / 8; w[2] = 3.0 / 8; }
        return 3;
    }
    if (I0 == 0) {
        for (int a = 0; a < 4; ++a) idx[a] = a;
        w[0] = 5.0 / 16; w[1] = 15.0 / 16; w[2] = -5.0 / 16; w[3] = 1.0 / 16;
    } else if (I0 == nc - 2) {
        for (int a = 0; a < 4; ++a) idx[a] = nc - 4 + a;
        w[0] = 1.0 / 16; w[1] = -5.0 / 16; w[2] = 15.0 / 16; w[3] = 5.0 / 16;
    } else {
        for (int a = 0; a < 4; ++a) idx[a] = I0 - 1 + a;
        w[0] = -1.0 / 16; w[1] = 9.0 / 16; w[2] = 9.0 / 16; w[3] = -1.0 / 16;
    }
    return 4;
}

/* Algorithm 2 step 4 with tricubic interpolation: the tensor product of the
 * per-axis cubic stencils, fine interior only (the shell keeps g). */
void orc_interpolate_cubic(const double *uc, int nc, double *uf, int nf)
{
    for (int k = 1; k <= nf - 2; ++k)
        for (int j = 1; j <= nf - 2; ++j)
            for (int i = 1; i <= nf - 2; ++i) {
                int ix[4], iy[4], iz[4];
                double wx[4], wy[4], wz[4];
                const int nx = cubic_stencil(i, nc, ix, wx);
                const int ny = cubic_stencil(j, nc, iy, wy);
                const int nz = cubic_stencil(k, nc, iz, wz);
                double s = 0.0;
                for (int c = 0; c < nz; ++c)
                    for (int b = 0; b < ny; ++b)
                        for (int a = 0; a < nx; ++a)
                            s += wz[c] * wy[b] * wx[a] * AT(uc, nc, ix[a], iy[b], iz[c]);
                AT(uf, nf, i, j, k) = s;
            }
}

/* Algorithm 1 step 5: b_H = S_H(w_H) + r_H on the coarse interior (S_H the
 * same discrete operator with step H, Section 3); 0 on the shell. */
void orc_coarse_rhs(const double *wc, const double *rc, double *bc, int nc, double H)
{
    memset(bc, 0, sizeof(double) * (size_t)nc * nc * nc);
    for (int K = 1; K <= nc - 2; ++K)
        for (int J = 1; J <= nc - 2; ++J)
            for (int I = 1; I <= nc - 2; ++I)
                AT(bc, nc, I, J, K) = discrete_ma(wc, nc, H, I, J, K) + AT(rc, nc, I, J, K);
}

/* ------------------------------------------------------------------------ */
/* FAS V-cycle (Algorithm 1) and FMG (Algorithm 2)                           */
/* ------------------------------------------------------------------------ */

typedef struct {
    int nu1, nu2;        /* pre- and post-smoothing sweeps (Section 4 uses 2, 2) */
    int coarsest_n;      /* points per side of the coarsest grid (3 or 5)        */
    int restrict_kind;   /* ORC_HALF_WEIGHTING or ORC_FULL_WEIGHTING              */
    int coarse_sweeps;   /* > 0: that many sweeps on the coarsest grid;
                            0: sweep until max|du| <= 1e-14 max|u| (cap 100)     */
    int ordering;        /* sweep ordering (ORC_COLOUR8 ...)                     */
    int approx_restrict; /* ORC_APPROX_INJECTION or ORC_APPROX_WEIGHTED            */
    int fmg_interp;      /* ORC_FMG_TRILINEAR or ORC_FMG_CUBIC (Algorithm 2 step 4) */
} orc_params;

typedef struct { int n; double h; double *u, *rhs, *r, *w; } orc_level;
typedef struct { int nlev; orc_level lev[24]; orc_params p; long events; } orc_hier;

static int hier_init(orc_hier *H, int n, double h, const orc_params *p)
{
    memset(H, 0, sizeof *H);
    H->p = *p;
    int m = n;
    double hh = h;
    while (1) {
        if (H->nlev >= 24) return -1;
        orc_level *L = &H->lev[H->nlev++];
        L->n = m; L->h = hh;
        const size_t sz = sizeof(double) * (size_t)m * m * m;
        L->u = (double *)calloc(1, sz); L->rhs = (double *)calloc(1, sz);
        L->r = (double *)calloc(1, sz); L->w = (double *)calloc(1, sz);
        if (!L->u || !L->rhs || !L->r || !L->w) return -1;
        if (m <= p->coarsest_n) break;
        if ((m - 1) % 2 != 0) return -1;
        m = (m + 1) / 2;
        hh *= 2.0;
    }
    return H->lev[H->nlev - 1].n == p->coarsest_n ? 0 : -1;
}

static void hier_free(orc_hier *H)
{
    for (int l = 0; l < H->nlev; ++l) {
        free(H->lev[l].u); free(H->lev[l].rhs); free(H->lev[l].r); free(H->lev[l].w);
    }
}

/* Algorithm 1 step 1: approximate solve on the coarsest grid. */
static void coarsest_solve(orc_hier *H, orc_level *L)
{
    if (H->p.coarse_sweeps > 0) {
        for (int s = 0; s < H->p.coarse_sweeps; ++s)
            H->events += orc_gs_sweep(L->u, L->rhs, L->n, L->h, H->p.ordering);
        return;
    }
    /* sweep to convergence; prev is private scratch (lev.w still holds w_H) */
    const size_t m = (size_t)L->n * L->n * L->n;
    double *prev = (double *)malloc(sizeof(double) * m);
    for (int s = 0; s < 100; ++s) {
        memcpy(prev, L->u, sizeof(double) * m);
        H->events += orc_gs_sweep(L->u, L->rhs, L->n, L->h, H->p.ordering);
        double du = 0.0, um = 0.0;
        for (size_t q = 0; q < m; ++q) {
            if (fabs(L->u[q] - prev[q]) > du) du = fabs(L->u[q] - prev[q]);
            if (fabs(L->u[q]) > um) um = fabs(L->u[q]);
        }
        if (du <= 1e-14 * um) break;
    }
    free(prev);
}

/* Algorithm 1 (FAS V-cycle) at level l; the iterate is lev[l].u, the
 * right-hand side lev[l].rhs. */
static void fas_vcycle(orc_hier *H, int l)
{
    orc_level *F = &H->lev[l];
    if (l == H->nlev - 1) { coarsest_solve(H, F); return; }
    orc_level *C = &H->lev[l + 1];
    for (int s = 0; s < H->p.nu1; ++s)                                  /* (2) */
        H->events += orc_gs_sweep(F->u, F->rhs, F->n, F->h, H->p.ordering);
    orc_residual(F->u, F->rhs, F->r, F->n, F->h);                       /* (3) */
    orc_restrict_residual(F->r, F->n, C->r, C->n, H->p.restrict_kind);
    /* (4) w_H = restricted approximation, and the coarse iterate u_H starts
     * from the same values, so that u_H - w_H in step (7) carries only what
     * the coarse solve changed.  The approximation restriction operator is
     * straight injection (Section 3) or, as an option, the residual's own
     * weighting (full weighting of u). */
    if (H->p.approx_restrict == ORC_APPROX_INJECTION)
        orc_inject(F->u, F->n, C->w, C->n);
    else
        orc_restrict_solution(F->u, F->n, C->w, C->n, H->p.restrict_kind);
    memcpy(C->u, C->w, sizeof(double) * (size_t)C->n * C->n * C->n);
    orc_coarse_rhs(C->w, C->r, C->rhs, C->n, C->h);                     /* (5) */
    fas_vcycle(H, l + 1);                                               /* (6) */
    orc_prolong_add(C->u, C->w, C->n, F->u, F->n);                      /* (7)-(8) */
    for (int s = 0; s < H->p.nu2; ++s)                                  /* (9) */
        H->events += orc_gs_sweep(F->u, F->rhs, F->n, F->h, H->p.ordering);
}

/* Algorithm 2 (FMG-FAS) at level l.  On entry lev[l].rhs holds b_h and the
 * shell of lev[l].u holds the Dirichlet data; the interior is overwritten. */
static void fmg(orc_hier *H, int l)
{
    orc_level *F = &H->lev[l];
    if (l == H->nlev - 1) {
        /* zero initial guess on the coarsest interior (Section 3, after
         * Algorithm 2), then the approximate solve */
        for (int k = 1; k <= F->n - 2; ++k)
            for (int j = 1; j <= F->n - 2; ++j)
                for (int i = 1; i <= F->n - 2; ++i) AT(F->u, F->n, i, j, k) = 0.0;
        coarsest_solve(H, F);
        return;
    }
    orc_level *C = &H->lev[l + 1];
    orc_inject(F->rhs, F->n, C->rhs, C->n);    /* (2) b_H = injection of b_h */
    orc_inject(F->u, F->n, C->u, C->n);        /*     coarse Dirichlet data  */
    fmg(H, l + 1);                             /* (3) */
    if (H->p.fmg_interp == ORC_FMG_CUBIC)      /* (4) */
        orc_interpolate_cubic(C->u, C->n, F->u, F->n);
    else
        orc_interpolate(C->u, C->n, F->u, F->n);
    fas_vcycle(H, l);                          /* (5) */
}

static int load(orc_hier *H, const double *u, const double *f, int n, double h, const orc_params *p)
{
    if (hier_init(H, n, h, p) != 0) { hier_free(H); return -1; }
    const size_t m = sizeof(double) * (size_t)n * n * n;
    memcpy(H->lev[0].u, u, m);
    memcpy(H->lev[0].rhs, f, m);
    return 0;
}

/* ncycles FAS V-cycles (Algorithm 1) on the finest level, in place on u.
 * Returns the number of nonconvex root events (rhs <= 0), or -1 on a bad
 * grid size. */
long orc_vcycle(double *u, const double *f, int n, double h, const orc_params *p, int ncycles)
{
    orc_hier H;
    if (load(&H, u, f, n, h, p) != 0) return -1;
    for (int c = 0; c < ncycles; ++c) fas_vcycle(&H, 0);
    memcpy(u, H.lev[0].u, sizeof(double) * (size_t)n * n * n);
    const long ev = H.events;
    hier_free(&H);
    return ev;
}

/* One FMG-FAS pass (Algorithm 2) on the finest level; u's shell supplies g,
 * its interior is overwritten.  Return value as orc_vcycle. */
long orc_fmg(double *u, const double *f, int n, double h, const orc_params *p)
{
    orc_hier H;
    if (load(&H, u, f, n, h, p) != 0) return -1;
    fmg(&H, 0);
    memcpy(u, H.lev[0].u, sizeof(double) * (size_t)n * n * n);
    const long ev = H.events;
    hier_free(&H);
    return ev;
}

/* Solve to tolerance: optional FMG initialisation (init = 1), then V-cycles
 * until ||f - S_h(u)|| / ref <= tol (norm kind over the fine interior) or
 * max_cycles.  ref_kind 0: ref = ||f||; 1: ref = the residual norm of the
 * initial iterate (Section 4's relative residual ||r^l|| / ||r^0||; with FMG
 * the initial iterate is the zero interior that FMG starts from).
 * res_hist[0..cycles] receives the relative residual after the
 * initialisation and after each cycle.  Returns the number of cycles, or -1. */
int orc_solve(double *u, const double *f, int n, double h, const orc_params *p,
              double tol, int norm, int max_cycles, int init, int ref_kind, double *res_hist, long *events)
{
    orc_hier H;
    if (load(&H, u, f, n, h, p) != 0) return -1;
    orc_level *F = &H.lev[0];
    double ref = orc_norm(f, n, h, norm);
    if (ref_kind == 1) {
        if (init)
            for (int k = 1; k <= n - 2; ++k)
                for (int j = 1; j <= n - 2; ++j)
                    for (int i = 1; i <= n - 2; ++i) AT(F->u, n, i, j, k) = 0.0;
        orc_residual(F->u, F->rhs, F->r, n, h);
        ref = orc_norm(F->r, n, h, norm);
    }
    if (init) fmg(&H, 0);
    orc_residual(F->u, F->rhs, F->r, n, h);
    double rel = orc_norm(F->r, n, h, norm) / ref;
    if (res_hist) res_hist[0] = rel;
    int c = 0;
    while (rel > tol && c < max_cycles) {
        fas_vcycle(&H, 0);
        ++c;
        orc_residual(F->u, F->rhs, F->r, n, h);
        rel = orc_norm(F->r, n, h, norm) / ref;
        if (res_hist) res_hist[c] = rel;
    }
    memcpy(u, F->u, sizeof(double) * (size_t)n * n * n);
    if (events) *events = H.events;
    hier_free(&H);
    return c;
}

/* ------------------------------------------------------------------------ */
/* Point-level entry points used by the pins                                 */
/* ------------------------------------------------------------------------ */

/* Smallest real root z of det(H - z I) - rhs for a symmetric H given as 9
 * row-major doubles. */
double orc_smallest_root(const double *Hrm, double rhs)
{
    double H[3][3];
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) H[a][b] = Hrm[3 * a + b];
    long ev = 0;
    return smallest_root(H, rhs, &ev);
}

/* New centre value from the stencil combinations q = (a, b, c, r, s, t), the
 * current centre value v0, the step h and the right-hand side. */
double orc_point_update(const double *q, double v0, double h, double rhs)
{
    long ev = 0;
    return point_update(q, v0, h, rhs, &ev);
}

/* Eigenvalues (ascending) of a symmetric 3x3 matrix given row-major. */
void orc_sym3_eigenvalues(const double *Hrm, double *lam)
{
    double H[3][3];
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) H[a][b] = Hrm[3 * a + b];
    sym3_eigenvalues(H, lam);
}

/* det(D^2_h u) at every interior point (0 on the shell). */
void orc_discrete_ma(const double *u, double *out, int n, double h)
{
    memset(out, 0, sizeof(double) * (size_t)n * n * n);
    for (int k = 1; k <= n - 2; ++k)
        for (int j = 1; j <= n - 2; ++j)
            for (int i = 1; i <= n - 2; ++i)
                AT(out, n, i, j, k) = discrete_ma(u, n, h, i, j, k);
}

/* The discrete Hessian at every interior point, six values per point in the
 * order xx, yy, zz, xy, xz, yz (shell points zero).  out holds 6 n^3 doubles. */
void orc_discrete_hessian(const double *u, double *out, int n, double h)
{
    const size_t m = (size_t)n * n * n;
    memset(out, 0, sizeof(double) * 6 * m);
    for (int k = 1; k <= n - 2; ++k)
        for (int j = 1; j <= n - 2; ++j)
            for (int i = 1; i <= n - 2; ++i) {
                double q[6], H[3][3];
                neighbour_sums(u, n, i, j, k, q);
                hessian_with_centre(q, AT(u, n, i, j, k), h, H);
                const size_t p = (((size_t)k) * n + j) * n + i;
                out[0 * m + p] = H[0][0]; out[1 * m + p] = H[1][1]; out[2 * m + p] = H[2][2];
                out[3 * m + p] = H[0][1]; out[4 * m + p] = H[0][2]; out[5 * m + p] = H[1][2];
            }
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
