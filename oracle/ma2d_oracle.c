/*
 * ma2d_oracle.c -- plain FP64 CPU statement of the two-dimensional version of
 * the FAS multigrid method (Section 4.1 of Liu, Froese, Oberman, Xiao, "A
 * multigrid scheme for 3D Monge-Ampere equations", arXiv:1411.7018):
 *     u_xx u_yy - u_xy^2 = f > 0 on a square, u = g on the boundary,
 * Eq. (MA2D), on the 9-point centred stencil, with the nonlinear Gauss-Seidel
 * smoother whose local equation is a quadratic in the centre value (the
 * scheme the paper takes from its reference on 2D Gauss-Seidel).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the package's smoke check and
 * the benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or constant with the CUDA path.  Pinned by tests/test_oracle2d_pins.py
 * (closed forms, library root finders, brute force, Tables 1 and 2).
 *
 * Grid: x_i = i h, i = 0..N, h = len / N; a level stores n = N + 1 points per
 * side, boundary included, as n^2 doubles in [j][i] order (i fastest).
 *
 * Local equation.  With a = u(i+1,j) + u(i-1,j), b = u(i,j+1) + u(i,j-1) and
 * r = (u(i+1,j+1) - u(i-1,j+1) - u(i+1,j-1) + u(i-1,j-1)) / 4, the centred
 * differences give u_xx = (a - 2v)/h^2, u_yy = (b - 2v)/h^2, u_xy = r/h^2 for
 * centre value v, and Eq. (MA2D) at the point reads
 *     (a - 2v)(b - 2v) - r^2 = h^4 f,
 * a quadratic in v whose smaller root is the convex choice (Section 2):
 *     v = ((a + b) - sqrt((a - b)^2 + 4 r^2 + 4 h^4 f)) / 4.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define AT2(u, n, i, j) ((u)[((size_t)(j)) * (size_t)(n) + (size_t)(i)])

enum { O2_REDBLACK = 0, O2_LEXICOGRAPHIC = 1, O2_COLOUR4 = 2 };
enum { O2_HALF_WEIGHTING = 0, O2_FULL_WEIGHTING = 1 };
enum { O2_NORM_MAX = 0, O2_NORM_L2 = 1 };
enum { O2_APPROX_INJECTION = 0, O2_APPROX_WEIGHTED = 1 };
enum { O2_FMG_BILINEAR = 0, O2_FMG_CUBIC = 1 };

static void sums2(const double *u, int n, int i, int j, double *a, double *b, double *r)
{
    *a = AT2(u, n, i + 1, j) + AT2(u, n, i - 1, j);
    *b = AT2(u, n, i, j + 1) + AT2(u, n, i, j - 1);
    *r = 0.25 * ((AT2(u, n, i + 1, j + 1) - AT2(u, n, i - 1, j + 1)) -
                 (AT2(u, n, i + 1, j - 1) - AT2(u, n, i - 1, j - 1)));
}

/* The smaller root of (a - 2v)(b - 2v) - r^2 = h^4 rhs.  A negative
 * discriminant (possible only for rhs < 0, e.g. a coarse-grid right-hand
 * side) has no real root: the vertex v = (a + b)/4 is taken and counted. */
static double quad_root(double a, double b, double r, double h, double rhs, long *ev)
{
    const double h4 = h * h * h * h;
    double disc = (a - b) * (a - b) + 4.0 * r * r + 4.0 * h4 * rhs;
    if (disc < 0.0) {
        ++*ev;
        disc = 0.0;
    }
    return 0.25 * ((a + b) - sqrt(disc));
}

double o2_point_update(double a, double b, double r, double h, double rhs)
{
    long ev = 0;
    return quad_root(a, b, r, h, rhs, &ev);
}

/* S_h(u) = u_xx u_yy - u_xy^2 at interior point (i, j). */
static double discrete_ma2(const double *u, int n, double h, int i, int j)
{
    double a, b, r;
    sums2(u, n, i, j, &a, &b, &r);
    const double v = AT2(u, n, i, j);
    const double h2 = h * h;
    return ((a - 2.0 * v) / h2) * ((b - 2.0 * v) / h2) - (r / h2) * (r / h2);
}

/* One Gauss-Seidel sweep over the interior.  Red-black: the points with
 * i + j even, then those with i + j odd, each colour updated at once from the
 * values before its update (diagonal neighbours share the colour); the
 * lexicographic order updates in place point by point; four colours
 * (i & 1) | (j & 1) << 1 separate all nine stencil points, so each colour's
 * in-place update is order-free.  Returns the count of negative
 * discriminants. */
long o2_gs_sweep(double *u, const double *rhs, int n, double h, int ordering)
{
    long ev = 0;
    if (ordering == O2_LEXICOGRAPHIC) {
        for (int j = 1; j <= n - 2; ++j)
            for (int i = 1; i <= n - 2; ++i) {
                double a, b, r;
                sums2(u, n, i, j, &a, &b, &r);
                AT2(u, n, i, j) = quad_root(a, b, r, h, AT2(rhs, n, i, j), &ev);
            }
        return ev;
    }
    if (ordering == O2_COLOUR4) {
        for (int c = 0; c < 4; ++c)
            for (int j = 1; j <= n - 2; ++j)
                for (int i = 1; i <= n - 2; ++i) {
                    if (((i & 1) | ((j & 1) << 1)) != c) continue;
                    double a, b, r;
                    sums2(u, n, i, j, &a, &b, &r);
                    AT2(u, n, i, j) = quad_root(a, b, r, h, AT2(rhs, n, i, j), &ev);
                }
        return ev;
    }
    double *nw = (double *)malloc(sizeof(double) * (size_t)n * n);
    for (int colour = 0; colour < 2; ++colour) {
        for (int j = 1; j <= n - 2; ++j)
            for (int i = 1; i <= n - 2; ++i) {
                if (((i + j) & 1) != colour) continue;
                double a, b, r;
                sums2(u, n, i, j, &a, &b, &r);
                AT2(nw, n, i, j) = quad_root(a, b, r, h, AT2(rhs, n, i, j), &ev);
            }
        for (int j = 1; j <= n - 2; ++j)
            for (int i = 1; i <= n - 2; ++i)
                if (((i + j) & 1) == colour) AT2(u, n, i, j) = AT2(nw, n, i, j);
    }
    free(nw);
    return ev;
}

void o2_residual(const double *u, const double *rhs, double *res, int n, double h)
{
    memset(res, 0, sizeof(double) * (size_t)n * n);
    for (int j = 1; j <= n - 2; ++j)
        for (int i = 1; i <= n - 2; ++i) AT2(res, n, i, j) = AT2(rhs, n, i, j) - discrete_ma2(u, n, h, i, j);
}

/* Max norm, or discrete L2 sqrt(h^2 sum v^2), over the interior. */
double o2_norm(const double *v, int n, double h, int kind)
{
    double m = 0.0, s = 0.0;
    for (int j = 1; j <= n - 2; ++j)
        for (int i = 1; i <= n - 2; ++i) {
            const double x = AT2(v, n, i, j);
            if (fabs(x) > m) m = fabs(x);
            s += x * x;
        }
    return kind == O2_NORM_MAX ? m : sqrt(h * h * s);
}

/* Restriction at fine point (2I, 2J): half weighting (4 centre + 4 faces)/8,
 * the 2D form of the 3D half weighting of Section 3, or full weighting
 * (1 2 1; 2 4 2; 1 2 1)/16. */
static double restrict_at2(const double *v, int nf, int i, int j, int kind)
{
    if (kind == O2_HALF_WEIGHTING)
        return (4.0 * AT2(v, nf, i, j) + AT2(v, nf, i + 1, j) + AT2(v, nf, i - 1, j) + AT2(v, nf, i, j + 1) +
                AT2(v, nf, i, j - 1)) / 8.0;
    double s = 0.0;
    for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di) {
            const double w = (di == 0 ? 2.0 : 1.0) * (dj == 0 ? 2.0 : 1.0);
            s += w * AT2(v, nf, i + di, j + dj);
        }
    return s / 16.0;
}

void o2_restrict_residual(const double *rf, int nf, double *rc, int nc, int kind)
{
    memset(rc, 0, sizeof(double) * (size_t)nc * nc);
    for (int J = 1; J <= nc - 2; ++J)
        for (int I = 1; I <= nc - 2; ++I) AT2(rc, nc, I, J) = restrict_at2(rf, nf, 2 * I, 2 * J, kind);
}

void o2_inject(const double *vf, int nf, double *vc, int nc)
{
    for (int J = 0; J < nc; ++J)
        for (int I = 0; I < nc; ++I) AT2(vc, nc, I, J) = AT2(vf, nf, 2 * I, 2 * J);
}

/* Approximation restriction of u: injection, or the residual's weighting
 * inside and injection on the boundary (the same reading as in 3D). */
void o2_restrict_solution(const double *uf, int nf, double *uc, int nc, int approx, int kind)
{
    o2_inject(uf, nf, uc, nc);
    if (approx == O2_APPROX_INJECTION) return;
    for (int J = 1; J <= nc - 2; ++J)
        for (int I = 1; I <= nc - 2; ++I) AT2(uc, nc, I, J) = restrict_at2(uf, nf, 2 * I, 2 * J, kind);
}

/* Bilinear interpolation at fine point (i, j) from coarse values d. */
static double bilinear_at(const double *d, int nc, int i, int j)
{
    const int I = i / 2, J = j / 2, oi = i & 1, oj = j & 1;
    double s = 0.0;
    for (int b = 0; b <= oj; ++b)
        for (int a = 0; a <= oi; ++a) s += AT2(d, nc, I + a, J + b);
    return s / (double)(1 << (oi + oj));
}

/* Algorithm 1 steps 7-8: u_h += I_H^h (u_H - w_H) on the fine interior. */
void o2_prolong_add(const double *uc, const double *wc, int nc, double *uf, int nf)
{
    double *d = (double *)malloc(sizeof(double) * (size_t)nc * nc);
    for (size_t p = 0; p < (size_t)nc * nc; ++p) d[p] = uc[p] - wc[p];
    for (int j = 1; j <= nf - 2; ++j)
        for (int i = 1; i <= nf - 2; ++i) AT2(uf, nf, i, j) += bilinear_at(d, nc, i, j);
    free(d);
}

/* Cubic interpolation along one axis: the same rule as in 3D (four
 * neighbouring coarse points, one-sided next to the ends, quadratic on a
 * 3-point grid). */
static int cubic_stencil2(int i, int nc, int idx[4], double w[4])
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

/* Algorithm 2 step 4: fine interior from the coarse solution, bilinear or
 * bicubic (tensor product of the one-axis stencils); the boundary keeps g. */
void o2_interpolate(const double *uc, int nc, double *uf, int nf, int cubic)
{
    for (int j = 1; j <= nf - 2; ++j)
        for (int i = 1; i <= nf - 2; ++i) {
            if (!cubic) { AT2(uf, nf, i, j) = bilinear_at(uc, nc, i, j); continue; }
            int ix[4], iy[4];
            double wx[4], wy[4];
            const int nx = cubic_stencil2(i, nc, ix, wx), ny = cubic_stencil2(j, nc, iy, wy);
            double s = 0.0;
            for (int b = 0; b < ny; ++b)
                for (int a = 0; a < nx; ++a) s += wy[b] * wx[a] * AT2(uc, nc, ix[a], iy[b]);
            AT2(uf, nf, i, j) = s;
        }
}

/* Algorithm 1 step 5: b_H = S_H(w_H) + r_H on the coarse interior. */
void o2_coarse_rhs(const double *wc, const double *rc, double *bc, int nc, double H)
{
    memset(bc, 0, sizeof(double) * (size_t)nc * nc);
    for (int J = 1; J <= nc - 2; ++J)
        for (int I = 1; I <= nc - 2; ++I) AT2(bc, nc, I, J) = discrete_ma2(wc, nc, H, I, J) + AT2(rc, nc, I, J);
}

typedef struct {
    int nu1, nu2, coarsest_n, restrict_kind, coarse_sweeps, ordering, approx_restrict, fmg_interp;
} o2_params;

typedef struct { int n; double h; double *u, *rhs, *r, *w; } o2_level;
typedef struct { int nlev; o2_level lev[24]; o2_params p; long events; } o2_hier;

static int hier2_init(o2_hier *H, int n, double h, const o2_params *p)
{
    memset(H, 0, sizeof *H);
    H->p = *p;
    int m = n;
    double hh = h;
    while (1) {
        if (H->nlev >= 24) return -1;
        o2_level *L = &H->lev[H->nlev++];
        L->n = m; L->h = hh;
        const size_t sz = sizeof(double) * (size_t)m * m;
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

static void hier2_free(o2_hier *H)
{
    for (int l = 0; l < H->nlev; ++l) {
        free(H->lev[l].u); free(H->lev[l].rhs); free(H->lev[l].r); free(H->lev[l].w);
    }
}

static void coarsest2(o2_hier *H, o2_level *L)
{
    if (H->p.coarse_sweeps > 0) {
        for (int s = 0; s < H->p.coarse_sweeps; ++s) H->events += o2_gs_sweep(L->u, L->rhs, L->n, L->h, H->p.ordering);
        return;
    }
    const size_t m = (size_t)L->n * L->n;
    double *prev = (double *)malloc(sizeof(double) * m);
    for (int s = 0; s < 100; ++s) {
        memcpy(prev, L->u, sizeof(double) * m);
        H->events += o2_gs_sweep(L->u, L->rhs, L->n, L->h, H->p.ordering);
        double du = 0.0, um = 0.0;
        for (size_t q = 0; q < m; ++q) {
            if (fabs(L->u[q] - prev[q]) > du) du = fabs(L->u[q] - prev[q]);
            if (fabs(L->u[q]) > um) um = fabs(L->u[q]);
        }
        if (du <= 1e-14 * um) break;
    }
    free(prev);
}

/* Algorithm 1 in 2D. */
static void vcycle2(o2_hier *H, int l)
{
    o2_level *F = &H->lev[l];
    if (l == H->nlev - 1) { coarsest2(H, F); return; }
    o2_level *C = &H->lev[l + 1];
    for (int s = 0; s < H->p.nu1; ++s) H->events += o2_gs_sweep(F->u, F->rhs, F->n, F->h, H->p.ordering);
    o2_residual(F->u, F->rhs, F->r, F->n, F->h);
    o2_restrict_residual(F->r, F->n, C->r, C->n, H->p.restrict_kind);
    o2_restrict_solution(F->u, F->n, C->w, C->n, H->p.approx_restrict, H->p.restrict_kind);
    memcpy(C->u, C->w, sizeof(double) * (size_t)C->n * C->n);
    o2_coarse_rhs(C->w, C->r, C->rhs, C->n, C->h);
    vcycle2(H, l + 1);
    o2_prolong_add(C->u, C->w, C->n, F->u, F->n);
    for (int s = 0; s < H->p.nu2; ++s) H->events += o2_gs_sweep(F->u, F->rhs, F->n, F->h, H->p.ordering);
}

/* Algorithm 2 in 2D. */
static void fmg2(o2_hier *H, int l)
{
    o2_level *F = &H->lev[l];
    if (l == H->nlev - 1) {
        for (int j = 1; j <= F->n - 2; ++j)
            for (int i = 1; i <= F->n - 2; ++i) AT2(F->u, F->n, i, j) = 0.0;
        coarsest2(H, F);
        return;
    }
    o2_level *C = &H->lev[l + 1];
    o2_inject(F->rhs, F->n, C->rhs, C->n);
    o2_inject(F->u, F->n, C->u, C->n);
    fmg2(H, l + 1);
    o2_interpolate(C->u, C->n, F->u, F->n, H->p.fmg_interp == O2_FMG_CUBIC);
    vcycle2(H, l);
}

/* FMG (init = 1) then V-cycles until ||f - S_h u|| / ref <= tol; ref_kind 0:
 * ||f||, 1: the residual norm of the initial iterate (the zero interior FMG
 * starts from).  res_hist[0..cycles] as in the 3D oracle.  Returns cycles, or
 * -1 for a grid size that does not coarsen to the coarsest grid. */
int o2_solve(double *u, const double *f, int n, double h, const o2_params *p, double tol, int norm, int max_cycles,
             int init, int ref_kind, double *res_hist, long *events)
{
    o2_hier H;
    if (hier2_init(&H, n, h, p) != 0) { hier2_free(&H); return -1; }
    o2_level *F = &H.lev[0];
    memcpy(F->u, u, sizeof(double) * (size_t)n * n);
    memcpy(F->rhs, f, sizeof(double) * (size_t)n * n);
    double ref = o2_norm(f, n, h, norm);
    if (ref_kind == 1) {
        if (init)
            for (int j = 1; j <= n - 2; ++j)
                for (int i = 1; i <= n - 2; ++i) AT2(F->u, n, i, j) = 0.0;
        o2_residual(F->u, F->rhs, F->r, n, h);
        ref = o2_norm(F->r, n, h, norm);
    }
    if (init) fmg2(&H, 0);
    o2_residual(F->u, F->rhs, F->r, n, h);
    double rel = o2_norm(F->r, n, h, norm) / ref;
    if (res_hist) res_hist[0] = rel;
    int c = 0;
    while (rel > tol && c < max_cycles) {
        vcycle2(&H, 0);
        ++c;
        o2_residual(F->u, F->rhs, F->r, n, h);
        rel = o2_norm(F->r, n, h, norm) / ref;
        if (res_hist) res_hist[c] = rel;
    }
    memcpy(u, F->u, sizeof(double) * (size_t)n * n);
    if (events) *events = H.events;
    hier2_free(&H);
    return c;
}

/* S_h(u) on the interior (0 on the boundary), for the pins. */
void o2_discrete_ma(const double *u, int n, double h, double *out)
{
    memset(out, 0, sizeof(double) * (size_t)n * n);
    for (int j = 1; j <= n - 2; ++j)
        for (int i = 1; i <= n - 2; ++i) AT2(out, n, i, j) = discrete_ma2(u, n, h, i, j);
}
