/*
 * ma2d.h -- C ABI of the two-dimensional version of the FAS multigrid method
 * for the Monge-Ampere equation (Eq. MA2D, Section 4.1 of Liu, Froese,
 * Oberman, Xiao, "A multigrid scheme for 3D Monge-Ampere equations"):
 *     u_xx u_yy - u_xy^2 = f > 0 in a square, u = g on its boundary, u convex,
 * on the 9-point centred stencil.  The local equation of the Gauss-Seidel
 * smoother is a quadratic in the centre value, whose smaller root is the
 * convex choice (Section 2).
 *
 * Conventions as in ma.h: n = N + 1 points per side (boundary included), h =
 * len / N, grids are n^2 doubles in [j][i] order (i fastest) in device
 * memory; calls return ma_status and never throw; the hierarchy's memory is a
 * caller-owned device workspace; a hierarchy is bound to one stream and is
 * not thread-safe.  Hierarchy calls require n = 2^L (coarsest_n - 1) + 1.
 */
#ifndef MA2D_H
#define MA2D_H

#include "ma.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Smoother ordering: red-black (the points with i + j even, then the odd
 * ones, each colour updated at once from the values before its update -- the
 * diagonal neighbours of the 9-point stencil share a colour; Table 1), or four
 * colours (i & 1) | (j & 1) << 1, which separate all nine stencil points, so
 * each colour updates in place. */
enum { MA2D_REDBLACK = 0, MA2D_COLOUR4 = 2 };

typedef struct ma2d_hierarchy ma2d_hierarchy;

typedef struct {
    int n;               /* points per side incl. boundary                              */
    double len;          /* square edge; h = len / (n - 1)                              */
    int nu1, nu2;        /* pre/post smoothing sweeps (Section 4: 2, 2)                 */
    int coarsest_n;      /* 3 (h0 = 1/2, one unknown), 5, 9 or 17                        */
    int restrict_kind;   /* MA_HALF_WEIGHTING ((4 centre + 4 faces)/8) | MA_FULL_WEIGHTING
                            ((1 2 1; 2 4 2; 1 2 1)/16)                                   */
    int approx_restrict; /* MA_APPROX_INJECTION | MA_APPROX_WEIGHTED (as in ma.h)         */
    int coarse_sweeps;   /* > 0: that many sweeps on the coarsest grid; 0: until
                            max|du| <= 1e-14 max|u| (at most 100)                       */
    int ordering;        /* MA2D_REDBLACK | MA2D_COLOUR4                                */
    int fmg_interp;      /* MA_FMG_TRILINEAR (bilinear in 2D) | MA_FMG_CUBIC (bicubic)    */
} ma2d_desc;

/* Bytes of device workspace a hierarchy needs.  Host only. */
ma_status ma2d_hierarchy_footprint(const ma2d_desc *desc, size_t *bytes);

/* Build a hierarchy in the caller's workspace (>= footprint bytes, 256-byte
 * aligned; the caller keeps it alive until ma2d_destroy_hierarchy). */
ma_status ma2d_create_hierarchy(const ma2d_desc *desc, void *dev_workspace, size_t bytes, ma_stream_t stream,
                                ma2d_hierarchy **out);

/* f (read on the interior; must be finite and > 0 there) and g (boundary
 * values; its interior is the initial iterate for MA_INIT_KEEP), n^2 each,
 * copied in.  MA_ERR_INVALID_ARG if f is not positive and finite inside. */
ma_status ma2d_set_rhs_bc(ma2d_hierarchy *H, const double *f_dev, const double *g_dev);

/* ncycles V-cycles (Algorithm 1 in 2D) from the current iterate. */
ma_status ma2d_vcycle(ma2d_hierarchy *H, int ncycles);

/* Algorithm 2 (or the chosen initial iterate) followed by V-cycles until the
 * stopping rule of opts holds (same rule and result fields as ma_solve; the
 * discrete L2 norm is sqrt(h^2 sum r^2)).  Blocks on the stream. */
ma_status ma2d_solve(ma2d_hierarchy *H, const ma_solve_opts *opts, ma_solve_result *res);

/* Copy the n^2 iterate out (async on the stream). */
ma_status ma2d_get_solution(const ma2d_hierarchy *H, double *u_dev);

ma_status ma2d_destroy_hierarchy(ma2d_hierarchy *H);

/* ---- single steps on caller arrays ------------------------------------- */

/* nsweeps Gauss-Seidel sweeps in place on u (shell untouched).  Red-black
 * needs scratch_dev of n^2 doubles (the second buffer); MA2D_COLOUR4 takes
 * null.  events_dev (optional) counts negative discriminants (no real root;
 * the vertex (a + b)/4 is taken). */
ma_status ma2d_smooth(double *u_dev, const double *rhs_dev, int n, double h, int nsweeps, int ordering,
                      double *scratch_dev, unsigned long long *events_dev, ma_stream_t stream);

/* r = rhs - (u_xx u_yy - u_xy^2) on the interior, 0 on the boundary. */
ma_status ma2d_residual(const double *u_dev, const double *rhs_dev, double *r_dev, int n, double h,
                        ma_stream_t stream);

/* Restriction of a fine residual (interior; coarse boundary 0), kind as in
 * ma2d_desc; nc = (nf + 1) / 2. */
ma_status ma2d_restrict_residual(const double *rf_dev, int nf, double *rc_dev, int kind, ma_stream_t stream);

/* uf += bilinear(uc - wc) on the fine interior (Algorithm 1 steps 7-8). */
ma_status ma2d_prolong_add(const double *uc_dev, const double *wc_dev, int nc, double *uf_dev, ma_stream_t stream);

/* Fine interior := bilinear (cubic = 0) or bicubic interpolation of uc. */
ma_status ma2d_interpolate(const double *uc_dev, int nc, double *uf_dev, int cubic, ma_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif
