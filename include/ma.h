/*
 * ma.h -- C ABI of libma, a GB300 (sm_103a) FAS multigrid solver for the 3D
 * elliptic Monge-Ampere equation
 *
 *     det(D^2 u) = f > 0 in the cube,   u = g on its boundary,   u convex
 *
 * (Liu, Froese, Oberman, Xiao, "A multigrid scheme for 3D Monge-Ampere
 * equations", Section 1, Eqs. (MA3D) and (DBC)).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Grids (Section 2): n = N + 1 points per side including the boundary
 *    shell, h = len / N, point (i, j, k) at x0 + (i h, j h, k h).  A grid
 *    array holds n^3 doubles in [k][j][i] order (i fastest), shell included.
 *    Hierarchy calls require n = 2^L (coarsest_n - 1) + 1.
 *  - Pointers named *_dev are device pointers (cudaMalloc'd or torch CUDA
 *    tensors) on the current device; *_host are host pointers.  The library
 *    never frees or keeps caller pointers beyond the call unless stated.
 *  - Every call is asynchronous on the given stream unless it says it blocks.
 *    A hierarchy is bound to the stream it was created with and is not
 *    thread-safe.
 *  - Every call returns ma_status; on failure ma_last_error_string() gives a
 *    one-line reason (thread-local).  No C++ exception crosses the ABI.
 *    MA_ERR_INVALID_ARG: a null pointer, a bad size or option, or a
 *    workspace smaller than the footprint.  MA_ERR_CUDA: a CUDA runtime error
 *    (the message names it).  MA_ERR_NOT_CONVERGED / MA_ERR_NONFINITE: see
 *    ma_solve.
 *  - The library allocates no device memory: every device buffer a hierarchy
 *    uses lives in the caller's workspace.  It allocates a few bytes of pinned
 *    host memory per hierarchy for norm read-back.
 */
#ifndef MA_H
#define MA_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MA_OK = 0,
    MA_ERR_INVALID_ARG = 1,
    MA_ERR_OOM = 2,
    MA_ERR_CUDA = 3,
    MA_ERR_NOT_CONVERGED = 4,
    MA_ERR_NONFINITE = 5
} ma_status;

/* Residual restriction I_h^H (Section 3): the printed 7-point half
 * weighting, or 27-point full weighting (weights 8/4/2/1 over 64). */
enum { MA_HALF_WEIGHTING = 0, MA_FULL_WEIGHTING = 1 };
/* Approximation restriction (Algorithm 1 step 4): straight injection
 * (Section 3), or the residual's own weighting applied to u.  The coarse
 * iterate u_H starts equal to w_H in both cases. */
enum { MA_APPROX_INJECTION = 0, MA_APPROX_WEIGHTED = 1 };
/* Arithmetic: everything in FP64; FP32 correction cycles under an FP64
 * fine-grid residual and update (defect correction); or everything in FP32
 * (the FP32 cycles on the solution itself, stopping on the FP32 residual): a
 * throughput mode whose accuracy is limited by FP32 round-off of the second
 * differences, ~eps_32 |u| / h^2 in the Hessian, which grows with N. */
enum { MA_FP64 = 0, MA_MIXED = 1, MA_FP32 = 2 };
/* Norms over the fine interior: max, or discrete L2 sqrt(h^3 sum v^2)
 * (stopping rule of Section 4). */
enum { MA_NORM_MAX = 0, MA_NORM_L2 = 1 };
/* Initial iterate for ma_solve: one FMG pass (Algorithm 2), the Dirichlet
 * data with a zero interior, or the current iterate. */
enum { MA_INIT_FMG = 0, MA_INIT_ZERO = 1, MA_INIT_KEEP = 2 };
/* Interpolation of the FMG pass (Algorithm 2 step 4): trilinear, or the
 * tricubic interpolation Section 3 recommends so that one FMG pass reaches
 * discretisation accuracy (one-sided cubics next to the boundary). */
enum { MA_FMG_TRILINEAR = 0, MA_FMG_CUBIC = 1 };
/* Reference of the stopping rule: none (absolute), ||f|| over the interior,
 * or the residual norm of the initial iterate (Section 4's relative residual
 * ||r^l|| / ||r^0||; with MA_INIT_FMG or MA_INIT_ZERO the initial iterate is
 * the Dirichlet data with a zero interior, which FMG starts from). */
enum { MA_REL_NONE = 0, MA_REL_RHS = 1, MA_REL_INITIAL = 2 };

/* A cudaStream_t (NULL = the legacy default stream). */
typedef void *ma_stream_t;

typedef struct ma_hierarchy ma_hierarchy;

/* Problem and cycle description (Sections 2-4). */
typedef struct {
    int n;               /* points per side incl. boundary; n = 2^L (coarsest_n-1) + 1 */
    double x0[3];        /* cube origin (informational; f and g are given on the grid) */
    double len;          /* cube edge; h = len / (n - 1)                               */
    int nu1, nu2;        /* pre/post smoothing sweeps (Section 4 uses 2, 2)            */
    int coarsest_n;      /* 3 (Section 4, h0 = 1/2: one unknown, so one sweep solves it
                            exactly) or 5, 9, 17                                       */
    int restrict_kind;   /* MA_HALF_WEIGHTING | MA_FULL_WEIGHTING                      */
    int approx_restrict; /* MA_APPROX_INJECTION | MA_APPROX_WEIGHTED                   */
    int precision;       /* MA_FP64 | MA_MIXED | MA_FP32.  MA_MIXED also runs each FMG
                            level below the finest as an outer iteration (FP64
                            residual, 2 FP32 correction cycles, FP64 update) in
                            place of an FP64 V-cycle                                    */
    int coarse_sweeps;   /* > 0: that many sweeps on the coarsest grid (Section 4 uses
                            1); 0: sweep until max|du| <= 1e-14 max|u| (cap 100)        */
    int inner_cycles;    /* MA_MIXED: FP32 correction V-cycles per FP64 residual and
                            update (0: the default, 3; 2 is faster for single solves
                            from 129^3 up); ignored in MA_FP64                          */
    int fmg_interp;      /* MA_FMG_TRILINEAR | MA_FMG_CUBIC (recommended: its start
                            leaves a ~1000x smaller residual)                           */
} ma_hier_desc;

/* Stopping rule for ma_solve.  Converged when ||f - det(D^2_h u)|| <= tol *
 * reference (MA_REL_*), norm over the fine interior, evaluated in FP64. */
typedef struct {
    double tol;
    int norm;            /* MA_NORM_MAX | MA_NORM_L2                        */
    int relative;        /* MA_REL_NONE | MA_REL_RHS | MA_REL_INITIAL         */
    int max_cycles;      /* V-cycles (outer iterations in MA_MIXED) at most    */
    int init;            /* MA_INIT_FMG | MA_INIT_ZERO | MA_INIT_KEEP          */
} ma_solve_opts;

typedef struct {
    int cycles;                       /* V-cycles run after the initial iterate        */
    double res0;                      /* residual norm after the initialisation (FMG)
                                         over the reference, as res                     */
    double res;                       /* final residual norm (same scaling as tol)      */
    int status;                       /* the ma_status ma_solve returned                */
    int floor_reached;                /* 1 if stopped because the residual stagnated at
                                         the round-off floor above tol                  */
    long long nonconvex_root_events;  /* point solves whose right-hand side was <= 0     */
} ma_solve_result;

/* ---- hierarchy (the method as a whole) ---------------------------------- */

/* Bytes of device workspace a hierarchy with this description needs
 * (all level grids and reduction scratch).  Host only; no CUDA call. */
ma_status ma_hierarchy_footprint(const ma_hier_desc *desc, size_t *bytes);

/* Build a hierarchy inside the caller's device workspace (>= footprint
 * bytes, 256-byte aligned).  The caller keeps ownership of the workspace and
 * must keep it alive until ma_destroy_hierarchy.  Fields are not initialised:
 * call ma_set_rhs_bc next. */
ma_status ma_create_hierarchy(const ma_hier_desc *desc, void *dev_workspace, size_t bytes,
                              ma_stream_t stream, ma_hierarchy **out);

/* Copy the data of Eqs. (MA3D)/(DBC) in: f_dev is read on the interior
 * (must be finite and > 0 there), g_dev on the boundary shell; the interior of
 * g_dev is taken as the initial iterate (used by MA_INIT_KEEP).  Both are n^3
 * doubles; they are copied, so the caller may free them after the stream
 * reaches this point.  Checks f > 0 on the device and blocks for that check. */
ma_status ma_set_rhs_bc(ma_hierarchy *h, const double *f_dev, const double *g_dev);

/* ma_set_rhs_bc with f and g in HOST memory (n^3 doubles each, [k][j][i]),
 * for callers whose data live on the host: both are copied to the device on
 * the hierarchy's stream (into the fine level's scratch fields), then checked
 * and moved into place as above.  Blocks for the check, so the host buffers
 * may be reused on return.  Page-locked (pinned) buffers make the copies
 * asynchronous DMA; pageable ones work but are staged by the driver. */
ma_status ma_set_rhs_bc_host(ma_hierarchy *h, const double *f_host, const double *g_host);

/* ncycles FAS V-cycles (Algorithm 1) on the finest level.  Asynchronous. */
ma_status ma_vcycle(ma_hierarchy *h, int ncycles);

/* Solve to tolerance: the chosen initial iterate, then V-cycles until the
 * stopping rule holds (MA_OK), max_cycles is reached, or the residual
 * stagnates above tol (two cycles in a row each reducing it by less than
 * 20 %: the round-off floor; result->floor_reached = 1).  Both of the latter
 * return MA_ERR_NOT_CONVERGED; a NaN/Inf residual returns MA_ERR_NONFINITE.
 * Blocks on the stream (one small read-back per cycle); result is filled in
 * every case. */
ma_status ma_solve(ma_hierarchy *h, const ma_solve_opts *opts, ma_solve_result *result);

/* The same solve without blocking, for callers that interleave many solves
 * (batching, serving).  ma_solve_begin queues the initial iterate and its
 * residual norm; each ma_solve_advance call returns at once: if the norms of
 * the last queued step have reached the host it applies the stopping rule
 * and, unless the solve is finished, queues the next cycle (one CUDA graph
 * launch and one 40-byte read-back on the hierarchy's stream); *done is set
 * to 1 when the solve has finished.  ma_solve_get_result then returns the
 * result and its status, as ma_solve would.  ma_solve is begin + advance
 * (waiting on the read-back) + get_result. */
ma_status ma_solve_begin(ma_hierarchy *h, const ma_solve_opts *opts);
ma_status ma_solve_advance(ma_hierarchy *h, int *done);
ma_status ma_solve_get_result(const ma_hierarchy *h, ma_solve_result *result);

/* Batched solve: every hierarchy in hs solves with opts, their cycles
 * overlapping on the GPU (each hierarchy runs on the stream it was created
 * with, so give them distinct streams).  Blocks until all have finished;
 * results[b] is filled for every b.  Returns MA_OK if all converged, else the
 * first non-MA_OK status. */
ma_status ma_batch_solve(ma_hierarchy *const *hs, int count, const ma_solve_opts *opts, ma_solve_result *results);

/* Shared per-level batch.  Binds `count` MA_MIXED hierarchies of any sizes
 * (n <= 1025; equal nu1, nu2, restrict_kind, approx_restrict, coarse_sweeps,
 * inner_cycles, coarsest_n, fmg_interp; one device; each at most once) so
 * that their solves share
 * kernel launches.  ma_batch_run starts every hierarchy as ma_solve_begin
 * does (FMG and the first outer iteration, each on its own stream; or as
 * batched launches, ma_set_batch_start), then runs the outer iterations
 * (Algorithm 1 V-cycles on the correction, the FP64 update and residual) of
 * all hierarchies still iterating as CUDA graphs, one per group of
 * hierarchies (ma_set_batch_groups), the first on `stream`.  Each group
 * advances on its own: its first outer iteration once its hierarchies'
 * starts are done, each next one once its own norms are back.  Each graph
 * kernel covers one level depth of every
 * hierarchy (its blocks find their hierarchy in a job table kept in the
 * workspace), the levels <= the fused-tail bound of every hierarchy take one
 * launch, and a hierarchy that has met the stopping rule is skipped.  Each
 * hierarchy executes the per-point operations of its own solve, so
 * results[b] and its solution are those ma_solve gives for it alone.
 *
 * ma_batch_footprint: device bytes the batch needs (job tables, flags and
 * norms; a few KB per hierarchy).  ma_create_batch: the caller owns the
 * 256-byte-aligned workspace, and the hierarchies, which must outlive the
 * batch and not be used by other calls while ma_batch_run runs; it reads the
 * fused-tail setting (ma_set_corr_tail) once, here.  MA_ERR_INVALID_ARG for a
 * null or repeated hierarchy, mismatched settings or a small workspace.
 * ma_batch_run blocks until every solve has finished; returns MA_OK if all
 * converged, else the first non-MA_OK status (results[b] is filled for every
 * b).  Later work on a hierarchy's own stream follows the batch's. */
typedef struct ma_batch ma_batch;
ma_status ma_batch_footprint(ma_hierarchy *const *hs, int count, size_t *bytes);
ma_status ma_create_batch(ma_hierarchy *const *hs, int count, void *dev_workspace, size_t bytes, ma_stream_t stream,
                          ma_batch **out);
ma_status ma_batch_run(ma_batch *b, const ma_solve_opts *opts, ma_solve_result *results);
ma_status ma_destroy_batch(ma_batch *b);

/* Batches split their hierarchies (by decreasing size, dealt in turn) into
 * min(count, groups) groups, each replayed as its own graph on its own stream
 * in every outer iteration, so that the groups' kernels overlap (an FP64
 * residual of one beside the FP32 sweeps of another).  1..16, default 2;
 * read by ma_batch_footprint and ma_create_batch.  The results do not
 * depend on it. */
ma_status ma_set_batch_groups(int groups);

/* How ma_batch_run starts its hierarchies: 0 (the default) runs each
 * hierarchy's own start graph on its own stream, concurrently; 1 runs the
 * start (the norms of f, FMG, the first outer iteration) as batched launches
 * too (with MA_INIT_FMG and a reference other than MA_REL_INITIAL).  With
 * FP64 V-cycles on the FMG levels the batched start measured ~4 % slower on
 * 64 mixed hierarchies of {33, 65, 129}^3.  The results do not depend on
 * it. */
ma_status ma_set_batch_start(int batched);

/* Norm of the fine-level FP64 residual f - det(D^2_h u) of the current
 * iterate (Algorithm 1 step 3; Section 4 norms).  Blocks on the stream. */
ma_status ma_residual_norm(ma_hierarchy *h, int norm, double *out);

/* Copy the current fine-level iterate (n^3 doubles, shell included) to u_dev.
 * Asynchronous. */
ma_status ma_get_solution(ma_hierarchy *h, double *u_dev);

/* Copy the current fine-level iterate (n^3 doubles, shell included) to HOST
 * memory u_host.  Blocks until the copy has landed (pinned memory makes it a
 * direct DMA). */
ma_status ma_get_solution_host(ma_hierarchy *h, double *u_host);

/* Replace the current fine-level iterate (shell included) from u_dev
 * (checkpoint/restart).  Asynchronous. */
ma_status ma_set_solution(ma_hierarchy *h, const double *u_dev);

/* Grid size, level count and workspace bytes of a hierarchy. */
ma_status ma_hierarchy_info(const ma_hierarchy *h, int *n, int *levels, size_t *bytes);

/* Release the host-side state; the caller frees the workspace afterwards.
 * Synchronises the hierarchy's stream first. */
ma_status ma_destroy_hierarchy(ma_hierarchy *h);

/* Thread-local text of the last failure ("" if none). */
const char *ma_last_error_string(void);

/* Diagnostics: the number of kernel launches this library has issued in this
 * process so far (all devices, all hierarchies).  Host only. */
ma_status ma_kernel_launch_count(unsigned long long *out);

/* Diagnostics: the FP64 fused-multiply-add rate of the current device,
 * measured (thread-level DFMA operations per second, one DFMA = one
 * operation), by independent chains of DFMAs on every SM timed with CUDA
 * events on the stream.  No counterpart in the paper: the FP64 kernels of
 * this library are bound by the FP64 pipe, and this is their peak.  Blocks
 * on the stream (~a millisecond). */
ma_status ma_probe_fp64_rate(double *ops_per_s, ma_stream_t stream);

/* Diagnostics: the cost per phase of a chain of `phases` dependent phases on
 * the current device, three ways, in microseconds per phase (best of 5 timed
 * runs after 2 untimed ones, CUDA events).  A phase computes
 * b[i] = a[i] * 1.0001 + 1 for i < n, and the next phase reads what it wrote
 * (a and b swap).  No counterpart in the paper: a multigrid cycle is such a
 * chain (colour sweeps, residual, transfers on every level), run here as
 * CUDA graphs, and this probe measures the persistent-kernel alternative.
 *    out_us[0]: a CUDA graph of `phases` launches, one element per thread;
 *    out_us[1]: the same graph with blocks_per_sm x (SM count) blocks, each
 *               striding over the elements;
 *    out_us[2]: one cooperative launch of that grid running all phases, a
 *               grid-wide barrier between consecutive ones.
 * out_us[2] - out_us[1] is the cost of a grid barrier over a launch edge.
 * a_dev, b_dev: n floats each on the device, sync_dev: 3 unsigned ints on the
 * device, all owned by the caller and overwritten.  n in [1, 2^40], phases in
 * [2, 4096], blocks_per_sm in [1, the resident limit of 128-thread blocks];
 * MA_ERR_INVALID_ARG otherwise or where the device has no cooperative launch.
 * Each barrier's wait is bounded (about a second); if one gives up, the
 * kernel ends and the call returns MA_ERR_CUDA.  Blocks until done. */
ma_status ma_probe_phase_chain(float *a_dev, float *b_dev, size_t n, int phases, int blocks_per_sm,
                               unsigned *sync_dev, double *out_us, ma_stream_t stream);

/* ---- single steps on raw device grids (each row of the V-cycle) ----------
 * These run exactly the kernels a hierarchy runs, on caller arrays of one
 * level (n^3 doubles, [k][j][i]).  n must be odd and >= 3.  All are
 * asynchronous on the given stream. */

/* nsweeps nonlinear Gauss-Seidel sweeps (Section 2, Eq. realroots) in place
 * on u_dev with right-hand side rhs_dev (f on the finest level, b_H on coarse
 * ones): eight colours c = (i&1)|(j&1)<<1|(k&1)<<2 in ascending order; each
 * point takes the smallest real root of its local cubic.  The shell is not
 * written.  If events_dev is not NULL, the count of point solves whose
 * right-hand side was <= 0 is added to *events_dev (one unsigned 64-bit
 * integer on the device). */
ma_status ma_smooth(double *u_dev, const double *rhs_dev, int n, double h, int nsweeps,
                    unsigned long long *events_dev, ma_stream_t stream);

/* r = rhs - det(D^2_h u) on the interior and 0 on the shell (Algorithm 1
 * step 3, the operator of Eq. MA_discrete). */
ma_status ma_residual(const double *u_dev, const double *rhs_dev, double *r_dev, int n, double h,
                      ma_stream_t stream);

/* The same residual (Algorithm 1 step 3, Eq. MA_discrete) as the fine-grid
 * residual of MA_MIXED solves computes it, without FP64 arithmetic: where the
 * 19 stencil values of a point share one sign and one binade, the second
 * differences are exact integer differences of their bit patterns, and the
 * determinant and rhs - det are taken in two-float (hi + lo FP32)
 * arithmetic, about 48 significant bits; elsewhere the FP64 evaluation of
 * ma_residual.  Same layout and arguments as ma_residual; asynchronous. */
ma_status ma_residual_f2(const double *u_dev, const double *rhs_dev, double *r_dev, int n, double h,
                         ma_stream_t stream);

/* Residual restriction r_H = I_h^H r_h (Section 3) from a fine grid of nf
 * points per side to the coarse grid of (nf+1)/2: kind MA_HALF_WEIGHTING or
 * MA_FULL_WEIGHTING on the coarse interior, 0 on the coarse shell. */
ma_status ma_restrict_residual(const double *rf_dev, int nf, double *rc_dev, int kind,
                               ma_stream_t stream);

/* Approximation restriction (Algorithm 1 step 4): with approx =
 * MA_APPROX_INJECTION, uc = uf(2I, 2J, 2K) everywhere; with
 * MA_APPROX_WEIGHTED, the kind weighting on the coarse interior and injection
 * on the shell. */
ma_status ma_restrict_solution(const double *uf_dev, int nf, double *uc_dev, int approx, int kind,
                               ma_stream_t stream);

/* tau-corrected coarse right-hand side b_H = det(D^2_H w_H) + r_H on the
 * coarse interior, 0 on the shell (Algorithm 1 step 5). */
ma_status ma_coarse_rhs(const double *wc_dev, const double *rc_dev, double *bc_dev, int nc, double H,
                        ma_stream_t stream);

/* u_h += I_H^h (u_H - w_H) on the fine interior, trilinear interpolation
 * (Algorithm 1 steps 7-8); nf = 2 nc - 1. */
ma_status ma_prolong_add(const double *uc_dev, const double *wc_dev, int nc, double *uf_dev,
                         ma_stream_t stream);

/* Fine interior := trilinear interpolation of the coarse solution (Algorithm
 * 2 step 4 with trilinear in place of cubic interpolation); shell untouched. */
ma_status ma_interpolate(const double *uc_dev, int nc, double *uf_dev, ma_stream_t stream);

/* Device scratch bytes of ma_interpolate_cubic for a coarse grid of nc. */
ma_status ma_interpolate_cubic_scratch_bytes(int nc, size_t *bytes);

/* Fine interior := tricubic interpolation of the coarse solution (Algorithm
 * 2 step 4, MA_FMG_CUBIC), as three one-axis passes through scratch_dev
 * (>= ma_interpolate_cubic_scratch_bytes(nc) bytes, 8-byte aligned); the fine
 * shell is untouched.  nc >= 3. */
ma_status ma_interpolate_cubic(const double *uc_dev, int nc, double *uf_dev, void *scratch_dev, size_t scratch_bytes,
                               ma_stream_t stream);

/* Approximate solve on a coarsest grid (Algorithm 1 step 1), one thread
 * block: sweeps > 0 runs that many sweeps, 0 sweeps until
 * max|du| <= 1e-14 max|u| (at most 100).  n <= 17. */
ma_status ma_coarsest_solve(double *u_dev, const double *rhs_dev, int n, double h, int sweeps,
                            unsigned long long *events_dev, ma_stream_t stream);

/* ---- single steps of the mixed-precision correction cycle -----------------
 * The correction problem for a fixed FP64 iterate u is
 *     N(e) = det(D^2_h (u + e)) - det(D^2_h u) = rhs,
 * i.e. det(D^2_h(u + e)) = f when rhs = f - det(D^2_h u); FP32 cycles solve it
 * for e and the FP64 driver updates u += e (defect correction; the FP64 work
 * is the fine residual and the update, motivated by the round-off remark of
 * Example 4).  N is evaluated as tr(cof(B) K) + tr(B cof(K)) + det(K) with
 * B = D^2_h u and K = D^2_h e, so its round-off scales with e.  u is passed as
 * an FP32 split u = u_hi + u_lo (u_hi = (float)u, u_lo = (float)(u - u_hi));
 * e, rhs and res are n^3 floats, [k][j][i]; e is 0 on the shell. */

/* Bytes of device scratch the two calls below need: the base Hessian
 * B = D^2_h u (FP32, six per interior point, colour-major order) and the
 * right-hand side in colour-major order. */
ma_status ma_correction_scratch_bytes(int n, size_t *bytes);

/* nsweeps 8-colour sweeps on e: at each point the new e is the one whose
 * u + e takes the smallest real root of the local cubic (Section 2, Eq.
 * realroots) for right-hand side det(D^2_h u) + rhs, with D^2_h u taken from
 * the FP32 store.  scratch_dev: >= ma_correction_scratch_bytes(n) bytes,
 * 256-byte aligned, overwritten. */
ma_status ma_smooth_correction(float *e_dev, const float *u_hi_dev, const float *u_lo_dev, const float *rhs_dev, int n,
                               double h, int nsweeps, void *scratch_dev, size_t scratch_bytes,
                               unsigned long long *events_dev, ma_stream_t stream);

/* One colour phase of that sweep: the points of colour
 * c = (i&1) | (j&1)<<1 | (k&1)<<2 (0 <= c < 8) only, in place; the eight
 * phases in ascending c are one sweep.  Same arguments otherwise;
 * MA_ERR_INVALID_ARG for a colour outside 0..7. */
ma_status ma_smooth_correction_colour(float *e_dev, const float *u_hi_dev, const float *u_lo_dev,
                                      const float *rhs_dev, int n, double h, int colour, void *scratch_dev,
                                      size_t scratch_bytes, unsigned long long *events_dev, ma_stream_t stream);

/* res = rhs - N(e) on the interior, 0 on the shell (same B store; same
 * scratch rules as ma_smooth_correction). */
ma_status ma_residual_correction(const float *e_dev, const float *u_hi_dev, const float *u_lo_dev,
                                 const float *rhs_dev, float *res_dev, int n, double h, void *scratch_dev,
                                 size_t scratch_bytes, ma_stream_t stream);

/* ---- kernel choice for the correction cycle (tile shapes, colour blocking) --
 * No counterpart in the paper.  A correction sweep visits the colours in
 * ascending order, either colour by colour (MA_CORR_BY_COLOUR: 8 launches in
 * place) or by k parity (MA_CORR_PLANE16/32/64: colours 0-3 of all even
 * planes, then colours 4-7 of all odd planes, 2 launches, in tiles of 16, 32
 * or 64 points per plane edge with a recomputed halo and a second e buffer),
 * which give the same bits; or in colour pairs (MA_CORR_PAIRS: colours c and
 * c^7, which share no stencil, in one launch, 4 launches in place), which is
 * the sequential sweep in the colour order 0, 7, 1, 6, 2, 5, 3, 4: another
 * 8-colour Gauss-Seidel sweep, other bits.  The
 * correction residual runs in plane tiles of 16, 32 or 64, or by columns
 * (MA_CORR_COLUMN: a warp walks 30 columns along k with the neighbour values
 * in registers and shuffles; residual only); all give the same bits.  The
 * choice is kept per grid size n (odd, 3 .. 4097) for the whole process;
 * hierarchy calls take it when they first record their CUDA graphs, so set or
 * tune before the first solve. */
enum {
    MA_CORR_BY_COLOUR = 0,
    MA_CORR_PLANE16 = 1,
    MA_CORR_PLANE32 = 2,
    MA_CORR_PLANE64 = 3,
    MA_CORR_COLUMN = 4,
    MA_CORR_PAIRS = 5
};

/* Sets the choice for grid size n (-1 restores the built-in default: colour
 * pairs at every size; the residual by columns).  The shared per-level batch
 * (ma_create_batch) and the fused tails (ma_set_corr_tail) sweep each grid
 * with the colour order of its size's choice, as a level-by-level cycle does.  MA_ERR_INVALID_ARG if n is not odd in [3, 4097] or a choice
 * is out of range (the residual has no MA_CORR_BY_COLOUR or MA_CORR_PAIRS,
 * the smoother no MA_CORR_COLUMN). */
ma_status ma_set_corr_tuning(int n, int smooth_choice, int residual_choice);

/* The choices in force for grid size n. */
ma_status ma_get_corr_tuning(int n, int *smooth_choice, int *residual_choice);

/* Fused tails.  The levels of a V-cycle with n <= max_n, down to the
 * coarsest grid, run as one single-block launch that keeps their grids in
 * shared memory and repeats the per-point arithmetic of the separate kernels,
 * so both forms give the same bits.  It saves the launches of those latency-
 * bound levels, but puts all their points on one SM: the default, 9, is the
 * fastest bound on whole solves (at 17 one SM takes longer over the 17^3
 * level than the launches it replaces).  max_n: 0 (level by level), 1 (the
 * default), or 3, 5, 9 or 17; MA_ERR_INVALID_ARG otherwise.  Hierarchies
 * take the setting when they first record their CUDA graphs.
 *
 * ma_set_corr_tail: the FP32 correction cycles of the mixed and FP32 modes. */
ma_status ma_set_corr_tail(int max_n);

/* ma_set_vcycle_tail: the FP64 V-cycles (ma_vcycle and the FP64 solves, FMG
 * included), with u, w, r and rhs of the
 * tail levels in shared memory.  The coarse levels' arrays in the workspace
 * are then left as they were; nothing outside the cycle reads them. */
ma_status ma_set_vcycle_tail(int max_n);

/* Autotuner: times every smoother variant (reps pairs of sweeps each) and
 * every residual variant (reps each) on the caller's data of one grid (the
 * arguments of ma_smooth_correction; e is overwritten by the sweeps), the way
 * hierarchies run them: each variant's launches are captured into a CUDA
 * graph and replayed, the fastest of 3 replays counting.  It records the
 * fastest of each for grid size n and writes the times in microseconds per
 * sweep (us_smooth[6], indexed by MA_CORR_*, entry 4 unused) and per residual
 * (us_residual[5], indexed by MA_CORR_*, entry 0 unused) when those are not
 * null.  Blocks on the stream. */
ma_status ma_tune_corr(float *e_dev, const float *u_hi_dev, const float *u_lo_dev, const float *rhs_dev, int n,
                       double h, int reps, void *scratch_dev, size_t scratch_bytes, double *us_smooth,
                       double *us_residual, ma_stream_t stream);

/* Bytes of device scratch ma_norm needs for a grid of n points per side. */
ma_status ma_norm_scratch_bytes(int n, size_t *bytes);

/* Max norm and discrete L2 norm sqrt(h^3 sum v^2) of v over the interior
 * (Section 4), written to out_host[0] and out_host[1].  scratch_dev holds at
 * least ma_norm_scratch_bytes(n) bytes.  Blocks on the stream. */
ma_status ma_norm(const double *v_dev, int n, double h, void *scratch_dev, size_t scratch_bytes,
                  double *out_host, ma_stream_t stream);

/* ---- norms without any scratch from the caller ------------------------------
 * No counterpart in the paper: an allocation-free variant of ma_norm for
 * callers that cannot allocate device memory where they need a norm (their
 * device memory is all owned and reserved by another allocator, or the
 * implicit device synchronisation of cudaMalloc/cudaFree is not acceptable
 * in their loop) and have no spare buffer to lend as scratch. */

/* Largest grid (points per side) ma_norm_static serves. */
#define MA_NORM_STATIC_MAX_N 513

/* Same result as ma_norm (max norm and discrete L2 norm of v over the
 * interior, into out_host[0] and out_host[1]; blocks on the stream), with the
 * reduction scratch taken from a fixed array of about 550 KB inside this
 * library's device memory instead of from the caller.  Every GPU that loads
 * the library holds that array until the process exits.  The library
 * allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 *  - n must be odd, 3 <= n <= MA_NORM_STATIC_MAX_N; larger grids return
 *    MA_ERR_INVALID_ARG with a message naming the limit.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress, with that device current) and caches it; make
 *    that first call before any stream capture.
 *  - All calls on a device share the one array and it keeps the last call's
 *    contents (each call overwrites every entry it reads, so nothing needs
 *    clearing).  Calls whose kernels overlap on the GPU -- on different
 *    streams, or from different host threads -- race on it and may return
 *    wrong norms; serialise them.
 *  - Each call waits for its stream (cudaStreamSynchronize) before it
 *    returns the norms on the host.
 *  - On failure the message for ma_last_error_string() is kept per host
 *    thread, like every other entry point's. */
ma_status ma_norm_static(const double *v_dev, int n, double h, double *out_host, ma_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* MA_H */
