// ma_capi.cu -- the C ABI of include/ma.h: hierarchy layout inside the
// caller's workspace, the FAS V-cycle and FMG drivers (Algorithms 1 and 2 of
// Liu, Froese, Oberman, Xiao), the stopping rule of Section 4, and the
// single-step entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ma.h"
#include "ma_hier.h"
#include "ma_internal.h"

namespace {

thread_local char g_err[512] = "";

ma_status fail(ma_status st, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

#define MA_CK(call)                                                                           \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return fail(MA_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool valid_step_grid(int n) { return n >= 3 && (n % 2) == 1 && n <= 4097; }

// Level sizes n_0 = n > n_1 > ... > n_{L-1} = coarsest_n with n_{l+1} = (n_l+1)/2.
int level_count(int n, int coarsest)
{
    int L = 1, m = n;
    while (m > coarsest) {
        if ((m - 1) % 2 != 0) return -1;
        m = (m + 1) / 2;
        ++L;
        if (L > ma::kMaxLevels) return -1;
    }
    return m == coarsest ? L : -1;
}

ma_status check_desc(const ma_hier_desc* d)
{
    if (!d) return fail(MA_ERR_INVALID_ARG, "null descriptor");
    if (!(d->coarsest_n == 3 || d->coarsest_n == 5 || d->coarsest_n == 9 || d->coarsest_n == 17))
        return fail(MA_ERR_INVALID_ARG, "coarsest_n must be 3, 5, 9 or 17 (got %d)", d->coarsest_n);
    if (d->n < d->coarsest_n || level_count(d->n, d->coarsest_n) < 1)
        return fail(MA_ERR_INVALID_ARG, "n = %d is not 2^L (coarsest_n - 1) + 1 for coarsest_n = %d", d->n,
                    d->coarsest_n);
    if (d->n > 4097) return fail(MA_ERR_INVALID_ARG, "n = %d exceeds 4097", d->n);
    if (!(d->len > 0.0) || !std::isfinite(d->len)) return fail(MA_ERR_INVALID_ARG, "len must be finite and > 0");
    if (d->nu1 < 0 || d->nu2 < 0 || d->nu1 > 64 || d->nu2 > 64 || d->nu1 + d->nu2 == 0)
        return fail(MA_ERR_INVALID_ARG, "nu1, nu2 must be in [0, 64] and not both 0");
    if (d->restrict_kind != MA_HALF_WEIGHTING && d->restrict_kind != MA_FULL_WEIGHTING)
        return fail(MA_ERR_INVALID_ARG, "bad restrict_kind %d", d->restrict_kind);
    if (d->approx_restrict != MA_APPROX_INJECTION && d->approx_restrict != MA_APPROX_WEIGHTED)
        return fail(MA_ERR_INVALID_ARG, "bad approx_restrict %d", d->approx_restrict);
    if (d->precision != MA_FP64 && d->precision != MA_MIXED && d->precision != MA_FP32)
        return fail(MA_ERR_INVALID_ARG, "bad precision %d", d->precision);
    if (d->coarse_sweeps < 0 || d->coarse_sweeps > 1000)
        return fail(MA_ERR_INVALID_ARG, "coarse_sweeps must be in [0, 1000]");
    if (d->inner_cycles < 0 || d->inner_cycles > 16)
        return fail(MA_ERR_INVALID_ARG, "inner_cycles must be in [0, 16]");
    if (d->fmg_interp != MA_FMG_TRILINEAR && d->fmg_interp != MA_FMG_CUBIC)
        return fail(MA_ERR_INVALID_ARG, "bad fmg_interp %d", d->fmg_interp);
    return MA_OK;
}

// Carves the workspace (or, with base == nullptr, only measures it).
size_t layout(ma_hierarchy* H, const ma_hier_desc* d, char* base)
{
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        char* p = base ? base + off : nullptr;
        off = align_up(off + bytes);
        return p;
    };
    const int L = level_count(d->n, d->coarsest_n);
    int m = d->n;
    double h = d->len / (d->n - 1);
    for (int l = 0; l < L; ++l) {
        const size_t pts = (size_t)m * m * m;
        ma::Level& lv = H->lev[l];
        lv.n = m;
        lv.h = h;
        lv.u = (double*)take(pts * sizeof(double));
        lv.rhs = (double*)take(pts * sizeof(double));
        lv.r = (double*)take(pts * sizeof(double));
        lv.w = (double*)take(pts * sizeof(double));
        if (d->precision == MA_MIXED || d->precision == MA_FP32) {
            lv.e = (float*)take(pts * sizeof(float));
            if (l < L - 1) lv.e2 = (float*)take(pts * sizeof(float));   // second buffer of the plane sweeps
            lv.bstore = (void*)take(ma::base_store_bytes(m));
            if (l > 0 && d->precision == MA_MIXED) {   // the finest B comes from the FP64 residual
                lv.hi = (float*)take(pts * sizeof(float));
                lv.lo = (float*)take(pts * sizeof(float));
            }
            lv.rhs32 = (float*)take(ma::cm_points(m) * sizeof(float));
            lv.res32 = (float*)take(pts * sizeof(float));
            lv.w32 = (float*)take(pts * sizeof(float));
        }
        m = (m + 1) / 2;
        h *= 2.0;
    }
    H->L = L;
    H->npartials = ma::residual_partial_count(d->n);
    H->partials = (double*)take(2 * sizeof(double) * (size_t)H->npartials);
    H->rb = (double*)take(5 * sizeof(double));
    H->out2 = H->rb;
    H->events = base ? (unsigned long long*)(H->rb + 4) : nullptr;
    H->flag = (int*)take(sizeof(int));
    return off;
}

// Algorithm 1 from level l0 down to the coarsest grid and back.  The levels
// with n <= 17 (the tail, down to the coarsest grid) run as one single-block
// launch with the same arithmetic.
cudaError_t vcycle_from(ma_hierarchy* H, int l0)
{
    cudaStream_t s = H->s;
    const ma_hier_desc& d = H->d;
    cudaError_t e;
    int lt = H->L - 1;   // first level of the fused tail
    while (lt > l0 && H->lev[lt - 1].n <= ma::vcycle_tail_max_n()) --lt;
    const bool fused = H->lev[lt].n <= ma::vcycle_tail_max_n();
    if (!fused) lt = H->L - 1;
    for (int l = l0; l < lt; ++l) {
        ma::Level& F = H->lev[l];
        ma::Level& C = H->lev[l + 1];
        if ((e = ma::launch_smooth(F.u, F.rhs, F.n, F.h, d.nu1, H->events, s)) != cudaSuccess) return e;   // (2)
        if ((e = ma::launch_residual(F.u, F.rhs, F.r, F.n, F.h, nullptr, s)) != cudaSuccess) return e;     // (3)
        if ((e = ma::launch_restrict_level(F.u, F.r, F.n, C.w, C.u, C.r, d.restrict_kind, d.approx_restrict, s)) !=
            cudaSuccess)
            return e;                                                                                        // (3)-(4)
        if ((e = ma::launch_coarse_rhs(C.w, C.r, C.rhs, C.n, C.h, s)) != cudaSuccess) return e;             // (5)
    }
    if (fused) {
        ma::TailSpec64 spec[4];
        const int nlev = H->L - lt;
        for (int q = 0; q < nlev; ++q) {
            ma::Level& A = H->lev[lt + q];
            spec[q] = ma::TailSpec64{A.n, A.h, A.u, A.rhs};
        }
        if ((e = ma::launch_vcycle_tail(spec, nlev, d.nu1, d.nu2, d.restrict_kind, d.approx_restrict,
                                        d.coarse_sweeps, H->events, s)) != cudaSuccess)
            return e;
    } else {
        ma::Level& B = H->lev[H->L - 1];
        if ((e = ma::launch_coarsest(B.u, B.rhs, B.n, B.h, d.coarse_sweeps, H->events, s)) != cudaSuccess)
            return e;                                                                                      // (1)
    }
    for (int l = lt - 1; l >= l0; --l) {
        ma::Level& F = H->lev[l];
        ma::Level& C = H->lev[l + 1];
        if ((e = ma::launch_prolong_add(C.u, C.w, C.n, F.u, s)) != cudaSuccess) return e;                  // (7)-(8)
        if ((e = ma::launch_smooth(F.u, F.rhs, F.n, F.h, d.nu2, H->events, s)) != cudaSuccess) return e;  // (9)
    }
    return cudaSuccess;
}

// Algorithm 2: inject f (and the Dirichlet data) down, solve the coarsest
// problem from a zero interior, then interpolate up with one V-cycle per level.
// With finest_vcycle false the finest level only receives the interpolated
// iterate (the mixed-precision solve continues from there).
cudaError_t refresh_base(ma_hierarchy* H, int apply, int l0 = 0);
cudaError_t corr_vcycle_from(ma_hierarchy* H, int l0);

// An FMG level of the mixed solve below the finest: one outer iteration with
// kFmgCorrCycles FP32 correction V-cycles from level l, in place of
// Algorithm 2's FP64 V-cycle there (cheaper, and at least as strong).  e_l = 0
// and the base Hessians below l from the FP32 split of u_l; the FP64 residual
// at l (the correction rhs and the B of level l); the cycles; u_l += e_l.
cudaError_t mixed_fmg_step(ma_hierarchy* H, int l)
{
    cudaError_t e;
    if ((e = refresh_base(H, 0, l)) != cudaSuccess) return e;
    ma::Level& F = H->lev[l];
    if ((e = ma::launch_residual64_to32(F.u, F.rhs, F.rhs32, F.bstore, F.n, F.h, H->partials, H->s)) != cudaSuccess)
        return e;
    for (int c = 0; c < ma::kFmgCorrCycles; ++c)
        if ((e = corr_vcycle_from(H, l)) != cudaSuccess) return e;
    return ma::launch_update(F.u, F.e, F.n, 1, H->s);
}

cudaError_t fmg(ma_hierarchy* H, bool finest_vcycle = true)
{
    cudaStream_t s = H->s;
    cudaError_t e;
    for (int l = 0; l < H->L - 1; ++l) {
        ma::Level& F = H->lev[l];
        ma::Level& C = H->lev[l + 1];
        if ((e = ma::launch_inject(F.rhs, F.n, C.rhs, s)) != cudaSuccess) return e;
        if ((e = ma::launch_inject(F.u, F.n, C.u, s)) != cudaSuccess) return e;
    }
    ma::Level& B = H->lev[H->L - 1];
    if ((e = ma::launch_zero_interior(B.u, B.n, s)) != cudaSuccess) return e;
    if ((e = ma::launch_coarsest(B.u, B.rhs, B.n, B.h, H->d.coarse_sweeps, H->events, s)) != cudaSuccess) return e;
    for (int l = H->L - 2; l >= 0; --l) {
        ma::Level& F = H->lev[l];
        ma::Level& C = H->lev[l + 1];
        // the fine level's r is free here and large enough for the cubic passes
        e = H->d.fmg_interp == MA_FMG_CUBIC ? ma::launch_interpolate_cubic(C.u, C.n, F.u, F.r, s)
                                            : ma::launch_interpolate(C.u, C.n, F.u, s);
        if (e != cudaSuccess) return e;
        if (l == 0 && !finest_vcycle) break;
        e = H->d.precision == MA_MIXED ? mixed_fmg_step(H, l) : vcycle_from(H, l);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ---- mixed precision: FP32 FAS cycle on the correction e --------------------

// u += e on the finest level (apply != 0), e = 0, and the base Hessians B of
// the coarse correction levels from the FP32 split of the injected iterate.
// The finest B is written by the FP64 residual (mixed_residual), which
// always follows.
cudaError_t refresh_base(ma_hierarchy* H, int apply, int l0)
{
    cudaStream_t s = H->s;
    cudaError_t e;
    ma::Level& F = H->lev[l0];
    if ((e = ma::launch_update(F.u, F.e, F.n, apply, s)) != cudaSuccess) return e;
    for (int l = l0 + 1; l < H->L; ++l) {
        ma::Level& A = H->lev[l];
        if ((e = ma::launch_split_inject(F.u, F.n, 1 << (l - l0), A.hi, A.lo, A.n, s)) != cudaSuccess) return e;
        if ((e = ma::launch_base_colour(A.hi, A.lo, A.bstore, A.n, A.h, s)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// One FAS V-cycle (Algorithm 1 structure) for N(e) = rhs32 from level l0
// down and back, starting from the current e on level l0.  The levels with
// n <= 17 (the tail, down to the coarsest grid) run as one single-block
// launch with the same arithmetic.
cudaError_t corr_vcycle_from(ma_hierarchy* H, int l0)
{
    cudaStream_t s = H->s;
    const ma_hier_desc& d = H->d;
    cudaError_t e;
    int lt = H->L - 1;   // first level of the fused tail
    while (lt > l0 && H->lev[lt - 1].n <= ma::corr_tail_max_n()) --lt;
    const bool fused = H->lev[lt].n <= ma::corr_tail_max_n();
    if (!fused) lt = H->L - 1;
    for (int l = l0; l < lt; ++l) {
        ma::Level& F = H->lev[l];
        ma::Level& C = H->lev[l + 1];
        if ((e = ma::launch_smooth_corr(F.e, F.e2, F.bstore, F.rhs32, F.n, F.h, d.nu1, H->events, s)) !=
            cudaSuccess)
            return e;
        if ((e = ma::launch_residual_corr(F.e, F.bstore, F.rhs32, F.res32, F.n, F.h, s)) != cudaSuccess) return e;
        if ((e = ma::launch_restrict_level_f32(F.e, F.res32, F.n, C.w32, C.e, C.res32, d.restrict_kind,
                                               d.approx_restrict, s)) != cudaSuccess)
            return e;
        if ((e = ma::launch_coarse_rhs_corr(C.w32, C.bstore, C.res32, C.rhs32, C.n, C.h, s)) != cudaSuccess)
            return e;
    }
    if (fused) {
        ma::TailSpec spec[4];
        const int nlev = H->L - lt;
        for (int q = 0; q < nlev; ++q) {
            ma::Level& A = H->lev[lt + q];
            spec[q] = ma::TailSpec{A.n, A.h, A.e, A.bstore, A.rhs32};
        }
        if ((e = ma::launch_corr_vcycle_tail(spec, nlev, d.nu1, d.nu2, d.restrict_kind, d.approx_restrict,
                                             d.coarse_sweeps, H->events, s)) != cudaSuccess)
            return e;
    } else {
        ma::Level& B = H->lev[H->L - 1];
        if ((e = ma::launch_coarsest_corr(B.e, B.bstore, B.rhs32, B.n, B.h, d.coarse_sweeps, H->events, s)) !=
            cudaSuccess)
            return e;
    }
    for (int l = lt - 1; l >= l0; --l) {
        ma::Level& F = H->lev[l];
        ma::Level& C = H->lev[l + 1];
        if ((e = ma::launch_prolong_add_f32(C.e, C.w32, C.n, F.e, s)) != cudaSuccess) return e;
        if ((e = ma::launch_smooth_corr(F.e, F.e2, F.bstore, F.rhs32, F.n, F.h, d.nu2, H->events, s)) !=
            cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

cudaError_t corr_vcycle(ma_hierarchy* H) { return corr_vcycle_from(H, 0); }

// ---- FP32 mode: the correction machinery with B = 0 -------------------------
// With B = 0 the correction operator N(e) = det(B + K(e)) - det(B) is
// det(D^2_h e) itself, so the FP32 FAS cycles solve det(D^2_h e) = f for the
// solution: e carries the Dirichlet data on its shell and rhs32 holds f.  No
// FP64 residual or update: the result carries FP32 round-off of the second
// differences, ~eps_32 |u| / h^2 in the Hessian.

// e = FP32(u) and rhs32 = FP32(f) (colour-major) on every level, f and the
// boundary data injected down in FP64 first; e2 gets e's shell.
cudaError_t fp32_prepare(ma_hierarchy* H)
{
    cudaStream_t s = H->s;
    cudaError_t e;
    for (int l = 0; l < H->L - 1; ++l) {
        ma::Level& F = H->lev[l];
        ma::Level& C = H->lev[l + 1];
        if ((e = ma::launch_inject(F.rhs, F.n, C.rhs, s)) != cudaSuccess) return e;
        if ((e = ma::launch_inject(F.u, F.n, C.u, s)) != cudaSuccess) return e;
    }
    for (int l = 0; l < H->L; ++l) {
        ma::Level& A = H->lev[l];
        if ((e = ma::launch_f64_to_f32(A.u, A.e, A.n, s)) != cudaSuccess) return e;
        if ((e = ma::launch_f64_to_f32(A.rhs, A.res32, A.n, s)) != cudaSuccess) return e;
        if ((e = ma::launch_to_cm(A.res32, A.rhs32, A.n, s)) != cudaSuccess) return e;
        if (A.e2 && (e = cudaMemcpyAsync(A.e2, A.e, sizeof(float) * (size_t)A.n * A.n * A.n,
                                         cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

// Algorithm 2 in FP32: zero coarsest interior, coarsest solve, then up the
// levels: interpolate and one cycle from that level.  The tricubic
// interpolation (MA_FMG_CUBIC) runs on the levels' FP64 arrays: coarse e to
// FP64, the fine interior interpolated, the fine grid back to FP32 (its shell
// holds the boundary data, which e carries as well).
cudaError_t fp32_fmg(ma_hierarchy* H)
{
    cudaStream_t s = H->s;
    cudaError_t e;
    ma::Level& B = H->lev[H->L - 1];
    if ((e = ma::launch_zero_interior_f32(B.e, B.n, s)) != cudaSuccess) return e;
    if ((e = ma::launch_coarsest_corr(B.e, B.bstore, B.rhs32, B.n, B.h, H->d.coarse_sweeps, H->events, s)) !=
        cudaSuccess)
        return e;
    for (int l = H->L - 2; l >= 0; --l) {
        ma::Level& F = H->lev[l];
        ma::Level& C = H->lev[l + 1];
        if (H->d.fmg_interp == MA_FMG_CUBIC) {
            if ((e = ma::launch_f32_to_f64(C.e, C.u, C.n, s)) != cudaSuccess) return e;
            if ((e = ma::launch_interpolate_cubic(C.u, C.n, F.u, F.r, s)) != cudaSuccess) return e;
            if ((e = ma::launch_f64_to_f32(F.u, F.e, F.n, s)) != cudaSuccess) return e;
        } else if ((e = ma::launch_interpolate_f32(C.e, C.n, F.e, s)) != cudaSuccess) {
            return e;
        }
        if ((e = corr_vcycle_from(H, l)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The FP32 residual f - det(D^2_h e) and its norms into out2; u = e in FP64.
cudaError_t fp32_residual(ma_hierarchy* H)
{
    ma::Level& F = H->lev[0];
    cudaError_t e = ma::launch_residual_corr(F.e, F.bstore, F.rhs32, F.res32, F.n, F.h, H->s);
    if (e == cudaSuccess) e = ma::launch_norm_partials_f32(F.res32, F.n, H->partials, H->s);
    if (e == cudaSuccess) e = ma::launch_norm_final(H->partials, H->npartials, F.h, H->out2, H->s);
    if (e == cudaSuccess) e = ma::launch_f32_to_f64(F.e, F.u, F.n, H->s);
    return e;
}

// FP64 fine residual into rhs32 (the correction problem's right-hand side)
// and the finest base Hessian B, with norm partials; the caller reads the
// norms.
cudaError_t mixed_residual(ma_hierarchy* H)
{
    ma::Level& F = H->lev[0];
    cudaError_t e = ma::launch_residual64_to32(F.u, F.rhs, F.rhs32, F.bstore, F.n, F.h, H->partials, H->s);
    if (e != cudaSuccess) return e;
    return ma::launch_norm_final(H->partials, H->npartials, F.h, H->out2, H->s);
}

// Runs body() as a CUDA graph captured once on the hierarchy's private
// stream and replayed on its own stream: one graph launch instead of the
// ~10^2 - 10^3 kernel launches of a cycle or an FMG pass.
template <typename F>
cudaError_t run_graph(ma_hierarchy* H, ma::GraphSlot& gs, F body)
{
    if (!gs.exec) {
        const unsigned long long before = ma::launch_count();
        cudaError_t e = cudaStreamBeginCapture(H->cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        cudaStream_t user = H->s;
        H->s = H->cap;
        const cudaError_t eb = body();
        H->s = user;
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(H->cap, &g);
        const unsigned long long captured = ma::launch_count() - before;
        ma::uncount_launches(captured);   // captured, not run
        if (eb != cudaSuccess || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return eb != cudaSuccess ? eb : e;
        }
        e = cudaGraphInstantiate(&gs.exec, g, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            gs.exec = nullptr;
            return e;
        }
        gs.graph = g;
        gs.launches = captured;
    }
    ma::count_launches(gs.launches);
    return cudaGraphLaunch(gs.exec, H->s);
}

void destroy_graphs(ma_hierarchy* H)
{
    ma::GraphSlot* slots[7] = {&H->g_init[0], &H->g_init[1], &H->g_init[2], &H->g_init[3],
                               &H->g_init[4], &H->g_init[5], &H->g_cycle};
    for (ma::GraphSlot* gs : slots) {
        if (gs->exec) cudaGraphExecDestroy(gs->exec);
        if (gs->graph) cudaGraphDestroy(gs->graph);
        *gs = ma::GraphSlot();
    }
}

// One outer (defect-correction) iteration: FP64 residual, FP32 correction
// V-cycle, FP64 update.  Leaves the base refreshed for the next iteration.
cudaError_t mixed_iteration(ma_hierarchy* H)
{
    cudaError_t e;
    if ((e = refresh_base(H, 0)) != cudaSuccess) return e;
    if ((e = mixed_residual(H)) != cudaSuccess) return e;
    const int inner = H->d.inner_cycles > 0 ? H->d.inner_cycles : 3;
    for (int c = 0; c < inner; ++c)
        if ((e = corr_vcycle(H)) != cudaSuccess) return e;
    return refresh_base(H, 1);
}

// Reads the reduced norms (max, L2) in out2 back to the host; blocks.
ma_status read_norms(ma_hierarchy* H, double* mx, double* l2)
{
    MA_CK(cudaMemcpyAsync(H->host, H->out2, 2 * sizeof(double), cudaMemcpyDeviceToHost, H->s));
    MA_CK(cudaStreamSynchronize(H->s));
    *mx = H->host[0];
    *l2 = H->host[1];
    return MA_OK;
}

// Fine-level FP64 residual norms (max, L2); blocks on the stream.
ma_status fine_residual_norms(ma_hierarchy* H, double* mx, double* l2)
{
    ma::Level& F = H->lev[0];
    MA_CK(ma::launch_residual(F.u, F.rhs, F.r, F.n, F.h, H->partials, H->s));
    MA_CK(ma::launch_norm_final(H->partials, H->npartials, F.h, H->out2, H->s));
    return read_norms(H, mx, l2);
}

// NVTX range over a host call (visible to ncu --nvtx and other tracers;
// a no-op unless a tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

void ma::set_last_error(const char* msg) { snprintf(g_err, sizeof g_err, "%s", msg); }

extern "C" {

const char* ma_last_error_string(void) { return g_err; }

ma_status ma_kernel_launch_count(unsigned long long* out)
{
    if (!out) return fail(MA_ERR_INVALID_ARG, "null out");
    *out = ma::launch_count();
    return MA_OK;
}

ma_status ma_hierarchy_footprint(const ma_hier_desc* desc, size_t* bytes)
{
    ma_status st = check_desc(desc);
    if (st != MA_OK) return st;
    if (!bytes) return fail(MA_ERR_INVALID_ARG, "null bytes");
    ma_hierarchy tmp;
    tmp.d = *desc;
    *bytes = layout(&tmp, desc, nullptr);
    return MA_OK;
}

ma_status ma_create_hierarchy(const ma_hier_desc* desc, void* dev_workspace, size_t bytes, ma_stream_t stream,
                              ma_hierarchy** out)
{
    ma_status st = check_desc(desc);
    if (st != MA_OK) return st;
    if (!out) return fail(MA_ERR_INVALID_ARG, "null out");
    *out = nullptr;
    if (!dev_workspace) return fail(MA_ERR_INVALID_ARG, "null workspace");
    if (((uintptr_t)dev_workspace) % kAlign != 0) return fail(MA_ERR_INVALID_ARG, "workspace not 256-byte aligned");
    ma_hierarchy* H = new (std::nothrow) ma_hierarchy();
    if (!H) return fail(MA_ERR_OOM, "host allocation failed");
    H->d = *desc;
    const size_t need = layout(H, desc, (char*)dev_workspace);
    if (bytes < need) {
        delete H;
        return fail(MA_ERR_INVALID_ARG, "workspace of %zu bytes < footprint %zu", bytes, need);
    }
    H->ws = (char*)dev_workspace;
    H->bytes = need;
    H->s = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&H->device);
    if (e == cudaSuccess) e = ma::prepare_kernels();
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&H->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&H->host, 8 * sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&H->sv.ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemsetAsync(H->events, 0, sizeof(unsigned long long), H->s);
    for (int l = 0; l < H->L && e == cudaSuccess; ++l) {
        // corrections start at zero; the shells of e, e2 and res32 stay zero
        const size_t pts = (size_t)H->lev[l].n * H->lev[l].n * H->lev[l].n;
        if (H->lev[l].e) e = cudaMemsetAsync(H->lev[l].e, 0, pts * sizeof(float), H->s);
        if (e == cudaSuccess && H->lev[l].e2) e = cudaMemsetAsync(H->lev[l].e2, 0, pts * sizeof(float), H->s);
        if (e == cudaSuccess && H->lev[l].res32) e = cudaMemsetAsync(H->lev[l].res32, 0, pts * sizeof(float), H->s);
        if (e == cudaSuccess && desc->precision == MA_FP32)   // B = 0: the operator is det(D^2_h e)
            e = cudaMemsetAsync(H->lev[l].bstore, 0, ma::base_store_bytes(H->lev[l].n), H->s);
    }
    if (e != cudaSuccess) {
        if (H->host) cudaFreeHost(H->host);
        if (H->cap) cudaStreamDestroy(H->cap);
        if (H->sv.ev) cudaEventDestroy(H->sv.ev);
        delete H;
        return fail(MA_ERR_CUDA, "create: %s", cudaGetErrorString(e));
    }
    *out = H;
    return MA_OK;
}

ma_status ma_destroy_hierarchy(ma_hierarchy* H)
{
    if (!H) return MA_OK;
    DeviceGuard g(H->device);
    cudaError_t e = cudaStreamSynchronize(H->s);
    destroy_graphs(H);
    if (H->cap) cudaStreamDestroy(H->cap);
    if (H->sv.ev) cudaEventDestroy(H->sv.ev);
    if (H->host) cudaFreeHost(H->host);
    delete H;
    if (e != cudaSuccess) return fail(MA_ERR_CUDA, "destroy: %s", cudaGetErrorString(e));
    return MA_OK;
}

ma_status ma_hierarchy_info(const ma_hierarchy* H, int* n, int* levels, size_t* bytes)
{
    if (!H) return fail(MA_ERR_INVALID_ARG, "null hierarchy");
    if (n) *n = H->d.n;
    if (levels) *levels = H->L;
    if (bytes) *bytes = H->bytes;
    return MA_OK;
}

ma_status ma_set_rhs_bc(ma_hierarchy* H, const double* f_dev, const double* g_dev)
{
    if (!H || !f_dev || !g_dev) return fail(MA_ERR_INVALID_ARG, "null argument");
    DeviceGuard g(H->device);
    ma::Level& F = H->lev[0];
    MA_CK(cudaMemsetAsync(H->flag, 0, sizeof(int), H->s));
    MA_CK(ma::launch_copy_rhs_bc(f_dev, g_dev, F.rhs, F.u, F.n, H->flag, H->s));
    int bad = 0;
    MA_CK(cudaMemcpyAsync(&H->host[6], H->flag, sizeof(int), cudaMemcpyDeviceToHost, H->s));
    MA_CK(cudaStreamSynchronize(H->s));
    std::memcpy(&bad, &H->host[6], sizeof(int));
    if (bad) return fail(MA_ERR_INVALID_ARG, "%d grid values invalid (f must be finite and > 0 inside, g finite)", bad);
    return MA_OK;
}

// Host-buffer variants: the inputs land in the fine level's residual and
// coarse-approximation fields (n^3 doubles each, scratch until the next cycle
// overwrites them), and the same validating copy kernel moves them into place.
ma_status ma_set_rhs_bc_host(ma_hierarchy* H, const double* f_host, const double* g_host)
{
    if (!H || !f_host || !g_host) return fail(MA_ERR_INVALID_ARG, "null argument");
    DeviceGuard g(H->device);
    ma::Level& F = H->lev[0];
    const size_t bytes = (size_t)F.n * F.n * F.n * sizeof(double);
    MA_CK(cudaMemcpyAsync(F.r, f_host, bytes, cudaMemcpyHostToDevice, H->s));
    MA_CK(cudaMemcpyAsync(F.w, g_host, bytes, cudaMemcpyHostToDevice, H->s));
    return ma_set_rhs_bc(H, F.r, F.w);
}

ma_status ma_get_solution_host(ma_hierarchy* H, double* u_host)
{
    if (!H || !u_host) return fail(MA_ERR_INVALID_ARG, "null argument");
    DeviceGuard g(H->device);
    const size_t pts = (size_t)H->d.n * H->d.n * H->d.n;
    MA_CK(cudaMemcpyAsync(u_host, H->lev[0].u, pts * sizeof(double), cudaMemcpyDeviceToHost, H->s));
    MA_CK(cudaStreamSynchronize(H->s));
    return MA_OK;
}

ma_status ma_vcycle(ma_hierarchy* H, int ncycles)
{
    NvtxRange nv("ma_vcycle");
    if (!H || ncycles < 0) return fail(MA_ERR_INVALID_ARG, "bad arguments");
    DeviceGuard g(H->device);
    if (H->d.precision == MA_FP32) {
        MA_CK(fp32_prepare(H));
        for (int c = 0; c < ncycles; ++c) MA_CK(corr_vcycle(H));
        MA_CK(ma::launch_f32_to_f64(H->lev[0].e, H->lev[0].u, H->lev[0].n, H->s));
        return MA_OK;
    }
    for (int c = 0; c < ncycles; ++c) {
        if (H->d.precision == MA_MIXED) MA_CK(mixed_iteration(H));
        else MA_CK(vcycle_from(H, 0));
    }
    return MA_OK;
}

ma_status ma_residual_norm(ma_hierarchy* H, int norm, double* out)
{
    if (!H || !out || (norm != MA_NORM_MAX && norm != MA_NORM_L2)) return fail(MA_ERR_INVALID_ARG, "bad arguments");
    DeviceGuard g(H->device);
    double mx, l2;
    ma_status st = fine_residual_norms(H, &mx, &l2);
    if (st != MA_OK) return st;
    *out = norm == MA_NORM_MAX ? mx : l2;
    return MA_OK;
}

ma_status ma_get_solution(ma_hierarchy* H, double* u_dev)
{
    if (!H || !u_dev) return fail(MA_ERR_INVALID_ARG, "null argument");
    DeviceGuard g(H->device);
    const size_t pts = (size_t)H->d.n * H->d.n * H->d.n;
    MA_CK(cudaMemcpyAsync(u_dev, H->lev[0].u, pts * sizeof(double), cudaMemcpyDeviceToDevice, H->s));
    return MA_OK;
}

ma_status ma_set_solution(ma_hierarchy* H, const double* u_dev)
{
    if (!H || !u_dev) return fail(MA_ERR_INVALID_ARG, "null argument");
    DeviceGuard g(H->device);
    const size_t pts = (size_t)H->d.n * H->d.n * H->d.n;
    MA_CK(cudaMemcpyAsync(H->lev[0].u, u_dev, pts * sizeof(double), cudaMemcpyDeviceToDevice, H->s));
    return MA_OK;
}

static void solve_state_reset(ma_hierarchy* H, const ma_solve_opts* opts)
{
    H->sv.o = *opts;
    H->sv.phase = 0;
    H->sv.stagnant = 0;
    H->sv.scale = 1.0;
    H->sv.rel = 0.0;
    std::memset(&H->sv.r, 0, sizeof H->sv.r);
}

static ma_status check_opts(const ma_solve_opts* o)
{
    if (!(o->tol >= 0.0) || o->max_cycles < 0 || (o->norm != MA_NORM_MAX && o->norm != MA_NORM_L2) ||
        o->init < MA_INIT_FMG || o->init > MA_INIT_KEEP || o->relative < MA_REL_NONE || o->relative > MA_REL_INITIAL)
        return fail(MA_ERR_INVALID_ARG, "bad solve options");
    return MA_OK;
}

// Copies the read-back block to the pinned host buffer and marks it.
static cudaError_t queue_readback(ma_hierarchy* H)
{
    cudaError_t e = cudaMemcpyAsync(H->host, H->rb, 5 * sizeof(double), cudaMemcpyDeviceToHost, H->s);
    if (e != cudaSuccess) return e;
    return cudaEventRecord(H->sv.ev, H->s);
}

ma_status ma_solve_begin(ma_hierarchy* H, const ma_solve_opts* opts)
{
    NvtxRange nv("ma_solve_begin: init + first cycle");
    if (!H || !opts) return fail(MA_ERR_INVALID_ARG, "null argument");
    ma_status st = check_opts(opts);
    if (st != MA_OK) return st;
    DeviceGuard g(H->device);
    solve_state_reset(H, opts);
    MA_CK(cudaMemsetAsync(H->events, 0, sizeof(unsigned long long), H->s));
    const bool mixed = H->d.precision == MA_MIXED;
    // rhs norms, the initial iterate and its residual norm as one graph.  In
    // mixed precision every FMG level runs an outer iteration (FP64
    // residual, FP32 correction cycles, FP64 update) in place of the FP64
    // V-cycle of Algorithm 2; the finest level's is the first outer
    // iteration of the solve.
    const int init = opts->init;
    const bool ref_initial = opts->relative == MA_REL_INITIAL;
    MA_CK(run_graph(H, H->g_init[init + (ref_initial ? 3 : 0)], [&]() -> cudaError_t {
        ma::Level& F = H->lev[0];
        cudaError_t e = cudaSuccess;
        if (ref_initial) {
            // reference: the residual of the initial iterate (zero interior
            // unless the current iterate is kept)
            if (init != MA_INIT_KEEP) e = ma::launch_zero_interior(F.u, F.n, H->s);
            if (e == cudaSuccess) e = ma::launch_residual(F.u, F.rhs, F.r, F.n, F.h, H->partials, H->s);
        } else {
            e = ma::launch_norm_partials(F.rhs, F.n, H->partials, H->s);
        }
        if (e == cudaSuccess) e = ma::launch_norm_final(H->partials, H->npartials, F.h, H->rb + 2, H->s);
        if (e != cudaSuccess) return e;
        if (H->d.precision == MA_FP32) {
            if ((e = fp32_prepare(H)) != cudaSuccess) return e;
            if (init == MA_INIT_FMG && (e = fp32_fmg(H)) != cudaSuccess) return e;
            if (init == MA_INIT_ZERO && (e = ma::launch_zero_interior_f32(F.e, F.n, H->s)) != cudaSuccess) return e;
            return fp32_residual(H);
        }
        if (init == MA_INIT_FMG) e = fmg(H, !mixed);
        if (e == cudaSuccess && init == MA_INIT_ZERO) e = ma::launch_zero_interior(F.u, F.n, H->s);
        if (e != cudaSuccess) return e;
        if (mixed) {
            if ((e = refresh_base(H, 0)) != cudaSuccess) return e;
            if ((e = mixed_residual(H)) != cudaSuccess) return e;
            if (init != MA_INIT_FMG) return cudaSuccess;
            // Algorithm 2 step 5 on the finest level: one outer iteration
            // (the FP32 correction cycles) completes the FMG pass
            const int inner = H->d.inner_cycles > 0 ? H->d.inner_cycles : 3;
            for (int c = 0; c < inner; ++c)
                if ((e = corr_vcycle(H)) != cudaSuccess) return e;
            if ((e = refresh_base(H, 1)) != cudaSuccess) return e;
            return mixed_residual(H);
        }
        if ((e = ma::launch_residual(F.u, F.rhs, F.r, F.n, F.h, H->partials, H->s)) != cudaSuccess) return e;
        return ma::launch_norm_final(H->partials, H->npartials, F.h, H->out2, H->s);
    }));
    MA_CK(queue_readback(H));
    H->sv.phase = 1;
    return MA_OK;
}

// One cycle (FP64 V-cycle, or in mixed precision inner FP32 correction
// cycles + FP64 update) and the new residual norm, as one graph.
static cudaError_t launch_cycle(ma_hierarchy* H)
{
    NvtxRange nv("cycle");
    const bool mixed = H->d.precision == MA_MIXED;
    return run_graph(H, H->g_cycle, [&]() -> cudaError_t {
        cudaError_t e;
        if (H->d.precision == MA_FP32) {
            if ((e = corr_vcycle(H)) != cudaSuccess) return e;
            return fp32_residual(H);
        }
        if (mixed) {
            const int inner = H->d.inner_cycles > 0 ? H->d.inner_cycles : 3;
            for (int c = 0; c < inner; ++c)
                if ((e = corr_vcycle(H)) != cudaSuccess) return e;
            if ((e = refresh_base(H, 1)) != cudaSuccess) return e;
            return mixed_residual(H);
        }
        if ((e = vcycle_from(H, 0)) != cudaSuccess) return e;
        ma::Level& F = H->lev[0];
        if ((e = ma::launch_residual(F.u, F.rhs, F.r, F.n, F.h, H->partials, H->s)) != cudaSuccess) return e;
        return ma::launch_norm_final(H->partials, H->npartials, F.h, H->out2, H->s);
    });
}

// Applies the stopping rule to the norms in the host read-back block (after
// the start, phase 1, or after a cycle, phase 2); returns true, with the
// result filled and phase 3, when the solve is finished.
static bool absorb_norms(ma_hierarchy* H)
{
    const ma_solve_opts& o = H->sv.o;
    const double resn = o.norm == MA_NORM_MAX ? H->host[0] : H->host[1];
    ma_solve_result& r = H->sv.r;
    if (H->sv.phase == 1) {
        double sc = 1.0;
        if (o.relative) {
            sc = o.norm == MA_NORM_MAX ? H->host[2] : H->host[3];
            if (!(sc > 0.0)) sc = 1.0;
        }
        H->sv.scale = sc;
        H->sv.rel = resn / sc;
        r.res0 = H->sv.rel;
    } else {
        const double nrel = resn / H->sv.scale;
        r.cycles += 1;
        // cycles in a row that barely reduce the residual: round-off floor
        H->sv.stagnant = (nrel > 0.8 * H->sv.rel) ? H->sv.stagnant + 1 : 0;
        H->sv.rel = nrel;
    }
    const double rel = H->sv.rel;
    // The max norm folds with fmax, which skips NaN entries; the sum of
    // squares behind the L2 norm does not, so both are checked.
    const bool finite = std::isfinite(rel) && std::isfinite(H->host[0]) && std::isfinite(H->host[1]);
    int out = -1;
    if (!finite) out = MA_ERR_NONFINITE;
    else if (rel <= o.tol) out = MA_OK;
    else if (r.cycles >= o.max_cycles) out = MA_ERR_NOT_CONVERGED;
    else if (H->sv.stagnant >= ma::kFloorStagnantCycles) {
        r.floor_reached = 1;
        out = MA_ERR_NOT_CONVERGED;
    }
    if (out >= 0) {
        unsigned long long ev = 0;
        std::memcpy(&ev, H->host + 4, sizeof ev);
        r.res = rel;
        r.status = out;
        r.nonconvex_root_events = (long long)ev;
        H->sv.phase = 3;
        return true;
    }
    return false;
}

ma_status ma_solve_advance(ma_hierarchy* H, int* done)
{
    if (!H || !done) return fail(MA_ERR_INVALID_ARG, "null argument");
    *done = 0;
    if (H->sv.phase == 0) return fail(MA_ERR_INVALID_ARG, "ma_solve_advance before ma_solve_begin");
    if (H->sv.phase == 3) {
        *done = 1;
        return MA_OK;
    }
    DeviceGuard g(H->device);
    const cudaError_t q = cudaEventQuery(H->sv.ev);
    if (q == cudaErrorNotReady) return MA_OK;
    if (q != cudaSuccess) return fail(MA_ERR_CUDA, "ma_solve_advance: %s", cudaGetErrorString(q));
    if (absorb_norms(H)) {
        *done = 1;
        return MA_OK;
    }
    MA_CK(launch_cycle(H));
    MA_CK(queue_readback(H));
    H->sv.phase = 2;
    return MA_OK;
}

ma_status ma_solve_get_result(const ma_hierarchy* H, ma_solve_result* res)
{
    if (!H || !res) return fail(MA_ERR_INVALID_ARG, "null argument");
    if (H->sv.phase != 3) return fail(MA_ERR_INVALID_ARG, "solve not finished");
    *res = H->sv.r;
    const int out = H->sv.r.status;
    if (out == MA_ERR_NONFINITE) return fail(MA_ERR_NONFINITE, "residual became non-finite after %d cycles", res->cycles);
    if (out == MA_ERR_NOT_CONVERGED)
        return fail(MA_ERR_NOT_CONVERGED, "not converged: residual %.3e > tol %.3e after %d cycles%s", res->res,
                    H->sv.o.tol, res->cycles, res->floor_reached ? " (round-off floor)" : "");
    return MA_OK;
}

ma_status ma_solve(ma_hierarchy* H, const ma_solve_opts* opts, ma_solve_result* res)
{
    NvtxRange nv("ma_solve");
    if (!H || !opts || !res) return fail(MA_ERR_INVALID_ARG, "null argument");
    std::memset(res, 0, sizeof *res);
    ma_status st = ma_solve_begin(H, opts);
    if (st != MA_OK) return st;
    int done = 0;
    while (!done) {
        {
            DeviceGuard g(H->device);
            MA_CK(cudaEventSynchronize(H->sv.ev));
        }
        st = ma_solve_advance(H, &done);
        if (st != MA_OK) return st;
    }
    return ma_solve_get_result(H, res);
}

ma_status ma_batch_solve(ma_hierarchy* const* hs, int count, const ma_solve_opts* opts, ma_solve_result* results)
{
    NvtxRange nv("ma_batch_solve");
    if (!hs || count < 0 || !opts || (count > 0 && !results)) return fail(MA_ERR_INVALID_ARG, "null argument");
    for (int b = 0; b < count; ++b) {
        if (!hs[b]) return fail(MA_ERR_INVALID_ARG, "null hierarchy %d", b);
        std::memset(&results[b], 0, sizeof results[b]);
    }
    for (int b = 0; b < count; ++b) {
        ma_status st = ma_solve_begin(hs[b], opts);
        if (st != MA_OK) return st;
    }
    int remaining = count;
    std::vector<char> done(count, 0);
    while (remaining > 0) {
        int first_pending = -1;
        for (int b = 0; b < count; ++b) {
            if (done[b]) continue;
            int d = 0;
            ma_status st = ma_solve_advance(hs[b], &d);
            if (st != MA_OK) return st;
            if (d) {
                done[b] = 1;
                --remaining;
            } else if (first_pending < 0) {
                first_pending = b;
            }
        }
        if (first_pending >= 0) {   // wait for one pending read-back instead of spinning
            DeviceGuard g(hs[first_pending]->device);
            MA_CK(cudaEventSynchronize(hs[first_pending]->sv.ev));
        }
    }
    ma_status worst = MA_OK;
    for (int b = 0; b < count; ++b) {
        const ma_status st = ma_solve_get_result(hs[b], &results[b]);
        if (st != MA_OK && worst == MA_OK) worst = st;
    }
    return worst;
}

// ---- shared per-level batches ----------------------------------------------

}  // extern "C"

struct ma_batch_group {
    std::vector<int> ids;             // the hierarchies of this group (indices into the batch)
    ma::BatchPlan* plan = nullptr;
    cudaStream_t s = nullptr;         // group 0: the batch's stream; others: created here
    cudaStream_t cap = nullptr;       // private capture stream
    ma::GraphSlot gs;                 // the start: FMG and the first outer iteration
    ma::GraphSlot g;                  // one outer iteration of the group
    cudaEvent_t done = nullptr;
};

// The active flags and packed norms are held once per group (group q's
// slice starts at q * count flags and 5 q * count norms, indexed by the
// hierarchy's place in the batch), so that each group uploads its flags and
// reads its norms on its own stream while the other groups run.
struct ma_batch {
    std::vector<ma_hierarchy*> hs;
    int device = 0;
    cudaStream_t s = nullptr;        // the caller's stream
    int* active_dev = nullptr;       // per group and hierarchy: 1 while it iterates
    double* packed_dev = nullptr;    // per group and hierarchy: (max, L2, -, -, events) after an iteration
    int* active_host = nullptr;      // pinned, the same shape
    double* packed_host = nullptr;   // pinned, the same shape
    std::vector<ma_batch_group> grp;
    cudaEvent_t flags_ev = nullptr;
    cudaEvent_t done_ev = nullptr;
};

namespace {

std::atomic<int> g_batch_groups{2};
std::atomic<int> g_batch_start{0};   // 1: the start as batched launches; 0: each hierarchy's own start graph

ma_status batch_describe(ma_hierarchy* const* hs, int count, std::vector<ma::BatchInstance>* in,
                         ma::BatchParams* p)
{
    if (!hs || count < 1) return fail(MA_ERR_INVALID_ARG, "batch: need at least one hierarchy");
    in->assign(count, ma::BatchInstance());
    for (int b = 0; b < count; ++b) {
        const ma_hierarchy* H = hs[b];
        if (!H) return fail(MA_ERR_INVALID_ARG, "batch: null hierarchy %d", b);
        for (int c = 0; c < b; ++c)
            if (hs[c] == H) return fail(MA_ERR_INVALID_ARG, "batch: hierarchy %d appears twice", b);
        const ma_hier_desc& d = H->d;
        const ma_hier_desc& d0 = hs[0]->d;
        if (d.precision != MA_MIXED) return fail(MA_ERR_INVALID_ARG, "batch: hierarchy %d is not MA_MIXED", b);
        if (d.n > 1025) return fail(MA_ERR_INVALID_ARG, "batch: n = %d exceeds 1025", d.n);
        if (d.nu1 != d0.nu1 || d.nu2 != d0.nu2 || d.restrict_kind != d0.restrict_kind ||
            d.approx_restrict != d0.approx_restrict || d.coarse_sweeps != d0.coarse_sweeps ||
            d.inner_cycles != d0.inner_cycles || d.coarsest_n != d0.coarsest_n || d.fmg_interp != d0.fmg_interp ||
            H->device != hs[0]->device)
            return fail(MA_ERR_INVALID_ARG, "batch: hierarchy %d differs from hierarchy 0 in its cycle settings "
                                            "or device", b);
        ma::BatchInstance& I = (*in)[b];
        I.id = b;
        I.L = H->L;
        for (int l = 0; l < H->L; ++l) {
            const ma::Level& A = H->lev[l];
            ma::BatchLevel& V = I.lev[l];
            V.n = A.n;
            V.h = A.h;
            V.u = A.u;
            V.rhs = A.rhs;
            V.r = A.r;
            V.w = A.w;
            V.e = A.e;
            V.e2 = A.e2;
            V.res32 = A.res32;
            V.w32 = A.w32;
            V.hi = A.hi;
            V.lo = A.lo;
            V.rhs32 = A.rhs32;
            V.bstore = A.bstore;
        }
        I.partials = H->partials;
        I.npartials = H->npartials;
        I.out2 = H->out2;
        I.ref_out2 = H->rb + 2;
        I.events = H->events;
    }
    const ma_hier_desc& d0 = hs[0]->d;
    p->nu1 = d0.nu1;
    p->nu2 = d0.nu2;
    p->kind = d0.restrict_kind;
    p->approx = d0.approx_restrict;
    p->coarse_sweeps = d0.coarse_sweeps;
    p->inner = d0.inner_cycles > 0 ? d0.inner_cycles : 3;
    p->tail_max = ma::corr_tail_max_n();
    p->vtail_max = ma::vcycle_tail_max_n();
    p->fmg_interp = d0.fmg_interp;
    return MA_OK;
}

// Groups of the batch: the hierarchies by decreasing size, dealt in turn to
// min(count, batch groups) groups, so that the groups carry similar work.
std::vector<std::vector<int>> batch_grouping(const std::vector<ma::BatchInstance>& in)
{
    const int count = (int)in.size();
    const int G = std::max(1, std::min(count, g_batch_groups.load(std::memory_order_relaxed)));
    std::vector<int> order(count);
    for (int b = 0; b < count; ++b) order[b] = b;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return in[x].lev[0].n > in[y].lev[0].n; });
    std::vector<std::vector<int>> grp(G);
    for (int q = 0; q < count; ++q) grp[q % G].push_back(order[q]);
    return grp;
}

std::vector<ma::BatchInstance> subset(const std::vector<ma::BatchInstance>& in, const std::vector<int>& ids)
{
    std::vector<ma::BatchInstance> out;
    for (int b : ids) out.push_back(in[b]);
    return out;
}

// Workspace: active flags and packed norms (one slice per group), then the
// job tables of each group.
size_t batch_layout(const std::vector<ma::BatchInstance>& in, const ma::BatchParams& p,
                    const std::vector<std::vector<int>>& grp, size_t* off_packed, std::vector<size_t>* off_tables)
{
    const size_t count = in.size(), ng = grp.size();
    *off_packed = align_up(sizeof(int) * count * ng);
    size_t off = *off_packed + align_up(5 * sizeof(double) * count * ng);
    off_tables->clear();
    for (const std::vector<int>& ids : grp) {
        off_tables->push_back(off);
        const std::vector<ma::BatchInstance> sub = subset(in, ids);
        off += align_up(ma::batch_tables_bytes(sub.data(), (int)sub.size(), p));
    }
    return off;
}

// Replays the group's start (start = true) or outer-iteration graph on its
// stream, capturing it on first use.
cudaError_t group_replay(ma_batch_group& G, bool start)
{
    ma::GraphSlot& gs = start ? G.gs : G.g;
    if (!gs.exec) {
        const unsigned long long before = ma::launch_count();
        cudaError_t e = cudaStreamBeginCapture(G.cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        const cudaError_t eb = start ? ma::batch_plan_start(G.plan, G.cap) : ma::batch_plan_iteration(G.plan, G.cap);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(G.cap, &g);
        const unsigned long long captured = ma::launch_count() - before;
        ma::uncount_launches(captured);
        if (eb != cudaSuccess || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return eb != cudaSuccess ? eb : e;
        }
        e = cudaGraphInstantiate(&gs.exec, g, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            gs.exec = nullptr;
            return e;
        }
        gs.graph = g;
        gs.launches = captured;
    }
    ma::count_launches(gs.launches);
    return cudaGraphLaunch(gs.exec, G.s);
}

// Uploads group q's active flags, replays its start (start = true) or
// outer-iteration graph and reads its packed norms back, all on the group's
// stream, and records G.done after them.  Touches only the group's slices.
cudaError_t group_launch(ma_batch* B, int q, const std::vector<char>& done, bool start)
{
    ma_batch_group& G = B->grp[q];
    const size_t count = B->hs.size();
    int* ah = B->active_host + (size_t)q * count;
    for (int b : G.ids) ah[b] = done[b] ? 0 : 1;
    cudaError_t e =
        cudaMemcpyAsync(B->active_dev + (size_t)q * count, ah, sizeof(int) * count, cudaMemcpyHostToDevice, G.s);
    if (e == cudaSuccess) e = group_replay(G, start);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(B->packed_host + 5 * (size_t)q * count, B->packed_dev + 5 * (size_t)q * count,
                            5 * sizeof(double) * count, cudaMemcpyDeviceToHost, G.s);
    if (e == cudaSuccess) e = cudaEventRecord(G.done, G.s);
    return e;
}

}  // namespace

extern "C" {

ma_status ma_set_batch_groups(int groups)
{
    if (groups < 1 || groups > 16) return fail(MA_ERR_INVALID_ARG, "ma_set_batch_groups: %d not in [1, 16]", groups);
    g_batch_groups.store(groups, std::memory_order_relaxed);
    return MA_OK;
}

ma_status ma_set_batch_start(int batched)
{
    if (batched != 0 && batched != 1) return fail(MA_ERR_INVALID_ARG, "ma_set_batch_start: %d is not 0 or 1", batched);
    g_batch_start.store(batched, std::memory_order_relaxed);
    return MA_OK;
}

ma_status ma_batch_footprint(ma_hierarchy* const* hs, int count, size_t* bytes)
{
    if (!bytes) return fail(MA_ERR_INVALID_ARG, "null bytes");
    std::vector<ma::BatchInstance> in;
    ma::BatchParams p;
    ma_status st = batch_describe(hs, count, &in, &p);
    if (st != MA_OK) return st;
    size_t op;
    std::vector<size_t> ot;
    *bytes = batch_layout(in, p, batch_grouping(in), &op, &ot);
    return MA_OK;
}

ma_status ma_create_batch(ma_hierarchy* const* hs, int count, void* dev_workspace, size_t bytes, ma_stream_t stream,
                          ma_batch** out)
{
    if (!out) return fail(MA_ERR_INVALID_ARG, "null out");
    *out = nullptr;
    std::vector<ma::BatchInstance> in;
    ma::BatchParams p;
    ma_status st = batch_describe(hs, count, &in, &p);
    if (st != MA_OK) return st;
    if (!dev_workspace || ((uintptr_t)dev_workspace) % kAlign != 0)
        return fail(MA_ERR_INVALID_ARG, "batch workspace null or not 256-byte aligned");
    const std::vector<std::vector<int>> grouping = batch_grouping(in);
    size_t op;
    std::vector<size_t> ot;
    const size_t need = batch_layout(in, p, grouping, &op, &ot);
    if (bytes < need) return fail(MA_ERR_INVALID_ARG, "batch workspace of %zu bytes < footprint %zu", bytes, need);
    DeviceGuard g(hs[0]->device);
    ma_batch* B = new (std::nothrow) ma_batch();
    if (!B) return fail(MA_ERR_OOM, "host allocation failed");
    B->hs.assign(hs, hs + count);
    B->device = hs[0]->device;
    B->s = (cudaStream_t)stream;
    char* ws = (char*)dev_workspace;
    const size_t ng = grouping.size();
    B->active_dev = (int*)ws;
    B->packed_dev = (double*)(ws + op);
    B->grp.resize(ng);
    cudaError_t e = cudaMallocHost((void**)&B->active_host, sizeof(int) * (size_t)count * ng);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&B->packed_host, 5 * sizeof(double) * (size_t)count * ng);
    if (e == cudaSuccess) {
        std::memset(B->active_host, 0, sizeof(int) * (size_t)count * ng);
        std::memset(B->packed_host, 0, 5 * sizeof(double) * (size_t)count * ng);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->flags_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->done_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws, 0, ot.empty() ? 0 : ot[0], B->s);
    for (size_t q = 0; q < grouping.size() && e == cudaSuccess; ++q) {
        ma_batch_group& G = B->grp[q];
        G.ids = grouping[q];
        if (q == 0) G.s = B->s;
        else e = cudaStreamCreateWithFlags(&G.s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&G.cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&G.done, cudaEventDisableTiming);
        if (e != cudaSuccess) break;
        const std::vector<ma::BatchInstance> sub = subset(in, G.ids);
        G.plan = ma::batch_plan_create(sub.data(), (int)sub.size(), p, ws + ot[q], B->active_dev + q * (size_t)count,
                                       B->packed_dev + 5 * q * (size_t)count, B->s, &e);
        if (!G.plan && e == cudaSuccess) e = cudaErrorMemoryAllocation;
    }
    if (e != cudaSuccess) {
        ma_destroy_batch(B);
        return fail(MA_ERR_CUDA, "create batch: %s", cudaGetErrorString(e));
    }
    *out = B;
    return MA_OK;
}

ma_status ma_batch_run(ma_batch* B, const ma_solve_opts* opts, ma_solve_result* results)
{
    NvtxRange nv("ma_batch_run");
    if (!B || !opts || !results) return fail(MA_ERR_INVALID_ARG, "null argument");
    ma_status st = check_opts(opts);
    if (st != MA_OK) return st;
    const int count = (int)B->hs.size();
    const int ng = (int)B->grp.size();
    DeviceGuard g(B->device);
    std::vector<char> done(count, 0), started(count, 0);
    // per group: WAIT for its hierarchies' own start graphs, READY to launch,
    // START or ITER in flight (its batched start or an outer iteration), OVER
    enum { WAIT, READY, START, ITER, OVER };
    std::vector<int> state(ng, WAIT);
    auto packed = [&](int q, int b) { return B->packed_host + 5 * ((size_t)q * count + b); };
    if (g_batch_start.load(std::memory_order_relaxed) && opts->init == MA_INIT_FMG &&
        opts->relative != MA_REL_INITIAL) {
        // the start of every hierarchy (the norms of f, FMG, the first outer
        // iteration) as batched launches too
        for (int b = 0; b < count; ++b) {
            ma_hierarchy* H = B->hs[b];
            std::memset(&results[b], 0, sizeof results[b]);
            solve_state_reset(H, opts);
            MA_CK(cudaEventRecord(H->sv.ev, H->s));   // after the caller's work on the hierarchy
            MA_CK(cudaStreamWaitEvent(B->s, H->sv.ev, 0));
            MA_CK(cudaMemsetAsync(H->events, 0, sizeof(unsigned long long), B->s));
            started[b] = 1;
        }
        MA_CK(cudaEventRecord(B->flags_ev, B->s));
        for (int q = 0; q < ng; ++q) {
            ma_batch_group& G = B->grp[q];
            if (G.s != B->s) MA_CK(cudaStreamWaitEvent(G.s, B->flags_ev, 0));
            MA_CK(group_launch(B, q, done, true));
            state[q] = START;
        }
    } else {
        // other starts: every hierarchy's own start graph on its own stream
        for (int b = 0; b < count; ++b) {
            std::memset(&results[b], 0, sizeof results[b]);
            if ((st = ma_solve_begin(B->hs[b], opts)) != MA_OK) return st;
        }
    }
    // Each group advances on its own: its first outer iteration once its
    // hierarchies' starts are in, each next one once its own norms are back.
    for (;;) {
        bool all_over = true, moved = false;
        cudaEvent_t pending = nullptr;
        for (int q = 0; q < ng; ++q) {
            ma_batch_group& G = B->grp[q];
            if (state[q] == OVER) continue;
            all_over = false;
            if (state[q] == WAIT) {
                bool ready = true;
                for (int b : G.ids) {
                    if (started[b]) continue;
                    ma_hierarchy* H = B->hs[b];
                    const cudaError_t qe = cudaEventQuery(H->sv.ev);
                    if (qe == cudaErrorNotReady) {
                        ready = false;
                        if (!pending) pending = H->sv.ev;
                        continue;
                    }
                    MA_CK(qe);
                    started[b] = 1;
                    done[b] = absorb_norms(H) ? 1 : 0;
                    if (!done[b]) H->sv.phase = 2;
                }
                if (!ready) continue;
                for (int b : G.ids) MA_CK(cudaStreamWaitEvent(G.s, B->hs[b]->sv.ev, 0));
                state[q] = READY;
                moved = true;
            } else if (state[q] == START || state[q] == ITER) {
                const cudaError_t qe = cudaEventQuery(G.done);
                if (qe == cudaErrorNotReady) {
                    if (!pending) pending = G.done;
                    continue;
                }
                MA_CK(qe);
                for (int b : G.ids) {
                    if (done[b]) continue;
                    ma_hierarchy* H = B->hs[b];
                    const double* pk = packed(q, b);
                    if (state[q] == START) {
                        for (int k = 0; k < 5; ++k) H->host[k] = pk[k];
                        H->sv.phase = 1;
                    } else {
                        H->host[0] = pk[0];
                        H->host[1] = pk[1];
                        H->host[4] = pk[4];
                    }
                    done[b] = absorb_norms(H) ? 1 : 0;
                    if (!done[b]) H->sv.phase = 2;
                }
                state[q] = READY;
                moved = true;
            }
            if (state[q] == READY) {
                bool any = false;
                for (int b : G.ids) any = any || !done[b];
                if (!any) {
                    state[q] = OVER;
                } else {
                    MA_CK(group_launch(B, q, done, false));
                    state[q] = ITER;
                }
                moved = true;
            }
        }
        if (all_over) break;
        if (!moved && pending) MA_CK(cudaEventSynchronize(pending));   // wait instead of spinning
    }
    // later work on the caller's stream and on each hierarchy's own stream
    // follows the batch's
    for (int q = 0; q < ng; ++q)
        if (B->grp[q].s != B->s) MA_CK(cudaStreamWaitEvent(B->s, B->grp[q].done, 0));
    for (int b = 0; b < count; ++b) MA_CK(cudaStreamWaitEvent(B->s, B->hs[b]->sv.ev, 0));
    MA_CK(cudaEventRecord(B->done_ev, B->s));
    ma_status worst = MA_OK;
    for (int b = 0; b < count; ++b) {
        MA_CK(cudaStreamWaitEvent(B->hs[b]->s, B->done_ev, 0));
        const ma_status sb = ma_solve_get_result(B->hs[b], &results[b]);
        if (sb != MA_OK && worst == MA_OK) worst = sb;
    }
    return worst;
}

ma_status ma_destroy_batch(ma_batch* B)
{
    if (!B) return MA_OK;
    DeviceGuard g(B->device);
    cudaError_t e = cudaSuccess;
    for (ma_batch_group& G : B->grp) {
        if (G.s) {
            const cudaError_t es = cudaStreamSynchronize(G.s);
            if (e == cudaSuccess) e = es;
        }
        if (G.g.exec) cudaGraphExecDestroy(G.g.exec);
        if (G.g.graph) cudaGraphDestroy(G.g.graph);
        if (G.gs.exec) cudaGraphExecDestroy(G.gs.exec);
        if (G.gs.graph) cudaGraphDestroy(G.gs.graph);
        if (G.cap) cudaStreamDestroy(G.cap);
        if (G.s && G.s != B->s) cudaStreamDestroy(G.s);
        if (G.done) cudaEventDestroy(G.done);
        ma::batch_plan_destroy(G.plan);
    }
    if (B->flags_ev) cudaEventDestroy(B->flags_ev);
    if (B->done_ev) cudaEventDestroy(B->done_ev);
    if (B->active_host) cudaFreeHost(B->active_host);
    if (B->packed_host) cudaFreeHost(B->packed_host);
    delete B;
    if (e != cudaSuccess) return fail(MA_ERR_CUDA, "destroy batch: %s", cudaGetErrorString(e));
    return MA_OK;
}

// ---- single steps ----------------------------------------------------------

ma_status ma_smooth(double* u, const double* rhs, int n, double h, int nsweeps, unsigned long long* events,
                    ma_stream_t stream)
{
    if (!u || !rhs || !valid_step_grid(n) || !(h > 0.0) || nsweeps < 0)
        return fail(MA_ERR_INVALID_ARG, "ma_smooth: bad arguments");
    MA_CK(ma::launch_smooth(u, rhs, n, h, nsweeps, events, (cudaStream_t)stream));
    return MA_OK;
}

ma_status ma_residual(const double* u, const double* rhs, double* r, int n, double h, ma_stream_t stream)
{
    if (!u || !rhs || !r || !valid_step_grid(n) || !(h > 0.0)) return fail(MA_ERR_INVALID_ARG, "ma_residual: bad arguments");
    MA_CK(ma::launch_residual(u, rhs, r, n, h, nullptr, (cudaStream_t)stream));
    return MA_OK;
}

ma_status ma_residual_f2(const double* u, const double* rhs, double* r, int n, double h, ma_stream_t stream)
{
    if (!u || !rhs || !r || !valid_step_grid(n) || !(h > 0.0))
        return fail(MA_ERR_INVALID_ARG, "ma_residual_f2: bad arguments");
    MA_CK(ma::launch_residual_f2(u, rhs, r, n, h, (cudaStream_t)stream));
    return MA_OK;
}

ma_status ma_restrict_residual(const double* rf, int nf, double* rc, int kind, ma_stream_t stream)
{
    if (!rf || !rc || !valid_step_grid(nf) || nf < 5 || (kind != MA_HALF_WEIGHTING && kind != MA_FULL_WEIGHTING))
        return fail(MA_ERR_INVALID_ARG, "ma_restrict_residual: bad arguments");
    MA_CK(ma::launch_restrict_residual(rf, nf, rc, kind, (cudaStream_t)stream));
    return MA_OK;
}

ma_status ma_restrict_solution(const double* uf, int nf, double* uc, int approx, int kind, ma_stream_t stream)
{
    if (!uf || !uc || !valid_step_grid(nf) || nf < 5 || (kind != MA_HALF_WEIGHTING && kind != MA_FULL_WEIGHTING) ||
        (approx != MA_APPROX_INJECTION && approx != MA_APPROX_WEIGHTED))
        return fail(MA_ERR_INVALID_ARG, "ma_restrict_solution: bad arguments");
    MA_CK(ma::launch_restrict_solution(uf, nf, uc, approx, kind, (cudaStream_t)stream));
    return MA_OK;
}

ma_status ma_coarse_rhs(const double* wc, const double* rc, double* bc, int nc, double Hs, ma_stream_t stream)
{
    if (!wc || !rc || !bc || !valid_step_grid(nc) || !(Hs > 0.0))
        return fail(MA_ERR_INVALID_ARG, "ma_coarse_rhs: bad arguments");
    MA_CK(ma::launch_coarse_rhs(wc, rc, bc, nc, Hs, (cudaStream_t)stream));
    return MA_OK;
}

ma_status ma_prolong_add(const double* uc, const double* wc, int nc, double* uf, ma_stream_t stream)
{
    if (!uc || !wc || !uf || !valid_step_grid(nc)) return fail(MA_ERR_INVALID_ARG, "ma_prolong_add: bad arguments");
    MA_CK(ma::launch_prolong_add(uc, wc, nc, uf, (cudaStream_t)stream));
    return MA_OK;
}

ma_status ma_interpolate(const double* uc, int nc, double* uf, ma_stream_t stream)
{
    if (!uc || !uf || !valid_step_grid(nc)) return fail(MA_ERR_INVALID_ARG, "ma_interpolate: bad arguments");
    MA_CK(ma::launch_interpolate(uc, nc, uf, (cudaStream_t)stream));
    return MA_OK;
}

ma_status ma_coarsest_solve(double* u, const double* rhs, int n, double h, int sweeps, unsigned long long* events,
                            ma_stream_t stream)
{
    if (!u || !rhs || !valid_step_grid(n) || n > 17 || !(h > 0.0) || sweeps < 0 || sweeps > 1000)
        return fail(MA_ERR_INVALID_ARG, "ma_coarsest_solve: bad arguments (n <= 17)");
    MA_CK(ma::prepare_kernels());
    MA_CK(ma::launch_coarsest(u, rhs, n, h, sweeps, events, (cudaStream_t)stream));
    return MA_OK;
}

ma_status ma_interpolate_cubic_scratch_bytes(int nc, size_t* bytes)
{
    if (!bytes || nc < 3 || nc > 2049) return fail(MA_ERR_INVALID_ARG, "ma_interpolate_cubic_scratch_bytes: bad arguments");
    *bytes = ma::interpolate_cubic_scratch(nc);
    return MA_OK;
}

ma_status ma_interpolate_cubic(const double* uc, int nc, double* uf, void* scratch, size_t scratch_bytes,
                               ma_stream_t stream)
{
    if (!uc || !uf || !scratch || nc < 3 || nc > 2049 || ((uintptr_t)scratch) % 8 != 0)
        return fail(MA_ERR_INVALID_ARG, "ma_interpolate_cubic: bad arguments");
    if (scratch_bytes < ma::interpolate_cubic_scratch(nc))
        return fail(MA_ERR_INVALID_ARG, "ma_interpolate_cubic: scratch %zu < %zu bytes", scratch_bytes,
                    ma::interpolate_cubic_scratch(nc));
    MA_CK(ma::launch_interpolate_cubic(uc, nc, uf, (double*)scratch, (cudaStream_t)stream));
    return MA_OK;
}

// Scratch of the correction step calls: the FP32 base-Hessian store, the
// colour-major right-hand side, and the second e buffer of the plane sweeps
// (each 256-byte aligned).
static size_t corr_scratch_rhs(int n) { return align_up(ma::base_store_bytes(n)); }
static size_t corr_scratch_e2(int n) { return corr_scratch_rhs(n) + align_up(ma::cm_points(n) * sizeof(float)); }

ma_status ma_correction_scratch_bytes(int n, size_t* bytes)
{
    if (!valid_step_grid(n) || !bytes) return fail(MA_ERR_INVALID_ARG, "ma_correction_scratch_bytes: bad arguments");
    *bytes = corr_scratch_e2(n) + (size_t)n * n * n * sizeof(float);
    return MA_OK;
}

static ma_status corr_setup(const float* hi, const float* lo, const float* rhs, int n, double h, void* scratch,
                            size_t scratch_bytes, cudaStream_t s, float** rhs_cm)
{
    size_t need = 0;
    ma_status st = ma_correction_scratch_bytes(n, &need);
    if (st != MA_OK) return st;
    if (scratch_bytes < need) return fail(MA_ERR_INVALID_ARG, "correction scratch %zu < %zu bytes", scratch_bytes, need);
    if (((uintptr_t)scratch) % kAlign != 0) return fail(MA_ERR_INVALID_ARG, "scratch not 256-byte aligned");
    MA_CK(ma::prepare_kernels());
    *rhs_cm = (float*)((char*)scratch + corr_scratch_rhs(n));
    MA_CK(ma::launch_base_colour(hi, lo, scratch, n, h, s));
    MA_CK(ma::launch_to_cm(rhs, *rhs_cm, n, s));
    return MA_OK;
}

ma_status ma_smooth_correction(float* e, const float* hi, const float* lo, const float* rhs, int n, double h,
                               int nsweeps, void* scratch, size_t scratch_bytes, unsigned long long* events,
                               ma_stream_t stream)
{
    if (!e || !scratch || !hi || !lo || !rhs || !valid_step_grid(n) || !(h > 0.0) || nsweeps < 0)
        return fail(MA_ERR_INVALID_ARG, "ma_smooth_correction: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    float* rhs_cm = nullptr;
    ma_status st = corr_setup(hi, lo, rhs, n, h, scratch, scratch_bytes, s, &rhs_cm);
    if (st != MA_OK) return st;
    float* e2 = (float*)((char*)scratch + corr_scratch_e2(n));
    MA_CK(cudaMemsetAsync(e2, 0, (size_t)n * n * n * sizeof(float), s));
    MA_CK(ma::launch_smooth_corr(e, e2, scratch, rhs_cm, n, h, nsweeps, events, s));
    return MA_OK;
}

ma_status ma_smooth_correction_colour(float* e, const float* hi, const float* lo, const float* rhs, int n, double h,
                                      int colour, void* scratch, size_t scratch_bytes, unsigned long long* events,
                                      ma_stream_t stream)
{
    if (!e || !scratch || !hi || !lo || !rhs || !valid_step_grid(n) || !(h > 0.0) || colour < 0 || colour > 7)
        return fail(MA_ERR_INVALID_ARG, "ma_smooth_correction_colour: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    float* rhs_cm = nullptr;
    ma_status st = corr_setup(hi, lo, rhs, n, h, scratch, scratch_bytes, s, &rhs_cm);
    if (st != MA_OK) return st;
    MA_CK(ma::launch_smooth_corr_colour(colour, e, scratch, rhs_cm, n, h, events, s));
    return MA_OK;
}

ma_status ma_residual_correction(const float* e, const float* hi, const float* lo, const float* rhs, float* res,
                                 int n, double h, void* scratch, size_t scratch_bytes, ma_stream_t stream)
{
    if (!e || !hi || !lo || !rhs || !res || !scratch || !valid_step_grid(n) || !(h > 0.0))
        return fail(MA_ERR_INVALID_ARG, "ma_residual_correction: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    float* rhs_cm = nullptr;
    ma_status st = corr_setup(hi, lo, rhs, n, h, scratch, scratch_bytes, s, &rhs_cm);
    if (st != MA_OK) return st;
    MA_CK(ma::launch_zero_shell_f32(res, n, s));
    MA_CK(ma::launch_residual_corr(e, scratch, rhs_cm, res, n, h, s));
    return MA_OK;
}

ma_status ma_set_corr_tail(int max_n)
{
    if (!ma::set_corr_tail(max_n)) return fail(MA_ERR_INVALID_ARG, "ma_set_corr_tail: bad value %d", max_n);
    return MA_OK;
}

ma_status ma_set_vcycle_tail(int max_n)
{
    if (!ma::set_vcycle_tail(max_n)) return fail(MA_ERR_INVALID_ARG, "ma_set_vcycle_tail: bad value %d", max_n);
    return MA_OK;
}

ma_status ma_set_corr_tuning(int n, int smooth_choice, int residual_choice)
{
    if (smooth_choice < -1 || smooth_choice == MA_CORR_COLUMN || smooth_choice > MA_CORR_PAIRS ||
        residual_choice < -1 || residual_choice == MA_CORR_BY_COLOUR || residual_choice > MA_CORR_COLUMN)
        return fail(MA_ERR_INVALID_ARG, "ma_set_corr_tuning: bad choice (%d, %d)", smooth_choice, residual_choice);
    if (!ma::set_corr_tuning(n, smooth_choice, residual_choice))
        return fail(MA_ERR_INVALID_ARG, "ma_set_corr_tuning: n = %d is not an odd size in [3, 4097]", n);
    return MA_OK;
}

ma_status ma_get_corr_tuning(int n, int* smooth_choice, int* residual_choice)
{
    if (!valid_step_grid(n)) return fail(MA_ERR_INVALID_ARG, "ma_get_corr_tuning: bad n %d", n);
    if (smooth_choice) *smooth_choice = ma::corr_smooth_choice(n);
    if (residual_choice) *residual_choice = ma::corr_resid_choice(n);
    return MA_OK;
}

// reps calls of launch(stream) timed as hierarchies run them: captured once
// into a CUDA graph on the private stream cap and replayed on s.  Inside a
// graph a dependent launch costs ~1 us against ~4 us for a stream launch, so
// timing stream launches would favour the variants with fewer launches on
// small grids.  The fastest of 3 replays after a warm-up one, in
// microseconds per call.
extern "C++" template <typename F>
cudaError_t graph_us(cudaStream_t s, cudaStream_t cap, int reps, cudaEvent_t t0, cudaEvent_t t1, F launch,
                            double* us)
{
    const unsigned long long before = ma::launch_count();
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t eb = cudaSuccess;
    for (int r = 0; r < reps && eb == cudaSuccess; ++r) eb = launch(cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cap, &g);
    const unsigned long long captured = ma::launch_count() - before;
    ma::uncount_launches(captured);   // captured, not run
    if (eb != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return eb != cudaSuccess ? eb : e;
    }
    cudaGraphExec_t ge = nullptr;
    e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return e;
    float best = 3.4e38f;
    for (int r = 0; r < 4 && e == cudaSuccess; ++r) {
        ma::count_launches(captured);
        e = cudaEventRecord(t0, s);
        if (e == cudaSuccess) e = cudaGraphLaunch(ge, s);
        if (e == cudaSuccess) e = cudaEventRecord(t1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (e == cudaSuccess && r > 0 && ms < best) best = ms;
    }
    cudaGraphExecDestroy(ge);
    if (e == cudaSuccess) *us = 1e3 * best / reps;
    return e;
}

ma_status ma_tune_corr(float* e, const float* hi, const float* lo, const float* rhs, int n, double h, int reps,
                       void* scratch, size_t scratch_bytes, double* us_smooth, double* us_residual,
                       ma_stream_t stream)
{
    if (!e || !scratch || !hi || !lo || !rhs || !valid_step_grid(n) || n < 5 || !(h > 0.0) || reps < 1 ||
        reps > 1000)
        return fail(MA_ERR_INVALID_ARG, "ma_tune_corr: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    float* rhs_cm = nullptr;
    ma_status st = corr_setup(hi, lo, rhs, n, h, scratch, scratch_bytes, s, &rhs_cm);
    if (st != MA_OK) return st;
    float* e2 = (float*)((char*)scratch + corr_scratch_e2(n));
    MA_CK(cudaMemsetAsync(e2, 0, (size_t)n * n * n * sizeof(float), s));
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaStream_t cap = nullptr;
    MA_CK(cudaEventCreate(&t0));
    cudaError_t ce = cudaEventCreate(&t1);
    if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    double ts[6] = {0, 0, 0, 0, 0, 0}, tr[5] = {0, 0, 0, 0, 0};
    for (int c = MA_CORR_BY_COLOUR; c <= MA_CORR_PAIRS && ce == cudaSuccess; ++c) {
        if (c == MA_CORR_COLUMN) continue;
        double us = 0.0;   // per call of 2 sweeps
        ce = graph_us(s, cap, reps, t0, t1,
                      [&](cudaStream_t q) {
                          return ma::launch_smooth_corr_choice(c, e, e2, scratch, rhs_cm, n, h, 2, nullptr, q);
                      },
                      &us);
        ts[c] = us / 2.0;
    }
    // the residual writes into the second buffer's interior (its shell stays 0)
    for (int c = MA_CORR_PLANE16; c <= MA_CORR_COLUMN && ce == cudaSuccess; ++c) {
        double us = 0.0;
        ce = graph_us(s, cap, reps, t0, t1,
                      [&](cudaStream_t q) { return ma::launch_residual_corr_choice(c, e, scratch, rhs_cm, e2, n, h, q); },
                      &us);
        tr[c] = us;
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (cap) cudaStreamDestroy(cap);
    if (ce != cudaSuccess) return fail(MA_ERR_CUDA, "ma_tune_corr: %s", cudaGetErrorString(ce));
    int bs = MA_CORR_BY_COLOUR, br = MA_CORR_PLANE16;
    for (int c = 1; c <= MA_CORR_PAIRS; ++c)
        if (c != MA_CORR_COLUMN && ts[c] < ts[bs]) bs = c;
    for (int c = MA_CORR_PLANE32; c <= MA_CORR_COLUMN; ++c)
        if (tr[c] < tr[br]) br = c;
    ma::set_corr_tuning(n, bs, br);
    for (int c = 0; c < 6; ++c) {
        if (us_smooth) us_smooth[c] = ts[c];
        if (us_residual && c < 5) us_residual[c] = tr[c];
    }
    return MA_OK;
}

ma_status ma_norm_scratch_bytes(int n, size_t* bytes)
{
    if (!valid_step_grid(n) || !bytes) return fail(MA_ERR_INVALID_ARG, "ma_norm_scratch_bytes: bad arguments");
    *bytes = (2 * (size_t)ma::norm_partial_count(n) + 2) * sizeof(double);
    return MA_OK;
}

ma_status ma_norm(const double* v, int n, double h, void* scratch, size_t scratch_bytes, double* out_host,
                  ma_stream_t stream)
{
    size_t need = 0;
    if (!v || !scratch || !out_host || !(h > 0.0) || ma_norm_scratch_bytes(n, &need) != MA_OK)
        return fail(MA_ERR_INVALID_ARG, "ma_norm: bad arguments");
    if (scratch_bytes < need) return fail(MA_ERR_INVALID_ARG, "ma_norm: scratch %zu < %zu bytes", scratch_bytes, need);
    cudaStream_t s = (cudaStream_t)stream;
    double* partials = (double*)scratch;
    const int count = ma::norm_partial_count(n);
    double* out2 = partials + 2 * (size_t)count;
    MA_CK(ma::launch_norm_partials(v, n, partials, s));
    MA_CK(ma::launch_norm_final(partials, count, h, out2, s));
    MA_CK(cudaMemcpyAsync(out_host, out2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    MA_CK(cudaStreamSynchronize(s));
    return MA_OK;
}

}  // extern "C"
