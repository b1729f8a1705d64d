// ma_internal.h -- launchers shared by the C-ABI layer (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include <functional>
#include <utility>
#include <vector>

namespace ma {

// Kernel launches issued by this library in this process (all devices).
void count_launches(unsigned long long k);
void uncount_launches(unsigned long long k);
// Sets the shared-memory limits of the kernels that need more than 48 KB
// (coarsest-grid solves up to n = 17, the 64-point plane tiles); call
// outside stream capture, once per device.
cudaError_t prepare_kernels();
unsigned long long launch_count();

// Sets the thread-local text ma_last_error_string() returns.
void set_last_error(const char* msg);

// FP64 kernels (ma_kernels_f64.cu).  All grids are n^3 doubles, [k][j][i].
cudaError_t launch_smooth(double* u, const double* rhs, int n, double h, int nsweeps,
                          unsigned long long* events, cudaStream_t s);
cudaError_t launch_residual(const double* u, const double* rhs, double* r, int n, double h,
                            double* partials, cudaStream_t s);
// The same residual with exact integer second differences and a two-float
// determinant (no FP64 arithmetic where a point's stencil lies in one binade).
cudaError_t launch_residual_f2(const double* u, const double* rhs, double* r, int n, double h, cudaStream_t s);
int residual_partial_count(int n);
cudaError_t launch_norm_partials(const double* v, int n, double* partials, cudaStream_t s);
int norm_partial_count(int n);
cudaError_t launch_norm_final(const double* partials, int count, double h, double* out2, cudaStream_t s);
cudaError_t launch_restrict_residual(const double* rf, int nf, double* rc, int kind, cudaStream_t s);
cudaError_t launch_restrict_solution(const double* uf, int nf, double* uc, int approx, int kind,
                                     cudaStream_t s);
cudaError_t launch_restrict_level(const double* uf, const double* rf, int nf, double* wc, double* uc, double* rc,
                                  int kind, int approx, cudaStream_t s);
cudaError_t launch_coarse_rhs(const double* wc, const double* rc, double* bc, int nc, double H,
                              cudaStream_t s);
cudaError_t launch_prolong_add(const double* uc, const double* wc, int nc, double* uf, cudaStream_t s);
cudaError_t launch_interpolate(const double* uc, int nc, double* uf, cudaStream_t s);
size_t interpolate_cubic_scratch(int nc);
cudaError_t launch_interpolate_cubic(const double* uc, int nc, double* uf, double* scratch, cudaStream_t s);
cudaError_t launch_inject(const double* vf, int nf, double* vc, cudaStream_t s);
cudaError_t launch_zero_interior(double* u, int n, cudaStream_t s);
cudaError_t launch_coarsest(double* u, const double* rhs, int n, double h, int sweeps,
                            unsigned long long* events, cudaStream_t s);
cudaError_t launch_copy_rhs_bc(const double* f, const double* g, double* rhs, double* u, int n,
                               int* bad, cudaStream_t s);
// One FP64 V-cycle over the levels with n <= vcycle_tail_max_n() (the first
// entry is the level the cycle enters there, the last the coarsest grid), in
// one single-block launch; the coarse levels' u, w, r, rhs stay on chip.
struct TailSpec64 {
    int n;
    double h;
    double* u;
    const double* rhs;
};
int vcycle_tail_max_n();          // 0 when the fused tail is switched off
bool set_vcycle_tail(int max_n);  // 0 off, 1 default, or 3 / 5 / 9 / 17; false otherwise
cudaError_t launch_vcycle_tail(const TailSpec64* lv, int nlev, int nu1, int nu2, int kind, int approx,
                               int coarse_sweeps, unsigned long long* events, cudaStream_t s);

// Mixed-precision kernels (ma_kernels_mixed.cu).  e, res, w are n^3 floats
// in the natural layout; hi + lo is the FP32 split of the FP64 iterate; the
// base Hessian store (FP32, six per interior point, base_store_bytes) and the
// correction right-hand side (cm_points floats) are in colour-major order.
size_t base_store_bytes(int n);
size_t cm_points(int n);
cudaError_t launch_base_colour(const float* hi, const float* lo, void* bstore, int n, double h, cudaStream_t s);
cudaError_t launch_to_cm(const float* nat, float* cm, int n, cudaStream_t s);
// nsweeps 8-colour sweeps; pairs of sweeps run by k parity through the second
// buffer e2 (n^3 floats, zero shell; null: every sweep by colour in place).
cudaError_t launch_smooth_corr(float* e, float* e2, const void* bstore, const float* rhs_cm, int n, double h,
                               int nsweeps, unsigned long long* events, cudaStream_t s);
cudaError_t launch_zero_shell_f32(float* v, int n, cudaStream_t s);
// Correction-smoother and residual variants (values of MA_CORR_* in ma.h) and
// the per-size choice table the launchers above consult.
constexpr int CORR_BY_COLOUR = 0, CORR_PLANE16 = 1, CORR_PLANE32 = 2, CORR_PLANE64 = 3;
constexpr int CORR_COLUMN = 4;   // residual only
constexpr int CORR_PAIRS = 5;    // smoother only: colours c and c^7 per launch
// FP32 correction V-cycles of each FMG level below the finest in a mixed solve
// (the FP64 V-cycle of Algorithm 2 step 5 there); solo and batched starts alike.
constexpr int kFmgCorrCycles = 2;
// Round-off floor of the stopping rule: this many cycles in a row that each
// cut the residual by less than 20 % end a solve as "floor reached".  Two:
// on every floor-limited solve measured (513^3 mixed and FP64, 257^3 FP64,
// the FP32 mode) a third such cycle left the error against the exact
// solution unchanged to seven digits.
constexpr int kFloorStagnantCycles = 2;
int corr_smooth_choice(int n);
int corr_resid_choice(int n);
bool set_corr_tuning(int n, int smooth, int resid);   // -1: built-in default; false unless n is odd in [3, 4097]
// One colour phase (colour 0..7) of the by-colour correction sweep, in place.
cudaError_t launch_smooth_corr_colour(int colour, float* e, const void* bstore, const float* rhs_cm, int n, double h,
                                      unsigned long long* events, cudaStream_t s);
cudaError_t launch_smooth_corr_choice(int choice, float* e, float* e2, const void* bstore, const float* rhs_cm, int n,
                                      double h, int nsweeps, unsigned long long* events, cudaStream_t s);
// One correction V-cycle over the levels with n <= corr_tail_max_n() (the
// first entry is the level the cycle enters there, the last the coarsest
// grid), in one single-block launch.
struct TailSpec {
    int n;
    double h;
    float* e;
    const void* bstore;
    const float* rhs_cm;
};
int corr_tail_max_n();            // 0 when the fused tail is switched off
bool set_corr_tail(int max_n);     // 0 off, 1 default, or 3 / 5 / 9 / 17; false otherwise
cudaError_t launch_corr_vcycle_tail(const TailSpec* lv, int nlev, int nu1, int nu2, int kind, int approx,
                                    int coarse_sweeps, unsigned long long* events, cudaStream_t s);
cudaError_t launch_residual_corr_choice(int choice, const float* e, const void* bstore, const float* rhs_cm,
                                        float* res, int n, double h, cudaStream_t s);
cudaError_t launch_residual_corr(const float* e, const void* bstore, const float* rhs_cm, float* res, int n,
                                 double h, cudaStream_t s);
cudaError_t launch_coarse_rhs_corr(const float* w, const void* bstore, const float* resc, float* rhs_cm, int nc,
                                   double H, cudaStream_t s);
cudaError_t launch_restrict_level_f32(const float* ef, const float* rf, int nf, float* wc, float* ec, float* rc,
                                      int kind, int approx, cudaStream_t s);
cudaError_t launch_prolong_add_f32(const float* ec, const float* wc, int nc, float* ef, cudaStream_t s);
cudaError_t launch_coarsest_corr(float* e, const void* bstore, const float* rhs_cm, int n, double h, int sweeps,
                                 unsigned long long* events, cudaStream_t s);
cudaError_t launch_update(double* u, float* e, int n, int apply, cudaStream_t s);
// FP32 mode (the correction machinery with B = 0 on the solution itself)
cudaError_t launch_f64_to_f32(const double* u, float* e, int n, cudaStream_t s);
cudaError_t launch_f32_to_f64(const float* e, double* u, int n, cudaStream_t s);
cudaError_t launch_interpolate_f32(const float* ec, int nc, float* ef, cudaStream_t s);
cudaError_t launch_zero_interior_f32(float* e, int n, cudaStream_t s);
cudaError_t launch_norm_partials_f32(const float* v, int n, double* partials, cudaStream_t s);
cudaError_t launch_split_inject(const double* u0, int n0, int stride, float* hi, float* lo, int nc, cudaStream_t s);
cudaError_t launch_residual64_to32(const double* u, const double* rhs, float* r_cm, void* bstore, int n, double h,
                                   double* partials, cudaStream_t s);

// Batched launches (ma_kernels_mixed.cu).  One outer iteration of the mixed-
// precision solve -- `inner` FP32 correction V-cycles, the update u += e with
// the coarse base refresh, the FP64 fine residual and its norms -- for several
// hierarchies of any sizes, as one launch per kernel and level depth over all
// of them: a block finds its hierarchy in a job table, and hierarchies whose
// active flag is 0 are skipped.  Every hierarchy runs exactly the per-point
// operations of its own cycle, so the results are those of solving it alone.
constexpr int kBatchMaxLevels = 16;
struct BatchLevel {
    int n;
    double h;
    double *u, *rhs, *r, *w;   // FP64 fields of the level (iterate, right-hand side, residual, restriction)
    float *e, *e2, *res32, *w32, *hi, *lo, *rhs32;   // e2: second buffer of the plane sweeps (null on the coarsest level)
    void* bstore;
};
struct BatchInstance {
    int id;                // index of the hierarchy in the batch (active flags, packed norms)
    int L;
    BatchLevel lev[kBatchMaxLevels];
    double* partials;      // norm partials of the fine residual
    int npartials;
    double* out2;          // the hierarchy's (max, L2) residual norms
    double* ref_out2;      // the (max, L2) norms of f, the stopping rule's reference
    unsigned long long* events;
};
struct BatchParams {
    int nu1, nu2, kind, approx, coarse_sweeps, inner;
    int tail_max;          // largest level of the fused correction tail
    int vtail_max;         // largest level of the fused FP64 tail (the FMG V-cycles)
    int fmg_interp;        // MA_FMG_TRILINEAR | MA_FMG_CUBIC
};
struct BatchPlan;
namespace batched {
struct BLaunch;
struct TableBuilder;
}  // namespace batched
// The FP64 part of the batched start (ma_kernels_f64.cu): the partials of
// the norms of f, and the FMG pass of Algorithm 2 with its FP64 V-cycles
// below the finest level, all hierarchies sharing the coarsest grid size so
// that every FMG step runs on one level size; and the launcher of its ops.
void emit_rhs_partials_f64(batched::TableBuilder& T, const BatchInstance* in, int count);
// level_step, when given, replaces the FP64 V-cycle of each FMG level below
// the finest: it receives (instance index, level) for the instances that
// have that level.
void emit_fmg_f64(batched::TableBuilder& T, const BatchInstance* in, int count, const BatchParams& p,
                  const std::function<void(const std::vector<std::pair<int, int>>&)>& level_step = nullptr);
cudaError_t batch_launch_f64(const char* tables, const batched::BLaunch& L, const int* active, cudaStream_t s);
// Bytes of the device job tables of a batch.
size_t batch_tables_bytes(const BatchInstance* in, int count, const BatchParams& p);
// Builds the job tables into tables_dev (batch_tables_bytes, 256-byte
// aligned; uploaded on s, which is synchronised) and returns the plan, or null
// with *err set.  active_dev: count ints; packed_dev: 5 doubles per instance,
// where each iteration leaves (max, L2, -, -, events).
BatchPlan* batch_plan_create(const BatchInstance* in, int count, const BatchParams& p, void* tables_dev,
                             const int* active_dev, double* packed_dev, cudaStream_t s, cudaError_t* err);
// The start (FMG, the first outer iteration and the norms) of every hierarchy;
// one outer iteration of every active hierarchy.
cudaError_t batch_plan_start(const BatchPlan* plan, cudaStream_t s);
cudaError_t batch_plan_iteration(const BatchPlan* plan, cudaStream_t s);
void batch_plan_destroy(BatchPlan* plan);

}  // namespace ma
