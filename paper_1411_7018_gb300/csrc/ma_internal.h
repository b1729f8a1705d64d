// ma_internal.h -- launchers shared by the C-ABI layer (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace ma {

// Kernel launches issued by this library in this process (all devices).
void count_launches(unsigned long long k);
void uncount_launches(unsigned long long k);
// Sets the coarsest-grid kernels' shared-memory limits for grids up to n = 17
// (call outside stream capture).
cudaError_t prepare_coarsest_kernels();
unsigned long long launch_count();

// Sets the thread-local text ma_last_error_string() returns.
void set_last_error(const char* msg);

// FP64 kernels (ma_kernels_f64.cu).  All grids are n^3 doubles, [k][j][i].
cudaError_t launch_smooth(double* u, const double* rhs, int n, double h, int nsweeps,
                          unsigned long long* events, cudaStream_t s);
cudaError_t launch_residual(const double* u, const double* rhs, double* r, int n, double h,
                            double* partials, cudaStream_t s);
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
cudaError_t launch_inject(const double* vf, int nf, double* vc, cudaStream_t s);
cudaError_t launch_zero_interior(double* u, int n, cudaStream_t s);
cudaError_t launch_coarsest(double* u, const double* rhs, int n, double h, int sweeps,
                            unsigned long long* events, cudaStream_t s);
cudaError_t launch_copy_rhs_bc(const double* f, const double* g, double* rhs, double* u, int n,
                               int* bad, cudaStream_t s);

// Mixed-precision kernels (ma_kernels_mixed.cu).  e, res, w are n^3 floats
// in the natural layout; hi + lo is the FP32 split of the FP64 iterate; the
// base Hessian store (BF16, base_store_bytes) and the correction right-hand
// side (cm_points floats) are in colour-major order.
size_t base_store_bytes(int n);
size_t cm_points(int n);
cudaError_t launch_base_colour(const float* hi, const float* lo, void* bstore, int n, double h, cudaStream_t s);
cudaError_t launch_to_cm(const float* nat, float* cm, int n, cudaStream_t s);
cudaError_t launch_smooth_corr(float* e, const void* bstore, const float* rhs_cm, int n, double h, int nsweeps,
                               unsigned long long* events, cudaStream_t s);
cudaError_t launch_residual_corr(const float* e, const void* bstore, const float* rhs_cm, float* res, int n,
                                 double h, cudaStream_t s);
cudaError_t launch_coarse_rhs_corr(const float* w, const void* bstore, const float* resc, float* rhs_cm, int nc,
                                   double H, cudaStream_t s);
cudaError_t launch_restrict_level_f32(const float* ef, const float* rf, int nf, float* wc, float* ec, float* rc,
                                      int kind, int approx, cudaStream_t s);
cudaError_t launch_prolong_add_f32(const float* ec, const float* wc, int nc, float* ef, cudaStream_t s);
cudaError_t launch_inject_f32(const float* vf, int nf, float* vc, cudaStream_t s);
cudaError_t launch_coarsest_corr(float* e, const void* bstore, const float* rhs_cm, int n, double h, int sweeps,
                                 unsigned long long* events, cudaStream_t s);
cudaError_t launch_split_update(double* u, float* e, float* hi, float* lo, int n, int apply, cudaStream_t s);
cudaError_t launch_residual64_to32(const double* u, const double* rhs, float* r_cm, int n, double h,
                                   double* partials, cudaStream_t s);

}  // namespace ma
