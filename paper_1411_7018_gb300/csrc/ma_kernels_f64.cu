// ma_kernels_f64.cu -- FP64 kernels of the FAS V-cycle (Algorithm 1 of Liu,
// Froese, Oberman, Xiao) on one level grid of n^3 doubles, [k][j][i] order,
// boundary shell included.
//
//   smoother        Section 2: 8-colour nonlinear Gauss-Seidel, smallest root
//   residual        Algorithm 1 step 3 (r = rhs - det D^2_h u), norm partials
//   restriction     Section 3: half/full weighting, injection (steps 3-4)
//   coarse rhs      Algorithm 1 step 5 (tau correction)
//   prolongation    Section 3 trilinear, Algorithm 1 steps 7-8
//   coarsest solve  Algorithm 1 step 1, one thread block
//
// FP64 throughput is the bound of these kernels on GB300 (FP64 issues at
// about 1/70 of the FP32 rate), so the point solve keeps its FP64 work to the
// stencil, one determinant and one Newton correction (ma_point.cuh).
#include <algorithm>
#include <atomic>
#include <cstring>
#include <vector>

#include "ma.h"
#include "ma_internal.h"
#include "ma_batched.cuh"
#include "ma_point.cuh"
#include "ma_transfer.cuh"
#include "ma_residual.cuh"

namespace ma {

namespace {

constexpr int BX = 32, BY = 4;

__device__ __forceinline__ long long lin(int i, int j, int k, int n)
{
    return ((long long)k * n + j) * n + i;
}

// ---------------------------------------------------------------------------
// Smoother: one colour phase.  Colour c = (i&1) | (j&1)<<1 | (k&1)<<2; the
// interior points of parity p along an axis start at 1 (p = 1) or 2 (p = 0).
// Every stencil neighbour differs from the centre in at least one index
// parity, so the points of one colour are independent and one launch may
// update them all in parallel.
// ---------------------------------------------------------------------------
template <int PI, int PJ, int PK>
__device__ __forceinline__ void smooth_colour_block(double* u, const double* __restrict__ rhs, int n, double h6,
                                                    unsigned long long* events, uint3 bid)
{
    const int i = (PI ? 1 : 2) + 2 * (int)(bid.x * BX + threadIdx.x);
    const int j = (PJ ? 1 : 2) + 2 * (int)(bid.y * BY + threadIdx.y);
    const int k = (PK ? 1 : 2) + 2 * (int)bid.z;
    if (i > n - 2 || j > n - 2 || k > n - 2) return;
    const long long sy = n, sz = (long long)n * n;
    const long long p = lin(i, j, k, n);
    const double v0 = u[p];
    const HessS H = gather_hess(u, p, sy, sz, v0);
    bool nonconvex = false;
    const double z = smallest_root(H, __dmul_rn(h6, rhs[p]), &nonconvex);   // h6 = 64 h^6: the 4 Hs scaling
    u[p] = fma(0.125, z, v0);
    if (nonconvex && events) atomicAdd(events, 1ull);
}

template <int PI, int PJ, int PK>
__global__ void __launch_bounds__(BX * BY) k_smooth_colour(double* u, const double* __restrict__ rhs, int n,
                                                            double h6, unsigned long long* events)
{
    smooth_colour_block<PI, PJ, PK>(u, rhs, n, h6, events, blockIdx);
}

// Interior indices of one parity along an axis of n points (n odd).
__host__ __device__ __forceinline__ int colour_count(int n, int parity) { return parity ? (n - 1) / 2 : (n - 3) / 2; }

template <int C>
cudaError_t launch_colour(double* u, const double* rhs, int n, double h6, unsigned long long* ev, cudaStream_t s)
{
    constexpr int PI = C & 1, PJ = (C >> 1) & 1, PK = (C >> 2) & 1;
    const int ni = colour_count(n, PI), nj = colour_count(n, PJ), nk = colour_count(n, PK);
    if (ni <= 0 || nj <= 0 || nk <= 0) return cudaSuccess;
    dim3 grid((ni + BX - 1) / BX, (nj + BY - 1) / BY, nk);
    count_launches(1);
    k_smooth_colour<PI, PJ, PK><<<grid, dim3(BX, BY), 0, s>>>(u, rhs, n, h6, ev);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Block reduction of (max |x|, sum x^2) in a fixed order (deterministic).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void block_reduce_store(double mx, double ss, double* partials, int slot)
{
    __shared__ double smx[BX * BY / 32], sss[BX * BY / 32];
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
        ss += __shfl_down_sync(0xffffffffu, ss, o);
    }
    const int t = threadIdx.y * BX + threadIdx.x;
    if ((t & 31) == 0) { smx[t >> 5] = mx; sss[t >> 5] = ss; }
    __syncthreads();
    if (t == 0) {
        double m = smx[0], q = sss[0];
        for (int w = 1; w < BX * BY / 32; ++w) { m = fmax(m, smx[w]); q += sss[w]; }
        partials[2 * slot] = m;
        partials[2 * slot + 1] = q;
    }
}

constexpr int KZ = 16;   // z-blocks of the reduction grids; each loops over k

dim3 reduce_grid(int n) { return dim3((n + BX - 1) / BX, (n + BY - 1) / BY, n < KZ ? n : KZ); }

template <typename T>
__device__ __forceinline__ void norm_partials_block(const T* __restrict__ v, int n, double* partials, uint3 bid,
                                                    uint3 gdim)
{
    const int i = bid.x * BX + threadIdx.x;
    const int j = bid.y * BY + threadIdx.y;
    double mx = 0.0, ss = 0.0;
    for (int k = bid.z; k < n; k += gdim.z) {
        if (i > 0 && j > 0 && k > 0 && i < n - 1 && j < n - 1 && k < n - 1) {
            const double x = (double)v[lin(i, j, k, n)];
            mx = fmax(mx, fabs(x));
            ss = fma(x, x, ss);
        }
    }
    block_reduce_store(mx, ss, partials, (bid.z * gdim.y + bid.y) * gdim.x + bid.x);
}

template <typename T>
__global__ void __launch_bounds__(BX * BY) k_norm_partials(const T* __restrict__ v, int n, double* partials)
{
    norm_partials_block<T>(v, n, partials, blockIdx, gridDim);
}

// One block folds the partials in a fixed order: out2 = (max, sqrt(h^3 sum)).
__global__ void __launch_bounds__(resid::NF) k_norm_final(const double* __restrict__ partials, int count, double h3,
                                                          double* out2)
{
    resid::norm_final_block(partials, count, h3, out2);
}

// b_H = det(D^2_H w_H) + r_H on the interior, 0 on the shell.
__device__ __forceinline__ void coarse_rhs_block(const double* __restrict__ wc, const double* __restrict__ rc,
                                                 double* __restrict__ bc, int nc, double inv_H6, uint3 bid)
{
    const int I = bid.x * BX + threadIdx.x;
    const int J = bid.y * BY + threadIdx.y;
    const int K = bid.z;
    if (I >= nc || J >= nc) return;
    const long long p = lin(I, J, K, nc);
    double b = 0.0;
    if (I > 0 && J > 0 && K > 0 && I < nc - 1 && J < nc - 1 && K < nc - 1) {
        const HessS H = gather_hess(wc, p, nc, (long long)nc * nc, wc[p]);
        b = fma(det0(H), inv_H6, rc[p]);
    }
    bc[p] = b;
}

__global__ void __launch_bounds__(BX * BY) k_coarse_rhs(const double* __restrict__ wc, const double* __restrict__ rc,
                                                        double* __restrict__ bc, int nc, double inv_H6)
{
    coarse_rhs_block(wc, rc, bc, nc, inv_H6, blockIdx);
}

// rhs := f, u := g (whole grids); counts interior points with f not finite
// or f <= 0 and shell points with g not finite.
__global__ void k_copy_rhs_bc(const double* __restrict__ f, const double* __restrict__ g, double* __restrict__ rhs,
                              double* __restrict__ u, int n, int* bad)
{
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= n || j >= n) return;
    const long long p = lin(i, j, k, n);
    const double fv = f[p], gv = g[p];
    rhs[p] = fv;
    u[p] = gv;
    const bool interior = i > 0 && j > 0 && k > 0 && i < n - 1 && j < n - 1 && k < n - 1;
    const bool ok = interior ? (isfinite(fv) && fv > 0.0 && isfinite(gv)) : isfinite(gv);
    if (!ok) atomicAdd(bad, 1);
}

// ---------------------------------------------------------------------------
// Coarsest grid: one thread block sweeps the whole grid in shared memory.
// ---------------------------------------------------------------------------
constexpr int COARSE_THREADS = 256;

__device__ __forceinline__ HessS gather_hess_plain(const double* u, int p, int sy, int sz, double v0)
{
    const double* q = u + p;
    const double a = q[1] + q[-1];
    const double b = q[sy] + q[-sy];
    const double c = q[sz] + q[-sz];
    const double r4 = (q[sy + 1] + q[-sy - 1]) - (q[sy - 1] + q[-sy + 1]);
    const double s4 = (q[sz + 1] + q[-sz - 1]) - (q[sz - 1] + q[-sz + 1]);
    const double t4 = (q[sz + sy] + q[-sz - sy]) - (q[sy - sz] + q[-sy + sz]);
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

__device__ __forceinline__ void coarsest64_body(double* u, const double* __restrict__ rhs, int n, double h6, int sweeps,
                                                unsigned long long* events)
{
    extern __shared__ double sm[];
    const int m = n * n * n;
    double* su = sm;
    double* sr = sm + m;
    __shared__ double red[COARSE_THREADS / 32][2];
    __shared__ int stop;
    for (int q = threadIdx.x; q < m; q += COARSE_THREADS) { su[q] = u[q]; sr[q] = rhs[q]; }
    __syncthreads();
    const int max_sweeps = sweeps > 0 ? sweeps : 100;
    unsigned long long ev = 0;
    for (int s = 0; s < max_sweeps; ++s) {
        double du = 0.0, um = 0.0;
        for (int c = 0; c < 8; ++c) {
            const int pi = c & 1, pj = (c >> 1) & 1, pk = (c >> 2) & 1;
            const int ni = colour_count(n, pi), nj = colour_count(n, pj), nk = colour_count(n, pk);
            const int cnt = (ni > 0 && nj > 0 && nk > 0) ? ni * nj * nk : 0;
            for (int t = threadIdx.x; t < cnt; t += COARSE_THREADS) {
                const int i = (pi ? 1 : 2) + 2 * (t % ni);
                const int j = (pj ? 1 : 2) + 2 * ((t / ni) % nj);
                const int k = (pk ? 1 : 2) + 2 * (t / (ni * nj));
                const int p = (k * n + j) * n + i;
                const double v0 = su[p];
                const HessS H = gather_hess_plain(su, p, n, n * n, v0);
                bool nonconvex = false;
                const double z = smallest_root_precise(H, __dmul_rn(h6, sr[p]), &nonconvex);
                const double v = fma(0.125, z, v0);
                su[p] = v;
                du = fmax(du, fabs(v - v0));
                um = fmax(um, fabs(v));
                ev += nonconvex ? 1ull : 0ull;
            }
            __syncthreads();
        }
        if (sweeps > 0) continue;
        // converged when max |du| <= 1e-14 max |u| over this sweep's updates
        for (int o = 16; o > 0; o >>= 1) {
            du = fmax(du, __shfl_down_sync(0xffffffffu, du, o));
            um = fmax(um, __shfl_down_sync(0xffffffffu, um, o));
        }
        if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5][0] = du; red[threadIdx.x >> 5][1] = um; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0, b = 0.0;
            for (int w = 0; w < COARSE_THREADS / 32; ++w) { a = fmax(a, red[w][0]); b = fmax(b, red[w][1]); }
            stop = (a <= 1e-14 * b) ? 1 : 0;
        }
        __syncthreads();
        if (stop) break;
    }
    for (int q = threadIdx.x; q < m; q += COARSE_THREADS) u[q] = su[q];
    if (events && ev) atomicAdd(events, ev);
}

__global__ void __launch_bounds__(COARSE_THREADS) k_coarsest(double* u, const double* __restrict__ rhs, int n,
                                                             double h6, int sweeps, unsigned long long* events)
{
    coarsest64_body(u, rhs, n, h6, sweeps, events);
}

// ---------------------------------------------------------------------------
// The tail of an FP64 V-cycle in one block: every level with n <= 17, from
// the level the cycle enters there down to the coarsest grid and back, with
// u, w, r and rhs of those levels in shared memory.  Each step repeats the
// per-point arithmetic of its separate kernel -- the colour sweeps of
// k_smooth_colour, the residual of resid::k_residual_col (its column
// grouping of the cross differences), the restriction of xfer::k_restrict,
// the tau-corrected right-hand side of k_coarse_rhs, the coarsest solve of
// k_coarsest, the prolongation of xfer::k_prolong -- so the result is the
// same bits; it replaces the ~100 launches these latency-bound levels take
// (8 colour launches per sweep) by one.  FMG runs such a cycle from every
// level, so it pays most there.
// ---------------------------------------------------------------------------
constexpr int T64 = 512;

struct Tail64Level {
    int n;
    double h6, inv_h6;   // 64 h^6 (the 4 Hs scaling) and its reciprocal
    double* u;           // global iterate (read on the top level, written back there)
    const double* rhs;   // global right-hand side (read on the top level)
};

struct Tail64Args {
    int nlev;
    Tail64Level lev[4];
    int nu1, nu2, kind, approx, coarse_sweeps;
    unsigned long long* events;
};

__host__ __device__ inline int tail64_level_doubles(int n, bool top)
{
    const int m = n * n * n;
    return m /* u */ + (top ? 0 : m) /* w */ + m /* r */ + m /* rhs */;
}

struct Tail64Smem {
    double *u, *w, *r, *rhs;
};

__device__ __forceinline__ void tail64_smooth(const Tail64Smem& S, int n, double h6, int nsw, unsigned long long* ev)
{
    for (int sw = 0; sw < nsw; ++sw) {
        for (int c = 0; c < 8; ++c) {
            const int pi = c & 1, pj = (c >> 1) & 1, pk = (c >> 2) & 1;
            const int ni = colour_count(n, pi), nj = colour_count(n, pj), nk = colour_count(n, pk);
            const int cnt = (ni > 0 && nj > 0 && nk > 0) ? ni * nj * nk : 0;
            for (int t = threadIdx.x; t < cnt; t += T64) {
                const int i = (pi ? 1 : 2) + 2 * (t % ni);
                const int j = (pj ? 1 : 2) + 2 * ((t / ni) % nj);
                const int k = (pk ? 1 : 2) + 2 * (t / (ni * nj));
                const int p = (k * n + j) * n + i;
                const double v0 = S.u[p];
                const HessS H = gather_hess_plain(S.u, p, n, n * n, v0);
                bool nonconvex = false;
                const double z = smallest_root(H, __dmul_rn(h6, S.rhs[p]), &nonconvex);
                S.u[p] = fma(0.125, z, v0);
                *ev += nonconvex ? 1ull : 0ull;
            }
            __syncthreads();
        }
    }
}

// rhs - det(D^2_h u) at interior point p, the cross differences grouped as
// the column-marching residual kernel forms them.
__device__ __forceinline__ double tail64_residual(const double* u, int p, int n, double rhs, double inv_h6)
{
    const int sy = n, sz = n * n;
    const double* q = u + p;
    const double a = q[1] + q[-1];
    const double b = q[sy] + q[-sy];
    const double c = q[sz] + q[-sz];
    const double r4 = (q[sy + 1] - q[sy - 1]) - (q[-sy + 1] - q[-sy - 1]);
    const double dxc = q[sz + 1] - q[sz - 1], dxa = q[-sz + 1] - q[-sz - 1];
    const double dyc = q[sz + sy] - q[sz - sy], dya = q[-sz + sy] - q[-sz - sy];
    HessS H;
    const double m8v = -8.0 * q[0];
    H.A = fma(4.0, a, m8v);
    H.B = fma(4.0, b, m8v);
    H.C = fma(4.0, c, m8v);
    H.R = r4;
    H.S = dxc - dxa;
    H.T = dyc - dya;
    return fma(-det0(H), inv_h6, rhs);
}

__device__ __forceinline__ double tail64_line(const double* uc, const double* wc, int nc, int Ic, int J0, int K0,
                                              int oj, int ok, double w)
{
    double s = 0.0;
    for (int dk = 0; dk <= ok; ++dk)
        for (int dj = 0; dj <= oj; ++dj) {
            const int q = ((K0 + dk) * nc + (J0 + dj)) * nc + Ic;
            s += uc[q] - wc[q];
        }
    return s * w;
}

__device__ __forceinline__ void vcycle_tail_body(const Tail64Args& A)
{
    extern __shared__ double t64sm[];
    Tail64Smem S[4];
    {
        double* q = t64sm;
        for (int l = 0; l < A.nlev; ++l) {
            const int m = A.lev[l].n * A.lev[l].n * A.lev[l].n;
            S[l].u = q; q += m;
            S[l].w = l > 0 ? q : nullptr; q += l > 0 ? m : 0;
            S[l].r = q; q += m;
            S[l].rhs = q; q += m;
        }
    }
    // inputs: the top level's iterate and right-hand side; residual shells 0
    // (the restriction reads only the interior, as in the separate path)
    for (int l = 0; l < A.nlev; ++l) {
        const int m = A.lev[l].n * A.lev[l].n * A.lev[l].n;
        for (int q = threadIdx.x; q < m; q += T64) S[l].r[q] = 0.0;
        if (l == 0)
            for (int q = threadIdx.x; q < m; q += T64) { S[0].u[q] = A.lev[0].u[q]; S[0].rhs[q] = A.lev[0].rhs[q]; }
    }
    __syncthreads();
    unsigned long long ev = 0;
    const int L = A.nlev;
    for (int l = 0; l < L - 1; ++l) {
        const Tail64Smem& F = S[l];
        const Tail64Smem& C = S[l + 1];
        const int nf = A.lev[l].n, nc = A.lev[l + 1].n;
        tail64_smooth(F, nf, A.lev[l].h6, A.nu1, &ev);                                       // (2)
        for (int q = threadIdx.x; q < (nf - 2) * (nf - 2) * (nf - 2); q += T64) {        // (3)
            const int i = 1 + q % (nf - 2), j = 1 + (q / (nf - 2)) % (nf - 2), k = 1 + q / ((nf - 2) * (nf - 2));
            const int p = (k * nf + j) * nf + i;
            F.r[p] = tail64_residual(F.u, p, nf, F.rhs[p], A.lev[l].inv_h6);
        }
        __syncthreads();
        for (int pc = threadIdx.x; pc < nc * nc * nc; pc += T64) {                        // (3)-(4)
            const int I = pc % nc, J = (pc / nc) % nc, K = pc / (nc * nc);
            const int pf = ((2 * K) * nf + 2 * J) * nf + 2 * I;
            const bool inside = I > 0 && J > 0 && K > 0 && I < nc - 1 && J < nc - 1 && K < nc - 1;
            C.r[pc] = inside ? xfer::weighted_restrict(F.r, pf, nf, (long long)nf * nf, A.kind) : 0.0;
            const double w = (inside && A.approx == 1) ? xfer::weighted_restrict(F.u, pf, nf, (long long)nf * nf, A.kind)
                                                      : F.u[pf];
            C.w[pc] = w;
            C.u[pc] = w;
        }
        __syncthreads();
        for (int p = threadIdx.x; p < nc * nc * nc; p += T64) {                           // (5)
            const int I = p % nc, J = (p / nc) % nc, K = p / (nc * nc);
            double b = 0.0;
            if (I > 0 && J > 0 && K > 0 && I < nc - 1 && J < nc - 1 && K < nc - 1) {
                const HessS H = gather_hess_plain(C.w, p, nc, nc * nc, C.w[p]);
                b = fma(det0(H), A.lev[l + 1].inv_h6, C.r[p]);
            }
            C.rhs[p] = b;
        }
        __syncthreads();
    }
    {   // (1) coarsest grid: sweeps until max|du| <= 1e-14 max|u| (at most 100), or a fixed count
        const Tail64Smem& Bt = S[L - 1];
        const int n = A.lev[L - 1].n;
        const double h6 = A.lev[L - 1].h6;
        __shared__ double red[T64 / 32][2];
        __shared__ int stop;
        const int max_sweeps = A.coarse_sweeps > 0 ? A.coarse_sweeps : 100;
        for (int s = 0; s < max_sweeps; ++s) {
            double du = 0.0, um = 0.0;
            for (int c = 0; c < 8; ++c) {
                const int pi = c & 1, pj = (c >> 1) & 1, pk = (c >> 2) & 1;
                const int ni = colour_count(n, pi), nj = colour_count(n, pj), nk = colour_count(n, pk);
                const int cnt = (ni > 0 && nj > 0 && nk > 0) ? ni * nj * nk : 0;
                for (int t = threadIdx.x; t < cnt; t += T64) {
                    const int i = (pi ? 1 : 2) + 2 * (t % ni);
                    const int j = (pj ? 1 : 2) + 2 * ((t / ni) % nj);
                    const int k = (pk ? 1 : 2) + 2 * (t / (ni * nj));
                    const int p = (k * n + j) * n + i;
                    const double v0 = Bt.u[p];
                    const HessS H = gather_hess_plain(Bt.u, p, n, n * n, v0);
                    bool nonconvex = false;
                    const double z = smallest_root_precise(H, __dmul_rn(h6, Bt.rhs[p]), &nonconvex);
                    const double v = fma(0.125, z, v0);
                    Bt.u[p] = v;
                    du = fmax(du, fabs(v - v0));
                    um = fmax(um, fabs(v));
                    ev += nonconvex ? 1ull : 0ull;
                }
                __syncthreads();
            }
            if (A.coarse_sweeps > 0) continue;
            for (int o = 16; o > 0; o >>= 1) {
                du = fmax(du, __shfl_down_sync(0xffffffffu, du, o));
                um = fmax(um, __shfl_down_sync(0xffffffffu, um, o));
            }
            if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5][0] = du; red[threadIdx.x >> 5][1] = um; }
            __syncthreads();
            if (threadIdx.x == 0) {
                double a = 0.0, b = 0.0;
                for (int w = 0; w < T64 / 32; ++w) { a = fmax(a, red[w][0]); b = fmax(b, red[w][1]); }
                stop = (a <= 1e-14 * b) ? 1 : 0;
            }
            __syncthreads();
            if (stop) break;
        }
    }
    for (int l = L - 2; l >= 0; --l) {
        const Tail64Smem& F = S[l];
        const Tail64Smem& C = S[l + 1];
        const int nf = A.lev[l].n, nc = A.lev[l + 1].n;
        // (7)-(8) u_h += I(u_H - w_H) on the fine interior, each value formed as xfer::k_prolong forms it
        for (int q = threadIdx.x; q < (nf - 2) * (nf - 2) * (nf - 2); q += T64) {
            const int i = 1 + q % (nf - 2), j = 1 + (q / (nf - 2)) % (nf - 2), k = 1 + q / ((nf - 2) * (nf - 2));
            const int J0 = j >> 1, K0 = k >> 1, oj = j & 1, ok = k & 1;
            const double w = 1.0 / (double)(1 << (oj + ok));
            double v;
            if (i & 1) {
                const int I = i >> 1;
                const double a = tail64_line(C.u, C.w, nc, I, J0, K0, oj, ok, w);
                const double b = tail64_line(C.u, C.w, nc, I + 1, J0, K0, oj, ok, w);
                v = (a + b) * 0.5;
            } else {
                v = tail64_line(C.u, C.w, nc, i >> 1, J0, K0, oj, ok, w);
            }
            const int p = (k * nf + j) * nf + i;
            F.u[p] = F.u[p] + v;
        }
        __syncthreads();
        tail64_smooth(F, nf, A.lev[l].h6, A.nu2, &ev);                                      // (9)
    }
    const int m0 = A.lev[0].n * A.lev[0].n * A.lev[0].n;
    for (int q = threadIdx.x; q < m0; q += T64) A.lev[0].u[q] = S[0].u[q];
    if (A.events && ev) atomicAdd(A.events, ev);
}

__global__ void __launch_bounds__(T64, 1) k_vcycle_tail(Tail64Args A) { vcycle_tail_body(A); }

int tail64_smem_bytes(const int* ns, int nlev)
{
    int d = 0;
    for (int l = 0; l < nlev; ++l) d += tail64_level_doubles(ns[l], l == 0);
    return d * (int)sizeof(double);
}

}  // namespace

// ---------------------------------------------------------------------------
// Batched FP64 launches (the start of a shared per-level batch): the norms
// of f and the FMG pass of Algorithm 2 over several hierarchies at once.
// With one coarsest grid size for all of them, FMG step j works on the level
// of size 2^j (coarsest_n - 1) + 1 in every hierarchy that has it, so the
// V-cycles of a step have the same level sizes everywhere.
// ---------------------------------------------------------------------------
namespace {

using batched::split_block;
using batched::TableBuilder;

enum F64OpId {
    F_SMOOTH0 = batched::kF64Ops,   // .. + 7
    F_RESID = batched::kF64Ops + 8, F_RESTRICT, F_COARSE_RHS, F_PROLONG, F_CUBIC0, F_CUBIC1, F_CUBIC2, F_INJECT,
    F_ZERO, F_COARSEST, F_TAIL, F_NORMPART
};

struct Smooth64Job {
    int inst, n, gx, gy;
    double h6;
    double* u;
    const double* rhs;
    unsigned long long* events;
};

template <int C>
struct OpSmooth64 {
    static constexpr int NT = BX * BY, MINB = 1;
    using Job = Smooth64Job;
    static __device__ __forceinline__ void run(const Job& J, int q)
    {
        smooth_colour_block<C & 1, (C >> 1) & 1, (C >> 2) & 1>(J.u, J.rhs, J.n, J.h6, J.events,
                                                               split_block(q, J.gx, J.gy));
    }
};

struct OpResid64 {
    static constexpr int NT = resid::RX * resid::RY, MINB = 1;
    struct Job {
        int inst, n, kchunk, gx, gy, gz;
        double inv_h6;
        const double* u;
        const double* rhs;
        double* r;
    };
    static __device__ __forceinline__ void run(const Job& J, int q)
    {
        resid::residual_col_block<resid::NaturalF64Out>(J.u, J.rhs, resid::NaturalF64Out{J.r}, J.n, J.inv_h6, nullptr,
                                                        J.kchunk, split_block(q, J.gx, J.gy),
                                                        make_uint3((unsigned)J.gx, (unsigned)J.gy, (unsigned)J.gz));
    }
};

struct OpRestrict64 {
    static constexpr int NT = BX * BY, MINB = 1;
    struct Job {
        int inst, nf, nc, kind, approx, gx, gy;
        const double* uf;
        const double* rf;
        double* wc;
        double* uc;
        double* rc;
    };
    static __device__ __forceinline__ void run(const Job& J, int q)
    {
        xfer::restrict_block<double>(J.uf, J.rf, J.nf, J.wc, J.uc, J.rc, J.nc, J.kind, J.approx,
                                     split_block(q, J.gx, J.gy));
    }
};

struct OpCoarseRhs64 {
    static constexpr int NT = BX * BY, MINB = 1;
    struct Job {
        int inst, nc, gx, gy;
        double inv_H6;
        const double* wc;
        const double* rc;
        double* bc;
    };
    static __device__ __forceinline__ void run(const Job& J, int q)
    {
        coarse_rhs_block(J.wc, J.rc, J.bc, J.nc, J.inv_H6, split_block(q, J.gx, J.gy));
    }
};

// add != 0: uf += I(uc - wc); add == 0: uf = I(uc) (trilinear)
struct OpProlong64 {
    static constexpr int NT = BX * BY, MINB = 1;
    struct Job {
        int inst, nc, nf, add, gx, gy;
        const double* uc;
        const double* wc;
        double* uf;
    };
    static __device__ __forceinline__ void run(const Job& J, int q)
    {
        xfer::prolong_block<double>(J.uc, J.wc, J.nc, J.uf, J.nf, J.add, split_block(q, J.gx, J.gy));
    }
};

struct CubicJob {
    int inst, nc, ox, oy, oz, interior_only, gx, gy;
    const double* in;
    double* out;
};

template <int AX>
struct OpCubic {
    static constexpr int NT = BX * BY, MINB = 1;
    using Job = CubicJob;
    static __device__ __forceinline__ void run(const Job& J, int q)
    {
        xfer::cubic_pass_block<AX>(J.in, J.out, J.nc, J.ox, J.oy, J.oz, J.interior_only, split_block(q, J.gx, J.gy));
    }
};

struct OpInject64 {
    static constexpr int NT = BX * BY, MINB = 1;
    struct Job {
        int inst, nf, nc, gx, gy;
        const double* vf;
        double* vc;
    };
    static __device__ __forceinline__ void run(const Job& J, int q)
    {
        xfer::inject_block<double>(J.vf, J.nf, J.vc, J.nc, split_block(q, J.gx, J.gy));
    }
};

struct OpZero64 {
    static constexpr int NT = BX * BY, MINB = 1;
    struct Job {
        int inst, n, gx, gy;
        double* u;
    };
    static __device__ __forceinline__ void run(const Job& J, int q)
    {
        xfer::zero_interior_block<double>(J.u, J.n, split_block(q, J.gx, J.gy));
    }
};

struct OpCoarsest64 {
    static constexpr int NT = COARSE_THREADS, MINB = 1;
    struct Job {
        int inst, n, sweeps;
        double h6;
        double* u;
        const double* rhs;
        unsigned long long* events;
    };
    static __device__ __forceinline__ void run(const Job& J, int)
    {
        coarsest64_body(J.u, J.rhs, J.n, J.h6, J.sweeps, J.events);
    }
};

struct OpTail64 {
    static constexpr int NT = T64, MINB = 1;
    struct Job {
        int inst;
        Tail64Args A;
    };
    static __device__ __forceinline__ void run(const Job& J, int) { vcycle_tail_body(J.A); }
};

struct OpNormPart64 {
    static constexpr int NT = BX * BY, MINB = 1;
    struct Job {
        int inst, n, gx, gy, gz;
        const double* v;
        double* partials;
    };
    static __device__ __forceinline__ void run(const Job& J, int q)
    {
        norm_partials_block<double>(J.v, J.n, J.partials, split_block(q, J.gx, J.gy),
                                    make_uint3((unsigned)J.gx, (unsigned)J.gy, (unsigned)J.gz));
    }
};

inline double pow6h(double h)
{
    const double h2 = h * h;
    return 64.0 * h2 * h2 * h2;
}

dim3 grid2(int n) { return dim3((n + BX - 1) / BX, (n + BY - 1) / BY, n); }

// An entry of a batched FP64 V-cycle: instance (index into the array) and the
// level its cycle starts from.
struct VEntry {
    int b, l0;
};

void emit_smooth64(TableBuilder& T, const BatchInstance* in, const std::vector<VEntry>& E, const std::vector<int>& lev,
                   int nsweeps)
{
    for (int sw = 0; sw < nsweeps; ++sw)
        for (int c = 0; c < 8; ++c) {
            std::vector<Smooth64Job> jobs;
            std::vector<int> blocks;
            for (size_t q = 0; q < E.size(); ++q) {
                if (lev[q] < 0) continue;
                const BatchInstance& I = in[E[q].b];
                const BatchLevel& F = I.lev[lev[q]];
                const int ni = colour_count(F.n, c & 1), nj = colour_count(F.n, (c >> 1) & 1),
                          nk = colour_count(F.n, (c >> 2) & 1);
                if (ni <= 0 || nj <= 0 || nk <= 0) continue;
                Smooth64Job J{I.id, F.n, (ni + BX - 1) / BX, (nj + BY - 1) / BY, pow6h(F.h), F.u, F.rhs, I.events};
                jobs.push_back(J);
                blocks.push_back(J.gx * J.gy * nk);
            }
            T.emit(F_SMOOTH0 + c, jobs, blocks, 0);
        }
}

// Algorithm 1 from level l0 of each entry down to the coarsest grid and
// back, with the fused FP64 tail: the launches of vcycle_from, depth by
// depth relative to l0.
void emit_vcycle64(TableBuilder& T, const BatchInstance* in, const std::vector<VEntry>& E, const BatchParams& p)
{
    if (E.empty()) return;
    std::vector<int> lt(E.size()), fused(E.size());
    int R = 0;
    for (size_t q = 0; q < E.size(); ++q) {
        const BatchInstance& I = in[E[q].b];
        int t = I.L - 1;
        while (t > E[q].l0 && I.lev[t - 1].n <= p.vtail_max) --t;
        fused[q] = I.lev[t].n <= p.vtail_max;
        lt[q] = fused[q] ? t : I.L - 1;
        R = std::max(R, lt[q] - E[q].l0);
    }
    auto level_at = [&](int r) {
        std::vector<int> lev(E.size(), -1);
        for (size_t q = 0; q < E.size(); ++q)
            if (r < lt[q] - E[q].l0) lev[q] = E[q].l0 + r;
        return lev;
    };
    for (int r = 0; r < R; ++r) {
        const std::vector<int> lev = level_at(r);
        emit_smooth64(T, in, E, lev, p.nu1);
        std::vector<OpResid64::Job> rj;
        std::vector<OpRestrict64::Job> sj;
        std::vector<OpCoarseRhs64::Job> cj;
        std::vector<int> rb, sb, cb;
        for (size_t q = 0; q < E.size(); ++q) {
            if (lev[q] < 0) continue;
            const BatchInstance& I = in[E[q].b];
            const BatchLevel& F = I.lev[lev[q]];
            const BatchLevel& C = I.lev[lev[q] + 1];
            const dim3 g = reduce_grid(F.n);
            const int kchunk = (F.n + (int)g.z - 1) / (int)g.z;
            rj.push_back(OpResid64::Job{I.id, F.n, kchunk, (int)g.x, (int)g.y, (int)g.z, 1.0 / pow6h(F.h), F.u, F.rhs,
                                        F.r});
            rb.push_back((int)(g.x * g.y * g.z));
            const dim3 gc = grid2(C.n);
            sj.push_back(OpRestrict64::Job{I.id, F.n, C.n, p.kind, p.approx, (int)gc.x, (int)gc.y, F.u, F.r, C.w, C.u,
                                           C.r});
            sb.push_back((int)(gc.x * gc.y * gc.z));
            cj.push_back(OpCoarseRhs64::Job{I.id, C.n, (int)gc.x, (int)gc.y, 1.0 / pow6h(C.h), C.w, C.r, C.rhs});
            cb.push_back((int)(gc.x * gc.y * gc.z));
        }
        T.emit(F_RESID, rj, rb, 0);
        T.emit(F_RESTRICT, sj, sb, 0);
        T.emit(F_COARSE_RHS, cj, cb, 0);
    }
    {
        std::vector<OpTail64::Job> tj;
        std::vector<OpCoarsest64::Job> kj;
        std::vector<int> tb, kb;
        int tsmem = 0, ksmem = 0;
        for (size_t q = 0; q < E.size(); ++q) {
            const BatchInstance& I = in[E[q].b];
            if (fused[q]) {
                OpTail64::Job J;
                std::memset(&J, 0, sizeof J);
                J.inst = I.id;
                Tail64Args& A = J.A;
                A.nlev = I.L - lt[q];
                int ns[4] = {0, 0, 0, 0};
                for (int v = 0; v < A.nlev; ++v) {
                    const BatchLevel& V = I.lev[lt[q] + v];
                    ns[v] = V.n;
                    A.lev[v].n = V.n;
                    A.lev[v].h6 = pow6h(V.h);
                    A.lev[v].inv_h6 = 1.0 / pow6h(V.h);
                    A.lev[v].u = V.u;
                    A.lev[v].rhs = V.rhs;
                }
                A.nu1 = p.nu1;
                A.nu2 = p.nu2;
                A.kind = p.kind;
                A.approx = p.approx;
                A.coarse_sweeps = p.coarse_sweeps;
                A.events = I.events;
                tsmem = std::max(tsmem, tail64_smem_bytes(ns, A.nlev));
                tj.push_back(J);
                tb.push_back(1);
            } else {
                const BatchLevel& V = I.lev[I.L - 1];
                kj.push_back(OpCoarsest64::Job{I.id, V.n, p.coarse_sweeps, pow6h(V.h), V.u, V.rhs, I.events});
                kb.push_back(1);
                ksmem = std::max(ksmem, (int)(2 * sizeof(double) * (size_t)V.n * V.n * V.n));
            }
        }
        T.emit(F_TAIL, tj, tb, tsmem);
        T.emit(F_COARSEST, kj, kb, ksmem);
    }
    for (int r = R - 1; r >= 0; --r) {
        const std::vector<int> lev = level_at(r);
        std::vector<OpProlong64::Job> pj;
        std::vector<int> pb;
        for (size_t q = 0; q < E.size(); ++q) {
            if (lev[q] < 0) continue;
            const BatchInstance& I = in[E[q].b];
            const BatchLevel& F = I.lev[lev[q]];
            const BatchLevel& C = I.lev[lev[q] + 1];
            const dim3 g = xfer::prolong_grid(F.n);
            pj.push_back(OpProlong64::Job{I.id, C.n, F.n, 1, (int)g.x, (int)g.y, C.u, C.w, F.u});
            pb.push_back((int)(g.x * g.y * g.z));
        }
        T.emit(F_PROLONG, pj, pb, 0);
        emit_smooth64(T, in, E, lev, p.nu2);
    }
}

}  // namespace

void emit_rhs_partials_f64(TableBuilder& T, const BatchInstance* in, int count)
{
    std::vector<OpNormPart64::Job> jobs;
    std::vector<int> blocks;
    for (int b = 0; b < count; ++b) {
        const BatchLevel& F = in[b].lev[0];
        const dim3 g = reduce_grid(F.n);
        jobs.push_back(OpNormPart64::Job{in[b].id, F.n, (int)g.x, (int)g.y, (int)g.z, F.rhs, in[b].partials});
        blocks.push_back((int)(g.x * g.y * g.z));
    }
    T.emit(F_NORMPART, jobs, blocks, 0);
}

// Algorithm 2 as fmg(H, false) runs it: inject f and the data down, solve the
// coarsest grid from a zero interior, then up the levels: interpolate and one
// V-cycle from that level, the finest level receiving the interpolation only.
void emit_fmg_f64(TableBuilder& T, const BatchInstance* in, int count, const BatchParams& p,
                  const std::function<void(const std::vector<std::pair<int, int>>&)>& level_step)
{
    int Lmax = 0;
    for (int b = 0; b < count; ++b) Lmax = std::max(Lmax, in[b].L);
    for (int d = 0; d + 1 < Lmax; ++d)
        for (int field = 0; field < 2; ++field) {   // f, then the iterate (its shell carries g)
            std::vector<OpInject64::Job> jobs;
            std::vector<int> blocks;
            for (int b = 0; b < count; ++b) {
                if (d + 1 >= in[b].L) continue;
                const BatchLevel& F = in[b].lev[d];
                const BatchLevel& C = in[b].lev[d + 1];
                const dim3 g = grid2(C.n);
                jobs.push_back(OpInject64::Job{in[b].id, F.n, C.n, (int)g.x, (int)g.y, field ? F.u : F.rhs,
                                               field ? C.u : C.rhs});
                blocks.push_back((int)(g.x * g.y * g.z));
            }
            T.emit(F_INJECT, jobs, blocks, 0);
        }
    {
        std::vector<OpZero64::Job> zj;
        std::vector<OpCoarsest64::Job> kj;
        std::vector<int> zb, kb;
        int ksmem = 0;
        for (int b = 0; b < count; ++b) {
            const BatchLevel& V = in[b].lev[in[b].L - 1];
            const dim3 g = grid2(V.n);
            zj.push_back(OpZero64::Job{in[b].id, V.n, (int)g.x, (int)g.y, V.u});
            zb.push_back((int)(g.x * g.y * g.z));
            kj.push_back(OpCoarsest64::Job{in[b].id, V.n, p.coarse_sweeps, pow6h(V.h), V.u, V.rhs, in[b].events});
            kb.push_back(1);
            ksmem = std::max(ksmem, (int)(2 * sizeof(double) * (size_t)V.n * V.n * V.n));
        }
        T.emit(F_ZERO, zj, zb, 0);
        T.emit(F_COARSEST, kj, kb, ksmem);
    }
    for (int j = 1; j < Lmax; ++j) {
        // interpolation into level l = L - 1 - j of every hierarchy that has it
        std::vector<OpProlong64::Job> lj;
        std::vector<CubicJob> c0, c1, c2;
        std::vector<int> lb, b0, b1, b2;
        std::vector<VEntry> E;
        for (int b = 0; b < count; ++b) {
            const int l = in[b].L - 1 - j;
            if (l < 0) continue;
            const BatchLevel& F = in[b].lev[l];
            const BatchLevel& C = in[b].lev[l + 1];
            const int nc = C.n, nf = F.n;
            if (p.fmg_interp == MA_FMG_CUBIC) {
                double* t1 = F.r;                              // the fine level's r is free here
                double* t2 = F.r + (size_t)nf * nc * nc;
                auto cj = [&](const double* src, double* dst, int ox, int oy, int oz, int io) {
                    return CubicJob{in[b].id, nc, ox, oy, oz, io, (ox + BX - 1) / BX, (oy + BY - 1) / BY, src, dst};
                };
                c0.push_back(cj(C.u, t1, nf, nc, nc, 0));
                b0.push_back(c0.back().gx * c0.back().gy * nc);
                c1.push_back(cj(t1, t2, nf, nf, nc, 0));
                b1.push_back(c1.back().gx * c1.back().gy * nc);
                c2.push_back(cj(t2, F.u, nf, nf, nf, 1));
                b2.push_back(c2.back().gx * c2.back().gy * nf);
            } else {
                const dim3 g = xfer::prolong_grid(nf);
                lj.push_back(OpProlong64::Job{in[b].id, nc, nf, 0, (int)g.x, (int)g.y, C.u, nullptr, F.u});
                lb.push_back((int)(g.x * g.y * g.z));
            }
            if (l >= 1) E.push_back(VEntry{b, l});
        }
        T.emit(F_PROLONG, lj, lb, 0);
        T.emit(F_CUBIC0, c0, b0, 0);
        T.emit(F_CUBIC1, c1, b1, 0);
        T.emit(F_CUBIC2, c2, b2, 0);
        if (level_step) {
            std::vector<std::pair<int, int>> steps;
            for (const VEntry& v : E) steps.emplace_back(v.b, v.l0);
            if (!steps.empty()) level_step(steps);
        } else {
            emit_vcycle64(T, in, E, p);
        }
    }
}

cudaError_t batch_launch_f64(const char* tables, const batched::BLaunch& L, const int* active, cudaStream_t s)
{
    using batched::launch;
    const dim3 b2(BX, BY);
    switch (L.op) {
    case F_SMOOTH0 + 0: return launch<OpSmooth64<0>>(tables, L, b2, active, s);
    case F_SMOOTH0 + 1: return launch<OpSmooth64<1>>(tables, L, b2, active, s);
    case F_SMOOTH0 + 2: return launch<OpSmooth64<2>>(tables, L, b2, active, s);
    case F_SMOOTH0 + 3: return launch<OpSmooth64<3>>(tables, L, b2, active, s);
    case F_SMOOTH0 + 4: return launch<OpSmooth64<4>>(tables, L, b2, active, s);
    case F_SMOOTH0 + 5: return launch<OpSmooth64<5>>(tables, L, b2, active, s);
    case F_SMOOTH0 + 6: return launch<OpSmooth64<6>>(tables, L, b2, active, s);
    case F_SMOOTH0 + 7: return launch<OpSmooth64<7>>(tables, L, b2, active, s);
    case F_RESID: return launch<OpResid64>(tables, L, dim3(resid::RX, resid::RY), active, s);
    case F_RESTRICT: return launch<OpRestrict64>(tables, L, b2, active, s);
    case F_COARSE_RHS: return launch<OpCoarseRhs64>(tables, L, b2, active, s);
    case F_PROLONG: return launch<OpProlong64>(tables, L, b2, active, s);
    case F_CUBIC0: return launch<OpCubic<0>>(tables, L, b2, active, s);
    case F_CUBIC1: return launch<OpCubic<1>>(tables, L, b2, active, s);
    case F_CUBIC2: return launch<OpCubic<2>>(tables, L, b2, active, s);
    case F_INJECT: return launch<OpInject64>(tables, L, b2, active, s);
    case F_ZERO: return launch<OpZero64>(tables, L, b2, active, s);
    case F_COARSEST: return launch<OpCoarsest64>(tables, L, dim3(COARSE_THREADS), active, s);
    case F_TAIL: return launch<OpTail64>(tables, L, dim3(T64), active, s);
    case F_NORMPART: return launch<OpNormPart64>(tables, L, b2, active, s);
    default: return cudaErrorInvalidValue;
    }
}

static std::atomic<unsigned long long> g_launches{0};
void count_launches(unsigned long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
void uncount_launches(unsigned long long k) { g_launches.fetch_sub(k, std::memory_order_relaxed); }
unsigned long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
// 64 h^6: determinants of the 4 Hs matrices the gathers return are 64 h^6 det(D^2 u).
static inline double pow6(double h) { const double h2 = h * h; return 64.0 * h2 * h2 * h2; }

cudaError_t launch_smooth(double* u, const double* rhs, int n, double h, int nsweeps,
                          unsigned long long* events, cudaStream_t s)
{
    const double h6 = pow6(h);
    for (int sw = 0; sw < nsweeps; ++sw) {
        cudaError_t e;
        if ((e = launch_colour<0>(u, rhs, n, h6, events, s)) != cudaSuccess) return e;
        if ((e = launch_colour<1>(u, rhs, n, h6, events, s)) != cudaSuccess) return e;
        if ((e = launch_colour<2>(u, rhs, n, h6, events, s)) != cudaSuccess) return e;
        if ((e = launch_colour<3>(u, rhs, n, h6, events, s)) != cudaSuccess) return e;
        if ((e = launch_colour<4>(u, rhs, n, h6, events, s)) != cudaSuccess) return e;
        if ((e = launch_colour<5>(u, rhs, n, h6, events, s)) != cudaSuccess) return e;
        if ((e = launch_colour<6>(u, rhs, n, h6, events, s)) != cudaSuccess) return e;
        if ((e = launch_colour<7>(u, rhs, n, h6, events, s)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int residual_partial_count(int n)
{
    const dim3 g = reduce_grid(n);
    return (int)(g.x * g.y * g.z);
}

int norm_partial_count(int n) { return residual_partial_count(n); }

cudaError_t launch_residual(const double* u, const double* rhs, double* r, int n, double h,
                            double* partials, cudaStream_t s)
{
    count_launches(1);
    const dim3 g = reduce_grid(n);
    const int kchunk = (n + (int)g.z - 1) / (int)g.z;
    resid::k_residual_col<resid::NaturalF64Out><<<resid::grid_for(n, g.z), dim3(resid::RX, resid::RY), 0, s>>>(
        u, rhs, resid::NaturalF64Out{r}, n, 1.0 / pow6(h), partials, kchunk);
    return cudaGetLastError();
}

cudaError_t launch_norm_partials(const double* v, int n, double* partials, cudaStream_t s)
{
    count_launches(1);
    k_norm_partials<double><<<reduce_grid(n), dim3(BX, BY), 0, s>>>(v, n, partials);
    return cudaGetLastError();
}

cudaError_t launch_norm_partials_f32(const float* v, int n, double* partials, cudaStream_t s)
{
    count_launches(1);
    k_norm_partials<float><<<reduce_grid(n), dim3(BX, BY), 0, s>>>(v, n, partials);
    return cudaGetLastError();
}

cudaError_t launch_norm_final(const double* partials, int count, double h, double* out2, cudaStream_t s)
{
    count_launches(1);
    k_norm_final<<<1, resid::NF, 0, s>>>(partials, count, h * h * h, out2);
    return cudaGetLastError();
}

using xfer::grid_of;

cudaError_t launch_restrict_residual(const double* rf, int nf, double* rc, int kind, cudaStream_t s)
{
    const int nc = (nf + 1) / 2;
    count_launches(1);
    xfer::k_restrict<double><<<grid_of(nc), dim3(BX, BY), 0, s>>>(nullptr, rf, nf, nullptr, nullptr, rc, nc, kind, 0);
    return cudaGetLastError();
}

cudaError_t launch_restrict_solution(const double* uf, int nf, double* uc, int approx, int kind, cudaStream_t s)
{
    const int nc = (nf + 1) / 2;
    count_launches(1);
    xfer::k_restrict<double><<<grid_of(nc), dim3(BX, BY), 0, s>>>(uf, nullptr, nf, nullptr, uc, nullptr, nc, kind, approx);
    return cudaGetLastError();
}

cudaError_t launch_restrict_level(const double* uf, const double* rf, int nf, double* wc, double* uc, double* rc,
                                  int kind, int approx, cudaStream_t s)
{
    const int nc = (nf + 1) / 2;
    count_launches(1);
    xfer::k_restrict<double><<<grid_of(nc), dim3(BX, BY), 0, s>>>(uf, rf, nf, wc, uc, rc, nc, kind, approx);
    return cudaGetLastError();
}

cudaError_t launch_coarse_rhs(const double* wc, const double* rc, double* bc, int nc, double H, cudaStream_t s)
{
    count_launches(1);
    k_coarse_rhs<<<grid_of(nc), dim3(BX, BY), 0, s>>>(wc, rc, bc, nc, 1.0 / pow6(H));
    return cudaGetLastError();
}

cudaError_t launch_prolong_add(const double* uc, const double* wc, int nc, double* uf, cudaStream_t s)
{
    const int nf = 2 * nc - 1;
    count_launches(1);
    xfer::k_prolong<double><<<xfer::prolong_grid(nf), dim3(BX, BY), 0, s>>>(uc, wc, nc, uf, nf, 1);
    return cudaGetLastError();
}

cudaError_t launch_interpolate(const double* uc, int nc, double* uf, cudaStream_t s)
{
    const int nf = 2 * nc - 1;
    count_launches(1);
    xfer::k_prolong<double><<<xfer::prolong_grid(nf), dim3(BX, BY), 0, s>>>(uc, nullptr, nc, uf, nf, 0);
    return cudaGetLastError();
}

size_t interpolate_cubic_scratch(int nc)
{
    const size_t nf = 2 * (size_t)nc - 1;
    return sizeof(double) * (nf * nc * nc + nf * nf * nc);
}

// Tricubic interpolation (Algorithm 2 step 4): passes x, y, z through the
// scratch t (interpolate_cubic_scratch(nc) bytes); the fine shell is kept.
cudaError_t launch_interpolate_cubic(const double* uc, int nc, double* uf, double* t, cudaStream_t s)
{
    const int nf = 2 * nc - 1;
    double* t1 = t;                                  // nc x nc x nf
    double* t2 = t + (size_t)nf * nc * nc;           // nc x nf x nf
    auto grid = [](int ox, int oy, int oz) { return dim3((ox + BX - 1) / BX, (oy + BY - 1) / BY, oz); };
    count_launches(3);
    xfer::k_cubic_pass<0><<<grid(nf, nc, nc), dim3(BX, BY), 0, s>>>(uc, t1, nc, nf, nc, nc, 0);
    xfer::k_cubic_pass<1><<<grid(nf, nf, nc), dim3(BX, BY), 0, s>>>(t1, t2, nc, nf, nf, nc, 0);
    xfer::k_cubic_pass<2><<<grid(nf, nf, nf), dim3(BX, BY), 0, s>>>(t2, uf, nc, nf, nf, nf, 1);
    return cudaGetLastError();
}

cudaError_t launch_inject(const double* vf, int nf, double* vc, cudaStream_t s)
{
    const int nc = (nf + 1) / 2;
    count_launches(1);
    xfer::k_inject<double><<<grid_of(nc), dim3(BX, BY), 0, s>>>(vf, nf, vc, nc);
    return cudaGetLastError();
}

cudaError_t launch_zero_interior(double* u, int n, cudaStream_t s)
{
    count_launches(1);
    xfer::k_zero_interior<double><<<grid_of(n), dim3(BX, BY), 0, s>>>(u, n);
    return cudaGetLastError();
}

cudaError_t launch_copy_rhs_bc(const double* f, const double* g, double* rhs, double* u, int n, int* bad,
                               cudaStream_t s)
{
    count_launches(1);
    k_copy_rhs_bc<<<grid_of(n), dim3(BX, BY), 0, s>>>(f, g, rhs, u, n, bad);
    return cudaGetLastError();
}

cudaError_t launch_coarsest(double* u, const double* rhs, int n, double h, int sweeps,
                            unsigned long long* events, cudaStream_t s)
{
    const size_t smem = 2 * sizeof(double) * (size_t)n * n * n;
    count_launches(1);
    k_coarsest<<<1, COARSE_THREADS, smem, s>>>(u, rhs, n, pow6(h), sweeps, events);
    return cudaGetLastError();
}

// Largest level of the fused FP64 tail.  One block runs the tail on one SM,
// whose FP64 pipe then does all the point solves: at 17^3 (3375 points a
// sweep) that costs more than 8 colour launches spread over the GPU, at 9^3
// and below the launches cost more.
constexpr int kVTailDefault = 9;
static std::atomic<int> g_vtail_max{kVTailDefault};

int vcycle_tail_max_n() { return g_vtail_max.load(std::memory_order_relaxed); }

bool set_vcycle_tail(int max_n)
{
    if (max_n == 1) max_n = kVTailDefault;
    if (!(max_n == 0 || max_n == 3 || max_n == 5 || max_n == 9 || max_n == 17)) return false;
    g_vtail_max.store(max_n, std::memory_order_relaxed);
    return true;
}

cudaError_t launch_vcycle_tail(const TailSpec64* lv, int nlev, int nu1, int nu2, int kind, int approx,
                               int coarse_sweeps, unsigned long long* events, cudaStream_t s)
{
    if (nlev < 1 || nlev > 4) return cudaErrorInvalidValue;
    Tail64Args A;
    A.nlev = nlev;
    int ns[4];
    for (int l = 0; l < nlev; ++l) {
        if (lv[l].n > 17 || (l > 0 && lv[l].n != (lv[l - 1].n + 1) / 2)) return cudaErrorInvalidValue;
        A.lev[l].n = ns[l] = lv[l].n;
        A.lev[l].h6 = pow6(lv[l].h);
        A.lev[l].inv_h6 = 1.0 / pow6(lv[l].h);
        A.lev[l].u = lv[l].u;
        A.lev[l].rhs = lv[l].rhs;
    }
    A.nu1 = nu1;
    A.nu2 = nu2;
    A.kind = kind;
    A.approx = approx;
    A.coarse_sweeps = coarse_sweeps;
    A.events = events;
    count_launches(1);
    k_vcycle_tail<<<1, T64, tail64_smem_bytes(ns, nlev), s>>>(A);
    return cudaGetLastError();
}

cudaError_t prepare_coarsest_f64()
{
    cudaError_t e = cudaFuncSetAttribute(k_coarsest, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(2 * sizeof(double) * 17 * 17 * 17));
    if (e != cudaSuccess) return e;
    const int tail_ns[4] = {17, 9, 5, 3};
    if ((e = cudaFuncSetAttribute(k_vcycle_tail, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  tail64_smem_bytes(tail_ns, 4))) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(batched::k_batched<OpTail64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  tail64_smem_bytes(tail_ns, 4))) != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(batched::k_batched<OpCoarsest64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(2 * sizeof(double) * 17 * 17 * 17));
}

}  // namespace ma
