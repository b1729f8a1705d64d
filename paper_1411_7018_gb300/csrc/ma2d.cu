// ma2d.cu -- the two-dimensional version of the method (Eq. MA2D, Section 4.1
// of Liu, Froese, Oberman, Xiao): kernels and the C ABI of include/ma2d.h.
//
// Local equation of the smoother at (i, j): with a = u(i+1,j) + u(i-1,j),
// b = u(i,j+1) + u(i,j-1) and r = the cross difference over 4,
//     (a - 2v)(b - 2v) - r^2 = h^4 f,
// whose smaller root v = ((a + b) - sqrt((a - b)^2 + 4 r^2 + 4 h^4 f)) / 4 is
// the convex one (Section 2).  A negative discriminant (possible only for a
// coarse right-hand side < 0) has no real root; the vertex (a + b)/4 is taken
// and counted.  FP64 throughout: the 2D point update is ~20 FP64 operations.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>

#include "ma.h"
#include "ma2d.h"
#include "ma_internal.h"

namespace {

constexpr int TX = 32, TY = 8;
constexpr int kMaxLevels2 = 16;

__device__ __forceinline__ void sums2(const double* u, int n, int i, int j, double& a, double& b, double& r)
{
    const double* p = u + (long long)j * n + i;
    a = p[1] + p[-1];
    b = p[n] + p[-n];
    r = 0.25 * ((p[n + 1] - p[n - 1]) - (p[-n + 1] - p[-n - 1]));
}

__device__ __forceinline__ double quad_root(double a, double b, double r, double h4, double rhs, bool* neg)
{
    double d = (a - b) * (a - b) + 4.0 * r * r + 4.0 * h4 * rhs;
    if (d < 0.0) {
        *neg = true;
        d = 0.0;
    }
    return 0.25 * ((a + b) - sqrt(d));
}

__device__ __forceinline__ double s_h(const double* u, int n, int i, int j, double inv_h2)
{
    double a, b, r;
    sums2(u, n, i, j, a, b, r);
    const double v = u[(long long)j * n + i];
    return ((a - 2.0 * v) * inv_h2) * ((b - 2.0 * v) * inv_h2) - (r * inv_h2) * (r * inv_h2);
}

// Red-black phase: dst = src with the points of one colour (i + j parity)
// updated from src.  A thread takes the pair i = 2 i2, 2 i2 + 1 of row j: it
// solves the point of this colour and copies the other, so every lane of a
// warp runs the root (colours alternate along a row).
__global__ void __launch_bounds__(TX * TY) k_rb_phase(const double* __restrict__ src, double* __restrict__ dst,
                                                       const double* __restrict__ rhs, int n, double h4, int colour,
                                                       unsigned long long* events)
{
    const int i0 = 2 * (int)(blockIdx.x * TX + threadIdx.x), j = blockIdx.y * TY + threadIdx.y;
    if (i0 >= n || j >= n) return;
    const long long row = (long long)j * n;
    const int ic = i0 + ((j + colour) & 1);   // (ic + j) & 1 == colour
    const int io = ic == i0 ? i0 + 1 : i0;
    if (io < n) dst[row + io] = src[row + io];
    if (ic >= n) return;
    if (ic > 0 && j > 0 && ic < n - 1 && j < n - 1) {
        double a, b, r;
        sums2(src, n, ic, j, a, b, r);
        bool neg = false;
        dst[row + ic] = quad_root(a, b, r, h4, rhs[row + ic], &neg);
        if (neg && events) atomicAdd(events, 1ull);
    } else {
        dst[row + ic] = src[row + ic];
    }
}

// Four-colour phase, in place: the points with i & 1 == pi, j & 1 == pj.
__global__ void __launch_bounds__(TX * TY) k_c4_phase(double* u, const double* __restrict__ rhs, int n, double h4,
                                                       int pi, int pj, unsigned long long* events)
{
    const int i = (pi ? 1 : 2) + 2 * (int)(blockIdx.x * TX + threadIdx.x);
    const int j = (pj ? 1 : 2) + 2 * (int)(blockIdx.y * TY + threadIdx.y);
    if (i > n - 2 || j > n - 2) return;
    double a, b, r;
    sums2(u, n, i, j, a, b, r);
    bool neg = false;
    const long long p = (long long)j * n + i;
    u[p] = quad_root(a, b, r, h4, rhs[p], &neg);
    if (neg && events) atomicAdd(events, 1ull);
}

// r = rhs - S_h(u) inside, 0 on the boundary; per-block (max |r|, sum r^2).
__global__ void __launch_bounds__(TX * TY) k_resid2(const double* __restrict__ u, const double* __restrict__ rhs,
                                                     double* __restrict__ res, int n, double inv_h2,
                                                     double* partials)
{
    const int i = blockIdx.x * TX + threadIdx.x, j = blockIdx.y * TY + threadIdx.y;
    double m = 0.0, s = 0.0;
    if (i < n && j < n) {
        const long long p = (long long)j * n + i;
        double v = 0.0;
        if (i > 0 && j > 0 && i < n - 1 && j < n - 1) {
            v = rhs[p] - s_h(u, n, i, j, inv_h2);
            m = fabs(v);
            s = v * v;
        }
        if (res) res[p] = v;
    }
    if (!partials) return;
    __shared__ double sm[TX * TY / 32][2];
    for (int o = 16; o > 0; o >>= 1) {
        m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
        s += __shfl_down_sync(0xffffffffu, s, o);
    }
    const int t = threadIdx.y * TX + threadIdx.x;
    if ((t & 31) == 0) { sm[t >> 5][0] = m; sm[t >> 5][1] = s; }
    __syncthreads();
    if (t == 0) {
        for (int w = 1; w < TX * TY / 32; ++w) { m = fmax(m, sm[w][0]); s += sm[w][1]; }
        const int slot = blockIdx.y * gridDim.x + blockIdx.x;
        partials[2 * slot] = m;
        partials[2 * slot + 1] = s;
    }
}

// Per-block (max |v|, sum v^2) over the interior of v.
__global__ void __launch_bounds__(TX * TY) k_norm_partials2(const double* __restrict__ v, int n, double* partials)
{
    const int i = blockIdx.x * TX + threadIdx.x, j = blockIdx.y * TY + threadIdx.y;
    double m = 0.0, s = 0.0;
    if (i > 0 && j > 0 && i < n - 1 && j < n - 1) {
        const double x = v[(long long)j * n + i];
        m = fabs(x);
        s = x * x;
    }
    __shared__ double sm[TX * TY / 32][2];
    for (int o = 16; o > 0; o >>= 1) {
        m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
        s += __shfl_down_sync(0xffffffffu, s, o);
    }
    const int t = threadIdx.y * TX + threadIdx.x;
    if ((t & 31) == 0) { sm[t >> 5][0] = m; sm[t >> 5][1] = s; }
    __syncthreads();
    if (t == 0) {
        for (int w = 1; w < TX * TY / 32; ++w) { m = fmax(m, sm[w][0]); s += sm[w][1]; }
        const int slot = blockIdx.y * gridDim.x + blockIdx.x;
        partials[2 * slot] = m;
        partials[2 * slot + 1] = s;
    }
}

// out2 = (max, sqrt(h^2 sum)) from the partials (one block).
__global__ void k_norm_final2(const double* partials, int count, double h, double* out2)
{
    double m = 0.0, s = 0.0;
    for (int q = threadIdx.x; q < count; q += blockDim.x) {
        m = fmax(m, partials[2 * q]);
        s += partials[2 * q + 1];
    }
    __shared__ double sm[32][2];
    for (int o = 16; o > 0; o >>= 1) {
        m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
        s += __shfl_down_sync(0xffffffffu, s, o);
    }
    if ((threadIdx.x & 31) == 0) { sm[threadIdx.x >> 5][0] = m; sm[threadIdx.x >> 5][1] = s; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x / 32); ++w) { m = fmax(m, sm[w][0]); s += sm[w][1]; }
        out2[0] = m;
        out2[1] = sqrt(h * h * s);
    }
}

__device__ __forceinline__ double restrict_at2(const double* v, int nf, int i, int j, int kind)
{
    const double* p = v + (long long)j * nf + i;
    if (kind == MA_HALF_WEIGHTING) return (4.0 * p[0] + ((p[1] + p[-1]) + (p[nf] + p[-nf]))) * 0.125;
    const double c = p[0], e = (p[1] + p[-1]) + (p[nf] + p[-nf]);
    const double d = (p[nf + 1] + p[nf - 1]) + (p[-nf + 1] + p[-nf - 1]);
    return (4.0 * c + 2.0 * e + d) * 0.0625;
}

// Coarse outputs (any may be null): rc = restricted residual (0 on the
// boundary); wc = approximation restriction of uf (injection on the
// boundary); uc = a copy of wc.
__global__ void __launch_bounds__(TX * TY) k_restrict2(const double* __restrict__ uf, const double* __restrict__ rf,
                                                        int nf, double* wc, double* uc, double* rc, int nc, int kind,
                                                        int approx)
{
    const int I = blockIdx.x * TX + threadIdx.x, J = blockIdx.y * TY + threadIdx.y;
    if (I >= nc || J >= nc) return;
    const long long pc = (long long)J * nc + I;
    const bool inside = I > 0 && J > 0 && I < nc - 1 && J < nc - 1;
    if (rc) rc[pc] = inside ? restrict_at2(rf, nf, 2 * I, 2 * J, kind) : 0.0;
    if (uf) {
        const double w = (inside && approx == MA_APPROX_WEIGHTED) ? restrict_at2(uf, nf, 2 * I, 2 * J, kind)
                                                                   : uf[(long long)(2 * J) * nf + 2 * I];
        if (wc) wc[pc] = w;
        if (uc) uc[pc] = w;
    }
}

__global__ void __launch_bounds__(TX * TY) k_inject2(const double* __restrict__ vf, int nf, double* vc, int nc)
{
    const int I = blockIdx.x * TX + threadIdx.x, J = blockIdx.y * TY + threadIdx.y;
    if (I >= nc || J >= nc) return;
    vc[(long long)J * nc + I] = vf[(long long)(2 * J) * nf + 2 * I];
}

// One axis of the cubic interpolation (the rule of the 3D cubic passes).
__device__ __forceinline__ int cubic_axis2(int i, int nc, double w[4], int* cnt)
{
    if ((i & 1) == 0) { w[0] = 1.0; *cnt = 1; return i >> 1; }
    const int I0 = i >> 1;
    if (nc == 2) { w[0] = w[1] = 0.5; *cnt = 2; return 0; }
    if (nc == 3) {
        *cnt = 3;
        if (I0 == 0) { w[0] = 0.375; w[1] = 0.75; w[2] = -0.125; }
        else { w[0] = -0.125; w[1] = 0.75; w[2] = 0.375; }
        return 0;
    }
    *cnt = 4;
    if (I0 == 0) { w[0] = 0.3125; w[1] = 0.9375; w[2] = -0.3125; w[3] = 0.0625; return 0; }
    if (I0 == nc - 2) { w[0] = 0.0625; w[1] = -0.3125; w[2] = 0.9375; w[3] = 0.3125; return nc - 4; }
    w[0] = -0.0625; w[1] = 0.5625; w[2] = 0.5625; w[3] = -0.0625;
    return I0 - 1;
}

// Fine interior from coarse values: add != 0: uf += bilinear(uc - wc);
// else uf = bilinear(uc) (cubic == 0) or bicubic(uc).
__global__ void __launch_bounds__(TX * TY) k_prolong2(const double* __restrict__ uc, const double* __restrict__ wc,
                                                       int nc, double* uf, int nf, int add, int cubic)
{
    const int i = blockIdx.x * TX + threadIdx.x, j = blockIdx.y * TY + threadIdx.y;
    if (i < 1 || j < 1 || i > nf - 2 || j > nf - 2) return;
    const long long p = (long long)j * nf + i;
    if (cubic) {
        double wx[4], wy[4];
        int cx, cy;
        const int I = cubic_axis2(i, nc, wx, &cx), J = cubic_axis2(j, nc, wy, &cy);
        double s = 0.0;
        for (int b = 0; b < cy; ++b) {
            double row = 0.0;
            for (int a = 0; a < cx; ++a) row = fma(wx[a], uc[(long long)(J + b) * nc + I + a], row);
            s = fma(wy[b], row, s);
        }
        uf[p] = s;
        return;
    }
    const int I = i >> 1, J = j >> 1, oi = i & 1, oj = j & 1;
    double s = 0.0;
    for (int b = 0; b <= oj; ++b)
        for (int a = 0; a <= oi; ++a) {
            const long long q = (long long)(J + b) * nc + I + a;
            s += add ? (uc[q] - wc[q]) : uc[q];
        }
    const double v = s * (1.0 / (double)(1 << (oi + oj)));
    uf[p] = add ? uf[p] + v : v;
}

// b = S_H(w) + r inside, 0 on the boundary (Algorithm 1 step 5).
__global__ void __launch_bounds__(TX * TY) k_coarse_rhs2(const double* __restrict__ w, const double* __restrict__ r,
                                                          double* __restrict__ b, int nc, double inv_h2)
{
    const int I = blockIdx.x * TX + threadIdx.x, J = blockIdx.y * TY + threadIdx.y;
    if (I >= nc || J >= nc) return;
    const long long p = (long long)J * nc + I;
    b[p] = (I > 0 && J > 0 && I < nc - 1 && J < nc - 1) ? s_h(w, nc, I, J, inv_h2) + r[p] : 0.0;
}

// Coarsest grid (n <= 17): one block, the grid in shared memory; sweeps > 0
// fixed sweeps, else until max|du| <= 1e-14 max|u| (at most 100).
constexpr int CT2 = 256;
__global__ void __launch_bounds__(CT2) k_coarsest2(double* u, const double* __restrict__ rhs, int n, double h4,
                                                   int sweeps, int ordering, unsigned long long* events)
{
    __shared__ double su[17 * 17];
    __shared__ double sr[17 * 17];
    __shared__ double red[CT2 / 32][2];
    __shared__ int stop;
    const int m = n * n;
    // the stopping test compares with max |u| over the whole grid, boundary
    // included (boundary values do not change)
    double bmax = 0.0;
    for (int q = threadIdx.x; q < m; q += CT2) {
        su[q] = u[q];
        sr[q] = rhs[q];
        const int i = q % n, j = q / n;
        if (i == 0 || j == 0 || i == n - 1 || j == n - 1) bmax = fmax(bmax, fabs(su[q]));
    }
    __syncthreads();
    unsigned long long ev = 0;
    const int phases = ordering == MA2D_COLOUR4 ? 4 : 2;
    const int max_sweeps = sweeps > 0 ? sweeps : 100;
    for (int s = 0; s < max_sweeps; ++s) {
        double du = 0.0, um = bmax;
        for (int ph = 0; ph < phases; ++ph) {
            // each thread takes at most two points per phase (n <= 17: <= 225 interior)
            double nv[2];
            int np[2], cnt = 0;
            for (int q = threadIdx.x; q < (n - 2) * (n - 2); q += CT2) {
                const int i = 1 + q % (n - 2), j = 1 + q / (n - 2);
                const bool mine = ordering == MA2D_COLOUR4 ? (((i & 1) | ((j & 1) << 1)) == ph) : (((i + j) & 1) == ph);
                if (!mine) continue;
                double a, b, r;
                sums2(su, n, i, j, a, b, r);
                bool neg = false;
                nv[cnt] = quad_root(a, b, r, h4, sr[j * n + i], &neg);
                np[cnt] = j * n + i;
                ++cnt;
                ev += neg ? 1 : 0;
            }
            __syncthreads();   // red-black: every point of the colour from the old values
            for (int c = 0; c < cnt; ++c) {
                du = fmax(du, fabs(nv[c] - su[np[c]]));
                su[np[c]] = nv[c];
                um = fmax(um, fabs(nv[c]));
            }
            __syncthreads();
        }
        if (sweeps > 0) continue;
        for (int o = 16; o > 0; o >>= 1) {
            du = fmax(du, __shfl_down_sync(0xffffffffu, du, o));
            um = fmax(um, __shfl_down_sync(0xffffffffu, um, o));
        }
        if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5][0] = du; red[threadIdx.x >> 5][1] = um; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0, b = 0.0;
            for (int w = 0; w < CT2 / 32; ++w) { a = fmax(a, red[w][0]); b = fmax(b, red[w][1]); }
            stop = a <= 1e-14 * b;
        }
        __syncthreads();
        if (stop) break;
    }
    for (int q = threadIdx.x; q < m; q += CT2) u[q] = su[q];
    if (events && ev) atomicAdd(events, ev);
}

// rhs = f, u = g; flag = 1 if f is not finite and > 0 inside.
__global__ void __launch_bounds__(TX * TY) k_copy_rhs_bc2(const double* __restrict__ f, const double* __restrict__ g,
                                                           double* rhs, double* u, int n, int* bad)
{
    const int i = blockIdx.x * TX + threadIdx.x, j = blockIdx.y * TY + threadIdx.y;
    if (i >= n || j >= n) return;
    const long long p = (long long)j * n + i;
    const bool inside = i > 0 && j > 0 && i < n - 1 && j < n - 1;
    const double fv = inside ? f[p] : 0.0;
    if (inside && !(fv > 0.0 && fv < INFINITY)) atomicExch(bad, 1);
    rhs[p] = fv;
    u[p] = g[p];
}

__global__ void __launch_bounds__(TX * TY) k_zero_interior2(double* u, int n)
{
    const int i = blockIdx.x * TX + threadIdx.x, j = blockIdx.y * TY + threadIdx.y;
    if (i < 1 || j < 1 || i > n - 2 || j > n - 2) return;
    u[(long long)j * n + i] = 0.0;
}

dim3 grid2(int nx, int ny) { return dim3((nx + TX - 1) / TX, (ny + TY - 1) / TY); }
int partial_count2(int n) { const dim3 g = grid2(n, n); return (int)(g.x * g.y); }

// ---- launchers ---------------------------------------------------------------

cudaError_t smooth2(double* u, double* t, const double* rhs, int n, double h, int nsweeps, int ordering,
                    unsigned long long* ev, cudaStream_t s)
{
    const double h4 = h * h * h * h;
    for (int sw = 0; sw < nsweeps; ++sw) {
        if (ordering == MA2D_COLOUR4) {
            for (int c = 0; c < 4; ++c) {
                const int pi = c & 1, pj = c >> 1;
                const int ni = pi ? (n - 1) / 2 : (n - 3) / 2, nj = pj ? (n - 1) / 2 : (n - 3) / 2;
                if (ni <= 0 || nj <= 0) continue;
                ma::count_launches(1);
                k_c4_phase<<<grid2(ni, nj), dim3(TX, TY), 0, s>>>(u, rhs, n, h4, pi, pj, ev);
            }
        } else {
            ma::count_launches(2);
            const dim3 g = grid2((n + 1) / 2, n);
            k_rb_phase<<<g, dim3(TX, TY), 0, s>>>(u, t, rhs, n, h4, 0, ev);
            k_rb_phase<<<g, dim3(TX, TY), 0, s>>>(t, u, rhs, n, h4, 1, ev);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t residual2(const double* u, const double* rhs, double* r, int n, double h, double* partials,
                      cudaStream_t s)
{
    ma::count_launches(1);
    k_resid2<<<grid2(n, n), dim3(TX, TY), 0, s>>>(u, rhs, r, n, 1.0 / (h * h), partials);
    return cudaGetLastError();
}

cudaError_t norm_final2(const double* partials, int count, double h, double* out2, cudaStream_t s)
{
    ma::count_launches(1);
    k_norm_final2<<<1, 1024, 0, s>>>(partials, count, h, out2);
    return cudaGetLastError();
}

thread_local char g_err2[512] = "";

ma_status fail2(ma_status st, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err2, sizeof g_err2, fmt, ap);
    va_end(ap);
    ma::set_last_error(g_err2);
    return st;
}

#define CK2(call)                                                                                \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return fail2(MA_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

bool valid_n2(int n) { return n >= 3 && (n % 2) == 1 && n <= 32769; }

}  // namespace

struct ma2d_hierarchy {
    ma2d_desc d;
    int L = 0;
    struct Lv {
        int n = 0;
        double h = 0.0;
        double *u = nullptr, *rhs = nullptr, *r = nullptr, *w = nullptr;
    } lev[kMaxLevels2];
    double* t = nullptr;          // second buffer of the red-black phases (finest size)
    double* partials = nullptr;
    int npartials = 0;
    double* out = nullptr;        // 4 doubles: residual (max, L2), reference (max, L2)
    int* flag = nullptr;
    double* host = nullptr;       // pinned, 4 doubles
    cudaStream_t s = nullptr;
};

namespace {

int levels2(int n, int coarsest)
{
    int L = 1, m = n;
    while (m > coarsest) {
        if ((m - 1) % 2) return -1;
        m = (m + 1) / 2;
        if (++L > kMaxLevels2) return -1;
    }
    return m == coarsest ? L : -1;
}

ma_status check_desc2(const ma2d_desc* d)
{
    if (!d) return fail2(MA_ERR_INVALID_ARG, "null descriptor");
    if (!(d->coarsest_n == 3 || d->coarsest_n == 5 || d->coarsest_n == 9 || d->coarsest_n == 17))
        return fail2(MA_ERR_INVALID_ARG, "coarsest_n must be 3, 5, 9 or 17");
    if (!valid_n2(d->n) || levels2(d->n, d->coarsest_n) < 1)
        return fail2(MA_ERR_INVALID_ARG, "n = %d is not 2^L (coarsest_n - 1) + 1 (<= 32769)", d->n);
    if (!(d->len > 0.0) || !std::isfinite(d->len)) return fail2(MA_ERR_INVALID_ARG, "len must be finite and > 0");
    if (d->nu1 < 0 || d->nu2 < 0 || d->nu1 > 64 || d->nu2 > 64 || d->nu1 + d->nu2 == 0)
        return fail2(MA_ERR_INVALID_ARG, "bad nu1, nu2");
    if (d->restrict_kind != MA_HALF_WEIGHTING && d->restrict_kind != MA_FULL_WEIGHTING)
        return fail2(MA_ERR_INVALID_ARG, "bad restrict_kind");
    if (d->approx_restrict != MA_APPROX_INJECTION && d->approx_restrict != MA_APPROX_WEIGHTED)
        return fail2(MA_ERR_INVALID_ARG, "bad approx_restrict");
    if (d->coarse_sweeps < 0 || d->coarse_sweeps > 1000) return fail2(MA_ERR_INVALID_ARG, "bad coarse_sweeps");
    if (d->ordering != MA2D_REDBLACK && d->ordering != MA2D_COLOUR4) return fail2(MA_ERR_INVALID_ARG, "bad ordering");
    if (d->fmg_interp != MA_FMG_TRILINEAR && d->fmg_interp != MA_FMG_CUBIC)
        return fail2(MA_ERR_INVALID_ARG, "bad fmg_interp");
    return MA_OK;
}

size_t layout2(ma2d_hierarchy* H, const ma2d_desc* d, char* base)
{
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        char* p = base ? base + off : nullptr;
        off = align256(off + bytes);
        return p;
    };
    const int L = levels2(d->n, d->coarsest_n);
    int m = d->n;
    double h = d->len / (d->n - 1);
    for (int l = 0; l < L; ++l) {
        const size_t pts = (size_t)m * m;
        auto& v = H->lev[l];
        v.n = m;
        v.h = h;
        v.u = (double*)take(pts * 8);
        v.rhs = (double*)take(pts * 8);
        v.r = (double*)take(pts * 8);
        v.w = (double*)take(pts * 8);
        m = (m + 1) / 2;
        h *= 2.0;
    }
    H->L = L;
    H->t = (double*)take((size_t)d->n * d->n * 8);
    H->npartials = partial_count2(d->n);
    H->partials = (double*)take(16 * (size_t)H->npartials);
    H->out = (double*)take(4 * 8);
    H->flag = (int*)take(sizeof(int));
    return off;
}

cudaError_t coarsest_solve2(ma2d_hierarchy* H, int l)
{
    auto& B = H->lev[l];
    const double h4 = B.h * B.h * B.h * B.h;
    ma::count_launches(1);
    k_coarsest2<<<1, CT2, 0, H->s>>>(B.u, B.rhs, B.n, h4, H->d.coarse_sweeps, H->d.ordering, nullptr);
    return cudaGetLastError();
}

// Algorithm 1 (2D) from level l0 down and back.
cudaError_t vcycle2_from(ma2d_hierarchy* H, int l0)
{
    cudaStream_t s = H->s;
    const ma2d_desc& d = H->d;
    cudaError_t e;
    for (int l = l0; l < H->L - 1; ++l) {
        auto& F = H->lev[l];
        auto& C = H->lev[l + 1];
        if ((e = smooth2(F.u, H->t, F.rhs, F.n, F.h, d.nu1, d.ordering, nullptr, s)) != cudaSuccess) return e;
        if ((e = residual2(F.u, F.rhs, F.r, F.n, F.h, nullptr, s)) != cudaSuccess) return e;
        ma::count_launches(2);
        k_restrict2<<<grid2(C.n, C.n), dim3(TX, TY), 0, s>>>(F.u, F.r, F.n, C.w, C.u, C.r, C.n, d.restrict_kind,
                                                             d.approx_restrict);
        k_coarse_rhs2<<<grid2(C.n, C.n), dim3(TX, TY), 0, s>>>(C.w, C.r, C.rhs, C.n, 1.0 / (C.h * C.h));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = coarsest_solve2(H, H->L - 1)) != cudaSuccess) return e;
    for (int l = H->L - 2; l >= l0; --l) {
        auto& F = H->lev[l];
        auto& C = H->lev[l + 1];
        ma::count_launches(1);
        k_prolong2<<<grid2(F.n, F.n), dim3(TX, TY), 0, s>>>(C.u, C.w, C.n, F.u, F.n, 1, 0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = smooth2(F.u, H->t, F.rhs, F.n, F.h, d.nu2, d.ordering, nullptr, s)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Algorithm 2 (2D).
cudaError_t fmg2(ma2d_hierarchy* H)
{
    cudaStream_t s = H->s;
    cudaError_t e;
    for (int l = 0; l < H->L - 1; ++l) {
        auto& F = H->lev[l];
        auto& C = H->lev[l + 1];
        ma::count_launches(2);
        k_inject2<<<grid2(C.n, C.n), dim3(TX, TY), 0, s>>>(F.rhs, F.n, C.rhs, C.n);
        k_inject2<<<grid2(C.n, C.n), dim3(TX, TY), 0, s>>>(F.u, F.n, C.u, C.n);
    }
    auto& B = H->lev[H->L - 1];
    ma::count_launches(1);
    k_zero_interior2<<<grid2(B.n, B.n), dim3(TX, TY), 0, s>>>(B.u, B.n);
    if ((e = coarsest_solve2(H, H->L - 1)) != cudaSuccess) return e;
    for (int l = H->L - 2; l >= 0; --l) {
        auto& F = H->lev[l];
        auto& C = H->lev[l + 1];
        ma::count_launches(1);
        k_prolong2<<<grid2(F.n, F.n), dim3(TX, TY), 0, s>>>(C.u, nullptr, C.n, F.u, F.n, 0,
                                                            H->d.fmg_interp == MA_FMG_CUBIC);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = vcycle2_from(H, l)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Residual norms of the finest level into out[slot], out[slot + 1]; reads
// them back when readback != 0 (blocks).
ma_status fine_norms2(ma2d_hierarchy* H, int slot, double* mx, double* l2)
{
    auto& F = H->lev[0];
    CK2(residual2(F.u, F.rhs, F.r, F.n, F.h, H->partials, H->s));
    CK2(norm_final2(H->partials, H->npartials, F.h, H->out + slot, H->s));
    CK2(cudaMemcpyAsync(H->host, H->out, 4 * sizeof(double), cudaMemcpyDeviceToHost, H->s));
    CK2(cudaStreamSynchronize(H->s));
    *mx = H->host[slot];
    *l2 = H->host[slot + 1];
    return MA_OK;
}

}  // namespace

extern "C" {

ma_status ma2d_hierarchy_footprint(const ma2d_desc* desc, size_t* bytes)
{
    ma_status st = check_desc2(desc);
    if (st != MA_OK) return st;
    if (!bytes) return fail2(MA_ERR_INVALID_ARG, "null bytes");
    ma2d_hierarchy tmp;
    *bytes = layout2(&tmp, desc, nullptr);
    return MA_OK;
}

ma_status ma2d_create_hierarchy(const ma2d_desc* desc, void* ws, size_t bytes, ma_stream_t stream,
                                ma2d_hierarchy** out)
{
    ma_status st = check_desc2(desc);
    if (st != MA_OK) return st;
    if (!out || !ws) return fail2(MA_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (((uintptr_t)ws) % 256 != 0) return fail2(MA_ERR_INVALID_ARG, "workspace not 256-byte aligned");
    ma2d_hierarchy* H = new (std::nothrow) ma2d_hierarchy();
    if (!H) return fail2(MA_ERR_OOM, "host allocation failed");
    H->d = *desc;
    const size_t need = layout2(H, desc, (char*)ws);
    if (bytes < need) {
        delete H;
        return fail2(MA_ERR_INVALID_ARG, "workspace of %zu bytes < footprint %zu", bytes, need);
    }
    H->s = (cudaStream_t)stream;
    cudaError_t e = cudaMallocHost((void**)&H->host, 4 * sizeof(double));
    if (e != cudaSuccess) {
        delete H;
        return fail2(MA_ERR_CUDA, "create: %s", cudaGetErrorString(e));
    }
    *out = H;
    return MA_OK;
}

ma_status ma2d_destroy_hierarchy(ma2d_hierarchy* H)
{
    if (!H) return MA_OK;
    cudaError_t e = cudaStreamSynchronize(H->s);
    if (H->host) cudaFreeHost(H->host);
    delete H;
    if (e != cudaSuccess) return fail2(MA_ERR_CUDA, "destroy: %s", cudaGetErrorString(e));
    return MA_OK;
}

ma_status ma2d_set_rhs_bc(ma2d_hierarchy* H, const double* f, const double* g)
{
    if (!H || !f || !g) return fail2(MA_ERR_INVALID_ARG, "null argument");
    auto& F = H->lev[0];
    CK2(cudaMemsetAsync(H->flag, 0, sizeof(int), H->s));
    ma::count_launches(1);
    k_copy_rhs_bc2<<<grid2(F.n, F.n), dim3(TX, TY), 0, H->s>>>(f, g, F.rhs, F.u, F.n, H->flag);
    CK2(cudaGetLastError());
    int bad = 0;
    CK2(cudaMemcpyAsync(&bad, H->flag, sizeof(int), cudaMemcpyDeviceToHost, H->s));
    CK2(cudaStreamSynchronize(H->s));
    if (bad) return fail2(MA_ERR_INVALID_ARG, "f must be finite and > 0 on the interior");
    return MA_OK;
}

ma_status ma2d_vcycle(ma2d_hierarchy* H, int ncycles)
{
    if (!H || ncycles < 0) return fail2(MA_ERR_INVALID_ARG, "bad arguments");
    for (int c = 0; c < ncycles; ++c) CK2(vcycle2_from(H, 0));
    return MA_OK;
}

ma_status ma2d_solve(ma2d_hierarchy* H, const ma_solve_opts* o, ma_solve_result* res)
{
    if (!H || !o || !res) return fail2(MA_ERR_INVALID_ARG, "null argument");
    if (!(o->tol >= 0.0) || o->max_cycles < 0 || (o->norm != MA_NORM_MAX && o->norm != MA_NORM_L2) ||
        o->init < MA_INIT_FMG || o->init > MA_INIT_KEEP || o->relative < MA_REL_NONE || o->relative > MA_REL_INITIAL)
        return fail2(MA_ERR_INVALID_ARG, "bad solve options");
    std::memset(res, 0, sizeof *res);
    auto& F = H->lev[0];
    double mx = 0.0, l2 = 0.0, scale = 1.0;
    if (o->relative == MA_REL_INITIAL) {
        if (o->init != MA_INIT_KEEP) {
            ma::count_launches(1);
            k_zero_interior2<<<grid2(F.n, F.n), dim3(TX, TY), 0, H->s>>>(F.u, F.n);
        }
        ma_status st = fine_norms2(H, 2, &mx, &l2);
        if (st != MA_OK) return st;
        scale = o->norm == MA_NORM_MAX ? mx : l2;
    } else if (o->relative == MA_REL_RHS) {
        ma::count_launches(2);
        k_norm_partials2<<<grid2(F.n, F.n), dim3(TX, TY), 0, H->s>>>(F.rhs, F.n, H->partials);
        k_norm_final2<<<1, 1024, 0, H->s>>>(H->partials, H->npartials, F.h, H->out + 2);
        CK2(cudaGetLastError());
        CK2(cudaMemcpyAsync(H->host, H->out, 4 * sizeof(double), cudaMemcpyDeviceToHost, H->s));
        CK2(cudaStreamSynchronize(H->s));
        scale = o->norm == MA_NORM_MAX ? H->host[2] : H->host[3];
    }
    if (!(scale > 0.0)) scale = 1.0;
    if (o->init == MA_INIT_FMG) CK2(fmg2(H));
    if (o->init == MA_INIT_ZERO) {
        ma::count_launches(1);
        k_zero_interior2<<<grid2(F.n, F.n), dim3(TX, TY), 0, H->s>>>(F.u, F.n);
    }
    ma_status st = fine_norms2(H, 0, &mx, &l2);
    if (st != MA_OK) return st;
    double rel = (o->norm == MA_NORM_MAX ? mx : l2) / scale;
    res->res0 = rel;
    int stagnant = 0;
    // the max norm folds with fmax, which skips NaN entries; the L2 norm's
    // sum of squares does not, so both are checked
    while (std::isfinite(rel) && std::isfinite(l2) && rel > o->tol && res->cycles < o->max_cycles &&
           stagnant < ma::kFloorStagnantCycles) {
        CK2(vcycle2_from(H, 0));
        res->cycles += 1;
        if ((st = fine_norms2(H, 0, &mx, &l2)) != MA_OK) return st;
        const double nrel = (o->norm == MA_NORM_MAX ? mx : l2) / scale;
        stagnant = nrel > 0.8 * rel ? stagnant + 1 : 0;
        rel = nrel;
    }
    res->res = rel;
    if (!std::isfinite(rel) || !std::isfinite(l2)) res->status = MA_ERR_NONFINITE;
    else if (rel <= o->tol) res->status = MA_OK;
    else {
        res->status = MA_ERR_NOT_CONVERGED;
        res->floor_reached = stagnant >= ma::kFloorStagnantCycles;
    }
    if (res->status == MA_ERR_NONFINITE) return fail2(MA_ERR_NONFINITE, "residual became non-finite");
    if (res->status == MA_ERR_NOT_CONVERGED)
        return fail2(MA_ERR_NOT_CONVERGED, "not converged: residual %.3e > tol %.3e after %d cycles", rel, o->tol,
                     res->cycles);
    return MA_OK;
}

ma_status ma2d_get_solution(const ma2d_hierarchy* H, double* u)
{
    if (!H || !u) return fail2(MA_ERR_INVALID_ARG, "null argument");
    const size_t m = (size_t)H->lev[0].n * H->lev[0].n;
    CK2(cudaMemcpyAsync(u, H->lev[0].u, m * sizeof(double), cudaMemcpyDeviceToDevice, H->s));
    return MA_OK;
}

ma_status ma2d_smooth(double* u, const double* rhs, int n, double h, int nsweeps, int ordering, double* scratch,
                      unsigned long long* events, ma_stream_t stream)
{
    if (!u || !rhs || !valid_n2(n) || !(h > 0.0) || nsweeps < 0 ||
        (ordering != MA2D_REDBLACK && ordering != MA2D_COLOUR4) || (ordering == MA2D_REDBLACK && !scratch))
        return fail2(MA_ERR_INVALID_ARG, "ma2d_smooth: bad arguments");
    CK2(smooth2(u, scratch, rhs, n, h, nsweeps, ordering, events, (cudaStream_t)stream));
    return MA_OK;
}

ma_status ma2d_residual(const double* u, const double* rhs, double* r, int n, double h, ma_stream_t stream)
{
    if (!u || !rhs || !r || !valid_n2(n) || !(h > 0.0)) return fail2(MA_ERR_INVALID_ARG, "ma2d_residual: bad arguments");
    CK2(residual2(u, rhs, r, n, h, nullptr, (cudaStream_t)stream));
    return MA_OK;
}

ma_status ma2d_restrict_residual(const double* rf, int nf, double* rc, int kind, ma_stream_t stream)
{
    if (!rf || !rc || !valid_n2(nf) || nf < 5 || (kind != MA_HALF_WEIGHTING && kind != MA_FULL_WEIGHTING))
        return fail2(MA_ERR_INVALID_ARG, "ma2d_restrict_residual: bad arguments");
    const int nc = (nf + 1) / 2;
    ma::count_launches(1);
    k_restrict2<<<grid2(nc, nc), dim3(TX, TY), 0, (cudaStream_t)stream>>>(nullptr, rf, nf, nullptr, nullptr, rc, nc,
                                                                          kind, 0);
    CK2(cudaGetLastError());
    return MA_OK;
}

ma_status ma2d_prolong_add(const double* uc, const double* wc, int nc, double* uf, ma_stream_t stream)
{
    if (!uc || !wc || !uf || nc < 2 || nc > 16385) return fail2(MA_ERR_INVALID_ARG, "ma2d_prolong_add: bad arguments");
    const int nf = 2 * nc - 1;
    ma::count_launches(1);
    k_prolong2<<<grid2(nf, nf), dim3(TX, TY), 0, (cudaStream_t)stream>>>(uc, wc, nc, uf, nf, 1, 0);
    CK2(cudaGetLastError());
    return MA_OK;
}

ma_status ma2d_interpolate(const double* uc, int nc, double* uf, int cubic, ma_stream_t stream)
{
    if (!uc || !uf || nc < 2 || nc > 16385) return fail2(MA_ERR_INVALID_ARG, "ma2d_interpolate: bad arguments");
    const int nf = 2 * nc - 1;
    ma::count_launches(1);
    k_prolong2<<<grid2(nf, nf), dim3(TX, TY), 0, (cudaStream_t)stream>>>(uc, nullptr, nc, uf, nf, 0, cubic ? 1 : 0);
    CK2(cudaGetLastError());
    return MA_OK;
}

}  // extern "C"
