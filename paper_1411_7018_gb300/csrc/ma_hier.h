// ma_hier.h -- host-side state of a hierarchy (internal).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "ma.h"

namespace ma {

constexpr int kMaxLevels = 16;

// One grid of the hierarchy: n points per side, step h; all fields are
// n^3 doubles in the caller's workspace.
struct Level {
    int n = 0;
    double h = 0.0;
    double* u = nullptr;     // iterate (w_h / u_H of Algorithm 1); shell = Dirichlet data
    double* rhs = nullptr;   // f on the finest level, b_H on coarse levels
    double* r = nullptr;     // residual; on coarse levels the restricted r_H
    double* w = nullptr;     // coarse levels: the restricted approximation w_H
    // mixed precision (FP32 correction cycle); null in FP64 mode
    float* e = nullptr;      // correction
    float* e2 = nullptr;     // second correction buffer of the plane sweeps (not on the coarsest level)
    void* bstore = nullptr;  // B = D^2_h u, colour-major FP32 (6 per interior point), refreshed per outer iteration
    float* hi = nullptr;     // coarse levels: base u = hi + lo (FP32 split of the injected iterate)
    float* lo = nullptr;
    float* rhs32 = nullptr;  // correction-problem right-hand side, colour-major (fine: the FP64 residual)
    float* res32 = nullptr;  // correction residual; on coarse levels the restricted one
    float* w32 = nullptr;    // coarse levels: the restricted correction
};

}  // namespace ma

namespace ma {
// A captured sequence of launches, replayed as one CUDA graph.
struct GraphSlot {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned long long launches = 0;   // kernels in the graph
};
}  // namespace ma

struct ma_hierarchy {
    ma_hier_desc d{};
    int L = 0;
    ma::Level lev[ma::kMaxLevels];
    cudaStream_t s = nullptr;
    int device = 0;
    char* ws = nullptr;
    size_t bytes = 0;
    double* partials = nullptr;          // norm partials (2 per block)
    int npartials = 0;
    // Device read-back block (5 x 8 bytes, copied to the host in one piece):
    // [0..1] residual norms (max, L2), [2..3] rhs norms, [4] nonconvex root
    // events (unsigned 64-bit).
    double* rb = nullptr;
    double* out2 = nullptr;                // = rb: where the residual norms land
    unsigned long long* events = nullptr;  // = rb + 4
    int* flag = nullptr;                 // device: input validation count
    double* host = nullptr;              // pinned host copy of the read-back block
    cudaStream_t cap = nullptr;          // private stream the graphs are captured on
    ma::GraphSlot g_init[6];             // per ma_solve init kind (and reference kind): init + first residual norm
    ma::GraphSlot g_cycle;               // one cycle + residual norm
    // Non-blocking solve state (ma_solve_begin / ma_solve_advance).
    struct {
        ma_solve_opts o{};
        int phase = 0;                   // 0 idle, 1 init norms pending, 2 cycle norms pending, 3 done
        double scale = 1.0, rel = 0.0;
        int stagnant = 0;
        ma_solve_result r{};
        cudaEvent_t ev = nullptr;        // marks the read-back of the latest norms
    } sv;
};
