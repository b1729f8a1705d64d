// ma_batched.cuh -- launches that cover the grids of several hierarchies at
// once.  A launch carries a table of jobs (one per hierarchy with work at this
// step: its pointers, sizes and grid shape) and the first block of each job;
// block b finds its job by binary search, skips it when the hierarchy's
// active flag is 0, and runs the block body of the single-grid kernel with
// its block index inside that job's grid, so both forms compute the same
// bits.  The job tables are built on the host (TableBuilder) and live in
// device memory the caller provides.
#pragma once

#include <cuda_runtime.h>

#include <cstring>
#include <vector>

namespace ma {

void count_launches(unsigned long long k);

namespace batched {

// One launch of a plan: operation id, jobs, total blocks, dynamic shared
// memory, and the offsets of its job table and block starts in the tables.
struct BLaunch {
    int op, njobs, blocks, smem;
    size_t jobs_off, starts_off;
};

// Accumulates the job tables of a plan in host memory, each table (jobs,
// then njobs + 1 block starts) 256-byte aligned.
struct TableBuilder {
    std::vector<char> buf;
    std::vector<BLaunch> seq;
    static size_t align(size_t x) { return (x + 255) / 256 * 256; }
    template <typename Job>
    void emit(int op, const std::vector<Job>& jobs, const std::vector<int>& blocks, int smem)
    {
        if (jobs.empty()) return;
        BLaunch L;
        L.op = op;
        L.njobs = (int)jobs.size();
        L.smem = smem;
        L.jobs_off = align(buf.size());
        L.starts_off = align(L.jobs_off + sizeof(Job) * jobs.size());
        buf.resize(align(L.starts_off + sizeof(int) * (jobs.size() + 1)), 0);
        std::memcpy(buf.data() + L.jobs_off, jobs.data(), sizeof(Job) * jobs.size());
        int* st = (int*)(buf.data() + L.starts_off);
        int acc = 0;
        for (size_t q = 0; q < jobs.size(); ++q) {
            st[q] = acc;
            acc += blocks[q];
        }
        st[jobs.size()] = acc;
        L.blocks = acc;
        if (acc > 0) seq.push_back(L);
    }
};

// Block q of a job grid of gx x gy x (any) blocks as a 3-D block index.
__device__ __forceinline__ uint3 split_block(int q, int gx, int gy)
{
    const int gxy = gx * gy;
    const int bz = q / gxy, r = q - bz * gxy;
    const int by = r / gx, bx = r - by * gx;
    return make_uint3((unsigned)bx, (unsigned)by, (unsigned)bz);
}

template <typename Op>
__global__ void __launch_bounds__(Op::NT, Op::MINB)
    k_batched(const typename Op::Job* __restrict__ jobs, const int* __restrict__ start, int njobs,
              const int* __restrict__ active)
{
    const int b = (int)blockIdx.x;
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    const typename Op::Job& J = jobs[lo];
    if (!active[J.inst]) return;   // uniform over the block
    Op::run(J, b - start[lo]);
}

template <typename Op>
cudaError_t launch(const char* tables, const BLaunch& L, dim3 block, const int* active, cudaStream_t s)
{
    count_launches(1);
    k_batched<Op><<<L.blocks, block, L.smem, s>>>((const typename Op::Job*)(tables + L.jobs_off),
                                                  (const int*)(tables + L.starts_off), L.njobs, active);
    return cudaGetLastError();
}

// Operation ids below kF64Ops belong to the mixed-precision kernels, the
// others to the FP64 kernels (each file dispatches its own).
constexpr int kF64Ops = 100;

}  // namespace batched
}  // namespace ma
