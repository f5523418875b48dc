// batched.h -- the per-problem descriptor of a batched solve, shared by the
// host layer (which builds the table) and the batched stage kernel.
#pragma once
#include "lsp_internal.h"

namespace lsp {

struct BatchProblem {
    StageArgs<float> a;  // geometry, alpha, parameters, ctl (stage fields set per launch)
    float* phi;
    float* w1;
    float* w2;
    const float* target;
    double dt, dt_last;  // regular CFL step and the last (shortened) one
    int nsteps;
    int ndim, dyn;
    int ch, nbx, nby, nchunks;  // tile grid: x-tiles, y-tiles, chunks along the march
    int block_start, nblocks;   // this problem's CTAs in the launch
    int tb, ta;                 // tile of the two fastest axes (tb x ta = kBatchThreads)
};

// Every batched CTA has kBatchThreads threads; each problem's tile of its two
// fastest axes is one of kBatchShapes (chosen per problem dimension by
// lsp_solve_opts.batch_tiles), thread t covering (t % tb, t / tb).
constexpr int kBatchThreads = 256;
constexpr int kBatchNumShapes = 3;
constexpr int kBatchShapes[kBatchNumShapes][2] = {{16, 16}, {32, 8}, {64, 4}};
// the largest haloed tile of the shapes, in floats, for ghost width G
__host__ __device__ constexpr int batch_max_tile(int G)
{
    return (16 + 2 * G) * (16 + 2 * G) > (8 + 2 * G) * (32 + 2 * G)
               ? ((16 + 2 * G) * (16 + 2 * G) > (4 + 2 * G) * (64 + 2 * G)
                      ? (16 + 2 * G) * (16 + 2 * G) : (4 + 2 * G) * (64 + 2 * G))
               : ((8 + 2 * G) * (32 + 2 * G) > (4 + 2 * G) * (64 + 2 * G)
                      ? (8 + 2 * G) * (32 + 2 * G) : (4 + 2 * G) * (64 + 2 * G));
}

// Persistent batched launch: work items (step k, stage s, tile b) are handed
// out in this order by one counter; the steps split into segments with a
// constant set of active problems (a prefix of the table).
struct BatchSegment {
    long long item_start;  // first item of the segment
    int k_start;           // first step of the segment
    int blocks;            // CTAs per stage in the segment
};

struct PersistCtl {
    unsigned long long next;  // next work item
    unsigned int abort;       // set once a CTA gave up waiting
    int stall_problem;        // test hook: this problem never reports done (-1: none)
    unsigned long long pad[30];
};
static_assert(sizeof(PersistCtl) <= 256, "persistent control block must fit 256 bytes");

}  // namespace lsp
