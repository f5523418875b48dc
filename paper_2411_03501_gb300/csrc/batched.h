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
};

constexpr int kBatchTB = 32, kBatchTA = 8;

}  // namespace lsp
