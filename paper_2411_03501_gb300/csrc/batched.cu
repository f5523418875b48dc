// batched.cu -- many independent level-set problems of different shapes,
// dynamics and step sizes advanced together.
//
// Each problem keeps its own grid, CFL step and step count (the FP64 time
// loop of a single solve, per problem).  One launch advances stage s of step
// k of every problem that still has steps left: a table maps each CTA of the
// launch to (problem, tile), and each CTA runs the tiled stage body of
// stage_tiled.cuh on its problem's fields.  Problems are ordered by
// decreasing step count, so the problems active at step k are a prefix of the
// table and the launch is simply shortened as problems finish.  The whole
// sequence of launches can be captured into one CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "batched.cuh"

namespace lsp {

cudaError_t launch_batched(int scheme, const BatchProblem* probs, const int* block_prob, int nblocks,
                           int step, int stage, int rk, bool local, cudaStream_t s)
{
    if (local) return launch_batched_local(scheme, probs, block_prob, nblocks, step, stage, rk, s);
    return launch_batched_t<false>(scheme, probs, block_prob, nblocks, step, stage, rk, s);
}

cudaError_t launch_batched_persistent(int scheme, const BatchProblem* probs, const int* block_prob,
                                      const BatchSegment* segs, int nseg, int rk,
                                      unsigned int* done, PersistCtl* pc, Ctl* ctl,
                                      unsigned long long wait_ns, bool local, cudaStream_t s)
{
    if (local)
        return launch_batched_persistent_local(scheme, probs, block_prob, segs, nseg, rk, done, pc,
                                               ctl, wait_ns, s);
    return launch_batched_persistent_t<false>(scheme, probs, block_prob, segs, nseg, rk, done, pc,
                                              ctl, wait_ns, s);
}

void batch_tile_dims(int* tb, int* ta)
{
    *tb = kBatchTB;
    *ta = kBatchTA;
}

bool batch_supported(int ndim, int dyn)
{
    if (ndim == 2) return dyn == NORMAL_SPEED || dyn == TRANSLATE || dyn == DOUBLE_INT;
    if (ndim == 3) return dyn == NORMAL_SPEED || dyn == TRANSLATE || dyn == AIR3D || dyn == ROCKETS;
    if (ndim == 4) return dyn == NORMAL_SPEED || dyn == TRANSLATE || dyn == CAR4D;
    return false;
}

}  // namespace lsp
