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

#include "batched.h"
#include "launch.h"

namespace lsp {

// the launches instantiated in the batched_*.cu translation units
// (batched.cuh)
template <int SCHEME, bool LOCAL, int CLS>
cudaError_t launch_batched_k(const BatchProblem* probs, const int* block_prob, int nblocks,
                             int step, int stage, int rk, cudaStream_t s);
template <int SCHEME, bool LOCAL, int CLS>
cudaError_t launch_persistent_k(const BatchProblem* probs, const int* block_prob,
                                const BatchSegment* segs, int nseg, int rk, unsigned int* done,
                                PersistCtl* pc, Ctl* ctl, unsigned long long wait_ns,
                                cudaStream_t s);

namespace {

// Local kernels cover every class; the two-class kernels exist for WENO5,
// the scheme of the mixed workload (the other schemes use the full set).
template <bool LOCAL>
cudaError_t batched_dispatch(int scheme, int cls, bool persistent, const BatchProblem* probs,
                             const int* block_prob, int nblocks, int step, int stage, int rk,
                             const BatchSegment* segs, int nseg, unsigned int* done, PersistCtl* pc,
                             Ctl* ctl, unsigned long long wait_ns, cudaStream_t s)
{
#define LSP_BATCHED_CALL(SCHEME, CLS)                                                              \
    return persistent ? launch_persistent_k<SCHEME, LOCAL, CLS>(probs, block_prob, segs, nseg, rk, \
                                                                done, pc, ctl, wait_ns, s)         \
                      : launch_batched_k<SCHEME, LOCAL, CLS>(probs, block_prob, nblocks, step,    \
                                                             stage, rk, s)
    switch (scheme) {
    case UPWIND1: LSP_BATCHED_CALL(UPWIND1, kBatchClsAll);
    case ENO2: LSP_BATCHED_CALL(ENO2, kBatchClsAll);
    case ENO3: LSP_BATCHED_CALL(ENO3, kBatchClsAll);
    case WENO5:
        if (!LOCAL && cls == kBatchClsNormal2Air3x16) LSP_BATCHED_CALL(WENO5, kBatchClsNormal2Air3x16);
        if (!LOCAL && cls == kBatchClsNormal2Air3) LSP_BATCHED_CALL(WENO5, kBatchClsNormal2Air3);
        LSP_BATCHED_CALL(WENO5, kBatchClsAll);
    }
#undef LSP_BATCHED_CALL
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_batched(int scheme, const BatchProblem* probs, const int* block_prob, int nblocks,
                           int step, int stage, int rk, bool local, int cls, cudaStream_t s)
{
    if (local)
        return batched_dispatch<true>(scheme, cls, false, probs, block_prob, nblocks, step, stage,
                                      rk, nullptr, 0, nullptr, nullptr, nullptr, 0, s);
    return batched_dispatch<false>(scheme, cls, false, probs, block_prob, nblocks, step, stage, rk,
                                   nullptr, 0, nullptr, nullptr, nullptr, 0, s);
}

cudaError_t launch_batched_persistent(int scheme, const BatchProblem* probs, const int* block_prob,
                                      const BatchSegment* segs, int nseg, int rk,
                                      unsigned int* done, PersistCtl* pc, Ctl* ctl,
                                      unsigned long long wait_ns, bool local, int cls,
                                      cudaStream_t s)
{
    if (local)
        return batched_dispatch<true>(scheme, cls, true, probs, block_prob, 0, 0, 0, rk, segs, nseg,
                                      done, pc, ctl, wait_ns, s);
    return batched_dispatch<false>(scheme, cls, true, probs, block_prob, 0, 0, 0, rk, segs, nseg,
                                   done, pc, ctl, wait_ns, s);
}

bool batch_tile_dims(int shape, int* tb, int* ta)
{
    if (shape < 0 || shape >= kBatchNumShapes) return false;
    *tb = kBatchShapes[shape][0];
    *ta = kBatchShapes[shape][1];
    return true;
}

bool batch_supported(int ndim, int dyn)
{
    if (ndim == 2) return dyn == NORMAL_SPEED || dyn == TRANSLATE || dyn == DOUBLE_INT;
    if (ndim == 3) return dyn == NORMAL_SPEED || dyn == TRANSLATE || dyn == AIR3D || dyn == ROCKETS;
    if (ndim == 4) return dyn == NORMAL_SPEED || dyn == TRANSLATE || dyn == CAR4D;
    return false;
}

}  // namespace lsp
