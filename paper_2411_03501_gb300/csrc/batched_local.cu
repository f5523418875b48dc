// batched_local.cu -- the batched kernels with local dissipation
// coefficients and the variational clip compiled in (batched.cuh, LOCAL =
// true); a translation unit of its own so that it compiles in parallel.
#include "batched.cuh"

namespace lsp {

cudaError_t launch_batched_local(int scheme, const BatchProblem* probs, const int* block_prob,
                                 int nblocks, int step, int stage, int rk, cudaStream_t s)
{
    return launch_batched_t<true>(scheme, probs, block_prob, nblocks, step, stage, rk, s);
}

cudaError_t launch_batched_persistent_local(int scheme, const BatchProblem* probs,
                                            const int* block_prob, const BatchSegment* segs,
                                            int nseg, int rk, unsigned int* done, PersistCtl* pc,
                                            Ctl* ctl, unsigned long long wait_ns, cudaStream_t s)
{
    return launch_batched_persistent_t<true>(scheme, probs, block_prob, segs, nseg, rk, done, pc,
                                             ctl, wait_ns, s);
}

}  // namespace lsp
