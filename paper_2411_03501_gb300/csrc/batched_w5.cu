// batched.cuh instantiations: WENO5, global-LF form, every problem class: the stage-synchronous kernel.
#include "batched.cuh"

namespace lsp {
LSP_BATCHED_INSTANTIATE_STAGE(WENO5, false, kClsAll)
}  // namespace lsp
