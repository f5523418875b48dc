// batched.cuh instantiations: WENO5, global-LF form, every problem class: the persistent kernel.
#include "batched.cuh"

namespace lsp {
LSP_BATCHED_INSTANTIATE_PERSISTENT(WENO5, false, kClsAll)
}  // namespace lsp
