// batched.cuh instantiations: first order, global-LF form, every problem class.
#include "batched.cuh"

namespace lsp {
LSP_BATCHED_INSTANTIATE(UPWIND1, false, kClsAll)
}  // namespace lsp
