// batched.cuh instantiations: ENO3, global-LF form, every problem class.
#include "batched.cuh"

namespace lsp {
LSP_BATCHED_INSTANTIATE(ENO3, false, kClsAll)
}  // namespace lsp
