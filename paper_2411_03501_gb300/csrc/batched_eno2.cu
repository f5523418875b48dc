// batched.cuh instantiations: ENO2, global-LF form, every problem class.
#include "batched.cuh"

namespace lsp {
LSP_BATCHED_INSTANTIATE(ENO2, false, kClsAll)
}  // namespace lsp
