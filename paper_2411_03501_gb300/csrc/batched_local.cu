// batched_local.cu -- batched.cuh instantiations with local dissipation
// coefficients and the variational clip compiled in (LOCAL = true), WENO5,
// every problem class; a translation unit of its own so that it compiles
// in parallel.
#include "batched.cuh"

namespace lsp {
LSP_BATCHED_INSTANTIATE(WENO5, true, kClsAll)
}  // namespace lsp
