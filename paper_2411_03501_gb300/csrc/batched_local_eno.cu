// batched.cuh instantiations with local dissipation coefficients and the
// variational clip compiled in (LOCAL = true): first order, ENO2, ENO3.
#include "batched.cuh"

namespace lsp {
LSP_BATCHED_INSTANTIATE(UPWIND1, true, kClsAll)
LSP_BATCHED_INSTANTIATE(ENO2, true, kClsAll)
LSP_BATCHED_INSTANTIATE(ENO3, true, kClsAll)
}  // namespace lsp
