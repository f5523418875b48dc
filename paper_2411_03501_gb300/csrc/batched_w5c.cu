// batched.cuh instantiations: WENO5, global-LF form, compiled for 2-D normal
// speed and 3-D air3d problems alone (the mixed workload), with every tile
// shape and with 16 x 16 tiles only.
#include "batched.cuh"

namespace lsp {
LSP_BATCHED_INSTANTIATE(WENO5, false, kClsNormal2Air3)
LSP_BATCHED_INSTANTIATE(WENO5, false, kClsNormal2Air3x16)
}  // namespace lsp
