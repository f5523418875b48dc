// launch.h -- host-side entry points of the kernels (defined in the
// per-precision translation units).
#pragma once
#include "lsp_internal.h"

namespace lsp {

struct GridGeom;

// Fused stage (generic one-thread-per-node kernel).
template <typename R>
cudaError_t launch_stage(int ndim, int scheme, int dyn, const StageArgs<R>& a, cudaStream_t s);

// Costate range reduction for H = |p|^2/2 (alpha from the current field).
template <typename R>
cudaError_t launch_prange(int ndim, int scheme, const StageArgs<R>& a, cudaStream_t s);

// State-only global-LF coefficients (FP64).
cudaError_t launch_alpha_state(int dyn, const GridGeom& g, unsigned long long* out, cudaStream_t s);

// Is there a kernel for this combination?
bool stage_supported(int ndim, int scheme, int dyn);

}  // namespace lsp
