// reduce.cu -- the once-per-grid reduction that yields the global-LF
// coefficients for state-only bounds (Listing 4: artificialDissipationGLF
// with partialFunc; alpha_k = max over the grid of the bound on |dH/dp_k|).
#include "launch.h"
#include "stage_generic.cuh"

namespace lsp {

cudaError_t launch_alpha_state(int dyn, const GridGeom& g, unsigned long long* out, cudaStream_t s)
{
    long long b = (g.npts + 255) / 256;
    const int nb = (int)(b < 152 * 8 ? (b < 1 ? 1 : b) : 152 * 8);
    switch (dyn) {
    case NORMAL_SPEED: alpha_state_kernel<NORMAL_SPEED><<<nb, 256, 0, s>>>(g, out); break;
    case TRANSLATE: alpha_state_kernel<TRANSLATE><<<nb, 256, 0, s>>>(g, out); break;
    case AIR3D: alpha_state_kernel<AIR3D><<<nb, 256, 0, s>>>(g, out); break;
    case CAR4D: alpha_state_kernel<CAR4D><<<nb, 256, 0, s>>>(g, out); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

bool stage_supported(int ndim, int scheme, int dyn)
{
    if (ndim < 1 || ndim > LSP_MAXD || scheme < UPWIND1 || scheme > WENO5) return false;
    if (dyn == AIR3D) return ndim == 3;
    if (dyn == CAR4D) return ndim == 4;
    return dyn >= NORMAL_SPEED && dyn <= QUADRATIC;
}

}  // namespace lsp
