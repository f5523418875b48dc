// reduce.cu -- the once-per-grid reduction that yields the global-LF
// coefficients for state-only bounds (Listing 4: artificialDissipationGLF
// with partialFunc; alpha_k = max over the grid of the bound on |dH/dp_k|).
#include "launch.h"
#include "stage_generic.cuh"
#include "stage_tiled.cuh"
#include "adjoint.cuh"

namespace lsp {

cudaError_t launch_alpha_state(int dyn, const GridGeom& g, unsigned long long* out, cudaStream_t s)
{
    long long b = (g.npts + 255) / 256;
    const long long cap = 8LL * sm_count();
    const int nb = (int)(b < cap ? (b < 1 ? 1 : b) : cap);
    switch (dyn) {
    case NORMAL_SPEED: alpha_state_kernel<NORMAL_SPEED><<<nb, 256, 0, s>>>(g, out); break;
    case TRANSLATE: alpha_state_kernel<TRANSLATE><<<nb, 256, 0, s>>>(g, out); break;
    case AIR3D: alpha_state_kernel<AIR3D><<<nb, 256, 0, s>>>(g, out); break;
    case CAR4D: alpha_state_kernel<CAR4D><<<nb, 256, 0, s>>>(g, out); break;
    case ROCKETS: alpha_state_kernel<ROCKETS><<<nb, 256, 0, s>>>(g, out); break;
    case DOUBLE_INT: alpha_state_kernel<DOUBLE_INT><<<nb, 256, 0, s>>>(g, out); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

bool tile_valid(int ndim, int scheme, const Tile& t, const int* n)
{
    if (ndim != 3 && ndim != 4) return false;
    const int G = ghost_width(scheme);
    if (t.tb < 1 || t.ta < 1 || t.ch < 1) return false;
    if (t.minb < 2 || t.minb > 4) return false;
    const int nS = n[ndim - 3];
    const long long nz = (long long)((nS + t.ch - 1) / t.ch) * (ndim == 4 ? n[0] : 1);
    if (t.pair == 5) return fused_tile_ok(ndim, scheme, t, n);  // temporally blocked RK2
    if (t.pair == 3 || t.pair == 4) {  // face-shared ENO runs of 4 or 2 nodes
        return (scheme == ENO2 || scheme == ENO3) &&
               run_tile_ok(ndim, scheme, t.pair == 3 ? 4 : 2, t.tb, t.ta) && nz <= 65535;
    }
    if (t.tb * t.ta > 256) return false;
    // pair 1: paired planes (WENO5, ENO2, ENO3); pair 2: WENO5 shared faces
    if (t.pair < 0 || t.pair > 2) return false;
    if (t.pair == 1 && scheme != WENO5 && scheme != ENO2 && scheme != ENO3) return false;
    if (t.pair == 2 && scheme != WENO5) return false;
    // each thread stages at most 3 values of the haloed plane tile (MAXE of
    // the tiled bodies; every shape the autotuner tries qualifies)
    if ((t.ta + 2 * G) * (t.tb + 2 * G) > 3 * t.ta * t.tb) return false;
    return nz <= 65535;
}

bool run_tile_ok(int ndim, int scheme, int run, int tb, int ta)
{
    if (tb != 16 && tb != 28 && tb != 32) return false;
    const int tbt = tb / run, G = ghost_width(scheme);
    const size_t floats = (size_t)(ta + 2 * G) * (tb + 8) +
                          (size_t)((ndim == 4 ? 2 * G : 0) + 3) * ta * tb;
    return ta >= 1 && tbt * ta <= 256 && 2 * sizeof(float) * floats <= kRunMaxSmem;
}

cudaError_t launch_stage_tiled(int ndim, int scheme, int dyn, const StageArgs<float>& a,
                               const Tile& t, cudaStream_t s)
{
    // local coefficients and the variational clip run the scalar local
    // bodies, except on the WENO5 shared-face tile with state-only bounds,
    // whose kernel has a local variant
    if ((a.local_alpha || a.varform) && !(scheme == WENO5 && t.pair == 2 && dyn != QUADRATIC)) {
        // the face-shared runs have no local variant: a one-node-per-thread
        // tile of the same chunking runs the local body
        const Tile tl = (t.pair == 3 || t.pair == 4) ? Tile{32, 8, t.ch, 3, 0}
                                                     : Tile{t.tb, t.ta, t.ch, t.minb, 0};
        return launch_stage_tiled_local(ndim, scheme, dyn, a, tl, s);
    }
    if (t.pair == 5) {  // a single stage on a fused-RK2 tile: the scalar body
        const Tile ts{t.tb, t.ta, t.ch, t.minb, 0};
        return launch_stage_tiled(ndim, scheme, dyn, a, ts, s);
    }
    if (t.pair == 3) return launch_stage_run_r<4>(ndim, scheme, dyn, a, t, s);
    if (t.pair == 4) return launch_stage_run_r<2>(ndim, scheme, dyn, a, t, s);
    switch (t.minb) {
    case 2: return launch_stage_tiled_m<2>(ndim, scheme, dyn, a, t, s);
    case 3: return launch_stage_tiled_m<3>(ndim, scheme, dyn, a, t, s);
    case 4: return launch_stage_tiled_m<4>(ndim, scheme, dyn, a, t, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_alpha_argmax(int dyn, const GridGeom& g, const double* alpha,
                                unsigned long long* out, cudaStream_t s)
{
    long long b = (g.npts + 255) / 256;
    const long long cap = 8LL * sm_count();
    const int nb = (int)(b < cap ? (b < 1 ? 1 : b) : cap);
    switch (dyn) {
    case NORMAL_SPEED: alpha_argmax_kernel<NORMAL_SPEED><<<nb, 256, 0, s>>>(g, alpha, out); break;
    case TRANSLATE: alpha_argmax_kernel<TRANSLATE><<<nb, 256, 0, s>>>(g, alpha, out); break;
    case AIR3D: alpha_argmax_kernel<AIR3D><<<nb, 256, 0, s>>>(g, alpha, out); break;
    case CAR4D: alpha_argmax_kernel<CAR4D><<<nb, 256, 0, s>>>(g, alpha, out); break;
    case ROCKETS: alpha_argmax_kernel<ROCKETS><<<nb, 256, 0, s>>>(g, alpha, out); break;
    case DOUBLE_INT: alpha_argmax_kernel<DOUBLE_INT><<<nb, 256, 0, s>>>(g, alpha, out); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

bool stage_supported(int ndim, int scheme, int dyn)
{
    if (ndim < 1 || ndim > LSP_MAXD || scheme < UPWIND1 || scheme > WENO5) return false;
    if (dyn == AIR3D) return ndim == 3;
    if (dyn == CAR4D) return ndim == 4;
    if (dyn == ROCKETS) return ndim == 3;
    if (dyn == DOUBLE_INT) return ndim == 2;
    return dyn >= NORMAL_SPEED && dyn <= QUADRATIC;
}

}  // namespace lsp
