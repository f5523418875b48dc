// stage_tiled.inl -- FP32 instantiations of the tiled stage kernel for one
// occupancy target LSP_MINB (included by stage_tiled_m{2,3,4}.cu).
#include "launch.h"
#include "stage_pair.cuh"
#include "stage_tiled.cuh"

namespace lsp {

template <int NDIM, int SCHEME, int DYN>
static cudaError_t tiled_one(const StageArgs<float>& a, const Tile& t, cudaStream_t s)
{
    constexpr int G = ghost_width(SCHEME);
    const int nB = a.n[NDIM - 1], nA = a.n[NDIM - 2], nS = a.n[NDIM - 3];
    const int nchunks = (nS + t.ch - 1) / t.ch;
    dim3 block(t.tb, t.ta, 1);
    dim3 grid((nB + t.tb - 1) / t.tb, (nA + t.ta - 1) / t.ta,
              nchunks * (NDIM == 4 ? a.n[0] : 1));
    const size_t smem = 2 * sizeof(float) * (t.ta + 2 * G) * (t.tb + 2 * G);
    // Local coefficients and the variational clip reach this file only on
    // the WENO5 shared-face tile with state-only bounds (its local variant);
    // launch_stage_tiled sends every other such stage to
    // stage_tiled_local.cu, and any other kernel here would drop them.
    constexpr bool kPairLocal = SCHEME == WENO5 && DYN != QUADRATIC;
    const bool local = a.local_alpha || a.varform;
    if (local && !(kPairLocal && t.pair == 2)) return cudaErrorInvalidValue;
    if constexpr (SCHEME == WENO5 || SCHEME == ENO2 || SCHEME == ENO3) {
        if (t.pair == 1) {
            stage_pair_kernel<NDIM, DYN, LSP_MINB, false, SCHEME><<<grid, block, 2 * smem, s>>>(a, t.ch, nchunks);
            return cudaGetLastError();
        }
    }
    if constexpr (SCHEME == WENO5) {
        if (t.pair == 2) {
            if constexpr (kPairLocal) {
                if (local) {
                    stage_pair_kernel<NDIM, DYN, LSP_MINB, true, WENO5, true>
                        <<<grid, block, 2 * smem, s>>>(a, t.ch, nchunks);
                    return cudaGetLastError();
                }
            }
            stage_pair_kernel<NDIM, DYN, LSP_MINB, true><<<grid, block, 2 * smem, s>>>(a, t.ch, nchunks);
            return cudaGetLastError();
        }
    }
    stage_tiled_kernel<NDIM, SCHEME, DYN, float, LSP_MINB><<<grid, block, smem, s>>>(a, t.ch, nchunks);
    return cudaGetLastError();
}

template <int NDIM, int SCHEME>
static cudaError_t tiled_dyn(int dyn, const StageArgs<float>& a, const Tile& t, cudaStream_t s)
{
    switch (dyn) {
    case NORMAL_SPEED: return tiled_one<NDIM, SCHEME, NORMAL_SPEED>(a, t, s);
    case TRANSLATE: return tiled_one<NDIM, SCHEME, TRANSLATE>(a, t, s);
    case QUADRATIC: return tiled_one<NDIM, SCHEME, QUADRATIC>(a, t, s);
    case AIR3D:
        if constexpr (NDIM == 3) return tiled_one<3, SCHEME, AIR3D>(a, t, s);
        break;
    case CAR4D:
        if constexpr (NDIM == 4) return tiled_one<4, SCHEME, CAR4D>(a, t, s);
        break;
    case ROCKETS:
        if constexpr (NDIM == 3) return tiled_one<3, SCHEME, ROCKETS>(a, t, s);
        break;
    }
    return cudaErrorInvalidValue;
}

template <int NDIM>
static cudaError_t tiled_scheme(int scheme, int dyn, const StageArgs<float>& a, const Tile& t,
                                cudaStream_t s)
{
    switch (scheme) {
    case UPWIND1: return tiled_dyn<NDIM, UPWIND1>(dyn, a, t, s);
    case ENO2: return tiled_dyn<NDIM, ENO2>(dyn, a, t, s);
    case ENO3: return tiled_dyn<NDIM, ENO3>(dyn, a, t, s);
    case WENO5: return tiled_dyn<NDIM, WENO5>(dyn, a, t, s);
    }
    return cudaErrorInvalidValue;
}

template <>
cudaError_t launch_stage_tiled_m<LSP_MINB>(int ndim, int scheme, int dyn,
                                           const StageArgs<float>& a, const Tile& t,
                                           cudaStream_t s)
{
    if (ndim == 3) return tiled_scheme<3>(scheme, dyn, a, t, s);
    if (ndim == 4) return tiled_scheme<4>(scheme, dyn, a, t, s);
    return cudaErrorInvalidValue;
}

}  // namespace lsp
