// stage_tiled_local.cu -- the tiled stage kernels with local dissipation
// coefficients (LLF / LLLF) and the variational clip compiled in
// (tiled_stage_body<..., LOCAL = true>), for every 3-D / 4-D dynamics and
// scheme, at the 3-CTAs-per-SM register budget whatever the tile's minb.
#include "launch.h"
#include "stage_tiled.cuh"

namespace lsp {

template <int NDIM, int SCHEME, int DYN>
static cudaError_t local_one(const StageArgs<float>& a, const Tile& t, cudaStream_t s)
{
    constexpr int G = ghost_width(SCHEME);
    const int nB = a.n[NDIM - 1], nA = a.n[NDIM - 2], nS = a.n[NDIM - 3];
    const int nchunks = (nS + t.ch - 1) / t.ch;
    dim3 block(t.tb, t.ta, 1);
    dim3 grid((nB + t.tb - 1) / t.tb, (nA + t.ta - 1) / t.ta, nchunks * (NDIM == 4 ? a.n[0] : 1));
    const size_t smem = 2 * sizeof(float) * (t.ta + 2 * G) * (t.tb + 2 * G);
    stage_tiled_kernel<NDIM, SCHEME, DYN, float, 3, true><<<grid, block, smem, s>>>(a, t.ch, nchunks);
    return cudaGetLastError();
}

template <int NDIM, int SCHEME>
static cudaError_t local_dyn(int dyn, const StageArgs<float>& a, const Tile& t, cudaStream_t s)
{
    switch (dyn) {
    case NORMAL_SPEED: return local_one<NDIM, SCHEME, NORMAL_SPEED>(a, t, s);
    case TRANSLATE: return local_one<NDIM, SCHEME, TRANSLATE>(a, t, s);
    case QUADRATIC: return local_one<NDIM, SCHEME, QUADRATIC>(a, t, s);
    case AIR3D:
        if constexpr (NDIM == 3) return local_one<3, SCHEME, AIR3D>(a, t, s);
        break;
    case ROCKETS:
        if constexpr (NDIM == 3) return local_one<3, SCHEME, ROCKETS>(a, t, s);
        break;
    case CAR4D:
        if constexpr (NDIM == 4) return local_one<4, SCHEME, CAR4D>(a, t, s);
        break;
    }
    return cudaErrorInvalidValue;
}

template <int NDIM>
static cudaError_t local_scheme(int scheme, int dyn, const StageArgs<float>& a, const Tile& t,
                                cudaStream_t s)
{
    switch (scheme) {
    case UPWIND1: return local_dyn<NDIM, UPWIND1>(dyn, a, t, s);
    case ENO2: return local_dyn<NDIM, ENO2>(dyn, a, t, s);
    case ENO3: return local_dyn<NDIM, ENO3>(dyn, a, t, s);
    case WENO5: return local_dyn<NDIM, WENO5>(dyn, a, t, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_stage_tiled_local(int ndim, int scheme, int dyn, const StageArgs<float>& a,
                                     const Tile& t, cudaStream_t s)
{
    if (ndim == 3) return local_scheme<3>(scheme, dyn, a, t, s);
    if (ndim == 4) return local_scheme<4>(scheme, dyn, a, t, s);
    return cudaErrorInvalidValue;
}

}  // namespace lsp
