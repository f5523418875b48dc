// stage_run.inl -- instantiations and launcher of the face-shared ENO2/ENO3
// stage kernel (stage_run.cuh) for 3-D and 4-D FP32 grids, for one run
// length LSP_RUN_R and register budget LSP_RUN_MINB (included by
// stage_run_r4.cu, Tile.pair = 3, and stage_run_r2.cu, Tile.pair = 4).
#include "launch.h"
#include "stage_run.cuh"

namespace lsp {

namespace {

constexpr int R = LSP_RUN_R;

template <int NDIM, int SCHEME, int DYN, int TBT>
cudaError_t run_launch(const StageArgs<float>& a, const Tile& t, cudaStream_t s)
{
    constexpr int TB = RunLayout<R, TBT>::TB;
    const int nB = a.n[NDIM - 1], nA = a.n[NDIM - 2], nS = a.n[NDIM - 3];
    const int nchunks = (nS + t.ch - 1) / t.ch;
    dim3 block(TBT, t.ta, 1);
    dim3 grid((nB + TB - 1) / TB, (nA + t.ta - 1) / t.ta, nchunks * (NDIM == 4 ? a.n[0] : 1));
    const size_t smem = 2 * sizeof(float) * (size_t)run_plane_floats<NDIM, SCHEME, R, TBT>(t.ta);
    if (smem > kRunMaxSmem) return cudaErrorInvalidValue;
    auto* fn = stage_run_kernel<NDIM, SCHEME, DYN, R, TBT, LSP_RUN_MINB>;
    static const cudaError_t attr =
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRunMaxSmem);
    if (attr != cudaSuccess) return attr;
    fn<<<grid, block, smem, s>>>(a, t.ch, nchunks);
    return cudaGetLastError();
}

template <int NDIM, int SCHEME, int DYN>
cudaError_t run_tbt(const StageArgs<float>& a, const Tile& t, cudaStream_t s)
{
    switch (t.tb / R) {
    case 16 / R: return run_launch<NDIM, SCHEME, DYN, 16 / R>(a, t, s);
    case 28 / R: return run_launch<NDIM, SCHEME, DYN, 28 / R>(a, t, s);
    case 32 / R: return run_launch<NDIM, SCHEME, DYN, 32 / R>(a, t, s);
    }
    return cudaErrorInvalidValue;
}

template <int NDIM, int SCHEME>
cudaError_t run_dyn(int dyn, const StageArgs<float>& a, const Tile& t, cudaStream_t s)
{
    switch (dyn) {
    case NORMAL_SPEED: return run_tbt<NDIM, SCHEME, NORMAL_SPEED>(a, t, s);
    case TRANSLATE: return run_tbt<NDIM, SCHEME, TRANSLATE>(a, t, s);
    case QUADRATIC: return run_tbt<NDIM, SCHEME, QUADRATIC>(a, t, s);
    case AIR3D:
        if constexpr (NDIM == 3) return run_tbt<3, SCHEME, AIR3D>(a, t, s);
        break;
    case ROCKETS:
        if constexpr (NDIM == 3) return run_tbt<3, SCHEME, ROCKETS>(a, t, s);
        break;
    case CAR4D:
        if constexpr (NDIM == 4) return run_tbt<4, SCHEME, CAR4D>(a, t, s);
        break;
    }
    return cudaErrorInvalidValue;
}

}  // namespace

template <>
cudaError_t launch_stage_run_r<LSP_RUN_R>(int ndim, int scheme, int dyn, const StageArgs<float>& a,
                                          const Tile& t, cudaStream_t s)
{
    if (t.tb % R) return cudaErrorInvalidValue;
    if (ndim == 3 && scheme == ENO2) return run_dyn<3, ENO2>(dyn, a, t, s);
    if (ndim == 3 && scheme == ENO3) return run_dyn<3, ENO3>(dyn, a, t, s);
    if (ndim == 4 && scheme == ENO2) return run_dyn<4, ENO2>(dyn, a, t, s);
    if (ndim == 4 && scheme == ENO3) return run_dyn<4, ENO3>(dyn, a, t, s);
    return cudaErrorInvalidValue;
}

}  // namespace lsp
