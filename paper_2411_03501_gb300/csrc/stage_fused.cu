// stage_fused.cu -- launches of the temporally blocked TVD-RK2 step
// (stage_fused.cuh): 3-D FP32 grids, every scheme, the dynamics with
// state-only dissipation bounds.
#include "launch.h"
#include "stage_fused.cuh"

namespace lsp {

bool fused_tile_ok(int ndim, int scheme, const Tile& t, const int* n)
{
    if (ndim != 3 || t.tb < 1 || t.ta < 1 || t.ch < 1 || t.tb * t.ta > 256) return false;
    if (t.minb < 2 || t.minb > 4) return false;
    const long long G = ghost_width(scheme), tb = t.tb, ta = t.ta;
    // slots per thread of the phi tile (2G halo) and of the W1 tile (G halo);
    // the W1 bound is also the one of the scalar body that runs single stages
    if ((ta + 4 * G) * (tb + 4 * G) > kFusedMaxP * ta * tb) return false;
    if ((ta + 2 * G) * (tb + 2 * G) > kFusedMaxW * ta * tb) return false;
    if (sizeof(float) * (size_t)fused_smem_floats((int)G, t.tb, t.ta) > kRunMaxSmem) return false;
    return (n[0] + t.ch - 1) / t.ch <= 65535;
}

template <int SCHEME, int DYN>
static cudaError_t fused_one(const StageArgs<float>& a, const Tile& t, cudaStream_t s)
{
    constexpr int G = ghost_width(SCHEME);
    const int nB = a.n[2], nA = a.n[1], nS = a.n[0];
    dim3 block(t.tb, t.ta, 1);
    dim3 grid((nB + t.tb - 1) / t.tb, (nA + t.ta - 1) / t.ta, (nS + t.ch - 1) / t.ch);
    const size_t smem = sizeof(float) * (size_t)fused_smem_floats(G, t.tb, t.ta);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(stage_fused_rk2_kernel<SCHEME, DYN>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    stage_fused_rk2_kernel<SCHEME, DYN><<<grid, block, smem, s>>>(a, t.ch);
    return cudaGetLastError();
}

template <int SCHEME>
static cudaError_t fused_dyn(int dyn, const StageArgs<float>& a, const Tile& t, cudaStream_t s)
{
    switch (dyn) {
    case NORMAL_SPEED: return fused_one<SCHEME, NORMAL_SPEED>(a, t, s);
    case TRANSLATE: return fused_one<SCHEME, TRANSLATE>(a, t, s);
    case AIR3D: return fused_one<SCHEME, AIR3D>(a, t, s);
    case ROCKETS: return fused_one<SCHEME, ROCKETS>(a, t, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_stage_fused_rk2(int scheme, int dyn, const StageArgs<float>& a, const Tile& t,
                                   cudaStream_t s)
{
    if (a.out == a.phi_s || a.local_alpha || a.varform || a.alpha_from_ctl)
        return cudaErrorInvalidValue;
    switch (scheme) {
    case UPWIND1: return fused_dyn<UPWIND1>(dyn, a, t, s);
    case ENO2: return fused_dyn<ENO2>(dyn, a, t, s);
    case ENO3: return fused_dyn<ENO3>(dyn, a, t, s);
    case WENO5: return fused_dyn<WENO5>(dyn, a, t, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lsp
