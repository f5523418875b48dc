// dispatch.inl -- explicit instantiation of the generic stage kernels for one
// precision LSP_REAL (included by stage_f32.cu / stage_f64.cu).
#include "launch.h"
#include "stage_generic.cuh"

namespace lsp {

static inline int stage_blocks(long long npts)
{
    long long b = (npts + 255) / 256;
    const long long cap = 16LL * sm_count();  // grid-stride beyond 16 blocks per SM
    return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

template <int NDIM, int SCHEME>
static cudaError_t stage_dyn(int dyn, const StageArgs<LSP_REAL>& a, cudaStream_t s)
{
    const int nb = stage_blocks(a.npts);
    switch (dyn) {
    case NORMAL_SPEED: stage_generic_kernel<NDIM, SCHEME, NORMAL_SPEED, LSP_REAL><<<nb, 256, 0, s>>>(a); break;
    case TRANSLATE: stage_generic_kernel<NDIM, SCHEME, TRANSLATE, LSP_REAL><<<nb, 256, 0, s>>>(a); break;
    case QUADRATIC: stage_generic_kernel<NDIM, SCHEME, QUADRATIC, LSP_REAL><<<nb, 256, 0, s>>>(a); break;
    case AIR3D:
        if constexpr (NDIM == 3) { stage_generic_kernel<3, SCHEME, AIR3D, LSP_REAL><<<nb, 256, 0, s>>>(a); break; }
        return cudaErrorInvalidValue;
    case CAR4D:
        if constexpr (NDIM == 4) { stage_generic_kernel<4, SCHEME, CAR4D, LSP_REAL><<<nb, 256, 0, s>>>(a); break; }
        return cudaErrorInvalidValue;
    case ROCKETS:
        if constexpr (NDIM == 3) { stage_generic_kernel<3, SCHEME, ROCKETS, LSP_REAL><<<nb, 256, 0, s>>>(a); break; }
        return cudaErrorInvalidValue;
    case DOUBLE_INT:
        if constexpr (NDIM == 2) { stage_generic_kernel<2, SCHEME, DOUBLE_INT, LSP_REAL><<<nb, 256, 0, s>>>(a); break; }
        return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int NDIM>
static cudaError_t stage_scheme(int scheme, int dyn, const StageArgs<LSP_REAL>& a, cudaStream_t s)
{
    switch (scheme) {
    case UPWIND1: return stage_dyn<NDIM, UPWIND1>(dyn, a, s);
    case ENO2: return stage_dyn<NDIM, ENO2>(dyn, a, s);
    case ENO3: return stage_dyn<NDIM, ENO3>(dyn, a, s);
    case WENO5: return stage_dyn<NDIM, WENO5>(dyn, a, s);
    }
    return cudaErrorInvalidValue;
}

template <>
cudaError_t launch_stage<LSP_REAL>(int ndim, int scheme, int dyn, const StageArgs<LSP_REAL>& a,
                                   cudaStream_t s)
{
    switch (ndim) {
    case 1: return stage_scheme<1>(scheme, dyn, a, s);
    case 2: return stage_scheme<2>(scheme, dyn, a, s);
    case 3: return stage_scheme<3>(scheme, dyn, a, s);
    case 4: return stage_scheme<4>(scheme, dyn, a, s);
    }
    return cudaErrorInvalidValue;
}

template <int NDIM>
static cudaError_t prange_scheme(int scheme, const StageArgs<LSP_REAL>& a, cudaStream_t s)
{
    const int nb = stage_blocks(a.npts);
    switch (scheme) {
    case UPWIND1: prange_kernel<NDIM, UPWIND1, LSP_REAL><<<nb, 256, 0, s>>>(a); break;
    case ENO2: prange_kernel<NDIM, ENO2, LSP_REAL><<<nb, 256, 0, s>>>(a); break;
    case ENO3: prange_kernel<NDIM, ENO3, LSP_REAL><<<nb, 256, 0, s>>>(a); break;
    case WENO5: prange_kernel<NDIM, WENO5, LSP_REAL><<<nb, 256, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <>
cudaError_t launch_prange<LSP_REAL>(int ndim, int scheme, const StageArgs<LSP_REAL>& a,
                                    cudaStream_t s)
{
    switch (ndim) {
    case 1: return prange_scheme<1>(scheme, a, s);
    case 2: return prange_scheme<2>(scheme, a, s);
    case 3: return prange_scheme<3>(scheme, a, s);
    case 4: return prange_scheme<4>(scheme, a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lsp
