// adjoint.inl -- instantiations of the adjoint stage kernels and the loss
// kernels for one precision LSP_REAL (included by adjoint_f32.cu /
// adjoint_f64.cu).
#include "adjoint.cuh"
#include "launch.h"

namespace lsp {

static inline int adj_blocks(long long npts)
{
    long long b = (npts + 255) / 256;
    const long long cap = 16LL * sm_count();
    return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

// Pass A: one wave of resident CTAs (occupancy x SMs, queried once per
// instantiation), so that each thread visits many nodes and the per-thread
// tail -- the promotion of its partial sums and the FP64 warp reduction --
// is paid once per ~30 nodes instead of once per ~3.
// 256 threads per CTA (the prefetch slices of FP32 pass A assume it).
template <int NDIM, int SCHEME, int DYN>
static cudaError_t launch_pass_a(const AdjArgs<LSP_REAL>& a, cudaStream_t s)
{
    constexpr size_t smem = adj_a_smem_bytes<NDIM, LSP_REAL>();
    static const int resident = [] {
        int nsm = sm_count(), per = 1;
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(adj_stage_a<NDIM, SCHEME, DYN, LSP_REAL>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per, adj_stage_a<NDIM, SCHEME, DYN, LSP_REAL>, 256, smem) != cudaSuccess || per < 1)
            per = 1;
        return nsm * per;
    }();
    long long b = (a.npts + 255) / 256;
    const int nb = (int)(b < resident ? (b < 1 ? 1 : b) : resident);
    adj_stage_a<NDIM, SCHEME, DYN, LSP_REAL><<<nb, 256, smem, s>>>(a);
    return cudaGetLastError();
}

template <int NDIM, int SCHEME>
static cudaError_t adj_dyn(int dyn, const AdjArgs<LSP_REAL>& a, cudaStream_t s)
{
    switch (dyn) {
    case NORMAL_SPEED: return launch_pass_a<NDIM, SCHEME, NORMAL_SPEED>(a, s);
    case TRANSLATE: return launch_pass_a<NDIM, SCHEME, TRANSLATE>(a, s);
    case AIR3D:
        if constexpr (NDIM == 3) return launch_pass_a<3, SCHEME, AIR3D>(a, s);
        return cudaErrorInvalidValue;
    case CAR4D:
        if constexpr (NDIM == 4) return launch_pass_a<4, SCHEME, CAR4D>(a, s);
        return cudaErrorInvalidValue;
    case ROCKETS:
        if constexpr (NDIM == 3) return launch_pass_a<3, SCHEME, ROCKETS>(a, s);
        return cudaErrorInvalidValue;
    case DOUBLE_INT:
        if constexpr (NDIM == 2) return launch_pass_a<2, SCHEME, DOUBLE_INT>(a, s);
        return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
    }
}

template <int NDIM>
static cudaError_t adj_scheme(int scheme, int dyn, const AdjArgs<LSP_REAL>& a, bool pass_b,
                              cudaStream_t s)
{
    if (pass_b) {
        adj_stage_b<NDIM, LSP_REAL><<<adj_blocks(a.npts), 256, 0, s>>>(a);
        return cudaGetLastError();
    }
    switch (scheme) {
    case UPWIND1: return adj_dyn<NDIM, UPWIND1>(dyn, a, s);
    case ENO2: return adj_dyn<NDIM, ENO2>(dyn, a, s);
    case ENO3: return adj_dyn<NDIM, ENO3>(dyn, a, s);
    case WENO5: return adj_dyn<NDIM, WENO5>(dyn, a, s);
    }
    return cudaErrorInvalidValue;
}

template <>
cudaError_t launch_adjoint_stage<LSP_REAL>(int ndim, int scheme, int dyn,
                                           const AdjArgs<LSP_REAL>& a, bool pass_b,
                                           cudaStream_t s)
{
    switch (ndim) {
    case 1: return adj_scheme<1>(scheme, dyn, a, pass_b, s);
    case 2: return adj_scheme<2>(scheme, dyn, a, pass_b, s);
    case 3: return adj_scheme<3>(scheme, dyn, a, pass_b, s);
    case 4: return adj_scheme<4>(scheme, dyn, a, pass_b, s);
    }
    return cudaErrorInvalidValue;
}

template <int NDIM>
static void loss_q(const LossArgs<LSP_REAL>& L, double* value, LSP_REAL* grad, cudaStream_t s)
{
    InterpArgs<LSP_REAL, NDIM> a;
    a.phi = L.phi;
    a.queries = L.queries;
    a.nq = L.nq;
    for (int k = 0; k < LSP_MAXD; ++k) {
        a.n[k] = L.n[k];
        a.stride[k] = L.stride[k];
        a.periodic[k] = L.periodic[k];
        a.lo[k] = L.lo[k];
        a.h[k] = L.h[k];
    }
    loss_query_kernel<LSP_REAL, NDIM><<<(L.nq + 127) / 128, 128, 0, s>>>(a, value, grad);
}

template <>
cudaError_t launch_loss<LSP_REAL>(const LossArgs<LSP_REAL>& L, double* value, LSP_REAL* grad,
                                  cudaStream_t s)
{
    loss_volume_kernel<LSP_REAL><<<adj_blocks(L.npts), 256, 0, s>>>(L.phi, L.npts, L.inv_eps,
                                                                      L.dV, value, grad);
    cudaError_t e = cudaGetLastError();
    if (e || L.nq <= 0) return e;
    switch (L.ndim) {
    case 1: loss_q<1>(L, value, grad, s); break;
    case 2: loss_q<2>(L, value, grad, s); break;
    case 3: loss_q<3>(L, value, grad, s); break;
    case 4: loss_q<4>(L, value, grad, s); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace lsp
