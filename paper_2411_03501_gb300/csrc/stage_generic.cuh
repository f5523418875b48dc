// stage_generic.cuh -- the fused Runge-Kutta stage kernel for any
// (dimension, scheme, dynamics, precision), one thread per node.
//
// One launch = one stage of TVD-RK (Sec. V-A):
//   out = c_n phi^n + c_s phi_s + c_l dt L(phi_s),  L = -Hhat (Sec. IV-D)
// with, per node: ghost substitution (Sec. III-B), left/right derivatives
// along every axis (Sec. IV), the Hamiltonian at the average costate and the
// Lax-Friedrichs dissipation sum_k alpha_k (p+_k - p-_k)/2 (global or local
// coefficients), the rate clipped at zero in the variational form, then
// (last stage of a tube step) the minimum with the target (Sec. VI-A).  Stencil reads go
// through the read-only cache; each node is written once.
#pragma once
#include "stencil.cuh"

namespace lsp {

template <int NDIM, int SCHEME, int DYN, typename R>
__global__ void __launch_bounds__(256) stage_generic_kernel(StageArgs<R> a)
{
    constexpr int G = ghost_width(SCHEME);
    R alpha[NDIM];
#pragma unroll
    for (int k = 0; k < NDIM; ++k)
        alpha[k] = a.alpha_from_ctl ? R(__longlong_as_double((long long)a.ctl->alpha_bits[k]))
                                    : a.alpha[k];
    const R dt = a.dt_from_ctl ? R(a.ctl->dt) : a.dt;
    const R cl = a.c_l * dt;

    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < a.npts;
         idx += (long long)gridDim.x * blockDim.x) {
        int c[NDIM];
        {
            long long r = idx;
#pragma unroll
            for (int k = NDIM - 1; k >= 0; --k) {
                c[k] = (int)(r % a.n[k]);
                r /= a.n[k];
            }
        }
        R x[NDIM], pbar[NDIM];
#pragma unroll
        for (int k = 0; k < NDIM; ++k) x[k] = a.lo[k] + R(c[k]) * a.h[k];
        R sth = R(0), cth = R(1);  // heading, for the local coefficients
        if constexpr (DYN == AIR3D || DYN == CAR4D || DYN == ROCKETS)
            if (a.local_alpha) rsincos(x[2], &sth, &cth);
        R diss = R(0);
#pragma unroll
        for (int k = 0; k < NDIM; ++k) {
            R u[2 * G + 1];
            load_window<R, G>(a.phi_s, idx, c[k], a.n[k], a.stride[k], a.periodic[k], u);
            R pm, pp;
            deriv<SCHEME>(u, a.inv_dx[k], pm, pp);
            pbar[k] = R(0.5) * (pp + pm);
            const R ak = a.local_alpha ? local_alpha<DYN>(x, k, a.prm, sth, cth, pm, pp) : alpha[k];
            diss += ak * R(0.5) * (pp - pm);
        }
        const R H = hamiltonian<DYN, NDIM>(x, pbar, a.prm);
        R L = -(H - diss);
        if (a.varform) L = rmin(L, R(0));
        R v = a.c_s * __ldg(a.phi_s + idx) + cl * L;
        if (a.phi_n) v += a.c_n * a.phi_n[idx];
        if (a.tube) v = rmin(v, __ldg(a.target + idx));
        if (!isfinite(v)) atomicOr(&a.ctl->flags, kFlagNonFinite);
        a.out[idx] = v;
    }
}

// Global-LF coefficients for state-only bounds: alpha_k = max over the grid
// nodes of the bound on |dH/dp_k| (FP64).  Block maximum, then one atomicMax
// per block and axis on the bit pattern of the non-negative double.
struct GridGeom {
    int ndim;
    int n[LSP_MAXD];
    double lo[LSP_MAXD];
    double h[LSP_MAXD];
    double prm[LSP_NPARAM];
    long long npts;
};

template <int DYN>
__global__ void __launch_bounds__(256) alpha_state_kernel(GridGeom g, unsigned long long* out)
{
    double m[LSP_MAXD] = {0.0, 0.0, 0.0, 0.0};
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < g.npts;
         idx += (long long)gridDim.x * blockDim.x) {
        double x[LSP_MAXD] = {0.0, 0.0, 0.0, 0.0};
        long long r = idx;
        for (int k = g.ndim - 1; k >= 0; --k) {
            x[k] = g.lo[k] + (double)(r % g.n[k]) * g.h[k];
            r /= g.n[k];
        }
        for (int k = 0; k < g.ndim; ++k) m[k] = fmax(m[k], partial_bound<DYN>(x, k, g.prm));
    }
    __shared__ double sm[LSP_MAXD][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < g.ndim; ++k) {
        double v = m[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) sm[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < (unsigned)g.ndim) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = fmax(v, sm[threadIdx.x][w]);
        atomicMax(out + threadIdx.x, (unsigned long long)__double_as_longlong(v));
    }
}

// Costate range for H = |p|^2/2: alpha_k = max over nodes of max(|p-_k|,
// |p+_k|) of the current stage field, into ctl->alpha_bits (zeroed before).
template <int NDIM, int SCHEME, typename R>
__global__ void __launch_bounds__(256) prange_kernel(StageArgs<R> a)
{
    constexpr int G = ghost_width(SCHEME);
    R m[NDIM];
#pragma unroll
    for (int k = 0; k < NDIM; ++k) m[k] = R(0);
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < a.npts;
         idx += (long long)gridDim.x * blockDim.x) {
        int c[NDIM];
        long long r = idx;
#pragma unroll
        for (int k = NDIM - 1; k >= 0; --k) {
            c[k] = (int)(r % a.n[k]);
            r /= a.n[k];
        }
#pragma unroll
        for (int k = 0; k < NDIM; ++k) {
            R u[2 * G + 1];
            load_window<R, G>(a.phi_s, idx, c[k], a.n[k], a.stride[k], a.periodic[k], u);
            R pm, pp;
            deriv<SCHEME>(u, a.inv_dx[k], pm, pp);
            m[k] = rmax(m[k], rmax(rabs(pm), rabs(pp)));
        }
    }
    __shared__ double sm[NDIM][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NDIM; ++k) {
        double v = (double)m[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) sm[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < NDIM) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = fmax(v, sm[threadIdx.x][w]);
        atomicMax(a.ctl->alpha_bits + threadIdx.x, (unsigned long long)__double_as_longlong(v));
    }
}

}  // namespace lsp
