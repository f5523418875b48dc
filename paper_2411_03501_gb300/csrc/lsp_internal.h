// lsp_internal.h -- structures shared by the host layer and the kernels of
// the level-set library.  Not part of the public ABI (see include/lsp.h).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define LSP_MAXD 4
#define LSP_NPARAM 8

namespace lsp {

enum Scheme { UPWIND1 = 0, ENO2 = 1, ENO3 = 2, WENO5 = 3 };
enum Dyn { NORMAL_SPEED = 0, TRANSLATE = 1, QUADRATIC = 2, AIR3D = 3, CAR4D = 4, ROCKETS = 5,
           DOUBLE_INT = 6 };

__host__ __device__ constexpr int ghost_width(int scheme) { return scheme == UPWIND1 ? 1 : (scheme == ENO2 ? 2 : 3); }

// Streaming multiprocessors of the current device, queried once per device
// index (152 on a GB300), for sizing grids in waves of resident CTAs.
inline int sm_count()
{
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (!cache[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            n = 1;
        cache[dev] = n;
    }
    return cache[dev];
}

// Device control block, the first 256 bytes of every workspace.
struct Ctl {
    unsigned long long alpha_bits[LSP_MAXD];  // p-dependent GLF alpha (bits of
                                              // a non-negative double; atomicMax)
    double dt;                                // step chosen on the device
    double t;                                 // time of the device loop
    unsigned int flags;                       // bit 0: non-finite value produced
    unsigned int pad0;
    unsigned long long reserved[24];
};
static_assert(sizeof(Ctl) <= 256, "control block must fit 256 bytes");
constexpr size_t kCtlBytes = 256;
constexpr unsigned int kFlagNonFinite = 1u;
constexpr unsigned int kFlagTimeout = 2u;

// Arguments of one fused stage launch.  Every launch computes, at every node,
//   out = c_n * phi_n + c_s * phi_s + c_l * dt * L(phi_s)
// (then min with the target if tube), with L the LF rate.
template <typename R>
struct StageArgs {
    const R* phi_s;     // stage input, read with the stencil
    const R* phi_n;     // phi^n, read pointwise (NULL when c_n == 0)
    const R* target;    // read pointwise when tube != 0
    R* out;             // may alias phi_n (pointwise read before write)
    int n[LSP_MAXD];    // nodes per axis
    int stride[LSP_MAXD];
    int periodic[LSP_MAXD];
    R inv_dx[LSP_MAXD];
    R lo[LSP_MAXD];     // coordinates: lo + i * h
    R h[LSP_MAXD];
    R alpha[LSP_MAXD];  // GLF coefficients (state-only dynamics)
    R prm[LSP_NPARAM];  // dynamics parameters
    R dt, c_n, c_s, c_l;
    int tube;
    int npts;
    Ctl* ctl;            // flags; alpha/dt for p-dependent dynamics
    int alpha_from_ctl;  // 1: read alpha from ctl->alpha_bits
    int dt_from_ctl;     // 1: read dt from ctl->dt
    int local_alpha;     // 1: LLF/LLLF coefficients per node instead of alpha[]
    int varform;         // 1: variational form, rate clipped at zero
};

}  // namespace lsp
