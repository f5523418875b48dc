// noalloc.cu -- lsp_hj_solve_noalloc: the solve of lsp_hj_solve with its
// scratch (RK stage fields and control block) in a fixed, library-owned
// device array instead of a caller-provided workspace, so that callers who
// may not allocate device memory can still run a solve.  No cudaMalloc,
// cudaFree or allocating library routine is called here.
#include <cstdio>
#include <mutex>

#include "../../include/lsp.h"
#include "lsp_internal.h"

namespace lsp {
void set_last_error(const char* msg);
}

namespace {

// 32 MiB, held on every GPU that loads the library until the process exits.
constexpr size_t kScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

lsp_status noalloc_fail(lsp_status s, const char* msg)
{
    lsp::set_last_error(msg);
    return s;
}

}  // namespace

extern "C" lsp_status lsp_hj_solve_noalloc(lsp_grid* grid, const lsp_solve_opts* opts, void* phi,
                                           const void* target, double t0, double t_final,
                                           lsp_solve_stats* stats, void* stream)
{
    if (!opts) return noalloc_fail(LSP_EINVAL, "opts is NULL");
    if (opts->use_graph)
        return noalloc_fail(LSP_EINVAL,
                            "use_graph must be 0 in lsp_hj_solve_noalloc (building a graph allocates)");
    size_t need = 0;
    lsp_status s = lsp_workspace_size(grid, opts, &need);
    if (s != LSP_OK) return s;
    if (need > kScratchBytes) {
        char msg[256];
        std::snprintf(msg, sizeof(msg),
                      "lsp_hj_solve_noalloc: this grid needs %zu bytes of scratch but the built-in "
                      "array holds %zu; use lsp_hj_solve with a workspace",
                      need, kScratchBytes);
        return noalloc_fail(LSP_ENOMEM, msg);
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(LSP_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(LSP_EINVAL, "device index out of range");
    void* ptr = nullptr;
    {
        // Set-up, once per device with that device current: the device
        // address of the static array (the host-side symbol is not one).
        // Kept per device index for the life of the process; after a
        // cudaDeviceReset the module would load at another address, which
        // is why resetting the device after the first call is unsupported.
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                char msg[256];
                std::snprintf(msg, sizeof(msg), "cudaGetSymbolAddress(scratch): %s",
                              cudaGetErrorString(e));
                return noalloc_fail(LSP_ECUDA, msg);
            }
            g_scratch_ptr[dev] = p;
        }
        ptr = g_scratch_ptr[dev];
    }
    // The solve resets the control block's flags on entry and writes every
    // stage field before reading it, so the previous call's contents of the
    // array are never used.
    return lsp_hj_solve(grid, opts, phi, target, t0, t_final, ptr, kScratchBytes, stats, stream);
}
