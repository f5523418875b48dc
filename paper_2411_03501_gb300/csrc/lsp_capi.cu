// lsp_capi.cu -- the C ABI of include/lsp.h: argument checking, workspace
// layout, the FP64 time loop and the enqueueing of the stage kernels.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <type_traits>
#include <vector>

#include "../../include/lsp.h"
#include "adjoint.cuh"
#include "batched.h"
#include "launch.h"
#include "stage_generic.cuh"
#include "stage_tiled.cuh"

struct lsp_grid {
    int ndim = 0;
    int n[LSP_MAXD] = {0, 0, 0, 0};
    double lo[LSP_MAXD] = {0, 0, 0, 0};
    double hi[LSP_MAXD] = {0, 0, 0, 0};
    double dx[LSP_MAXD] = {0, 0, 0, 0};
    int periodic[LSP_MAXD] = {0, 0, 0, 0};
    long long npts = 0;
    int dyn = -1;
    double prm[LSP_NPARAM] = {0, 0, 0, 0, 0, 0, 0, 0};
    double alpha[LSP_MAXD] = {0, 0, 0, 0};
    bool alpha_state = false;  // alpha known on the host (state-only bound)

    // tile of the tiled 3-D/4-D FP32 stage kernel: mode 0 = default shape,
    // 1 = set explicitly (or by the autotuner), -1 = use the generic kernel
    int tile_mode = 0;
    lsp::Tile tile{0, 0, 0, 3, 0};

    // cached CUDA graph of the last lsp_hj_solve with use_graph
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t capture_stream = nullptr;
    struct Key {
        void* phi;
        const void* target;
        void* ws;
        double t0, t1;
        lsp_solve_opts opts;
    } gkey{};
    lsp_solve_stats gstats{};
};

namespace {

thread_local char g_err[512] = "";

lsp_status fail(lsp_status s, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

lsp_status cuda_fail(cudaError_t e, const char* where)
{
    return fail(LSP_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

int nfields(int rk) { return rk == 3 ? 2 : 1; }

size_t elem_size(int dtype) { return dtype == LSP_F64 ? 8 : 4; }

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

lsp_status check_opts(const lsp_grid* g, const lsp_solve_opts* o)
{
    if (!g) return fail(LSP_EINVAL, "grid is NULL");
    if (!o) return fail(LSP_EINVAL, "opts is NULL");
    if (g->dyn < 0) return fail(LSP_EINVAL, "no dynamics set on the grid (lsp_set_dynamics)");
    if (o->rk_order < 1 || o->rk_order > 3) return fail(LSP_EINVAL, "rk_order must be 1, 2 or 3");
    if (o->scheme < LSP_UPWIND1 || o->scheme > LSP_WENO5) return fail(LSP_EINVAL, "bad scheme");
    if (o->dtype != LSP_F32 && o->dtype != LSP_F64) return fail(LSP_EINVAL, "bad dtype");
    if (!(o->cfl > 0.0 && o->cfl <= 1.0)) return fail(LSP_EINVAL, "cfl must be in (0, 1]");
    for (int d = 2; d <= 4; ++d)
        if (((o->batch_tiles >> (2 * (d - 2))) & 3) == 3)
            return fail(LSP_EINVAL, "batch_tiles: shape 3 is not defined (dimension %d)", d);
    if (o->batch_tiles >> 6) return fail(LSP_EINVAL, "batch_tiles: bits above 5 must be zero");
    if (o->diss < LSP_DISS_GLF || o->diss > LSP_DISS_LLLF) return fail(LSP_EINVAL, "bad diss");
    if (o->varform != 0 && o->varform != 1) return fail(LSP_EINVAL, "varform must be 0 or 1");
    if (o->batch_chunk < 0) return fail(LSP_EINVAL, "batch_chunk must be >= 0");
    if (o->batch_persistent != 0 && o->batch_persistent != 1)
        return fail(LSP_EINVAL, "batch_persistent must be 0 or 1");
    if (o->batch_wait_ms < 0) return fail(LSP_EINVAL, "batch_wait_ms must be >= 0");
    const int G = lsp::ghost_width(o->scheme);
    for (int k = 0; k < g->ndim; ++k)
        if (g->n[k] < 2 * G + 1)
            return fail(LSP_EINVAL, "axis %d has %d nodes; the scheme needs at least %d", k,
                        g->n[k], 2 * G + 1);
    if (!lsp::stage_supported(g->ndim, o->scheme, g->dyn))
        return fail(LSP_EUNSUPPORTED, "no kernel for ndim=%d scheme=%d dyn=%d", g->ndim,
                    o->scheme, g->dyn);
    return LSP_OK;
}

size_t ws_bytes(const lsp_grid* g, const lsp_solve_opts* o)
{
    return lsp::kCtlBytes + nfields(o->rk_order) * round256((size_t)g->npts * elem_size(o->dtype));
}

lsp_status check_ws(const lsp_grid* g, const lsp_solve_opts* o, const void* ws, size_t bytes)
{
    if (!ws) return fail(LSP_EINVAL, "workspace is NULL");
    if (!aligned16(ws)) return fail(LSP_EINVAL, "workspace must be 16-byte aligned");
    const size_t need = ws_bytes(g, o);
    if (bytes < need)
        return fail(LSP_ENOMEM, "workspace has %zu bytes, needs %zu", bytes, need);
    return LSP_OK;
}

double cfl_dt_host(const lsp_grid* g, double cfl, double t, double t_final)
{
    double s = 0.0;
    for (int k = 0; k < g->ndim; ++k) s += g->alpha[k] / g->dx[k];
    double dt = (s > 0.0) ? cfl / s : (t_final - t);
    if (t_final - t < dt) dt = t_final - t;
    return dt;
}

// Default tile: 32 x 8 threads over the two fastest axes, the march along
// the third split into chunks so that at least ~2 waves of 2 CTAs per SM
// are launched.
// The tile used without lsp_set_tile / lsp_autotune: WENO5 runs the paired
// shared-face kernel on 16 x 16 tiles, chunked so that the launch has about
// three waves of 3 CTAs per SM, with an even chunk length (the pairs of
// planes); the other schemes the scalar kernel on 32 x 8 tiles, about two
// waves of 2 CTAs per SM.
lsp::Tile default_tile(const lsp_grid* g, int scheme)
{
    const int d = g->ndim;
    const bool paired = scheme == LSP_WENO5;
    lsp::Tile t;
    t.tb = paired ? 16 : 32;
    t.ta = paired ? 16 : 8;
    t.minb = 3;
    t.pair = paired ? 2 : 0;
    const long long nplane = (long long)((g->n[d - 1] + t.tb - 1) / t.tb) *
                             ((g->n[d - 2] + t.ta - 1) / t.ta) * (d == 4 ? g->n[0] : 1);
    const long long want = (paired ? 3LL * 3 : 2LL * 2) * lsp::sm_count();
    long long nch = (want + nplane - 1) / nplane;
    const int nS = g->n[d - 3];
    if (nch > nS / 4) nch = nS / 4;
    if (nch < 1) nch = 1;
    t.ch = (int)((nS + nch - 1) / nch);
    if (paired && (t.ch & 1)) t.ch += 1;
    return t;
}

// The tile the FP32 3-D/4-D stages use, or ch = 0 for the generic kernel.
lsp::Tile tile_in_effect(const lsp_grid* g, const lsp_solve_opts* o)
{
    lsp::Tile none{0, 0, 0, 0, 0};
    if (o->dtype != LSP_F32 || (g->ndim != 3 && g->ndim != 4) || g->tile_mode < 0) return none;
    lsp::Tile t = g->tile_mode == 1 ? g->tile : default_tile(g, o->scheme);
    return lsp::tile_valid(g->ndim, o->scheme, t, g->n) ? t : none;
}

template <typename R>
lsp::StageArgs<R> base_args(const lsp_grid* g, lsp::Ctl* ctl)
{
    lsp::StageArgs<R> a;
    std::memset(&a, 0, sizeof(a));
    long long s = 1;
    for (int k = g->ndim - 1; k >= 0; --k) {
        a.n[k] = g->n[k];
        a.stride[k] = (int)s;
        s *= g->n[k];
        a.periodic[k] = g->periodic[k];
        a.inv_dx[k] = R(1.0 / g->dx[k]);
        a.lo[k] = R(g->lo[k]);
        a.h[k] = R(g->dx[k]);
        a.alpha[k] = R(g->alpha[k]);
    }
    for (int i = 0; i < LSP_NPARAM; ++i) a.prm[i] = R(g->prm[i]);
    a.npts = (int)g->npts;
    a.ctl = ctl;
    a.alpha_from_ctl = g->alpha_state ? 0 : 1;
    return a;
}

// One stage: out = c_n phi_n + c_s phi_s + c_l dt L(phi_s) [min target].
template <typename R>
lsp_status enqueue_stage(const lsp_grid* g, const lsp_solve_opts* o, lsp::Ctl* ctl,
                         const R* phi_s, const R* phi_n, const R* target, R* out, double dt,
                         double c_n, double c_s, double c_l, bool tube, cudaStream_t st)
{
    lsp::StageArgs<R> a = base_args<R>(g, ctl);
    a.phi_s = phi_s;
    a.phi_n = phi_n;
    a.target = target;
    a.out = out;
    a.dt = R(dt);
    a.c_n = R(c_n);
    a.c_s = R(c_s);
    a.c_l = R(c_l);
    a.tube = tube ? 1 : 0;
    a.local_alpha = o->diss != LSP_DISS_GLF;
    a.varform = o->varform;
    cudaError_t e;
    if (!g->alpha_state) {  // alpha from the costate range of phi_s
        e = cudaMemsetAsync(ctl->alpha_bits, 0, sizeof(ctl->alpha_bits), st);
        if (e != cudaSuccess) return cuda_fail(e, "memset alpha");
        e = lsp::launch_prange<R>(g->ndim, o->scheme, a, st);
        if (e != cudaSuccess) return cuda_fail(e, "costate range kernel");
    }
    if constexpr (std::is_same<R, float>::value) {
        const lsp::Tile t = tile_in_effect(g, o);
        if (t.ch > 0) {
            e = lsp::launch_stage_tiled(g->ndim, o->scheme, g->dyn, a, t, st);
            if (e != cudaSuccess) return cuda_fail(e, "tiled stage kernel");
            return LSP_OK;
        }
    }
    e = lsp::launch_stage<R>(g->ndim, o->scheme, g->dyn, a, st);
    if (e != cudaSuccess) return cuda_fail(e, "stage kernel");
    return LSP_OK;
}

// One TVD-RK step of size dt, phi in place (Sec. V-A), tube in the last stage.
template <typename R>
lsp_status enqueue_step(const lsp_grid* g, const lsp_solve_opts* o, R* phi, const R* target,
                        double dt, void* ws, cudaStream_t st, R* w1_at = nullptr,
                        R* w2_at = nullptr)
{
    // stage fields: the workspace's, or the caller's (w1_at, w2_at: the
    // adjoint keeps a segment's stage inputs)
    lsp::Ctl* ctl = (lsp::Ctl*)ws;
    R* w1 = w1_at ? w1_at : (R*)((char*)ws + lsp::kCtlBytes);
    R* w2 = w2_at ? w2_at : (R*)((char*)ws + lsp::kCtlBytes + round256((size_t)g->npts * sizeof(R)));
    const bool tube = o->tube != 0;
    lsp_status s;
    switch (o->rk_order) {
    case 1:
        s = enqueue_stage<R>(g, o, ctl, phi, nullptr, target, w1, dt, 0.0, 1.0, 1.0, tube, st);
        if (s) return s;
        if (cudaError_t e = cudaMemcpyAsync(phi, w1, (size_t)g->npts * sizeof(R),
                                            cudaMemcpyDeviceToDevice, st))
            return cuda_fail(e, "copy back");
        return LSP_OK;
    case 2:
        s = enqueue_stage<R>(g, o, ctl, phi, nullptr, nullptr, w1, dt, 0.0, 1.0, 1.0, false, st);
        if (s) return s;
        return enqueue_stage<R>(g, o, ctl, w1, phi, target, phi, dt, 0.5, 0.5, 0.5, tube, st);
    default:
        s = enqueue_stage<R>(g, o, ctl, phi, nullptr, nullptr, w1, dt, 0.0, 1.0, 1.0, false, st);
        if (s) return s;
        s = enqueue_stage<R>(g, o, ctl, w1, phi, nullptr, w2, dt, 0.75, 0.25, 0.25, false, st);
        if (s) return s;
        return enqueue_stage<R>(g, o, ctl, w2, phi, target, phi, dt, 1.0 / 3.0, 2.0 / 3.0,
                                2.0 / 3.0, tube, st);
    }
}

// Does an RK2 step with these options run as one temporally blocked launch
// (tile pair 5; 3-D FP32, GLF with state-only bounds)?
bool fused_rk2(const lsp_grid* g, const lsp_solve_opts* o)
{
    if (o->rk_order != 2 || o->dtype != LSP_F32 || g->ndim != 3 || !g->alpha_state) return false;
    if (o->diss != LSP_DISS_GLF || o->varform) return false;
    const lsp::Tile t = tile_in_effect(g, o);
    return t.ch > 0 && t.pair == 5;
}

// One RK2 step from phi into out (distinct fields) in one launch.
lsp_status enqueue_fused_rk2(const lsp_grid* g, const lsp_solve_opts* o, const float* phi,
                             float* out, const float* target, double dt, void* ws, cudaStream_t st)
{
    lsp::StageArgs<float> a = base_args<float>(g, (lsp::Ctl*)ws);
    a.phi_s = phi;
    a.out = out;
    a.target = target;
    a.dt = float(dt);
    a.c_n = 0.5f;
    a.c_s = 0.5f;
    a.c_l = 0.5f;
    a.tube = o->tube ? 1 : 0;
    cudaError_t e = lsp::launch_stage_fused_rk2(o->scheme, g->dyn, a, tile_in_effect(g, o), st);
    if (e != cudaSuccess) return cuda_fail(e, "fused RK2 kernel");
    return LSP_OK;
}

// One step of phi in place.  allow_fused: a fused-RK2 tile runs the step
// as one launch into the workspace's stage field, copied back to phi (the
// solve alternates the two fields instead of copying).
lsp_status step_any(const lsp_grid* g, const lsp_solve_opts* o, void* phi, const void* target,
                    double dt, void* ws, cudaStream_t st, bool allow_fused = false)
{
    if (allow_fused && fused_rk2(g, o)) {
        float* w1 = (float*)((char*)ws + lsp::kCtlBytes);
        lsp_status s = enqueue_fused_rk2(g, o, (const float*)phi, w1, (const float*)target, dt, ws, st);
        if (s) return s;
        if (cudaError_t e = cudaMemcpyAsync(phi, w1, (size_t)g->npts * sizeof(float),
                                            cudaMemcpyDeviceToDevice, st))
            return cuda_fail(e, "copy back");
        return LSP_OK;
    }
    if (o->dtype == LSP_F64)
        return enqueue_step<double>(g, o, (double*)phi, (const double*)target, dt, ws, st);
    return enqueue_step<float>(g, o, (float*)phi, (const float*)target, dt, ws, st);
}

// dt for p-dependent alpha: reduce the costate range of phi on the device and
// read it back (the call waits for the stream).
lsp_status device_alpha(const lsp_grid* g, const lsp_solve_opts* o, const void* phi, void* ws,
                        cudaStream_t st, double* alpha)
{
    lsp::Ctl* ctl = (lsp::Ctl*)ws;
    cudaError_t e = cudaMemsetAsync(ctl->alpha_bits, 0, sizeof(ctl->alpha_bits), st);
    if (e) return cuda_fail(e, "memset alpha");
    if (o->dtype == LSP_F64) {
        lsp::StageArgs<double> a = base_args<double>(g, ctl);
        a.phi_s = (const double*)phi;
        e = lsp::launch_prange<double>(g->ndim, o->scheme, a, st);
    } else {
        lsp::StageArgs<float> a = base_args<float>(g, ctl);
        a.phi_s = (const float*)phi;
        e = lsp::launch_prange<float>(g->ndim, o->scheme, a, st);
    }
    if (e) return cuda_fail(e, "costate range kernel");
    unsigned long long bits[LSP_MAXD];
    e = cudaMemcpyAsync(bits, ctl->alpha_bits, sizeof(bits), cudaMemcpyDeviceToHost, st);
    if (e) return cuda_fail(e, "read alpha");
    e = cudaStreamSynchronize(st);
    if (e) return cuda_fail(e, "synchronize");
    for (int k = 0; k < g->ndim; ++k) {
        double v;
        std::memcpy(&v, &bits[k], sizeof(v));
        alpha[k] = v;
    }
    return LSP_OK;
}

lsp_status reset_flags(void* ws, cudaStream_t st)
{
    lsp::Ctl* ctl = (lsp::Ctl*)ws;
    cudaError_t e = cudaMemsetAsync(&ctl->flags, 0, sizeof(ctl->flags), st);
    return e ? cuda_fail(e, "reset flags") : LSP_OK;
}

lsp_status read_flags(const void* ws, cudaStream_t st)
{
    const lsp::Ctl* ctl = (const lsp::Ctl*)ws;
    unsigned int f = 0;
    cudaError_t e = cudaMemcpyAsync(&f, &ctl->flags, sizeof(f), cudaMemcpyDeviceToHost, st);
    if (e) return cuda_fail(e, "read flags");
    e = cudaStreamSynchronize(st);
    if (e) return cuda_fail(e, "synchronize");
    if (f & lsp::kFlagTimeout)
        return fail(LSP_ETIMEOUT, "a device-side wait ran out; the results are incomplete");
    if (f & lsp::kFlagNonFinite) return fail(LSP_ENONFINITE, "a non-finite value was produced");
    return LSP_OK;
}

lsp_status check_field(const void* p, const char* name)
{
    if (!p) return fail(LSP_EINVAL, "%s is NULL", name);
    if (!aligned16(p)) return fail(LSP_EINVAL, "%s must be 16-byte aligned", name);
    return LSP_OK;
}

}  // namespace

namespace lsp {
// Record the thread's last-error text from another translation unit.
void set_last_error(const char* msg)
{
    std::snprintf(g_err, sizeof(g_err), "%s", msg);
}
}  // namespace lsp

extern "C" {

int lsp_version(void) { return 100; }

const char* lsp_status_string(lsp_status s)
{
    switch (s) {
    case LSP_OK: return "ok";
    case LSP_EINVAL: return "invalid argument";
    case LSP_ENOMEM: return "workspace too small";
    case LSP_ECUDA: return "CUDA error";
    case LSP_EUNSUPPORTED: return "unsupported combination";
    case LSP_ENONFINITE: return "non-finite value produced";
    case LSP_ETIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

const char* lsp_last_error(void) { return g_err; }

lsp_status lsp_grid_create(int ndim, const double* gmin, const double* gmax, const int64_t* n,
                           const int* bc, lsp_grid** out)
{
    if (!out) return fail(LSP_EINVAL, "out is NULL");
    *out = nullptr;
    if (ndim < 1 || ndim > LSP_MAXD) return fail(LSP_EINVAL, "ndim must be 1..4");
    if (!gmin || !gmax || !n || !bc) return fail(LSP_EINVAL, "NULL argument");
    long long npts = 1;
    for (int k = 0; k < ndim; ++k) {
        if (!std::isfinite(gmin[k]) || !std::isfinite(gmax[k]) || !(gmax[k] > gmin[k]))
            return fail(LSP_EINVAL, "axis %d: bounds must be finite with gmax > gmin", k);
        if (n[k] < 7 || n[k] > (1 << 30)) return fail(LSP_EINVAL, "axis %d: need 7 <= n", k);
        if (bc[k] != LSP_BC_EXTRAPOLATE && bc[k] != LSP_BC_PERIODIC)
            return fail(LSP_EINVAL, "axis %d: bad boundary condition", k);
        npts *= n[k];
        if (npts >= (1LL << 31)) return fail(LSP_EINVAL, "grid exceeds 2^31 - 1 nodes");
    }
    lsp_grid* g = new (std::nothrow) lsp_grid();
    if (!g) return fail(LSP_EINVAL, "out of host memory");
    g->ndim = ndim;
    g->npts = npts;
    for (int k = 0; k < ndim; ++k) {
        g->n[k] = (int)n[k];
        g->lo[k] = gmin[k];
        g->hi[k] = gmax[k];
        g->periodic[k] = bc[k] == LSP_BC_PERIODIC;
        g->dx[k] = g->periodic[k] ? (gmax[k] - gmin[k]) / (double)n[k]
                                  : (gmax[k] - gmin[k]) / (double)(n[k] - 1);
    }
    *out = g;
    return LSP_OK;
}

void lsp_grid_destroy(lsp_grid* g)
{
    if (!g) return;
    if (g->gexec) cudaGraphExecDestroy(g->gexec);
    if (g->capture_stream) cudaStreamDestroy(g->capture_stream);
    delete g;
}

lsp_status lsp_set_dynamics(lsp_grid* g, int dyn, const double* params, int nparams)
{
    if (!g) return fail(LSP_EINVAL, "grid is NULL");
    int need;
    switch (dyn) {
    case LSP_DYN_NORMAL_SPEED: need = 1; break;
    case LSP_DYN_TRANSLATE: need = g->ndim; break;
    case LSP_DYN_QUADRATIC: need = 0; break;
    case LSP_DYN_AIR3D:
        if (g->ndim != 3) return fail(LSP_EINVAL, "AIR3D needs a 3-D grid");
        need = 4;
        break;
    case LSP_DYN_CAR4D:
        if (g->ndim != 4) return fail(LSP_EINVAL, "CAR4D needs a 4-D grid");
        need = 2;
        break;
    case LSP_DYN_ROCKETS:
        if (g->ndim != 3) return fail(LSP_EINVAL, "ROCKETS needs a 3-D grid");
        need = 4;
        break;
    case LSP_DYN_DOUBLE_INTEGRATOR:
        if (g->ndim != 2) return fail(LSP_EINVAL, "DOUBLE_INTEGRATOR needs a 2-D grid");
        need = 1;
        break;
    default: return fail(LSP_EINVAL, "unknown dynamics %d", dyn);
    }
    if (nparams != need) return fail(LSP_EINVAL, "dynamics %d takes %d parameters, got %d", dyn, need, nparams);
    if (need && !params) return fail(LSP_EINVAL, "params is NULL");
    for (int i = 0; i < need; ++i)
        if (!std::isfinite(params[i])) return fail(LSP_EINVAL, "parameter %d is not finite", i);
    if (g->gexec) {
        cudaGraphExecDestroy(g->gexec);
        g->gexec = nullptr;
    }
    for (int i = 0; i < LSP_NPARAM; ++i) g->prm[i] = i < need ? params[i] : 0.0;
    g->dyn = dyn;
    g->alpha_state = false;
    for (int k = 0; k < LSP_MAXD; ++k) g->alpha[k] = 0.0;
    if (dyn == LSP_DYN_QUADRATIC) return LSP_OK;

    // alpha_k = max over the grid nodes of the bound on |dH/dp_k|
    lsp::GridGeom geo;
    std::memset(&geo, 0, sizeof(geo));
    geo.ndim = g->ndim;
    geo.npts = g->npts;
    for (int k = 0; k < g->ndim; ++k) {
        geo.n[k] = g->n[k];
        geo.lo[k] = g->lo[k];
        geo.h[k] = g->dx[k];
    }
    for (int i = 0; i < LSP_NPARAM; ++i) geo.prm[i] = g->prm[i];
    unsigned long long* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(unsigned long long) * LSP_MAXD);
    if (e) return cuda_fail(e, "cudaMalloc (alpha)");
    e = cudaMemset(d, 0, sizeof(unsigned long long) * LSP_MAXD);
    if (!e) e = lsp::launch_alpha_state(dyn, geo, d, 0);
    unsigned long long bits[LSP_MAXD] = {0, 0, 0, 0};
    if (!e) e = cudaMemcpy(bits, d, sizeof(bits), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e) {
        g->dyn = -1;
        return cuda_fail(e, "alpha reduction");
    }
    for (int k = 0; k < g->ndim; ++k) std::memcpy(&g->alpha[k], &bits[k], sizeof(double));
    g->alpha_state = true;
    return LSP_OK;
}

lsp_status lsp_get_alpha(const lsp_grid* g, double* alpha)
{
    if (!g || !alpha) return fail(LSP_EINVAL, "NULL argument");
    if (g->dyn < 0) return fail(LSP_EINVAL, "no dynamics set");
    if (!g->alpha_state) return fail(LSP_EUNSUPPORTED, "alpha depends on phi for this dynamics");
    for (int k = 0; k < g->ndim; ++k) alpha[k] = g->alpha[k];
    return LSP_OK;
}

lsp_status lsp_workspace_size(const lsp_grid* g, const lsp_solve_opts* o, size_t* bytes)
{
    if (!bytes) return fail(LSP_EINVAL, "bytes is NULL");
    lsp_status s = check_opts(g, o);
    if (s) return s;
    *bytes = ws_bytes(g, o);
    return LSP_OK;
}

lsp_status lsp_cfl_dt(const lsp_grid* g, const lsp_solve_opts* o, double t, double t_final,
                      double* dt)
{
    if (!dt) return fail(LSP_EINVAL, "dt is NULL");
    lsp_status s = check_opts(g, o);
    if (s) return s;
    if (!g->alpha_state) return fail(LSP_EUNSUPPORTED, "the step depends on phi for this dynamics");
    *dt = cfl_dt_host(g, o->cfl, t, t_final);
    return LSP_OK;
}

lsp_status lsp_hj_rate(lsp_grid* g, const lsp_solve_opts* o, const void* phi, void* rate,
                       void* ws, size_t ws_size, void* stream)
{
    lsp_status s = check_opts(g, o);
    if (!s) s = check_field(phi, "phi");
    if (!s) s = check_field(rate, "rate");
    if (!s) s = check_ws(g, o, ws, ws_size);
    if (s) return s;
    if (phi == rate) return fail(LSP_EINVAL, "rate must not alias phi");
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = reset_flags(ws, st))) return s;
    lsp::Ctl* ctl = (lsp::Ctl*)ws;
    if (o->dtype == LSP_F64)
        s = enqueue_stage<double>(g, o, ctl, (const double*)phi, nullptr, nullptr, (double*)rate,
                                  1.0, 0.0, 0.0, 1.0, false, st);
    else
        s = enqueue_stage<float>(g, o, ctl, (const float*)phi, nullptr, nullptr, (float*)rate,
                                 1.0, 0.0, 0.0, 1.0, false, st);
    if (s) return s;
    if (o->check_finite) return read_flags(ws, st);
    return LSP_OK;
}

lsp_status lsp_hj_step(lsp_grid* g, const lsp_solve_opts* o, void* phi, const void* target,
                       double t, double* dt_io, void* ws, size_t ws_size, void* stream)
{
    lsp_status s = check_opts(g, o);
    if (!s) s = check_field(phi, "phi");
    if (!s && o->tube) s = check_field(target, "target");
    if (!s) s = check_ws(g, o, ws, ws_size);
    if (s) return s;
    if (!dt_io) return fail(LSP_EINVAL, "dt_io is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = reset_flags(ws, st))) return s;
    double dt = *dt_io;
    if (!g->alpha_state) {
        if (dt > 0.0) return fail(LSP_EINVAL, "QUADRATIC dynamics choose their own step: pass *dt_io <= 0");
        double a[LSP_MAXD];
        if ((s = device_alpha(g, o, phi, ws, st, a))) return s;
        double sum = 0.0;
        for (int k = 0; k < g->ndim; ++k) sum += a[k] / g->dx[k];
        if (!(sum > 0.0)) return fail(LSP_EINVAL, "zero costate range: no CFL step");
        dt = o->cfl / sum;
    } else if (!(dt > 0.0)) {
        dt = cfl_dt_host(g, o->cfl, t, INFINITY);
    }
    if (!std::isfinite(dt) || !(dt > 0.0)) return fail(LSP_EINVAL, "step size must be finite and > 0");
    *dt_io = dt;
    if ((s = step_any(g, o, phi, target, dt, ws, st, true))) return s;
    if (o->check_finite) return read_flags(ws, st);
    return LSP_OK;
}

lsp_status lsp_hj_solve(lsp_grid* g, const lsp_solve_opts* o, void* phi, const void* target,
                        double t0, double t_final, void* ws, size_t ws_size, lsp_solve_stats* stats,
                        void* stream)
{
    lsp_status s = check_opts(g, o);
    if (!s) s = check_field(phi, "phi");
    if (!s && o->tube) s = check_field(target, "target");
    if (!s) s = check_ws(g, o, ws, ws_size);
    if (s) return s;
    if (!std::isfinite(t0) || !std::isfinite(t_final)) return fail(LSP_EINVAL, "times must be finite");
    cudaStream_t st = (cudaStream_t)stream;
    lsp_solve_stats sts{0, 0, INFINITY, 0.0, t0};
    const double t_stop = t_final - 1e-12 * std::fabs(t_final);

    if (!g->alpha_state) {  // alpha from phi: one device round trip per step
        if ((s = reset_flags(ws, st))) return s;
        double t = t0;
        while (t < t_stop) {
            double a[LSP_MAXD];
            if ((s = device_alpha(g, o, phi, ws, st, a))) return s;
            double sum = 0.0;
            for (int k = 0; k < g->ndim; ++k) sum += a[k] / g->dx[k];
            double dt = sum > 0.0 ? o->cfl / sum : t_final - t;
            if (t_final - t < dt) dt = t_final - t;
            if ((s = step_any(g, o, phi, target, dt, ws, st))) return s;
            t += dt;
            sts.steps++;
            sts.dt_min = std::fmin(sts.dt_min, dt);
            sts.dt_max = std::fmax(sts.dt_max, dt);
        }
        sts.t_end = t;
        sts.stages = sts.steps * o->rk_order;
        if (stats) *stats = sts;
        if (o->check_finite) return read_flags(ws, st);
        return LSP_OK;
    }

    const bool graph = o->use_graph != 0;
    if (graph && g->gexec) {
        const lsp_grid::Key& k = g->gkey;
        if (k.phi == phi && k.target == target && k.ws == ws && k.t0 == t0 && k.t1 == t_final &&
            std::memcmp(&k.opts, o, sizeof(*o)) == 0) {
            cudaError_t e = cudaGraphLaunch(g->gexec, st);
            if (e) return cuda_fail(e, "graph launch");
            if (stats) *stats = g->gstats;
            if (o->check_finite) return read_flags(ws, st);
            return LSP_OK;
        }
        cudaGraphExecDestroy(g->gexec);
        g->gexec = nullptr;
    }
    cudaStream_t es = st;
    if (graph) {
        if (!g->capture_stream) {
            cudaError_t e = cudaStreamCreateWithFlags(&g->capture_stream, cudaStreamNonBlocking);
            if (e) return cuda_fail(e, "create capture stream");
        }
        es = g->capture_stream;
        cudaError_t e = cudaStreamBeginCapture(es, cudaStreamCaptureModeThreadLocal);
        if (e) return cuda_fail(e, "begin capture");
    }
    s = reset_flags(ws, es);
    double t = t0;
    // fused RK2: each step reads one field and writes the other (phi and the
    // workspace's stage field in turn), the result copied to phi at the end
    const bool fused = fused_rk2(g, o);
    float* cur = (float*)phi;
    float* alt = (float*)((char*)ws + lsp::kCtlBytes);
    while (!s && t < t_stop) {
        const double dt = cfl_dt_host(g, o->cfl, t, t_final);
        if (!(dt > 0.0)) {
            s = fail(LSP_EINVAL, "non-positive CFL step");
            break;
        }
        if (fused) {
            s = enqueue_fused_rk2(g, o, cur, alt, (const float*)target, dt, ws, es);
            std::swap(cur, alt);
        } else {
            s = step_any(g, o, phi, target, dt, ws, es);
        }
        t += dt;
        sts.steps++;
        sts.dt_min = std::fmin(sts.dt_min, dt);
        sts.dt_max = std::fmax(sts.dt_max, dt);
    }
    if (!s && fused && cur != (float*)phi) {
        if (cudaError_t e = cudaMemcpyAsync(phi, cur, (size_t)g->npts * sizeof(float),
                                            cudaMemcpyDeviceToDevice, es))
            s = cuda_fail(e, "copy back");
    }
    sts.t_end = t;
    sts.stages = sts.steps * o->rk_order;
    if (graph) {
        cudaGraph_t gr = nullptr;
        cudaError_t e = cudaStreamEndCapture(es, &gr);
        if (s) {
            if (gr) cudaGraphDestroy(gr);
            return s;
        }
        if (e) return cuda_fail(e, "end capture");
        e = cudaGraphInstantiate(&g->gexec, gr, 0);
        cudaGraphDestroy(gr);
        if (e) {
            g->gexec = nullptr;
            return cuda_fail(e, "graph instantiate");
        }
        g->gkey = lsp_grid::Key{phi, target, ws, t0, t_final, *o};
        g->gstats = sts;
        e = cudaGraphLaunch(g->gexec, st);
        if (e) return cuda_fail(e, "graph launch");
    }
    if (s) return s;
    if (stats) *stats = sts;
    if (o->check_finite) return read_flags(ws, st);
    return LSP_OK;
}

lsp_status lsp_set_tile(lsp_grid* g, int tb, int ta, int ch, int minb, int pair)
{
    if (!g) return fail(LSP_EINVAL, "grid is NULL");
    if (g->gexec) {
        cudaGraphExecDestroy(g->gexec);
        g->gexec = nullptr;
    }
    if (tb < 0) {
        g->tile_mode = -1;
        return LSP_OK;
    }
    if (tb == 0 && ta == 0 && ch == 0) {
        g->tile_mode = 0;
        return LSP_OK;
    }
    lsp::Tile t{tb, ta, ch, minb, pair};
    // validated for a scheme that has the variant (the step re-checks the
    // tile against its own scheme and runs the generic kernel if it fails)
    if (!lsp::tile_valid(g->ndim, pair == 5 ? LSP_ENO2 : (pair >= 3 ? LSP_ENO3 : LSP_WENO5), t,
                         g->n))
        return fail(LSP_EINVAL, "tile %dx%dx%d (%d CTAs/SM) is not valid for this grid", tb, ta,
                    ch, minb);
    g->tile = t;
    g->tile_mode = 1;
    return LSP_OK;
}

lsp_status lsp_get_tile(const lsp_grid* g, const lsp_solve_opts* o, int* tb, int* ta, int* ch,
                        int* minb, int* pair)
{
    lsp_status s = check_opts(g, o);
    if (s) return s;
    if (!tb || !ta || !ch || !minb || !pair) return fail(LSP_EINVAL, "NULL argument");
    const lsp::Tile t = tile_in_effect(g, o);
    if (t.ch == 0) {
        *tb = *ta = *ch = *minb = *pair = -1;
    } else {
        *tb = t.tb;
        *ta = t.ta;
        *ch = t.ch;
        *minb = t.minb;
        *pair = t.pair;
    }
    return LSP_OK;
}

lsp_status lsp_autotune(lsp_grid* g, const lsp_solve_opts* o, const void* phi, void* ws,
                        size_t ws_size, void* stream, int* tb_out, int* ta_out, int* ch_out,
                        int* minb_out, int* pair_out)
{
    lsp_status s = check_opts(g, o);
    if (!s) s = check_field(phi, "phi");
    if (!s) s = check_ws(g, o, ws, ws_size);
    if (s) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if (o->dtype != LSP_F32 || (g->ndim != 3 && g->ndim != 4)) {
        g->tile_mode = -1;
        if (tb_out) *tb_out = -1;
        if (ta_out) *ta_out = -1;
        if (ch_out) *ch_out = -1;
        if (minb_out) *minb_out = -1;
        if (pair_out) *pair_out = -1;
        return LSP_OK;
    }
    if (!g->alpha_state) return fail(LSP_EUNSUPPORTED, "autotune needs state-only LF bounds");
    const int d = g->ndim;
    // fixed shapes, then two fitted to the grid: about 32 (16) nodes of the
    // fastest axis and as many rows as 256 threads allow, each rounded up so
    // that the tiles divide the two axes evenly (81 nodes: 27 x 9, 14 x 17),
    // which leaves fewer idle threads in the last tile of a row or column
    int shapes[9][2] = {{32, 8}, {32, 4}, {16, 8}, {16, 16}, {64, 4}, {32, 6}, {48, 4}};
    int nshapes = 7;
    for (const int wmax : {32, 16}) {
        const int nB = g->n[d - 1], nA = g->n[d - 2];
        const int tb = (nB + (nB + wmax - 1) / wmax - 1) / ((nB + wmax - 1) / wmax);
        const int hmax = 256 / tb;
        const int ta = (nA + (nA + hmax - 1) / hmax - 1) / ((nA + hmax - 1) / hmax);
        bool dup = false;
        for (int i = 0; i < nshapes; ++i) dup |= shapes[i][0] == tb && shapes[i][1] == ta;
        if (!dup) {
            shapes[nshapes][0] = tb;
            shapes[nshapes][1] = ta;
            ++nshapes;
        }
    }
    const int splits[] = {1, 2, 3, 4, 6, 8, 12};
    lsp::Ctl* ctl = (lsp::Ctl*)ws;
    float* w1 = (float*)((char*)ws + lsp::kCtlBytes);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) || cudaEventCreate(&e1)) return fail(LSP_ECUDA, "event create");
    lsp_grid trial = *g;
    trial.gexec = nullptr;
    trial.capture_stream = nullptr;
    // Candidates are timed on whole RK steps of a scratch copy of phi (the
    // caller's field is never written), with a copy of phi standing in for
    // the tube target: the later stages read the previous level and the
    // target besides the stencil field, and single first stages (which read
    // phi alone) ranked the tiles differently from the solve.  Without room
    // for the two scratch fields the first stage alone is timed.
    const size_t F = round256((size_t)g->npts * sizeof(float));
    char* scratch = nullptr;
    if (cudaMalloc(&scratch, 2 * F) != cudaSuccess) {
        cudaGetLastError();
        scratch = nullptr;
    }
    float* sphi = (float*)scratch;
    float* stgt = scratch ? (float*)(scratch + F) : nullptr;
    if (scratch && (cudaMemcpyAsync(sphi, phi, (size_t)g->npts * sizeof(float),
                                    cudaMemcpyDeviceToDevice, st) ||
                    cudaMemcpyAsync(stgt, phi, (size_t)g->npts * sizeof(float),
                                    cudaMemcpyDeviceToDevice, st))) {
        cudaFree(scratch);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return fail(LSP_ECUDA, "autotune scratch copy");
    }
    float best_ms = 1e30f;
    lsp::Tile best{0, 0, 0, 0, 0};
    // the fastest few of the first round, re-timed over longer windows
    constexpr int kFinal = 6;
    float top_ms[kFinal];
    lsp::Tile top[kFinal];
    int ntop = 0;
    const double dt = cfl_dt_host(g, o->cfl, 0.0, INFINITY);
    auto run_once = [&]() -> lsp_status {
        if (scratch) return enqueue_step<float>(&trial, o, sphi, o->tube ? stgt : nullptr, dt, ws, st);
        return enqueue_stage<float>(&trial, o, ctl, (const float*)phi, nullptr, nullptr, w1, dt,
                                    0.0, 1.0, 1.0, false, st);
    };
    // the face-shared ENO runs (pair 3: 4 nodes per thread, pair 4: 2): 16,
    // 28 or 32 nodes of the fastest axis per CTA and 4, 8 or 16 rows, or as
    // many rows as split the second-fastest axis evenly into tiles of at most
    // 16, 10 or 6 rows (81 nodes: 14, 9 and 6 rows; 9 x 9 rows ran the car4d
    // stage 5 % faster than 8 or 14)
    constexpr int kRunRows = 6;
    int run_rows[kRunRows] = {4, 8, 16, 0, 0, 0};
    {
        const int nA = g->n[d - 2];
        const int target[3] = {16, 10, 6};
        for (int q = 0; q < 3; ++q) {
            const int k = (nA + target[q] - 1) / target[q];
            run_rows[3 + q] = (nA + k - 1) / k;
        }
    }
    const bool eno = o->scheme == LSP_ENO2 || o->scheme == LSP_ENO3;
    const int nrun = eno ? 3 * kRunRows : 0;
    for (int si = 0; si < nshapes + nrun; ++si) {
        const bool run = si >= nshapes;
        const int run_tb[3] = {16, 28, 32};
        const int ri = (si - nshapes) % kRunRows;
        const int sh[2] = {run ? run_tb[(si - nshapes) / kRunRows] : shapes[si][0],
                           run ? run_rows[ri] : shapes[si][1]};
        if (run && ri >= 3) {
            bool dup = false;
            for (int q = 0; q < ri; ++q) dup |= run_rows[q] == sh[1];
            if (dup) continue;
        }
        for (int cand = 0; cand < 63; ++cand) {
            const int sp = splits[cand % 7];
            const int minb = 2 + (cand / 7) % 3;
            int pair = cand / 21;
            if (run) {  // runs of 4 (128 registers) and of 2 (80 registers)
                if (cand >= 14) break;
                pair = cand < 7 ? 3 : 4;
            }
            if (pair == 2 && o->scheme != LSP_WENO5) continue;
            if (pair == 1 && o->scheme == LSP_UPWIND1) continue;
            const int nS = g->n[d - 3];
            lsp::Tile t{sh[0], sh[1], (nS + sp - 1) / sp, run ? (pair == 3 ? 2 : 3) : minb, pair};
            if (!lsp::tile_valid(d, o->scheme, t, g->n)) continue;
            trial.tile = t;
            trial.tile_mode = 1;
            float ms_min = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                cudaEventRecord(e0, st);
                s = run_once();
                cudaEventRecord(e1, st);
                if (s) break;
                cudaEventSynchronize(e1);
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0 && ms < ms_min) ms_min = ms;  // first run warms up
            }
            if (s) break;
            // keep the kFinal fastest, sorted
            int pos = ntop < kFinal ? ntop++ : kFinal;
            if (pos == kFinal && ms_min >= top_ms[kFinal - 1]) continue;
            if (pos == kFinal) pos = kFinal - 1;
            while (pos > 0 && top_ms[pos - 1] > ms_min) {
                top_ms[pos] = top_ms[pos - 1];
                top[pos] = top[pos - 1];
                --pos;
            }
            top_ms[pos] = ms_min;
            top[pos] = t;
        }
        if (s) break;
    }
    // second round: each finalist timed as the best of 3 windows of 3
    // back-to-back runs (single runs of ~0.1-1 ms differ by a few %)
    for (int i = 0; i < ntop && !s; ++i) {
        trial.tile = top[i];
        trial.tile_mode = 1;
        float ms_min = 1e30f;
        for (int rep = 0; rep < 3 && !s; ++rep) {
            cudaEventRecord(e0, st);
            for (int k = 0; k < 3 && !s; ++k) s = run_once();
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < ms_min) ms_min = ms;
        }
        if (!s && ms_min < best_ms) {
            best_ms = ms_min;
            best = top[i];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (scratch) {
        cudaError_t e = cudaStreamSynchronize(st);
        cudaFree(scratch);
        if (!s && e != cudaSuccess) return cuda_fail(e, "autotune");
    }
    if (s) return s;
    if (best.ch == 0) return fail(LSP_EUNSUPPORTED, "no valid tile for this grid");
    g->tile = best;
    g->tile_mode = 1;
    if (g->gexec) {
        cudaGraphExecDestroy(g->gexec);
        g->gexec = nullptr;
    }
    if (tb_out) *tb_out = best.tb;
    if (ta_out) *ta_out = best.ta;
    if (ch_out) *ch_out = best.ch;
    if (minb_out) *minb_out = best.minb;
    if (pair_out) *pair_out = best.pair;
    return LSP_OK;
}

}  // extern "C"

namespace {

struct BatchPlanEntry {
    int p;  // index in the caller's arrays
    int nsteps;
    double dt, dt_last;
    int nbx, nby, nchunks, ch, nblocks;
    int tb, ta;          // tile of the two fastest axes
    size_t field_bytes;  // one stage field, rounded to 256
};

// Prefix the thread's last-error text with the problem index.
lsp_status fail_problem(lsp_status s, int i)
{
    char tmp[sizeof(g_err)];
    std::snprintf(tmp, sizeof(tmp), "%s", g_err);
    return fail(s, "problem %d: %s", i, tmp);
}

lsp_status batch_check(int nprob, lsp_grid* const* grids, const lsp_solve_opts* o)
{
    if (nprob < 1) return fail(LSP_EINVAL, "nprob must be >= 1");
    if (!grids) return fail(LSP_EINVAL, "grids is NULL");
    if (!o) return fail(LSP_EINVAL, "opts is NULL");
    if (o->dtype != LSP_F32) return fail(LSP_EUNSUPPORTED, "batched solves are FP32");
    if (o->rk_order != 2 && o->rk_order != 3)
        return fail(LSP_EUNSUPPORTED, "batched solves use TVD-RK2 or RK3");
    for (int i = 0; i < nprob; ++i) {
        const lsp_grid* g = grids[i];
        lsp_status s = check_opts(g, o);
        if (s) return fail_problem(s, i);
        if (!g->alpha_state)
            return fail(LSP_EUNSUPPORTED, "problem %d: batched solves need state-only LF bounds", i);
        if (!lsp::batch_supported(g->ndim, g->dyn))
            return fail(LSP_EUNSUPPORTED, "problem %d: no batched kernel for ndim=%d dyn=%d", i,
                        g->ndim, g->dyn);
    }
    return LSP_OK;
}

// Persistent launch state: control block, per-problem completion counters,
// segment table (at most one segment per problem, plus the end marker).
size_t batch_persist_bytes(int nprob)
{
    return round256(sizeof(lsp::PersistCtl)) + round256((size_t)nprob * sizeof(unsigned int)) +
           round256((size_t)(nprob + 1) * sizeof(lsp::BatchSegment));
}

// Test hook of the persistent batched launch (lsp_debug_stall_problem).
int g_stall_problem = -1;

// Tile grid and field sizes of every problem; the total workspace bytes.
// any_shape: size the block table for the largest tile count over every
// shape (a workspace that serves any opts->batch_tiles).
void batch_geometry(int nprob, lsp_grid* const* grids, const lsp_solve_opts* o,
                    std::vector<BatchPlanEntry>& plan, size_t* bytes, long long* total_blocks,
                    bool any_shape = false)
{
    // 128 planes per CTA by default (a whole column of every problem up to
    // 128 nodes along the march): the persistent launch's per-item overhead
    // (counter, fences, dependency poll) is paid per tile, and the graph form
    // gains too (256-problem workload: 67.5 / 67.0 G updates/s at 128 against
    // 65.8 / 66.3 G at 64, 61.7 / 65.0 G at 32 and 54.3 / 61.5 G at 16,
    // persistent / graph)
    const int chunk = o->batch_chunk > 0 ? o->batch_chunk : 128;
    plan.resize(nprob);
    size_t fields = 0;
    long long blocks = 0;
    for (int i = 0; i < nprob; ++i) {
        const lsp_grid* g = grids[i];
        BatchPlanEntry& e = plan[i];
        const int d = g->ndim;
        e.p = i;
        e.nsteps = 0;
        e.dt = e.dt_last = 0.0;
        // the local-coefficient / clipped kernels are compiled for 16 x 16 tiles
        const bool local = o->diss != LSP_DISS_GLF || o->varform;
        const int shape = local ? 0 : (o->batch_tiles >> (2 * (d - 2))) & 3;
        long long nb_max = 0;
        for (int sh = 0; sh < 3; ++sh) {
            if (!any_shape && sh != shape) continue;
            int tb = 16, ta = 16;
            lsp::batch_tile_dims(sh, &tb, &ta);
            const int nbx = (g->n[d - 1] + tb - 1) / tb, nby = (g->n[d - 2] + ta - 1) / ta;
            int ch = 1, nchunks = 1;
            if (d >= 3) {
                const int nS = g->n[d - 3];
                ch = std::min(chunk, nS);
                nchunks = (nS + ch - 1) / ch;
            }
            const long long nb = (long long)nbx * nby * nchunks * (d == 4 ? g->n[0] : 1);
            nb_max = std::max(nb_max, nb);
            if (sh == shape) {
                e.tb = tb;
                e.ta = ta;
                e.nbx = nbx;
                e.nby = nby;
                e.ch = ch;
                e.nchunks = nchunks;
                e.nblocks = (int)nb;
            }
        }
        e.field_bytes = round256((size_t)g->npts * sizeof(float));
        fields += nfields(o->rk_order) * e.field_bytes;
        blocks += any_shape ? nb_max : e.nblocks;
    }
    *total_blocks = blocks;
    *bytes = lsp::kCtlBytes + round256((size_t)nprob * sizeof(lsp::BatchProblem)) +
             round256((size_t)blocks * sizeof(int)) + batch_persist_bytes(nprob) + fields;
}

// The persistent variant of lsp_hj_solve_batched: segments of steps with a
// constant set of active problems (a prefix of `order`, sorted by decreasing
// step count), items (step, stage, tile) numbered in that order, one
// cooperative launch.
lsp_status solve_batched_persistent(int nprob, const lsp_solve_opts* o,
                                    const std::vector<BatchPlanEntry>& order,
                                    const std::vector<int>& prefix, const lsp::BatchProblem* d_table,
                                    const int* d_block_prob, lsp::PersistCtl* d_pc,
                                    unsigned int* d_done, lsp::BatchSegment* d_segs, lsp::Ctl* ctl,
                                    void* ws, int cls, cudaStream_t st)
{
    const int rk = o->rk_order;
    std::vector<lsp::BatchSegment> segs;
    long long items = 0;
    int nactive = nprob, k = 0;
    for (;;) {
        while (nactive > 0 && order[nactive - 1].nsteps <= k) --nactive;
        if (nactive == 0) break;
        const int k_end = order[nactive - 1].nsteps;
        lsp::BatchSegment sg;
        sg.item_start = items;
        sg.k_start = k;
        sg.blocks = prefix[nactive];
        segs.push_back(sg);
        items += (long long)(k_end - k) * rk * prefix[nactive];
        k = k_end;
    }
    for (int j = 0; j < nprob; ++j)
        if ((long long)order[j].nsteps * rk * order[j].nblocks > 0xffffffffLL)
            return fail(LSP_EINVAL, "problem %d: too many tile stages for one persistent launch",
                        order[j].p);
    const int nseg = (int)segs.size();
    lsp::BatchSegment end;
    end.item_start = items;
    end.k_start = k;
    end.blocks = 0;
    segs.push_back(end);

    lsp::PersistCtl pc;
    std::memset(&pc, 0, sizeof(pc));
    pc.stall_problem = -1;
    for (int j = 0; j < nprob; ++j)
        if (order[j].p == g_stall_problem) pc.stall_problem = j;

    lsp_status s = reset_flags(ws, st);
    if (s) return s;
    // pageable sources: the copies are staged before the calls return
    cudaError_t e = cudaMemcpyAsync(d_pc, &pc, sizeof(pc), cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(d_segs, segs.data(), segs.size() * sizeof(segs[0]),
                                cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemsetAsync(d_done, 0, (size_t)nprob * sizeof(unsigned int), st);
    if (e) return cuda_fail(e, "upload persistent state");
    if (items == 0) return LSP_OK;
    const unsigned long long wait_ns =
        (unsigned long long)(o->batch_wait_ms > 0 ? o->batch_wait_ms : 1000) * 1000000ULL;
    e = lsp::launch_batched_persistent(o->scheme, d_table, d_block_prob, d_segs, nseg, rk, d_done,
                                       d_pc, ctl, wait_ns, o->diss != LSP_DISS_GLF || o->varform,
                                       cls, st);
    if (e) return cuda_fail(e, "persistent batched kernel");
    return LSP_OK;
}

}  // namespace

extern "C" {

int lsp_debug_stall_problem(int problem)
{
    const int prev = g_stall_problem;
    g_stall_problem = problem;
    return prev;
}

lsp_status lsp_batched_workspace_size(int nprob, lsp_grid* const* grids, const lsp_solve_opts* o,
                                      size_t* bytes)
{
    if (!bytes) return fail(LSP_EINVAL, "bytes is NULL");
    lsp_status s = batch_check(nprob, grids, o);
    if (s) return s;
    std::vector<BatchPlanEntry> plan;
    long long blocks = 0;
    batch_geometry(nprob, grids, o, plan, bytes, &blocks, true);
    return LSP_OK;
}

lsp_status lsp_hj_solve_batched(int nprob, lsp_grid* const* grids, const lsp_solve_opts* o,
                                void* const* phis, const void* const* targets,
                                const double* t_final, void* ws, size_t ws_size,
                                lsp_solve_stats* stats, void* stream)
{
    lsp_status s = batch_check(nprob, grids, o);
    if (s) return s;
    if (!phis || !t_final) return fail(LSP_EINVAL, "phis and t_final must not be NULL");
    if (o->tube && !targets) return fail(LSP_EINVAL, "targets is NULL with tube on");
    for (int i = 0; i < nprob; ++i) {
        if ((s = check_field(phis[i], "phi"))) return fail_problem(s, i);
        if (o->tube && (s = check_field(targets[i], "target"))) return fail_problem(s, i);
        if (!std::isfinite(t_final[i])) return fail(LSP_EINVAL, "problem %d: t_final not finite", i);
    }
    if (!ws || !aligned16(ws)) return fail(LSP_EINVAL, "workspace must be non-NULL and 16-byte aligned");
    std::vector<BatchPlanEntry> plan;
    size_t need = 0;
    long long total_blocks = 0;
    batch_geometry(nprob, grids, o, plan, &need, &total_blocks);
    if (ws_size < need) return fail(LSP_ENOMEM, "workspace has %zu bytes, needs %zu", ws_size, need);
    if (total_blocks > 0x7fffffffLL) return fail(LSP_EINVAL, "too many tiles");

    // per-problem FP64 time loop (the same as a single solve's)
    for (auto& e : plan) {
        const lsp_grid* g = grids[e.p];
        const double tf = t_final[e.p];
        const double t_stop = tf - 1e-12 * std::fabs(tf);
        double t = 0.0;
        e.dt = cfl_dt_host(g, o->cfl, 0.0, INFINITY);
        while (t < t_stop) {
            const double dt = cfl_dt_host(g, o->cfl, t, tf);
            if (!(dt > 0.0)) return fail(LSP_EINVAL, "problem %d: non-positive CFL step", e.p);
            e.dt_last = dt;
            t += dt;
            e.nsteps++;
        }
        if (stats) {
            lsp_solve_stats& st = stats[e.p];
            st.steps = e.nsteps;
            st.stages = (int64_t)e.nsteps * o->rk_order;
            st.dt_min = e.nsteps ? std::fmin(e.dt, e.dt_last) : INFINITY;
            st.dt_max = e.nsteps ? std::fmax(e.dt, e.dt_last) : 0.0;
            st.t_end = t;
        }
    }
    // longest first: the problems still running at step k are a prefix
    std::vector<BatchPlanEntry> order = plan;
    std::stable_sort(order.begin(), order.end(),
                     [](const BatchPlanEntry& a, const BatchPlanEntry& b) { return a.nsteps > b.nsteps; });

    lsp::Ctl* ctl = (lsp::Ctl*)ws;
    char* base = (char*)ws + lsp::kCtlBytes;
    lsp::BatchProblem* d_table = (lsp::BatchProblem*)base;
    base += round256((size_t)nprob * sizeof(lsp::BatchProblem));
    int* d_block_prob = (int*)base;
    base += round256((size_t)total_blocks * sizeof(int));
    lsp::PersistCtl* d_pc = (lsp::PersistCtl*)base;
    base += round256(sizeof(lsp::PersistCtl));
    unsigned int* d_done = (unsigned int*)base;
    base += round256((size_t)nprob * sizeof(unsigned int));
    lsp::BatchSegment* d_segs = (lsp::BatchSegment*)base;
    base += round256((size_t)(nprob + 1) * sizeof(lsp::BatchSegment));

    std::vector<lsp::BatchProblem> table(nprob);
    std::vector<int> block_prob((size_t)total_blocks);
    std::vector<int> prefix(nprob + 1, 0);
    for (int j = 0; j < nprob; ++j) {
        const BatchPlanEntry& e = order[j];
        const lsp_grid* g = grids[e.p];
        lsp::BatchProblem& P = table[j];
        std::memset(&P, 0, sizeof(P));
        P.a = base_args<float>(g, ctl);
        P.a.tube = o->tube ? 1 : 0;
        P.a.local_alpha = o->diss != LSP_DISS_GLF;
        P.a.varform = o->varform;
        P.phi = (float*)phis[e.p];
        P.target = o->tube ? (const float*)targets[e.p] : nullptr;
        P.w1 = (float*)base;
        base += e.field_bytes;
        P.w2 = o->rk_order == 3 ? (float*)base : nullptr;
        if (o->rk_order == 3) base += e.field_bytes;
        P.dt = e.dt;
        P.dt_last = e.dt_last;
        P.nsteps = e.nsteps;
        P.ndim = g->ndim;
        P.dyn = g->dyn;
        P.ch = e.ch;
        P.nbx = e.nbx;
        P.nby = e.nby;
        P.nchunks = e.nchunks;
        P.tb = e.tb;
        P.ta = e.ta;
        P.block_start = prefix[j];
        P.nblocks = e.nblocks;
        prefix[j + 1] = prefix[j] + e.nblocks;
        for (int b = 0; b < e.nblocks; ++b) block_prob[(size_t)prefix[j] + b] = j;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // pageable sources: the copies are staged before the calls return
    cudaError_t e = cudaMemcpyAsync(d_table, table.data(), table.size() * sizeof(table[0]),
                                    cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(d_block_prob, block_prob.data(), block_prob.size() * sizeof(int),
                                cudaMemcpyHostToDevice, st);
    if (e) return cuda_fail(e, "upload batch table");

    // the class set the kernels are compiled for: 2-D normal speed and 3-D
    // air3d alone when those are the only problems, else every class
    int cls = lsp::kBatchClsNormal2Air3;
    for (int i = 0; i < nprob; ++i) {
        const lsp_grid* g = grids[i];
        if (!((g->ndim == 2 && g->dyn == LSP_DYN_NORMAL_SPEED) ||
              (g->ndim == 3 && g->dyn == LSP_DYN_AIR3D)))
            cls = lsp::kBatchClsAll;
    }
    if (cls == lsp::kBatchClsNormal2Air3 && o->batch_tiles == 0) cls = lsp::kBatchClsNormal2Air3x16;
    if (o->batch_persistent) {
        s = solve_batched_persistent(nprob, o, order, prefix, d_table, d_block_prob, d_pc, d_done,
                                     d_segs, ctl, ws, cls, st);
        if (s) return s;
        if (o->check_finite) return read_flags(ws, st);
        return LSP_OK;
    }

    cudaStream_t es = st;
    cudaStream_t cap = nullptr;
    if (o->use_graph) {
        if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking))) return cuda_fail(e, "create stream");
        es = cap;
        if ((e = cudaStreamBeginCapture(es, cudaStreamCaptureModeThreadLocal))) {
            cudaStreamDestroy(cap);
            return cuda_fail(e, "begin capture");
        }
    }
    s = reset_flags(ws, es);
    int nactive = nprob;
    const int maxsteps = nprob ? order[0].nsteps : 0;
    for (int k = 0; !s && k < maxsteps; ++k) {
        while (nactive > 0 && order[nactive - 1].nsteps <= k) --nactive;
        for (int stage = 0; stage < o->rk_order && !s; ++stage) {
            e = lsp::launch_batched(o->scheme, d_table, d_block_prob, prefix[nactive], k, stage,
                                    o->rk_order, o->diss != LSP_DISS_GLF || o->varform, cls, es);
            if (e) s = cuda_fail(e, "batched stage kernel");
        }
    }
    if (o->use_graph) {
        cudaGraph_t gr = nullptr;
        e = cudaStreamEndCapture(es, &gr);
        if (!s && e) s = cuda_fail(e, "end capture");
        cudaGraphExec_t ex = nullptr;
        if (!s && (e = cudaGraphInstantiate(&ex, gr, 0))) s = cuda_fail(e, "graph instantiate");
        if (!s && (e = cudaGraphLaunch(ex, st))) s = cuda_fail(e, "graph launch");
        if (ex) cudaGraphExecDestroy(ex);
        if (gr) cudaGraphDestroy(gr);
        cudaStreamDestroy(cap);
    }
    if (s) return s;
    if (o->check_finite) return read_flags(ws, st);
    return LSP_OK;
}

lsp_status lsp_batched_autotune(int nprob, lsp_grid* const* grids, const lsp_solve_opts* o,
                                const void* const* phis, const void* const* targets,
                                const double* t_final, void* ws, size_t ws_size, void* stream,
                                int* batch_tiles)
{
    lsp_status s = batch_check(nprob, grids, o);
    if (s) return s;
    if (!phis || !t_final || !batch_tiles) return fail(LSP_EINVAL, "NULL argument");
    if (o->tube && !targets) return fail(LSP_EINVAL, "targets is NULL with tube on");
    cudaStream_t st = (cudaStream_t)stream;
    // scratch copies of the fields: trial solves never write the caller's
    size_t total = 0;
    std::vector<size_t> off(nprob);
    for (int i = 0; i < nprob; ++i) {
        if ((s = check_field(phis[i], "phi"))) return fail_problem(s, i);
        off[i] = total;
        total += round256((size_t)grids[i]->npts * sizeof(float));
    }
    char* scratch = nullptr;
    cudaError_t e = cudaMalloc(&scratch, total);
    if (e) return cuda_fail(e, "batched autotune scratch");
    std::vector<void*> sp(nprob);
    for (int i = 0; i < nprob; ++i) sp[i] = scratch + off[i];
    // a short horizon of every problem (at most 8 of its CFL steps), so
    // that the trials see the full mix of problems
    std::vector<double> tf(nprob);
    for (int i = 0; i < nprob; ++i)
        tf[i] = std::fmin(t_final[i], 8.0 * cfl_dt_host(grids[i], o->cfl, 0.0, INFINITY));
    lsp_solve_opts trial = *o;
    trial.use_graph = 0;
    trial.check_finite = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) || cudaEventCreate(&e1)) {
        cudaFree(scratch);
        return fail(LSP_ECUDA, "event create");
    }
    auto time_tiles = [&](int tiles, float* ms_out) -> lsp_status {
        trial.batch_tiles = tiles;
        float best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            for (int i = 0; i < nprob; ++i) {
                cudaError_t ce = cudaMemcpyAsync(sp[i], phis[i], grids[i]->npts * sizeof(float),
                                                 cudaMemcpyDeviceToDevice, st);
                if (ce) return cuda_fail(ce, "batched autotune copy");
            }
            cudaEventRecord(e0, st);
            lsp_status r = lsp_hj_solve_batched(nprob, grids, &trial, sp.data(), targets,
                                                tf.data(), ws, ws_size, nullptr, st);
            cudaEventRecord(e1, st);
            if (r) return r;
            cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < best) best = ms;  // the first run warms up
        }
        *ms_out = best;
        return LSP_OK;
    };
    // coordinate descent over the dimensions present, from opts->batch_tiles
    int best_tiles = o->batch_tiles;
    float best_ms = 0.0f;
    s = time_tiles(best_tiles, &best_ms);
    for (int d = 2; d <= 4 && !s; ++d) {
        bool present = false;
        for (int i = 0; i < nprob; ++i) present |= grids[i]->ndim == d;
        if (!present) continue;
        for (int shape = 0; shape < 3 && !s; ++shape) {
            const int tiles = (best_tiles & ~(3 << (2 * (d - 2)))) | (shape << (2 * (d - 2)));
            if (tiles == best_tiles) continue;
            float ms = 0.0f;
            s = time_tiles(tiles, &ms);
            if (!s && ms < best_ms) {
                best_ms = ms;
                best_tiles = tiles;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    e = cudaStreamSynchronize(st);
    cudaFree(scratch);
    if (s) return s;
    if (e) return cuda_fail(e, "batched autotune");
    *batch_tiles = best_tiles;
    return LSP_OK;
}

}  // extern "C"

namespace {

// ----------------------------------------------------------------- adjoint
// Workspace of a checkpointed forward solve and its reverse sweep:
// [ctl 256][W1][W2][acc 256][ckpt: C fields][seg: K fields][seg stage
// inputs: (rk-1) K fields][lam][lam_n][lam_a][lam_b][lam_v][contrib: 7*ndim
// fields], K = ceil(nsteps / C).  The recomputation of a segment keeps every
// step's stage inputs (W1, W2), which the reverse sweep of that segment reads
// instead of recomputing them.
struct AdjLayout {
    int C, K;
    bool keep_all;  // ncheck < 0: every state and stage input stored by the forward
    size_t F;  // one field, rounded to 256 bytes
    size_t off_acc, off_ckpt, off_seg, off_segw, off_w1, off_w2, off_lam, off_lamn, off_lama,
        off_lamb, off_lamv, off_contrib, total;
};

AdjLayout adj_layout(const lsp_grid* g, const lsp_solve_opts* o, int nsteps, int ncheck)
{
    AdjLayout L;
    L.keep_all = ncheck < 0;
    L.C = ncheck > 0 ? ncheck : ncheck < 0 ? nsteps
                                          : (int)std::ceil(std::sqrt((double)std::max(nsteps, 1)));
    if (L.C > nsteps) L.C = std::max(nsteps, 1);
    L.K = (nsteps + L.C - 1) / L.C;
    if (L.K < 1) L.K = 1;
    L.F = round256((size_t)g->npts * elem_size(o->dtype));
    // W1 and W2 come first so that the stage launches of a plain step (which
    // expect [ctl][W1][W2]) can run on this workspace unchanged
    size_t off = lsp::kCtlBytes;
    L.off_w1 = off; off += L.F;
    L.off_w2 = off; off += L.F;
    L.off_acc = off; off += 256;
    L.off_ckpt = off; off += (size_t)L.C * L.F;
    // keep_all: the checkpoints are the states, and the stage inputs of
    // every step follow them (no recomputation segment)
    L.off_seg = off; off += L.keep_all ? 0 : (size_t)L.K * L.F;
    L.off_segw = off;
    off += (size_t)(o->rk_order - 1) * (L.keep_all ? (size_t)L.C : (size_t)L.K) * L.F;
    L.off_lam = off; off += L.F;
    L.off_lamn = off; off += L.F;
    L.off_lama = off; off += L.F;
    L.off_lamb = off; off += L.F;
    L.off_lamv = off; off += L.F;
    // two sets of 7 ndim coefficient fields: a stage's pass A writes one
    // while the same launch gathers the previous stage's from the other
    L.off_contrib = off; off += (size_t)2 * 7 * g->ndim * L.F;
    L.total = off;
    return L;
}

lsp_status adj_check(const lsp_grid* g, const lsp_solve_opts* o, int nsteps)
{
    lsp_status s = check_opts(g, o);
    if (s) return s;
    if (!g->alpha_state) return fail(LSP_EUNSUPPORTED, "the adjoint needs state-only LF bounds");
    if (g->dyn == LSP_DYN_QUADRATIC)
        return fail(LSP_EUNSUPPORTED, "no adjoint for dynamics %d", g->dyn);
    if (o->diss != LSP_DISS_GLF || o->varform)
        return fail(LSP_EUNSUPPORTED, "the adjoint reverses the GLF form without the clip");
    if (nsteps < 1) return fail(LSP_EINVAL, "nsteps must be >= 1");
    return LSP_OK;
}

// One reversed RK stage: v = c_n phin + c_s u + c_l dt L(u), out = min(v, g)
// in a tube stage; dLoss/du is collected in lam_u, c_n dLoss/dv in lam_n.
template <typename R>
struct AdjStage {
    const R* u;
    const R* phin;
    const R* target;
    R* lam_u;
    R* lam_n;
    R* lam_g;
    double c_n, c_s, c_l;
    bool tube;
};

// Launch pass A of stage d, fused with pass B of `prev` (the stage reversed
// just before, NULL for the first), writing coefficient set `set`; or, with
// pass_b, pass B of d alone (its coefficients in set `set`).  lam: dLoss/dout
// of d when prev is NULL.
template <typename R>
lsp_status adj_stage(const lsp_grid* g, const lsp_solve_opts* o, void* ws, const AdjLayout& Lo,
                     const AdjStage<R>& d, const AdjStage<R>* prev, const R* lam, int set,
                     bool pass_b, double dt, cudaStream_t st)
{
    lsp::AdjArgs<R> a;
    std::memset(&a, 0, sizeof(a));
    const size_t set_bytes = (size_t)7 * g->ndim * Lo.F;
    a.u = d.u;
    a.phin = d.phin;
    a.target = d.target;
    a.lam = lam;
    a.lam_v = (R*)((char*)ws + Lo.off_lamv);
    a.contrib = (R*)((char*)ws + Lo.off_contrib + (size_t)set * set_bytes);
    a.cstride = (long long)(Lo.F / sizeof(R));
    a.lam_u = d.lam_u;
    a.lam_n = d.lam_n;
    a.lam_g = d.tube ? d.lam_g : nullptr;
    if (prev && !pass_b) {
        a.gcontrib = (const R*)((char*)ws + Lo.off_contrib + (size_t)(1 - set) * set_bytes);
        a.glam_u = prev->lam_u;
        a.glam_n = prev->lam_n;
        a.gc_s = R(prev->c_s);
        a.gc_n = R(prev->c_n);
        a.gatomic = prev->lam_n && prev->lam_n != prev->lam_u && prev->lam_n == d.lam_u;
    }
    a.acc = (lsp::AdjAcc*)((char*)ws + Lo.off_acc);
    long long sd = 1;
    for (int k = g->ndim - 1; k >= 0; --k) {
        a.n[k] = g->n[k];
        a.stride[k] = (int)sd;
        sd *= g->n[k];
        a.periodic[k] = g->periodic[k];
        a.inv_dx[k] = R(1.0 / g->dx[k]);
        a.lo[k] = R(g->lo[k]);
        a.h[k] = R(g->dx[k]);
        a.alpha[k] = R(g->alpha[k]);
    }
    for (int i = 0; i < LSP_NPARAM; ++i) a.prm[i] = R(g->prm[i]);
    a.dt = R(dt);
    a.c_n = R(d.c_n);
    a.c_s = R(d.c_s);
    a.c_l = R(d.c_l);
    a.tube = d.tube ? 1 : 0;
    a.npts = (int)g->npts;
    cudaError_t e = lsp::launch_adjoint_stage<R>(g->ndim, o->scheme, g->dyn, a, pass_b, st);
    return e ? cuda_fail(e, "adjoint stage kernels") : LSP_OK;
}

// d alpha_k / d prm_j at the node attaining alpha_k (FP64, host).
void alpha_param_grads(const lsp_grid* g, const double* x, int k, double* gk)
{
    const double* c = g->prm;
    for (int j = 0; j < LSP_NPARAM; ++j) gk[j] = 0.0;
    auto sg = [](double v) { return v >= 0.0 ? 1.0 : -1.0; };
    switch (g->dyn) {
    case LSP_DYN_NORMAL_SPEED: gk[0] = g->prm[0] >= 0.0 ? 1.0 : -1.0; break;  // d|a|/da
    case LSP_DYN_TRANSLATE: gk[k] = sg(c[k]); break;
    case LSP_DYN_AIR3D:
        if (k == 0) {
            const double w = -c[0] + c[1] * std::cos(x[2]);
            gk[0] = -sg(w);
            gk[1] = sg(w) * std::cos(x[2]);
            gk[2] = std::fabs(x[1]);
        } else if (k == 1) {
            gk[1] = std::fabs(std::sin(x[2]));
            gk[2] = std::fabs(x[0]);
        } else {
            gk[2] = 1.0;
            gk[3] = 1.0;
        }
        break;
    case LSP_DYN_CAR4D:
        if (k == 2) gk[0] = 1.0;
        if (k == 3) gk[1] = 1.0;
        break;
    case LSP_DYN_ROCKETS:
        if (k == 0) {  // a |cos th| + ue |x|
            gk[0] = std::fabs(std::cos(x[2]));
            gk[2] = std::fabs(x[0]);
        } else if (k == 1) {  // |a sin th + a - g| + up |x|
            const double w = c[0] * std::sin(x[2]) + c[0] - c[1];
            gk[0] = sg(w) * (std::sin(x[2]) + 1.0);
            gk[1] = -sg(w);
            gk[3] = std::fabs(x[0]);
        } else {  // ue + up
            gk[2] = 1.0;
            gk[3] = 1.0;
        }
        break;
    case LSP_DYN_DOUBLE_INTEGRATOR:
        if (k == 1) gk[0] = sg(c[0]);  // |umax|
        break;
    }
}

template <typename R>
lsp_status adjoint_sweep(const lsp_grid* g, const lsp_solve_opts* o, const R* target, int nsteps,
                         const R* lamT, R* lam0, R* lam_target, double* dprm, void* ws,
                         const AdjLayout& Lo, cudaStream_t st)
{
    const size_t N = (size_t)g->npts;
    const size_t NB = N * sizeof(R);
    char* W = (char*)ws;
    lsp::Ctl* ctl = (lsp::Ctl*)ws;
    R* ckpt = (R*)(W + Lo.off_ckpt);
    R* seg = (R*)(W + Lo.off_seg);
    R* segw0 = (R*)(W + Lo.off_segw);
    R* w1 = (R*)(W + Lo.off_w1);
    R* w2 = (R*)(W + Lo.off_w2);
    R* lam = (R*)(W + Lo.off_lam);
    R* lamn = (R*)(W + Lo.off_lamn);
    R* lama = (R*)(W + Lo.off_lama);
    R* lamb = (R*)(W + Lo.off_lamb);
    const size_t FE = Lo.F / sizeof(R);  // field stride in elements
    const bool tube = o->tube != 0;
    const int rk = o->rk_order;
    const double dt = cfl_dt_host(g, o->cfl, 0.0, INFINITY);
    cudaError_t e;
    lsp_status s = LSP_OK;
    if ((e = cudaMemsetAsync(W + Lo.off_acc, 0, 256, st))) return cuda_fail(e, "memset acc");
    if ((e = cudaMemcpyAsync(lam, lamT, NB, cudaMemcpyDeviceToDevice, st))) return cuda_fail(e, "copy lamT");
    if (lam_target && (e = cudaMemsetAsync(lam_target, 0, NB, st))) return cuda_fail(e, "memset lam_target");
    // lamn, lama, lamb start at zero; every launch zeroes the buffer it reads
    for (R* b : {lamn, lama, lamb})
        if ((e = cudaMemsetAsync(b, 0, NB, st))) return cuda_fail(e, "memset");
    // the stage reversed last and the coefficient set its pass A wrote
    AdjStage<R> prev{};
    bool have_prev = false;
    int set = 0;
    auto run_stage = [&](const AdjStage<R>& d) -> lsp_status {
        lsp_status r = adj_stage<R>(g, o, ws, Lo, d, have_prev ? &prev : nullptr, lam, set, false,
                                    dt, st);
        prev = d;
        have_prev = true;
        set ^= 1;
        return r;
    };
    for (int sg = (nsteps - 1) / Lo.K; sg >= 0 && !s; --sg) {
        const int n0 = sg * Lo.K, n1 = std::min(n0 + Lo.K, nsteps);
        // stage inputs of step n of the segment (RK2/RK3): W1, then W2; with
        // keep_all, every step's as the forward stored them
        const int base = Lo.keep_all ? 0 : n0;
        auto segw = [&](int n, int q) { return segw0 + ((size_t)(n - base) * (rk - 1) + q) * FE; };
        if (Lo.keep_all) seg = ckpt + (size_t)n0 * FE;  // phi^n0, stored by the forward
        // states phi^n, n0 <= n < n1, recomputed from the checkpoint
        if (!Lo.keep_all) {
            e = cudaMemcpyAsync(seg, ckpt + (size_t)sg * FE, NB, cudaMemcpyDeviceToDevice, st);
            if (e) return cuda_fail(e, "restore checkpoint");
        }
        for (int n = n0; n < n1 && !s && !Lo.keep_all; ++n) {
            R* cur = seg + (size_t)(n - n0) * FE;
            if (n + 1 < n1) {  // phi^{n+1}, keeping step n's stage inputs
                R* nxt = seg + (size_t)(n - n0 + 1) * FE;
                e = cudaMemcpyAsync(nxt, cur, NB, cudaMemcpyDeviceToDevice, st);
                if (e) return cuda_fail(e, "copy state");
                s = enqueue_step<R>(g, o, nxt, target, dt, ws, st, rk >= 2 ? segw(n, 0) : nullptr,
                                    rk == 3 ? segw(n, 1) : nullptr);
            } else {  // the last step of the segment: its stage inputs alone
                if (rk >= 2)
                    s = enqueue_stage<R>(g, o, ctl, cur, nullptr, nullptr, segw(n, 0), dt, 0.0, 1.0,
                                         1.0, false, st);
                if (!s && rk == 3)
                    s = enqueue_stage<R>(g, o, ctl, segw(n, 0), cur, nullptr, segw(n, 1), dt, 0.75,
                                         0.25, 0.25, false, st);
            }
        }
        for (int n = n1 - 1; n >= n0 && !s; --n) {
            const R* phin = seg + (size_t)(n - n0) * FE;
            // the stage inputs of step n, as the recomputation (or, with
            // keep_all, the forward) left them
            if (rk >= 2) w1 = segw(n, 0);
            if (rk == 3) w2 = segw(n, 1);
            // Stages in reverse order.  dLoss/du of a stage goes to its own
            // buffer (lamb, lama, then lamn, which also collects the c_n
            // parts of the later stages: dLoss/dphi^n); RK1 alternates two
            // buffers by step, so that a launch never reads and clears the
            // buffer its own pass A folds into.
            if (rk == 1) {
                // phi^{n+1} = [phi^n + dt L(phi^n)]_tube
                R* lu = (n & 1) ? lama : lamn;
                s = run_stage({phin, nullptr, target, lu, lu, lam_target, 0.0, 1.0, 1.0, tube});
            } else if (rk == 2) {
                // phi^{n+1} = [1/2 phi^n + 1/2 W1 + 1/2 dt L(W1)]_tube
                s = run_stage({w1, phin, target, lama, lamn, lam_target, 0.5, 0.5, 0.5, tube});
                // W1 = phi^n + dt L(phi^n)
                if (!s) s = run_stage({phin, nullptr, nullptr, lamn, lamn, nullptr, 0.0, 1.0, 1.0, false});
            } else {
                // phi^{n+1} = [1/3 phi^n + 2/3 W2 + 2/3 dt L(W2)]_tube
                s = run_stage({w2, phin, target, lamb, lamn, lam_target, 1.0 / 3.0, 2.0 / 3.0,
                               2.0 / 3.0, tube});
                // W2 = 3/4 phi^n + 1/4 W1 + 1/4 dt L(W1)
                if (!s) s = run_stage({w1, phin, nullptr, lama, lamn, nullptr, 0.75, 0.25, 0.25, false});
                // W1 = phi^n + dt L(phi^n)
                if (!s) s = run_stage({phin, nullptr, nullptr, lamn, lamn, nullptr, 0.0, 1.0, 1.0, false});
            }
        }
    }
    // pass B of the last stage alone: dLoss/dphi^0
    if (!s) s = adj_stage<R>(g, o, ws, Lo, prev, nullptr, nullptr, set ^ 1, true, dt, st);
    lam = prev.lam_u;
    if (s) return s;
    if ((e = cudaMemcpyAsync(lam0, lam, NB, cudaMemcpyDeviceToDevice, st))) return cuda_fail(e, "copy lam0");
    // parameters: direct (through H) + through alpha (dissipation and dt)
    lsp::AdjAcc acc;
    if ((e = cudaMemcpyAsync(&acc, W + Lo.off_acc, sizeof(acc), cudaMemcpyDeviceToHost, st)))
        return cuda_fail(e, "read accumulators");
    // the node attaining each alpha_k
    lsp::GridGeom geo;
    std::memset(&geo, 0, sizeof(geo));
    geo.ndim = g->ndim;
    geo.npts = g->npts;
    for (int k = 0; k < g->ndim; ++k) {
        geo.n[k] = g->n[k];
        geo.lo[k] = g->lo[k];
        geo.h[k] = g->dx[k];
    }
    for (int i = 0; i < LSP_NPARAM; ++i) geo.prm[i] = g->prm[i];
    double* d_alpha = (double*)((char*)ctl->reserved);                       // 4 doubles
    unsigned long long* d_arg = (unsigned long long*)((char*)ctl->reserved + 32);  // 4 indices
    if ((e = cudaMemcpyAsync(d_alpha, g->alpha, 4 * sizeof(double), cudaMemcpyHostToDevice, st)))
        return cuda_fail(e, "upload alpha");
    if ((e = cudaMemsetAsync(d_arg, 0xff, 4 * sizeof(unsigned long long), st))) return cuda_fail(e, "memset");
    if ((e = lsp::launch_alpha_argmax(g->dyn, geo, d_alpha, d_arg, st))) return cuda_fail(e, "argmax");
    unsigned long long arg[4];
    if ((e = cudaMemcpyAsync(arg, d_arg, sizeof(arg), cudaMemcpyDeviceToHost, st)))
        return cuda_fail(e, "read argmax");
    if ((e = cudaStreamSynchronize(st))) return cuda_fail(e, "synchronize");
    double S = 0.0;
    for (int k = 0; k < g->ndim; ++k) S += g->alpha[k] / g->dx[k];
    for (int j = 0; j < LSP_NPARAM; ++j) dprm[j] = j < 4 ? acc.hprm[j] : 0.0;
    for (int k = 0; k < g->ndim; ++k) {
        double x[LSP_MAXD] = {0, 0, 0, 0};
        long long r = (long long)arg[k];
        for (int q = g->ndim - 1; q >= 0; --q) {
            x[q] = g->lo[q] + (double)(r % g->n[q]) * g->dx[q];
            r /= g->n[q];
        }
        double gk[LSP_NPARAM];
        alpha_param_grads(g, x, k, gk);
        const double dL_dalpha = acc.alpha[k] - acc.dt * o->cfl / (S * S * g->dx[k]);
        for (int j = 0; j < LSP_NPARAM; ++j) dprm[j] += dL_dalpha * gk[j];
    }
    return LSP_OK;
}

}  // namespace

extern "C" {

lsp_status lsp_adjoint_workspace_size(const lsp_grid* g, const lsp_solve_opts* o, int nsteps,
                                      int ncheck, size_t* bytes)
{
    if (!bytes) return fail(LSP_EINVAL, "bytes is NULL");
    lsp_status s = adj_check(g, o, nsteps);
    if (s) return s;
    *bytes = adj_layout(g, o, nsteps, ncheck).total;
    return LSP_OK;
}

lsp_status lsp_hj_solve_ckpt(lsp_grid* g, const lsp_solve_opts* o, void* phi, const void* target,
                             int nsteps, int ncheck, void* ws, size_t ws_size, void* stream)
{
    lsp_status s = adj_check(g, o, nsteps);
    if (!s) s = check_field(phi, "phi");
    if (!s && o->tube) s = check_field(target, "target");
    if (s) return s;
    if (!ws || !aligned16(ws)) return fail(LSP_EINVAL, "workspace must be non-NULL and 16-byte aligned");
    const AdjLayout Lo = adj_layout(g, o, nsteps, ncheck);
    if (ws_size < Lo.total) return fail(LSP_ENOMEM, "workspace has %zu bytes, needs %zu", ws_size, Lo.total);
    cudaStream_t st = (cudaStream_t)stream;
    const double dt = cfl_dt_host(g, o->cfl, 0.0, INFINITY);
    const size_t NB = (size_t)g->npts * elem_size(o->dtype);
    if ((s = reset_flags(ws, st))) return s;
    const int rk = o->rk_order;
    for (int n = 0; n < nsteps && !s; ++n) {
        if (n % Lo.K == 0) {
            cudaError_t e = cudaMemcpyAsync((char*)ws + Lo.off_ckpt + (size_t)(n / Lo.K) * Lo.F, phi,
                                            NB, cudaMemcpyDeviceToDevice, st);
            if (e) return cuda_fail(e, "store checkpoint");
        }
        if (Lo.keep_all && rk > 1) {  // the stage inputs written where the reverse reads them
            char* w1 = (char*)ws + Lo.off_segw + (size_t)n * (rk - 1) * Lo.F;
            char* w2 = rk == 3 ? w1 + Lo.F : nullptr;
            s = o->dtype == LSP_F64
                    ? enqueue_step<double>(g, o, (double*)phi, (const double*)target, dt, ws, st,
                                           (double*)w1, (double*)w2)
                    : enqueue_step<float>(g, o, (float*)phi, (const float*)target, dt, ws, st,
                                          (float*)w1, (float*)w2);
        } else {
            s = step_any(g, o, phi, target, dt, ws, st);
        }
    }
    if (s) return s;
    if (o->check_finite) return read_flags(ws, st);
    return LSP_OK;
}

lsp_status lsp_hj_adjoint(lsp_grid* g, const lsp_solve_opts* o, const void* target, int nsteps,
                          int ncheck, const void* lamT, void* lam0, void* lam_target, double* dprm,
                          void* ws, size_t ws_size, void* stream)
{
    lsp_status s = adj_check(g, o, nsteps);
    if (!s) s = check_field(lamT, "lamT");
    if (!s) s = check_field(lam0, "lam0");
    if (!s && o->tube) s = check_field(target, "target");
    if (!s && lam_target) s = check_field(lam_target, "lam_target");
    if (s) return s;
    if (!dprm) return fail(LSP_EINVAL, "dprm is NULL");
    if (!ws || !aligned16(ws)) return fail(LSP_EINVAL, "workspace must be non-NULL and 16-byte aligned");
    const AdjLayout Lo = adj_layout(g, o, nsteps, ncheck);
    if (ws_size < Lo.total) return fail(LSP_ENOMEM, "workspace has %zu bytes, needs %zu", ws_size, Lo.total);
    cudaStream_t st = (cudaStream_t)stream;
    if (o->dtype == LSP_F64)
        return adjoint_sweep<double>(g, o, (const double*)target, nsteps, (const double*)lamT,
                                     (double*)lam0, (double*)lam_target, dprm, ws, Lo, st);
    return adjoint_sweep<float>(g, o, (const float*)target, nsteps, (const float*)lamT,
                                (float*)lam0, (float*)lam_target, dprm, ws, Lo, st);
}

lsp_status lsp_loss_tube(const lsp_grid* g, int dtype, const void* phi, const void* queries,
                         int nq, double* value_dev, void* grad, void* stream)
{
    if (!g) return fail(LSP_EINVAL, "grid is NULL");
    lsp_status s = check_field(phi, "phi");
    if (s) return s;
    if (nq < 0 || (nq > 0 && !queries)) return fail(LSP_EINVAL, "bad queries");
    if (!value_dev) return fail(LSP_EINVAL, "value_dev is NULL");
    if (dtype != LSP_F32 && dtype != LSP_F64) return fail(LSP_EINVAL, "bad dtype");
    cudaStream_t st = (cudaStream_t)stream;
    double eps = 0.0, dV = 1.0;
    for (int k = 0; k < g->ndim; ++k) {
        eps = std::fmax(eps, g->dx[k]);
        dV *= g->dx[k];
    }
    cudaError_t e = cudaMemsetAsync(value_dev, 0, sizeof(double), st);
    if (!e && grad) e = cudaMemsetAsync(grad, 0, (size_t)g->npts * elem_size(dtype), st);
    if (e) return cuda_fail(e, "memset");
    auto fill = [&](auto& L) {
        L.nq = nq;
        L.ndim = g->ndim;
        L.npts = (int)g->npts;
        long long sd = 1;
        for (int k = g->ndim - 1; k >= 0; --k) {
            L.n[k] = g->n[k];
            L.stride[k] = (int)sd;
            sd *= g->n[k];
            L.periodic[k] = g->periodic[k];
            L.lo[k] = g->lo[k];
            L.h[k] = g->dx[k];
        }
        L.inv_eps = 1.0 / eps;
        L.dV = dV;
    };
    if (dtype == LSP_F64) {
        lsp::LossArgs<double> L;
        std::memset(&L, 0, sizeof(L));
        L.phi = (const double*)phi;
        L.queries = (const double*)queries;
        fill(L);
        e = lsp::launch_loss<double>(L, value_dev, (double*)grad, st);
    } else {
        lsp::LossArgs<float> L;
        std::memset(&L, 0, sizeof(L));
        L.phi = (const float*)phi;
        L.queries = (const float*)queries;
        fill(L);
        e = lsp::launch_loss<float>(L, value_dev, (float*)grad, st);
    }
    return e ? cuda_fail(e, "loss kernels") : LSP_OK;
}

}  // extern "C"

namespace {

// geometry and the shared checks of the shape primitives
lsp_status shape_prep(const lsp_grid* g, int dtype, const void* out, unsigned ignore,
                      lsp::ShapeGeom& geo)
{
    if (!g) return fail(LSP_EINVAL, "grid is NULL");
    if (dtype != LSP_F32 && dtype != LSP_F64) return fail(LSP_EINVAL, "bad dtype");
    if (!out) return fail(LSP_EINVAL, "out is NULL");
    unsigned used = 0;
    for (int k = 0; k < g->ndim; ++k)
        if (!((ignore >> k) & 1u)) used++;
    if (used == 0) return fail(LSP_EINVAL, "every dimension is ignored");
    geo.ndim = g->ndim;
    for (int k = 0; k < g->ndim; ++k) {
        geo.n[k] = g->n[k];
        geo.lo[k] = g->lo[k];
        geo.h[k] = g->dx[k];
    }
    geo.npts = g->npts;
    return LSP_OK;
}

lsp_status shape_run(const lsp::ShapeGeom& geo, const lsp::ShapeArgs& sa, int dtype,
                     void* out, void* stream)
{
    cudaError_t e = lsp::launch_shape(geo, sa, dtype, out, (cudaStream_t)stream);
    return e ? cuda_fail(e, "shape kernel") : LSP_OK;
}

}  // namespace

extern "C" {

lsp_status lsp_shape_sphere(const lsp_grid* g, int dtype, const double* center, double radius,
                            unsigned ignore, void* out, void* stream)
{
    lsp::ShapeGeom geo;
    lsp_status s = shape_prep(g, dtype, out, ignore, geo);
    if (s) return s;
    if (!center) return fail(LSP_EINVAL, "center is NULL");
    if (!(radius >= 0.0)) return fail(LSP_EINVAL, "radius must be >= 0");
    lsp::ShapeArgs sa{};
    sa.kind = lsp::SHAPE_SPHERE;
    sa.ignore = ignore;
    for (int k = 0; k < g->ndim; ++k) sa.c[k] = center[k];
    sa.r = radius;
    return shape_run(geo, sa, dtype, out, stream);
}

lsp_status lsp_shape_box(const lsp_grid* g, int dtype, const double* lo, const double* hi,
                         unsigned ignore, void* out, void* stream)
{
    lsp::ShapeGeom geo;
    lsp_status s = shape_prep(g, dtype, out, ignore, geo);
    if (s) return s;
    if (!lo || !hi) return fail(LSP_EINVAL, "lo and hi must not be NULL");
    lsp::ShapeArgs sa{};
    sa.kind = lsp::SHAPE_BOX;
    sa.ignore = ignore;
    for (int k = 0; k < g->ndim; ++k) {
        if (!((ignore >> k) & 1u) && !(lo[k] <= hi[k]))
            return fail(LSP_EINVAL, "box dimension %d has lo > hi", k);
        sa.c[k] = lo[k];
        sa.d[k] = hi[k];
    }
    return shape_run(geo, sa, dtype, out, stream);
}

lsp_status lsp_shape_quadric(const lsp_grid* g, int dtype, const double* center,
                             const double* weights, double offset, unsigned ignore, void* out,
                             void* stream)
{
    lsp::ShapeGeom geo;
    lsp_status s = shape_prep(g, dtype, out, ignore, geo);
    if (s) return s;
    if (!center || !weights) return fail(LSP_EINVAL, "center and weights must not be NULL");
    lsp::ShapeArgs sa{};
    sa.kind = lsp::SHAPE_QUADRIC;
    sa.ignore = ignore;
    for (int k = 0; k < g->ndim; ++k) {
        sa.c[k] = center[k];
        sa.d[k] = weights[k];
    }
    sa.r = offset;
    return shape_run(geo, sa, dtype, out, stream);
}

lsp_status lsp_shape_halfspace(const lsp_grid* g, int dtype, const double* normal,
                               const double* point, unsigned ignore, void* out, void* stream)
{
    lsp::ShapeGeom geo;
    lsp_status s = shape_prep(g, dtype, out, ignore, geo);
    if (s) return s;
    if (!normal || !point) return fail(LSP_EINVAL, "normal and point must not be NULL");
    lsp::ShapeArgs sa{};
    sa.kind = lsp::SHAPE_HALFSPACE;
    sa.ignore = ignore;
    double nn = 0.0;
    for (int k = 0; k < g->ndim; ++k) {
        sa.c[k] = point[k];
        sa.d[k] = normal[k];
        if (!((ignore >> k) & 1u)) nn += normal[k] * normal[k];
    }
    if (!(nn > 0.0)) return fail(LSP_EINVAL, "the normal is zero in the dimensions used");
    return shape_run(geo, sa, dtype, out, stream);
}

lsp_status lsp_shape_op(int op, int dtype, const void* a, const void* b, void* out, int64_t n,
                        void* stream)
{
    if (op < LSP_SHAPE_UNION || op > LSP_SHAPE_DIFFERENCE) return fail(LSP_EINVAL, "bad op");
    if (dtype != LSP_F32 && dtype != LSP_F64) return fail(LSP_EINVAL, "bad dtype");
    if (n < 0 || n >= (1LL << 31)) return fail(LSP_EINVAL, "n must be in [0, 2^31)");
    if (n > 0 && (!a || !out || (op != LSP_SHAPE_COMPLEMENT && !b)))
        return fail(LSP_EINVAL, "NULL field");
    cudaError_t e = lsp::launch_shape_op(op, dtype, a, b, out, (long long)n, (cudaStream_t)stream);
    return e ? cuda_fail(e, "shape op kernel") : LSP_OK;
}

lsp_status lsp_check_status(const void* ws, void* stream)
{
    if (!ws) return fail(LSP_EINVAL, "workspace is NULL");
    return read_flags(ws, (cudaStream_t)stream);
}

}  // extern "C"
