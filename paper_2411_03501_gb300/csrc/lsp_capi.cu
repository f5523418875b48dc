// lsp_capi.cu -- the C ABI of include/lsp.h: argument checking, workspace
// layout, the FP64 time loop and the enqueueing of the stage kernels.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "../../include/lsp.h"
#include "launch.h"
#include "stage_generic.cuh"

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
    for (int i = 0; i < 6; ++i)
        if (o->reserved[i]) return fail(LSP_EINVAL, "reserved option fields must be zero");
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
    cudaError_t e;
    if (!g->alpha_state) {  // alpha from the costate range of phi_s
        e = cudaMemsetAsync(ctl->alpha_bits, 0, sizeof(ctl->alpha_bits), st);
        if (e != cudaSuccess) return cuda_fail(e, "memset alpha");
        e = lsp::launch_prange<R>(g->ndim, o->scheme, a, st);
        if (e != cudaSuccess) return cuda_fail(e, "costate range kernel");
    }
    e = lsp::launch_stage<R>(g->ndim, o->scheme, g->dyn, a, st);
    if (e != cudaSuccess) return cuda_fail(e, "stage kernel");
    return LSP_OK;
}

// One TVD-RK step of size dt, phi in place (Sec. V-A), tube in the last stage.
template <typename R>
lsp_status enqueue_step(const lsp_grid* g, const lsp_solve_opts* o, R* phi, const R* target,
                        double dt, void* ws, cudaStream_t st)
{
    lsp::Ctl* ctl = (lsp::Ctl*)ws;
    R* w1 = (R*)((char*)ws + lsp::kCtlBytes);
    R* w2 = (R*)((char*)w1 + round256((size_t)g->npts * sizeof(R)));
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

lsp_status step_any(const lsp_grid* g, const lsp_solve_opts* o, void* phi, const void* target,
                    double dt, void* ws, cudaStream_t st)
{
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
    if ((s = step_any(g, o, phi, target, dt, ws, st))) return s;
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
    while (!s && t < t_stop) {
        const double dt = cfl_dt_host(g, o->cfl, t, t_final);
        if (!(dt > 0.0)) {
            s = fail(LSP_EINVAL, "non-positive CFL step");
            break;
        }
        s = step_any(g, o, phi, target, dt, ws, es);
        t += dt;
        sts.steps++;
        sts.dt_min = std::fmin(sts.dt_min, dt);
        sts.dt_max = std::fmax(sts.dt_max, dt);
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

lsp_status lsp_check_status(const void* ws, void* stream)
{
    if (!ws) return fail(LSP_EINVAL, "workspace is NULL");
    return read_flags(ws, (cudaStream_t)stream);
}

}  // extern "C"
