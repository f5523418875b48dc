// launch.h -- host-side entry points of the kernels (defined in the
// per-precision translation units).
#pragma once
#include "lsp_internal.h"

namespace lsp {

struct GridGeom;

// Fused stage (generic one-thread-per-node kernel).
template <typename R>
cudaError_t launch_stage(int ndim, int scheme, int dyn, const StageArgs<R>& a, cudaStream_t s);

// Costate range reduction for H = |p|^2/2 (alpha from the current field).
template <typename R>
cudaError_t launch_prange(int ndim, int scheme, const StageArgs<R>& a, cudaStream_t s);

// State-only global-LF coefficients (FP64).
cudaError_t launch_alpha_state(int dyn, const GridGeom& g, unsigned long long* out, cudaStream_t s);

struct Tile;

// Tiled fused stage for 3-D and 4-D FP32 grids (stage_tiled.cuh); one
// instantiation set per occupancy target MINB (stage_tiled_m*.cu).
template <int MINB>
cudaError_t launch_stage_tiled_m(int ndim, int scheme, int dyn, const StageArgs<float>& a,
                                 const Tile& t, cudaStream_t s);
cudaError_t launch_stage_tiled(int ndim, int scheme, int dyn, const StageArgs<float>& a,
                               const Tile& t, cudaStream_t s);
bool tile_valid(int ndim, int scheme, const Tile& t, const int* n);
// Face-shared ENO2/ENO3 kernel with R-node runs per thread (stage_run.cuh):
// Tile.pair = 3 runs of 4 (stage_run_r4.cu), 4 runs of 2 (stage_run_r2.cu);
// tb = nodes of the fastest axis per CTA (16, 28 or 32).
constexpr size_t kRunMaxSmem = 200 * 1024;  // dynamic shared memory of a launch
template <int R>
cudaError_t launch_stage_run_r(int ndim, int scheme, int dyn, const StageArgs<float>& a,
                               const Tile& t, cudaStream_t s);
bool run_tile_ok(int ndim, int scheme, int run, int tb, int ta);
// The two stages of a TVD-RK2 step in one launch (stage_fused.cuh, Tile.pair
// = 5): 3-D FP32 grids, GLF with state-only bounds; a.phi_s = phi^n, a.out =
// phi^{n+1} (a different field), a.dt the step.
cudaError_t launch_stage_fused_rk2(int scheme, int dyn, const StageArgs<float>& a, const Tile& t,
                                   cudaStream_t s);
bool fused_tile_ok(int ndim, int scheme, const Tile& t, const int* n);
// The same stage with local coefficients / the variational clip compiled in
// (stage_tiled_local.cu); launch_stage_tiled routes there when a asks for them.
cudaError_t launch_stage_tiled_local(int ndim, int scheme, int dyn, const StageArgs<float>& a,
                                     const Tile& t, cudaStream_t s);

// Batched stages (batched.cu): RK2/RK3, FP32, problems of 2 to 4 dimensions.
struct BatchProblem;
struct BatchSegment;
struct PersistCtl;
// local: the problems use local dissipation coefficients or the variational
// clip (batched_local.cu's instantiation).  cls: the class set the kernel is
// compiled for (kBatchClsNormal2Air3: every problem is 2-D normal speed or
// 3-D air3d; kBatchClsAll otherwise; local kernels cover every class).
// kBatchClsNormal2Air3x16: the same two classes, every tile 16 x 16.
enum { kBatchClsAll = 0, kBatchClsNormal2Air3 = 1, kBatchClsNormal2Air3x16 = 2 };
cudaError_t launch_batched(int scheme, const BatchProblem* probs, const int* block_prob, int nblocks,
                           int step, int stage, int rk, bool local, int cls, cudaStream_t s);
// The whole batched solve as one cooperative launch of resident CTAs.
cudaError_t launch_batched_persistent(int scheme, const BatchProblem* probs, const int* block_prob,
                                      const BatchSegment* segs, int nseg, int rk,
                                      unsigned int* done, PersistCtl* pc, Ctl* ctl,
                                      unsigned long long wait_ns, bool local, int cls,
                                      cudaStream_t s);
// Tile shape `shape` (0: 16 x 16, 1: 32 x 8, 2: 64 x 4) of batched problems;
// false for other values.
bool batch_tile_dims(int shape, int* tb, int* ta);
bool batch_supported(int ndim, int dyn);

// Implicit-surface primitives and set operations (shapes.cu).
struct ShapeGeom {
    int ndim;
    int n[LSP_MAXD];
    double lo[LSP_MAXD];
    double h[LSP_MAXD];
    long long npts;
};
enum { SHAPE_SPHERE = 0, SHAPE_BOX = 1, SHAPE_QUADRIC = 2, SHAPE_HALFSPACE = 3 };
struct ShapeArgs {
    int kind;
    unsigned ignore;     // bit k set: dimension k is ignored
    double c[LSP_MAXD];  // centre / box lower corner / quadric centre / plane point
    double d[LSP_MAXD];  // box upper corner / quadric weights / plane normal
    double r;            // radius / quadric offset
};
cudaError_t launch_shape(const ShapeGeom& g, const ShapeArgs& s, int dtype, void* out,
                         cudaStream_t st);
cudaError_t launch_shape_op(int op, int dtype, const void* a, const void* b, void* out,
                            long long n, cudaStream_t st);

// Adjoint of one stage (adjoint.cuh): pass A (with the previous stage's
// pass B when a.gcontrib is set) when pass_b is false, pass B alone when it
// is true.
template <typename R> struct AdjArgs;
template <typename R>
cudaError_t launch_adjoint_stage(int ndim, int scheme, int dyn, const AdjArgs<R>& a,
                                 bool pass_b, cudaStream_t s);
cudaError_t launch_alpha_argmax(int dyn, const GridGeom& g, const double* alpha,
                                unsigned long long* out, cudaStream_t s);

// Loss of the differentiation workload (value accumulated into *value).
template <typename R>
struct LossArgs {
    const R* phi;
    const R* queries;
    int nq, ndim, npts;
    int n[LSP_MAXD], stride[LSP_MAXD], periodic[LSP_MAXD];
    double lo[LSP_MAXD], h[LSP_MAXD];
    double inv_eps, dV;
};
template <typename R>
cudaError_t launch_loss(const LossArgs<R>& L, double* value, R* grad, cudaStream_t s);

// Is there a kernel for this combination?
bool stage_supported(int ndim, int scheme, int dyn);

}  // namespace lsp
