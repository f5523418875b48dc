// batched.cuh -- the kernels of the batched solve (see batched.cu), as
// templates over LOCAL (local dissipation coefficients and the variational
// clip compiled in or not); batched.cu instantiates LOCAL = false,
// batched_local.cu LOCAL = true.
#pragma once
#include "../../include/lsp.h"
#include "batched.h"
#include "launch.h"
#include "stage_pair.cuh"
#include "stage_tiled.cuh"

namespace lsp {

// Stage fields and TVD-RK coefficients (Sec. V-A) of stage `stage` of a
// problem's step; the target only in the last stage.
__device__ __forceinline__ void batch_stage_args(const BatchProblem& P, int step, int stage, int rk,
                                                 StageArgs<float>& sa)
{
    sa = P.a;
    sa.dt = float((step == P.nsteps - 1) ? P.dt_last : P.dt);
    sa.dt_from_ctl = 0;
    sa.alpha_from_ctl = 0;
    sa.tube = 0;
    sa.phi_n = nullptr;
    if (stage == 0) {
        sa.phi_s = P.phi; sa.out = P.w1;
        sa.c_n = 0.f; sa.c_s = 1.f; sa.c_l = 1.f;
    } else if (stage == 1 && rk == 2) {
        sa.phi_s = P.w1; sa.phi_n = P.phi; sa.out = P.phi;
        sa.c_n = 0.5f; sa.c_s = 0.5f; sa.c_l = 0.5f;
        sa.tube = P.a.tube;
    } else if (stage == 1) {
        sa.phi_s = P.w1; sa.phi_n = P.phi; sa.out = P.w2;
        sa.c_n = 0.75f; sa.c_s = 0.25f; sa.c_l = 0.25f;
    } else {
        sa.phi_s = P.w2; sa.phi_n = P.phi; sa.out = P.phi;
        sa.c_n = float(1.0 / 3.0); sa.c_s = float(2.0 / 3.0); sa.c_l = float(2.0 / 3.0);
        sa.tube = P.a.tube;
    }
    sa.target = P.target;
}

// The body of one tile of a 3-D / 4-D problem: the paired shared-face body
// for the WENO5 stage (as single-problem solves run it by default; its local
// variant for local coefficients or the clip, state-only bounds), the scalar
// body otherwise.
template <int NDIM, int SCHEME, int DYN, bool COH, bool LOCAL>
__device__ __forceinline__ void batch_body(const StageArgs<float>& sa, int TB, int TA, int bx,
                                           int by, int chunk, int outer, int ch, float* tile,
                                           int tx, int ty)
{
    if constexpr (SCHEME == WENO5 && (!LOCAL || DYN != QUADRATIC))
        tiled_pair_body<NDIM, DYN, true, COH, WENO5, LOCAL>(sa, TB, TA, bx, by, chunk, outer, ch,
                                                            tile, tx, ty);
    else
        tiled_stage_body<NDIM, SCHEME, DYN, float, COH, LOCAL>(sa, TB, TA, bx, by, chunk, outer,
                                                               ch, tile, tx, ty);
}

// Shared tile of a batched CTA: two double-buffered planes, four for the
// paired body (WENO5), of the largest tile shape.
template <int SCHEME, bool LOCAL>
__host__ __device__ constexpr int batch_tile_floats()
{
    return (SCHEME == WENO5 ? 4 : 2) * batch_max_tile(ghost_width(SCHEME));
}

// Problem classes a batched kernel is compiled for: every supported
// (dimension, dynamics) pair, or only 2-D normal speed and 3-D air3d (the
// mixed workload of reachability problems), so that the kernel's register
// allocation is that of those two bodies alone.
enum {
    kClsAll = kBatchClsAll,
    kClsNormal2Air3 = kBatchClsNormal2Air3,
    kClsNormal2Air3x16 = kBatchClsNormal2Air3x16  // the same, 16 x 16 tiles only
};
__host__ __device__ constexpr bool cls_has(int cls, int ndim, int dyn)
{
    return cls == kClsAll || (ndim == 2 && dyn == NORMAL_SPEED) || (ndim == 3 && dyn == AIR3D);
}

// One tile of shape TB x TA (compile-time: the bodies' index arithmetic
// folds the tile extents).
template <int SCHEME, bool COH, bool LOCAL, int CLS, int TB, int TA>
__device__ __forceinline__ void batch_tile_shape(const BatchProblem& P, const StageArgs<float>& sa,
                                                 int local, float* tile)
{
    const int bx = local % P.nbx;
    const int by = (local / P.nbx) % P.nby;
    const int z = local / (P.nbx * P.nby);
    const int chunk = z % P.nchunks, outer = z / P.nchunks;
    const int ty = threadIdx.x / TB, tx = threadIdx.x - ty * TB;
    switch (P.ndim * 8 + P.dyn) {
    case 2 * 8 + NORMAL_SPEED:
        if constexpr (cls_has(CLS, 2, NORMAL_SPEED))
            tiled_stage_body<2, SCHEME, NORMAL_SPEED, float, COH, LOCAL>(sa, TB, TA, bx, by, 0, 0, 1, tile, tx, ty);
        break;
    case 2 * 8 + TRANSLATE:
        if constexpr (cls_has(CLS, 2, TRANSLATE))
            tiled_stage_body<2, SCHEME, TRANSLATE, float, COH, LOCAL>(sa, TB, TA, bx, by, 0, 0, 1, tile, tx, ty);
        break;
    case 3 * 8 + NORMAL_SPEED:
        if constexpr (cls_has(CLS, 3, NORMAL_SPEED))
            batch_body<3, SCHEME, NORMAL_SPEED, COH, LOCAL>(sa, TB, TA, bx, by, chunk, 0, P.ch, tile, tx, ty);
        break;
    case 3 * 8 + TRANSLATE:
        if constexpr (cls_has(CLS, 3, TRANSLATE))
            batch_body<3, SCHEME, TRANSLATE, COH, LOCAL>(sa, TB, TA, bx, by, chunk, 0, P.ch, tile, tx, ty);
        break;
    case 3 * 8 + AIR3D:
        if constexpr (cls_has(CLS, 3, AIR3D))
            batch_body<3, SCHEME, AIR3D, COH, LOCAL>(sa, TB, TA, bx, by, chunk, 0, P.ch, tile, tx, ty);
        break;
    case 3 * 8 + ROCKETS:
        if constexpr (cls_has(CLS, 3, ROCKETS))
            batch_body<3, SCHEME, ROCKETS, COH, LOCAL>(sa, TB, TA, bx, by, chunk, 0, P.ch, tile, tx, ty);
        break;
    case 2 * 8 + DOUBLE_INT:
        if constexpr (cls_has(CLS, 2, DOUBLE_INT))
            tiled_stage_body<2, SCHEME, DOUBLE_INT, float, COH, LOCAL>(sa, TB, TA, bx, by, 0, 0, 1, tile, tx, ty);
        break;
    case 4 * 8 + NORMAL_SPEED:
        if constexpr (cls_has(CLS, 4, NORMAL_SPEED))
            batch_body<4, SCHEME, NORMAL_SPEED, COH, LOCAL>(sa, TB, TA, bx, by, chunk, outer, P.ch, tile, tx, ty);
        break;
    case 4 * 8 + TRANSLATE:
        if constexpr (cls_has(CLS, 4, TRANSLATE))
            batch_body<4, SCHEME, TRANSLATE, COH, LOCAL>(sa, TB, TA, bx, by, chunk, outer, P.ch, tile, tx, ty);
        break;
    case 4 * 8 + CAR4D:
        if constexpr (cls_has(CLS, 4, CAR4D))
            batch_body<4, SCHEME, CAR4D, COH, LOCAL>(sa, TB, TA, bx, by, chunk, outer, P.ch, tile, tx, ty);
        break;
    default:
        break;  // rejected on the host
    }
}

template <int SCHEME, bool COH, bool LOCAL, int CLS = kClsAll>
__device__ __forceinline__ void batch_tile(const BatchProblem& P, const StageArgs<float>& sa,
                                           int local, float* tile)
{
    static_assert(kBatchShapes[1][0] == 32 && kBatchShapes[2][0] == 64, "tile shapes");
    if constexpr (LOCAL || CLS == kClsNormal2Air3x16) {  // 16 x 16 tiles only (local
                                                          // coefficients / the clip: see the plan)
        batch_tile_shape<SCHEME, COH, LOCAL, CLS, 16, 16>(P, sa, local, tile);
        return;
    }
    if (P.tb == 32) batch_tile_shape<SCHEME, COH, LOCAL, CLS, 32, 8>(P, sa, local, tile);
    else if (P.tb == 64) batch_tile_shape<SCHEME, COH, LOCAL, CLS, 64, 4>(P, sa, local, tile);
    else batch_tile_shape<SCHEME, COH, LOCAL, CLS, 16, 16>(P, sa, local, tile);
}

// One RK stage of every active problem: CTA i runs tile i - block_start of
// problem block_prob[i].
template <int SCHEME, bool LOCAL, int CLS>
__global__ void __launch_bounds__(kBatchThreads, 3)
    stage_batched_kernel(const BatchProblem* __restrict__ probs, const int* __restrict__ block_prob,
                         int step, int stage, int rk)
{
    constexpr int G = ghost_width(SCHEME);
    __shared__ StageArgs<float> sa;
    __shared__ __align__(16) float tile[batch_tile_floats<SCHEME, LOCAL>()];
    const int p = block_prob[blockIdx.x];
    const BatchProblem& P = probs[p];
    const int tid = threadIdx.x;
    if (tid == 0) batch_stage_args(P, step, stage, rk, sa);
    __syncthreads();
    batch_tile<SCHEME, false, LOCAL, CLS>(P, sa, blockIdx.x - P.block_start, tile);
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// The whole batched solve in one launch.  Every CTA takes the next work item
// (k, s, b) from one counter; items go out in (step, stage, tile) order, so
// every item an item depends on -- all tiles of the previous stage of the
// same problem -- was handed out earlier to a CTA that is running (the launch
// is cooperative: all CTAs are resident).  A CTA waits for its dependency on
// the problem's completion counter; the wait is bounded by wait_ns, after
// which it raises kFlagTimeout, sets the abort flag (other waiters leave at
// once) and stops: the launch always ends.
template <int SCHEME, bool LOCAL, int CLS>
__global__ void __launch_bounds__(kBatchThreads, 3)
    stage_batched_persistent(const BatchProblem* __restrict__ probs,
                             const int* __restrict__ block_prob,
                             const BatchSegment* __restrict__ segs, int nseg, int rk,
                             unsigned int* done, PersistCtl* pc, Ctl* ctl,
                             unsigned long long wait_ns)
{
    constexpr int G = ghost_width(SCHEME);
    __shared__ StageArgs<float> sa;
    __shared__ __align__(16) float tile[batch_tile_floats<SCHEME, LOCAL>()];
    __shared__ int s_p, s_local, s_stop;
    const int tid = threadIdx.x;
    const long long total = segs[nseg].item_start;
    for (;;) {
        if (tid == 0) {
            int stop = 0;
            const long long it = (long long)atomicAdd(&pc->next, 1ULL);
            if (it >= total || *(volatile unsigned*)&pc->abort) {
                stop = 1;
            } else {
                int lo = 0, hi = nseg;  // segs[lo].item_start <= it < segs[hi].item_start
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (segs[mid].item_start <= it) lo = mid;
                    else hi = mid;
                }
                const BatchSegment sg = segs[lo];
                const long long off = it - sg.item_start;
                const long long per_step = (long long)rk * sg.blocks;
                const int k = sg.k_start + (int)(off / per_step);
                const int r = (int)(off % per_step);
                const int stage = r / sg.blocks, b = r % sg.blocks;
                const int p = block_prob[b];
                const BatchProblem& P = probs[p];
                const unsigned target = (unsigned)(k * rk + stage) * (unsigned)P.nblocks;
                const unsigned long long t0 = global_ns();
                while (*(volatile unsigned*)(done + p) < target) {
                    if (*(volatile unsigned*)&pc->abort) {
                        stop = 1;
                        break;
                    }
                    if (global_ns() - t0 > wait_ns) {
                        atomicOr(&ctl->flags, kFlagTimeout);
                        atomicExch(&pc->abort, 1u);
                        stop = 1;
                        break;
                    }
                    __nanosleep(256);
                }
                __threadfence();  // acquire: the producers' stores are visible
                if (!stop) {
                    batch_stage_args(P, k, stage, rk, sa);
                    s_p = p;
                    s_local = b - P.block_start;
                }
            }
            s_stop = stop;
        }
        __syncthreads();
        if (s_stop) break;
        batch_tile<SCHEME, true, LOCAL, CLS>(probs[s_p], sa, s_local, tile);
        __syncthreads();
        if (tid == 0) {
            __threadfence();  // release this tile's stores before counting it done
            if (s_p != pc->stall_problem) atomicAdd(done + s_p, 1u);
        }
    }
}

// The launches of one (scheme, local, class set) instantiation.  They are
// instantiated explicitly in separate translation units (batched_*.cu) so
// that the kernels compile in parallel; batched.cu dispatches to them.
template <int SCHEME, bool LOCAL, int CLS>
cudaError_t launch_batched_k(const BatchProblem* probs, const int* block_prob, int nblocks,
                             int step, int stage, int rk, cudaStream_t s)
{
    if (nblocks <= 0) return cudaSuccess;
    stage_batched_kernel<SCHEME, LOCAL, CLS><<<nblocks, dim3(kBatchThreads, 1, 1), 0, s>>>(
        probs, block_prob, step, stage, rk);
    return cudaGetLastError();
}

template <int SCHEME, bool LOCAL, int CLS>
cudaError_t launch_persistent_k(const BatchProblem* probs, const int* block_prob,
                                const BatchSegment* segs, int nseg, int rk, unsigned int* done,
                                PersistCtl* pc, Ctl* ctl, unsigned long long wait_ns,
                                cudaStream_t s)
{
    const void* fn = (const void*)stage_batched_persistent<SCHEME, LOCAL, CLS>;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBatchThreads, 0);
    if (e) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    dim3 grid(sm_count() * per_sm), block(kBatchThreads, 1, 1);
    void* args[] = {(void*)&probs, (void*)&block_prob, (void*)&segs, (void*)&nseg, (void*)&rk,
                    (void*)&done, (void*)&pc, (void*)&ctl, (void*)&wait_ns};
    return cudaLaunchCooperativeKernel(fn, grid, block, args, 0, s);
}

#define LSP_BATCHED_INSTANTIATE_STAGE(SCHEME, LOCAL, CLS)                                         \
    template cudaError_t launch_batched_k<SCHEME, LOCAL, CLS>(                                    \
        const BatchProblem*, const int*, int, int, int, int, cudaStream_t);
#define LSP_BATCHED_INSTANTIATE_PERSISTENT(SCHEME, LOCAL, CLS)                                    \
    template cudaError_t launch_persistent_k<SCHEME, LOCAL, CLS>(                                 \
        const BatchProblem*, const int*, const BatchSegment*, int, int, unsigned int*,           \
        PersistCtl*, Ctl*, unsigned long long, cudaStream_t);
#define LSP_BATCHED_INSTANTIATE(SCHEME, LOCAL, CLS)                                               \
    LSP_BATCHED_INSTANTIATE_STAGE(SCHEME, LOCAL, CLS)                                             \
    LSP_BATCHED_INSTANTIATE_PERSISTENT(SCHEME, LOCAL, CLS)

}  // namespace lsp
