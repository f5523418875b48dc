// batched.cu -- many independent level-set problems of different shapes,
// dynamics and step sizes advanced together.
//
// Each problem keeps its own grid, CFL step and step count (the FP64 time
// loop of a single solve, per problem).  One launch advances stage s of step
// k of every problem that still has steps left: a table maps each CTA of the
// launch to (problem, tile), and each CTA runs the tiled stage body of
// stage_tiled.cuh on its problem's fields.  Problems are ordered by
// decreasing step count, so the problems active at step k are a prefix of the
// table and the launch is simply shortened as problems finish.  The whole
// sequence of launches can be captured into one CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/lsp.h"
#include "batched.h"
#include "launch.h"
#include "stage_tiled.cuh"

namespace lsp {

template <int SCHEME>
__global__ void __launch_bounds__(kBatchTB * kBatchTA, 3)
    stage_batched_kernel(const BatchProblem* __restrict__ probs, const int* __restrict__ block_prob,
                         int step, int stage, int rk)
{
    constexpr int G = ghost_width(SCHEME);
    __shared__ StageArgs<float> sa;
    __shared__ float tile[2 * (kBatchTA + 2 * G) * (kBatchTB + 2 * G)];
    const int p = block_prob[blockIdx.x];
    const BatchProblem& P = probs[p];
    const int tid = threadIdx.y * kBatchTB + threadIdx.x;
    if (tid == 0) {
        sa = P.a;
        const double dt = (step == P.nsteps - 1) ? P.dt_last : P.dt;
        sa.dt = float(dt);
        sa.dt_from_ctl = 0;
        sa.alpha_from_ctl = 0;
        // stage fields and coefficients of TVD-RK (Sec. V-A); the target only
        // in the last stage of a step
        sa.tube = 0;
        sa.phi_n = nullptr;
        if (stage == 0) {
            sa.phi_s = P.phi;
            sa.out = P.w1;
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
    __syncthreads();
    const int local = blockIdx.x - P.block_start;
    const int bx = local % P.nbx;
    const int by = (local / P.nbx) % P.nby;
    const int z = local / (P.nbx * P.nby);
    const int chunk = z % P.nchunks, outer = z / P.nchunks;
    const int tx = threadIdx.x, ty = threadIdx.y;
    switch (P.ndim * 8 + P.dyn) {
    case 2 * 8 + NORMAL_SPEED:
        tiled_stage_body<2, SCHEME, NORMAL_SPEED, float>(sa, kBatchTB, kBatchTA, bx, by, 0, 0, 1, tile, tx, ty);
        break;
    case 2 * 8 + TRANSLATE:
        tiled_stage_body<2, SCHEME, TRANSLATE, float>(sa, kBatchTB, kBatchTA, bx, by, 0, 0, 1, tile, tx, ty);
        break;
    case 3 * 8 + NORMAL_SPEED:
        tiled_stage_body<3, SCHEME, NORMAL_SPEED, float>(sa, kBatchTB, kBatchTA, bx, by, chunk, 0, P.ch, tile, tx, ty);
        break;
    case 3 * 8 + TRANSLATE:
        tiled_stage_body<3, SCHEME, TRANSLATE, float>(sa, kBatchTB, kBatchTA, bx, by, chunk, 0, P.ch, tile, tx, ty);
        break;
    case 3 * 8 + AIR3D:
        tiled_stage_body<3, SCHEME, AIR3D, float>(sa, kBatchTB, kBatchTA, bx, by, chunk, 0, P.ch, tile, tx, ty);
        break;
    case 4 * 8 + NORMAL_SPEED:
        tiled_stage_body<4, SCHEME, NORMAL_SPEED, float>(sa, kBatchTB, kBatchTA, bx, by, chunk, outer, P.ch, tile, tx, ty);
        break;
    case 4 * 8 + TRANSLATE:
        tiled_stage_body<4, SCHEME, TRANSLATE, float>(sa, kBatchTB, kBatchTA, bx, by, chunk, outer, P.ch, tile, tx, ty);
        break;
    case 4 * 8 + CAR4D:
        tiled_stage_body<4, SCHEME, CAR4D, float>(sa, kBatchTB, kBatchTA, bx, by, chunk, outer, P.ch, tile, tx, ty);
        break;
    default:
        break;  // rejected on the host
    }
}

cudaError_t launch_batched(int scheme, const BatchProblem* probs, const int* block_prob, int nblocks,
                           int step, int stage, int rk, cudaStream_t s)
{
    if (nblocks <= 0) return cudaSuccess;
    dim3 block(kBatchTB, kBatchTA, 1);
    switch (scheme) {
    case UPWIND1: stage_batched_kernel<UPWIND1><<<nblocks, block, 0, s>>>(probs, block_prob, step, stage, rk); break;
    case ENO2: stage_batched_kernel<ENO2><<<nblocks, block, 0, s>>>(probs, block_prob, step, stage, rk); break;
    case ENO3: stage_batched_kernel<ENO3><<<nblocks, block, 0, s>>>(probs, block_prob, step, stage, rk); break;
    case WENO5: stage_batched_kernel<WENO5><<<nblocks, block, 0, s>>>(probs, block_prob, step, stage, rk); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

void batch_tile_dims(int* tb, int* ta)
{
    *tb = kBatchTB;
    *ta = kBatchTA;
}

bool batch_supported(int ndim, int dyn)
{
    if (ndim == 2) return dyn == NORMAL_SPEED || dyn == TRANSLATE;
    if (ndim == 3) return dyn == NORMAL_SPEED || dyn == TRANSLATE || dyn == AIR3D;
    if (ndim == 4) return dyn == NORMAL_SPEED || dyn == TRANSLATE || dyn == CAR4D;
    return false;
}

}  // namespace lsp
