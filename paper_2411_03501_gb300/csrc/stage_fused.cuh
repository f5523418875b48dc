// stage_fused.cuh -- temporal blocking of the two stages of a TVD-RK2 step
// (Sec. V-A) in one kernel, for 3-D FP32 grids with state-only dissipation
// bounds.
//
// Unfused, a step is two launches: W1 = phi + dt L(phi) (written to HBM or
// L2), then phi' = phi/2 + (W1 + dt L(W1))/2 [min target].  Here one CTA
// owns a TA x TB tile of the two fastest axes (A, B) and marches along the
// third (S) over a chunk of planes, carrying both stages:
//  - phi planes, with a 2G-cell halo in A and B (ghost values substituted
//    while loading), sit in a ring of 2G+2 shared-memory planes;
//  - the first stage is evaluated on the tile plus a G-cell halo in A and B
//    and on G extra planes at each end of the chunk (what the second stage's
//    stencils read), into a ring of 2G+1 shared-memory W1 planes; W1's own
//    ghost cells (Sec. III-B) are formed from the computed W1 values after
//    the plane is complete: periodic positions are computed at their wrapped
//    node, extrapolated ones are filled from the two nodes next to the edge;
//  - the second stage is evaluated on the tile, reading W1 from shared
//    memory only, and written to `out` (a field other than phi: the halo of
//    phi is read by neighbouring CTAs while this one writes).
// Every value is computed by the same operations as the stage kernels
// (stage_tiled.cuh) on the same operands, so the result equals two launches
// of the scalar tiled body.  The price is the first stage on the halo:
// (TA+2G)(TB+2G)(CH+2G) / (TA TB CH) evaluations per node instead of one.
#pragma once
#include "stage_tiled.cuh"

namespace lsp {

// The LF rate L = -Hhat at one node of a 3-D grid from its three windows
// (axis order S, A, B as in the stage kernels; GLF coefficients).
template <int SCHEME, int DYN>
__device__ __forceinline__ float fused_rate(const float* uS, const float* uA, const float* uB,
                                            const StageArgs<float>& a, const float* x, float sth,
                                            float cth)
{
    float pm, pp, pbar[3], diss = 0.0f;
    deriv_fast<SCHEME>(uS, a.inv_dx[0], weno_floor12(a.inv_dx[0]), pm, pp);
    pbar[0] = 0.5f * (pp + pm);
    diss = rfma(a.alpha[0] * 0.5f, pp - pm, diss);
    deriv_fast<SCHEME>(uA, a.inv_dx[1], weno_floor12(a.inv_dx[1]), pm, pp);
    pbar[1] = 0.5f * (pp + pm);
    diss = rfma(a.alpha[1] * 0.5f, pp - pm, diss);
    deriv_fast<SCHEME>(uB, a.inv_dx[2], weno_floor12(a.inv_dx[2]), pm, pp);
    pbar[2] = 0.5f * (pp + pm);
    diss = rfma(a.alpha[2] * 0.5f, pp - pm, diss);
    const float Hv = hamiltonian_sc<DYN, 3>(x, pbar, a.prm, sth, cth);
    return -(Hv - diss);
}

// Linear extrapolation of a line's ghost value j (j < 0 from nodes 0, 1;
// j >= n from nodes n-1, n-2): the expression line_value uses.
__device__ __forceinline__ float extrap_ghost(float u0, float u1, int k)
{
    return u0 + float(k) * (u0 - u1);
}

// Shared memory (floats) of a fused launch.
__host__ __device__ constexpr int fused_smem_floats(int G, int tb, int ta)
{
    return (2 * G + 2) * (tb + 4 * G) * (ta + 4 * G) + (2 * G + 1) * (tb + 2 * G) * (ta + 2 * G);
}

// Slots per thread: phi tile (with 2G halo) and W1 tile (with G halo).
constexpr int kFusedMaxP = 4;
constexpr int kFusedMaxW = 3;

// blockDim = (TB, TA); gridDim = (ceil(nB/TB), ceil(nA/TA), nchunks).
// a.phi_s = phi^n, a.out = phi^{n+1} (distinct fields), a.target read when
// a.tube, a.dt the step; alpha from a.alpha (state-only bounds).
template <int SCHEME, int DYN>
__global__ void __launch_bounds__(256, 2) stage_fused_rk2_kernel(StageArgs<float> a, int ch)
{
    constexpr int G = ghost_width(SCHEME);
    constexpr int NPR = 2 * G + 2, NWR = 2 * G + 1;
    extern __shared__ float fsm[];
    const int TB = blockDim.x, TA = blockDim.y;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TB + tx, nthr = TB * TA;
    const int PW = TB + 4 * G, PH = TA + 4 * G, PSZ = PW * PH;
    const int WW = TB + 2 * G, WH = TA + 2 * G, WSZ = WW * WH;
    float* pring = fsm;
    float* wring = fsm + NPR * PSZ;
    const int nS = a.n[0], nA = a.n[1], nB = a.n[2];
    const int sS = a.stride[0], sA = a.stride[1];
    const int perS = a.periodic[0], perA = a.periodic[1], perB = a.periodic[2];
    const int b0 = blockIdx.x * TB, a0 = blockIdx.y * TA;
    const int s0 = blockIdx.z * ch, s1 = min(s0 + ch, nS);
    // last node of the tile along A and B (partial tiles) and the reach of
    // the stencils beyond it
    const int aEnd = min(a0 + TA, nA) - 1, bEnd = min(b0 + TB, nB) - 1;
    const float dtf = a.dt;

    // distance of a tile position outside the tile's own nodes along A / B
    auto dist = [](int j, int lo, int hi) { return j < lo ? lo - j : (j > hi ? j - hi : 0); };
    // one period suffices: positions lie within 2G <= 6 nodes of the grid and
    // every axis has at least 7 nodes
    auto wrap = [](int j, int n) { return j < 0 ? j + n : (j >= n ? j - n : j); };

    // ---- phi tile slots (the node after the wrap of periodic axes): kinds
    // 0 in the grid, 1 extrapolated ghost along B, 2 along A, 3 not read.
    // The first stage runs on the tile and its G-wide bands along A and B,
    // so it reads phi on the tile, bands 2G wide and G x G corners.
    int pja[kFusedMaxP], pjb[kFusedMaxP];
    unsigned pkinds = 0;
#pragma unroll
    for (int k = 0; k < kFusedMaxP; ++k) {
        const int e = tid + k * nthr;
        const int r = e / PW, c = e - r * PW;
        int ja = a0 - 2 * G + r, jb = b0 - 2 * G + c;
        const int dA = dist(ja, a0, aEnd), dB = dist(jb, b0, bEnd);
        const bool read = e < PSZ && ((dA == 0 && dB <= 2 * G) || (dB == 0 && dA <= 2 * G) ||
                                      (dA <= G && dB <= G));
        if (perA) ja = wrap(ja, nA);
        if (perB) jb = wrap(jb, nB);
        const bool inA = ja >= 0 && ja < nA, inB = jb >= 0 && jb < nB;
        const unsigned kind = !read ? 3u : (inA && inB) ? 0u : inA ? 1u : inB ? 2u : 3u;
        pkinds |= kind << (2 * k);
        pja[k] = ja;
        pjb[k] = jb;
    }
    // phi plane p (ghost planes of S substituted) into this thread's slots
    auto fetch = [&](int p, float* pf) {
        bool sghost = p < 0 || p >= nS;
        int ps = p;
        if (sghost && perS) {
            ps = wrap(p, nS);
            sghost = false;
        }
#pragma unroll
        for (int k = 0; k < kFusedMaxP; ++k) {
            const unsigned kind = (pkinds >> (2 * k)) & 3u;
            float v = 0.0f;
            if (!sghost) {
                const float* plane = a.phi_s + (size_t)ps * sS;
                if (kind == 0u) v = __ldg(plane + pja[k] * sA + pjb[k]);
                else if (kind == 1u) v = line_value<float>(plane + pja[k] * sA, pjb[k], nB, 1, 0);
                else if (kind == 2u) v = line_value<float>(plane + pjb[k], pja[k], nA, sA, 0);
            } else if (kind == 0u) {  // extrapolated S: only in-grid (A, B) columns are read
                v = line_value<float>(a.phi_s + pja[k] * sA + pjb[k], p, nS, sS, 0);
            }
            pf[k] = v;
        }
    };

    // ---- W1 tile slots: the tile and its G-wide bands along A and B (what
    // the second stage reads).  Kinds 0 computed (periodic positions at
    // their wrapped node), 1 extrapolated ghost along A, 2 along B, 3 unused
    int wpc[kFusedMaxW];  // phi-tile offset of the slot's node
    int wja[kFusedMaxW], wjb[kFusedMaxW];
    float wxa[kFusedMaxW], wxb[kFusedMaxW], wsn[kFusedMaxW], wcs[kFusedMaxW];
    unsigned wkinds = 0;
#pragma unroll
    for (int k = 0; k < kFusedMaxW; ++k) {
        const int e = tid + k * nthr;
        const int r = e / WW, c = e - r * WW;
        int ja = a0 - G + r, jb = b0 - G + c;
        const int dA = dist(ja, a0, aEnd), dB = dist(jb, b0, bEnd);
        const bool read = e < WSZ && ((dA == 0 && dB <= G) || (dB == 0 && dA <= G));
        if (perA) ja = wrap(ja, nA);
        if (perB) jb = wrap(jb, nB);
        const bool inA = ja >= 0 && ja < nA, inB = jb >= 0 && jb < nB;
        const unsigned kind = !read ? 3u : (inA && inB) ? 0u : inB ? 1u : inA ? 2u : 3u;
        wkinds |= kind << (2 * k);
        wja[k] = ja;
        wjb[k] = jb;
        wpc[k] = (r + G) * PW + c + G;
        wxa[k] = rfma(float(ja), a.h[1], a.lo[1]);
        wxb[k] = rfma(float(jb), a.h[2], a.lo[2]);
        wsn[k] = 0.0f;
        wcs[k] = 1.0f;
        if constexpr (DYN == AIR3D || DYN == ROCKETS)
            if (kind == 0u) rsincos(wxb[k], &wsn[k], &wcs[k]);
    }
    // block-uniform: W1 has extrapolated ghost cells inside this tile
    const bool fillA = !perA && (a0 - G < 0 || aEnd + G >= nA);
    const bool fillB = !perB && (b0 - G < 0 || bEnd + G >= nB);

    // ---- this thread's output node
    const int ia = a0 + ty, ib = b0 + tx;
    const bool active = ia < nA && ib < nB;
    float ox[3];
    ox[1] = rfma(float(ia), a.h[1], a.lo[1]);
    ox[2] = rfma(float(ib), a.h[2], a.lo[2]);
    float osn = 0.0f, ocs = 1.0f;
    if constexpr (DYN == AIR3D || DYN == ROCKETS) rsincos(ox[2], &osn, &ocs);

    auto pslot = [&](int p) { return ((p + 4 * NPR) % NPR) * PSZ; };
    auto wslot = [&](int q) { return ((q + 4 * NWR) % NWR) * WSZ; };
    bool nonfinite = false;

    // prologue: phi planes s0-2G .. s0-1 staged, plane s0 in registers
    float pf[kFusedMaxP];
    for (int p = s0 - 2 * G; p < s0; ++p) {
        fetch(p, pf);
        float* dst = pring + pslot(p);
#pragma unroll
        for (int k = 0; k < kFusedMaxP; ++k)
            if (((pkinds >> (2 * k)) & 3u) != 3u) dst[tid + k * nthr] = pf[k];
    }
    fetch(s0, pf);

    for (int t = s0 - G; t < s1 + G; ++t) {
        {  // phi plane t+G into the ring (its slot was last read two barriers ago)
            float* dst = pring + pslot(t + G);
#pragma unroll
            for (int k = 0; k < kFusedMaxP; ++k)
                if (((pkinds >> (2 * k)) & 3u) != 3u) dst[tid + k * nthr] = pf[k];
        }
        __syncthreads();
        if (t + G + 1 < s1 + 2 * G) fetch(t + G + 1, pf);

        // first stage on W1 plane t
        const bool computed = perS || (t >= 0 && t < nS);
        float* wt = wring + wslot(t);
        if (computed) {
            const int ts = t < 0 ? t + nS : (t >= nS ? t - nS : t);
            float x[3];
            x[0] = rfma(float(ts), a.h[0], a.lo[0]);
            const float* pt = pring + pslot(t);
#pragma unroll
            for (int k = 0; k < kFusedMaxW; ++k) {
                if (((wkinds >> (2 * k)) & 3u) != 0u) continue;
                const int pc = wpc[k];
                float uS[2 * G + 1], uA[2 * G + 1], uB[2 * G + 1];
#pragma unroll
                for (int o = -G; o <= G; ++o) {
                    uS[o + G] = pring[pslot(t + o) + pc];
                    uA[o + G] = pt[pc + o * PW];
                    uB[o + G] = pt[pc + o];
                }
                x[1] = wxa[k];
                x[2] = wxb[k];
                const float L = fused_rate<SCHEME, DYN>(uS, uA, uB, a, x, wsn[k], wcs[k]);
                const float v = rfma(dtf, L, uS[G]);
                nonfinite |= !isfinite(v);
                wt[tid + k * nthr] = v;
            }
            if (fillA || fillB) {  // W1's extrapolated ghost cells of this plane
                __syncthreads();
#pragma unroll
                for (int k = 0; k < kFusedMaxW; ++k) {
                    const unsigned kind = (wkinds >> (2 * k)) & 3u;
                    const int e = tid + k * nthr;
                    if (kind == 1u) {
                        const int c = e - (e / WW) * WW, j = wja[k];
                        const int r0 = (j < 0 ? 0 : nA - 1) - (a0 - G);
                        const int r1 = (j < 0 ? 1 : nA - 2) - (a0 - G);
                        wt[e] = extrap_ghost(wt[r0 * WW + c], wt[r1 * WW + c],
                                             j < 0 ? -j : j - nA + 1);
                    } else if (kind == 2u) {
                        const int rb = (e / WW) * WW, j = wjb[k];
                        const int c0 = (j < 0 ? 0 : nB - 1) - (b0 - G);
                        const int c1 = (j < 0 ? 1 : nB - 2) - (b0 - G);
                        wt[e] = extrap_ghost(wt[rb + c0], wt[rb + c1], j < 0 ? -j : j - nB + 1);
                    }
                }
            }
        } else if (t >= nS) {  // extrapolated S, ghost plane above the grid
            const float* un = wring + wslot(nS - 1);
            const float* um = wring + wslot(nS - 2);
#pragma unroll
            for (int k = 0; k < kFusedMaxW; ++k) {
                const int e = tid + k * nthr;
                if (e < WSZ) wt[e] = extrap_ghost(un[e], um[e], t - nS + 1);
            }
        }
        if (!perS && t == 1 && s0 - G < 0) {  // ghost planes below the grid from planes 0, 1
            __syncthreads();
            const float* u0 = wring + wslot(0);
            const float* u1 = wring + wslot(1);
            for (int q = -G; q < 0; ++q) {
                float* wq = wring + wslot(q);
#pragma unroll
                for (int k = 0; k < kFusedMaxW; ++k) {
                    const int e = tid + k * nthr;
                    if (e < WSZ) wq[e] = extrap_ghost(u0[e], u1[e], -q);
                }
            }
        }
        __syncthreads();

        // second stage on output plane s = t - G
        const int s = t - G;
        if (s >= s0 && active) {
            const int wc = (ty + G) * WW + tx + G;
            const float* ws = wring + wslot(s);
            float uS[2 * G + 1], uA[2 * G + 1], uB[2 * G + 1];
#pragma unroll
            for (int o = -G; o <= G; ++o) {
                uS[o + G] = wring[wslot(s + o) + wc];
                uA[o + G] = ws[wc + o * WW];
                uB[o + G] = ws[wc + o];
            }
            ox[0] = rfma(float(s), a.h[0], a.lo[0]);
            const float L = fused_rate<SCHEME, DYN>(uS, uA, uB, a, ox, osn, ocs);
            const float phin = pring[pslot(s) + (ty + 2 * G) * PW + tx + 2 * G];
            float v = rfma(0.5f * dtf, L, 0.5f * uS[G]);
            v = rfma(0.5f, phin, v);
            const size_t idx = (size_t)s * sS + ia * sA + ib;
            if (a.tube) v = rmin(v, __ldg(a.target + idx));
            nonfinite |= !isfinite(v);
            a.out[idx] = v;
        }
    }
    if (nonfinite) atomicOr(&a.ctl->flags, kFlagNonFinite);
}

}  // namespace lsp
