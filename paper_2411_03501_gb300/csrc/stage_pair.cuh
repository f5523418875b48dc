// stage_pair.cuh -- the tiled stage body (WENO5, ENO2, ENO3) evaluating two
// consecutive planes of the march per iteration with paired FP32
// instructions.
//
// Same computation as tiled_stage_body<.., SCHEME, .., float>
// (stage_tiled.cuh); each thread carries the nodes (s, ia, ib) and
// (s+1, ia, ib) together in F2 values, so every add/mul/fma of the
// derivatives, the Hamiltonian and the combination is issued once for both
// (the ENO stencil choices are made per node, on the same differences as the
// scalar body).  Each axis' central costate and dissipation are formed from
// the scheme's parts (axis_pair) rather than from the rounded one-sided
// derivatives, so the two bodies agree to rounding, not bit for bit.  The
// plane tiles of s and s+1 are staged interleaved (a float2 per node, one
// 64-bit shared access for both planes), double-buffered; the marching
// window holds 2G+2 values.
#pragma once
#include "pair2.cuh"
#include "stage_tiled.cuh"

namespace lsp {

// phi^n may be written by the same launch when COH (persistent batched
// solve, after the CTA's acquire): a weak load cached at every level then, a
// plain one otherwise.
template <bool COH>
__device__ __forceinline__ float ld_phin(const float* p)
{
    if constexpr (COH) return __ldca(p);
    else return *p;
}

template <int DYN, int NDIM>
__device__ __forceinline__ F2 hamiltonian_pair(const F2* x, const F2* p, const float* prm, float s,
                                               float c)
{
    if constexpr (DYN == NORMAL_SPEED) {
        F2 n2 = p[0] * p[0];
#pragma unroll
        for (int k = 1; k < NDIM; ++k) n2 = fma2(p[k], p[k], n2);
        return F2(prm[0]) * sqrt2(n2);
    } else if constexpr (DYN == TRANSLATE) {
        F2 h = F2(prm[0]) * p[0];
#pragma unroll
        for (int k = 1; k < NDIM; ++k) h = fma2(F2(prm[k]), p[k], h);
        return h;
    } else if constexpr (DYN == AIR3D) {
        const float ve = prm[0], vp = prm[1], um = prm[2], dm = prm[3];
        const F2 sw = p[0] * x[1] - p[1] * x[0] - p[2];
        const F2 v = p[0] * F2(fmaf(vp, c, -ve)) + p[1] * F2(vp * s) + F2(um) * abs2(sw) -
                     F2(dm) * abs2(p[2]);
        return -v;
    } else if constexpr (DYN == CAR4D) {
        const F2 m = p[0] * x[3] * F2(c) + p[1] * x[3] * F2(s) - F2(prm[0]) * abs2(p[2]) -
                     F2(prm[1]) * abs2(p[3]);
        return -m;
    } else if constexpr (DYN == ROCKETS) {  // hamiltonian_rockets for two nodes
        const float a = prm[0], ue = prm[2], up = prm[3];
        const F2 fx(a * c), fz(fmaf(a, s, a - prm[1]));
        F2 v = fma2(p[0], fx, p[1] * fz);
        v = fma2(F2(ue), abs2(fma2(p[0], x[0], -p[2])), v);
        v = fma2(F2(-up), abs2(fma2(p[1], x[0], p[2])), v);
        return -v;
    } else {
        static_assert(DYN == QUADRATIC, "no paired Hamiltonian for these dynamics");
        F2 n2 = p[0] * p[0];
#pragma unroll
        for (int k = 1; k < NDIM; ++k) n2 = fma2(p[k], p[k], n2);
        return F2(0.5f) * n2;
    }
}

// One axis of the paired LF rate from the window u[0..2G] of both nodes:
// adds the axis' central costate to pbar and its dissipation to diss, with
// hax = alpha / (2 dx) per node.  WENO5 delivers both multiplied by 6
// (lf_axis2); ENO2/ENO3 as they are: pbar = (p+ + p-)/2, dissipation
// alpha (p+ - p-)/2 from dx p-, dx p+.
template <int SCHEME>
__device__ __forceinline__ void axis_pair(const F2* u, float floor4, float inv_dx, F2 hax,
                                          F2& pbar, F2& diss)
{
    if constexpr (SCHEME == WENO5) {
        F2 cen6, phim6, phip6;
        weno5_jp2(u, floor4, cen6, phim6, phip6);
        lf_axis2(cen6, phim6, phip6, F2(inv_dx), hax, pbar, diss);
    } else {
        static_assert(SCHEME == ENO2 || SCHEME == ENO3, "paired ENO2, ENO3 or WENO5");
        F2 am, ap;
        if constexpr (SCHEME == ENO2) eno2_parts2(u, am, ap);
        else eno3_parts2(u, am, ap);
        pbar = (ap + am) * F2(0.5f * inv_dx);
        diss = fma2(hax, ap - am, diss);
    }
}

// FACES = true (WENO5): the marching axis' derivatives come from shared
// faces (weno5_face2): one face evaluation per node instead of two one-sided
// ones, the left-biased correction of the next plane carried in a register.
// The results are bit-identical to FACES = false.  SCHEME: WENO5, ENO2 or
// ENO3.  LOCAL (WENO5, state-only bounds): the stage's local-coefficient and
// variational flags are honoured -- per-node dissipation coefficients
// alpha_k(x) of each plane's node (LLF = LLLF for these bounds, Sec. IV-D)
// and the rate of the variational form min[0, H] (Sec. VI-A, Eq. 30)
// clipped at zero (the clip acts on 6 L, the same sign).
template <int NDIM, int DYN, bool FACES = false, bool COH = false, int SCHEME = WENO5,
          bool LOCAL = false>
__device__ __forceinline__ void tiled_pair_body(const StageArgs<float>& a, int TB, int TA, int bx,
                                                int by, int chunk, int outer, int ch, float* tile,
                                                int tx, int ty)
{
    static_assert(NDIM == 3 || NDIM == 4, "paired planes need a marching axis");
    static_assert(SCHEME == WENO5 || !FACES, "shared faces are a WENO5 form");
    static_assert(!LOCAL || (SCHEME == WENO5 && DYN != QUADRATIC),
                  "paired local coefficients: WENO5 with state-only bounds");
    constexpr int G = ghost_width(SCHEME);
    constexpr int AS = NDIM - 3, AA = NDIM - 2, AB = NDIM - 1;
    const int W = TB + 2 * G, H = TA + 2 * G, HW = H * W;
    const int nB = a.n[AB], nA = a.n[AA], nS = a.n[AS];
    const int sA = a.stride[AA], sS = a.stride[AS];
    const int b0 = bx * TB, a0 = by * TA;
    const int base_outer = (NDIM == 4) ? outer * a.stride[0] : 0;
    const int s_begin = chunk * ch;
    const int s_end = min(s_begin + ch, nS);
    const int ib = b0 + tx, ia = a0 + ty;
    const bool active = (ib < nB) && (ia < nA);
    const int tid = ty * TB + tx, nthr = TB * TA;

    float alpha[NDIM];
#pragma unroll
    for (int k = 0; k < NDIM; ++k)
        alpha[k] = a.alpha_from_ctl ? float(__longlong_as_double((long long)a.ctl->alpha_bits[k]))
                                    : a.alpha[k];
    const float dt = a.dt_from_ctl ? float(a.ctl->dt) : a.dt;
    // WENO5: the axes deliver 6 x the central costate and 6 x the
    // dissipation (lf_axis2); the Hamiltonians are positively homogeneous in
    // p (degree 1, the quadratic one degree 2, rescaled below), so the rate
    // comes out as 6 L and the 1/6 goes into the stage's time coefficient.
    constexpr float kRate = SCHEME == WENO5 ? 6.0f : 1.0f;
    const F2 clk(a.c_l * dt * (1.0f / kRate)), cs(a.c_s), cn(a.c_n);
    const float fl_s = weno_floor4(a.inv_dx[AS]);
    const float fl_a = weno_floor4(a.inv_dx[AA]);
    const float fl_b = weno_floor4(a.inv_dx[AB]);

    F2 x[NDIM];
    if constexpr (NDIM == 4) x[0] = F2(fmaf(float(outer), a.h[0], a.lo[0]));
    x[AA] = F2(fmaf(float(ia), a.h[AA], a.lo[AA]));
    x[AB] = F2(fmaf(float(ib), a.h[AB], a.lo[AB]));
    float sth = 0.f, cth = 1.f;
    if constexpr (DYN == AIR3D || DYN == CAR4D || DYN == ROCKETS) sincosf(x[2].x(), &sth, &cth);

    const int ia_c = min(ia, nA - 1), ib_c = min(ib, nB - 1);
    const float* col = a.phi_s + base_outer + ia_c * sA + ib_c;
    float w[2 * G + 2];
#pragma unroll
    for (int o = -G; o < G; ++o) w[o + G] = line_value<float, COH>(col, s_begin + o, nS, sS, a.periodic[AS]);

    constexpr int MAXE = 3;
    int e_off[MAXE];
    unsigned kinds = 0;
#pragma unroll
    for (int k = 0; k < MAXE; ++k) {
        const int e = tid + k * nthr;
        const int r = e / W, c = e - r * W;
        const int ja = a0 - G + r, jb = b0 - G + c;
        const bool inA = ja >= 0 && ja < nA, inB = jb >= 0 && jb < nB;
        const unsigned kind = (e >= HW) ? 3u : (inA && inB) ? 0u : inA ? 1u : inB ? 2u : 3u;
        kinds |= kind << (2 * k);
        e_off[k] = (kind == 0u) ? ja * sA + jb : (kind == 1u ? ja : (kind == 2u ? jb : 0));
    }
    // tiles whose halo lies inside the grid in A and B load without ghost
    // handling (block-uniform); nvalid = slots inside the tile
    const bool inner = a0 - G >= 0 && a0 + TA + G <= nA && b0 - G >= 0 && b0 + TB + G <= nB;
    const int nvalid = min(MAXE, max(0, (HW - tid + nthr - 1) / nthr));
    auto fetch = [&](int s, float* pf) {
        const float* plane = a.phi_s + base_outer + s * sS;
        if (inner) {
#pragma unroll
            for (int k = 0; k < MAXE; ++k)
                if (k < nvalid) pf[k] = ld_in<COH>(plane + e_off[k]);
            return;
        }
#pragma unroll
        for (int k = 0; k < MAXE; ++k) {
            const unsigned kind = (kinds >> (2 * k)) & 3u;
            float v = 0.f;
            if (kind == 0u) {
                v = ld_in<COH>(plane + e_off[k]);
            } else if (kind == 1u) {
                const int e = tid + k * nthr;
                v = line_value<float, COH>(plane + e_off[k] * sA, b0 - G + (e - (e / W) * W), nB, 1,
                               a.periodic[AB]);
            } else if (kind == 2u) {
                const int e = tid + k * nthr;
                v = line_value<float, COH>(plane + e_off[k], a0 - G + e / W, nA, sA, a.periodic[AA]);
            }
            pf[k] = v;
        }
    };
    float pfA[MAXE], pfB[MAXE];
    fetch(s_begin, pfA);
    fetch(min(s_begin + 1, nS - 1), pfB);
    // value j >= 0 of this thread's column along S (plain load inside the grid)
    auto col_value = [&](int j) -> float {
        if (j < nS) return ld_in<COH>(col + j * sS);
        return line_value<float, COH>(col, j, nS, sS, a.periodic[AS]);
    };
    float wnA = col_value(s_begin + G);
    float wnB = col_value(s_begin + G + 1);
    bool nonfinite = false;
    // FACES: left-biased correction of node s from the face s - 1/2 (values
    // s-3 .. s+2 = w[0..5] at the start of the chunk)
    float phim_next = 0.f;
    if constexpr (FACES) {
        F2 v[6], fm, fp, c;
#pragma unroll
        for (int o = 0; o < 6; ++o) v[o] = F2(w[o]);
        weno5_face2(v, fl_s, fm, fp, c);
        phim_next = fm.x();
    }

    for (int s = s_begin; s < s_end; s += 2) {
        // planes s and s+1 interleaved: one 64-bit shared access moves a
        // node's value on both planes, already in the pair layout
        float2* cur = reinterpret_cast<float2*>(tile) + (((s - s_begin) >> 1) & 1) * HW;
#pragma unroll
        for (int k = 0; k < MAXE; ++k)
            if (((kinds >> (2 * k)) & 3u) != 3u) cur[tid + k * nthr] = make_float2(pfA[k], pfB[k]);
        w[2 * G] = wnA;
        w[2 * G + 1] = wnB;
        __syncthreads();  // planes s, s+1 staged; the other buffer pair is free
        if (s + 2 < s_end) {
            fetch(s + 2, pfA);
            fetch(min(s + 3, nS - 1), pfB);
            wnA = col_value(s + 2 + G);
            wnB = col_value(s + 3 + G);
        }
        if (active) {
            const bool second = s + 1 < s_end;
            F2 u[2 * G + 1], pbar[NDIM], diss(0.f);
            // alpha_k / (2 dx_k) of the two nodes: global, or (LOCAL with the
            // stage's local flag) local to each node's state
            F2 hx[NDIM];
            if constexpr (LOCAL) {
                x[AS] = F2(fmaf(float(s), a.h[AS], a.lo[AS]), fmaf(float(s + 1), a.h[AS], a.lo[AS]));
                if (a.local_alpha) {
                    float xa[NDIM], xb[NDIM];
#pragma unroll
                    for (int k = 0; k < NDIM; ++k) {
                        xa[k] = x[k].x();
                        xb[k] = x[k].y();
                    }
#pragma unroll
                    for (int k = 0; k < NDIM; ++k)
                        hx[k] = F2(local_alpha<DYN>(xa, k, a.prm, sth, cth, 0.f, 0.f) * (0.5f * a.inv_dx[k]),
                                   local_alpha<DYN>(xb, k, a.prm, sth, cth, 0.f, 0.f) * (0.5f * a.inv_dx[k]));
                } else {
#pragma unroll
                    for (int k = 0; k < NDIM; ++k) hx[k] = F2(0.5f * alpha[k] * a.inv_dx[k]);
                }
            }
            // the global form forms its factor where it is used (not held in
            // a live array across the loop)
            auto hax = [&](int k) -> F2 {
                if constexpr (LOCAL) return hx[k];
                else return F2(0.5f * alpha[k] * a.inv_dx[k]);
            };
            if constexpr (FACES) {
                // faces s + 1/2 (x) and s + 3/2 (y): values w[1..6] and w[2..7]
                F2 fm, cen, phip;
#pragma unroll
                for (int o = 0; o < 6; ++o) u[o] = F2(w[o + 1], w[o + 2]);
                weno5_face2(u, fl_s, fm, phip, cen);
                const F2 phim(phim_next, fm.x());
                phim_next = fm.y();
                lf_axis2(cen, phim, phip, F2(a.inv_dx[AS]), hax(AS), pbar[AS], diss);
            } else {
#pragma unroll
                for (int o = 0; o <= 2 * G; ++o) u[o] = F2(w[o], w[o + 1]);
                axis_pair<SCHEME>(u, fl_s, a.inv_dx[AS], hax(AS), pbar[AS], diss);
            }
#pragma unroll
            for (int o = 0; o <= 2 * G; ++o)
                u[o] = F2(cur[(ty + o) * W + tx + G]);
            axis_pair<SCHEME>(u, fl_a, a.inv_dx[AA], hax(AA), pbar[AA], diss);
#pragma unroll
            for (int o = 0; o <= 2 * G; ++o)
                u[o] = F2(cur[(ty + G) * W + tx + o]);
            const F2 center = u[G];
            axis_pair<SCHEME>(u, fl_b, a.inv_dx[AB], hax(AB), pbar[AB], diss);
            if constexpr (NDIM == 4) {
                const float* c0 = a.phi_s + s * sS + ia * sA + ib;
                const float* c1 = c0 + (second ? sS : 0);
                if (outer >= G && outer + G < a.n[0]) {  // block-uniform: no ghost cells
#pragma unroll
                    for (int o = -G; o <= G; ++o)
                        u[o + G] = F2(ld_in<COH>(c0 + (outer + o) * a.stride[0]),
                                      ld_in<COH>(c1 + (outer + o) * a.stride[0]));
                } else {
#pragma unroll
                    for (int o = -G; o <= G; ++o)
                        u[o + G] = F2(line_value<float, COH>(c0, outer + o, a.n[0], a.stride[0], a.periodic[0]),
                                      line_value<float, COH>(c1, outer + o, a.n[0], a.stride[0],
                                                 a.periodic[0]));
                }
                axis_pair<SCHEME>(u, weno_floor4(a.inv_dx[0]), a.inv_dx[0], hax(0), pbar[0], diss);
            }
            x[AS] = F2(fmaf(float(s), a.h[AS], a.lo[AS]), fmaf(float(s + 1), a.h[AS], a.lo[AS]));
            F2 Hv = hamiltonian_pair<DYN, NDIM>(x, pbar, a.prm, sth, cth);  // kRate x H
            if constexpr (SCHEME == WENO5 && DYN == QUADRATIC)
                Hv = Hv * F2(1.0f / 6.0f);  // 36 H -> 6 H
            F2 L = diss - Hv;
            if constexpr (LOCAL)
                if (a.varform) L = min2(L, F2(0.f));
            const int idx = base_outer + s * sS + ia * sA + ib;
            F2 v = fma2(cs, center, clk * L);
            if (a.phi_n)
                v = fma2(cn, F2(ld_phin<COH>(a.phi_n + idx), second ? ld_phin<COH>(a.phi_n + idx + sS) : 0.f), v);
            if (a.tube) v = min2(v, F2(__ldg(a.target + idx), second ? __ldg(a.target + idx + sS) : 0.f));
            nonfinite |= !isfinite(v.x()) || (second && !isfinite(v.y()));
            a.out[idx] = v.x();
            if (second) a.out[idx + sS] = v.y();
        }
#pragma unroll
        for (int o = 0; o < 2 * G; ++o) w[o] = w[o + 2];
    }
    if (nonfinite) atomicOr(&a.ctl->flags, kFlagNonFinite);
}

// Single-problem launch of the paired body (FP32): blockDim = (tb, ta);
// gridDim = (ceil(nB/tb), ceil(nA/ta), nchunks * nOuter).
template <int NDIM, int DYN, int MINB, bool FACES, int SCHEME = WENO5, bool LOCAL = false>
__global__ void __launch_bounds__(256, MINB) stage_pair_kernel(StageArgs<float> a, int ch, int nchunks)
{
    extern __shared__ __align__(16) unsigned char smem_pair[];
    float* tile = reinterpret_cast<float*>(smem_pair);
    tiled_pair_body<NDIM, DYN, FACES, false, SCHEME, LOCAL>(a, blockDim.x, blockDim.y, blockIdx.x, blockIdx.y,
                               blockIdx.z % nchunks, blockIdx.z / nchunks, ch, tile, threadIdx.x,
                               threadIdx.y);
}

}  // namespace lsp
