// stage_tiled.cuh -- the fused Runge-Kutta stage kernel for 3-D and 4-D
// grids, tiled for GB300.
//
// Same computation as stage_generic_kernel (one TVD-RK stage, Sec. V-A, of
// the LF rate of Sec. IV-D with ghost cells of Sec. III-B and the tube of
// Sec. VI-A), organised for the memory system:
//  - a CTA owns a TA x TB tile of the two fastest axes (A, B) and marches
//    along the third-fastest axis S over a chunk of CH planes; a 4-D grid
//    adds the slowest axis as a grid dimension;
//  - each plane of the tile, with a G-cell halo in A and B (ghost values
//    substituted while loading), is staged in shared memory; the A and B
//    stencils read it from there;
//  - the S stencil lives in a register window of 2G+1 values per thread that
//    slides by one plane per iteration (one coalesced load per node);
//  - coordinates that are constant along the march (everything but S) and
//    their sin/cos are computed once per thread.
// Every node of the grid is read once from DRAM per stage in the best case
// (tiles overlap only in L2) and written once.
#pragma once
#include "stencil.cuh"

namespace lsp {

// HJ-WENO5 in the equivalent form of Jiang and Peng (the form the paper's
// Sec. IV-C follows): with second differences S_m = u_{m+1} - 2u_m + u_{m-1}
//   p- = [ (-d_{-2} + 7 d_{-1} + 7 d_0 - d_1) / 12 - Phi(S_-2, S_-1, S_0, S_1) ] / dx
//   p+ = [ (-d_{-2} + 7 d_{-1} + 7 d_0 - d_1) / 12 + Phi(S_2, S_1, S_0, S_-1) ] / dx
//   Phi(a,b,c,d) = w0 (a - 2b + c) / 3 + (w2 - 1/2)(b - 2c + d) / 6
// with IS0 = 13(a-b)^2 + 3(a-3b)^2, IS1 = 13(b-c)^2 + 3(b+c)^2,
// IS2 = 13(c-d)^2 + 3(3c-d)^2 (= 12 x the paper's sigma_k in units of the
// unscaled differences) and weights proportional to (1, 6, 3)/(IS_k + e)^2,
// e = 12 x the paper's eps.  Algebraically identical to the three weighted
// substencils; it shares the differences of both sides and needs one
// reciprocal per side: w0 = Q1 Q2 / P, w2 = 3 Q0 Q1 / P with Q_k = (IS_k+e)^2
// scaled by a power of two ~ 1/e (exact, keeps the products in range) and
// P = Q1 Q2 + 6 Q0 Q2 + 3 Q0 Q1.
__device__ __forceinline__ float weno_phi(float is0, float is1, float is2, float e, float A,
                                          float B)
{
    // power of two close to 1/e (e >= 1e-17 is a normal number)
    const float sc = __uint_as_float(0x7f000000u - (__float_as_uint(e) & 0x7f800000u));
    const float q0 = (is0 + e) * sc, q1 = (is1 + e) * sc, q2 = (is2 + e) * sc;
    const float Q0 = q0 * q0, Q1 = q1 * q1, Q2 = q2 * q2;
    const float Q12 = Q1 * Q2, Q01 = Q0 * Q1;
    const float P = fmaf(6.0f * Q0, Q2, fmaf(3.0f, Q01, Q12));
    const float r = __fdividef(1.0f, P);
    const float w0 = Q12 * r, w2 = 3.0f * Q01 * r;
    return w0 * A * (1.0f / 3.0f) + (w2 - 0.5f) * B * (1.0f / 6.0f);
}

__device__ __forceinline__ double weno_phi(double is0, double is1, double is2, double e,
                                           double A, double B)
{
    const double q0 = is0 + e, q1 = is1 + e, q2 = is2 + e;
    const double a0 = 1.0 / (q0 * q0), a1 = 6.0 / (q1 * q1), a2 = 3.0 / (q2 * q2);
    const double r = 1.0 / (a0 + a1 + a2);
    return a0 * r * A * (1.0 / 3.0) + (a2 * r - 0.5) * B * (1.0 / 6.0);
}

template <typename R>
__device__ __forceinline__ void deriv_weno5_jp(const R* u, R inv_dx, R floor12, R& pm, R& pp)
{
    const R dm3 = u[1] - u[0], dm2 = u[2] - u[1], dm1 = u[3] - u[2];
    const R d0 = u[4] - u[3], d1 = u[5] - u[4], d2 = u[6] - u[5];
    const R Sm2 = dm2 - dm3, Sm1 = dm1 - dm2, S0 = d0 - dm1, S1 = d1 - d0, S2 = d2 - d1;
    const R cen = (R(7) * (dm1 + d0) - (dm2 + d1)) * R(1.0 / 12.0);
    // max_k d_k^2 as (max_k |d_k|)^2: the same number (squaring rounds
    // monotonically on [0, inf)), one multiply instead of six
    const R m4 = rmax(rmax(rabs(dm2), rabs(dm1)), rmax(rabs(d0), rabs(d1)));
    const R mL = rmax(m4, rabs(dm3)), mR = rmax(m4, rabs(d2));
    const R eL = R(1.2e-5) * (mL * mL) + floor12;
    const R eR = R(1.2e-5) * (mR * mR) + floor12;
    const R e1 = (Sm2 - Sm1) * (Sm2 - Sm1), e2 = (Sm1 - S0) * (Sm1 - S0);
    const R e3 = (S0 - S1) * (S0 - S1), e4 = (S1 - S2) * (S1 - S2);
    const R f0m = Sm2 - R(3) * Sm1, f1m = Sm1 + S0, f2m = R(3) * S0 - S1;
    const R f0p = S2 - R(3) * S1, f1p = S1 + S0, f2p = R(3) * S0 - Sm1;
    const R is0m = R(13) * e1 + R(3) * f0m * f0m;
    const R is1m = R(13) * e2 + R(3) * f1m * f1m;
    const R is2m = R(13) * e3 + R(3) * f2m * f2m;
    const R is0p = R(13) * e4 + R(3) * f0p * f0p;
    const R is1p = R(13) * e3 + R(3) * f1p * f1p;
    const R is2p = R(13) * e2 + R(3) * f2p * f2p;
    const R Tm1 = Sm2 - R(2) * Sm1 + S0, T0 = Sm1 - R(2) * S0 + S1, T1 = S0 - R(2) * S1 + S2;
    pm = (cen - weno_phi(is0m, is1m, is2m, eL, Tm1, T0)) * inv_dx;
    pp = (cen + weno_phi(is0p, is1p, is2p, eR, T1, T0)) * inv_dx;
}

// 12 x the regulariser floor on unscaled differences (see Num<R>).
template <typename R>
__device__ __forceinline__ R weno_floor12(R inv_dx)
{
    return R(12) * Num<R>::eps_floor(inv_dx);
}

// 4 x the floor, for the indicators scaled by 1/3 of the paired form (pair2.cuh).
template <typename R>
__device__ __forceinline__ R weno_floor4(R inv_dx)
{
    return R(4) * Num<R>::eps_floor(inv_dx);
}

template <int SCHEME, typename R>
__device__ __forceinline__ void deriv_fast(const R* u, R inv_dx, R floor12, R& pm, R& pp)
{
    if constexpr (SCHEME == WENO5) deriv_weno5_jp(u, inv_dx, floor12, pm, pp);
    else deriv<SCHEME>(u, inv_dx, pm, pp);
}

// Loads of the stage input.  COH = false: through the read-only cache (the
// field does not change during the launch).  COH = true: the persistent
// batched launch, in which other CTAs of the same launch wrote the field
// before this CTA's acquire (the fence after it observed their completion
// count): a weak load cached at every level (ld.global.ca), which that
// acquire orders, not the read-only path, which no fence orders.
template <bool COH, typename R>
__device__ __forceinline__ R ld_in(const R* p)
{
    if constexpr (COH) return __ldca(p);
    else return __ldg(p);
}

// Value at index j of a line of n nodes whose node 0 is at p[0] with stride
// s, ghost cells substituted (periodic wrap or linear extrapolation).
template <typename R, bool COH = false>
__device__ __forceinline__ R line_value(const R* __restrict__ p, int j, int n, int s, int periodic)
{
    if (j >= 0 && j < n) return ld_in<COH>(p + j * s);
    if (periodic) return ld_in<COH>(p + (j < 0 ? j + n : j - n) * s);
    if (j < 0) {
        const R u0 = ld_in<COH>(p), u1 = ld_in<COH>(p + s);
        return u0 + R(-j) * (u0 - u1);
    }
    const R un = ld_in<COH>(p + (n - 1) * s), um = ld_in<COH>(p + (n - 2) * s);
    return un + R(j - n + 1) * (un - um);
}

struct Tile {
    int tb, ta, ch;  // tile width (fastest axis), tile rows, planes per CTA
    int minb;        // occupancy target of the kernel variant (2, 3 or 4)
    int pair;        // 0 scalar body; 1 two planes per iteration in paired FP32;
                     // 2 the same with shared WENO5 faces; 3 / 4 face-shared
                     // ENO runs of 4 / 2 nodes (stage_run.cuh)
};

// One CTA's share of a stage: the tile (bx, by) of the two fastest axes,
// chunk `chunk` of the march along axis S and, for 4-D grids, index `outer`
// along axis 0.  2-D grids have no march (one plane).  Block of TB x TA
// threads (tx, ty); `tile` holds (TA + 2G) x (TB + 2G) values.
// LOCAL = true compiles the per-node dissipation coefficients (LLF/LLLF) and
// the variational clip in, each taken when its StageArgs flag is set;
// LOCAL = false is the global-LF form alone (the code the benchmark runs,
// kept free of the local variants so that every kernel that inlines it
// rounds it the same way).
template <int NDIM, int SCHEME, int DYN, typename R, bool COH = false, bool LOCAL = false>
__device__ __forceinline__ void tiled_stage_body(const StageArgs<R>& a, int TB, int TA, int bx,
                                                 int by, int chunk, int outer, int ch, R* tile,
                                                 int tx, int ty)
{
    static_assert(NDIM >= 2 && NDIM <= 4, "tiled stage is for 2-D to 4-D grids");
    constexpr int G = ghost_width(SCHEME);
    constexpr bool HAS_S = NDIM >= 3;
    constexpr int AS = HAS_S ? NDIM - 3 : 0, AA = NDIM - 2, AB = NDIM - 1;

    const int W = TB + 2 * G;           // tile row length with halo
    const int H = TA + 2 * G;           // tile rows with halo
    const int nB = a.n[AB], nA = a.n[AA];
    const int nS = HAS_S ? a.n[AS] : 1;
    const int sA = a.stride[AA], sS = HAS_S ? a.stride[AS] : 0;
    const int b0 = bx * TB, a0 = by * TA;
    const int base_outer = (NDIM == 4) ? outer * a.stride[0] : 0;
    const int s_begin = HAS_S ? chunk * ch : 0;
    const int s_end = HAS_S ? min(s_begin + ch, nS) : 1;
    const int ib = b0 + tx, ia = a0 + ty;
    const bool active = (ib < nB) && (ia < nA);
    const int tid = ty * TB + tx, nthr = TB * TA;

    R alpha[NDIM];
#pragma unroll
    for (int k = 0; k < NDIM; ++k)
        alpha[k] = a.alpha_from_ctl ? R(__longlong_as_double((long long)a.ctl->alpha_bits[k]))
                                    : a.alpha[k];
    const R dt = a.dt_from_ctl ? R(a.ctl->dt) : a.dt;
    const R cl = a.c_l * dt;
    const R fl_a = weno_floor12(a.inv_dx[AA]);
    const R fl_b = weno_floor12(a.inv_dx[AB]);

    // coordinates fixed for this thread (and the heading's sin/cos: theta
    // is axis 2, one of the tile axes, for both 3-D and 4-D games)
    R x[NDIM];
    if constexpr (NDIM == 4) x[0] = rfma(R(outer), a.h[0], a.lo[0]);
    x[AA] = rfma(R(ia), a.h[AA], a.lo[AA]);
    x[AB] = rfma(R(ib), a.h[AB], a.lo[AB]);
    R sth = R(0), cth = R(1);
    if constexpr (DYN == AIR3D || DYN == CAR4D || DYN == ROCKETS) rsincos(x[2], &sth, &cth);

    // own column along S (clamped so inactive threads stay in bounds)
    const int ia_c = min(ia, nA - 1), ib_c = min(ib, nB - 1);
    const R* col = a.phi_s + base_outer + ia_c * sA + ib_c;
    R w[2 * G + 1];
    if constexpr (HAS_S) {
#pragma unroll
        for (int o = -G; o < G; ++o)
            w[o + G] = line_value<R, COH>(col, s_begin + o, nS, sS, a.periodic[AS]);
    }

    // This thread's share of the plane tile (with halo): at most 3 slots.
    // Kinds, packed 2 bits per slot: 0 interior, 1 ghost along B, 2 ghost
    // along A, 3 corner (never read by the axis stencils) or unused.
    constexpr int MAXE = 3;
    int e_off[MAXE];
    unsigned kinds = 0;
#pragma unroll
    for (int k = 0; k < MAXE; ++k) {
        const int e = tid + k * nthr;
        const int r = e / W, c = e - r * W;
        const int ja = a0 - G + r, jb = b0 - G + c;
        const bool inA = ja >= 0 && ja < nA, inB = jb >= 0 && jb < nB;
        const unsigned kind = (e >= H * W) ? 3u : (inA && inB) ? 0u : inA ? 1u : inB ? 2u : 3u;
        kinds |= kind << (2 * k);
        e_off[k] = (kind == 0u) ? ja * sA + jb : (kind == 1u ? ja : (kind == 2u ? jb : 0));
    }
    // Tiles whose halo lies inside the grid in A and B (block-uniform) load
    // their slots without ghost handling; nvalid = slots inside the tile.
    const bool inner = a0 - G >= 0 && a0 + TA + G <= nA && b0 - G >= 0 && b0 + TB + G <= nB;
    const int nvalid = min(MAXE, max(0, (H * W - tid + nthr - 1) / nthr));
    // Fetch this thread's slots of plane s (ghost values substituted).
    auto fetch = [&](int s, R* pf) {
        const R* plane = a.phi_s + base_outer + s * sS;
        if (inner) {
#pragma unroll
            for (int k = 0; k < MAXE; ++k)
                if (k < nvalid) pf[k] = ld_in<COH>(plane + e_off[k]);
            return;
        }
#pragma unroll
        for (int k = 0; k < MAXE; ++k) {
            const unsigned kind = (kinds >> (2 * k)) & 3u;
            R v = R(0);
            if (kind == 0u) {
                v = ld_in<COH>(plane + e_off[k]);
            } else if (kind == 1u) {  // e_off = ja; jb recomputed from the slot
                const int e = tid + k * nthr;
                v = line_value<R, COH>(plane + e_off[k] * sA, b0 - G + (e - (e / W) * W), nB, 1,
                               a.periodic[AB]);
            } else if (kind == 2u) {  // e_off = jb
                const int e = tid + k * nthr;
                v = line_value<R, COH>(plane + e_off[k], a0 - G + e / W, nA, sA, a.periodic[AA]);
            }
            pf[k] = v;
        }
    };
    R pf[MAXE];
    fetch(s_begin, pf);
    // value j of this thread's column along S (plain load inside the grid)
    auto col_value = [&](int j) -> R {
        if (j < nS) return ld_in<COH>(col + j * sS);
        return line_value<R, COH>(col, j, nS, sS, a.periodic[AS]);
    };
    R wnext = R(0);
    if constexpr (HAS_S) wnext = col_value(s_begin + G);
    bool nonfinite = false;

    for (int s = s_begin; s < s_end; ++s) {
        // double buffer: the buffer written here was last read two planes
        // ago, before every thread passed the previous plane's barrier
        R* cur = tile + ((s - s_begin) & 1) * (H * W);
#pragma unroll
        for (int k = 0; k < MAXE; ++k)
            if (((kinds >> (2 * k)) & 3u) != 3u) cur[tid + k * nthr] = pf[k];
        if constexpr (HAS_S) w[2 * G] = wnext;
        __syncthreads();  // plane s staged
        if (s + 1 < s_end) {  // issue plane s+1's loads before computing plane s
            fetch(s + 1, pf);
            if constexpr (HAS_S) wnext = col_value(s + 1 + G);
        }
        const R* tile_s = cur;
        if (active) {
            const R* tile = tile_s;
            R pm, pp, pbar[NDIM], diss = R(0);
            if constexpr (HAS_S) x[AS] = rfma(R(s), a.h[AS], a.lo[AS]);
            // dissipation coefficient of axis k: global, or local (LLF/LLLF)
            auto coef = [&](int k, R m, R p) -> R {
                if constexpr (LOCAL)
                    return a.local_alpha ? local_alpha<DYN>(x, k, a.prm, sth, cth, m, p) : alpha[k];
                else
                    return alpha[k];
            };
            if constexpr (HAS_S) {  // S axis from the register window
                deriv_fast<SCHEME>(w, a.inv_dx[AS], weno_floor12(a.inv_dx[AS]), pm, pp);
                pbar[AS] = R(0.5) * (pp + pm);
                diss = rfma(coef(AS, pm, pp) * R(0.5), pp - pm, diss);
            }
            {  // A axis from the tile column
                R u[2 * G + 1];
#pragma unroll
                for (int o = 0; o <= 2 * G; ++o) u[o] = tile[(ty + o) * W + tx + G];
                deriv_fast<SCHEME>(u, a.inv_dx[AA], fl_a, pm, pp);
                pbar[AA] = R(0.5) * (pp + pm);
                diss = rfma(coef(AA, pm, pp) * R(0.5), pp - pm, diss);
            }
            R center;
            {  // B axis from the tile row
                R u[2 * G + 1];
#pragma unroll
                for (int o = 0; o <= 2 * G; ++o) u[o] = tile[(ty + G) * W + tx + o];
                center = u[G];
                deriv_fast<SCHEME>(u, a.inv_dx[AB], fl_b, pm, pp);
                pbar[AB] = R(0.5) * (pp + pm);
                diss = rfma(coef(AB, pm, pp) * R(0.5), pp - pm, diss);
            }
            if constexpr (NDIM == 4) {
                // axis 0 (a grid dimension): window straight from global memory
                R u[2 * G + 1];
                const R* col0 = a.phi_s + s * sS + ia * sA + ib;
                if (outer >= G && outer + G < a.n[0]) {  // block-uniform: no ghost cells
#pragma unroll
                    for (int o = -G; o <= G; ++o)
                        u[o + G] = ld_in<COH>(col0 + (outer + o) * a.stride[0]);
                } else {
#pragma unroll
                    for (int o = -G; o <= G; ++o)
                        u[o + G] = line_value<R, COH>(col0, outer + o, a.n[0], a.stride[0],
                                                      a.periodic[0]);
                }
                deriv_fast<SCHEME>(u, a.inv_dx[0], weno_floor12(a.inv_dx[0]), pm, pp);
                pbar[0] = R(0.5) * (pp + pm);
                diss = rfma(coef(0, pm, pp) * R(0.5), pp - pm, diss);
            }
            const R Hv = hamiltonian_sc<DYN, NDIM>(x, pbar, a.prm, sth, cth);
            R L = -(Hv - diss);
            if constexpr (LOCAL)
                if (a.varform) L = rmin(L, R(0));
            const int idx = base_outer + s * sS + ia * sA + ib;
            R v = rfma(cl, L, a.c_s * center);
            if (a.phi_n) v = rfma(a.c_n, COH ? __ldca(a.phi_n + idx) : a.phi_n[idx], v);
            if (a.tube) v = rmin(v, __ldg(a.target + idx));
            nonfinite |= !isfinite(v);
            a.out[idx] = v;
        }
        if constexpr (HAS_S) {
#pragma unroll
            for (int o = 0; o < 2 * G; ++o) w[o] = w[o + 1];
        }
    }
    if (nonfinite) atomicOr(&a.ctl->flags, kFlagNonFinite);
}

// Single-problem launch: blockDim = (tb, ta); gridDim = (ceil(nB/tb),
// ceil(nA/ta), nchunks * nOuter).
// MINB: CTAs of 256 threads that must fit on one SM (2: up to 128
// registers per thread, 3: 80, 4: 64).
template <int NDIM, int SCHEME, int DYN, typename R, int MINB, bool LOCAL = false>
__global__ void __launch_bounds__(256, MINB) stage_tiled_kernel(StageArgs<R> a, int ch, int nchunks)
{
    extern __shared__ unsigned char smem_raw[];
    R* tile = reinterpret_cast<R*>(smem_raw);
    tiled_stage_body<NDIM, SCHEME, DYN, R, false, LOCAL>(a, blockDim.x, blockDim.y, blockIdx.x, blockIdx.y,
                                           blockIdx.z % nchunks, blockIdx.z / nchunks, ch, tile,
                                           threadIdx.x, threadIdx.y);
}

}  // namespace lsp
