// stencil.cuh -- device building blocks of one Runge-Kutta stage of the
// level-set method of LevelSetPy (arXiv 2411.03501): one-sided derivatives
// (Sec. IV-A..IV-C), Hamiltonians with optimal inputs (Sec. VI-A pattern) and
// the Lax-Friedrichs numerical Hamiltonian (Sec. IV-D).
//
// Derivatives are written on a window u[0..2G] holding the values at axis
// offsets -G..G of the node (ghost cells already substituted).  Differences
// are kept unscaled (u_{j+1} - u_j) and multiplied by 1/dx once at the end,
// which leaves every ENO comparison and every WENO weight unchanged (both are
// invariant under a common positive scale).
#pragma once
#include <cuda_runtime.h>
#include "lsp_internal.h"

namespace lsp {

// Additive floor of the WENO regulariser eps, on UNSCALED differences.
// FP64 keeps the paper's 1e-99 on differences scaled by 1/dx (1e-99 dx^2
// unscaled).  In FP32 that underflows and (sigma + eps)^2 would flush to
// zero on a flat stencil (0/0 weights); 1e-18 on the unscaled differences
// keeps (sigma + eps)^2 >= 1e-36, a normal number, and only matters where
// every difference of the stencil is below ~1e-9, where all substencils
// agree to rounding anyway.
template <typename R> struct Num;
template <> struct Num<float> {
    static __device__ __forceinline__ float eps_floor(float /*inv_dx*/) { return 1e-18f; }
};
template <> struct Num<double> {
    static __device__ __forceinline__ double eps_floor(double inv_dx)
    {
        return 1e-99 / (inv_dx * inv_dx);
    }
};

__device__ __forceinline__ float rabs(float x) { return fabsf(x); }
// explicit fused multiply-add: the same rounding in every kernel that inlines
// the caller, whatever the compiler would contract there
__device__ __forceinline__ float rfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ double rabs(double x) { return fabs(x); }
__device__ __forceinline__ float rmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double rmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float rmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double rmin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float real_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double real_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ void rsincos(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void rsincos(double x, double* s, double* c) { sincos(x, s, c); }

// ---------------------------------------------------------------------------
// First-order upwinding (Sec. IV-A): p- = D- u, p+ = D+ u.   Window G = 1.
template <typename R>
__device__ __forceinline__ void deriv_upwind1(const R* u, R inv_dx, R& pm, R& pp)
{
    pm = (u[1] - u[0]) * inv_dx;
    pp = (u[2] - u[1]) * inv_dx;
}

// ENO stencil choices once per cell face.  The ENO polynomial of the
// right-biased derivative at node j and of the left-biased one at node j+1
// starts from the same interval [x_j, x_j+1] (k = j for both, Eqs. 11-14),
// so the second-difference choice, the base index k* and the third-difference
// choice are the same for both; only the evaluation point differs:
//   p+_j = d - c/2 + cs f+/6,  p-_{j+1} = d + c/2 + cs f-/6,
//   (f+, f-) = (-1, 2) if the left second difference was taken, else (2, -1),
// with d = u_{j+1} - u_j, c the chosen second difference S and cs the chosen
// third difference T (unscaled; the caller applies 1/dx).  With M_j the
// smaller in magnitude of T_{j-1/2}, T_{j+1/2} (ties to the left, the <= of
// Eq. 13), cs = M_j when the left second difference is taken, else M_{j+1}.
// Every choice is a select on a comparison (no branches).

// The one of a, b smaller in magnitude, ties to a.
template <typename R>
__device__ __forceinline__ R eno_smaller(R a, R b)
{
    return rabs(a) <= rabs(b) ? a : b;
}

// Face j+1/2 of ENO3 from d, S_j, S_{j+1}, M_j, M_{j+1}: pp = dx p+_j,
// pm = dx p-_{j+1}.
template <typename R>
__device__ __forceinline__ void eno3_face(R d, R Sj, R Sj1, R Mj, R Mj1, R& pp, R& pm)
{
    const bool left = rabs(Sj) <= rabs(Sj1);
    const R c = left ? Sj : Sj1;
    const R cs = left ? Mj : Mj1;
    const R fp = left ? R(-1.0 / 6.0) : R(1.0 / 3.0);
    const R fm = left ? R(1.0 / 3.0) : R(-1.0 / 6.0);
    pp = rfma(cs, fp, rfma(R(-0.5), c, d));
    pm = rfma(cs, fm, rfma(R(0.5), c, d));
}

// Face j+1/2 of ENO2: pp = dx p+_j, pm = dx p-_{j+1}.
template <typename R>
__device__ __forceinline__ void eno2_face(R d, R Sj, R Sj1, R& pp, R& pm)
{
    const R c = eno_smaller(Sj, Sj1);
    pp = rfma(R(-0.5), c, d);
    pm = rfma(R(0.5), c, d);
}

// dx p- and dx p+ at NN consecutive nodes of a line from the window
// w[0 .. NN+2G-1] (w[k] = value at node k - G), each face evaluated once.
template <int SCHEME, int NN, typename R>
__device__ __forceinline__ void eno_line(const R* w, R* pm, R* pp)
{
    constexpr int G = SCHEME == ENO2 ? 2 : 3;
    R d[NN + 2 * G - 1];  // d[k]: face (k - G) + 1/2
#pragma unroll
    for (int k = 0; k < NN + 2 * G - 1; ++k) d[k] = w[k + 1] - w[k];
    R S[NN + 2 * G - 2];  // S[k]: node k - G + 1
#pragma unroll
    for (int k = 0; k < NN + 2 * G - 2; ++k) S[k] = d[k + 1] - d[k];
    if constexpr (SCHEME == ENO2) {
#pragma unroll
        for (int j = -1; j < NN; ++j) {  // face j+1/2: S_j = S[j+1], d = d[j+2]
            R a, b;
            eno2_face(d[j + 2], S[j + 1], S[j + 2], a, b);
            if (j >= 0) pp[j] = a;
            if (j + 1 < NN) pm[j + 1] = b;
        }
    } else {
        static_assert(SCHEME == ENO3, "ENO2 or ENO3");
        R T[NN + 3];  // T[k]: face (k - 2) + 1/2
#pragma unroll
        for (int k = 0; k < NN + 3; ++k) T[k] = S[k + 1] - S[k];
        R M[NN + 2];  // M[j+1] = M_j = smaller of T_{j-1/2}, T_{j+1/2}
#pragma unroll
        for (int j = -1; j <= NN; ++j) M[j + 1] = eno_smaller(T[j + 1], T[j + 2]);
#pragma unroll
        for (int j = -1; j < NN; ++j) {  // face j+1/2: S_j = S[j+2], d = d[j+3]
            R a, b;
            eno3_face(d[j + 3], S[j + 2], S[j + 3], M[j + 1], M[j + 2], a, b);
            if (j >= 0) pp[j] = a;
            if (j + 1 < NN) pm[j + 1] = b;
        }
    }
}

// ENO2 (Sec. IV-B, Eqs. 11-12).  Window G = 2, u[m+2] = value at offset m.
// With d_m = u_{m+1} - u_m and S_m = d_m - d_{m-1} (= 2 dx^2 D2_m):
//   left  (k = i-1): p- = (d_{-1} + S_c / 2) / dx, S_c the smaller in
//                    magnitude of S_{-1}, S_0 (ties to the left one)
//   right (k = i)  : p+ = (d_0 - S_c / 2) / dx, S_c from S_0, S_1
// (Per node, as written: on the 4-D ENO3 stage this form runs 19 % faster
// than the per-node use of eno_line, 686 vs 849 us per launch.)
template <typename R>
__device__ __forceinline__ void deriv_eno2(const R* u, R inv_dx, R& pm, R& pp)
{
    const R dm2 = u[1] - u[0], dm1 = u[2] - u[1], d0 = u[3] - u[2], d1 = u[4] - u[3];
    const R Sm1 = dm1 - dm2, S0 = d0 - dm1, S1 = d1 - d0;
    const R cl = (rabs(Sm1) <= rabs(S0)) ? Sm1 : S0;
    const R cr = (rabs(S0) <= rabs(S1)) ? S0 : S1;
    pm = (dm1 + R(0.5) * cl) * inv_dx;
    pp = (d0 - R(0.5) * cr) * inv_dx;
}

// ENO3 (Sec. IV-B, Eqs. 11-14).  Window G = 3, u[m+3] = value at offset m.
// T_m = S_{m+1} - S_m (= 6 dx^3 D3_{m+1/2}); after the ENO2 choice the base
// index k* is k-1 if the left second difference was taken, else k; the cubic
// term is T_c (3 s^2 - 6 s + 2) / 6 / dx with s = i - k* and T_c the smaller
// in magnitude of T_{k*}, T_{k*+1}.
template <typename R>
__device__ __forceinline__ void deriv_eno3(const R* u, R inv_dx, R& pm, R& pp)
{
    const R dm3 = u[1] - u[0], dm2 = u[2] - u[1], dm1 = u[3] - u[2];
    const R d0 = u[4] - u[3], d1 = u[5] - u[4], d2 = u[6] - u[5];
    const R Sm2 = dm2 - dm3, Sm1 = dm1 - dm2, S0 = d0 - dm1, S1 = d1 - d0, S2 = d2 - d1;
    const R Tm2 = Sm1 - Sm2, Tm1 = S0 - Sm1, T0 = S1 - S0, T1 = S2 - S1;
    // left derivative, k = i-1
    {
        R c, ta, tb, f;
        if (rabs(Sm1) <= rabs(S0)) { c = Sm1; ta = Tm2; tb = Tm1; f = R(2); }   // k* = i-2, s = 2
        else                       { c = S0;  ta = Tm1; tb = T0;  f = R(-1); }  // k* = i-1, s = 1
        const R cs = (rabs(ta) <= rabs(tb)) ? ta : tb;
        pm = (dm1 + R(0.5) * c + cs * f * R(1.0 / 6.0)) * inv_dx;
    }
    // right derivative, k = i
    {
        R c, ta, tb, f;
        if (rabs(S0) <= rabs(S1)) { c = S0; ta = Tm1; tb = T0; f = R(-1); }  // k* = i-1, s = 1
        else                      { c = S1; ta = T0;  tb = T1; f = R(2); }   // k* = i,   s = 0
        const R cs = (rabs(ta) <= rabs(tb)) ? ta : tb;
        pp = (d0 - R(0.5) * c + cs * f * R(1.0 / 6.0)) * inv_dx;
    }
}

// HJ-WENO5 combination (Sec. IV-C, Eqs. 15-20) of five differences v1..v5
// (unscaled: the result is multiplied by 1/dx by the caller).  Substencils
// with +1/3 on the first term of the third one, smoothness indicators with
// v2 - 2 v3 + v4 in the second, eps = 1e-6 max(v_k^2) + floor, optimal
// weights 0.1, 0.6, 0.3.
template <typename R>
__device__ __forceinline__ R weno5_combine(R v1, R v2, R v3, R v4, R v5, R floor_)
{
    const R phi1 = v1 * R(1.0 / 3.0) - v2 * R(7.0 / 6.0) + v3 * R(11.0 / 6.0);
    const R phi2 = -v2 * R(1.0 / 6.0) + v3 * R(5.0 / 6.0) + v4 * R(1.0 / 3.0);
    const R phi3 = v3 * R(1.0 / 3.0) + v4 * R(5.0 / 6.0) - v5 * R(1.0 / 6.0);
    const R a1 = v1 - R(2) * v2 + v3, b1 = v1 - R(4) * v2 + R(3) * v3;
    const R a2 = v2 - R(2) * v3 + v4, b2 = v2 - v4;
    const R a3 = v3 - R(2) * v4 + v5, b3 = R(3) * v3 - R(4) * v4 + v5;
    const R s1 = R(13.0 / 12.0) * a1 * a1 + R(0.25) * b1 * b1;
    const R s2 = R(13.0 / 12.0) * a2 * a2 + R(0.25) * b2 * b2;
    const R s3 = R(13.0 / 12.0) * a3 * a3 + R(0.25) * b3 * b3;
    R mx = rmax(rmax(v1 * v1, v2 * v2), rmax(v3 * v3, v4 * v4));
    mx = rmax(mx, v5 * v5);
    const R eps = R(1e-6) * mx + floor_;
    const R q1 = s1 + eps, q2 = s2 + eps, q3 = s3 + eps;
    const R al1 = R(0.1) / (q1 * q1);
    const R al2 = R(0.6) / (q2 * q2);
    const R al3 = R(0.3) / (q3 * q3);
    const R inv = R(1) / (al1 + al2 + al3);
    return (al1 * phi1 + al2 * phi2 + al3 * phi3) * inv;
}

// Left derivative from D+u_{i-3..i+1}, right one from the mirror image
// D+u_{i+2}, D+u_{i+1}, D+u_i, D+u_{i-1}, D+u_{i-2}.  Window G = 3.
template <typename R>
__device__ __forceinline__ void deriv_weno5(const R* u, R inv_dx, R& pm, R& pp)
{
    const R dm3 = u[1] - u[0], dm2 = u[2] - u[1], dm1 = u[3] - u[2];
    const R d0 = u[4] - u[3], d1 = u[5] - u[4], d2 = u[6] - u[5];
    const R fl = Num<R>::eps_floor(inv_dx);
    pm = weno5_combine(dm3, dm2, dm1, d0, d1, fl) * inv_dx;
    pp = weno5_combine(d2, d1, d0, dm1, dm2, fl) * inv_dx;
}

template <int SCHEME, typename R>
__device__ __forceinline__ void deriv(const R* u, R inv_dx, R& pm, R& pp)
{
    if constexpr (SCHEME == UPWIND1) deriv_upwind1(u, inv_dx, pm, pp);
    else if constexpr (SCHEME == ENO2) deriv_eno2(u, inv_dx, pm, pp);
    else if constexpr (SCHEME == ENO3) deriv_eno3(u, inv_dx, pm, pp);
    else deriv_weno5(u, inv_dx, pm, pp);
}

// ---------------------------------------------------------------------------
// Rockets game (Sec. VI-A, Eq. 31): f = (a cos th + u_e x, a sin th + a +
// u_p x - g, u_p - u_e), evader u_e in [-ue, ue] maximises, pursuer u_p in
// [-up, up] minimises, H = -max min p.f; with p.f = p1 a cos th +
// p2 (a sin th + a - g) + u_e (p1 x - p3) + u_p (p2 x + p3) the optimum is
// p1 a cos th + p2 (a sin th + a - g) + ue |p1 x - p3| - up |p2 x + p3|.
// (Eq. 32 prints this closed form with three sign slips; the definition is
// what is evaluated.)  Explicit operations: see hamiltonian_sc.
template <typename R>
__device__ __forceinline__ R hamiltonian_rockets(const R* x, const R* p, const R* prm, R s, R c)
{
    const R a = prm[0], g = prm[1], ue = prm[2], up = prm[3];
    const R fx = a * c, fz = rfma(a, s, a - g);
    R v = rfma(p[0], fx, p[1] * fz);
    v = rfma(ue, rabs(rfma(p[0], x[0], -p[2])), v);
    v = rfma(-up, rabs(rfma(p[1], x[0], p[2])), v);
    return -v;
}

// ---------------------------------------------------------------------------
// Hamiltonians at (x, p).  Reachability games follow H = -max_u min_d p.f
// (Sec. VI-A, Eq. 31) evaluated in closed form: the optimal bounded inputs
// are picked by the sign of their costate coefficient, which produces the
// |.| switching terms (the pattern of Eq. 32).
template <int DYN, int NDIM, typename R>
__device__ __forceinline__ R hamiltonian(const R* x, const R* p, const R* prm)
{
    if constexpr (DYN == NORMAL_SPEED) {
        R s = R(0);
#pragma unroll
        for (int k = 0; k < NDIM; ++k) s += p[k] * p[k];
        return prm[0] * real_sqrt(s);
    } else if constexpr (DYN == TRANSLATE) {
        R s = R(0);
#pragma unroll
        for (int k = 0; k < NDIM; ++k) s += prm[k] * p[k];
        return s;
    } else if constexpr (DYN == QUADRATIC) {
        R s = R(0);
#pragma unroll
        for (int k = 0; k < NDIM; ++k) s += p[k] * p[k];
        return R(0.5) * s;
    } else if constexpr (DYN == AIR3D) {
        // relative dynamics: xdot = -v_e + v_p cos th + u y, ydot = v_p sin th - u x,
        // thdot = d - u; evader input u in [-u_max, u_max] maximises, pursuer
        // input d in [-d_max, d_max] minimises.
        R s, c;
        rsincos(x[2], &s, &c);
        const R ve = prm[0], vp = prm[1], um = prm[2], dm = prm[3];
        const R v = p[0] * (-ve + vp * c) + p[1] * (vp * s) +
                    um * rabs(p[0] * x[1] - p[1] * x[0] - p[2]) - dm * rabs(p[2]);
        return -v;
    } else if constexpr (DYN == CAR4D) {  // xdot = v cos th, ydot = v sin th, thdot = w,
                                         // vdot = a; both inputs minimise p.f (reach)
        R s, c;
        rsincos(x[2], &s, &c);
        const R v = x[3];
        const R m = p[0] * v * c + p[1] * v * s - prm[0] * rabs(p[2]) - prm[1] * rabs(p[3]);
        return -m;
    } else if constexpr (DYN == ROCKETS) {
        R s, c;
        rsincos(x[2], &s, &c);
        return hamiltonian_rockets(x, p, prm, s, c);
    } else {  // DOUBLE_INT: x1dot = x2, x2dot = u, |u| <= umax minimises p.f (reach)
        return -rfma(p[0], x[1], -prm[0] * rabs(p[1]));
    }
}

// Hamiltonian with the coordinate-only factors (sin/cos of the heading)
// precomputed by the caller: hamiltonian_sc(x, p, prm, sin th, cos th).
// Every product and sum is an explicit operation here (and in local_alpha
// below, which shares factors with it), so the rounding does not depend on
// how the compiler fuses them in the kernel that inlines the call: the tiled
// body gives the same bits in the single-problem and the batched kernels.
template <int DYN, int NDIM, typename R>
__device__ __forceinline__ R hamiltonian_sc(const R* x, const R* p, const R* prm, R s, R c)
{
    if constexpr (DYN == AIR3D) {
        const R ve = prm[0], vp = prm[1], um = prm[2], dm = prm[3];
        const R fx = rfma(vp, c, -ve);  // -v_e + v_p cos th
        const R fy = vp * s;
        const R sw = rfma(p[0], x[1], -(p[1] * x[0])) - p[2];
        R v = rfma(p[0], fx, p[1] * fy);
        v = rfma(um, rabs(sw), v);
        v = rfma(-dm, rabs(p[2]), v);
        return -v;
    } else if constexpr (DYN == CAR4D) {
        const R vc = x[3] * c, vs = x[3] * s;
        R m = rfma(p[0], vc, p[1] * vs);
        m = rfma(-prm[0], rabs(p[2]), m);
        m = rfma(-prm[1], rabs(p[3]), m);
        return -m;
    } else if constexpr (DYN == ROCKETS) {
        return hamiltonian_rockets(x, p, prm, s, c);
    } else {
        return hamiltonian<DYN, NDIM>(x, p, prm);
    }
}

// Local dissipation coefficient of axis k at one node (LLF / LLLF, Sec.
// IV-D's Lax-Friedrichs term with the toolbox's local siblings of the GLF
// routine): the bound on |dH/dp_k| at the node's state, or for H = |p|^2/2
// over the node's own costate interval, max(|p-_k|, |p+_k|).  The bounds
// involve at most the costate of axis k, so LLF and LLLF coincide.  s, c:
// sin and cos of the heading x[2] (AIR3D, CAR4D).
template <int DYN, typename R>
__device__ __forceinline__ R local_alpha(const R* x, int k, const R* prm, R s, R c, R pm, R pp)
{
    if constexpr (DYN == NORMAL_SPEED) {
        return rabs(prm[0]);
    } else if constexpr (DYN == TRANSLATE) {
        return rabs(prm[k]);
    } else if constexpr (DYN == QUADRATIC) {
        return rmax(rabs(pm), rabs(pp));
    } else if constexpr (DYN == AIR3D) {
        if (k == 0) return rfma(prm[2], rabs(x[1]), rabs(rfma(prm[1], c, -prm[0])));
        if (k == 1) return rfma(prm[2], rabs(x[0]), prm[1] * rabs(s));
        return prm[2] + prm[3];
    } else if constexpr (DYN == CAR4D) {
        if (k == 0) return rabs(x[3] * c);
        if (k == 1) return rabs(x[3] * s);
        if (k == 2) return prm[0];
        return prm[1];
    } else if constexpr (DYN == ROCKETS) {
        if (k == 0) return rfma(prm[2], rabs(x[0]), rabs(prm[0] * c));
        if (k == 1) return rfma(prm[3], rabs(x[0]), rabs(rfma(prm[0], s, prm[0] - prm[1])));
        return prm[2] + prm[3];
    } else {  // DOUBLE_INT
        return k == 0 ? rabs(x[1]) : rabs(prm[0]);
    }
}

// Per-node bound on |dH/dp_k| for state-only bounds (FP64, used once per
// grid by the reduction that yields the global-LF coefficients).
template <int DYN>
__device__ __forceinline__ double partial_bound(const double* x, int k, const double* prm)
{
    if constexpr (DYN == NORMAL_SPEED) {
        return fabs(prm[0]);  // |dH/dp_k| = |a| |p_k| / |p| <= |a|
    } else if constexpr (DYN == TRANSLATE) {
        return fabs(prm[k]);
    } else if constexpr (DYN == AIR3D) {
        double s, c;
        sincos(x[2], &s, &c);
        if (k == 0) return fabs(-prm[0] + prm[1] * c) + prm[2] * fabs(x[1]);
        if (k == 1) return prm[1] * fabs(s) + prm[2] * fabs(x[0]);
        return prm[2] + prm[3];
    } else if constexpr (DYN == CAR4D) {
        double s, c;
        sincos(x[2], &s, &c);
        if (k == 0) return fabs(x[3] * c);
        if (k == 1) return fabs(x[3] * s);
        if (k == 2) return prm[0];
        return prm[1];
    } else if constexpr (DYN == ROCKETS) {
        double s, c;
        sincos(x[2], &s, &c);
        if (k == 0) return prm[0] * fabs(c) + prm[2] * fabs(x[0]);
        if (k == 1) return fabs(prm[0] * s + prm[0] - prm[1]) + prm[3] * fabs(x[0]);
        return prm[2] + prm[3];
    } else if constexpr (DYN == DOUBLE_INT) {
        return k == 0 ? fabs(x[1]) : fabs(prm[0]);
    } else {
        return 0.0;
    }
}

// ---------------------------------------------------------------------------
// Ghost-cell substitution for a window along one axis (Sec. III-B): the
// value at axis coordinate j = i + o; periodic axes wrap, other axes
// extrapolate linearly from the two boundary nodes.
template <typename R, int G>
__device__ __forceinline__ void load_window(const R* __restrict__ phi, long long base, int i, int n,
                                            int s, int periodic, R* u)
{
#pragma unroll
    for (int o = -G; o <= G; ++o) {
        const int j = i + o;
        R v;
        if (j >= 0 && j < n) {
            v = __ldg(phi + base + (long long)o * s);
        } else if (periodic) {
            const int jj = (j < 0) ? j + n : j - n;
            v = __ldg(phi + base + (long long)(jj - i) * s);
        } else if (j < 0) {
            const R u0 = __ldg(phi + base - (long long)i * s);
            const R u1 = __ldg(phi + base - (long long)i * s + s);
            v = u0 + R(-j) * (u0 - u1);
        } else {
            const R un = __ldg(phi + base + (long long)(n - 1 - i) * s);
            const R um = __ldg(phi + base + (long long)(n - 2 - i) * s);
            v = un + R(j - n + 1) * (un - um);
        }
        u[o + G] = v;
    }
}

}  // namespace lsp
