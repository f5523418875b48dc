// pair2.cuh -- two FP32 values carried together through Blackwell's paired
// FP32 instructions (FADD2 / FMUL2 / FFMA2: one issue, two results).  Used to
// evaluate the same stencil at two nodes at once (two consecutive planes of
// the march), halving the issued FP32 instructions of the WENO5 and ENO
// arithmetic (the ENO stencil choices stay per component).
#pragma once
#include <cuda_runtime.h>

namespace lsp {

struct F2 {
    float2 v;
    __device__ __forceinline__ F2() {}
    __device__ __forceinline__ explicit F2(float2 x) : v(x) {}
    __device__ __forceinline__ F2(float a) : v(make_float2(a, a)) {}
    __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
    __device__ __forceinline__ float x() const { return v.x; }
    __device__ __forceinline__ float y() const { return v.y; }
};

__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2(__fmul2_rn(a.v, b.v)); }
// a - b as one paired FMA: b * (-1) + a is exact
__device__ __forceinline__ F2 operator-(F2 a, F2 b)
{
    return F2(__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v));
}
__device__ __forceinline__ F2 operator-(F2 a) { return F2(__fmul2_rn(a.v, make_float2(-1.f, -1.f))); }
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ F2 max2(F2 a, F2 b) { return F2(fmaxf(a.v.x, b.v.x), fmaxf(a.v.y, b.v.y)); }
__device__ __forceinline__ F2 min2(F2 a, F2 b) { return F2(fminf(a.v.x, b.v.x), fminf(a.v.y, b.v.y)); }
__device__ __forceinline__ F2 abs2(F2 a) { return F2(fabsf(a.v.x), fabsf(a.v.y)); }
__device__ __forceinline__ F2 sqrt2(F2 a) { return F2(sqrtf(a.v.x), sqrtf(a.v.y)); }

// The paired WENO5 works with scaled copies of the quantities of
// deriv_weno5_jp (stage_tiled.cuh), each scaling exact in real arithmetic:
//  - a third of each smoothness indicator, is/3 = (13/3) (.)^2 + f^2, with
//    the regulariser scaled alike (e/3 = 4e-6 max d^2 + 4 floor): the
//    weights depend only on the ratios (is_k + e)/(is_l + e);
//  - six times each correction, 6 Phi = r (2 Q12 A + 3 Q01 B) - B/2 with
//    r = 1/P (w0 = Q12 r, w2 = 3 Q01 r substituted into
//    Phi = w0 A/3 + (w2 - 1/2) B/6), and six times the centred term,
//    6 cen = (7 (d_{-1} + d_0) - (d_{-2} + d_1)) / 2; the stage body takes
//    the 1/6 out after the Hamiltonian (see tiled_pair_body).
// The values agree with the scalar form to FP32 rounding.

// 6 Phi for two nodes from the scaled indicators, the regulariser, 2A and
// -B/2 (same exact power-of-two rescaling of the squares, per component).
__device__ __forceinline__ F2 weno_phi2(F2 is0, F2 is1, F2 is2, F2 e, F2 A2, F2 nB2, F2 B)
{
    const F2 sc(__uint_as_float(0x7f000000u - (__float_as_uint(e.v.x) & 0x7f800000u)),
                __uint_as_float(0x7f000000u - (__float_as_uint(e.v.y) & 0x7f800000u)));
    // (is + e) sc as fma(is, sc, e sc): the same value (sc is a power of two)
    const F2 esc = e * sc;
    const F2 q0 = fma2(is0, sc, esc), q1 = fma2(is1, sc, esc), q2 = fma2(is2, sc, esc);
    const F2 Q0 = q0 * q0, Q1 = q1 * q1, Q2 = q2 * q2;
    const F2 Q12 = Q1 * Q2, Q01 = Q0 * Q1, t01 = F2(3.0f) * Q01;
    const F2 P = fma2(F2(6.0f) * Q0, Q2, t01 + Q12);
    const F2 r(__fdividef(1.0f, P.v.x), __fdividef(1.0f, P.v.y));
    return fma2(r, fma2(t01, B, Q12 * A2), nB2);
}

// The parts of deriv_weno5_jp for two nodes: u[o] holds the window values
// at offset o-3 of both nodes; floor4 = 4 x the regulariser floor.  Returns
// 6 cen, 6 phim and 6 phip (p- = (cen - phim) / dx, p+ = (cen + phip) / dx;
// the caller combines them, see lf_axis2).
__device__ __forceinline__ void weno5_jp2(const F2* u, float floor4, F2& cen6, F2& phim6, F2& phip6)
{
    const F2 dm3 = u[1] - u[0], dm2 = u[2] - u[1], dm1 = u[3] - u[2];
    const F2 d0 = u[4] - u[3], d1 = u[5] - u[4], d2 = u[6] - u[5];
    const F2 Sm2 = dm2 - dm3, Sm1 = dm1 - dm2, S0 = d0 - dm1, S1 = d1 - d0, S2 = d2 - d1;
    // from its negation: fma(-7, x, y) is exactly -fma(7, x, -y), so no
    // paired negation is issued
    cen6 = fma2(F2(-7.0f), dm1 + d0, dm2 + d1) * F2(-0.5f);
    // max_k d_k^2 as (max_k |d_k|)^2: squaring rounds monotonically on
    // [0, inf), so the two are the same number; the max runs on the ALU
    const F2 m4 = max2(max2(abs2(dm2), abs2(dm1)), max2(abs2(d0), abs2(d1)));
    const F2 mL = max2(m4, abs2(dm3)), mR = max2(m4, abs2(d2));
    const F2 eL = fma2(F2(4e-6f), mL * mL, F2(floor4));
    const F2 eR = fma2(F2(4e-6f), mR * mR, F2(floor4));
    const F2 g1 = Sm2 - Sm1, g2 = Sm1 - S0, g3 = S0 - S1, g4 = S1 - S2;
    const F2 e1 = g1 * g1, e2 = g2 * g2, e3 = g3 * g3, e4 = g4 * g4;
    // f2m and f2p enter only squared: their negations -(3 S0 - S1) and
    // -(3 S0 - Sm1) are one FMA each and give the same squares
    const F2 f0m = fma2(F2(-3.0f), Sm1, Sm2), f1m = Sm1 + S0, f2m = fma2(F2(-3.0f), S0, S1);
    const F2 f0p = fma2(F2(-3.0f), S1, S2), f1p = S1 + S0, f2p = fma2(F2(-3.0f), S0, Sm1);
    const F2 k13(13.0f / 3.0f);
    const F2 is0m = fma2(k13, e1, f0m * f0m);
    const F2 is1m = fma2(k13, e2, f1m * f1m);
    const F2 is2m = fma2(k13, e3, f2m * f2m);
    const F2 is0p = fma2(k13, e4, f0p * f0p);
    const F2 is1p = fma2(k13, e3, f1p * f1p);
    const F2 is2p = fma2(k13, e2, f2p * f2p);
    const F2 two(2.0f);
    const F2 Tm1 = fma2(-two, Sm1, Sm2 + S0), T0 = fma2(-two, S0, Sm1 + S1);
    const F2 T1 = fma2(-two, S1, S0 + S2);
    const F2 nT0h = T0 * F2(-0.5f);
    phim6 = weno_phi2(is0m, is1m, is2m, eL, Tm1 + Tm1, nT0h, T0);
    phip6 = weno_phi2(is0p, is1p, is2p, eR, T1 + T1, nT0h, T0);
}

// One axis' share of the LF rate (Sec. IV-D) from the parts of its WENO5
// derivatives: the central costate (p+ + p-)/2 = (cen + (phip - phim)/2)/dx
// and the dissipation alpha (p+ - p-)/2 = alpha/(2 dx) (phip + phim), added
// to diss; sx = 1/dx, hax = alpha/(2 dx).  With the parts multiplied by 6
// both results are 6 x theirs.  The centred term cancels from the
// difference instead of being subtracted after rounding.
__device__ __forceinline__ void lf_axis2(F2 cen6, F2 phim6, F2 phip6, F2 sx, F2 hax, F2& pbar6,
                                         F2& diss6)
{
    pbar6 = fma2(F2(0.5f), phip6 - phim6, cen6) * sx;
    diss6 = fma2(hax, phip6 + phim6, diss6);
}

// The two WENO5 corrections that share the face between nodes j and j+1,
// from the six values v[o] = phi_{j-2+o}: phim6 for the left-biased
// derivative at node j+1 and phip6 for the right-biased derivative at node j
// (scaled as in weno5_jp2).  Both sides of a face see the same five first
// differences, so their smoothness indicators are the same three numbers in
// reversed order and their regulariser is the same; everything up to the
// squared scaled indicators is computed once.  Each result is bit-identical
// to the corresponding weno_phi2 call of weno5_jp2 (the same operations on
// the same operands: negated FMAs round symmetrically and products commute).
// cen6_j receives 6 x the centred term of node j.
__device__ __forceinline__ void weno5_face2(const F2* v, float floor4, F2& phim6, F2& phip6,
                                            F2& cen6_j)
{
    const F2 da = v[1] - v[0], db = v[2] - v[1], dc = v[3] - v[2];
    const F2 dd = v[4] - v[3], de = v[5] - v[4];
    cen6_j = fma2(F2(-7.0f), db + dc, da + dd) * F2(-0.5f);  // as in weno5_jp2
    // second differences S_{j-1} .. S_{j+2}
    const F2 Sa = db - da, Sb = dc - db, Sc = dd - dc, Sd = de - dd;
    const F2 m5 = max2(max2(max2(abs2(db), abs2(dc)), max2(abs2(dd), abs2(de))), abs2(da));
    const F2 e = fma2(F2(4e-6f), m5 * m5, F2(floor4));
    const F2 g1 = Sa - Sb, g2 = Sb - Sc, g3 = Sc - Sd;
    const F2 e1 = g1 * g1, e2 = g2 * g2, e3 = g3 * g3;
    const F2 f0 = fma2(F2(-3.0f), Sb, Sa), f1 = Sb + Sc, f2 = fma2(F2(-3.0f), Sc, Sd);
    const F2 k13(13.0f / 3.0f), two(2.0f);
    const F2 b0 = fma2(k13, e1, f0 * f0);
    const F2 b1 = fma2(k13, e2, f1 * f1);
    const F2 b2 = fma2(k13, e3, f2 * f2);
    const F2 Tj = fma2(-two, Sb, Sa + Sc), Tj1 = fma2(-two, Sc, Sb + Sd);
    const F2 sc(__uint_as_float(0x7f000000u - (__float_as_uint(e.v.x) & 0x7f800000u)),
                __uint_as_float(0x7f000000u - (__float_as_uint(e.v.y) & 0x7f800000u)));
    const F2 esc = e * sc;
    const F2 q0 = fma2(b0, sc, esc), q1 = fma2(b1, sc, esc), q2 = fma2(b2, sc, esc);
    const F2 Q0 = q0 * q0, Q1 = q1 * q1, Q2 = q2 * q2;
    const F2 Q12 = Q1 * Q2, Q01 = Q0 * Q1;
    // left-biased side of node j+1: indicators (b0, b1, b2), A = T_j, B = T_{j+1}
    const F2 t01 = F2(3.0f) * Q01;
    const F2 Pm = fma2(F2(6.0f) * Q0, Q2, t01 + Q12);
    const F2 rm(__fdividef(1.0f, Pm.v.x), __fdividef(1.0f, Pm.v.y));
    phim6 = fma2(rm, fma2(t01, Tj1, Q12 * (Tj + Tj)), Tj1 * F2(-0.5f));
    // right-biased side of node j: indicators (b2, b1, b0), A = T_{j+1}, B = T_j
    const F2 t12 = F2(3.0f) * Q12;
    const F2 Pp = fma2(F2(6.0f) * Q2, Q0, t12 + Q01);
    const F2 rp(__fdividef(1.0f, Pp.v.x), __fdividef(1.0f, Pp.v.y));
    phip6 = fma2(rp, fma2(t12, Tj, Q01 * (Tj1 + Tj1)), Tj * F2(-0.5f));
}

// x or y per component: a where |ka| <= |kb|, else b (ties to a, as the
// scalar ENO choices)
__device__ __forceinline__ F2 sel_smaller2(F2 ka, F2 kb, F2 a, F2 b)
{
    return F2(fabsf(ka.v.x) <= fabsf(kb.v.x) ? a.v.x : b.v.x,
              fabsf(ka.v.y) <= fabsf(kb.v.y) ? a.v.y : b.v.y);
}

// deriv_eno2 for two nodes (stencil choices per component), as dx p- and
// dx p+: am = d_{-1} + S_c / 2, ap = d_0 - S_c / 2.
__device__ __forceinline__ void eno2_parts2(const F2* u, F2& am, F2& ap)
{
    const F2 dm2 = u[1] - u[0], dm1 = u[2] - u[1], d0 = u[3] - u[2], d1 = u[4] - u[3];
    const F2 Sm1 = dm1 - dm2, S0 = d0 - dm1, S1 = d1 - d0;
    am = fma2(F2(0.5f), sel_smaller2(Sm1, S0, Sm1, S0), dm1);
    ap = fma2(F2(-0.5f), sel_smaller2(S0, S1, S0, S1), d0);
}

// deriv_eno3 for two nodes (stencil choices per component), as dx p- and
// dx p+; the cubic factor f/6 of the chosen base index is 1/3 (s = 2, f = 2)
// or -1/6 (s = 1, f = -1).
__device__ __forceinline__ void eno3_parts2(const F2* u, F2& am, F2& ap)
{
    const F2 dm3 = u[1] - u[0], dm2 = u[2] - u[1], dm1 = u[3] - u[2];
    const F2 d0 = u[4] - u[3], d1 = u[5] - u[4], d2 = u[6] - u[5];
    const F2 Sm2 = dm2 - dm3, Sm1 = dm1 - dm2, S0 = d0 - dm1, S1 = d1 - d0, S2 = d2 - d1;
    const F2 Tm2 = Sm1 - Sm2, Tm1 = S0 - Sm1, T0 = S1 - S0, T1 = S2 - S1;
    {  // left derivative, k = i-1: base i-2 (s = 2) if |S_-1| <= |S_0|, else i-1 (s = 1)
        const bool lx = fabsf(Sm1.v.x) <= fabsf(S0.v.x), ly = fabsf(Sm1.v.y) <= fabsf(S0.v.y);
        const F2 c(lx ? Sm1.v.x : S0.v.x, ly ? Sm1.v.y : S0.v.y);
        const F2 ta(lx ? Tm2.v.x : Tm1.v.x, ly ? Tm2.v.y : Tm1.v.y);
        const F2 tb(lx ? Tm1.v.x : T0.v.x, ly ? Tm1.v.y : T0.v.y);
        const F2 f6(lx ? 1.0f / 3.0f : -1.0f / 6.0f, ly ? 1.0f / 3.0f : -1.0f / 6.0f);
        am = fma2(sel_smaller2(ta, tb, ta, tb), f6, fma2(F2(0.5f), c, dm1));
    }
    {  // right derivative, k = i: base i-1 (s = 1) if |S_0| <= |S_1|, else i (s = 0)
        const bool rx = fabsf(S0.v.x) <= fabsf(S1.v.x), ry = fabsf(S0.v.y) <= fabsf(S1.v.y);
        const F2 c(rx ? S0.v.x : S1.v.x, ry ? S0.v.y : S1.v.y);
        const F2 ta(rx ? Tm1.v.x : T0.v.x, ry ? Tm1.v.y : T0.v.y);
        const F2 tb(rx ? T0.v.x : T1.v.x, ry ? T0.v.y : T1.v.y);
        const F2 f6(rx ? -1.0f / 6.0f : 1.0f / 3.0f, ry ? -1.0f / 6.0f : 1.0f / 3.0f);
        ap = fma2(sel_smaller2(ta, tb, ta, tb), f6, fma2(F2(-0.5f), c, d0));
    }
}

}  // namespace lsp
