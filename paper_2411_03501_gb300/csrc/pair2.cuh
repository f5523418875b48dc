// pair2.cuh -- two FP32 values carried together through Blackwell's paired
// FP32 instructions (FADD2 / FMUL2 / FFMA2: one issue, two results).  Used to
// evaluate the same stencil at two nodes at once (two consecutive planes of
// the march), halving the issued FP32 instructions of the WENO5 arithmetic.
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

// Jiang-Peng Phi of deriv_weno5_jp for two nodes (same formulas and the same
// exact power-of-two rescaling, per component).
__device__ __forceinline__ F2 weno_phi2(F2 is0, F2 is1, F2 is2, F2 e, F2 A, F2 B)
{
    const F2 sc(__uint_as_float(0x7f000000u - (__float_as_uint(e.v.x) & 0x7f800000u)),
                __uint_as_float(0x7f000000u - (__float_as_uint(e.v.y) & 0x7f800000u)));
    // (is + e) sc as fma(is, sc, e sc): the same value (sc is a power of two)
    const F2 esc = e * sc;
    const F2 q0 = fma2(is0, sc, esc), q1 = fma2(is1, sc, esc), q2 = fma2(is2, sc, esc);
    const F2 Q0 = q0 * q0, Q1 = q1 * q1, Q2 = q2 * q2;
    const F2 Q12 = Q1 * Q2, Q01 = Q0 * Q1;
    const F2 P = fma2(F2(6.0f) * Q0, Q2, fma2(F2(3.0f), Q01, Q12));
    const F2 r(__fdividef(1.0f, P.v.x), __fdividef(1.0f, P.v.y));
    const F2 w0 = Q12 * r, w2 = F2(3.0f) * Q01 * r;
    return fma2(w0 * F2(1.0f / 3.0f), A, (w2 - F2(0.5f)) * (B * F2(1.0f / 6.0f)));
}

// The parts of deriv_weno5_jp for two nodes: u[o] holds the window values
// at offset o-3 of both nodes; p- = (cen - phim) / dx, p+ = (cen + phip) / dx
// (the caller combines them, see lf_axis2).
__device__ __forceinline__ void weno5_jp2(const F2* u, float floor12, F2& cen, F2& phim, F2& phip)
{
    const F2 dm3 = u[1] - u[0], dm2 = u[2] - u[1], dm1 = u[3] - u[2];
    const F2 d0 = u[4] - u[3], d1 = u[5] - u[4], d2 = u[6] - u[5];
    const F2 Sm2 = dm2 - dm3, Sm1 = dm1 - dm2, S0 = d0 - dm1, S1 = d1 - d0, S2 = d2 - d1;
    // (7 (dm1 + d0) - (dm2 + d1)) / 12 from its negation: fma(-7, x, y) is
    // exactly -fma(7, x, -y), and the product of two negated factors rounds
    // like the plain one (no paired negation is issued)
    cen = fma2(F2(-7.0f), dm1 + d0, dm2 + d1) * F2(-1.0f / 12.0f);
    // max_k d_k^2 as (max_k |d_k|)^2: squaring rounds monotonically on
    // [0, inf), so the two are the same number; the max runs on the ALU
    const F2 m4 = max2(max2(abs2(dm2), abs2(dm1)), max2(abs2(d0), abs2(d1)));
    const F2 mL = max2(m4, abs2(dm3)), mR = max2(m4, abs2(d2));
    const F2 eL = fma2(F2(1.2e-5f), mL * mL, F2(floor12));
    const F2 eR = fma2(F2(1.2e-5f), mR * mR, F2(floor12));
    const F2 g1 = Sm2 - Sm1, g2 = Sm1 - S0, g3 = S0 - S1, g4 = S1 - S2;
    const F2 e1 = g1 * g1, e2 = g2 * g2, e3 = g3 * g3, e4 = g4 * g4;
    // f2m and f2p enter only squared: their negations -(3 S0 - S1) and
    // -(3 S0 - Sm1) are one FMA each and give the same squares
    const F2 f0m = fma2(F2(-3.0f), Sm1, Sm2), f1m = Sm1 + S0, f2m = fma2(F2(-3.0f), S0, S1);
    const F2 f0p = fma2(F2(-3.0f), S1, S2), f1p = S1 + S0, f2p = fma2(F2(-3.0f), S0, Sm1);
    const F2 three(3.0f), thirteen(13.0f);
    const F2 is0m = fma2(thirteen, e1, three * f0m * f0m);
    const F2 is1m = fma2(thirteen, e2, three * f1m * f1m);
    const F2 is2m = fma2(thirteen, e3, three * f2m * f2m);
    const F2 is0p = fma2(thirteen, e4, three * f0p * f0p);
    const F2 is1p = fma2(thirteen, e3, three * f1p * f1p);
    const F2 is2p = fma2(thirteen, e2, three * f2p * f2p);
    const F2 two(2.0f);
    const F2 Tm1 = fma2(-two, Sm1, Sm2 + S0), T0 = fma2(-two, S0, Sm1 + S1);
    const F2 T1 = fma2(-two, S1, S0 + S2);
    phim = weno_phi2(is0m, is1m, is2m, eL, Tm1, T0);
    phip = weno_phi2(is0p, is1p, is2p, eR, T1, T0);
}

// One axis' share of the LF rate (Sec. IV-D) from the parts of its WENO5
// derivatives: the central costate (p+ + p-)/2 = (cen + (phip - phim)/2)/dx
// and the dissipation alpha (p+ - p-)/2 = alpha/(2 dx) (phip + phim), added
// to diss; hax = alpha/(2 dx).  The centred term cancels from the
// difference instead of being subtracted after rounding, and the pair costs
// five paired instructions instead of eight.
__device__ __forceinline__ void lf_axis2(F2 cen, F2 phim, F2 phip, F2 sx, F2 hax, F2& pbar,
                                         F2& diss)
{
    pbar = fma2(F2(0.5f), phip - phim, cen) * sx;
    diss = fma2(hax, phip + phim, diss);
}

// The two WENO5 corrections that share the face between nodes j and j+1,
// from the six values v[o] = phi_{j-2+o}: phim for the left-biased
// derivative at node j+1 and phip for the right-biased derivative at node j.
// Both sides of a face see the same five first differences, so their
// smoothness indicators are the same three numbers in reversed order and
// their regulariser is the same; everything up to the squared scaled
// indicators is computed once.  Each result is bit-identical to the
// corresponding weno_phi2 call of weno5_jp2 (the same operations on the
// same operands: negated FMAs round symmetrically, products commute, and the
// scaling by an exact power of two commutes with rounding, so
// fma(is, sc, e*sc) == (is + e) * sc).  cen receives the centred term of
// node j (x: (7 (d_{j-1} + d_j) - (d_{j-2} + d_{j+1})) / 12).
__device__ __forceinline__ void weno5_face2(const F2* v, float floor12, F2& phim, F2& phip,
                                            F2& cen_j)
{
    const F2 da = v[1] - v[0], db = v[2] - v[1], dc = v[3] - v[2];
    const F2 dd = v[4] - v[3], de = v[5] - v[4];
    cen_j = fma2(F2(-7.0f), db + dc, da + dd) * F2(-1.0f / 12.0f);  // as in weno5_jp2
    // second differences S_{j-1} .. S_{j+2}
    const F2 Sa = db - da, Sb = dc - db, Sc = dd - dc, Sd = de - dd;
    const F2 m5 = max2(max2(max2(abs2(db), abs2(dc)), max2(abs2(dd), abs2(de))), abs2(da));
    const F2 e = fma2(F2(1.2e-5f), m5 * m5, F2(floor12));
    const F2 g1 = Sa - Sb, g2 = Sb - Sc, g3 = Sc - Sd;
    const F2 e1 = g1 * g1, e2 = g2 * g2, e3 = g3 * g3;
    const F2 f0 = fma2(F2(-3.0f), Sb, Sa), f1 = Sb + Sc, f2 = fma2(F2(-3.0f), Sc, Sd);
    const F2 three(3.0f), thirteen(13.0f), two(2.0f);
    const F2 b0 = fma2(thirteen, e1, three * f0 * f0);
    const F2 b1 = fma2(thirteen, e2, three * f1 * f1);
    const F2 b2 = fma2(thirteen, e3, three * f2 * f2);
    const F2 Tj = fma2(-two, Sb, Sa + Sc), Tj1 = fma2(-two, Sc, Sb + Sd);
    const F2 sc(__uint_as_float(0x7f000000u - (__float_as_uint(e.v.x) & 0x7f800000u)),
                __uint_as_float(0x7f000000u - (__float_as_uint(e.v.y) & 0x7f800000u)));
    const F2 esc = e * sc;
    const F2 q0 = fma2(b0, sc, esc), q1 = fma2(b1, sc, esc), q2 = fma2(b2, sc, esc);
    const F2 Q0 = q0 * q0, Q1 = q1 * q1, Q2 = q2 * q2;
    const F2 Q12 = Q1 * Q2, Q01 = Q0 * Q1;
    // left-biased side of node j+1: indicators (b0, b1, b2), A = T_j, B = T_{j+1}
    const F2 Pm = fma2(F2(6.0f) * Q0, Q2, fma2(three, Q01, Q12));
    const F2 rm(__fdividef(1.0f, Pm.v.x), __fdividef(1.0f, Pm.v.y));
    const F2 w0m = Q12 * rm, w2m = three * Q01 * rm;
    phim = fma2(w0m * F2(1.0f / 3.0f), Tj, (w2m - F2(0.5f)) * (Tj1 * F2(1.0f / 6.0f)));
    // right-biased side of node j: indicators (b2, b1, b0), A = T_{j+1}, B = T_j
    const F2 Pp = fma2(F2(6.0f) * Q2, Q0, fma2(three, Q12, Q01));
    const F2 rp(__fdividef(1.0f, Pp.v.x), __fdividef(1.0f, Pp.v.y));
    const F2 w0p = Q01 * rp, w2p = three * Q12 * rp;
    phip = fma2(w0p * F2(1.0f / 3.0f), Tj1, (w2p - F2(0.5f)) * (Tj * F2(1.0f / 6.0f)));
}

}  // namespace lsp
