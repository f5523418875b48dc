// adjoint.cuh -- reverse of one fused Runge-Kutta stage.
//
// Forward stage (stage_generic.cuh / stage_tiled.cuh):
//   v   = c_n phi^n + c_s u + c_l dt L(u),   out = min(v, g) in a tube stage
//   L_i = -H(x_i, pbar_i) + sum_k alpha_k (p+_k,i - p-_k,i) / 2
// Given lam = dLoss/dout, the reverse gives dLoss/du, dLoss/dphi^n,
// dLoss/dg and the sensitivities to the dynamics parameters, alpha and dt.
// Every selection the forward made (ENO stencils, the argmax inside the WENO
// regulariser, the signs of the optimal inputs, the min with the target) is
// recomputed from the same stage input and frozen; the smooth remainder --
// WENO weights included -- is differentiated exactly.
//
// Two passes per stage.  Pass A (one thread per node i) recomputes the
// node's forward quantities, forms the weighted sensitivities of p+-_k,i and
// stores, per axis, the 7 coefficients c_k,i[o] = dLoss/du at window offset
// o; window positions that fall on ghost cells of an extrapolated axis are
// folded onto their boundary nodes right away (atomics, boundary nodes only).
// Pass B (node j) gathers sum_k sum_o c_k,(j-o e_k)[o] (periodic axes wrap)
// -- deterministic, no atomics on the interior.  Pass B of a stage needs
// only the node's own values besides the coefficients, and it yields the
// node's dLoss/dout of the stage reversed next, which is all that stage's
// pass A needs at the node: adj_stage_a runs the later stage's pass B and
// this stage's pass A in one launch (two coefficient buffers, alternating);
// adj_stage_b runs the last stage's pass B alone.
#pragma once
#include "stage_generic.cuh"
#include "stage_tiled.cuh"

namespace lsp {

// ---------------------------------------------------------------------------
// Window gradients: gm[o], gp[o] = d p-/du[o], d p+/du[o], o = 0..6 for the
// window offsets -3..3 (the stencils of G < 3 use the middle entries).

template <typename R>
__device__ __forceinline__ void grad_upwind1(R inv_dx, R* gm, R* gp)
{
    gm[2] += -inv_dx; gm[3] += inv_dx;
    gp[3] += -inv_dx; gp[4] += inv_dx;
}

// ENO2/ENO3 on the window u[0..6] (offset -3..3): the same unscaled
// differences and the same comparisons as deriv_eno2 / deriv_eno3, so the
// frozen stencil is the forward's; the derivative is then a fixed linear
// combination of window values.
template <typename R>
__device__ __forceinline__ void add_D(R* g, int m, R w)  // D_m = u_{m+1} - u_m
{
    g[m + 4] += w; g[m + 3] -= w;
}
template <typename R>
__device__ __forceinline__ void add_S(R* g, int m, R w)  // S_m = u_{m+1} - 2u_m + u_{m-1}
{
    g[m + 4] += w; g[m + 3] -= R(2) * w; g[m + 2] += w;
}
template <typename R>
__device__ __forceinline__ void add_T(R* g, int m, R w)  // T_m = S_{m+1} - S_m
{
    add_S(g, m + 1, w); add_S(g, m, -w);
}

template <typename R, int ORDER>
__device__ __forceinline__ void grad_eno(const R* u7, R inv_dx, R* gm, R* gp)
{
    // unscaled differences at offsets, as in the forward kernels
    const R dm3 = u7[1] - u7[0], dm2 = u7[2] - u7[1], dm1 = u7[3] - u7[2];
    const R d0 = u7[4] - u7[3], d1 = u7[5] - u7[4], d2 = u7[6] - u7[5];
    const R Sm2 = dm2 - dm3, Sm1 = dm1 - dm2, S0 = d0 - dm1, S1 = d1 - d0, S2 = d2 - d1;
    const R Tm2 = Sm1 - Sm2, Tm1 = S0 - Sm1, T0 = S1 - S0, T1 = S2 - S1;
    (void)Tm2; (void)T1;
    // left: p- = (d_-1 + S_c / 2 [+ T_c f / 6]) / dx
    add_D(gm, -1, inv_dx);
    if (rabs(Sm1) <= rabs(S0)) {
        add_S(gm, -1, R(0.5) * inv_dx);
        if (ORDER == 3) {
            if (rabs(Tm2) <= rabs(Tm1)) add_T(gm, -2, R(2.0 / 6.0) * inv_dx);
            else add_T(gm, -1, R(2.0 / 6.0) * inv_dx);
        }
    } else {
        add_S(gm, 0, R(0.5) * inv_dx);
        if (ORDER == 3) {
            if (rabs(Tm1) <= rabs(T0)) add_T(gm, -1, R(-1.0 / 6.0) * inv_dx);
            else add_T(gm, 0, R(-1.0 / 6.0) * inv_dx);
        }
    }
    // right: p+ = (d_0 - S_c / 2 [+ T_c f / 6]) / dx
    add_D(gp, 0, inv_dx);
    if (rabs(S0) <= rabs(S1)) {
        add_S(gp, 0, R(-0.5) * inv_dx);
        if (ORDER == 3) {
            if (rabs(Tm1) <= rabs(T0)) add_T(gp, -1, R(-1.0 / 6.0) * inv_dx);
            else add_T(gp, 0, R(-1.0 / 6.0) * inv_dx);
        }
    } else {
        add_S(gp, 1, R(-0.5) * inv_dx);
        if (ORDER == 3) {
            if (rabs(T0) <= rabs(T1)) add_T(gp, 0, R(2.0 / 6.0) * inv_dx);
            else add_T(gp, 1, R(2.0 / 6.0) * inv_dx);
        }
    }
}

// Gradient of the Jiang-Peng term Phi(a,b,c,d) (see deriv_weno5_jp) with
// respect to a, b, c, d and to the regulariser e:
//   Phi = w0 A + (w2 - 1/2) B,  A = (a - 2b + c)/3,  B = (b - 2c + d)/6,
//   w_k = C_k/(IS_k + e)^2 / sum_l C_l/(IS_l + e)^2,  C = (1, 6, 3),
//   dw_k = w_k (g_k - sum_l w_l g_l),  g_k = -2 (dIS_k + de)/(IS_k + e).
__device__ __forceinline__ void weno_phi_grad(double a, double b, double c, double d, double e,
                                              double* gabcd, double* ge)
{
    const double f0 = a - 3.0 * b, f1 = b + c, f2 = 3.0 * c - d;
    const double is0 = 13.0 * (a - b) * (a - b) + 3.0 * f0 * f0;
    const double is1 = 13.0 * (b - c) * (b - c) + 3.0 * f1 * f1;
    const double is2 = 13.0 * (c - d) * (c - d) + 3.0 * f2 * f2;
    const double q0 = is0 + e, q1 = is1 + e, q2 = is2 + e;
    // weights (the common scale of q cancels; 1/q^2 may be large, so form
    // ratios to the largest weight)
    const double r0 = 1.0 / q0, r1 = 1.0 / q1, r2 = 1.0 / q2;
    const double a0 = r0 * r0, a1 = 6.0 * r1 * r1, a2 = 3.0 * r2 * r2;
    const double inv = 1.0 / (a0 + a1 + a2);
    const double w0 = a0 * inv, w1 = a1 * inv, w2 = a2 * inv;
    const double A = (a - 2.0 * b + c) * (1.0 / 3.0), B = (b - 2.0 * c + d) * (1.0 / 6.0);
    const double E = A * w0 + B * w2;
    // coefficient of g_k in dPhi: gamma_k; times -2/q_k
    const double k0 = (A * w0 - w0 * E) * -2.0 * r0;
    const double k1 = (-w1 * E) * -2.0 * r1;
    const double k2 = (B * w2 - w2 * E) * -2.0 * r2;
    // dIS / d(a,b), d(b,c), d(c,d)
    const double i0a = 26.0 * (a - b) + 6.0 * f0, i0b = -26.0 * (a - b) - 18.0 * f0;
    const double i1b = 26.0 * (b - c) + 6.0 * f1, i1c = -26.0 * (b - c) + 6.0 * f1;
    const double i2c = 26.0 * (c - d) + 18.0 * f2, i2d = -26.0 * (c - d) - 6.0 * f2;
    gabcd[0] = w0 * (1.0 / 3.0) + k0 * i0a;
    gabcd[1] = w0 * (-2.0 / 3.0) + (w2 - 0.5) * (1.0 / 6.0) + k0 * i0b + k1 * i1b;
    gabcd[2] = w0 * (1.0 / 3.0) + (w2 - 0.5) * (-2.0 / 6.0) + k1 * i1c + k2 * i2c;
    gabcd[3] = (w2 - 0.5) * (1.0 / 6.0) + k2 * i2d;
    *ge = k0 + k1 + k2;
}

// FP32: the weights as the forward forms them (q_k scaled by a power of two
// close to 1/e, one reciprocal of P = Q1 Q2 + 6 Q0 Q2 + 3 Q0 Q1), and the
// three reciprocals 1/q_k from one reciprocal of q0 q1 q2 (the products stay
// below 1e24: IS_k <= 400 max D^2 while e >= 1.2e-5 max D^2).  Two
// approximate reciprocals in place of four divisions; the gradient's error
// stays a few FP32 ulps.
__device__ __forceinline__ void weno_phi_grad(float a, float b, float c, float d, float e,
                                              float* gabcd, float* ge)
{
    const float f0 = a - 3.0f * b, f1 = b + c, f2 = 3.0f * c - d;
    const float is0 = 13.0f * (a - b) * (a - b) + 3.0f * f0 * f0;
    const float is1 = 13.0f * (b - c) * (b - c) + 3.0f * f1 * f1;
    const float is2 = 13.0f * (c - d) * (c - d) + 3.0f * f2 * f2;
    const float sc = __uint_as_float(0x7f000000u - (__float_as_uint(e) & 0x7f800000u));
    const float q0 = (is0 + e) * sc, q1 = (is1 + e) * sc, q2 = (is2 + e) * sc;
    const float Q0 = q0 * q0, Q1 = q1 * q1, Q2 = q2 * q2;
    const float Q12 = Q1 * Q2, Q01 = Q0 * Q1, Q02 = Q0 * Q2;
    const float P = fmaf(6.0f * Q0, Q2, fmaf(3.0f, Q01, Q12));
    const float r = __fdividef(1.0f, P);
    const float w0 = Q12 * r, w1 = 6.0f * Q02 * r, w2 = 3.0f * Q01 * r;
    // sc / q_k = 1 / (IS_k + e)
    const float q12 = q1 * q2;
    const float rq = __fdividef(sc, q0 * q12);
    const float r0 = q12 * rq, r1 = q0 * q2 * rq, r2 = q0 * q1 * rq;
    const float A = (a - 2.0f * b + c) * (1.0f / 3.0f), B = (b - 2.0f * c + d) * (1.0f / 6.0f);
    const float E = A * w0 + B * w2;
    const float k0 = (A * w0 - w0 * E) * -2.0f * r0;
    const float k1 = (-w1 * E) * -2.0f * r1;
    const float k2 = (B * w2 - w2 * E) * -2.0f * r2;
    const float i0a = 26.0f * (a - b) + 6.0f * f0, i0b = -26.0f * (a - b) - 18.0f * f0;
    const float i1b = 26.0f * (b - c) + 6.0f * f1, i1c = -26.0f * (b - c) + 6.0f * f1;
    const float i2c = 26.0f * (c - d) + 18.0f * f2, i2d = -26.0f * (c - d) - 6.0f * f2;
    gabcd[0] = w0 * (1.0f / 3.0f) + k0 * i0a;
    gabcd[1] = w0 * (-2.0f / 3.0f) + (w2 - 0.5f) * (1.0f / 6.0f) + k0 * i0b + k1 * i1b;
    gabcd[2] = w0 * (1.0f / 3.0f) + (w2 - 0.5f) * (-2.0f / 6.0f) + k1 * i1c + k2 * i2c;
    gabcd[3] = (w2 - 0.5f) * (1.0f / 6.0f) + k2 * i2d;
    *ge = k0 + k1 + k2;
}

template <typename R>
__device__ __forceinline__ void grad_weno5(const R* u7, R inv_dx, R floor12, R* gm, R* gp)
{
    R D[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) D[m] = u7[m + 1] - u7[m];  // D[m] = D_{m-3}
    R S[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) S[j] = D[j + 1] - D[j];    // S[j] = S_{j-2}
    // the central part (shared by both sides): (-D_-2 + 7 D_-1 + 7 D_0 - D_1)/12
    const R cw[4] = {R(-1.0 / 12.0), R(7.0 / 12.0), R(7.0 / 12.0), R(-1.0 / 12.0)};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        add_D(gm, q - 2, cw[q] * inv_dx);
        add_D(gp, q - 2, cw[q] * inv_dx);
    }
    // regulariser e = 1.2e-5 max(D^2 over the side's five differences) + floor;
    // argmax frozen (the first of equal values).  The maxima are tracked by
    // value and the argmax only selects among unrolled updates, so that no
    // array is indexed at run time (that would place D, gm and gp in local
    // memory).
    int mL = 0, mR = 1;
    R DL = D[0], DL2 = D[0] * D[0], DR = D[1], DR2 = D[1] * D[1];
#pragma unroll
    for (int m = 1; m < 5; ++m) {
        const R q = D[m] * D[m];
        if (q > DL2) { DL2 = q; DL = D[m]; mL = m; }
    }
#pragma unroll
    for (int m = 2; m < 6; ++m) {
        const R q = D[m] * D[m];
        if (q > DR2) { DR2 = q; DR = D[m]; mR = m; }
    }
    const R eL = R(1.2e-5) * DL * DL + floor12;
    const R eR = R(1.2e-5) * DR * DR + floor12;
    R g4[4], ge;
    // p- = (cen - Phi(S_-2, S_-1, S_0, S_1)) / dx
    weno_phi_grad(S[0], S[1], S[2], S[3], eL, g4, &ge);
#pragma unroll
    for (int q = 0; q < 4; ++q) add_S(gm, q - 2, -g4[q] * inv_dx);
    const R wL = -ge * R(2.4e-5) * DL * inv_dx;
#pragma unroll
    for (int m = 0; m < 5; ++m)
        if (m == mL) add_D(gm, m - 3, wL);
    // p+ = (cen + Phi(S_2, S_1, S_0, S_-1)) / dx
    weno_phi_grad(S[4], S[3], S[2], S[1], eR, g4, &ge);
#pragma unroll
    for (int q = 0; q < 4; ++q) add_S(gp, 2 - q, g4[q] * inv_dx);
    const R wR = ge * R(2.4e-5) * DR * inv_dx;
#pragma unroll
    for (int m = 1; m < 6; ++m)
        if (m == mR) add_D(gp, m - 3, wR);
}

template <int SCHEME, typename R>
__device__ __forceinline__ void window_grad(const R* u7, R inv_dx, R floor12, R* gm, R* gp)
{
#pragma unroll
    for (int o = 0; o < 7; ++o) gm[o] = gp[o] = R(0);
    if constexpr (SCHEME == UPWIND1) grad_upwind1(inv_dx, gm, gp);
    else if constexpr (SCHEME == ENO2) grad_eno<R, 2>(u7, inv_dx, gm, gp);
    else if constexpr (SCHEME == ENO3) grad_eno<R, 3>(u7, inv_dx, gm, gp);
    else grad_weno5(u7, inv_dx, floor12, gm, gp);
}

// ---------------------------------------------------------------------------
// dH/dp_k (frozen input selections, sign(0) = +1) and dH/dprm_j.
__device__ __forceinline__ float sgn1(float v) { return v >= 0.f ? 1.f : -1.f; }
__device__ __forceinline__ double sgn1(double v) { return v >= 0.0 ? 1.0 : -1.0; }

template <int DYN, int NDIM, typename R>
__device__ __forceinline__ void ham_grad(const R* x, const R* p, const R* prm, R s, R c, R* hp,
                                         R* hprm)
{
#pragma unroll
    for (int j = 0; j < 4; ++j) hprm[j] = R(0);
    if constexpr (DYN == NORMAL_SPEED) {
        R n2 = R(0);
#pragma unroll
        for (int k = 0; k < NDIM; ++k) n2 += p[k] * p[k];
        const R n = real_sqrt(n2);
#pragma unroll
        for (int k = 0; k < NDIM; ++k) hp[k] = n > R(0) ? prm[0] * p[k] / n : R(0);
        hprm[0] = n;
    } else if constexpr (DYN == TRANSLATE) {
#pragma unroll
        for (int k = 0; k < NDIM; ++k) {
            hp[k] = prm[k];
            if (k < 4) hprm[k] = p[k];
        }
    } else if constexpr (DYN == AIR3D) {
        const R ve = prm[0], vp = prm[1], um = prm[2], dm = prm[3];
        const R s1 = p[0] * x[1] - p[1] * x[0] - p[2];
        const R g1 = sgn1(s1), g3 = sgn1(p[2]);
        hp[0] = -((-ve + vp * c) + um * g1 * x[1]);
        hp[1] = -(vp * s - um * g1 * x[0]);
        hp[2] = um * g1 + dm * g3;
        hprm[0] = p[0];
        hprm[1] = -(p[0] * c + p[1] * s);
        hprm[2] = -rabs(s1);
        hprm[3] = rabs(p[2]);
    } else if constexpr (DYN == CAR4D) {
        const R v = x[3];
        hp[0] = -v * c;
        hp[1] = -v * s;
        hp[2] = prm[0] * sgn1(p[2]);
        hp[3] = prm[1] * sgn1(p[3]);
        hprm[0] = rabs(p[2]);
        hprm[1] = rabs(p[3]);
    } else if constexpr (DYN == ROCKETS) {
        // H = -[p1 a cos th + p2 (a sin th + a - g) + ue |p1 x - p3| - up |p2 x + p3|];
        // the switching arguments as hamiltonian_rockets forms them, so the
        // frozen input signs are the forward's
        const R a = prm[0], g = prm[1], ue = prm[2], up = prm[3];
        const R s1 = rfma(p[0], x[0], -p[2]), s2 = rfma(p[1], x[0], p[2]);
        const R g1 = sgn1(s1), g2 = sgn1(s2);
        hp[0] = -rfma(ue * g1, x[0], a * c);
        hp[1] = -rfma(-up * g2, x[0], rfma(a, s, a - g));
        hp[2] = ue * g1 + up * g2;
        hprm[0] = -rfma(p[0], c, p[1] * (s + R(1)));
        hprm[1] = p[1];
        hprm[2] = -rabs(s1);
        hprm[3] = rabs(s2);
    } else if constexpr (DYN == DOUBLE_INT) {
        // H = -(p1 x2 - umax |p2|)
        hp[0] = -x[1];
        hp[1] = prm[0] * sgn1(p[1]);
        hprm[0] = rabs(p[1]);
    } else {
#pragma unroll
        for (int k = 0; k < NDIM; ++k) hp[k] = p[k];
    }
}

// ---------------------------------------------------------------------------
struct AdjAcc {        // FP64 accumulators (device)
    double hprm[4];    // sum_i w_i (-dH/dprm_j)
    double alpha[4];   // sum_i w_i (p+_k - p-_k)/2
    double dt;         // sum_i lam_v,i c_l L_i
    double pad[7];
};

template <typename R>
struct AdjArgs {
    const R* u;        // stage input (stencil)
    const R* phin;     // phi^n (pointwise; NULL when c_n == 0)
    const R* target;   // read when tube
    const R* lam;      // dLoss/d out
    R* lam_v;          // out: dLoss/dv per node
    R* contrib;        // out: 7 NDIM coefficient fields, field q = 7 k + (o + 3)
                       // (axis k, window offset o) at contrib + q * cstride
    long long cstride; // elements between coefficient fields
    R* lam_u;          // ghost folds (atomics) here; pass B adds the rest
    R* lam_n;          // pass B: += c_n lam_v (may equal lam_u)
    R* lam_g;          // tube: += lam where the min took the target (nullable)
    // Pass A only: the pass B of the stage reversed before this one, done
    // node by node in the same launch (gcontrib NULL: none, lam is read).
    // At node i it forms that stage's dLoss/du_i -- this stage's dLoss/dout_i
    // -- from glam_u[i] (then zeroed for reuse), its own lam_v[i] and the
    // neighbours' coefficients in gcontrib.
    const R* gcontrib; // the later stage's coefficient fields (not contrib)
    R* glam_u;         // the later stage's lam_u (never this stage's lam_u)
    R* glam_n;         // the later stage's lam_n (NULL or == glam_u: into the sum)
    R gc_s, gc_n;      // the later stage's c_s, c_n
    int gatomic;       // glam_n is this stage's fold target: add atomically
    AdjAcc* acc;
    int n[LSP_MAXD];
    int stride[LSP_MAXD];
    int periodic[LSP_MAXD];
    R inv_dx[LSP_MAXD];
    R lo[LSP_MAXD];
    R h[LSP_MAXD];
    R alpha[LSP_MAXD];
    R prm[LSP_NPARAM];
    R dt, c_n, c_s, c_l;
    int tube;
    int npts;
};

// sum over axes k and offsets o of the coefficient c_k,(i - o e_k)[o]: what
// node i's value contributed, through every window that contains it, to the
// stage's reverse (periodic axes wrap; positions beyond an extrapolated end
// were folded by pass A).  Added to acc in the order k, o.
template <int NDIM, typename R>
__device__ __forceinline__ R gather_coeffs(const AdjArgs<R>& a, const R* contrib, int idx,
                                           const int* c, R acc)
{
#pragma unroll
    for (int k = 0; k < NDIM; ++k) {
        const int n = a.n[k], s = a.stride[k];
        const R* ck = contrib + (long long)(7 * k + 3) * a.cstride + idx;  // offset 0
        if (c[k] >= 3 && c[k] < n - 3) {
#pragma unroll
            for (int o = -3; o <= 3; ++o) acc += ck[(long long)o * a.cstride - (long long)o * s];
            continue;
        }
#pragma unroll
        for (int o = -3; o <= 3; ++o) {
            int i = c[k] - o;  // the node whose window offset o is this node
            if (i < 0 || i >= n) {
                if (!a.periodic[k]) continue;
                i = i < 0 ? i + n : i - n;
            }
            acc += ck[(long long)o * a.cstride + (long long)(i - c[k]) * s];
        }
    }
    return acc;
}

// Asynchronous 4-byte copy global -> shared (cp.async): complete after
// adj_cp_wait() in the issuing thread.
__device__ __forceinline__ void adj_cp4(float* smem_dst, const float* gsrc)
{
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void adj_cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void adj_cp_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// FP32 pass A prefetches the gather of the next node it visits into shared
// memory while it computes the current one: per thread two slices of
// adj_gather_slots(NDIM) floats (lam_v, glam_u, then the 7 NDIM
// coefficients in gather order), slot q of slice b at [(b NQ + q) 256 + tid].
__host__ __device__ constexpr int adj_gather_slots(int ndim) { return 7 * ndim + 2; }
template <int NDIM, typename R>
__host__ __device__ constexpr size_t adj_a_smem_bytes() { return sizeof(R) == 4 ? 2 * adj_gather_slots(NDIM) * 256 * sizeof(float) : 0; }

// Element k of a small array, k known only at run time: a select over the
// compile-time indices (the array stays in registers).
template <int N, typename T>
__device__ __forceinline__ T pick(const T* arr, int k)
{
    T v = arr[0];
#pragma unroll
    for (int j = 1; j < N; ++j)
        if (k == j) v = arr[j];
    return v;
}
template <int N, typename T>
__device__ __forceinline__ void put(T* arr, int k, T v)
{
#pragma unroll
    for (int j = 0; j < N; ++j)
        if (k == j) arr[j] = v;
}

// 3 CTAs of 256 per SM in FP32: the kernel fits 80 registers without spills
// (left to itself the compiler takes 128 and runs 2 CTAs per SM; 64
// registers spill); FP64 (the oracle comparisons) keeps 2.
template <typename R>
constexpr int adj_a_min_blocks() { return sizeof(R) == 4 ? 3 : 2; }

template <int NDIM, int SCHEME, int DYN, typename R>
__global__ void __launch_bounds__(256, adj_a_min_blocks<R>()) adj_stage_a(AdjArgs<R> a)
{
    constexpr int G = ghost_width(SCHEME);
    // per-thread partial sums in the field precision (a thread visits a few
    // nodes), promoted to FP64 once for the block reduction: per-node FP64
    // arithmetic would run on GB300's slow FP64 pipe
    R acc_h[4] = {0, 0, 0, 0}, acc_a[4] = {0, 0, 0, 0}, acc_dt = R(0);
    // grid-stride loop with the node's coordinates advanced by the stride's
    // mixed-radix digits (one carry per axis) instead of divided out per node
    const int step = gridDim.x * blockDim.x;
    int c[NDIM], dc[NDIM];
    {
        int r = blockIdx.x * blockDim.x + threadIdx.x, q = step;
#pragma unroll
        for (int k = NDIM - 1; k >= 0; --k) {
            c[k] = r % a.n[k];
            r /= a.n[k];
            dc[k] = q % a.n[k];
            q /= a.n[k];
        }
        c[0] += r * a.n[0];  // a thread past the last node leaves at once
        dc[0] += q * a.n[0];
    }
    // the gather's operands of node pidx (coordinates pc) into slice buf
    constexpr bool kPF = sizeof(R) == 4;
    constexpr int NQ = adj_gather_slots(NDIM);
    extern __shared__ __align__(16) unsigned char adj_smem_raw[];
    float* slices = reinterpret_cast<float*>(adj_smem_raw) + threadIdx.x;
    auto prefetch = [&](int pidx, const int* pc, int buf) {
        if constexpr (kPF) {
            float* sl = slices + buf * NQ * 256;
            adj_cp4(sl, reinterpret_cast<const float*>(a.lam_v + pidx));
            adj_cp4(sl + 256, reinterpret_cast<const float*>(a.glam_u + pidx));
#pragma unroll
            for (int k = 0; k < NDIM; ++k) {
                const int n = a.n[k], s = a.stride[k];
                const float* ck =
                    reinterpret_cast<const float*>(a.gcontrib) + (long long)(7 * k + 3) * a.cstride + pidx;
                const bool inner = pc[k] >= 3 && pc[k] < n - 3;
#pragma unroll
                for (int o = -3; o <= 3; ++o) {
                    float* dst = sl + (2 + 7 * k + o + 3) * 256;
                    int i = pc[k] - o;
                    if (!inner && (i < 0 || i >= n)) {
                        if (!a.periodic[k]) {  // folded by the later stage's pass A
                            *dst = 0.0f;
                            continue;
                        }
                        i = i < 0 ? i + n : i - n;
                    }
                    adj_cp4(dst, ck + (long long)o * a.cstride + (long long)(i - pc[k]) * s);
                }
            }
            adj_cp_commit();
        }
    };
    const bool gather = a.gcontrib != nullptr;
    if (kPF && gather && blockIdx.x * blockDim.x + threadIdx.x < a.npts)
        prefetch(blockIdx.x * blockDim.x + threadIdx.x, c, 0);
    int it = 0;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < a.npts; idx += step, ++it) {
        // coordinates of the next node of this thread
        int cn[NDIM];
        {
            int carry = 0;
#pragma unroll
            for (int k = NDIM - 1; k >= 1; --k) {
                cn[k] = c[k] + dc[k] + carry;
                carry = cn[k] >= a.n[k];
                if (carry) cn[k] -= a.n[k];
            }
            cn[0] = c[0] + dc[0] + carry;
        }
        // dLoss/dout at this node: the later stage's pass B here, or lam
        R lam_in;
        if (gather) {
            R lvp, glu, acc;
            if constexpr (kPF) {
                adj_cp_wait();
                const float* sl = slices + (it & 1) * NQ * 256;
                lvp = sl[0];
                glu = sl[256];
                acc = a.gc_s * lvp;
#pragma unroll
                for (int q = 0; q < 7 * NDIM; ++q) acc += sl[(2 + q) * 256];
                if (idx + step < a.npts) prefetch(idx + step, cn, (it + 1) & 1);
            } else {
                lvp = a.lam_v[idx];
                glu = a.glam_u[idx];
                acc = gather_coeffs<NDIM>(a, a.gcontrib, idx, c, a.gc_s * lvp);
            }
            if (a.glam_n && a.glam_n != a.glam_u) {
                if (a.gatomic) atomicAdd(a.glam_n + idx, a.gc_n * lvp);
                else a.glam_n[idx] += a.gc_n * lvp;
            } else {
                acc += a.gc_n * lvp;
            }
            lam_in = glu + acc;
            a.glam_u[idx] = R(0);
        } else {
            lam_in = a.lam[idx];
        }
        // The per-axis work runs in loops that are not unrolled (one copy of
        // the window load, the derivative and the window gradient in the
        // code instead of NDIM: the unrolled form was bound by instruction
        // fetch); per-axis values go in and out of the small arrays by
        // selects over compile-time indices, so they stay in registers.
        R x[NDIM], pm[NDIM], pp[NDIM], pbar[NDIM];
        R diss = R(0);
        // the stencil window of axis k at this node (ghost cells substituted)
        auto window = [&](int k, R* u) {
            const int nk = pick<NDIM>(a.n, k), ck = pick<NDIM>(c, k);
            const int sk = pick<NDIM>(a.stride, k);
            if (ck >= 3 && ck < nk - 3) {  // no ghost cells in the window
                const R* p0 = a.u + idx;
#pragma unroll
                for (int o = -3; o <= 3; ++o) u[o + 3] = __ldg(p0 + (long long)o * sk);
            } else {
                load_window<R, 3>(a.u, idx, ck, nk, sk, pick<NDIM>(a.periodic, k), u);
            }
        };
#pragma unroll 1
        for (int k = 0; k < NDIM; ++k) {
            R u[7];
            window(k, u);
            const R idk = pick<NDIM>(a.inv_dx, k);
            R pmk, ppk;
            deriv_fast<SCHEME>(u + (3 - G), idk, weno_floor12(idk), pmk, ppk);
            put<NDIM>(pm, k, pmk);
            put<NDIM>(pp, k, ppk);
            put<NDIM>(pbar, k, R(0.5) * (ppk + pmk));
            diss += pick<NDIM>(a.alpha, k) * R(0.5) * (ppk - pmk);
            put<NDIM>(x, k, pick<NDIM>(a.lo, k) + R(pick<NDIM>(c, k)) * pick<NDIM>(a.h, k));
        }
        R sth = R(0), cth = R(1);
        if constexpr (DYN == AIR3D || DYN == CAR4D || DYN == ROCKETS) rsincos(x[2], &sth, &cth);
        const R H = hamiltonian_sc<DYN, NDIM>(x, pbar, a.prm, sth, cth);
        const R L = -(H - diss);
        R v = a.c_s * a.u[idx] + (a.c_l * a.dt) * L;
        if (a.phin) v += a.c_n * a.phin[idx];
        R lv = lam_in;
        if (a.tube) {
            const R g = a.target[idx];
            if (g < v) {  // the min took the target
                if (a.lam_g) a.lam_g[idx] += lv;
                lv = R(0);
            }
        }
        a.lam_v[idx] = lv;
        const R w = a.c_l * a.dt * lv;
        acc_dt += (a.c_l * lv) * L;
        R hp[NDIM], hprm[4];
        ham_grad<DYN, NDIM>(x, pbar, a.prm, sth, cth, hp, hprm);
#pragma unroll
        for (int j = 0; j < 4; ++j) acc_h[j] += w * -hprm[j];
#pragma unroll 1
        for (int k = 0; k < NDIM; ++k) {
            put<NDIM>(acc_a, k,
                      pick<NDIM>(acc_a, k) + w * R(0.5) * (pick<NDIM>(pp, k) - pick<NDIM>(pm, k)));
            R u[7], gm[7], gp[7];
            window(k, u);  // again: cheaper than holding NDIM windows in registers
            const R idk = pick<NDIM>(a.inv_dx, k), alk = pick<NDIM>(a.alpha, k);
            window_grad<SCHEME>(u, idk, weno_floor12(idk), gm, gp);
            const R hpk = pick<NDIM>(hp, k);
            const R sp = w * (R(-0.5) * hpk + R(0.5) * alk);
            const R sm = w * (R(-0.5) * hpk - R(0.5) * alk);
            R* out = a.contrib + (long long)(7 * k + 3) * a.cstride + idx;  // offset 0
            const int n = pick<NDIM>(a.n, k), s = pick<NDIM>(a.stride, k), ck = pick<NDIM>(c, k);
            const int perk = pick<NDIM>(a.periodic, k);
            if (perk || (ck >= 3 && ck < n - 3)) {  // no ghost position to fold
#pragma unroll
                for (int o = -3; o <= 3; ++o)
                    out[(long long)o * a.cstride] = sp * gp[o + 3] + sm * gm[o + 3];
                continue;
            }
#pragma unroll
            for (int o = -3; o <= 3; ++o) {
                R cf = sp * gp[o + 3] + sm * gm[o + 3];
                const int j = ck + o;
                if (j < 0 || j >= n) {
                    // ghost of an extrapolated axis: u_j = (1+q) u_b - q u_b', fold now
                    if (cf != R(0)) {
                        const long long line0 = (long long)idx - (long long)ck * s;
                        if (j < 0) {
                            const R q = R(-j);
                            atomicAdd(a.lam_u + line0, (R(1) + q) * cf);
                            atomicAdd(a.lam_u + line0 + s, -q * cf);
                        } else {
                            const R q = R(j - n + 1);
                            atomicAdd(a.lam_u + line0 + (long long)(n - 1) * s, (R(1) + q) * cf);
                            atomicAdd(a.lam_u + line0 + (long long)(n - 2) * s, -q * cf);
                        }
                    }
                    cf = R(0);
                }
                out[(long long)o * a.cstride] = cf;
            }
        }
#pragma unroll
        for (int k = 0; k < NDIM; ++k) c[k] = cn[k];
    }
    // block reductions of the accumulators, one FP64 atomic each per block
    __shared__ double red[9][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double vals[9] = {(double)acc_h[0], (double)acc_h[1], (double)acc_h[2], (double)acc_h[3],
                            (double)acc_a[0], (double)acc_a[1], (double)acc_a[2], (double)acc_a[3],
                            (double)acc_dt};
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        double v = vals[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[q][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
        double* dst = threadIdx.x < 4 ? a.acc->hprm + threadIdx.x
                    : threadIdx.x < 8 ? a.acc->alpha + (threadIdx.x - 4)
                                      : &a.acc->dt;
        if (v != 0.0) atomicAdd(dst, v);
    }
}

template <int NDIM, typename R>
__global__ void __launch_bounds__(256) adj_stage_b(AdjArgs<R> a)
{
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < a.npts;
         idx += gridDim.x * blockDim.x) {
        int c[NDIM];
        {
            int r = idx;
#pragma unroll
            for (int k = NDIM - 1; k >= 0; --k) {
                c[k] = r % a.n[k];
                r /= a.n[k];
            }
        }
        const R lv = a.lam_v[idx];
        R acc = gather_coeffs<NDIM>(a, a.contrib, idx, c, a.c_s * lv);
        if (a.lam_n != a.lam_u && a.lam_n) a.lam_n[idx] += a.c_n * lv;
        else acc += a.c_n * lv;
        a.lam_u[idx] += acc;
    }
}

// First node (C order) whose per-node LF bound on axis k equals alpha_k:
// the node the GLF coefficient's derivative is taken at.
template <int DYN>
__global__ void __launch_bounds__(256) alpha_argmax_kernel(GridGeom g, const double* alpha,
                                                          unsigned long long* out)
{
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < g.npts;
         idx += (long long)gridDim.x * blockDim.x) {
        double x[LSP_MAXD] = {0.0, 0.0, 0.0, 0.0};
        long long r = idx;
        for (int k = g.ndim - 1; k >= 0; --k) {
            x[k] = g.lo[k] + (double)(r % g.n[k]) * g.h[k];
            r /= g.n[k];
        }
        for (int k = 0; k < g.ndim; ++k)
            if (partial_bound<DYN>(x, k, g.prm) == alpha[k])
                atomicMin(out + k, (unsigned long long)idx);
    }
}

// ---------------------------------------------------------------------------
// Loss of the differentiation workload on the device:
//   sum_i H_eps(-phi_i) dV + sum_q phi(x_q),  H_eps(s) = 1/(1 + exp(-s/eps))
// with multilinear interpolation at the query states (periodic axes wrap,
// the others clamp), and its gradient.
template <typename R, int NDIM>
struct InterpArgs {
    const R* phi;
    const R* queries;  // nq x NDIM
    int nq;
    int n[LSP_MAXD];
    int stride[LSP_MAXD];
    int periodic[LSP_MAXD];
    double lo[LSP_MAXD], h[LSP_MAXD];
};

template <typename R>
__global__ void __launch_bounds__(256) loss_volume_kernel(const R* phi, int npts, double inv_eps,
                                                         double dV, double* value, R* grad)
{
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npts; i += gridDim.x * blockDim.x) {
        const double Hs = 1.0 / (1.0 + exp((double)phi[i] * inv_eps));  // H_eps(-phi)
        acc += Hs * dV;
        if (grad) grad[i] = R(-Hs * (1.0 - Hs) * inv_eps * dV);
    }
    __shared__ double red[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
        atomicAdd(value, v);
    }
}

template <typename R, int NDIM>
__global__ void __launch_bounds__(128) loss_query_kernel(InterpArgs<R, NDIM> a, double* value,
                                                        R* grad)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= a.nq) return;
    int i0[NDIM], i1[NDIM];
    double f[NDIM];
#pragma unroll
    for (int k = 0; k < NDIM; ++k) {
        double t = ((double)a.queries[q * NDIM + k] - a.lo[k]) / a.h[k];
        const int n = a.n[k];
        if (a.periodic[k]) {
            const double fl = floor(t);
            f[k] = t - fl;
            int b = (int)fl % n;
            if (b < 0) b += n;
            i0[k] = b;
            i1[k] = (b + 1) % n;
        } else {
            t = fmin(fmax(t, 0.0), (double)(n - 1));
            int b = (int)floor(t);
            if (b > n - 2) b = n - 2;
            f[k] = t - b;
            i0[k] = b;
            i1[k] = b + 1;
        }
    }
    double val = 0.0;
    for (int corner = 0; corner < (1 << NDIM); ++corner) {
        double w = 1.0;
        long long off = 0;
#pragma unroll
        for (int k = 0; k < NDIM; ++k) {
            const int bit = (corner >> (NDIM - 1 - k)) & 1;
            w *= bit ? f[k] : 1.0 - f[k];
            off += (long long)(bit ? i1[k] : i0[k]) * a.stride[k];
        }
        val += w * (double)a.phi[off];
        if (grad) atomicAdd(grad + off, R(w));
    }
    atomicAdd(value, val);
}

}  // namespace lsp
