/*
 * lsp_oracle.c -- plain, slow, FP64 CPU oracle for the explicit Hamilton-Jacobi
 * level-set integrator of "LevelSetPy" (arXiv 2411.03501).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the yardstick the GPU path is checked
 * against.  It is called from tests/, from the smoke check and from the CPU
 * baseline leg of the benchmark; the product path never links or calls it, and
 * it shares no code, header, table or constant with the CUDA sources.
 *
 * Everything is written point by point in double precision, in the order the
 * paper states the method:
 *   grid + ghost cells          Sec. III-B (grid fields, ghost-cell boundaries)
 *   one-sided derivatives       Sec. IV-A (Eq. 6, first-order upwinding),
 *                               Sec. IV-B (Eqs. 8, 11-14, ENO2 / ENO3),
 *                               Sec. IV-C (Eqs. 15-20, HJ-WENO5)
 *   Lax-Friedrichs term + GLF   Sec. IV-D, Listing 4 (termLaxFriedrichs,
 *                               artificialDissipationGLF, partialFunc)
 *   CFL step                    Sec. IV-D (CFL condition), Sec. V-A
 *   TVD-RK1/2/3                 Sec. V-A (Eqs. 24-27 and the averaging steps)
 *   min with target (tube)      Sec. VI-A (variational HJI, Eq. 30)
 *   Hamiltonians with optimal   Sec. VI-A (Eqs. 31-32: H = -max_u min_d p.f,
 *   inputs                      closed form with |.| switching terms)
 *
 * Where the paper is silent or its printed formulas are garbled, the reading
 * used is stated at the spot (each one is listed in the design notes).  The
 * equation numbers are those of the numbered displays of the paper, counted
 * in order.
 *
 * Layout: C order, last axis fastest (the paper: "generalizes a row-major
 * layout", Sec. III-C).
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

#define ORC_MAXD 4

/* scheme ids */
enum { ORC_UPWIND1 = 0, ORC_ENO2 = 1, ORC_ENO3 = 2, ORC_WENO5 = 3 };
/* dynamics ids */
enum {
    ORC_DYN_NORMAL_SPEED = 0, /* H = a |p|                                   */
    ORC_DYN_TRANSLATE = 1,    /* H = v . p                                   */
    ORC_DYN_QUADRATIC = 2,    /* H = |p|^2 / 2   (alpha depends on p)        */
    ORC_DYN_AIR3D = 3,        /* relative pursuit-evasion (x, y, theta)      */
    ORC_DYN_CAR4D = 4,        /* car (x, y, theta, v), reach game            */
    ORC_DYN_ROCKETS = 5,      /* two rockets, relative (x, z, theta), game   */
    ORC_DYN_DOUBLE_INT = 6    /* double integrator (x1, x2), reach           */
};

/* dissipation coefficient variants (artificialDissipationGLF of Listing 4
 * and its local siblings of the toolbox the paper follows) */
enum { ORC_DISS_GLF = 0, ORC_DISS_LLF = 1, ORC_DISS_LLLF = 2 };

typedef struct {
    int ndim;
    int scheme;
    int dyn;
    int diss;    /* ORC_DISS_*                                              */
    int64_t n[ORC_MAXD];
    double lo[ORC_MAXD];
    double hi[ORC_MAXD];
    int periodic[ORC_MAXD];
    double prm[8];
    int varform; /* 1: the variational form of the BRT PDE (rate <= 0)    */
    int pad_;
} orc_problem;

typedef struct {
    int64_t steps;
    int64_t stages;
    double dt_min;
    double dt_max;
    double t_end;
} orc_stats;

/* ------------------------------------------------------------------------ */
/* Grid (Sec. III-B, Listing 1).                                             */
/* Reading: a non-periodic axis has nodes lo + i*dx, i = 0..n-1, with        */
/* dx = (hi-lo)/(n-1); a periodic axis has dx = (hi-lo)/n so that hi itself  */
/* is the image of lo and is not a node (theta in [0, 2 pi)).                */
/* ------------------------------------------------------------------------ */
double orc_dx(const orc_problem* P, int k)
{
    if (P->periodic[k]) return (P->hi[k] - P->lo[k]) / (double)P->n[k];
    return (P->hi[k] - P->lo[k]) / (double)(P->n[k] - 1);
}

double orc_node(const orc_problem* P, int k, int64_t i)
{
    return P->lo[k] + (double)i * orc_dx(P, k);
}

int64_t orc_npoints(const orc_problem* P)
{
    int64_t N = 1;
    for (int k = 0; k < P->ndim; ++k) N *= P->n[k];
    return N;
}

static int64_t stride_of(const orc_problem* P, int k)
{
    int64_t s = 1;
    for (int j = P->ndim - 1; j > k; --j) s *= P->n[j];
    return s;
}

/* Ghost width needed by each scheme: the stencils of Sec. IV reach
 * i-1..i+1 (first order), i-2..i+2 (ENO2), i-3..i+3 (ENO3, WENO5). */
int orc_ghost_width(int scheme)
{
    switch (scheme) {
    case ORC_UPWIND1: return 1;
    case ORC_ENO2: return 2;
    default: return 3;
    }
}

/* Fill one extended line u[-G .. n-1+G] (stored at offset G) from the n node
 * values of a grid line.  Sec. III-B: boundary conditions enter through the
 * ghost cells that extend each line.  Periodic: wrap around.  Otherwise (reading; the
 * paper names no other condition): linear extrapolation from the two nodes
 * nearest the boundary, u[-k] = u[0] + k (u[0] - u[1]). */
static void fill_line(const double* line, int64_t n, int G, int periodic, double* ext)
{
    for (int64_t i = 0; i < n; ++i) ext[G + i] = line[i];
    for (int k = 1; k <= G; ++k) {
        if (periodic) {
            ext[G - k] = line[((n - k) % n + n) % n];
            ext[G + n - 1 + k] = line[(k - 1) % n];
        } else {
            ext[G - k] = line[0] + (double)k * (line[0] - line[1]);
            ext[G + n - 1 + k] = line[n - 1] + (double)k * (line[n - 1] - line[n - 2]);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* One-sided derivatives on one extended line.  `u` points at node 0 of the  */
/* extended line, so u[-G..n-1+G] is valid.  Outputs pm[i] = phi_x^-(x_i),   */
/* pp[i] = phi_x^+(x_i).  `tie` (nullable) receives, per node, the largest   */
/* change of p^- or p^+ that flipping a near-tied ENO selection there would  */
/* cause (0 when none is near a tie, always 0 for the other schemes): where  */
/* it is large, another implementation may validly take the other stencil.   */
/* ------------------------------------------------------------------------ */

/* Sec. IV-A, Eq. 6 and the text below it: D^- looks left, D^+ looks right.
 * (Eq. 6 prints the two labels the other way round; the text fixes the
 * standard reading: use D^- phi when information travels left to right.) */
static void upwind1_line(const double* u, int64_t n, double dx, double* pm, double* pp)
{
    for (int64_t i = 0; i < n; ++i) {
        pm[i] = (u[i] - u[i - 1]) / dx;
        pp[i] = (u[i + 1] - u[i]) / dx;
    }
}

/* Divided differences of Sec. IV-B (Eq. 8):
 *   D1_{j+1/2} = (u_{j+1} - u_j) / dx
 *   D2_j       = (D1_{j+1/2} - D1_{j-1/2}) / (2 dx)
 *   D3_{j+1/2} = (D2_{j+1} - D2_j) / (3 dx)                                 */
static double D1h(const double* u, int64_t j, double dx) /* D1_{j+1/2} */
{
    return (u[j + 1] - u[j]) / dx;
}
static double D2(const double* u, int64_t j, double dx) /* D2_j */
{
    return (D1h(u, j, dx) - D1h(u, j - 1, dx)) / (2.0 * dx);
}
static double D3h(const double* u, int64_t j, double dx) /* D3_{j+1/2} */
{
    return (D2(u, j + 1, dx) - D2(u, j, dx)) / (3.0 * dx);
}

/* Relative gap between |a| and |b|: a selection by |a| <= |b| whose gap is
 * below 1e-4 may be taken the other way by a computation in another
 * precision or order of operations. */
static double rel_gap(double a, double b)
{
    double s = fabs(a) + fabs(b);
    return s == 0.0 ? 1.0 : fabs(fabs(a) - fabs(b)) / s;
}

/* ENO polynomial derivative at node i built on base index k (k = i-1 for the
 * left derivative, k = i for the right one), Sec. IV-B:
 *   phi_x(x_i) = Q1'(x_i) + Q2'(x_i) [+ Q3'(x_i)]                (Eq. 10)
 *   Q1'(x_i)   = D1_{k+1/2}                                          (Eq. 11)
 *   c          = D2_k if |D2_k| <= |D2_{k+1}| else D2_{k+1}          (Eq. 12)
 *   Q2'(x_i)   = c (2(i-k) - 1) dx
 *   c*         = D3_{k*+1/2} if |D3_{k*+1/2}| <= |D3_{k*+3/2}|
 *                else D3_{k*+3/2}                                    (Eq. 13)
 *   Q3'(x_i)   = c* (3(i-k*)^2 - 6(i-k*) + 2) dx^2                   (Eq. 14b)
 * Reading for k* (the paper uses it without defining it; this is the rule of
 * the Osher-Fedkiw text the paper follows): k* = k-1 when c took D2_k, else
 * k* = k.  The product in Eq. 14a is read as (x-x_{k*})(x-x_{k*+1})(x-x_{k*+2}),
 * whose derivative at x_i is the printed Eq. 14b.                           */
/* force2 / force3: -1 to select by the rule, 0 / 1 to take the first /
 * second candidate regardless (used only to size the effect of a flip). */
static double eno_eval(const double* u, int64_t i, int64_t k, double dx, int order, int force2,
                       int force3)
{
    double q1 = D1h(u, k, dx);
    double a = D2(u, k, dx), b = D2(u, k + 1, dx);
    double c;
    int64_t kstar;
    int first = force2 < 0 ? (fabs(a) <= fabs(b)) : (force2 == 0);
    if (first) {
        c = a;
        kstar = k - 1;
    } else {
        c = b;
        kstar = k;
    }
    double r = q1 + c * (double)(2 * (i - k) - 1) * dx;
    if (order >= 3) {
        double e = D3h(u, kstar, dx), f = D3h(u, kstar + 1, dx);
        int first3 = force3 < 0 ? (fabs(e) <= fabs(f)) : (force3 == 0);
        double cs = first3 ? e : f;
        double s = (double)(i - kstar);
        r += cs * (3.0 * s * s - 6.0 * s + 2.0) * dx * dx;
    }
    return r;
}

/* The ENO derivative, and in *flip (nullable) the largest change of it that
 * taking a near-tied selection the other way would cause; 0 when no
 * selection is near a tie.  Near a tie: the compared magnitudes differ by
 * less than 1e-4 of their sum, or by less than what FP32 rounding of the
 * window values can move a divided difference (about 4 ulps of the largest
 * |u| in the window for a second difference, 8 for a third, over their
 * denominators 2 dx^2 and 6 dx^3, doubled).  (*flip is diagnostic output for
 * the comparisons with other implementations; it enters no computed value.) */
static double eno_at(const double* u, int64_t i, int64_t k, double dx, int order, double* flip)
{
    double r = eno_eval(u, i, k, dx, order, -1, -1);
    if (flip) {
        const double u32 = 5.9604644775390625e-8; /* 2^-24 */
        double M = 0.0;
        for (int o = -order; o <= order; ++o) M = fmax(M, fabs(u[i + o]));
        double fl = 0.0;
        double a = D2(u, k, dx), b = D2(u, k + 1, dx);
        int first = fabs(a) <= fabs(b);
        double tie2 = 8.0 * u32 * M / (2.0 * dx * dx);
        if (rel_gap(a, b) < 1e-4 || fabs(fabs(a) - fabs(b)) <= tie2)
            fl = fabs(eno_eval(u, i, k, dx, order, first ? 1 : 0, -1) - r);
        if (order >= 3) {
            int64_t kstar = first ? k - 1 : k;
            double e = D3h(u, kstar, dx), f = D3h(u, kstar + 1, dx);
            double tie3 = 16.0 * u32 * M / (6.0 * dx * dx * dx);
            if (rel_gap(e, f) < 1e-4 || fabs(fabs(e) - fabs(f)) <= tie3) {
                double alt = eno_eval(u, i, k, dx, order, first ? 0 : 1,
                                      fabs(e) <= fabs(f) ? 1 : 0);
                if (fabs(alt - r) > fl) fl = fabs(alt - r);
            }
        }
        *flip = fl;
    }
    return r;
}

static void eno_line(const double* u, int64_t n, double dx, int order, double* pm,
                     double* pp, double* tie)
{
    for (int64_t i = 0; i < n; ++i) {
        double m1, m2;
        pm[i] = eno_at(u, i, i - 1, dx, order, &m1);
        pp[i] = eno_at(u, i, i, dx, order, &m2);
        if (tie) tie[i] = (m1 > m2) ? m1 : m2;
    }
}

/* HJ-WENO5 of Sec. IV-C on five first differences v1..v5.
 *   substencils (Eq. 15):
 *     phi1 = v1/3 - 7 v2/6 + 11 v3/6
 *     phi2 = -v2/6 + 5 v3/6 + v4/3
 *     phi3 = v3/3 + 5 v4/6 - v5/6
 *   Reading: Eq. 15c is printed with -1/3 on its first term; its coefficients
 *   must sum to 1 for consistency and only +1/3 reproduces the optimal
 *   fifth-order combination printed after Eq. 16 with weights (0.1, 0.6, 0.3).
 *   smoothness (Eq. 18), with sigma2 read as 13/12 (v2 - 2 v3 + v4)^2 +
 *   1/4 (v2 - v4)^2 (the print repeats the index i-3 in its first bracket):
 *     s1 = 13/12 (v1 - 2 v2 + v3)^2 + 1/4 (v1 - 4 v2 + 3 v3)^2
 *     s2 = 13/12 (v2 - 2 v3 + v4)^2 + 1/4 (v2 - v4)^2
 *     s3 = 13/12 (v3 - 2 v4 + v5)^2 + 1/4 (3 v3 - 4 v4 + v5)^2
 *   eps (Eq. 19), read with squares: 1e-6 max(v1^2..v5^2) + 1e-99
 *   alpha (Eq. 17), read with 0.3 on the third weight (the text states the
 *   optimal weights 0.1, 0.6, 0.3): alpha_k = d_k / (s_k + eps)^2
 *   w_k = alpha_k / sum alpha (Eq. 20);  result = sum w_k phi_k (Eq. 16).  */
static double weno5_combine(double v1, double v2, double v3, double v4, double v5)
{
    double phi1 = v1 / 3.0 - 7.0 * v2 / 6.0 + 11.0 * v3 / 6.0;
    double phi2 = -v2 / 6.0 + 5.0 * v3 / 6.0 + v4 / 3.0;
    double phi3 = v3 / 3.0 + 5.0 * v4 / 6.0 - v5 / 6.0;

    double t;
    double s1 = 13.0 / 12.0 * (v1 - 2.0 * v2 + v3) * (v1 - 2.0 * v2 + v3);
    t = v1 - 4.0 * v2 + 3.0 * v3;
    s1 += 0.25 * t * t;
    double s2 = 13.0 / 12.0 * (v2 - 2.0 * v3 + v4) * (v2 - 2.0 * v3 + v4);
    t = v2 - v4;
    s2 += 0.25 * t * t;
    double s3 = 13.0 / 12.0 * (v3 - 2.0 * v4 + v5) * (v3 - 2.0 * v4 + v5);
    t = 3.0 * v3 - 4.0 * v4 + v5;
    s3 += 0.25 * t * t;

    double mx = v1 * v1;
    if (v2 * v2 > mx) mx = v2 * v2;
    if (v3 * v3 > mx) mx = v3 * v3;
    if (v4 * v4 > mx) mx = v4 * v4;
    if (v5 * v5 > mx) mx = v5 * v5;
    double eps = 1e-6 * mx + 1e-99;

    double a1 = 0.1 / ((s1 + eps) * (s1 + eps));
    double a2 = 0.6 / ((s2 + eps) * (s2 + eps));
    double a3 = 0.3 / ((s3 + eps) * (s3 + eps));
    double sum = a1 + a2 + a3;
    return (a1 / sum) * phi1 + (a2 / sum) * phi2 + (a3 / sum) * phi3;
}

/* Left derivative: v1..v5 = D+u_{i-3} .. D+u_{i+1} (Sec. IV-C).
 * Right derivative (reading; the paper gives only the left one): the mirror
 * image, v1..v5 = D+u_{i+2}, D+u_{i+1}, D+u_i, D+u_{i-1}, D+u_{i-2}.
 * D+u_j = (u_{j+1} - u_j) / dx.                                            */
static void weno5_line(const double* u, int64_t n, double dx, double* pm, double* pp)
{
    for (int64_t i = 0; i < n; ++i) {
        double d[6]; /* d[m] = D+u_{i-3+m}, m = 0..5 */
        for (int m = 0; m < 6; ++m) d[m] = (u[i - 3 + m + 1] - u[i - 3 + m]) / dx;
        pm[i] = weno5_combine(d[0], d[1], d[2], d[3], d[4]);
        pp[i] = weno5_combine(d[5], d[4], d[3], d[2], d[1]);
    }
}

/* Derivatives of phi along `axis` at every node.  pm, pp: N doubles each;
 * tie (nullable): N doubles, size of a near-tie flip (see above). */
int orc_derivs(const orc_problem* P, const double* phi, int axis, double* pm, double* pp,
               double* tie)
{
    if (axis < 0 || axis >= P->ndim) return -1;
    int G = orc_ghost_width(P->scheme);
    int64_t n = P->n[axis];
    if (n < 2 * G + 1) return -2;
    int64_t s = stride_of(P, axis);
    int64_t N = orc_npoints(P);
    int64_t nlines = N / n;
    double dx = orc_dx(P, axis);

#pragma omp parallel
    {
        double* line = (double*)malloc(sizeof(double) * (size_t)n);
        double* ext = (double*)malloc(sizeof(double) * (size_t)(n + 2 * G));
        double* lm = (double*)malloc(sizeof(double) * (size_t)n);
        double* lp = (double*)malloc(sizeof(double) * (size_t)n);
        double* lt = (double*)malloc(sizeof(double) * (size_t)n);
#pragma omp for schedule(static)
        for (int64_t L = 0; L < nlines; ++L) {
            /* line L: the index with the axis coordinate removed */
            int64_t outer = L / s, inner = L % s;
            int64_t base = outer * s * n + inner;
            for (int64_t i = 0; i < n; ++i) line[i] = phi[base + i * s];
            fill_line(line, n, G, P->periodic[axis], ext);
            const double* u = ext + G;
            for (int64_t i = 0; i < n; ++i) lt[i] = 0.0;
            switch (P->scheme) {
            case ORC_UPWIND1: upwind1_line(u, n, dx, lm, lp); break;
            case ORC_ENO2: eno_line(u, n, dx, 2, lm, lp, lt); break;
            case ORC_ENO3: eno_line(u, n, dx, 3, lm, lp, lt); break;
            default: weno5_line(u, n, dx, lm, lp); break;
            }
            for (int64_t i = 0; i < n; ++i) {
                pm[base + i * s] = lm[i];
                pp[base + i * s] = lp[i];
                if (tie) tie[base + i * s] = lt[i];
            }
        }
        free(line);
        free(ext);
        free(lm);
        free(lp);
        free(lt);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Hamiltonians (Sec. VI-A pattern: H = -max_u min_d p.f evaluated in closed */
/* form, the optimal inputs picked by the sign of a costate combination).    */
/* x: node coordinates, p: costate, d: dimension count.                      */
/* ------------------------------------------------------------------------ */
static double ham(const orc_problem* P, const double* x, const double* p)
{
    const double* c = P->prm;
    int d = P->ndim;
    switch (P->dyn) {
    case ORC_DYN_NORMAL_SPEED: { /* H = a |p|: fronts move outward at speed a */
        double s = 0.0;
        for (int k = 0; k < d; ++k) s += p[k] * p[k];
        return c[0] * sqrt(s);
    }
    case ORC_DYN_TRANSLATE: { /* phi_t + v.grad phi = 0 */
        double s = 0.0;
        for (int k = 0; k < d; ++k) s += c[k] * p[k];
        return s;
    }
    case ORC_DYN_QUADRATIC: {
        double s = 0.0;
        for (int k = 0; k < d; ++k) s += p[k] * p[k];
        return 0.5 * s;
    }
    case ORC_DYN_AIR3D: {
        /* relative dynamics, evader (control, maximises) turn rate u, pursuer
         * (disturbance, minimises) turn rate d:
         *   xdot = -v_e + v_p cos th + u y,  ydot = v_p sin th - u x,
         *   thdot = d - u.
         * max_u min_d p.f = p1(-v_e + v_p cos th) + p2 v_p sin th
         *                   + ue_max |p1 y - p2 x - p3| - ud_max |p3|
         * and H = -(that), the sign convention of Eq. 31.                 */
        double ve = c[0], vp = c[1], we = c[2], wp = c[3];
        double X = x[0], Y = x[1], th = x[2];
        double v = p[0] * (-ve + vp * cos(th)) + p[1] * vp * sin(th) +
                   we * fabs(p[0] * Y - p[1] * X - p[2]) - wp * fabs(p[2]);
        return -v;
    }
    case ORC_DYN_CAR4D: {
        /* xdot = v cos th, ydot = v sin th, thdot = w, vdot = acc; the
         * control minimises p.f (reach): H = -min_u p.f                     */
        double wm = c[0], am = c[1];
        double th = x[2], v = x[3];
        double m = p[0] * v * cos(th) + p[1] * v * sin(th) - wm * fabs(p[2]) - am * fabs(p[3]);
        return -m;
    }
    case ORC_DYN_ROCKETS: {
        /* Sec. VI-A, Eq. 31: f = (a cos th + u_e x, a sin th + a + u_p x - g,
         * u_p - u_e) with a_e = a_p = a; the evader input u_e in [-ue, ue]
         * maximises, the pursuer input u_p in [-up, up] minimises, and
         * H = -max_{u_e} min_{u_p} p.f.  Reading: this definition is used and
         * its closed form derived from it, because the printed closed form
         * (Eq. 32) disagrees with it in the sign of the p_2 term and in both
         * switching terms.  p.f = p1 a cos th + p2 (a sin th + a - g)
         *   + u_e (p1 x - p3) + u_p (p2 x + p3).                              */
        double a = c[0], g = c[1], ue = c[2], up = c[3];
        double X = x[0], th = x[2];
        double v = p[0] * a * cos(th) + p[1] * (a * sin(th) + a - g) + ue * fabs(p[0] * X - p[2]) -
                   up * fabs(p[1] * X + p[2]);
        return -v;
    }
    case ORC_DYN_DOUBLE_INT: {
        /* Table I names the double integrator without stating it.  Reading:
         * x1dot = x2, x2dot = u, |u| <= umax, the input drives the state into
         * the target (reach): H = -min_u p.f = -(p1 x2 - umax |p2|).         */
        double um = c[0];
        return -(p[0] * x[1] - um * fabs(p[1]));
    }
    }
    return 0.0;
}

/* Per-node bound on |dH/dp_k| for the dynamics whose bound does not depend
 * on p ("partialFunc" of Listing 4).                                        */
static double partial_bound(const orc_problem* P, const double* x, int k)
{
    const double* c = P->prm;
    switch (P->dyn) {
    case ORC_DYN_NORMAL_SPEED: return fabs(c[0]); /* |dH/dp_k| = |a| |p_k| / |p| */
    case ORC_DYN_TRANSLATE: return fabs(c[k]);
    case ORC_DYN_AIR3D: {
        double ve = c[0], vp = c[1], we = c[2], wp = c[3];
        if (k == 0) return fabs(-ve + vp * cos(x[2])) + we * fabs(x[1]);
        if (k == 1) return vp * fabs(sin(x[2])) + we * fabs(x[0]);
        return we + wp;
    }
    case ORC_DYN_CAR4D: {
        if (k == 0) return fabs(x[3] * cos(x[2]));
        if (k == 1) return fabs(x[3] * sin(x[2]));
        if (k == 2) return c[0];
        return c[1];
    }
    case ORC_DYN_ROCKETS: { /* |dH/dp_k| over both input choices */
        double a = c[0], g = c[1], ue = c[2], up = c[3];
        if (k == 0) return a * fabs(cos(x[2])) + ue * fabs(x[0]);
        if (k == 1) return fabs(a * sin(x[2]) + a - g) + up * fabs(x[0]);
        return ue + up;
    }
    case ORC_DYN_DOUBLE_INT:
        return k == 0 ? fabs(x[1]) : c[0];
    }
    return 0.0;
}

/* Bound on |dH/dp_k| at state x over the costate box [clo_j, chi_j] of
 * every dimension j (the "partialFunc" of Listing 4 receives the costate
 * range).  The state-only bounds ignore the box; for H = |p|^2/2,
 * dH/dp_k = p_k and the bound over the box is max(|clo_k|, |chi_k|).       */
static double partial_bound_box(const orc_problem* P, const double* x, const double* clo,
                                const double* chi, int k)
{
    if (P->dyn == ORC_DYN_QUADRATIC) return fmax(fabs(clo[k]), fabs(chi[k]));
    return partial_bound(P, x, k);
}

static void node_coords(const orc_problem* P, int64_t idx, double* x)
{
    for (int k = P->ndim - 1; k >= 0; --k) {
        int64_t i = idx % P->n[k];
        idx /= P->n[k];
        x[k] = orc_node(P, k, i);
    }
}

/* Global Lax-Friedrichs coefficients (artificialDissipationGLF, Listing 4;
 * the paper names the routine without stating it).  Reading: alpha_k is the
 * maximum over the whole grid of the bound on |dH/dp_k|.  For H = |p|^2/2 the
 * bound is p-dependent and is taken from the current one-sided derivative
 * fields: alpha_k = max(|min p_k|, |max p_k|) over p^- and p^+.
 * pm/pp (ndim arrays of N each) are needed only for that case.             */
static void alpha_from(const orc_problem* P, double* const* pm, double* const* pp,
                       double* alpha)
{
    int64_t N = orc_npoints(P);
    for (int k = 0; k < P->ndim; ++k) alpha[k] = 0.0;
    if (P->dyn == ORC_DYN_QUADRATIC) {
        for (int k = 0; k < P->ndim; ++k) {
            double lo = INFINITY, hi = -INFINITY;
            for (int64_t i = 0; i < N; ++i) {
                if (pm[k][i] < lo) lo = pm[k][i];
                if (pm[k][i] > hi) hi = pm[k][i];
                if (pp[k][i] < lo) lo = pp[k][i];
                if (pp[k][i] > hi) hi = pp[k][i];
            }
            alpha[k] = fmax(fabs(lo), fabs(hi));
        }
        return;
    }
    for (int64_t i = 0; i < N; ++i) {
        double x[ORC_MAXD];
        node_coords(P, i, x);
        for (int k = 0; k < P->ndim; ++k) {
            double b = partial_bound(P, x, k);
            if (b > alpha[k]) alpha[k] = b;
        }
    }
}

/* Lax-Friedrichs numerical Hamiltonian (termLaxFriedrichs, Sec. IV-D and
 * Listing 4).  Reading of the HJ form (the paper prints only the
 * conservation-law scheme):
 *   Hhat(x) = H(x, (p^+ + p^-)/2) - sum_k alpha_k (p^+_k - p^-_k)/2
 * and the method-of-lines rate (Sec. V-A, Eq. 24) is L = -Hhat.
 * Dissipation coefficients (P->diss):
 *   GLF   alpha_k: one number per dimension, the grid maximum of the bound
 *         over the global costate box (alpha_from; alpha_in overrides it)
 *   LLF   alpha_k(x): the bound at node x over the box that is the node's
 *         own [min, max] of p^-_k, p^+_k in dimension k and the global
 *         costate range in the other dimensions
 *   LLLF  alpha_k(x): the bound at node x over the node's own box in every
 *         dimension
 * (the paper names only the global routine; the local ones are its
 * siblings in the toolbox whose layout the paper follows).
 * Variational form (P->varform, Eq. 30): in time-to-go, with this sign
 * convention, phi_t + min[0, H] = 0 of the paper's backward-time statement
 * becomes phi_t = min(0, L): every stage's rate is clipped at zero, so
 * phi never increases.
 * If alpha_in is NULL alpha is computed from this phi (alpha_out, nullable,
 * receives the GLF coefficients in every mode).  rate: N doubles.          */
int orc_rate(const orc_problem* P, const double* phi, const double* alpha_in,
             double* alpha_out, double* rate)
{
    int d = P->ndim;
    int64_t N = orc_npoints(P);
    double* pm[ORC_MAXD];
    double* pp[ORC_MAXD];
    int rc = 0;
    for (int k = 0; k < d; ++k) {
        pm[k] = (double*)malloc(sizeof(double) * (size_t)N);
        pp[k] = (double*)malloc(sizeof(double) * (size_t)N);
    }
    for (int k = 0; k < d && rc == 0; ++k) rc = orc_derivs(P, phi, k, pm[k], pp[k], NULL);
    if (rc == 0) {
        double alpha[ORC_MAXD];
        if (alpha_in) {
            for (int k = 0; k < d; ++k) alpha[k] = alpha_in[k];
        } else {
            alpha_from(P, pm, pp, alpha);
        }
        if (alpha_out)
            for (int k = 0; k < d; ++k) alpha_out[k] = alpha[k];
        /* global costate box, for the local variants */
        double glo[ORC_MAXD], ghi[ORC_MAXD];
        for (int k = 0; k < d; ++k) {
            glo[k] = INFINITY;
            ghi[k] = -INFINITY;
            for (int64_t i = 0; i < N; ++i) {
                glo[k] = fmin(glo[k], fmin(pm[k][i], pp[k][i]));
                ghi[k] = fmax(ghi[k], fmax(pm[k][i], pp[k][i]));
            }
        }
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < N; ++i) {
            double x[ORC_MAXD], pbar[ORC_MAXD];
            node_coords(P, i, x);
            double diss = 0.0;
            for (int k = 0; k < d; ++k) {
                double ak = alpha[k];
                if (P->diss != ORC_DISS_GLF) {
                    double clo[ORC_MAXD], chi[ORC_MAXD];
                    for (int j = 0; j < d; ++j) {
                        int local = (P->diss == ORC_DISS_LLLF) || (j == k);
                        clo[j] = local ? fmin(pm[j][i], pp[j][i]) : glo[j];
                        chi[j] = local ? fmax(pm[j][i], pp[j][i]) : ghi[j];
                    }
                    ak = partial_bound_box(P, x, clo, chi, k);
                }
                pbar[k] = 0.5 * (pp[k][i] + pm[k][i]);
                diss += ak * 0.5 * (pp[k][i] - pm[k][i]);
            }
            double hhat = ham(P, x, pbar) - diss;
            rate[i] = -hhat;
            if (P->varform && rate[i] > 0.0) rate[i] = 0.0;
        }
    }
    for (int k = 0; k < d; ++k) {
        free(pm[k]);
        free(pp[k]);
    }
    return rc;
}

/* GLF coefficients for the field phi (see alpha_from). */
int orc_alpha(const orc_problem* P, const double* phi, double* alpha)
{
    int d = P->ndim;
    if (P->dyn != ORC_DYN_QUADRATIC) {
        alpha_from(P, NULL, NULL, alpha);
        return 0;
    }
    int64_t N = orc_npoints(P);
    double* pm[ORC_MAXD];
    double* pp[ORC_MAXD];
    int rc = 0;
    for (int k = 0; k < d; ++k) {
        pm[k] = (double*)malloc(sizeof(double) * (size_t)N);
        pp[k] = (double*)malloc(sizeof(double) * (size_t)N);
    }
    for (int k = 0; k < d && rc == 0; ++k) rc = orc_derivs(P, phi, k, pm[k], pp[k], NULL);
    if (rc == 0) alpha_from(P, pm, pp, alpha);
    for (int k = 0; k < d; ++k) {
        free(pm[k]);
        free(pp[k]);
    }
    return rc;
}

/* CFL step (Sec. IV-D: lambda max|f'| <= 1; Sec. V-A: adaptive step):
 *   dt = min(cfl / sum_k(alpha_k / dx_k), t_final - t)
 * with the GLF coefficients in every dissipation mode: the local
 * coefficients' grid maxima are the GLF ones for every bound above.        */
double orc_cfl_dt(const orc_problem* P, const double* alpha, double cfl, double t,
                  double t_final)
{
    double s = 0.0;
    for (int k = 0; k < P->ndim; ++k) s += alpha[k] / orc_dx(P, k);
    double dt = (s > 0.0) ? cfl / s : (t_final - t);
    if (t_final - t < dt) dt = t_final - t;
    return dt;
}

/* One TVD-RK step of size dt (Sec. V-A):
 *   RK1: phi^{n+1} = phi^n + dt L(phi^n)
 *   RK2: phi1 = phi^n + dt L(phi^n);  phi^{n+1} = 1/2 (phi^n + phi1 + dt L(phi1))
 *   RK3: phi1 = phi^n + dt L(phi^n);
 *        phi2 = 3/4 phi^n + 1/4 (phi1 + dt L(phi1));
 *        phi^{n+1} = 1/3 phi^n + 2/3 (phi2 + dt L(phi2))
 * Each stage takes its own GLF coefficients from its own field.  Then, for
 * a reachable tube (g non-NULL), phi^{n+1} <- min(phi^{n+1}, g) (reading of
 * the variational inequality of Eq. 30, applied after each full step).
 * phi is updated in place.                                                */
int orc_step(const orc_problem* P, double* phi, const double* g, int rk_order, double dt)
{
    int64_t N = orc_npoints(P);
    double* L = (double*)malloc(sizeof(double) * (size_t)N);
    double* p1 = (double*)malloc(sizeof(double) * (size_t)N);
    double* p2 = (double*)malloc(sizeof(double) * (size_t)N);
    int rc = orc_rate(P, phi, NULL, NULL, L);
    if (rc == 0) {
        for (int64_t i = 0; i < N; ++i) p1[i] = phi[i] + dt * L[i];
        if (rk_order == 1) {
            for (int64_t i = 0; i < N; ++i) phi[i] = p1[i];
        } else if (rk_order == 2) {
            rc = orc_rate(P, p1, NULL, NULL, L);
            for (int64_t i = 0; i < N; ++i) phi[i] = 0.5 * (phi[i] + p1[i] + dt * L[i]);
        } else {
            rc = orc_rate(P, p1, NULL, NULL, L);
            for (int64_t i = 0; i < N; ++i) p2[i] = 0.75 * phi[i] + 0.25 * (p1[i] + dt * L[i]);
            if (rc == 0) rc = orc_rate(P, p2, NULL, NULL, L);
            for (int64_t i = 0; i < N; ++i)
                phi[i] = phi[i] / 3.0 + 2.0 / 3.0 * (p2[i] + dt * L[i]);
        }
        if (g)
            for (int64_t i = 0; i < N; ++i)
                if (g[i] < phi[i]) phi[i] = g[i];
    }
    free(L);
    free(p1);
    free(p2);
    return rc;
}

/* Integrate from t0 to t_final (odeCFLx of Listing 3): at the start of each
 * step the GLF coefficients of the current field give dt (FP64, reused by
 * all stages of the step), the time is accumulated in FP64 and the solve
 * stops once t >= t_final - 1e-12 |t_final|.  max_steps <= 0: no limit.     */
int orc_solve(const orc_problem* P, double* phi, const double* g, int rk_order, double cfl,
              double t0, double t_final, int64_t max_steps, orc_stats* st)
{
    double t = t0;
    int64_t steps = 0;
    double dtmin = INFINITY, dtmax = 0.0;
    int rc = 0;
    while (t < t_final - 1e-12 * fabs(t_final)) {
        if (max_steps > 0 && steps >= max_steps) break;
        double alpha[ORC_MAXD];
        rc = orc_alpha(P, phi, alpha);
        if (rc) break;
        double dt = orc_cfl_dt(P, alpha, cfl, t, t_final);
        if (!(dt > 0.0)) {
            rc = -3;
            break;
        }
        rc = orc_step(P, phi, g, rk_order, dt);
        if (rc) break;
        t += dt;
        ++steps;
        if (dt < dtmin) dtmin = dt;
        if (dt > dtmax) dtmax = dt;
    }
    if (st) {
        st->steps = steps;
        st->stages = steps * rk_order;
        st->dt_min = dtmin;
        st->dt_max = dtmax;
        st->t_end = t;
    }
    return rc;
}

/* Number of OpenMP threads this build uses (1 without OpenMP). */
int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Set the number of OpenMP threads of later calls (no effect without
 * OpenMP); used to time the oracle on one core and on all cores. */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Point evaluations, exported for the tests that pin the closed forms:
 * the Hamiltonian at one state/costate, and the per-node bound on |dH/dp_k|. */
double orc_ham(const orc_problem* P, const double* x, const double* p)
{
    return ham(P, x, p);
}

double orc_partial_bound(const orc_problem* P, const double* x, int k)
{
    return partial_bound(P, x, k);
}

/* ======================================================================== */
/* Discrete adjoint of a solve with a FIXED number of steps.                 */
/*                                                                          */
/* The forward map is the scheme above with dt = cfl / sum_k alpha_k/dx_k   */
/* (no shortened last step).  Its reverse is written out by hand: every     */
/* selection the forward makes -- ENO stencils, the argmax inside the WENO  */
/* regulariser, the signs of the optimal inputs, the min with the target,   */
/* the grid node attaining each GLF coefficient -- is frozen at the forward */
/* value, and the derivative of the smooth remainder is taken exactly (the  */
/* WENO weights included).  Parameters act through H, through the GLF       */
/* coefficients (via their argmax node) and through dt.                     */
/* ======================================================================== */

/* d(weno5_combine)/dv_m at v (same formula as weno5_combine):
 *   F = sum_k w_k phi_k,  w_k = a_k / sum a,  a_k = d_k / (s_k + eps)^2
 *   dF/dv = sum_k w_k dphi_k/dv - sum_k b_k (ds_k/dv + deps/dv),
 *   b_k = 2 w_k (phi_k - F) / (s_k + eps). */
static void weno5_combine_grad(const double* v, double* gv)
{
    double v1 = v[0], v2 = v[1], v3 = v[2], v4 = v[3], v5 = v[4];
    double phi[3] = {v1 / 3.0 - 7.0 * v2 / 6.0 + 11.0 * v3 / 6.0,
                     -v2 / 6.0 + 5.0 * v3 / 6.0 + v4 / 3.0,
                     v3 / 3.0 + 5.0 * v4 / 6.0 - v5 / 6.0};
    static const double dphi[3][5] = {{1.0 / 3.0, -7.0 / 6.0, 11.0 / 6.0, 0.0, 0.0},
                                      {0.0, -1.0 / 6.0, 5.0 / 6.0, 1.0 / 3.0, 0.0},
                                      {0.0, 0.0, 1.0 / 3.0, 5.0 / 6.0, -1.0 / 6.0}};
    double a[3] = {v1 - 2.0 * v2 + v3, v2 - 2.0 * v3 + v4, v3 - 2.0 * v4 + v5};
    double b[3] = {v1 - 4.0 * v2 + 3.0 * v3, v2 - v4, 3.0 * v3 - 4.0 * v4 + v5};
    static const double da[3][5] = {{1, -2, 1, 0, 0}, {0, 1, -2, 1, 0}, {0, 0, 1, -2, 1}};
    static const double db[3][5] = {{1, -4, 3, 0, 0}, {0, 1, 0, -1, 0}, {0, 0, 3, -4, 1}};
    double s[3];
    for (int k = 0; k < 3; ++k) s[k] = 13.0 / 12.0 * a[k] * a[k] + 0.25 * b[k] * b[k];
    int mstar = 0; /* argmax of v^2 (first one on ties), frozen */
    for (int m = 1; m < 5; ++m)
        if (v[m] * v[m] > v[mstar] * v[mstar]) mstar = m;
    double eps = 1e-6 * v[mstar] * v[mstar] + 1e-99;
    static const double d[3] = {0.1, 0.6, 0.3};
    double al[3], sum = 0.0;
    for (int k = 0; k < 3; ++k) {
        al[k] = d[k] / ((s[k] + eps) * (s[k] + eps));
        sum += al[k];
    }
    double F = 0.0, w[3];
    for (int k = 0; k < 3; ++k) {
        w[k] = al[k] / sum;
        F += w[k] * phi[k];
    }
    double bsum = 0.0, bk[3];
    for (int k = 0; k < 3; ++k) {
        bk[k] = 2.0 * w[k] * (phi[k] - F) / (s[k] + eps);
        bsum += bk[k];
    }
    for (int m = 0; m < 5; ++m) {
        double gm = 0.0;
        for (int k = 0; k < 3; ++k) {
            double ds = 13.0 / 6.0 * a[k] * da[k][m] + 0.5 * b[k] * db[k][m];
            gm += w[k] * dphi[k][m] - bk[k] * ds;
        }
        if (m == mstar) gm -= bsum * 2e-6 * v[mstar];
        gv[m] = gm;
    }
}

/* Coefficients of the ENO derivative at node i built on base index k, as a
 * combination of the extended line values u[i-3..i+3] (c[o+3]); the same
 * selections as eno_at. */
static void eno_at_coeffs(const double* u, int64_t i, int64_t k, double dx, int order, double* c)
{
    for (int o = 0; o < 7; ++o) c[o] = 0.0;
    /* Q1' = D1_{k+1/2} = (u[k+1] - u[k]) / dx */
    c[(k + 1) - i + 3] += 1.0 / dx;
    c[k - i + 3] -= 1.0 / dx;
    double a = D2(u, k, dx), b = D2(u, k + 1, dx);
    int64_t j, kstar;
    if (fabs(a) <= fabs(b)) {
        j = k;
        kstar = k - 1;
    } else {
        j = k + 1;
        kstar = k;
    }
    /* c (2(i-k) - 1) dx with c = D2_j = (u[j+1] - 2u[j] + u[j-1]) / (2 dx^2) */
    double f2 = (double)(2 * (i - k) - 1) * dx / (2.0 * dx * dx);
    c[(j + 1) - i + 3] += f2;
    c[j - i + 3] -= 2.0 * f2;
    c[(j - 1) - i + 3] += f2;
    if (order >= 3) {
        double e = D3h(u, kstar, dx), f = D3h(u, kstar + 1, dx);
        int64_t jj = (fabs(e) <= fabs(f)) ? kstar : kstar + 1;
        /* D3_{jj+1/2} = (u[jj+2] - 3u[jj+1] + 3u[jj] - u[jj-1]) / (6 dx^3) */
        double ss = (double)(i - kstar);
        double f3 = (3.0 * ss * ss - 6.0 * ss + 2.0) * dx * dx / (6.0 * dx * dx * dx);
        c[(jj + 2) - i + 3] += f3;
        c[(jj + 1) - i + 3] -= 3.0 * f3;
        c[jj - i + 3] += 3.0 * f3;
        c[(jj - 1) - i + 3] -= f3;
    }
}

/* Gradients of p^- and p^+ at node i w.r.t. u[i-3..i+3] (extended line). */
static void deriv_window_grad(int scheme, const double* u, int64_t i, double dx, double* gm,
                              double* gp)
{
    for (int o = 0; o < 7; ++o) gm[o] = gp[o] = 0.0;
    if (scheme == ORC_UPWIND1) {
        gm[3] = 1.0 / dx;
        gm[2] = -1.0 / dx;
        gp[4] = 1.0 / dx;
        gp[3] = -1.0 / dx;
    } else if (scheme == ORC_ENO2 || scheme == ORC_ENO3) {
        int order = scheme == ORC_ENO2 ? 2 : 3;
        eno_at_coeffs(u, i, i - 1, dx, order, gm);
        eno_at_coeffs(u, i, i, dx, order, gp);
    } else {
        double d[6], vm[5], vp[5], g5[5];
        for (int m = 0; m < 6; ++m) d[m] = (u[i - 3 + m + 1] - u[i - 3 + m]) / dx;
        for (int m = 0; m < 5; ++m) {
            vm[m] = d[m];
            vp[m] = d[5 - m];
        }
        /* d[m] = (u[i-2+m] - u[i-3+m]) / dx  ->  window offsets m-2 and m-3 */
        weno5_combine_grad(vm, g5);
        for (int m = 0; m < 5; ++m) {
            gm[m + 1] += g5[m] / dx;
            gm[m] -= g5[m] / dx;
        }
        weno5_combine_grad(vp, g5);
        for (int m = 0; m < 5; ++m) {
            int dm = 5 - m; /* vp[m] = d[5-m] */
            gp[dm + 1] += g5[m] / dx;
            gp[dm] -= g5[m] / dx;
        }
    }
}

/* dH/dp_k (frozen input selections, sgn(0) = +1) and dH/dprm_j at (x, p). */
static double sgn1(double v) { return v >= 0.0 ? 1.0 : -1.0; }

static void ham_grads(const orc_problem* P, const double* x, const double* p, double* hp,
                      double* hprm)
{
    const double* c = P->prm;
    int d = P->ndim;
    for (int j = 0; j < 8; ++j) hprm[j] = 0.0;
    switch (P->dyn) {
    case ORC_DYN_NORMAL_SPEED: {
        double s = 0.0;
        for (int k = 0; k < d; ++k) s += p[k] * p[k];
        s = sqrt(s);
        for (int k = 0; k < d; ++k) hp[k] = s > 0.0 ? c[0] * p[k] / s : 0.0;
        hprm[0] = s;
        break;
    }
    case ORC_DYN_TRANSLATE:
        for (int k = 0; k < d; ++k) {
            hp[k] = c[k];
            hprm[k] = p[k];
        }
        break;
    case ORC_DYN_AIR3D: {
        double ve = c[0], vp = c[1], um = c[2], dm = c[3];
        double X = x[0], Y = x[1], th = x[2];
        double s1 = p[0] * Y - p[1] * X - p[2];
        double g1 = sgn1(s1), g3 = sgn1(p[2]);
        hp[0] = -((-ve + vp * cos(th)) + um * g1 * Y);
        hp[1] = -(vp * sin(th) - um * g1 * X);
        hp[2] = um * g1 + dm * g3;
        hprm[0] = p[0];
        hprm[1] = -(p[0] * cos(th) + p[1] * sin(th));
        hprm[2] = -fabs(s1);
        hprm[3] = fabs(p[2]);
        break;
    }
    case ORC_DYN_CAR4D: {
        double th = x[2], v = x[3];
        hp[0] = -v * cos(th);
        hp[1] = -v * sin(th);
        hp[2] = c[0] * sgn1(p[2]);
        hp[3] = c[1] * sgn1(p[3]);
        hprm[0] = fabs(p[2]);
        hprm[1] = fabs(p[3]);
        break;
    }
    case ORC_DYN_ROCKETS: {
        /* H = -[p1 a cos th + p2 (a sin th + a - g) + ue |p1 x - p3|
         *       - up |p2 x + p3|]  (the closed form derived from Eq. 31)    */
        double a = c[0], g = c[1], ue = c[2], up = c[3];
        double X = x[0], th = x[2];
        double s1 = p[0] * X - p[2], s2 = p[1] * X + p[2];
        double g1 = sgn1(s1), g2 = sgn1(s2);
        hp[0] = -(a * cos(th) + ue * g1 * X);
        hp[1] = -(a * sin(th) + a - g - up * g2 * X);
        hp[2] = ue * g1 + up * g2;
        hprm[0] = -(p[0] * cos(th) + p[1] * (sin(th) + 1.0));
        hprm[1] = p[1];
        hprm[2] = -fabs(s1);
        hprm[3] = fabs(s2);
        break;
    }
    case ORC_DYN_DOUBLE_INT: /* H = -(p1 x2 - umax |p2|) */
        hp[0] = -x[1];
        hp[1] = c[0] * sgn1(p[1]);
        hprm[0] = fabs(p[1]);
        break;
    }
}

/* d alpha_k / d prm_j through the grid node attaining alpha_k (the first
 * one in C order, as alpha_from finds it). */
static void alpha_grads(const orc_problem* P, double* dalpha /* [4][8] */)
{
    int64_t N = orc_npoints(P);
    int d = P->ndim;
    double best[ORC_MAXD];
    int64_t at[ORC_MAXD];
    for (int k = 0; k < d; ++k) {
        best[k] = -1.0;
        at[k] = 0;
    }
    for (int64_t i = 0; i < N; ++i) {
        double x[ORC_MAXD];
        node_coords(P, i, x);
        for (int k = 0; k < d; ++k) {
            double b = partial_bound(P, x, k);
            if (b > best[k]) {
                best[k] = b;
                at[k] = i;
            }
        }
    }
    for (int j = 0; j < 4 * 8; ++j) dalpha[j] = 0.0;
    const double* c = P->prm;
    for (int k = 0; k < d; ++k) {
        double x[ORC_MAXD];
        node_coords(P, at[k], x);
        double* g = dalpha + 8 * k;
        switch (P->dyn) {
        case ORC_DYN_NORMAL_SPEED: g[0] = sgn1(c[0]); break; /* d|a|/da */
        case ORC_DYN_TRANSLATE: g[k] = sgn1(c[k]); break;
        case ORC_DYN_AIR3D:
            if (k == 0) {
                double w = -c[0] + c[1] * cos(x[2]);
                g[0] = -sgn1(w);
                g[1] = sgn1(w) * cos(x[2]);
                g[2] = fabs(x[1]);
            } else if (k == 1) {
                g[1] = fabs(sin(x[2]));
                g[2] = fabs(x[0]);
            } else {
                g[2] = 1.0;
                g[3] = 1.0;
            }
            break;
        case ORC_DYN_CAR4D:
            if (k == 2) g[0] = 1.0;
            if (k == 3) g[1] = 1.0;
            break;
        case ORC_DYN_ROCKETS:
            if (k == 0) { /* a |cos th| + ue |x| */
                g[0] = fabs(cos(x[2]));
                g[2] = fabs(x[0]);
            } else if (k == 1) { /* |a sin th + a - g| + up |x| */
                double w = c[0] * sin(x[2]) + c[0] - c[1];
                g[0] = sgn1(w) * (sin(x[2]) + 1.0);
                g[1] = -sgn1(w);
                g[3] = fabs(x[0]);
            } else { /* ue + up */
                g[2] = 1.0;
                g[3] = 1.0;
            }
            break;
        case ORC_DYN_DOUBLE_INT:
            if (k == 1) g[0] = 1.0; /* the bound umax */
            break;
        }
    }
}

/* Node index of extended-line position e on a line (base, stride s, n
 * nodes) and its weight, for ghost positions expressed through real nodes:
 * up to two (node, weight) pairs. */
static int ghost_terms(int64_t e, int64_t n, int periodic, int64_t* node, double* wt)
{
    if (e >= 0 && e < n) {
        node[0] = e;
        wt[0] = 1.0;
        return 1;
    }
    if (periodic) {
        node[0] = ((e % n) + n) % n;
        wt[0] = 1.0;
        return 1;
    }
    if (e < 0) { /* u0 + k (u0 - u1), k = -e */
        double k = (double)(-e);
        node[0] = 0;
        wt[0] = 1.0 + k;
        node[1] = 1;
        wt[1] = -k;
        return 2;
    }
    {
        double k = (double)(e - (n - 1));
        node[0] = n - 1;
        wt[0] = 1.0 + k;
        node[1] = n - 2;
        wt[1] = -k;
        return 2;
    }
}

/* Reverse of one rate evaluation L(u) scaled by the per-node weights lam:
 *   lam_u += J_L(u)^T lam,  hprm_acc += sum_i lam_i (-dH/dprm)(x_i, pbar_i),
 *   alpha_acc[k] += sum_i lam_i (p+_k - p-_k)/2,  and returns sum_i lam_i L_i
 * (the coefficient of dt). */
static double rate_adjoint(const orc_problem* P, const double* u, const double* alpha,
                           const double* lam, double* lam_u, double* hprm_acc, double* alpha_acc)
{
    int d = P->ndim;
    int G = orc_ghost_width(P->scheme);
    int64_t N = orc_npoints(P);
    double* pm[ORC_MAXD];
    double* pp[ORC_MAXD];
    for (int k = 0; k < d; ++k) {
        pm[k] = (double*)malloc(sizeof(double) * (size_t)N);
        pp[k] = (double*)malloc(sizeof(double) * (size_t)N);
        orc_derivs(P, u, k, pm[k], pp[k], NULL);
    }
    double dt_coef = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        if (lam[i] == 0.0) continue;
        double x[ORC_MAXD], pbar[ORC_MAXD], hp[ORC_MAXD], hprm[8];
        node_coords(P, i, x);
        double diss = 0.0;
        for (int k = 0; k < d; ++k) {
            pbar[k] = 0.5 * (pp[k][i] + pm[k][i]);
            diss += alpha[k] * 0.5 * (pp[k][i] - pm[k][i]);
            alpha_acc[k] += lam[i] * 0.5 * (pp[k][i] - pm[k][i]);
        }
        dt_coef += lam[i] * (-(ham(P, x, pbar) - diss));
        ham_grads(P, x, pbar, hp, hprm);
        for (int j = 0; j < 8; ++j) hprm_acc[j] += lam[i] * (-hprm[j]);
        /* scatter through every axis' window */
        int64_t rem = i, coord[ORC_MAXD];
        for (int k = d - 1; k >= 0; --k) {
            coord[k] = rem % P->n[k];
            rem /= P->n[k];
        }
        for (int k = 0; k < d; ++k) {
            int64_t n = P->n[k], s = stride_of(P, k);
            int64_t base = i - coord[k] * s; /* node 0 of this line */
            /* extended line of this node's axis */
            double* line = (double*)malloc(sizeof(double) * (size_t)n);
            double* ext = (double*)malloc(sizeof(double) * (size_t)(n + 2 * G));
            for (int64_t q = 0; q < n; ++q) line[q] = u[base + q * s];
            fill_line(line, n, G, P->periodic[k], ext);
            double gm[7], gp[7];
            deriv_window_grad(P->scheme, ext + G, coord[k], orc_dx(P, k), gm, gp);
            double sp = lam[i] * (-0.5 * hp[k] + 0.5 * alpha[k]);
            double sm = lam[i] * (-0.5 * hp[k] - 0.5 * alpha[k]);
            for (int o = -3; o <= 3; ++o) {
                double c = sp * gp[o + 3] + sm * gm[o + 3];
                if (c == 0.0) continue;
                int64_t nodes[2];
                double wts[2];
                int cnt = ghost_terms(coord[k] + o, n, P->periodic[k], nodes, wts);
                for (int q = 0; q < cnt; ++q) lam_u[base + nodes[q] * s] += c * wts[q];
            }
            free(line);
            free(ext);
        }
    }
    for (int k = 0; k < d; ++k) {
        free(pm[k]);
        free(pp[k]);
    }
    return dt_coef;
}

/* Forward solve with a fixed number of steps (dt from the CFL condition of
 * the state-only GLF coefficients, no shortened last step). */
int orc_solve_steps(const orc_problem* P, double* phi, const double* g, int rk_order, double cfl,
                    int64_t nsteps)
{
    double alpha[ORC_MAXD];
    int rc = orc_alpha(P, phi, alpha);
    if (rc) return rc;
    double dt = orc_cfl_dt(P, alpha, cfl, 0.0, INFINITY);
    for (int64_t n = 0; n < nsteps && rc == 0; ++n) rc = orc_step(P, phi, g, rk_order, dt);
    return rc;
}

/* Reverse sweep of orc_solve_steps (state-only GLF bounds).
 *  lamT   dLoss/dphi(t_end)                                   (N, in)
 *  lam0   dLoss/dphi0                                          (N, out)
 *  lam_g  dLoss/dtarget (nullable; only with a target)         (N, out)
 *  dprm   dLoss/dprm_j, j < 8, through H, alpha and dt          (out)
 *  phiT   the forward end state (nullable)                     (N, out)
 * Every forward stage input is stored, so memory is (steps * stages * N). */
int orc_adjoint(const orc_problem* P, const double* phi0, const double* g, int rk, double cfl,
                int64_t nsteps, const double* lamT, double* lam0, double* lam_g, double* dprm,
                double* phiT)
{
    if (P->dyn == ORC_DYN_QUADRATIC) return -5; /* reverse written for state-only bounds */
    if (P->diss != ORC_DISS_GLF || P->varform) return -6; /* reverse of the GLF form only */
    int d = P->ndim;
    int64_t N = orc_npoints(P);
    double alpha[ORC_MAXD];
    orc_alpha(P, phi0, alpha);
    double S = 0.0;
    for (int k = 0; k < d; ++k) S += alpha[k] / orc_dx(P, k);
    double dt = cfl / S;
    /* forward, storing the stage inputs u_0 = phi^n, u_1, u_2 */
    size_t NS = (size_t)N;
    double* st = (double*)malloc(sizeof(double) * NS * (size_t)(rk * nsteps + 1));
    if (!st) return -4;
    double* L = (double*)malloc(sizeof(double) * NS);
    double* cur = (double*)malloc(sizeof(double) * NS);
    memcpy(cur, phi0, sizeof(double) * NS);
    for (int64_t n = 0; n < nsteps; ++n) {
        double* u0 = st + NS * (size_t)(rk * n);
        memcpy(u0, cur, sizeof(double) * NS);
        orc_rate(P, u0, alpha, NULL, L);
        if (rk == 1) {
            for (size_t i = 0; i < NS; ++i) cur[i] = u0[i] + dt * L[i];
        } else {
            double* u1 = u0 + NS;
            for (size_t i = 0; i < NS; ++i) u1[i] = u0[i] + dt * L[i];
            orc_rate(P, u1, alpha, NULL, L);
            if (rk == 2) {
                for (size_t i = 0; i < NS; ++i) cur[i] = 0.5 * (u0[i] + u1[i] + dt * L[i]);
            } else {
                double* u2 = u1 + NS;
                for (size_t i = 0; i < NS; ++i) u2[i] = 0.75 * u0[i] + 0.25 * (u1[i] + dt * L[i]);
                orc_rate(P, u2, alpha, NULL, L);
                for (size_t i = 0; i < NS; ++i)
                    cur[i] = u0[i] / 3.0 + 2.0 / 3.0 * (u2[i] + dt * L[i]);
            }
        }
        if (g)
            for (size_t i = 0; i < NS; ++i)
                if (g[i] < cur[i]) cur[i] = g[i];
    }
    if (phiT) memcpy(phiT, cur, sizeof(double) * NS);

    /* reverse */
    double* lam = (double*)malloc(sizeof(double) * NS);  /* dLoss/dphi^{n+1} */
    double* ln = (double*)malloc(sizeof(double) * NS);   /* -> dLoss/dphi^n */
    double* lv = (double*)malloc(sizeof(double) * NS);   /* before the min */
    double* la = (double*)malloc(sizeof(double) * NS);   /* stage adjoints */
    double* lb = (double*)malloc(sizeof(double) * NS);
    double* w = (double*)malloc(sizeof(double) * NS);
    memcpy(lam, lamT, sizeof(double) * NS);
    if (lam_g) memset(lam_g, 0, sizeof(double) * NS);
    double hprm_acc[8] = {0}, alpha_acc[ORC_MAXD] = {0, 0, 0, 0}, dt_acc = 0.0;
    for (int64_t n = nsteps - 1; n >= 0; --n) {
        double* u0 = st + NS * (size_t)(rk * n);
        double* ulast = u0 + NS * (size_t)(rk - 1); /* input of the last stage */
        /* value before the min: recompute the last stage */
        orc_rate(P, ulast, alpha, NULL, L);
        for (size_t i = 0; i < NS; ++i) {
            double v;
            if (rk == 1) v = u0[i] + dt * L[i];
            else if (rk == 2) v = 0.5 * (u0[i] + ulast[i] + dt * L[i]);
            else v = u0[i] / 3.0 + 2.0 / 3.0 * (ulast[i] + dt * L[i]);
            if (g && g[i] < v) { /* the min took the target */
                lv[i] = 0.0;
                if (lam_g) lam_g[i] += lam[i];
            } else {
                lv[i] = lam[i];
            }
        }
        memset(ln, 0, sizeof(double) * NS);
        if (rk == 1) {
            /* phi^{n+1} = u0 + dt L(u0) */
            for (size_t i = 0; i < NS; ++i) {
                ln[i] += lv[i];
                w[i] = dt * lv[i];
            }
            dt_acc += rate_adjoint(P, u0, alpha, w, ln, hprm_acc, alpha_acc) / dt;
        } else if (rk == 2) {
            double* u1 = u0 + NS;
            /* phi^{n+1} = 1/2 u0 + 1/2 u1 + 1/2 dt L(u1) */
            memset(la, 0, sizeof(double) * NS);
            for (size_t i = 0; i < NS; ++i) {
                ln[i] += 0.5 * lv[i];
                la[i] += 0.5 * lv[i];
                w[i] = 0.5 * dt * lv[i];
            }
            dt_acc += rate_adjoint(P, u1, alpha, w, la, hprm_acc, alpha_acc) / dt;
            /* u1 = u0 + dt L(u0) */
            for (size_t i = 0; i < NS; ++i) {
                ln[i] += la[i];
                w[i] = dt * la[i];
            }
            dt_acc += rate_adjoint(P, u0, alpha, w, ln, hprm_acc, alpha_acc) / dt;
        } else {
            double* u1 = u0 + NS;
            double* u2 = u1 + NS;
            /* phi^{n+1} = 1/3 u0 + 2/3 u2 + 2/3 dt L(u2) */
            memset(lb, 0, sizeof(double) * NS);
            for (size_t i = 0; i < NS; ++i) {
                ln[i] += lv[i] / 3.0;
                lb[i] += 2.0 / 3.0 * lv[i];
                w[i] = 2.0 / 3.0 * dt * lv[i];
            }
            dt_acc += rate_adjoint(P, u2, alpha, w, lb, hprm_acc, alpha_acc) / dt;
            /* u2 = 3/4 u0 + 1/4 u1 + 1/4 dt L(u1) */
            memset(la, 0, sizeof(double) * NS);
            for (size_t i = 0; i < NS; ++i) {
                ln[i] += 0.75 * lb[i];
                la[i] += 0.25 * lb[i];
                w[i] = 0.25 * dt * lb[i];
            }
            dt_acc += rate_adjoint(P, u1, alpha, w, la, hprm_acc, alpha_acc) / dt;
            /* u1 = u0 + dt L(u0) */
            for (size_t i = 0; i < NS; ++i) {
                ln[i] += la[i];
                w[i] = dt * la[i];
            }
            dt_acc += rate_adjoint(P, u0, alpha, w, ln, hprm_acc, alpha_acc) / dt;
        }
        memcpy(lam, ln, sizeof(double) * NS);
    }
    memcpy(lam0, lam, sizeof(double) * NS);
    /* hprm_acc and alpha_acc were accumulated with weights c dt lam: they are
     * already dLoss/dprm (direct) and dLoss/dalpha (dissipation).  dt_acc is
     * dLoss/ddt.  dt = cfl / S(alpha):  ddt/dalpha_k = -cfl / (S^2 dx_k). */
    double dal[4 * 8];
    alpha_grads(P, dal);
    for (int j = 0; j < 8; ++j) {
        double v = hprm_acc[j];
        for (int k = 0; k < d; ++k) {
            double dL_dalpha = alpha_acc[k] - dt_acc * cfl / (S * S * orc_dx(P, k));
            v += dL_dalpha * dal[8 * k + j];
        }
        dprm[j] = v;
    }
    free(st);
    free(L);
    free(cur);
    free(lam);
    free(ln);
    free(lv);
    free(la);
    free(lb);
    free(w);
    return 0;
}
