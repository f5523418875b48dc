"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks a closed form,
an exactness or convergence property, a value printed in the paper, a
brute-force definition, or an invariant, chosen so that a dropped term, a
wrong sign or index, or a swapped operand in the oracle fails at least one.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2411_03501_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SCHEME_DEGREE = {"upwind1": 1, "eno2": 2, "eno3": 3, "weno5": 3}
SCHEME_G = {"upwind1": 1, "eno2": 2, "eno3": 3, "weno5": 3}


def _spec1d(n, scheme, periodic=False, lo=-1.0, hi=1.0, dyn="translate", params=(1.0,)):
    return W.problem(1, [n], [lo], [hi], [periodic], scheme, dyn, list(params))


# --------------------------------------------------------------- derivatives
@pytest.mark.parametrize("scheme", ["upwind1", "eno2", "eno3", "weno5"])
def test_polynomial_exactness(orc, scheme):
    """Sec. IV-A..IV-C: first-order upwinding is exact on lines, ENO2 on
    quadratics, ENO3 (and any convex WENO5 combination of third-order
    substencils) on cubics -- at every node whose stencil is inside the grid."""
    deg = SCHEME_DEGREE[scheme]
    G = SCHEME_G[scheme]
    rng = np.random.default_rng(1)
    for axis in range(2):
        spec = W.problem(2, [17, 19], [-1.3, 0.2], [0.9, 2.1], [False, False], scheme,
                         "translate", [1.0, 1.0])
        xs = W.mesh(spec)
        c = rng.uniform(-1, 1, size=deg + 1)
        u = xs[axis]
        phi = sum(c[m] * u ** m for m in range(deg + 1)) + 0.7 * xs[1 - axis] ** 2
        exact = sum(m * c[m] * u ** (m - 1) for m in range(1, deg + 1))
        pm, pp = orc.derivs(spec, phi, axis)
        sl = [slice(None)] * 2
        sl[axis] = slice(G, spec["n"][axis] - G)
        sl = tuple(sl)
        scale = np.abs(exact).max() + 1.0
        assert np.abs(pm[sl] - exact[sl]).max() < 1e-10 * scale
        assert np.abs(pp[sl] - exact[sl]).max() < 1e-10 * scale
    # one degree more is not reproduced (the test can fail)
    spec = _spec1d(21, scheme)
    x = W.axis_nodes(spec, 0)
    pm, _ = orc.derivs(spec, x ** (deg + 1), 0)
    assert np.abs(pm[G:-G] - (deg + 1) * x[G:-G] ** deg).max() > 1e-6


@pytest.mark.parametrize("scheme", ["upwind1", "eno2", "eno3", "weno5"])
def test_extrapolation_ghosts_exact_for_linear(orc, scheme):
    """Ghost cells by linear extrapolation continue a linear field exactly,
    so every scheme is exact on a linear field at the boundary nodes too."""
    spec = W.problem(2, [12, 9], [-2, -1], [3, 1], [False, False], scheme, "translate",
                     [1.0, 1.0])
    xs = W.mesh(spec)
    phi = 0.7 - 1.9 * xs[0] + 0.4 * xs[1]
    for axis, slope in ((0, -1.9), (1, 0.4)):
        pm, pp = orc.derivs(spec, phi, axis)
        assert np.abs(pm - slope).max() < 1e-12
        assert np.abs(pp - slope).max() < 1e-12


@pytest.mark.parametrize("scheme,order", [("upwind1", 1), ("eno2", 2), ("eno3", 3),
                                          ("weno5", 5)])
def test_convergence_order_periodic(orc, scheme, order):
    """Observed order of accuracy on smooth periodic data matches the order
    each scheme is built for (Sec. IV: first order, ENO2, ENO3, fifth-order
    WENO in smooth regions).  Also exercises the periodic ghost wrap at the
    ends of the line."""
    errs = []
    for n in (20, 40, 80):
        spec = _spec1d(n, scheme, periodic=True, lo=0.0, hi=1.0)
        x = W.axis_nodes(spec, 0)
        pm, pp = orc.derivs(spec, np.sin(2 * np.pi * x + 0.3), 0)
        ex = 2 * np.pi * np.cos(2 * np.pi * x + 0.3)
        errs.append(max(np.abs(pm - ex).max(), np.abs(pp - ex).max()))
    obs = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert obs.min() > order - 0.25, obs


@pytest.mark.parametrize("scheme", ["eno2", "eno3", "weno5"])
def test_eno_picks_smooth_stencil_at_kink(orc, scheme):
    """Sec. IV-B/IV-C: ENO chooses the smoother of the candidate stencils
    (smaller |divided difference|); WENO gives stencils that cross a kink a
    vanishing weight.  For phi = |x - c| (kink between two nodes) the left
    derivative just left of the kink and the right derivative just right of
    it are the exact one-sided slopes."""
    n = 41
    spec = _spec1d(n, scheme)
    x = W.axis_nodes(spec, 0)
    c = 0.013  # between nodes
    phi = np.abs(x - c)
    pm, pp = orc.derivs(spec, phi, 0)
    iL = np.where(x < c)[0][-1]  # last node left of the kink
    tol = 1e-9 if scheme != "weno5" else 1e-8
    # every left derivative at nodes left of the kink has a smooth stencil
    for i in range(3, iL + 1):
        assert abs(pm[i] + 1.0) < tol, (i, pm[i])
    for i in range(iL + 1, n - 3):
        assert abs(pp[i] - 1.0) < tol, (i, pp[i])


def _golden_weno():
    with open(os.path.join(GOLDEN, "weno5_optimal.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    return np.array([float(Fraction(v)) for v in rows[0]])


def test_weno5_optimal_formula_is_fifth_order_exact():
    """The printed optimal combination (Sec. IV-C) differentiates
    polynomials of degree <= 5 exactly -- a check of the fixture itself."""
    w = _golden_weno()
    dx = 0.37
    xi = 0.4
    for deg in range(6):
        f = lambda x: (x - 0.1) ** deg  # noqa: E731
        nodes = xi + dx * np.arange(-3, 3)  # x_{i-3} .. x_{i+2}
        d = np.diff(f(nodes)) / dx  # D+phi_{i-3} .. D+phi_{i+1}
        exact = deg * (xi - 0.1) ** (deg - 1) if deg > 0 else 0.0
        assert abs(np.dot(w, d) - exact) < 1e-11


def test_weno5_reduces_to_printed_optimal_combination(orc):
    """When every smoothness indicator is far below eps, the weights equal
    the optimal ones and the oracle's left derivative equals the printed
    fifth-order formula (Sec. IV-C).  Pins the substencil coefficients
    (including the sign of the first term of the third substencil) and the
    optimal weights 0.1, 0.6, 0.3."""
    w = _golden_weno()
    rng = np.random.default_rng(7)
    for _ in range(20):
        dx = rng.uniform(0.05, 0.5)
        v = 1.0 + 1e-6 * rng.standard_normal(7)  # differences, nearly constant
        phi = np.concatenate([[0.0], np.cumsum(v * dx)])  # 8 nodes
        spec = _spec1d(8, "weno5", lo=0.0, hi=7 * dx)
        pm, pp = orc.derivs(spec, phi, 0)
        i = 3
        got = pm[i]
        want = np.dot(w, v[i - 3: i + 2])
        # the weights deviate from optimal by O(sigma/eps) ~ 1e-6 and the
        # substencils differ by O(1e-6): expected agreement ~ 1e-12, while a
        # wrong optimal weight would move the result by ~ 1e-7
        assert abs(got - want) < 1e-10, (got, want)
        # right derivative: the mirror image
        i = 4
        want_p = np.dot(w, v[i - 2: i + 3][::-1])
        assert abs(pp[i] - want_p) < 1e-10


def test_weno5_differs_from_optimal_on_rough_data(orc):
    """With strongly varying smoothness the nonlinear weights move away from
    the optimal ones (the test above could not pass with fixed weights
    by accident)."""
    w = _golden_weno()
    v = np.array([0.0, 0.0, 0.0, 5.0, 5.0, 5.0, 5.0])
    phi = np.concatenate([[0.0], np.cumsum(v)])
    spec = _spec1d(8, "weno5", lo=0.0, hi=7.0)
    pm, _ = orc.derivs(spec, phi, 0)
    assert abs(pm[3] - np.dot(w, v[0:5])) > 0.1


@pytest.mark.parametrize("scheme", ["upwind1", "eno2", "eno3", "weno5"])
def test_derivative_is_homogeneous(orc, scheme):
    """The derivative of lam*phi is lam times the derivative of phi.  For
    WENO5 this holds only if eps scales like the smoothness indicators, i.e.
    eps = 1e-6 max(v_k^2) (the reading with squares): data whose indicators
    are comparable to eps make any other scaling visible."""
    rng = np.random.default_rng(12)
    v = 1.0 + 1e-3 * rng.standard_normal(40)
    phi = np.concatenate([[0.0], np.cumsum(v)]) * 0.1
    spec = _spec1d(41, scheme, lo=0.0, hi=4.0)
    pm0, pp0 = orc.derivs(spec, phi, 0)
    for lam in (1e3, 1e-3, -7.0):
        pm, pp = orc.derivs(spec, lam * phi, 0)
        assert np.abs(pm - lam * pm0).max() < 1e-11 * abs(lam)
        assert np.abs(pp - lam * pp0).max() < 1e-11 * abs(lam)


def test_eno_flip_size_reported(orc):
    """The diagnostic next to ENO derivatives: the change a near-tied
    selection would cause if taken the other way.  At a step (second
    differences +1 and -1, an exact tie) it is the jump between the two
    stencils; on a parabola (equal candidates) it vanishes to rounding; the
    schemes without selections report 0."""
    spec = _spec1d(9, "eno2", lo=0.0, hi=8.0)
    step = np.array([0.0, 0.0, 0.0, 0.0, 1.0, 1.0, 1.0, 1.0, 1.0])
    pm, pp, flip = orc.derivs(spec, step, 0, with_ties=True)
    assert flip.max() == pytest.approx(1.0)  # |S_a - S_b| dx / 2 with S = +-1
    x = W.axis_nodes(spec, 0)
    _, _, flip = orc.derivs(spec, x ** 2, 0, with_ties=True)
    assert flip.max() < 1e-12
    spec = _spec1d(9, "weno5")
    _, _, flip = orc.derivs(spec, step, 0, with_ties=True)
    assert np.all(flip == 0.0)


# --------------------------------------------------------------- Hamiltonians
def _air3d_f(x, u, d, ve, vp):
    X, Y, th = x
    return np.array([-ve + vp * np.cos(th) + u * Y, vp * np.sin(th) - u * X, d - u])


def _car4d_f(x, w, a):
    return np.array([x[3] * np.cos(x[2]), x[3] * np.sin(x[2]), w, a])


def test_air3d_hamiltonian_is_maxmin_of_dynamics(orc):
    """Sec. VI-A, Eqs. 31-32: H(x, p) = -max_u min_d p.f(x, u, d); the closed
    form with |.| switching terms equals the brute-force max-min over the
    input boxes (the optimum of a bilinear game sits at the box corners,
    which the sampling includes)."""
    spec, _, _ = W.air3d(n=9)
    ve, vp, we, wp = spec["params"]
    rng = np.random.default_rng(3)
    us = np.linspace(-we, we, 41)
    ds = np.linspace(-wp, wp, 41)
    for _ in range(50):
        x = np.array([rng.uniform(-6, 20), rng.uniform(-10, 10), rng.uniform(0, 2 * np.pi)])
        p = rng.standard_normal(3)
        best = max(min(p @ _air3d_f(x, u, d, ve, vp) for d in ds) for u in us)
        assert abs(orc.ham(spec, x, p) - (-best)) < 1e-12 * (1 + abs(best))


def test_car4d_hamiltonian_is_min_of_dynamics(orc):
    """Reach game: H = -min_u p.f (control minimises), brute force over the
    input box."""
    spec, _, _ = W.car4d(n=9)
    wm, am = spec["params"]
    rng = np.random.default_rng(4)
    ws = np.linspace(-wm, wm, 21)
    acs = np.linspace(-am, am, 21)
    for _ in range(50):
        x = np.array([rng.uniform(-4, 4), rng.uniform(-4, 4), rng.uniform(0, 2 * np.pi),
                      rng.uniform(0, 2)])
        p = rng.standard_normal(4)
        best = min(p @ _car4d_f(x, w, a) for w in ws for a in acs)
        assert abs(orc.ham(spec, x, p) - (-best)) < 1e-12 * (1 + abs(best))


def test_normal_speed_hamiltonian(orc):
    """H = a|p| is the support function of the ball of radius a."""
    spec, _, _ = W.normal_speed_2d(n=9)
    rng = np.random.default_rng(5)
    ang = np.linspace(0, 2 * np.pi, 20001)
    dirs = np.stack([np.cos(ang), np.sin(ang)], 1)
    for _ in range(20):
        p = rng.standard_normal(2)
        assert abs(orc.ham(spec, [0.1, 0.2], p) - (dirs @ p).max()) < 1e-6


@pytest.mark.parametrize("maker", ["air3d", "car4d"])
def test_partial_bounds_dominate_and_are_tight(orc, maker):
    """partialFunc (Listing 4): the per-node bound dominates |dH/dp_k| for
    every costate (central differences) and is attained for some costate."""
    spec = W.air3d(n=9)[0] if maker == "air3d" else W.car4d(n=9)[0]
    d = spec["ndim"]
    rng = np.random.default_rng(6)
    h = 1e-6
    for _ in range(30):
        x = np.array([rng.uniform(spec["lo"][k], spec["hi"][k]) for k in range(d)])
        best = np.zeros(d)
        for _ in range(200):
            p = rng.standard_normal(d)
            for k in range(d):
                e = np.zeros(d)
                e[k] = h
                g = (orc.ham(spec, x, p + e) - orc.ham(spec, x, p - e)) / (2 * h)
                b = orc.partial_bound(spec, x, k)
                assert abs(g) <= b + 1e-6
                best[k] = max(best[k], abs(g))
        for k in range(d):
            assert best[k] >= orc.partial_bound(spec, x, k) * 0.8


# --------------------------------------------------------------- LF and RK
def test_lf_with_exact_alpha_is_first_order_upwinding(orc):
    """Sec. IV-A + IV-D: for H = v p and first-order differences, the LF
    numerical Hamiltonian with alpha = |v| is exactly the upwind scheme of
    Eq. 7 (D^- phi when v > 0, D^+ phi when v < 0)."""
    for v in (1.7, -0.6):
        spec = _spec1d(30, "upwind1", periodic=True, lo=0, hi=1, params=(v,))
        x = W.axis_nodes(spec, 0)
        phi = np.sin(2 * np.pi * x) + 0.3 * np.cos(6 * np.pi * x)
        L, a = orc.rate(spec, phi)
        assert abs(a[0] - abs(v)) < 1e-15
        h = 1.0 / 30
        up = (phi - np.roll(phi, 1)) / h if v > 0 else (np.roll(phi, -1) - phi) / h
        assert np.abs(L - (-v * up)).max() < 1e-12


@pytest.mark.parametrize("rk", [1, 2, 3])
def test_tvd_rk_equals_taylor_polynomial_for_linear_rate(orc, rk):
    """Sec. V-A: for a linear semi-discrete system dphi/dt = A phi, TVD-RK1/2/3
    of step dt equal the Taylor polynomial of exp(dt A) of degree 1, 2, 3."""
    spec = W.problem(2, [13, 11], [0, 0], [1, 1], [True, True], "upwind1", "translate",
                     [0.8, -1.3])
    phi = W.smooth_field(spec, seed=11)
    dt = 0.01
    terms = [phi]
    for _ in range(rk):
        terms.append(orc.rate(spec, terms[-1])[0])
    want = sum(dt ** m / np.prod(range(1, m + 1)) * terms[m] for m in range(rk + 1))
    got = orc.step(spec, phi, dt, rk)
    assert np.abs(got - want).max() < 1e-12


def test_cfl_dt_and_step_count_config1(orc):
    """CFL step (Sec. IV-D, V-A) on the 2-D unit-speed front: alpha = (1, 1),
    dx = 0.02, CFL 0.9 -> dt = 0.009, 56 steps ending with 0.005."""
    g = dict(ln.split() for ln in open(os.path.join(GOLDEN, "normal_speed_2d.txt"))
             if ln.strip() and not ln.startswith("#"))
    spec, phi0, _ = W.normal_speed_2d(101)
    a = orc.alpha(spec, phi0)
    assert np.allclose(a, [1.0, 1.0])
    assert abs(orc.cfl_dt(spec, a, 0.9, 0.0, 0.5) - float(g["dt"])) < 1e-15
    _, st = orc.solve(spec, phi0, 0.5, 2, 0.9, max_steps=0)
    assert st["steps"] == int(g["steps"])
    assert abs(st["dt_min"] - float(g["dt_last"])) < 1e-12
    assert abs(st["t_end"] - 0.5) < 1e-12


# --------------------------------------------------------------- closed forms
def _zero_radius_along_x(phi, spec):
    n = spec["n"][0]
    mid = n // 2
    line = phi[mid:, mid]
    xx = W.axis_nodes(spec, 0)[mid:]
    j = np.where(line > 0)[0][0]
    return xx[j - 1] - line[j - 1] * (xx[j] - xx[j - 1]) / (line[j] - line[j - 1])


def test_normal_speed_closed_form_and_refinement(orc):
    """phi_t + a|grad phi| = 0 from a cone: phi(x, t) = max(|x| - a t, 0) - r0.
    The zero level set reaches radius 0.8 at t = 0.5 within half a cell, sign
    disagreements with the closed form occur only within one cell of the
    interface, and the error near the interface falls under refinement."""
    band_err = []
    for n in (51, 101, 201):
        spec, phi0, _ = W.normal_speed_2d(n)
        phi, _ = orc.solve(spec, phi0, 0.5, 2, 0.9)
        xs = W.mesh(spec)
        r = np.sqrt(xs[0] ** 2 + xs[1] ** 2)
        exact = np.maximum(r - 0.5, 0.0) - 0.3
        h = 2.0 / (n - 1)
        assert abs(_zero_radius_along_x(phi, spec) - 0.8) < 0.5 * h
        bad = (np.sign(phi) != np.sign(exact)) & (np.abs(exact) > h)
        assert not bad.any()
        band_err.append(np.abs(phi - exact)[np.abs(exact) < 0.1].max())
    assert band_err[0] > 3 * band_err[1] > 9 * band_err[2]


def test_translation_is_rigid_shift(orc):
    """Constant velocity (Eq. 4 with constant F): phi(x, t) = phi0(x - v t);
    with v = (1, -1) on the periodic unit square the field returns after
    t = 1.  WENO5 + RK3 error falls at third order or better."""
    errs = []
    for n in (24, 48):
        spec = W.problem(2, [n, n], [0, 0], [1, 1], [True, True], "weno5", "translate",
                         [1.0, -1.0])
        xs = W.mesh(spec)
        phi0 = np.sin(2 * np.pi * xs[0]) * np.cos(2 * np.pi * xs[1]) + 0.5 * np.sin(
            2 * np.pi * (xs[0] + xs[1]))
        phi, st = orc.solve(spec, phi0, 1.0, 3, 0.5)
        errs.append(np.abs(phi - phi0).max())
    assert errs[1] < 0.02
    assert errs[0] / errs[1] > 6.0


def test_hopf_lax_quadratic(orc):
    """Convex H = |p|^2/2: phi(x, t) = min_y phi0(y) + |x - y|^2 / (2 t)
    (Hopf-Lax), by brute force over the grid nodes; the LF coefficients here
    depend on the current costate range.  Error is O(dx) and shrinks."""
    errs = []
    for n in (17, 33):
        spec = W.problem(2, [n, n], [-1, -1], [1, 1], [False, False], "eno2", "quadratic",
                         [], rk=2)
        xs = W.mesh(spec)
        phi0 = np.sqrt(xs[0] ** 2 + xs[1] ** 2) - 0.5
        t = 0.3
        phi, _ = orc.solve(spec, phi0, t, 2, 0.5)
        X = np.stack([xs[0].ravel(), xs[1].ravel()], 1)
        d2 = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
        hl = (phi0.ravel()[None, :] + d2 / (2 * t)).min(1).reshape(spec["n"])
        inner = np.abs(xs[0]) < 0.7
        inner &= np.abs(xs[1]) < 0.7
        errs.append(np.abs(phi - hl)[inner].max())
    assert errs[1] < 0.06
    assert errs[1] < errs[0]


# --------------------------------------------------------------- monotone scheme
def test_monotone_first_order_scheme(orc):
    """Sec. IV-D: LF with first-order upwinding under CFL <= 1 is monotone:
    phi0 <= psi0 implies phi <= psi, and sup-norm differences do not grow.
    (Periodic axes: linear-extrapolation ghosts give the node next to the
    boundary a negative weight, so they are not monotone by construction.)"""
    spec = W.problem(2, [40, 40], [-1, -1], [1, 1], [True, True], "upwind1",
                     "normal_speed", [1.0])
    rng = np.random.default_rng(9)
    phi0 = W.rough_field(spec, seed=2)
    psi0 = phi0 + np.abs(rng.standard_normal(spec["n"])) * 0.1
    phi, _ = orc.solve(spec, phi0, 0.3, 1, 0.9)
    psi, _ = orc.solve(spec, psi0, 0.3, 1, 0.9)
    assert np.all(phi <= psi + 1e-13)
    assert np.abs(phi - psi).max() <= np.abs(phi0 - psi0).max() + 1e-13


@pytest.mark.parametrize("rk", [1, 2, 3])
def test_total_variation_non_increasing_1d(orc, rk):
    """1-D advection with first-order upwinding and TVD-RK (Sec. V-A) at
    CFL <= 1: total variation never grows, step by step."""
    spec = _spec1d(64, "upwind1", periodic=True, lo=0, hi=1, params=(1.0,))
    x = W.axis_nodes(spec, 0)
    phi = np.where((x > 0.2) & (x < 0.5), 1.0, 0.0) + 0.3 * np.sin(6 * np.pi * x)
    tv = lambda f: np.abs(np.diff(np.concatenate([f, f[:1]]))).sum()  # noqa: E731
    a = orc.alpha(spec, phi)
    dt = orc.cfl_dt(spec, a, 0.9, 0.0, 10.0)
    prev = tv(phi)
    for _ in range(40):
        phi = orc.step(spec, phi, dt, rk)
        cur = tv(phi)
        assert cur <= prev + 1e-12
        prev = cur


# --------------------------------------------------------------- reachable tube
def test_air3d_tube_invariants(orc):
    """Sec. VI-A (variational HJI, Eq. 30; tube by min with the target):
    phi <= g everywhere, the set {phi <= 0} only grows, and the game is
    symmetric under (x, y, theta) -> (x, -y, -theta), so is the solution."""
    spec, phi, g = W.air3d(n=25, t_final=0.6)
    n = spec["n"]
    vol_prev = (phi <= 0).sum()
    a = orc.alpha(spec, phi)
    t = 0.0
    for _ in range(6):
        dt = orc.cfl_dt(spec, a, 0.75, t, spec["t_final"])
        phi = orc.step(spec, phi, dt, 3, target=g)
        t += dt
        assert np.all(phi <= g)
        vol = (phi <= 0).sum()
        assert vol >= vol_prev
        vol_prev = vol
    mirrored = phi[:, ::-1, :]
    mirrored = mirrored[:, :, (-np.arange(n[2])) % n[2]]
    assert np.abs(phi - mirrored).max() < 1e-9
    assert vol_prev > (g <= 0).sum()


# --------------------------------------------------------------- more dynamics
def _rockets_f(x, ue, up, a, g):
    X, Z, th = x
    return np.array([a * np.cos(th) + ue * X, a * np.sin(th) + a + up * X - g, up - ue])


def test_rockets_hamiltonian_is_maxmin_of_eq31_dynamics(orc):
    """Sec. VI-A, Eq. 31: H = -max_{u_e} min_{u_p} p.f with the dynamics the
    equation displays (a_e = a_p = a), by brute force over the input boxes;
    the evader maximises, the pursuer minimises."""
    spec = W.rockets(n=9)[0]
    a, g, ue, up = spec["params"]
    rng = np.random.default_rng(13)
    ues = np.linspace(-ue, ue, 41)
    ups = np.linspace(-up, up, 41)
    for _ in range(50):
        x = np.array([rng.uniform(-64, 64), rng.uniform(-64, 64), rng.uniform(-1.5, 1.5)])
        p = rng.standard_normal(3)
        best = max(min(p @ _rockets_f(x, e, q, a, g) for q in ups) for e in ues)
        assert abs(orc.ham(spec, x, p) - (-best)) < 1e-12 * (1 + abs(best))


def test_double_integrator_hamiltonian_is_min_of_dynamics(orc):
    """Reach: the input minimises p.f over |u| <= umax."""
    spec = W.double_integrator(n=9)[0]
    um = spec["params"][0]
    rng = np.random.default_rng(14)
    us = np.linspace(-um, um, 41)
    for _ in range(50):
        x = rng.uniform(-1, 1, 2)
        p = rng.standard_normal(2)
        best = min(p @ np.array([x[1], u]) for u in us)
        assert abs(orc.ham(spec, x, p) - (-best)) < 1e-12 * (1 + abs(best))


@pytest.mark.parametrize("maker", ["rockets", "double_integrator"])
def test_partial_bounds_dominate_and_are_tight_new_dynamics(orc, maker):
    spec = W.rockets(n=9)[0] if maker == "rockets" else W.double_integrator(n=9)[0]
    d = spec["ndim"]
    rng = np.random.default_rng(15)
    h = 1e-6
    for _ in range(20):
        x = np.array([rng.uniform(spec["lo"][k], spec["hi"][k]) for k in range(d)])
        best = np.zeros(d)
        for _ in range(200):
            p = rng.standard_normal(d)
            for k in range(d):
                e = np.zeros(d)
                e[k] = h
                gk = (orc.ham(spec, x, p + e) - orc.ham(spec, x, p - e)) / (2 * h)
                assert abs(gk) <= orc.partial_bound(spec, x, k) + 1e-6 * (1 + abs(gk))
                best[k] = max(best[k], abs(gk))
        for k in range(d):
            assert best[k] >= orc.partial_bound(spec, x, k) * 0.8


def _double_integrator_time(x1, x2):
    """Minimum time to the origin for x1dot = x2, x2dot = u, |u| <= 1
    (bang-bang with one switch on the curve x1 = -x2|x2|/2)."""
    above = x1 > -x2 * np.abs(x2) / 2
    ta = x2 + 2 * np.sqrt(np.maximum(x1 + x2 ** 2 / 2, 0.0))
    tb = -x2 + 2 * np.sqrt(np.maximum(-x1 + x2 ** 2 / 2, 0.0))
    return np.where(above, ta, tb)


def test_double_integrator_tube_is_the_minimum_time_sublevel_set(orc):
    """The reachable tube of a small disc D around the origin after time t
    brackets {T <= t}, T the closed-form minimum time to the origin: since
    T(x) <= T_D(x) + max_{y in D} T(y) (reach D, then the origin) and
    T_D <= T, nodes with T < t - m are in the computed tube and nodes with
    T > t + max_D T + m are not; m covers the grid's numerical diffusion."""
    spec, phi0, g = W.double_integrator(n=81, radius=0.05, t_final=0.6)
    phi, _ = orc.solve(spec, phi0, 0.6, 2, 0.75, target=g)
    xs = W.mesh(spec)
    T = _double_integrator_time(xs[0], xs[1])
    ang = np.linspace(0, 2 * np.pi, 721)
    rad = np.linspace(0, 0.05, 51)[:, None]
    tmax_disc = _double_integrator_time(rad * np.cos(ang), rad * np.sin(ang)).max()
    m = 0.1
    inside, outside = T < 0.6 - m, T > 0.6 + tmax_disc + m
    assert np.all(phi[inside] <= 0)
    assert np.all(phi[outside] > 0)
    assert inside.sum() > 50 and outside.sum() > 1000
