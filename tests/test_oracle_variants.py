"""Pins of the oracle's local dissipation coefficients (LLF, LLLF: the local
siblings of the global-LF routine the paper names) and of the variational
form of the reachable-tube PDE (Eq. 30), against what the mathematics fixes:
reductions to the global form where the bound is constant, the comparison
principle of the Rusanov (local-LF) flux, the Hopf-Lax solution, exact
freezing of a receding front, monotone decrease in time, and agreement with
the min-with-target tube to O(dt)."""
import numpy as np
import pytest

from paper_2411_03501_gb300 import workloads as W


def _with(spec, **kw):
    s = dict(spec)
    s.update(kw)
    return s


# ------------------------------------------------------------ local LF
@pytest.mark.parametrize("dyn,params", [("normal_speed", [1.3]), ("translate", [0.7, -1.1])])
@pytest.mark.parametrize("diss", ["llf", "lllf"])
def test_local_equals_global_for_constant_bounds(orc, dyn, params, diss):
    """Where |dH/dp_k| has a constant bound the local coefficients are the
    global ones: identical rates."""
    spec = W.problem(2, [23, 19], [-1, -1], [1, 1], [False, True], "eno3", dyn, params)
    phi = W.smooth_field(spec, seed=3) + 0.3 * W.rough_field(spec, seed=4)
    want, _ = orc.rate(spec, phi)
    got, _ = orc.rate(_with(spec, diss=diss), phi)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("maker", ["air3d", "car4d", "quadratic"])
def test_llf_equals_lllf_for_separable_bounds(orc, maker):
    """The bounds provided depend on the state and at most on the costate of
    their own dimension, so the box of the other dimensions (global for LLF,
    local for LLLF) does not enter: both give the same rate."""
    if maker == "air3d":
        spec = W.air3d(nx=[13, 12, 14])[0]
    elif maker == "car4d":
        spec = W.car4d(n=9)[0]
    else:
        spec = W.problem(2, [21, 17], [-1, -1], [1, 1], [False, False], "weno5", "quadratic",
                         [])
    phi = W.smooth_field(spec, seed=5) + 0.3 * W.rough_field(spec, seed=6)
    a, _ = orc.rate(_with(spec, diss="llf"), phi)
    b, _ = orc.rate(_with(spec, diss="lllf"), phi)
    assert np.array_equal(a, b)


def test_local_dissipation_is_smaller_and_keeps_the_cfl_step(orc):
    """The local coefficient at a node never exceeds the global one (the grid
    maximum of the same bound), so with p+ >= p- (convex data, first-order
    differences) the local rate is never below... the global rate is never
    above the local one; the CFL step is the global one in every mode."""
    spec, phi, _ = W.air3d(nx=[15, 13, 16], scheme="upwind1")
    xs = W.mesh(spec)
    phi = xs[0] ** 2 + 0.5 * xs[1] ** 2 + 0.1 * np.cos(xs[2])  # convex in x, y
    glf, ag = orc.rate(spec, phi)
    llf, al = orc.rate(_with(spec, diss="llf"), phi)
    np.testing.assert_array_equal(ag, al)
    # dissipation enters the rate as + alpha (p+ - p-)/2 >= 0 on x, y; theta is
    # periodic and cos(theta) is not convex, but its bound is constant
    assert np.all(llf <= glf + 1e-12)
    assert (llf < glf - 1e-9).mean() > 0.5


def test_local_lf_is_monotone_first_order(orc):
    """The local-LF flux with alpha = the bound over the node's own costate
    interval (the Rusanov flux) is monotone for H = |p|^2/2 with first-order
    upwinding, forward Euler and CFL <= 1: ordered data stay ordered and
    sup-norm differences do not grow."""
    spec = W.problem(2, [36, 36], [-1, -1], [1, 1], [True, True], "upwind1", "quadratic", [],
                     diss="llf")
    rng = np.random.default_rng(12)
    phi0 = 0.5 * W.rough_field(spec, seed=7)
    psi0 = phi0 + np.abs(rng.standard_normal(spec["n"])) * 0.05
    phi, _ = orc.solve(spec, phi0, 0.2, 1, 0.5)
    psi, _ = orc.solve(spec, psi0, 0.2, 1, 0.5)
    assert np.all(phi <= psi + 1e-13)
    assert np.abs(phi - psi).max() <= np.abs(phi0 - psi0).max() + 1e-13


def test_local_lf_hopf_lax(orc):
    """H = |p|^2/2 with local coefficients converges to the Hopf-Lax
    solution min_y phi0(y) + |x - y|^2 / (2t) (brute force over the grid
    nodes), at least as closely as the global form."""
    errs = {}
    for diss in ("glf", "llf"):
        errs[diss] = []
        for n in (17, 33):
            spec = W.problem(2, [n, n], [-1, -1], [1, 1], [False, False], "eno2", "quadratic",
                             [], rk=2, diss=diss)
            xs = W.mesh(spec)
            phi0 = np.sqrt(xs[0] ** 2 + xs[1] ** 2) - 0.5
            t = 0.3
            phi, _ = orc.solve(spec, phi0, t, 2, 0.5)
            X = np.stack([xs[0].ravel(), xs[1].ravel()], 1)
            d2 = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
            hl = (phi0.ravel()[None, :] + d2 / (2 * t)).min(1).reshape(spec["n"])
            inner = (np.abs(xs[0]) < 0.7) & (np.abs(xs[1]) < 0.7)
            errs[diss].append(np.abs(phi - hl)[inner].max())
    assert errs["llf"][1] < errs["llf"][0]
    assert errs["llf"][1] < 0.06
    assert errs["llf"][1] <= errs["glf"][1] + 1e-12


# ------------------------------------------------------------ variational form
def test_variational_form_freezes_a_receding_front(orc):
    """phi_t + min[0, H] = 0 (Eq. 30) only lets phi decrease.  With a
    receding front (normal speed a < 0: the plain rate -a|grad phi| plus the
    LF dissipation is >= 0 on convex data with first-order differences) the
    clipped rate is zero everywhere and phi stays exactly where it started,
    while the plain PDE moves it."""
    spec = W.problem(2, [31, 27], [-1, -1], [1, 1], [False, False], "upwind1",
                     "normal_speed", [-0.8], rk=1, varform=True)
    xs = W.mesh(spec)
    phi0 = xs[0] ** 2 + 0.7 * xs[1] ** 2 - 0.3
    phi, st = orc.solve(spec, phi0, 0.25, 1, 0.9)
    assert st["steps"] > 5
    assert np.array_equal(phi, phi0)
    plain, _ = orc.solve(_with(spec, varform=False), phi0, 0.25, 1, 0.9)
    assert np.abs(plain - phi0).max() > 0.05


@pytest.mark.parametrize("rk", [1, 2, 3])
def test_variational_form_never_increases(orc, rk):
    """Every stage rate is <= 0 and TVD-RK steps are convex combinations of
    Euler steps, so phi^{n+1} <= phi^n at every node, for a game whose plain
    rate has both signs."""
    spec, phi, _ = W.air3d(nx=[17, 15, 16], scheme="weno5", rk=rk)
    spec = _with(spec, varform=True, tube=False)
    phi = phi + 0.5 * W.smooth_field(spec, seed=8)
    plain, _ = orc.rate(_with(spec, varform=False), phi)
    assert (plain > 1e-3).any() and (plain < -1e-3).any()
    a = orc.alpha(spec, phi)
    dt = orc.cfl_dt(spec, a, 0.75, 0.0, 1.0)
    for _ in range(3):
        nxt = orc.step(spec, phi, dt, rk)
        assert np.all(nxt <= phi + 1e-12 * np.abs(phi).max())
        phi = nxt


def test_variational_form_and_tube_converge_together(orc):
    """From phi0 = g the variational form and the min-with-target tube are
    two discretisations of the same reachable tube: on a fixed grid they
    differ (the tube lets phi rise again below g, the clipped rate never
    does), and the difference shrinks as grid and step are refined together
    -- about first order for the expanding front, and for the air3d game."""
    diffs = []
    for n in (41, 81, 161):
        spec, phi0, _ = W.normal_speed_2d(n)
        tube, _ = orc.solve(spec, phi0, 0.5, 2, 0.9, target=phi0)
        var, _ = orc.solve(_with(spec, varform=True), phi0, 0.5, 2, 0.9)
        diffs.append(np.abs(tube - var).max())
    assert diffs[0] > 1.8 * diffs[1] > 1.8 ** 2 * diffs[2]
    game = []
    for n in (17, 33):
        spec, phi0, g = W.air3d(nx=[n, n, n], scheme="eno2", rk=2, t_final=0.4)
        tube, _ = orc.solve(spec, phi0, 0.4, 2, 0.75, target=g)
        var, _ = orc.solve(_with(spec, varform=True), phi0, 0.4, 2, 0.75)
        game.append(np.abs(tube - var).max())
    assert game[0] > 1.4 * game[1]
