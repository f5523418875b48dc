"""Pins of the oracle's discrete adjoint against central finite differences
of the FP64 oracle's forward map (fixed step count), in random directions of
the initial field and the target and along every dynamics parameter (every
dynamics with state-only LF bounds: the parameters act through H, through
the GLF coefficients and through dt)."""
import numpy as np
import pytest

from paper_2411_03501_gb300 import workloads as W


def _case(kind, scheme):
    if kind == "air3d":
        spec = W.air3d(nx=[13, 12, 14], scheme=scheme, ve=4.0, vp=5.5, we=1.1, wp=0.9)[0]
        nsteps = 4
    elif kind == "car4d":
        spec = W.car4d(n=8, scheme=scheme)[0]
        spec["n"] = [9, 8, 9, 8]
        nsteps = 3
    elif kind == "rockets":  # Sec. VI-A's game, every axis extrapolated
        spec = W.rockets(n=12, scheme=scheme, a=1.1, g=30.0, ue=0.9, up=1.2)[0]
        spec["n"] = [13, 12, 11]
        nsteps = 4
    elif kind == "double_integrator":
        spec = W.double_integrator(n=17, scheme=scheme, umax=0.8)[0]
        spec["n"] = [17, 15]
        nsteps = 5
    else:
        spec = W.problem(2, [17, 15], [-1, -1], [1, 1], [False, True], scheme, "normal_speed",
                         [1.3], rk=3, cfl=0.75, tube=True)
        nsteps = 5
    phi0 = W.smooth_field(spec, seed=21) + 0.5 * W.circle_sdf(spec, 0.4 * (spec["hi"][0] - spec["lo"][0]) / 2)
    g = phi0 + 0.2 + 0.3 * W.smooth_field(spec, seed=22)
    return spec, phi0, g, nsteps


def _J(orc, spec, phi0, g, nsteps, c):
    return float(np.sum(c * orc.solve_steps(spec, phi0, nsteps, spec["rk"], spec["cfl"], target=g)))


@pytest.mark.parametrize("kind,scheme", [("air3d", "weno5"), ("air3d", "eno3"), ("air3d", "eno2"),
                                         ("air3d", "upwind1"), ("car4d", "eno3"),
                                         ("normal2d", "weno5"), ("rockets", "eno2"),
                                         ("rockets", "weno5"), ("double_integrator", "eno2")])
def test_adjoint_matches_central_differences(orc, kind, scheme):
    spec, phi0, g, nsteps = _case(kind, scheme)
    rng = np.random.default_rng(5)
    c = rng.standard_normal(spec["n"])
    lam0, lamg, dprm, phiT = orc.adjoint(spec, phi0, nsteps, spec["rk"], spec["cfl"], c, target=g)
    np.testing.assert_allclose(phiT, orc.solve_steps(spec, phi0, nsteps, spec["rk"], spec["cfl"], g))
    # h = 1e-7: small enough not to cross a selection (ENO stencil, input
    # sign, min with the target) for these data, large enough for FP64
    h = 1e-7
    for trial in range(3):
        dphi = rng.standard_normal(spec["n"])
        fd = (_J(orc, spec, phi0 + h * dphi, g, nsteps, c) - _J(orc, spec, phi0 - h * dphi, g, nsteps, c)) / (2 * h)
        ad = float(np.sum(lam0 * dphi))
        assert abs(fd - ad) <= 2e-6 * (abs(fd) + 1.0), (trial, fd, ad)
        dg = rng.standard_normal(spec["n"])
        fd = (_J(orc, spec, phi0, g + h * dg, nsteps, c) - _J(orc, spec, phi0, g - h * dg, nsteps, c)) / (2 * h)
        ad = float(np.sum(lamg * dg))
        assert abs(fd - ad) <= 2e-6 * (abs(fd) + 1.0), (trial, fd, ad)
    for j, p0 in enumerate(spec["params"]):
        sp, sm = dict(spec), dict(spec)
        sp["params"] = list(spec["params"])
        sm["params"] = list(spec["params"])
        sp["params"][j] = p0 + h
        sm["params"][j] = p0 - h
        fd = (_J(orc, sp, phi0, g, nsteps, c) - _J(orc, sm, phi0, g, nsteps, c)) / (2 * h)
        assert abs(fd - dprm[j]) <= 2e-6 * (abs(fd) + 1.0), (j, fd, dprm[j])


def test_loss_gradient_matches_central_differences(orc):
    spec = W.air3d(nx=[11, 10, 12])[0]
    phi = W.circle_sdf(spec, 5.0) + 0.3 * W.smooth_field(spec, seed=2)
    rng = np.random.default_rng(20241106)
    q = np.stack([rng.uniform(spec["lo"][k], spec["hi"][k], 64) for k in range(3)], 1)
    g = orc.loss_grad(spec, phi, q)
    h = 1e-6
    for _ in range(3):
        d = rng.standard_normal(spec["n"])
        fd = (orc.loss(spec, phi + h * d, q) - orc.loss(spec, phi - h * d, q)) / (2 * h)
        assert abs(fd - np.sum(g * d)) <= 1e-7 * (1 + abs(fd))
    # interpolation reproduces a field that is linear in every coordinate
    xs = W.mesh(spec)
    lin = 0.3 + 0.2 * xs[0] - 0.7 * xs[1]
    val = sum(np.sum(w * lin.ravel()[f]) for f, w in orc._interp_weights(spec, q))
    want = np.sum(0.3 + 0.2 * q[:, 0] - 0.7 * q[:, 1])
    assert abs(val - want) < 1e-9
