"""The rockets game (Sec. VI-A, Eq. 31) and the double integrator (Table I)
on the GPU through the C ABI against the FP64 oracle: GLF coefficients,
rates of every scheme and kernel family (generic, tiled, paired WENO5
variants; global and local coefficients), whole tube solves and batched
solves (their adjoint: test_gpu_adjoint.py)."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import (check_fp32_solve, compare, flip_allowance, gpu_rate, noise_spread,
                         rate_tol, rounded, to_dev, trajectory_check)
from paper_2411_03501_gb300 import binding as B
from paper_2411_03501_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _rockets(scheme, dtype, n=(19, 17, 21)):
    spec = W.rockets(n=9, scheme=scheme, dtype=dtype)[0]
    spec["n"] = list(n)
    return spec


def _di(scheme, dtype):
    spec = W.double_integrator(n=9, scheme=scheme, dtype=dtype)[0]
    spec["n"] = [37, 29]
    return spec


@pytest.mark.parametrize("diss", ["glf", "llf"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("scheme", ["upwind1", "eno2", "eno3", "weno5"])
@pytest.mark.parametrize("kind", ["rockets", "double_integrator"])
def test_rate_parity(kind, scheme, dtype, diss):
    spec = _rockets(scheme, dtype) if kind == "rockets" else _di(scheme, dtype)
    spec["diss"] = diss
    phi = W.smooth_field(spec, seed=31) * (30.0 if kind == "rockets" else 1.0)
    phi = rounded(phi + 0.2 * W.rough_field(spec, seed=32) * (30.0 if kind == "rockets" else 1.0),
                  dtype)
    got, P = gpu_rate(spec, phi)
    want, alpha = oracle.rate(spec, phi)
    np.testing.assert_allclose(P.alpha(), alpha, rtol=1e-12)
    compare(got, want, rate_tol(spec, phi, want, alpha),
            flip_allowance(spec, phi, alpha) if dtype == "f32" else None, max_frac=0.05)


@pytest.mark.parametrize("pair", [1, 2])
def test_rockets_paired_variants(pair):
    """The paired WENO5 kernels carry the rockets Hamiltonian too."""
    spec = _rockets("weno5", "f32", n=(23, 19, 26))
    phi = rounded(30.0 * W.smooth_field(spec, seed=33) + 6.0 * W.rough_field(spec, seed=34), "f32")
    P = B.Problem(spec, check_finite=True)
    P.set_tile(16, 16, 8, 3, pair)
    x = to_dev(phi, "f32")
    out = torch.empty_like(x)
    P.rate(x, out)
    want, alpha = oracle.rate(spec, phi)
    compare(out.double().cpu().numpy(), want, rate_tol(spec, phi, want, alpha), max_frac=0.05)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_rockets_tube_solve(dtype):
    spec, phi0, g = W.rockets(n=9, dtype=dtype, t_final=0.4)
    spec["n"] = [25, 23, 21]
    phi0 = rounded(W.circle_sdf(spec, 8.0), dtype)
    g = phi0.copy()
    want, st_o = oracle.solve(spec, phi0, 0.4, 2, 0.75, target=g)
    P = B.Problem(spec, check_finite=True)
    x = to_dev(phi0, dtype)
    st = P.solve(x, to_dev(g, dtype), 0.0, 0.4)
    assert st["steps"] == st_o["steps"]
    got = x.double().cpu().numpy()
    if dtype == "f64":
        assert np.abs(got - want).max() <= 1e-9 * np.abs(want).max()
    else:
        check_fp32_solve(got, want, noise_spread(spec, phi0, g, 0.4, want), spec)
        # ENO2: every step against the oracle's step from the same FP32 input
        y = to_dev(phi0, dtype)
        trajectory_check(spec, P, y, to_dev(g, dtype), g, oracle.alpha(spec, phi0), 0.4,
                         st_o["steps"])
    assert np.all(got <= g + 1e-6 * np.abs(g).max())


def test_double_integrator_tube_solve_fp64():
    spec, phi0, g = W.double_integrator(n=61, t_final=0.5)
    want, st_o = oracle.solve(spec, phi0, 0.5, 2, 0.75, target=g)
    P = B.Problem(spec, check_finite=True)
    x = to_dev(phi0, "f64")
    st = P.solve(x, to_dev(g, "f64"), 0.0, 0.5)
    assert st["steps"] == st_o["steps"]
    assert np.abs(x.cpu().numpy() - want).max() <= 1e-9 * np.abs(want).max()


def test_batched_new_dynamics_match_single_solves():
    """Rockets (3-D, bit for bit) and double integrator (2-D, to rounding)
    problems share batched launches with an air3d problem (one scheme and
    RK order per batch: ENO2, RK2)."""
    specs, phis, gs = [], [], []
    for sp, p0, g in (W.rockets(n=21, t_final=0.3), W.double_integrator(n=41, dtype="f32", t_final=0.4),
                      W.air3d(n=17, t_final=0.3, scheme="eno2", rk=2)):
        specs.append(sp)
        phis.append(rounded(p0, "f32"))
        gs.append(to_dev(rounded(g, "f32"), "f32"))
    xs = [to_dev(p, "f32") for p in phis]
    B.Batch(specs, check_finite=True).solve(xs, gs)
    for i, sp in enumerate(specs):
        P = B.Problem(sp)
        y = to_dev(phis[i], "f32")
        P.solve(y, gs[i])
        torch.cuda.synchronize()
        if sp["ndim"] == 3:
            assert torch.equal(xs[i], y), i
        else:
            assert float((xs[i] - y).abs().max()) <= 1e-5 * float(y.abs().max())

