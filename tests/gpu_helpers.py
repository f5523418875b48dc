"""Shared helpers of the GPU parity tests: run the CUDA path through the
C ABI and the FP64 oracle on the same seeded inputs, and compare.

Tolerances.  FP64 kernels: rounding only, so 1e-11 relative to the scale of
the compared quantity.  FP32 kernels: every one-sided derivative is a
combination (coefficients summing in magnitude to < 4 after the 1/dx) of
differences of stencil values, each carrying a relative rounding of u = 2^-24
of max|phi|, so |dp_k| <~ 8 u max|phi| / dx_k; the rate then moves by at
most sum_k (|dH/dp_k| + alpha_k) |dp_k| <= sum_k 2 alpha_k |dp_k| plus u |L|.
The tests allow 8 times that:
    tol_rate = 8 * (16 u max|phi| sum_k alpha_k / dx_k + u max|L|).
A stage adds dt times that plus the rounding of the combination.  Where an
ENO stencil choice is within 1e-4 (relative) of a tie, the FP32 and FP64
choices may differ; there the bar grows by what the other stencil changes
(flip_allowance), and such nodes must be few.
"""
import numpy as np
import torch

import oracle
from conditioning import BAR, conditioning_mask, dilate, noise_response
from paper_2411_03501_gb300 import binding as B

U32 = 2.0 ** -24
U64 = 2.0 ** -53


def to_dev(arr, dtype):
    t = torch.float64 if dtype == "f64" else torch.float32
    return torch.as_tensor(np.ascontiguousarray(arr)).to("cuda", t).contiguous()


def rounded(arr, dtype):
    """The input as the GPU sees it, in float64."""
    return np.asarray(arr, dtype=np.float32 if dtype == "f32" else np.float64).astype(np.float64)


def gpu_rate(spec, phi):
    P = B.Problem(spec, check_finite=True)
    x = to_dev(phi, spec["dtype"])
    out = torch.empty_like(x)
    P.rate(x, out)
    torch.cuda.synchronize()
    return out.double().cpu().numpy(), P


def flip_allowance(spec, phi, alpha):
    """Per node, how much the rate L may validly differ because a near-tied
    ENO selection can go either way in another precision: the oracle reports
    the change of p-/p+ a flip would cause (flip_k); the rate moves by at most
    sum_k alpha_k (|dp+_k| + |dp-_k|) <= 2 sum_k alpha_k flip_k.  Zero for the
    schemes without selections."""
    out = np.zeros(spec["n"])
    if spec["scheme"] in ("eno2", "eno3"):
        for k in range(spec["ndim"]):
            _, _, f = oracle.derivs(spec, phi, k, with_ties=True)
            out += 2.0 * float(alpha[k]) * f
    return out


def step_flip_allowance(spec, phi, dt, rk, alpha, tol, max_frac=0.05):
    """The same for one RK step: the flip allowances of the stage inputs
    (phi, W1, W2 as the oracle computes them), weighted by dt, spread over the
    stencil width and doubled for what the next stages make of them.  Checks
    that at most max_frac of the nodes carry a flip larger than tol before
    the spreading."""
    if spec["scheme"] not in ("eno2", "eno3"):
        return np.zeros(spec["n"])
    u = [np.asarray(phi, dtype=np.float64)]
    L0, _ = oracle.rate(spec, u[0])
    if rk >= 2:
        u.append(u[0] + dt * L0)
    if rk >= 3:
        L1, _ = oracle.rate(spec, u[1])
        u.append(0.75 * u[0] + 0.25 * (u[1] + dt * L1))
    tot = sum(flip_allowance(spec, ui, alpha) for ui in u)
    frac = float((2.0 * dt * tot > tol).mean())
    assert frac <= max_frac, f"{frac:.3%} of nodes near an ENO tie"
    return 2.0 * dt * dilate(tot, spec)


def rate_tol(spec, phi, L, alpha):
    dx = oracle.dx(spec)
    M = np.abs(phi).max()
    if spec["dtype"] == "f64":
        return 1e-11 * (M * float(np.sum(np.asarray(alpha) / dx)) + np.abs(L).max() + 1e-30)
    return 8.0 * (16 * U32 * M * float(np.sum(np.asarray(alpha) / dx)) + U32 * np.abs(L).max())


def noise_spread(spec, phi0, target, t_final, ref, samples=2, rel=6e-8, seed=0):
    """Per node, how far the FP64 oracle's own solve moves when every step's
    field is perturbed by independent relative noise of FP32 size
    (conditioning.noise_response): the conditioning of the discrete problem
    (boundary closures, ENO selections, symmetric states that are unstable
    to asymmetric perturbations) at FP32 precision."""
    return noise_response(oracle, spec, phi0, target, t_final, ref, samples, rel, seed)


def adjoint_noise_spread(spec, phi0, g, nsteps, rk, lamT, ref0, ref_g, samples=3, rel=6e-8,
                         seed=0):
    """How far the FP64 oracle's adjoint (lam0, lam_target) moves when phi0 and
    lamT carry independent relative noise of FP32 size: the conditioning of
    the discrete adjoint (WENO weight derivatives, the regulariser's argmax,
    near-tied selections) at FP32 precision.  Returns (spread_lam0,
    spread_lam_target)."""
    rng = np.random.default_rng(seed)
    w0 = wg = 0.0
    for _ in range(samples):
        p = phi0 * (1.0 + rel * rng.standard_normal(phi0.shape))
        lt = lamT * (1.0 + rel * rng.standard_normal(lamT.shape))
        a0, ag, _, _ = oracle.adjoint(spec, p, nsteps, rk, spec["cfl"], lt, target=g)
        w0 = max(w0, float(np.abs(a0 - ref0).max()))
        wg = max(wg, float(np.abs(ag - ref_g).max()))
    return w0, wg


def check_fp32_solve(got, want, response, spec, factor=3.0, max_frac=0.05):
    """The FP32 precision bar for whole solves, node by node:
      * |got - want| <= 1e-4 max|want| (the bar asked of the path) at every
        node outside the ill-conditioned set C of conditioning_mask: the
        nodes where the FP64 oracle itself, perturbed by FP32-sized noise,
        moves by more than a third of that bar (`response` from
        noise_spread, per node);
      * on C, |got - want| <= factor x the oracle's own (dilated) response
        there, and C is at most max_frac of the nodes.
    ENO2/ENO3 solves are a discontinuous function of the rounding (a stencil
    choice near a tie can go either way in another precision, and the two
    trajectories then differ by more than rounding): for them the end state
    is held to max(1e-4 max|want|, factor x the largest response), and the
    tests check every step of the trajectory against the oracle's step from
    the same input instead (trajectory_check, near-tied choices apart).
    Returns {"err": max|got-want|/max|want|, "err_outside": the same off C,
    "frac_c": |C| / nodes}."""
    scale = float(np.abs(want).max())
    err = np.abs(got - want)
    if spec["scheme"] in ("eno2", "eno3"):
        bar = max(BAR * scale, factor * float(response.max()))
        assert float(err.max()) <= bar, (float(err.max()) / scale, bar / scale)
        return {"err": float(err.max()) / scale, "err_outside": None, "frac_c": None}
    mask, R = conditioning_mask(response, scale, spec, factor)
    frac = float(mask.mean())
    assert frac <= max_frac, f"ill-conditioned set covers {frac:.2%} of the nodes"
    out = float(err[~mask].max()) if (~mask).any() else 0.0
    assert out <= BAR * scale, (f"max|dphi| off the ill-conditioned set {out / scale:.3e} "
                                f"max|phi| > {BAR:g} at "
                                f"{np.unravel_index(np.where(mask, 0.0, err).argmax(), err.shape)}")
    if mask.any():
        over = err - np.maximum(BAR * scale, factor * R)
        assert not (mask & (over > 0)).any(), (
            f"max|dphi| on the ill-conditioned set exceeds {factor}x the oracle's response by "
            f"{over[mask].max():.3e} at {np.unravel_index(np.where(mask, over, -np.inf).argmax(), err.shape)}")
    return {"err": float(err.max()) / scale, "err_outside": out / scale, "frac_c": frac}


def trajectory_check(spec, P, x, gt, g32, a, t_final, nsteps):
    """Every step of the GPU trajectory against the oracle's step from the
    same FP32 input (stage tolerance; near-tied ENO selections apart)."""
    t = 0.0
    for _ in range(nsteps):
        dt = oracle.cfl_dt(spec, a, spec["cfl"], t, t_final)
        before = x.double().cpu().numpy()
        P.step(x, gt, t=t, dt=dt)
        got_step = x.double().cpu().numpy()
        want_step = oracle.step(spec, before, dt, spec["rk"], target=g32)
        L, _ = oracle.rate(spec, before)
        tol = spec["rk"] * dt * rate_tol(spec, before, L, a) + 8 * U32 * np.abs(before).max()
        compare(got_step, want_step, tol,
                step_flip_allowance(spec, before, dt, spec["rk"], a, tol))
        t += dt


def sign_ok(got, want, spec):
    """Sign disagreements only at nodes next to the oracle's zero level set
    (an axis neighbour of the node has the other oracle sign)."""
    s = want > 0
    near = np.zeros_like(s)
    for k in range(spec["ndim"]):
        for sh in (1, -1):
            near |= np.roll(s, sh, axis=k) != s
    return not (((got > 0) != s) & ~near).any()


def compare(got, want, tol, allowance=None, max_frac=1.0):
    """Element-wise |got - want| <= tol + allowance.  `allowance` (per node,
    from flip_allowance / step_flip_allowance) admits the other valid ENO
    stencil where a selection is near a tie; the nodes where it exceeds tol
    must be at most max_frac (flip_allowance callers pass 0.05; the spread
    step allowance checks its own count before spreading)."""
    err = np.abs(got - want)
    assert np.isfinite(got).all()
    bound = tol if allowance is None else tol + allowance
    bad = err > bound
    assert not bad.any(), (f"max excess {(err - bound).max():.3e} (tol {tol:.3e}) at "
                           f"{np.unravel_index((err - bound).argmax(), err.shape)}")
    if allowance is not None:
        frac = float((allowance > tol).mean())
        assert frac <= max_frac, f"{frac:.3%} of nodes near an ENO tie"
    return float(err.max())
