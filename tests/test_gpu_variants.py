"""Local dissipation coefficients (LLF, LLLF) and the variational form of the
reachable-tube PDE on the GPU (through the C ABI) against the FP64 oracle:
rates of every kernel family, steps and solves, the exact freezing of a
receding front, the paired WENO5 variants (the shared-face kernel's local
variant, the plane-paired fallback), batched solves, and the adjoint's
refusal."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import (check_fp32_solve, compare, flip_allowance, gpu_rate, noise_spread,
                         rate_tol, rounded, to_dev)
from paper_2411_03501_gb300 import binding as B
from paper_2411_03501_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _spec(kind, scheme, dtype):
    if kind == "air3d":  # tiled kernel in FP32 (3-D), generic in FP64
        return W.air3d(nx=[19, 17, 21], scheme=scheme, dtype=dtype)[0]
    if kind == "car4d":
        spec = W.car4d(n=9, scheme=scheme, dtype=dtype)[0]
        spec["n"] = [11, 13, 17, 23]
        return spec
    if kind == "quadratic3d":
        return W.problem(3, [15, 14, 17], [-1, -1, -1], [1, 1, 1], [False, True, False], scheme,
                         "quadratic", [], dtype=dtype)
    return W.problem(2, [23, 19], [-1, -1], [1, 1], [False, True], scheme, "quadratic", [],
                     dtype=dtype)


CASES = [(k, s, d) for d in ("f32", "f64") for k, s in
         (("air3d", "weno5"), ("air3d", "eno3"), ("car4d", "eno3"), ("car4d", "eno2"),
          ("car4d", "weno5"), ("quadratic3d", "weno5"), ("quadratic2d", "eno2"))]


@pytest.mark.parametrize("diss,varform", [("llf", False), ("lllf", False), ("glf", True),
                                          ("llf", True)])
@pytest.mark.parametrize("kind,scheme,dtype", CASES)
def test_rate_parity(kind, scheme, dtype, diss, varform):
    """L(phi) with local coefficients and/or the clip at zero, every node,
    against the oracle (the generic kernel in FP64 and in 2-D, the tiled one
    for 3-D/4-D FP32)."""
    spec = _spec(kind, scheme, dtype)
    spec.update(diss=diss, varform=varform)
    phi = rounded(W.smooth_field(spec, seed=11) + 0.2 * W.rough_field(spec, seed=12), dtype)
    got, _ = gpu_rate(spec, phi)
    want, alpha = oracle.rate(spec, phi)
    compare(got, want, rate_tol(spec, phi, want, alpha),
            flip_allowance(spec, phi, alpha) if dtype == "f32" else None, max_frac=0.05)
    if varform:
        assert (got <= 0).all()


def _rates_over_pairs(spec, phi, pairs):
    outs = []
    for p in pairs:
        P = B.Problem(spec, check_finite=True)
        P.set_tile(16, 16, 7, 3, p)
        x = to_dev(phi, "f32")
        o = torch.empty_like(x)
        P.rate(x, o)
        outs.append(o)
    return outs


def test_plane_paired_tile_falls_back_to_the_scalar_body():
    """The plane-paired WENO5 variant (pair = 1) evaluates the GLF form only:
    with local coefficients or the clip the tile runs the scalar local body,
    giving the scalar tile's bits."""
    spec = _spec("air3d", "weno5", "f32")
    spec.update(diss="llf", varform=True)
    phi = rounded(W.smooth_field(spec, seed=3) + 0.2 * W.rough_field(spec, seed=4), "f32")
    outs = _rates_over_pairs(spec, phi, (0, 1))
    assert torch.equal(outs[0], outs[1])


@pytest.mark.parametrize("kind", ["air3d", "car4d"])
@pytest.mark.parametrize("diss,varform", [("llf", False), ("lllf", True), ("glf", True)])
def test_shared_face_local_variant_agrees_with_the_scalar_local_body(kind, diss, varform):
    """The shared-face WENO5 kernel (pair = 2) has a local variant for
    state-only bounds: per-node coefficients of each plane's state and the
    clip.  It agrees with the scalar local body to FP32 rounding (the two
    arrange the same WENO5 arithmetic differently): within the rate tolerance
    of the oracle comparison, and both against the oracle."""
    spec = _spec(kind, "weno5", "f32")
    spec.update(diss=diss, varform=varform)
    phi = rounded(W.smooth_field(spec, seed=3) + 0.2 * W.rough_field(spec, seed=4), "f32")
    scalar, paired = (o.double().cpu().numpy() for o in _rates_over_pairs(spec, phi, (0, 2)))
    want, alpha = oracle.rate(spec, phi)
    tol = rate_tol(spec, phi, want, alpha)
    compare(paired, scalar, tol, None, max_frac=0.0)
    compare(paired, want, tol, None, max_frac=0.05)
    if varform:
        assert (paired <= 0).all()


def test_receding_front_is_frozen_on_the_gpu():
    """Normal speed a < 0 on convex data with first-order differences: the
    clipped rate is zero at every node, so RK1 steps leave phi unchanged bit
    for bit (and the plain form moves it)."""
    spec = W.problem(2, [31, 27], [-1, -1], [1, 1], [False, False], "upwind1", "normal_speed",
                     [-0.8], rk=1, varform=True)
    xs = W.mesh(spec)
    phi0 = rounded(xs[0] ** 2 + 0.7 * xs[1] ** 2 - 0.3, "f32")
    P = B.Problem(spec, check_finite=True)
    x = to_dev(phi0, "f32")
    st = P.solve(x, None, 0.0, 0.25)
    assert st["steps"] > 5
    assert torch.equal(x, to_dev(phi0, "f32"))
    spec["varform"] = False
    Q = B.Problem(spec)
    y = to_dev(phi0, "f32")
    Q.solve(y, None, 0.0, 0.25)
    assert float((y - x).abs().max()) > 0.05


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("diss,varform", [("llf", False), ("glf", True), ("lllf", True)])
def test_solve_parity(dtype, diss, varform):
    """Whole solves of the air3d game (WENO5, RK3) with the new options
    against the oracle: FP64 to 1e-9 of max|phi|, FP32 with the calibrated
    bar of the single-problem tests."""
    spec, phi0, g = W.air3d(nx=[21, 19, 18], scheme="weno5", dtype=dtype, t_final=0.3)
    spec.update(diss=diss, varform=varform, tube=not varform)
    phi0 = rounded(phi0, dtype)
    g = rounded(g, dtype)
    tgt = None if varform else g
    want, st_o = oracle.solve(spec, phi0, 0.3, 3, spec["cfl"], target=tgt)
    P = B.Problem(spec, check_finite=True)
    x = to_dev(phi0, dtype)
    st = P.solve(x, to_dev(g, dtype) if tgt is not None else None, 0.0, 0.3)
    assert st["steps"] == st_o["steps"]
    got = x.double().cpu().numpy()
    if dtype == "f64":
        assert np.abs(got - want).max() <= 1e-9 * np.abs(want).max()
    else:
        check_fp32_solve(got, want, noise_spread(spec, phi0, tgt, 0.3, want), spec)
    if varform:
        assert (got <= phi0 + 1e-6 * np.abs(phi0).max()).all()


def test_batched_with_local_dissipation_matches_single_solves():
    """Batched solves carry the options to every problem: 3-D problems end
    where their single-problem solves end, to a few FP32 ulps (the two
    kernels inline the local-coefficient code separately and may round the
    shared game terms differently; the global-LF form is compared bit for
    bit in the batched tests)."""
    probs = W.batched(count=6, seed=5, scale=0.15)
    specs = [p[0] for p in probs]
    for sp in specs:
        sp.update(diss="llf", varform=True)
    phis = [rounded(p[1], "f32") for p in probs]
    gs = [to_dev(rounded(p[2], "f32"), "f32") for p in probs]
    xs = [to_dev(p, "f32") for p in phis]
    B.Batch(specs, check_finite=True).solve(xs, gs)
    for i, sp in enumerate(specs):
        if sp["ndim"] != 3:
            continue
        P = B.Problem(sp)
        y = to_dev(phis[i], "f32")
        P.solve(y, gs[i])
        torch.cuda.synchronize()
        assert float((xs[i] - y).abs().max()) <= 1e-6 * float(y.abs().max()), i


def test_adjoint_refuses_the_new_forms():
    spec = W.air3d(nx=[13, 12, 14], dtype="f64")[0]
    for kw in ({"diss": "llf"}, {"varform": True}):
        sp = dict(spec, **kw)
        P = B.Problem(sp)
        with pytest.raises(B.LspError) as e:
            B.lsp_adjoint_workspace_size(P.grid, P.opts, 4, 0)
        assert e.value.status == B.LSP_EUNSUPPORTED
