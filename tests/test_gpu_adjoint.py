"""The discrete adjoint on the GPU (through the C ABI) against the FP64
oracle's adjoint, against central finite differences of the GPU forward
map, across checkpoint counts, and through the autograd wrapper."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import adjoint_noise_spread, rounded, to_dev
from paper_2411_03501_gb300 import binding as B
from paper_2411_03501_gb300 import workloads as W
from paper_2411_03501_gb300.autograd import HJTube

pytestmark = pytest.mark.gpu


def _case(kind, scheme, dtype, rk=3):
    if kind == "air3d":
        spec = W.air3d(nx=[13, 12, 14], scheme=scheme, ve=4.0, vp=5.5, we=1.1, wp=0.9,
                       dtype=dtype, rk=rk)[0]
        nsteps = 4
    elif kind == "car4d":
        spec = W.car4d(n=8, scheme=scheme, dtype=dtype)[0]
        spec["n"] = [9, 8, 9, 8]
        nsteps = 3
    elif kind == "rockets":
        spec = W.rockets(n=12, scheme=scheme, a=1.1, g=30.0, ue=0.9, up=1.2, dtype=dtype)[0]
        spec["n"] = [13, 12, 11]
        spec["rk"] = rk
        nsteps = 4
    elif kind == "double_integrator":
        spec = W.double_integrator(n=17, scheme=scheme, umax=0.8, dtype=dtype)[0]
        spec["n"] = [17, 15]
        spec["rk"] = rk
        nsteps = 5
    else:
        spec = W.problem(2, [17, 15], [-1, -1], [1, 1], [False, True], scheme, "normal_speed",
                         [1.3], rk=rk, cfl=0.75, tube=True, dtype=dtype)
        nsteps = 5
    phi0 = W.smooth_field(spec, seed=21) + 0.5 * W.circle_sdf(
        spec, 0.4 * (spec["hi"][0] - spec["lo"][0]) / 2)
    g = phi0 + 0.2 + 0.3 * W.smooth_field(spec, seed=22)
    return spec, rounded(phi0, dtype), rounded(g, dtype), nsteps


def _gpu_adjoint(spec, phi0, g, nsteps, lamT, ncheck=0):
    P = B.Problem(spec)
    nbytes = B.lsp_adjoint_workspace_size(P.grid, P.opts, nsteps, ncheck)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    dt = spec["dtype"]
    phi = to_dev(phi0, dt)
    gt = to_dev(g, dt)
    B.lsp_hj_solve_ckpt(P.grid, P.opts, phi, gt, nsteps, ncheck, ws)
    lam0 = torch.empty_like(phi)
    lamg = torch.empty_like(phi)
    dprm = B.lsp_hj_adjoint(P.grid, P.opts, gt, nsteps, ncheck, to_dev(lamT, dt), lam0, lamg, ws)
    torch.cuda.synchronize()
    c = lambda t: t.double().cpu().numpy()  # noqa: E731
    return c(phi), c(lam0), c(lamg), np.array(dprm)


CASES = [("air3d", "weno5", 3), ("air3d", "eno3", 3), ("air3d", "eno2", 2),
         ("air3d", "upwind1", 1), ("car4d", "eno3", 3), ("normal2d", "weno5", 3),
         ("rockets", "eno2", 2), ("rockets", "weno5", 3), ("double_integrator", "eno2", 2)]


@pytest.mark.parametrize("kind,scheme,rk", CASES)
def test_fp64_adjoint_matches_oracle(kind, scheme, rk):
    """FP64 GPU adjoint (JP-form WENO gradient, two-pass gather) against the
    oracle's hand-written reverse (paper-form WENO gradient): the same
    derivative up to rounding."""
    spec, phi0, g, nsteps = _case(kind, scheme, "f64", rk)
    lamT = np.random.default_rng(3).standard_normal(spec["n"])
    phiT, lam0, lamg, dprm = _gpu_adjoint(spec, phi0, g, nsteps, lamT)
    o0, og, oprm, ophiT = oracle.adjoint(spec, phi0, nsteps, rk, spec["cfl"], lamT, target=g)
    assert np.abs(phiT - ophiT).max() <= 1e-11 * np.abs(ophiT).max()
    assert np.abs(lam0 - o0).max() <= 1e-9 * np.abs(o0).max(), np.abs(lam0 - o0).max()
    assert np.abs(lamg - og).max() <= 1e-9 * max(np.abs(og).max(), 1e-300)
    # parameter gradients may vanish (normal speed: dt L does not depend on
    # the speed); the absolute floor follows the scale of the field gradient
    npar = len(spec["params"])
    floor = 1e-9 * max(np.abs(oprm).max(), np.abs(o0).max())
    np.testing.assert_allclose(dprm[:npar], oprm[:npar], rtol=1e-8, atol=floor)


@pytest.mark.parametrize("kind,scheme,rk", CASES)
def test_fp32_adjoint_matches_oracle(kind, scheme, rk):
    """FP32 adjoint against the FP64 oracle with the bar of the FP32 solves:
    max(1e-4 max|lam|, 3 x the oracle's own spread under FP32-sized input
    noise) -- the WENO5 air3d adjoint is conditioned so that the FP64 oracle
    itself moves by ~2e-4 relative under such noise."""
    spec, phi0, g, nsteps = _case(kind, scheme, "f32", rk)
    lamT = rounded(np.random.default_rng(4).standard_normal(spec["n"]), "f32")
    _, lam0, lamg, dprm = _gpu_adjoint(spec, phi0, g, nsteps, lamT)
    o0, og, oprm, _ = oracle.adjoint(spec, phi0, nsteps, rk, spec["cfl"], lamT, target=g)
    s0, sg = adjoint_noise_spread(spec, phi0, g, nsteps, rk, lamT, o0, og)
    bar0 = max(1e-4 * np.abs(o0).max(), 3.0 * s0)
    barg = max(1e-4 * max(np.abs(og).max(), 1e-30), 3.0 * sg)
    assert np.abs(lam0 - o0).max() <= bar0, (np.abs(lam0 - o0).max(), bar0)
    assert np.abs(lamg - og).max() <= barg, (np.abs(lamg - og).max(), barg)
    npar = len(spec["params"])
    floor = 1e-4 * max(np.abs(oprm).max(), np.abs(o0).max())
    np.testing.assert_allclose(dprm[:npar], oprm[:npar], rtol=1e-3, atol=floor)


@pytest.mark.parametrize("rk,scheme", [(1, "upwind1"), (2, "eno2"), (3, "weno5")])
def test_fp32_keep_all_matches_checkpoints(rk, scheme):
    """FP32 (the fused passes with the gather prefetched through shared
    memory): keeping every stage input gives the gradient of sqrt(N)
    checkpointing, for each RK order's buffer rotation (RK1 alternates two
    buffers by step), up to the order of the FP32 boundary folds."""
    spec, phi0, g, _ = _case("air3d", scheme, "f32", rk)
    nsteps = 7
    lamT = rounded(np.random.default_rng(6).standard_normal(spec["n"]), "f32")
    ref = _gpu_adjoint(spec, phi0, g, nsteps, lamT, ncheck=0)
    got = _gpu_adjoint(spec, phi0, g, nsteps, lamT, ncheck=-1)
    assert np.array_equal(got[0], ref[0])  # the same forward
    for a, b in ((got[1], ref[1]), (got[2], ref[2])):
        assert np.abs(a - b).max() <= 1e-5 * max(np.abs(b).max(), 1e-30)
    np.testing.assert_allclose(got[3], ref[3], rtol=1e-5, atol=1e-6 * np.abs(ref[3]).max())


def test_checkpoint_counts_agree():
    """sqrt(N) checkpointing recomputes the same states: any checkpoint
    count, and keeping every state and stage input (ncheck < 0), gives the
    same gradient (up to the order of the FP64 parameter sums and of the
    boundary folds)."""
    spec, phi0, g, _ = _case("air3d", "weno5", "f64")
    nsteps = 9
    lamT = np.random.default_rng(5).standard_normal(spec["n"])
    ref = _gpu_adjoint(spec, phi0, g, nsteps, lamT, ncheck=0)
    for nc in (1, 2, 9, -1):
        got = _gpu_adjoint(spec, phi0, g, nsteps, lamT, ncheck=nc)
        assert np.abs(got[1] - ref[1]).max() <= 1e-12 * np.abs(ref[1]).max()
        np.testing.assert_allclose(got[3], ref[3], rtol=1e-12, atol=1e-14)


def _air3d_adjoint_problem(n, nsteps, dtype, radius=5.0):
    spec = W.air3d(n=n, dtype=dtype)[0]
    sdf = W.circle_sdf(spec, 0.0)  # distance to the cylinder axis
    rng = np.random.default_rng(20241106)
    q = np.stack([rng.uniform(spec["lo"][k], spec["hi"][k], 1024) for k in range(3)], 1)
    return spec, sdf, q


def _loss_of(tube, sdf_t, q_t, r, params):
    target = sdf_t - r
    phiT = tube(target, target, params)
    return tube.loss(phiT, q_t)


def test_autograd_matches_central_differences_fp64():
    """dLoss/d(v_e, v_p, turn bounds, target radius) through the autograd
    wrapper (FP64) against central differences of the same forward map."""
    spec, sdf, q = _air3d_adjoint_problem(21, 12, "f64")
    tube = HJTube(spec, nsteps=12)
    sdf_t = torch.as_tensor(sdf, device="cuda")
    q_t = torch.as_tensor(q, device="cuda")
    params = torch.tensor(spec["params"], dtype=torch.float64, requires_grad=True)
    r = torch.tensor(5.0, dtype=torch.float64, device="cuda", requires_grad=True)
    L = _loss_of(tube, sdf_t, q_t, r, params)
    L.backward()
    h = 1e-6
    with torch.no_grad():
        for j in range(4):
            pp = params.detach().clone()
            pm = params.detach().clone()
            pp[j] += h
            pm[j] -= h
            fd = (_loss_of(tube, sdf_t, q_t, r, pp) - _loss_of(tube, sdf_t, q_t, r, pm)).item() / (2 * h)
            assert abs(fd - params.grad[j].item()) <= 1e-5 * (abs(fd) + 1e-3), (j, fd, params.grad[j])
        fd = (_loss_of(tube, sdf_t, q_t, r + h, params) - _loss_of(tube, sdf_t, q_t, r - h, params)).item() / (2 * h)
        assert abs(fd - r.grad.item()) <= 1e-5 * (abs(fd) + 1e-3), (fd, r.grad)


@pytest.mark.slow
def test_adjoint_workload_fp32_against_fd_and_fp64():
    """The differentiation workload: air3d tube at 129^3, 200 RK3 steps,
    loss = smoothed volume + values at 1024 seeded query states; gradients
    with respect to v_e, v_p, the shared turn-rate bound w and the target
    radius r.

    * FP64 adjoint against FP64 central differences with h = 1e-6 (1e-5
      relative): the discrete map is piecewise smooth (input signs, the min
      with the target, ENO/WENO selections switch), so finite differences
      converge to the adjoint only once h is below the distance to the
      nearest switch -- at h = 1e-3 they are off by ~2% on v_p even in FP64.
    * FP32 adjoint (autotuned tile, as the benchmark runs it) against the
      FP64 adjoint, within 3x the spread of the FP64 gradients themselves
      when phi0 and the target carry independent relative noise of FP32 size
      (two samples; measured 2.3e-2, 2.5e-2 and 1.1e-2 on v_e, v_p, w:
      the v_p gradient is a small difference of large terms, so the map from
      rounding-sized input changes to it is what bounds any FP32 computation
      of it) plus 1e-4 relative for the FP32 reductions; and against FP32
      central differences with
      h = 1e-3 (6e-2 relative: the kinks above plus FP32 rounding of the
      loss)."""
    n, nsteps = 129, 200
    res = {}
    fd = {}
    for dtype, h in (("f64", 1e-6), ("f32", 1e-3)):
        spec, sdf, q = _air3d_adjoint_problem(n, nsteps, dtype)
        tube = HJTube(spec, nsteps=nsteps)
        tdt = torch.float64 if dtype == "f64" else torch.float32
        sdf_t = torch.as_tensor(sdf, device="cuda").to(tdt)
        q_t = torch.as_tensor(q, device="cuda").to(tdt)
        if dtype == "f32":  # the tile the benchmark runs this workload with
            tb, ta, ch, minb, pair = tube.autotune(sdf_t - 5.0)
            assert tb > 0 and ch > 0
        base = torch.tensor([5.0, 5.0, 1.0], dtype=torch.float64, requires_grad=True)
        r = torch.tensor(5.0, dtype=torch.float64, requires_grad=True)

        def run(b, rr, field=None):
            params = torch.stack([b[0], b[1], b[2], b[2]])
            target = (sdf_t if field is None else field) - rr.to("cuda").to(tdt)
            return tube.loss(tube(target, target, params), q_t)

        L = run(base, r)
        L.backward()
        res[dtype] = np.concatenate([base.grad.numpy(), [r.grad.item()]])
        if dtype == "f64":  # the gradients' own spread under FP32-sized input noise
            spread = np.zeros(4)
            for seed in (1, 2):
                rng = np.random.default_rng(seed)
                noisy = torch.as_tensor(sdf * (1 + 6e-8 * rng.standard_normal(sdf.shape)),
                                        device="cuda")
                b2 = base.detach().clone().requires_grad_(True)
                r2 = r.detach().clone().requires_grad_(True)
                run(b2, r2, noisy).backward()
                g2 = np.concatenate([b2.grad.numpy(), [r2.grad.item()]])
                spread = np.maximum(spread, np.abs(g2 - res["f64"]))
        vals = []
        with torch.no_grad():
            for j in range(3):
                bp = base.detach().clone()
                bm = base.detach().clone()
                bp[j] += h
                bm[j] -= h
                vals.append((run(bp, r) - run(bm, r)).item() / (2 * h))
            vals.append((run(base, r + h) - run(base, r - h)).item() / (2 * h))
        fd[dtype] = np.array(vals)
    np.testing.assert_allclose(res["f64"], fd["f64"], rtol=1e-5, atol=1e-6)
    # plus the FP32 rounding of the reductions that form the gradients (the
    # r gradient sums the FP32 field gradient over 2.1 M nodes; its input
    # spread is ~1e-9 relative, its FP32 sum ~5e-6 relative): 1e-4 relative
    dev = np.abs(res["f32"] - res["f64"])
    assert np.all(dev <= 3 * spread + 1e-4 * np.abs(res["f64"])), (dev, spread, res)
    np.testing.assert_allclose(res["f32"], fd["f32"], rtol=6e-2, atol=1e-2)


def _seam_and_edge_queries(spec, rng, nq):
    """Seeded query states uniform over the domain, plus states across the
    periodic theta seam (just below 2 pi, above it, below 0) and beyond the
    clamped x and y edges."""
    q = np.stack([rng.uniform(spec["lo"][k], spec["hi"][k], nq) for k in range(3)], 1)
    dth = 2 * np.pi / spec["n"][2]
    extra = np.array([[3.3, -1.7, 2 * np.pi - dth / 2], [0.4, 2.2, 2 * np.pi + dth / 4],
                      [-2.0, 5.0, -dth / 3], [25.0, 1.0, 0.4], [-8.0, -12.0, 5.0],
                      [4.0, 12.5, 2 * np.pi - 1e-3]])
    return np.concatenate([q, extra], 0)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_device_loss_matches_oracle(dtype):
    """lsp_loss_tube (smoothed volume of {phi <= 0} plus multilinear values at
    query states) against oracle.loss and oracle.loss_grad, value and
    gradient field element by element, with queries across the periodic
    theta seam and beyond the clamped edges.  The value is accumulated in
    FP64 from the field's values and the query coordinates as stored (the
    oracle gets the same rounded inputs), so it agrees to FP64 rounding in
    both precisions; the FP32 gradient is the volume term rounded to FP32
    plus the query weights added by FP32 atomics (a few u relative, u = 2^-24,
    plus u per unit weight)."""
    spec = W.air3d(nx=[33, 29, 31], dtype=dtype)[0]
    rng = np.random.default_rng(20241106)
    phi = rounded(W.circle_sdf(spec, 4.0, center=[7.0, 0.5]) + 0.3 * W.smooth_field(spec, seed=2),
                  dtype)
    q = rounded(_seam_and_edge_queries(spec, rng, 64), dtype)
    P = B.Problem(spec)
    val = torch.zeros(1, dtype=torch.float64, device="cuda")
    grad = torch.empty(spec["n"], dtype=torch.float64 if dtype == "f64" else torch.float32,
                       device="cuda")
    B.lsp_loss_tube(P.grid, dtype, to_dev(phi, dtype), to_dev(q, dtype), val, grad)
    torch.cuda.synchronize()
    want = oracle.loss(spec, phi, q)
    want_g = oracle.loss_grad(spec, phi, q)
    got_g = grad.double().cpu().numpy()
    if dtype == "f64":
        assert abs(val.item() - want) <= 1e-12 * abs(want)
        np.testing.assert_allclose(got_g, want_g, rtol=1e-12, atol=1e-15)
    else:
        assert abs(val.item() - want) <= 1e-10 * abs(want), (val.item(), want)
        tol_g = 8 * 2.0 ** -24 * (np.abs(want_g) + 1.0)
        assert np.all(np.abs(got_g - want_g) <= tol_g), np.abs(got_g - want_g).max()


def test_backward_through_an_overwritten_forward_raises():
    """Two forwards on one tube, then the backward of the first: its
    checkpoints were overwritten by the second forward, so the backward
    raises instead of returning another forward's gradients; the backward of
    the second forward equals that of a tube used once."""
    spec, sdf, q = _air3d_adjoint_problem(17, 6, "f64")
    sdf_t = torch.as_tensor(sdf, device="cuda")
    q_t = torch.as_tensor(q, device="cuda")

    def grads(tube, r0):
        params = torch.tensor(spec["params"], dtype=torch.float64, requires_grad=True)
        r = torch.tensor(r0, dtype=torch.float64, device="cuda", requires_grad=True)
        return _loss_of(tube, sdf_t, q_t, r, params), params

    tube = HJTube(spec, nsteps=6)
    L1, p1 = grads(tube, 5.0)
    L2, p2 = grads(tube, 4.5)
    with pytest.raises(RuntimeError, match="reused by a later forward"):
        L1.backward()
    L2.backward()
    fresh = HJTube(spec, nsteps=6)
    L3, p3 = grads(fresh, 4.5)
    L3.backward()
    # the same computation up to the order of FP64 atomic accumulations
    assert L2.item() == pytest.approx(L3.item(), rel=1e-12)
    torch.testing.assert_close(p2.grad, p3.grad, rtol=1e-10, atol=1e-12)
