"""Batched solves (many problems of different shapes, dynamics and step
sizes in shared launches) against single-problem solves and the oracle."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import check_fp32_solve, noise_spread, rounded, sign_ok, to_dev
from paper_2411_03501_gb300 import binding as B
from paper_2411_03501_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _mixed(scale=0.15, count=12, seed=20241105):
    probs = W.batched(count=count, seed=seed, scale=scale)
    specs = [p[0] for p in probs]
    phis = [rounded(p[1], "f32") for p in probs]
    gs = [rounded(p[2], "f32") for p in probs]
    return specs, phis, gs


@pytest.mark.parametrize("use_graph", [False, True])
def test_batched_equals_single_problem_solves(use_graph):
    """Every problem of a mixed 2-D / 3-D batch ends where its own
    single-problem solve ends: bit for bit for the 3-D problems run with the
    paired shared-face body (the one the batched kernel inlines for WENO5;
    same arithmetic per node), to FP32 rounding for the 2-D ones (the
    single-problem path runs the generic kernel there)."""
    specs, phis, gs = _mixed()
    Bt = B.Batch(specs, use_graph=use_graph, check_finite=True)
    xs = [to_dev(p, "f32") for p in phis]
    gts = [to_dev(g, "f32") for g in gs]
    stats = Bt.solve(xs, gts)
    torch.cuda.synchronize()
    for i, sp in enumerate(specs):
        P = B.Problem(sp)
        if sp["ndim"] == 3:
            P.set_tile(16, 16, 64, 3, 2)  # the paired body the batched kernel runs for WENO5
        y = to_dev(phis[i], "f32")
        st = P.solve(y, gts[i])
        torch.cuda.synchronize()
        assert stats[i]["steps"] == st["steps"], (i, stats[i], st)
        if sp["ndim"] == 3:
            assert torch.equal(xs[i], y), (i, float((xs[i] - y).abs().max()))
        else:
            err = float((xs[i] - y).abs().max())
            assert err <= 1e-5 * float(y.abs().max()), (i, err)


def test_batched_matches_oracle_on_small_problems():
    """A few batched problems against the FP64 oracle's own solves, with the
    FP32 precision bar of the single-problem tests (check_fp32_solve: 1e-4
    max|phi| at every node except the few where the oracle itself, perturbed
    by FP32-sized noise, moves by more than a third of that -- e.g. the
    symmetric valley at theta = 0, y = 0 of an air3d tube, which FP32
    rounding desymmetrises -- and 3x the oracle's own response there)."""
    specs, phis, gs = _mixed(scale=0.3, count=6, seed=7)
    Bt = B.Batch(specs)
    xs = [to_dev(p, "f32") for p in phis]
    Bt.solve(xs, [to_dev(g, "f32") for g in gs])
    torch.cuda.synchronize()
    for i, sp in enumerate(specs):
        want, _ = oracle.solve(sp, phis[i], sp["t_final"], sp["rk"], sp["cfl"], target=gs[i])
        got = xs[i].double().cpu().numpy()
        resp = noise_spread(sp, phis[i], gs[i], sp["t_final"], want)
        check_fp32_solve(got, want, resp, sp)
        assert sign_ok(got, want, sp)


def test_batched_zero_and_uneven_horizons():
    """Per-problem t_final: a zero horizon leaves the field untouched, and
    problems with very different step counts share the launches."""
    specs, phis, gs = _mixed(count=4, seed=3)
    Bt = B.Batch(specs)
    xs = [to_dev(p, "f32") for p in phis]
    tf = [0.0, specs[1]["t_final"], 0.3 * specs[2]["t_final"], specs[3]["t_final"]]
    stats = Bt.solve(xs, [to_dev(g, "f32") for g in gs], t_final=tf)
    torch.cuda.synchronize()
    assert stats[0]["steps"] == 0
    assert torch.equal(xs[0], to_dev(phis[0], "f32"))
    for i in (1, 2, 3):
        assert stats[i]["steps"] > 0
        assert stats[i]["t_end"] == pytest.approx(tf[i], rel=1e-12)


def test_batched_rejections():
    specs, phis, gs = _mixed(count=2)
    q = W.problem(2, [16, 16], [-1, -1], [1, 1], [False, False], "weno5", "quadratic", [])
    with pytest.raises(B.LspError) as e:
        B.Batch(specs + [q])
    assert e.value.status == B.LSP_EUNSUPPORTED
    Bt = B.Batch(specs)
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(B.LspError) as e:
        B.lsp_hj_solve_batched(Bt.grids, Bt.opts, [to_dev(p, "f32") for p in phis],
                               [to_dev(g, "f32") for g in gs], [s["t_final"] for s in specs], small)
    assert e.value.status == B.LSP_ENOMEM
    o = B.make_opts(rk_order=1, scheme="weno5", dtype="f32", tube=True)
    with pytest.raises(B.LspError) as e:
        B.lsp_batched_workspace_size(Bt.grids, o)
    assert e.value.status == B.LSP_EUNSUPPORTED


def _mixed_with_4d(scheme, rk, seed=11):
    specs, phis, gs = _mixed(count=8, seed=seed)
    sp, phi, g = W.car4d(n=12, t_final=0.4)
    specs.append(sp)
    phis.append(rounded(phi, "f32"))
    gs.append(rounded(g, "f32"))
    for s in specs:
        s["scheme"] = scheme
        s["rk"] = rk
    return specs, phis, gs


@pytest.mark.parametrize("scheme,rk", [("weno5", 3), ("eno2", 2), ("eno3", 3)])
def test_persistent_equals_stage_synchronous(scheme, rk):
    """The persistent launch (one cooperative launch, work items taken in
    (step, stage, tile) order, per-problem completion counters) runs the same
    tile computations as the stage-synchronous launches: identical fields
    bit for bit, for 2-D, 3-D and 4-D problems with uneven horizons (one of
    them zero)."""
    specs, phis, gs = _mixed_with_4d(scheme, rk)
    tf = [s["t_final"] * f for s, f in zip(specs, [1.0, 0.0, 0.5, 1.0, 0.2, 1.0, 0.7, 1.0, 1.0])]
    gts = [to_dev(g, "f32") for g in gs]
    ref = [to_dev(p, "f32") for p in phis]
    st_ref = B.Batch(specs, check_finite=True).solve(ref, gts, t_final=tf)
    got = [to_dev(p, "f32") for p in phis]
    st_got = B.Batch(specs, check_finite=True, persistent=True).solve(got, gts, t_final=tf)
    torch.cuda.synchronize()
    assert st_got == st_ref
    assert st_got[1]["steps"] == 0
    for i in range(len(specs)):
        assert torch.equal(got[i], ref[i]), (i, float((got[i] - ref[i]).abs().max()))


def test_persistent_wait_runs_out_and_context_survives():
    """A problem whose tiles are never counted done (the library's testing
    hook) makes the first wait on it run out: the launch ends, the solve
    reports LSP_ETIMEOUT (directly with check_finite, else through
    lsp_check_status), and the context stays usable -- the next solve on the
    same workspace succeeds and matches the stage-synchronous result."""
    specs, phis, gs = _mixed(count=4, seed=3)
    gts = [to_dev(g, "f32") for g in gs]
    Bt = B.Batch(specs, check_finite=True, persistent=True, wait_ms=50)
    Bq = B.Batch(specs, check_finite=False, persistent=True, wait_ms=50)
    prev = B.lsp_debug_stall_problem(1)
    try:
        with pytest.raises(B.LspError) as e:
            Bt.solve([to_dev(p, "f32") for p in phis], gts)
        assert e.value.status == B.LSP_ETIMEOUT
        Bq.solve([to_dev(p, "f32") for p in phis], gts)
        with pytest.raises(B.LspError) as e:
            B.lsp_check_status(Bq.workspace)
        assert e.value.status == B.LSP_ETIMEOUT
    finally:
        B.lsp_debug_stall_problem(prev)
    got = [to_dev(p, "f32") for p in phis]
    Bt.solve(got, gts)
    ref = [to_dev(p, "f32") for p in phis]
    B.Batch(specs).solve(ref, gts)
    torch.cuda.synchronize()
    for i in range(len(specs)):
        assert torch.equal(got[i], ref[i]), i


@pytest.mark.parametrize("tiles", [0b000101, 0b001010, 0b000110])
def test_batched_tile_shapes(tiles):
    """Per-dimension tile shapes (opts.batch_tiles: 16 x 16, 32 x 8, 64 x 4,
    256 threads each): the 3-D problems end bit for bit where single-problem
    solves on the same tile end (the paired shared-face body for WENO5), the
    2-D ones to FP32 rounding; the persistent launch equals the
    stage-synchronous one bit for bit."""
    shapes = [(16, 16), (32, 8), (64, 4)]
    specs, phis, gs = _mixed()
    gts = [to_dev(g, "f32") for g in gs]
    xs = [to_dev(p, "f32") for p in phis]
    stats = B.Batch(specs, check_finite=True, tiles=tiles).solve(xs, gts)
    ys = [to_dev(p, "f32") for p in phis]
    B.Batch(specs, check_finite=True, tiles=tiles, persistent=True).solve(ys, gts)
    torch.cuda.synchronize()
    for i, sp in enumerate(specs):
        assert torch.equal(xs[i], ys[i]), i
        P = B.Problem(sp)
        if sp["ndim"] == 3:
            tb, ta = shapes[(tiles >> 2) & 3]
            P.set_tile(tb, ta, 64, 3, 2)
        y = to_dev(phis[i], "f32")
        st = P.solve(y, gts[i])
        torch.cuda.synchronize()
        assert stats[i]["steps"] == st["steps"]
        if sp["ndim"] == 3:
            assert torch.equal(xs[i], y), (i, float((xs[i] - y).abs().max()))
        else:
            assert float((xs[i] - y).abs().max()) <= 1e-5 * float(y.abs().max()), i


def test_batched_autotune_picks_valid_tiles_and_leaves_fields():
    """lsp_batched_autotune returns a valid batch_tiles value for the
    dimensions present, leaves the caller's fields untouched, and later
    solves with it equal solves with the value set explicitly."""
    specs, phis, gs = _mixed_with_4d("weno5", 3)
    gts = [to_dev(g, "f32") for g in gs]
    xs = [to_dev(p, "f32") for p in phis]
    Bt = B.Batch(specs)
    tiles = Bt.autotune(xs, gts)
    assert tiles >> 6 == 0 and all(((tiles >> (2 * k)) & 3) != 3 for k in range(3))
    for i in range(len(specs)):
        assert torch.equal(xs[i], to_dev(phis[i], "f32"))
    Bt.solve(xs, gts)
    ys = [to_dev(p, "f32") for p in phis]
    B.Batch(specs, tiles=tiles).solve(ys, gts)
    torch.cuda.synchronize()
    for i in range(len(specs)):
        assert torch.equal(xs[i], ys[i]), i
    with pytest.raises(B.LspError) as e:
        B.Batch(specs, tiles=0b11)
    assert e.value.status == B.LSP_EINVAL
