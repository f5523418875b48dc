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
    single-problem solve ends: bit for bit for the 3-D problems (same tiled
    stage body, same arithmetic per node), to FP32 rounding for the 2-D ones
    (the single-problem path runs the generic kernel there)."""
    specs, phis, gs = _mixed()
    Bt = B.Batch(specs, use_graph=use_graph, check_finite=True)
    xs = [to_dev(p, "f32") for p in phis]
    gts = [to_dev(g, "f32") for g in gs]
    stats = Bt.solve(xs, gts)
    torch.cuda.synchronize()
    for i, sp in enumerate(specs):
        P = B.Problem(sp)
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
    max|phi|, or 3x the oracle's own spread under FP32-sized noise where the
    discrete problem is worse conditioned -- e.g. the symmetric valley at
    theta = 0, y = 0 of an air3d tube, which FP32 rounding desymmetrises)."""
    specs, phis, gs = _mixed(scale=0.3, count=6, seed=7)
    Bt = B.Batch(specs)
    xs = [to_dev(p, "f32") for p in phis]
    Bt.solve(xs, [to_dev(g, "f32") for g in gs])
    torch.cuda.synchronize()
    for i, sp in enumerate(specs):
        want, _ = oracle.solve(sp, phis[i], sp["t_final"], sp["rk"], sp["cfl"], target=gs[i])
        got = xs[i].double().cpu().numpy()
        spread = noise_spread(sp, phis[i], gs[i], sp["t_final"], want)
        check_fp32_solve(got, want, spread)
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
