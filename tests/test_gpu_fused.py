"""Temporal blocking of TVD-RK2 (tile pair 5: both stages of a step in one
launch, the first stage on the tile plus its halo in shared memory) against
two launches of the scalar tiled body on the same tile and against the FP64
oracle's step (Sec. V-A's RK2 with Sec. IV-D's rate and Sec. VI-A's tube).

The fused kernel performs the same operations on the same operands as the
scalar body, so the two agree bit for bit; the oracle comparison holds it to
the stage tolerance of the other kernels.  Grids are ragged (partial tiles
along both tile axes, partial chunks along the march) with periodic and
extrapolated axes in every role."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import U32, compare, rate_tol, rounded, step_flip_allowance, to_dev
from paper_2411_03501_gb300 import binding as B
from paper_2411_03501_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TILES = [(32, 8, 5, 3, 5), (16, 16, 1, 2, 5), (25, 10, 200, 3, 5), (32, 4, 3, 4, 5)]


def _spec(kind, scheme):
    if kind == "air3d":  # x, y extrapolated, theta periodic (the fastest axis)
        spec = W.air3d(nx=[37, 29, 45], scheme=scheme, rk=2)[0]
    elif kind == "rockets":  # every axis extrapolated
        spec = W.rockets(n=25, scheme=scheme)[0]
        spec["n"] = [27, 23, 41]
    elif kind == "periodic":
        spec = W.problem(3, [19, 22, 35], [-1, -1, -1], [1, 1, 1], [True, True, True], scheme,
                         "translate", [0.7, -1.1, 0.4], rk=2, cfl=0.75)
    else:  # march periodic, second axis extrapolated, fastest periodic
        spec = W.problem(3, [13, 30, 39], [-1, -1, 0], [1, 1.5, 2 * np.pi], [True, False, True],
                         scheme, "normal_speed", [1.3], rk=2, cfl=0.75)
    spec["tube"] = True
    return spec


@pytest.mark.parametrize("scheme", ["upwind1", "eno2", "eno3", "weno5"])
@pytest.mark.parametrize("kind", ["air3d", "rockets", "periodic", "mixed"])
def test_fused_rk2_step_equals_two_stages(kind, scheme):
    spec = _spec(kind, scheme)
    phi = rounded(W.smooth_field(spec, seed=8) + 0.2 * W.rough_field(spec, seed=9), "f32")
    g = rounded(phi + 0.05 * W.smooth_field(spec, seed=3), "f32")
    a = oracle.alpha(spec, phi)
    dt = oracle.cfl_dt(spec, a, 0.75, 0.0, 10.0)
    want = oracle.step(spec, phi, dt, 2, target=g)
    L, alpha = oracle.rate(spec, phi)
    tol = 2 * dt * rate_tol(spec, phi, L, alpha) + 8 * U32 * np.abs(phi).max()
    allow = step_flip_allowance(spec, phi, dt, 2, alpha, tol)
    gt = to_dev(g, "f32")
    ran = 0
    for tile in TILES:
        F = B.Problem(spec, check_finite=True)
        F.set_tile(*tile)
        if F.tile()[4] != 5:  # this scheme's halo does not fit the tile
            continue
        ran += 1
        S = B.Problem(spec, check_finite=True)
        S.set_tile(*tile[:4], 0)
        xf = to_dev(phi, "f32")
        xs = to_dev(phi, "f32")
        F.step(xf, gt, t=0.0, dt=dt)
        S.step(xs, gt, t=0.0, dt=dt)
        got = xf.cpu().numpy()
        np.testing.assert_array_equal(got, xs.cpu().numpy(), err_msg=f"tile {tile}")
        compare(got.astype(np.float64), want, tol, allow)
        assert np.all(got <= g)
    assert ran >= 3


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("nsteps", [5, 6])
def test_fused_rk2_solve_equals_unfused(graph, nsteps):
    """Whole solves of the rockets game (ENO2, RK2, tube): the fused solve
    alternates phi and the stage field; with an odd and an even step count
    the result lands in phi, equal bit for bit to the two-launch solve."""
    spec = W.rockets(n=29)[0]
    spec["n"] = [29, 27, 31]
    phi0 = rounded(W.circle_sdf(spec, 1.5) + 0.1 * W.smooth_field(spec, seed=2), "f32")
    gt = to_dev(W.circle_sdf(spec, 1.5), "f32")
    F = B.Problem(spec, check_finite=True, use_graph=graph)
    F.set_tile(16, 16, 4, 2, 5)
    S = B.Problem(spec, check_finite=True, use_graph=graph)
    S.set_tile(16, 16, 4, 2, 0)
    dt = B.lsp_cfl_dt(F.grid, F.opts, 0.0, 1e30)
    t_final = (nsteps - 0.5) * dt  # nsteps - 1 full steps and a half one
    xf = to_dev(phi0, "f32")
    xs = to_dev(phi0, "f32")
    st_f = F.solve(xf, gt, 0.0, t_final)
    st_s = S.solve(xs, gt, 0.0, t_final)
    assert st_f["steps"] == st_s["steps"] == nsteps
    np.testing.assert_array_equal(xf.cpu().numpy(), xs.cpu().numpy())
    if graph:  # the replay of the captured solve, from the same input
        xf.copy_(to_dev(phi0, "f32"))
        F.solve(xf, gt, 0.0, t_final)
        np.testing.assert_array_equal(xf.cpu().numpy(), xs.cpu().numpy())


def test_fused_tile_other_stages_run_the_scalar_body():
    """On a fused-RK2 tile, RK3 steps and single rates run the scalar body of
    the same tile (bitwise equal to pair 0); pair 5 is refused on 4-D grids,
    and a scheme whose halo does not fit the tile runs the generic kernel."""
    spec = _spec("air3d", "eno3")
    spec["rk"] = 3
    phi = rounded(W.smooth_field(spec, seed=8) + 0.2 * W.rough_field(spec, seed=9), "f32")
    F = B.Problem(spec, check_finite=True)
    F.set_tile(32, 8, 5, 3, 5)
    S = B.Problem(spec, check_finite=True)
    S.set_tile(32, 8, 5, 3, 0)
    xf, xs = to_dev(phi, "f32"), to_dev(phi, "f32")
    dt = B.lsp_cfl_dt(F.grid, F.opts, 0.0, 10.0)
    F.step(xf, to_dev(phi, "f32"), t=0.0, dt=dt)
    S.step(xs, to_dev(phi, "f32"), t=0.0, dt=dt)
    np.testing.assert_array_equal(xf.cpu().numpy(), xs.cpu().numpy())
    of, os_ = torch.empty_like(xf), torch.empty_like(xs)
    F.rate(xf, of)
    S.rate(xf, os_)
    np.testing.assert_array_equal(of.cpu().numpy(), os_.cpu().numpy())
    # 64 x 4: the ENO2 halo fits, the ENO3 one does not
    E = B.Problem(_spec("air3d", "eno2"))
    E.set_tile(64, 4, 5, 3, 5)
    assert E.tile()[4] == 5
    T = B.Problem(_spec("air3d", "eno3"))
    T.set_tile(64, 4, 5, 3, 5)
    assert T.tile() == (-1, -1, -1, -1, -1)
    spec4 = W.car4d(n=9)[0]
    Q = B.Problem(spec4)
    with pytest.raises(B.LspError):
        Q.set_tile(16, 8, 5, 3, 5)
