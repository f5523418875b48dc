#!/usr/bin/env python
"""Per-configuration precision of the FP32 GPU path against the FP64 oracle
at the benchmark sizes (a report, not a test: the oracle needs tens of
minutes of host time per configuration at these sizes).

For each configuration the GPU solve runs through the C ABI in the launch
configuration the benchmark uses (autotuned tile), the oracle solves the
same FP32-rounded inputs on every host core, and one JSON line reports
  err            max|phi_gpu - phi_oracle| / max|phi_oracle| at t_final
  err_interior   the same more than 6 nodes from every extrapolated edge
  frac_over_bar  fraction of nodes above 1e-4 max|phi| (the spec bar)
  sign_ok        sign disagreements only next to the oracle's zero level set
  steps          CFL steps of both (must be equal)
The adjoint configuration reports the FP32 gradients against the FP64
oracle adjoint instead.

  python tests/precision_report.py air3d_201 car4d_81 batched adjoint
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
from conditioning import BAR, boundary_distance  # noqa: E402
from gpu_helpers import rounded, sign_ok  # noqa: E402


def _solve_pair(spec, phi0, g):
    import torch

    from paper_2411_03501_gb300 import binding as B
    phi0 = rounded(phi0, "f32")
    g = rounded(g, "f32") if g is not None else None
    P = B.Problem(spec, check_finite=True)
    x = torch.as_tensor(phi0, dtype=torch.float32, device="cuda")
    tile = P.autotune(x)
    gt = torch.as_tensor(g, dtype=torch.float32, device="cuda") if g is not None else None
    st = P.solve(x, gt, 0.0, spec["t_final"])
    got = x.double().cpu().numpy()
    t0 = time.time()
    want, so = oracle.solve(spec, phi0, spec["t_final"], spec["rk"], spec["cfl"], target=g)
    return got, want, st, so, tile, time.time() - t0


def _report(name, spec, got, want, st, so, tile, secs):
    scale = float(np.abs(want).max())
    err = np.abs(got - want)
    bd = boundary_distance(spec)
    inner = bd >= 6
    return {"config": name, "nodes": int(np.prod(spec["n"])), "tile": list(tile),
            "steps_gpu": st["steps"], "steps_oracle": so["steps"],
            "err": float(err.max()) / scale,
            "err_interior": float(err[inner].max()) / scale if inner.any() else None,
            "frac_over_bar": float((err > BAR * scale).mean()),
            "sign_ok": bool(sign_ok(got, want, spec)), "oracle_s": secs,
            "oracle_threads": oracle.threads()}


def solve_config(name):
    from paper_2411_03501_gb300 import workloads as W
    if name.startswith("air3d_"):
        spec, phi0, g = W.air3d(n=int(name[6:]))
    elif name.startswith("car4d_"):
        spec, phi0, g = W.car4d(n=int(name[6:]))
    else:
        raise SystemExit(f"unknown configuration {name}")
    return [_report(name, spec, *_solve_pair(spec, phi0, g))]


def batched_config(every=16):
    """Every `every`-th problem of the 256-problem workload (seeded), each
    solved by the batched launch and by the oracle."""
    import torch

    from paper_2411_03501_gb300 import binding as B
    from paper_2411_03501_gb300 import workloads as W
    allp = W.batched(256)
    pick = list(range(0, 256, every))
    specs = [allp[i][0] for i in pick]
    phis = [rounded(allp[i][1], "f32") for i in pick]
    gs = [rounded(allp[i][2], "f32") for i in pick]
    Bt = B.Batch(specs, use_graph=True, check_finite=True)
    xs = [torch.as_tensor(p, dtype=torch.float32, device="cuda") for p in phis]
    stats = Bt.solve(xs, [torch.as_tensor(g, dtype=torch.float32, device="cuda") for g in gs])
    torch.cuda.synchronize()
    out = []
    for k, i in enumerate(pick):
        sp = specs[k]
        t0 = time.time()
        want, so = oracle.solve(sp, phis[k], sp["t_final"], sp["rk"], sp["cfl"], target=gs[k])
        out.append(_report(f"batched[{i}]", sp, xs[k].double().cpu().numpy(), want, stats[k], so,
                           (16, 16), time.time() - t0))
    return out


def adjoint_config():
    """The differentiation workload (air3d 129^3, 200 RK3 steps, loss =
    smoothed volume + 1024 query values): the FP32 GPU adjoint's field and
    parameter gradients against the FP64 oracle adjoint of the same map."""
    import torch

    from paper_2411_03501_gb300 import binding as B
    from paper_2411_03501_gb300 import workloads as W
    n, nsteps = 129, 200
    spec = W.air3d(n=n)[0]
    sdf = W.circle_sdf(spec, 0.0)
    rng = np.random.default_rng(20241106)
    q = rounded(np.stack([rng.uniform(spec["lo"][k], spec["hi"][k], 1024) for k in range(3)], 1),
                "f32")
    phi0 = rounded(sdf - 5.0, "f32")
    P = B.Problem(spec)
    x = torch.as_tensor(phi0, dtype=torch.float32, device="cuda")
    tile = P.autotune(x)
    ws = torch.empty(B.lsp_adjoint_workspace_size(P.grid, P.opts, nsteps, 0), dtype=torch.uint8,
                     device="cuda")
    gt = x.clone()
    B.lsp_hj_solve_ckpt(P.grid, P.opts, x, gt, nsteps, 0, ws)
    phiT = x.double().cpu().numpy()
    lamT = oracle.loss_grad(spec, phiT, q)
    lam0 = torch.empty_like(x)
    lamg = torch.empty_like(x)
    dprm = B.lsp_hj_adjoint(P.grid, P.opts, gt, nsteps, 0,
                            torch.as_tensor(lamT, dtype=torch.float32, device="cuda"), lam0, lamg,
                            ws)
    torch.cuda.synchronize()
    t0 = time.time()
    o0, og, oprm, oT = oracle.adjoint(spec, phi0, nsteps, 3, spec["cfl"], rounded(lamT, "f32"),
                                      target=phi0)
    secs = time.time() - t0
    g_gpu = (lam0 + lamg).double().cpu().numpy()  # phi0 = target: both paths
    g_orc = o0 + og
    s = float(np.abs(g_orc).max())
    return [{"config": "adjoint_air3d_129^3_200xrk3", "tile": list(tile),
             "phiT_err": float(np.abs(phiT - oT).max() / np.abs(oT).max()),
             "grad_phi0_err": float(np.abs(g_gpu - g_orc).max()) / s,
             "grad_phi0_frac_over_1e-4": float((np.abs(g_gpu - g_orc) > 1e-4 * s).mean()),
             "dparams_gpu": [float(v) for v in dprm[:4]],
             "dparams_oracle": [float(v) for v in oprm[:4]],
             "dparams_rel_err": [float(abs(a - b) / max(abs(b), 1e-30))
                                 for a, b in zip(dprm[:4], oprm[:4])],
             "oracle_s": secs, "oracle_threads": oracle.threads()}]


def main(argv):
    names = argv or ["air3d_201", "car4d_81", "batched", "adjoint"]
    for name in names:
        if name == "batched":
            rows = batched_config()
        elif name == "adjoint":
            rows = adjoint_config()
        else:
            rows = solve_config(name)
        for r in rows:
            print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
