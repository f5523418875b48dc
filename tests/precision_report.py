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
  python tests/precision_report.py --gpu-only DIR air3d_201 batched adjoint
  python tests/precision_report.py --oracle-only DIR air3d_201 batched adjoint
  python tests/precision_report.py --oracle-only DIR --conditioning air3d_121 car4d_51

With --conditioning the oracle side also computes, for the single-problem
configurations, its own per-node response R to FP32-sized noise injected into
every step (two realisations, tests/conditioning.py) and the ill-conditioned
set C (R above a third of the bar, grown by one node), and reports
  frac_C                the fraction of nodes in C
  frac_over_bar_off_C   nodes above the bar outside C (the kernel's share)
  err_off_C             max|dphi| / max|phi| outside C
  worst_in_C_over_3R    max over C of |dphi| / (3 R)

The two-phase form runs the GPU side on a GPU host and writes its results
(FP32 fields, gradients, step counts, tiles) to DIR/<config>.npz; the oracle
side then runs on any host with the same inputs (the seeded workloads) and
reports.
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
from conditioning import BAR, boundary_distance, conditioning_mask, noise_response  # noqa: E402
from gpu_helpers import rounded, sign_ok  # noqa: E402


def _gpu_solve(spec, phi0, g):
    import torch

    from paper_2411_03501_gb300 import binding as B
    P = B.Problem(spec, check_finite=True)
    x = torch.as_tensor(phi0, dtype=torch.float32, device="cuda")
    tile = P.autotune(x)
    gt = torch.as_tensor(g, dtype=torch.float32, device="cuda") if g is not None else None
    st = P.solve(x, gt, 0.0, spec["t_final"])
    return x.cpu().numpy(), st["steps"], tile


def _report(name, spec, got, want, steps_gpu, steps_orc, tile, secs):
    scale = float(np.abs(want).max())
    err = np.abs(got - want)
    bd = boundary_distance(spec)
    inner = bd >= 6
    return {"config": name, "nodes": int(np.prod(spec["n"])), "tile": [int(v) for v in tile],
            "steps_gpu": int(steps_gpu), "steps_oracle": int(steps_orc),
            "err": float(err.max()) / scale,
            "err_interior": float(err[inner].max()) / scale if inner.any() else None,
            "frac_over_bar": float((err > BAR * scale).mean()),
            "frac_over_bar_interior": float((err[inner] > BAR * scale).mean()) if inner.any() else None,
            "sign_ok": bool(sign_ok(got, want, spec)), "oracle_s": secs,
            "oracle_threads": oracle.threads()}


def _inputs(name):
    from paper_2411_03501_gb300 import workloads as W
    if name.startswith("air3d_"):
        spec, phi0, g = W.air3d(n=int(name[6:]))
    elif name.startswith("car4d_"):
        spec, phi0, g = W.car4d(n=int(name[6:]))
    else:
        raise SystemExit(f"unknown configuration {name}")
    return spec, rounded(phi0, "f32"), rounded(g, "f32")


BATCH_PICK = list(range(0, 256, 16))  # every 16th problem of the seeded workload


def gpu_phase(name, out):
    """Run the GPU side of one configuration; return its arrays."""
    import torch

    from paper_2411_03501_gb300 import binding as B
    if name == "batched":
        from paper_2411_03501_gb300 import workloads as W
        allp = W.batched(256)
        specs = [allp[i][0] for i in BATCH_PICK]
        phis = [rounded(allp[i][1], "f32") for i in BATCH_PICK]
        gs = [rounded(allp[i][2], "f32") for i in BATCH_PICK]
        Bt = B.Batch(specs, use_graph=True, check_finite=True)
        xs = [torch.as_tensor(p, dtype=torch.float32, device="cuda") for p in phis]
        stats = Bt.solve(xs, [torch.as_tensor(g, dtype=torch.float32, device="cuda") for g in gs])
        torch.cuda.synchronize()
        res = {f"phi{k}": x.cpu().numpy() for k, x in enumerate(xs)}
        res["steps"] = np.array([st["steps"] for st in stats])
        return res
    if name == "adjoint":
        return _adjoint_gpu()
    spec, phi0, g = _inputs(name)
    got, steps, tile = _gpu_solve(spec, phi0, g)
    return {"phi": got, "steps": np.array(steps), "tile": np.array(tile)}


def oracle_phase(name, d, conditioning=False):
    """Compare one configuration's GPU arrays `d` with the oracle."""
    if name == "batched":
        from paper_2411_03501_gb300 import workloads as W
        allp = W.batched(256)
        rows = []
        for k, i in enumerate(BATCH_PICK):
            sp = allp[i][0]
            phi0, g = rounded(allp[i][1], "f32"), rounded(allp[i][2], "f32")
            t0 = time.time()
            want, so = oracle.solve(sp, phi0, sp["t_final"], sp["rk"], sp["cfl"], target=g)
            rows.append(_report(f"batched[{i}] {sp['ndim']}-D {sp['n'][0]}^{sp['ndim']}", sp,
                                d[f"phi{k}"].astype(np.float64), want, d["steps"][k], so["steps"],
                                (16, 16), time.time() - t0))
        return rows
    if name == "adjoint":
        return [_adjoint_oracle(d)]
    spec, phi0, g = _inputs(name)
    t0 = time.time()
    want, so = oracle.solve(spec, phi0, spec["t_final"], spec["rk"], spec["cfl"], target=g)
    got = d["phi"].astype(np.float64)
    rep = _report(name, spec, got, want, int(d["steps"]), so["steps"], d["tile"],
                  time.time() - t0)
    if conditioning:
        t1 = time.time()
        R = noise_response(oracle, spec, phi0, g, spec["t_final"], want)
        scale = float(np.abs(want).max())
        C, Rd = conditioning_mask(R, scale, spec)
        err = np.abs(got - want)
        off = ~C
        rep.update({"frac_C": float(C.mean()),
                    "frac_over_bar_off_C": float(((err > BAR * scale) & off).mean()),
                    "err_off_C": float(err[off].max()) / scale if off.any() else None,
                    "worst_in_C_over_3R": (float((err[C] / (3.0 * Rd[C])).max())
                                           if C.any() else None),
                    "noise_response_max": float(R.max()) / scale,
                    "conditioning_s": time.time() - t1})
    return [rep]


ADJ_N, ADJ_STEPS = 129, 200


def _adjoint_inputs():
    from paper_2411_03501_gb300 import workloads as W
    spec = W.air3d(n=ADJ_N)[0]
    rng = np.random.default_rng(20241106)
    q = rounded(np.stack([rng.uniform(spec["lo"][k], spec["hi"][k], 1024) for k in range(3)], 1),
                "f32")
    phi0 = rounded(W.circle_sdf(spec, 0.0) - 5.0, "f32")
    return spec, q, phi0


def _adjoint_gpu():
    """The differentiation workload (air3d 129^3, 200 RK3 steps, loss =
    smoothed volume + 1024 query values, phi0 = target): the FP32 GPU
    adjoint's field and parameter gradients."""
    import torch

    from paper_2411_03501_gb300 import binding as B
    spec, q, phi0 = _adjoint_inputs()
    P = B.Problem(spec)
    x = torch.as_tensor(phi0, dtype=torch.float32, device="cuda")
    tile = P.autotune(x)
    ws = torch.empty(B.lsp_adjoint_workspace_size(P.grid, P.opts, ADJ_STEPS, 0),
                     dtype=torch.uint8, device="cuda")
    gt = x.clone()
    B.lsp_hj_solve_ckpt(P.grid, P.opts, x, gt, ADJ_STEPS, 0, ws)
    phiT = x.double().cpu().numpy()
    lamT = oracle.loss_grad(spec, phiT, q)
    lam0 = torch.empty_like(x)
    lamg = torch.empty_like(x)
    dprm = B.lsp_hj_adjoint(P.grid, P.opts, gt, ADJ_STEPS, 0,
                            torch.as_tensor(lamT, dtype=torch.float32, device="cuda"), lam0, lamg,
                            ws)
    torch.cuda.synchronize()
    return {"phiT": x.cpu().numpy(), "grad": (lam0 + lamg).cpu().numpy(),
            "dprm": np.array(dprm[:4]), "tile": np.array(tile)}


def _adjoint_oracle(d):
    spec, q, phi0 = _adjoint_inputs()
    # the oracle's adjoint of its own forward, seeded with the loss gradient
    # at its own phi_T
    t0 = time.time()
    phiT_o = oracle.solve_steps(spec, phi0, ADJ_STEPS, 3, spec["cfl"], target=phi0)
    lamT = rounded(oracle.loss_grad(spec, phiT_o, q), "f32")
    o0, og, oprm, _ = oracle.adjoint(spec, phi0, ADJ_STEPS, 3, spec["cfl"], lamT, target=phi0)
    secs = time.time() - t0
    g_orc = o0 + og
    s = float(np.abs(g_orc).max())
    g_gpu = d["grad"].astype(np.float64)
    return {"config": f"adjoint_air3d_{ADJ_N}^3_{ADJ_STEPS}xrk3", "tile": [int(v) for v in d["tile"]],
            "phiT_err": float(np.abs(d["phiT"] - phiT_o).max() / np.abs(phiT_o).max()),
            "grad_phi0_err": float(np.abs(g_gpu - g_orc).max()) / s,
            "grad_phi0_frac_over_1e-4": float((np.abs(g_gpu - g_orc) > 1e-4 * s).mean()),
            "dparams_gpu[v_e,v_p,w_e,w_p]": [float(v) for v in d["dprm"]],
            "dparams_oracle": [float(v) for v in oprm[:4]],
            "dparams_rel_err": [float(abs(a - b) / max(abs(b), 1e-30))
                                for a, b in zip(d["dprm"], oprm[:4])],
            "oracle_s": secs, "oracle_threads": oracle.threads()}


def main(argv):
    mode, outdir = "both", None
    if argv and argv[0] in ("--gpu-only", "--oracle-only"):
        mode, outdir, argv = argv[0][2:], argv[1], argv[2:]
        os.makedirs(outdir, exist_ok=True)
    conditioning = "--conditioning" in argv
    argv = [a for a in argv if a != "--conditioning"]
    names = argv or ["air3d_201", "car4d_81", "batched", "adjoint"]
    for name in names:
        path = os.path.join(outdir, f"{name}.npz") if outdir else None
        if mode in ("both", "gpu-only"):
            d = gpu_phase(name, outdir)
            if path:
                np.savez(path, **d)
                print(json.dumps({"config": name, "saved": path}), flush=True)
        if mode == "oracle-only":
            d = dict(np.load(path))
        if mode in ("both", "oracle-only"):
            for r in oracle_phase(name, d, conditioning):
                print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
