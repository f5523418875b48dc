#!/usr/bin/env python
"""Benchmark: grid-point updates per second per RK stage of the explicit HJ
level-set solve on one GB300, with its roofline position and the FP64 oracle
timed on the host cores beside it.

One benchmark step = one complete reachable-tube solve of the workload
(phi0 -> t_final: every RK stage of every step, CFL steps, tube), so the
metric is  points * stages / time.  Default workload: the 4-D car at 81^4
(ENO3, RK3, CFL 0.75, t_final 1.0, FP32; 124 steps, 372 stages; 43 M nodes,
fields of 172 MB), the largest configuration that fits one GPU; the air3d
game at 201^3 (WENO5, RK3, t_final 2.8; 5241 stages), the batched workload
(256 problems in one persistent launch) and the differentiation workload
(air3d 129^3, 200 RK3 steps, gradient by the discrete adjoint) are measured
first and reported inside the same line under "also".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   # the FP64 oracle on the host cores

Under torchrun (N > 1) every rank solves its own copy of the workload
(independent replicas: a single solve has no data-parallel split), the
time is the maximum over ranks, and the value counts every rank's updates.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid-point updates/s per RK stage"
UNIT = "updates/s"
L2_FLUSH_BYTES = 512 << 20  # > 129 MB of L2


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def workload(name: str):
    from paper_2411_03501_gb300 import workloads as W
    # air3d_<n>, car4d_<n>: the game workloads at n nodes per axis (the
    # benchmark lines use 201 and 81; smaller n serve profiler captures)
    if name.startswith("air3d_") and name[6:].isdigit():
        spec, phi0, g = W.air3d(n=int(name[6:]))
    elif name.startswith("car4d_") and name[6:].isdigit():
        spec, phi0, g = W.car4d(n=int(name[6:]))
    elif name.startswith("rockets_") and name[8:].isdigit():
        spec, phi0, g = W.rockets(n=int(name[8:]))
    elif name.startswith("double_integrator_") and name[18:].isdigit():
        spec, phi0, g = W.double_integrator(n=int(name[18:]))
    elif name == "normal_speed_2d":
        spec, phi0, g = W.normal_speed_2d(101)
    else:
        raise SystemExit(f"unknown workload {name}")
    return spec, phi0, g


def workload_for(args):
    """The workload of the command line with its dissipation / variational
    options applied (the name records them)."""
    spec, phi0, g = workload(args.workload)
    if args.diss != "glf":
        spec["diss"] = args.diss
        spec["name"] += "_" + args.diss
    if args.varform:
        spec["varform"] = True
        spec["tube"] = False  # the variational form stands in for the min with the target
        spec["name"] += "_varform"
    return spec, phi0, g


# Algorithmic work per node per stage (derivation in the design notes).
#  bytes: stage 1 reads phi and writes W1 (2 words); stage 2 reads W1 and
#  phi and writes W2 (3); stage 3 reads W2, phi and the target and writes
#  phi (4): RK3 with a tube averages 3 words per node per stage (RK2 without
#  a tube: 2.5).  Stencil neighbours and ghost cells are not counted.
#  flops: FP32 operations of the per-node formulas as the method states them
#  (FMA = 2, a division = 1, compare/max = 1), with no sharing between
#  nodes: one-sided derivatives along one axis, both sides (WENO5 156,
#  ENO3 32, ENO2 15, first order 4); the LF terms of one axis (average
#  costate 2, dissipation 3); the Hamiltonian (coordinate-only factors such
#  as sin/cos(theta) excluded); the stage combination with the tube (7).
DERIV_FLOPS = {"weno5": 156, "eno3": 32, "eno2": 15, "upwind1": 4}
LF_FLOPS_PER_AXIS = 5
COMBINE_FLOPS = 7


def ham_flops(dyn: str, d: int) -> int:
    return {"air3d": 15, "car4d": 10, "normal_speed": 2 * d + 1, "translate": 2 * d - 1,
            "quadratic": 2 * d, "rockets": 14, "double_integrator": 4}[dyn]


def algorithmic(spec) -> tuple[float, float]:
    """(bytes, flops) per node per stage, averaged over the stages of a step."""
    word = 8 if spec["dtype"] == "f64" else 4
    rk = spec["rk"]
    # fields read + written by the stages of one step (the last stage also
    # reads the previous level, the tube's stage the target):
    # RK1 phi -> W1; RK2 +(W1, phi -> phi); RK3 +(W1, phi -> W2), (W2, phi -> phi)
    words = {1: 2.0, 2: 5.0 / 2, 3: 8.0 / 3}[rk]
    if spec.get("tube"):
        words += 1.0 / rk
    d = spec["ndim"]
    flops = d * (DERIV_FLOPS[spec["scheme"]] + LF_FLOPS_PER_AXIS) + ham_flops(spec["dyn"], d) \
        + COMBINE_FLOPS
    return words * word, float(flops)


def launch_accounting(spec, tile, stats) -> tuple[int, float, float, bool]:
    """(stage-kernel launches per solve, algorithmic FLOPs per launch,
    algorithmic bytes per launch, fused) of a solve with `stats` on `tile`.
    A fused-RK2 tile (pair 5) runs both stages of a step in one launch, which
    reads phi (and the target) and writes phi': twice the stage FLOPs and
    2 or 3 words per node; otherwise one launch per stage."""
    import numpy as np
    npts = float(np.prod(spec["n"]))
    bpn, fpn = algorithmic(spec)
    fused = bool(tile[0] > 0 and tile[4] == 5 and spec["rk"] == 2)
    if fused:
        word = 8 if spec["dtype"] == "f64" else 4
        return int(stats["steps"]), 2 * fpn * npts, word * (2 + bool(spec.get("tube"))) * npts, True
    return int(stats["stages"]), fpn * npts, bpn * npts, False


KERNEL_SOURCES = ["stencil.cuh", "stage_tiled.cuh", "stage_tiled.inl", "stage_generic.cuh",
                  "pair2.cuh", "stage_pair.cuh", "stage_run.cuh", "stage_run.inl"]


def kernel_hash() -> str:
    """Hash of the stage-kernel sources: a DRAM-traffic figure taken by ncu is
    reported only while the kernel it was measured on is unchanged."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2411_03501_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload_name: str, pair: int):
    """dram__bytes_read.sum + dram__bytes_write.sum per stage launch from the
    committed ncu summary of this workload and stage-kernel variant (tile
    pair) (profiles/*.md lines `traffic_bytes_per_launch[<workload>]: <bytes>
    kernel_hash=<hash> pair=<pair>`), or None when no summary matches the
    current kernel sources and the variant that ran."""
    import glob
    want = kernel_hash()
    for f in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for ln in open(f):
            tag = f"traffic_bytes_per_launch[{workload_name}]:"
            if ln.strip().startswith(tag):
                parts = ln.strip()[len(tag):].split()
                if (len(parts) >= 3 and parts[1] == f"kernel_hash={want}"
                        and parts[2] == f"pair={pair}"):
                    return float(parts[0])
    return None


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    def __init__(self, index: int, path: str):
        self.index, self.path, self.proc = index, path, None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}",
                                          f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        rows = []
        for ln in open(self.path):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx,
                "reasons": reasons, "samples": len(rows)}


def sm_count() -> int:
    """Streaming multiprocessors of the current device (152 on a GB300); 152
    when no device is visible (the CPU tests of the accounting)."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.get_device_properties(torch.cuda.current_device())
                       .multi_processor_count)
    except Exception:
        pass
    return 152


def roofline_of(flops: float, nbytes: float, seconds: float, traffic):
    """Roofline object of a kernel that does `flops` algorithmic FLOPs and
    moves `nbytes` algorithmic bytes per launch in `seconds`: the FP32 ALU
    roof (SM count x 128 lanes x 2 x max SM clock) and the measured HBM copy
    roof; the binding one (larger fraction) first, the other inside."""
    peaks, src = _peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    nsm = sm_count()
    alu_peak = nsm * 128 * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s
    hbm_peak = float(peaks["hbm_gbs"])
    flop_ach = flops / seconds / 1e12
    hbm_ach = nbytes / seconds / 1e9
    alu = {"bound": "alu", "achieved": flop_ach, "peak": alu_peak, "unit": "TFLOP/s",
           "frac": flop_ach / alu_peak, "traffic": traffic,
           "peak_note": f"{nsm} SMs (queried) x 128 FP32 lanes x 2 (FMA) x max SM clock "
                        f"({sm_mhz:.0f} MHz, {src})"}
    hbm = {"bound": "hbm", "achieved": hbm_ach, "peak": hbm_peak, "unit": "GB/s",
           "frac": hbm_ach / hbm_peak, "traffic": traffic,
           "peak_note": f"{src} STREAM copy"}
    roof = dict(alu if alu["frac"] >= hbm["frac"] else hbm)
    roof["other"] = hbm if roof["bound"] == "alu" else alu
    return roof


def cpu_oracle_rate(spec, phi0, g, steps: int = 1):
    """The FP64 oracle as it stands, on the host cores: `steps` full RK steps
    of the workload from phi0.  Returns (updates/s, seconds, threads)."""
    import numpy as np
    import oracle
    p = np.asarray(phi0, dtype=np.float64)
    a = oracle.alpha(spec, p)
    dt = oracle.cfl_dt(spec, a, spec["cfl"], 0.0, spec["t_final"])
    t0 = time.perf_counter()
    for _ in range(steps):
        p = oracle.step(spec, p, dt, spec["rk"], target=g if spec["tube"] else None)
    el = time.perf_counter() - t0
    npts = int(np.prod(spec["n"]))
    return npts * spec["rk"] * steps / el, el, oracle.threads()


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return 0
    spec, phi0, g = workload_for(args)
    import numpy as np
    import oracle
    npts = int(np.prod(spec["n"]))
    # one benchmark step = one stage of the workload (a forward-Euler step
    # from phi0 with the workload's first CFL step): npts updates
    p0 = np.asarray(phi0, dtype=np.float64)
    a = oracle.alpha(spec, p0)
    dt = oracle.cfl_dt(spec, a, spec["cfl"], 0.0, spec["t_final"])
    tgt = g if spec["tube"] else None

    def one_stage():
        t0 = time.perf_counter()
        oracle.step(spec, p0, dt, 1, target=tgt)
        return time.perf_counter() - t0

    for _ in range(args.warmup):
        one_stage()
    t_all = sum(one_stage() for _ in range(args.steps))
    thr = oracle.threads()
    v = npts * args.steps / t_all
    sample = (f"1 stage (forward-Euler step, {npts} node updates) of {spec['name']} from phi0 "
              f"per benchmark step, FP64, OpenMP over {thr} threads, {cpu_model()}")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": spec["name"], "points": npts,
                   "parallelism": "single" if world == 1 else f"rank 0 alone of {world}",
                   "l2": "n/a (host)"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": thr, "kind": "oracle",
                         "sample": sample, "cpu_model": cpu_model()},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def measure_solve(args, name: str, rank: int, world: int, local_rank: int, clk_tag: str):
    """One workload's measurement: K timed solves (device-resident inputs,
    L2 flushed between solves), the pipelined end-to-end leg from pinned
    host buffers and the roofline of the stage kernel.  Returns the fields of
    its JSON line (rank 0) or None."""
    import numpy as np
    import torch

    from paper_2411_03501_gb300 import binding as B

    saved = args.workload
    args.workload = name
    spec, phi0, g = workload_for(args)
    args.workload = saved
    npts = int(np.prod(spec["n"]))
    P = B.Problem(spec, use_graph=args.graph)
    tdt = P.torch_dtype
    phi0_d = torch.as_tensor(phi0).to("cuda", tdt).contiguous()
    if args.tile:
        P.set_tile(*[int(v) for v in args.tile.split(",")])
        tile = P.tile()
    else:
        tile = P.autotune(phi0_d) if args.autotune else P.tile()
    g_d = torch.as_tensor(g).to("cuda", tdt).contiguous() if g is not None else None
    phi = torch.empty_like(phi0_d)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def one_solve():
        return P.solve(phi, g_d, 0.0, spec["t_final"])

    # warm-up (also captures the graph when enabled)
    for _ in range(args.warmup):
        phi.copy_(phi0_d)
        stats = one_solve()
    torch.cuda.synchronize()
    stages = stats["stages"]

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timed region: events around each solve, L2
    # flushed (and phi reset) between solves, outside the events
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clk = ClockSampler(local_rank, os.path.join(args.outdir, f"clocks_rank{rank}_{clk_tag}.csv"))
    barrier()
    with clk:
        for i in range(args.steps):
            phi.copy_(phi0_d)
            flush.zero_()
            ev[i][0].record(stream)
            one_solve()
            ev[i][1].record(stream)
        barrier()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    tmax = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if world > 1:
        torch.distributed.all_reduce(tmax, op=torch.distributed.ReduceOp.MAX)
    ms = float(tmax.item())
    units = world * npts * stages * args.steps
    value = units / (ms / 1e3)

    # ---- end to end through the public API: every step copies its inputs
    # (phi0 and the target) from pinned host memory, solves, and copies the
    # result back.  Two buffer sets and a copy stream: the copies of step
    # i+1's inputs and of step i-1's result run while step i solves (a
    # pipelined job of K solves); the timed region runs from the first
    # upload to the last download.
    h_phi0 = torch.as_tensor(phi0).to(tdt).pin_memory()
    h_g = torch.as_tensor(g).to(tdt).pin_memory() if g is not None else None
    h_out = [torch.empty_like(h_phi0).pin_memory() for _ in range(2)]
    d_phi = [torch.empty_like(phi0_d) for _ in range(2)]
    d_g = [torch.empty_like(g_d) for _ in range(2)] if g_d is not None else [None, None]
    bi = h_phi0.numel() * h_phi0.element_size() + (h_g.numel() * h_g.element_size() if h_g is not None else 0)
    bo = h_out[0].numel() * h_out[0].element_size()
    copy = torch.cuda.Stream()
    P_e2e = [P, P]
    if args.graph:  # a captured graph belongs to its buffers: one per buffer set
        P_e2e = [B.Problem(spec, use_graph=True) for _ in range(2)]
        for Q in P_e2e:
            if tile[0] > 0:
                Q.set_tile(*tile)

    def e2e_run(K):
        up = [torch.cuda.Event() for _ in range(2)]
        done = [torch.cuda.Event() for _ in range(2)]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(copy)

        def upload(i):
            with torch.cuda.stream(copy):
                d_phi[i % 2].copy_(h_phi0, non_blocking=True)
                if h_g is not None:
                    d_g[i % 2].copy_(h_g, non_blocking=True)
                up[i % 2].record(copy)

        upload(0)
        for i in range(K):
            stream.wait_event(up[i % 2])
            P_e2e[i % 2].solve(d_phi[i % 2], d_g[i % 2], 0.0, spec["t_final"], stream=stream)
            done[i % 2].record(stream)
            if i + 1 < K:
                upload(i + 1)  # after step i-1's download on the copy stream
            copy.wait_event(done[i % 2])
            with torch.cuda.stream(copy):
                h_out[i % 2].copy_(d_phi[i % 2], non_blocking=True)
        e1.record(copy)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    e2e_run(max(2, args.warmup))
    barrier()
    ms2 = e2e_run(args.steps)
    t2 = torch.tensor([ms2], dtype=torch.float64, device="cuda")
    if world > 1:
        torch.distributed.all_reduce(t2, op=torch.distributed.ReduceOp.MAX)
    e2e_value = units / (float(t2.item()) / 1e3)
    # the same copies alone, to account for the e2e leg (not overlapped)
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    d_phi[0].copy_(h_phi0, non_blocking=True)
    if h_g is not None:
        d_g[0].copy_(h_g, non_blocking=True)
    h_out[0].copy_(d_phi[0], non_blocking=True)
    c1.record(stream)
    torch.cuda.synchronize()
    copy_ms = c0.elapsed_time(c1)
    if rank != 0:
        return None

    # ---- roofline of the dominant kernel (the fused stage kernel): its
    # average launch time over the timed region = solve time / stage launches
    launches, fpl, bpl, fused = launch_accounting(spec, tile, stats)
    per_launch_s = (ms / 1e3) / (launches * args.steps)
    roof = roofline_of(fpl, bpl, per_launch_s,
                       None if fused else measured_traffic(spec["name"], int(tile[4])))
    return {
        "spec": spec, "phi0": phi0, "g": g, "value": value, "ms_per_step": ms / args.steps,
        "config": {"workload": spec["name"], "points": npts, "stages_per_step": stages,
                   "rk_steps_per_step": stats["steps"],
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "flushed (512 MB write) between timed solves",
                   "graph": bool(args.graph), "tile": list(tile),
                   "fused_rk2_steps": fused},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": bi,
                "d2h_bytes_per_step": bo,
                "pipelined": "step i+1's uploads and step i-1's download overlap step i's solve "
                             "(second stream, two buffer sets)",
                "copy_ms_per_step_alone": copy_ms},
        "gpu_launches": launches * args.steps,
        "roofline": roof,
        "clocks": clk.summary(),
    }


def cpu_model() -> str:
    try:
        for ln in subprocess.run(["lscpu"], capture_output=True, text=True).stdout.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline_of(spec, phi0, g):
    """The FP64 oracle as it stands on this host: one RK step of the
    workload on every core (OpenMP), and one stage (a forward-Euler step) on
    one core over a slab of the grid (the first slices of the slowest axis,
    same spacing, at least 7) so that it stays within seconds."""
    import numpy as np
    import oracle
    v, el, thr = cpu_oracle_rate(spec, phi0, g, 1)
    n0 = spec["n"][0]
    k = max(7, n0 // 16) if spec["ndim"] >= 3 else n0
    sub = dict(spec)
    sub["n"] = [k] + list(spec["n"][1:])
    h0 = (spec["hi"][0] - spec["lo"][0]) / ((n0) if spec["periodic"][0] else (n0 - 1))
    sub["hi"] = [spec["lo"][0] + h0 * (k if spec["periodic"][0] else k - 1)] + list(spec["hi"][1:])
    p = np.ascontiguousarray(np.asarray(phi0, dtype=np.float64)[:k])
    gs = np.ascontiguousarray(np.asarray(g, dtype=np.float64)[:k]) if g is not None else None
    a = oracle.alpha(spec, phi0)
    dt = oracle.cfl_dt(spec, a, spec["cfl"], 0.0, spec["t_final"])
    oracle.set_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.step(sub, p, dt, 1, target=gs if spec["tube"] else None)
        el1 = time.perf_counter() - t0
    finally:
        oracle.set_threads(thr)
    v1 = int(np.prod(sub["n"])) / el1
    return {"value": v, "unit": UNIT, "cores": thr, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": f"1 RK{spec['rk']} step ({spec['rk']} stages, {el:.1f} s) of "
                      f"{spec['name']} from phi0, FP64, OpenMP over {thr} threads",
            "one_thread_value": v1,
            "one_thread_sample": f"1 stage (forward-Euler step, {el1:.1f} s) on the first {k} "
                                 f"slices of axis 0 ({int(np.prod(sub['n']))} nodes), 1 thread"}


def run_ours(args, rank: int, world: int, local_rank: int):
    from paper_2411_03501_gb300 import build as BLD
    import torch

    torch.cuda.set_device(local_rank)
    if rank == 0 or not os.path.exists(BLD.LIB):
        BLD.build()
    if world > 1:
        torch.distributed.barrier()
    also = [] if args.also in ("", "none") else args.also.split(",")
    others = {}
    for name in also:  # secondary workloads first; the headline line is measured last
        r = measure_solve(args, name, rank, world, local_rank, name)
        if r is not None:
            others[r["config"]["workload"]] = {
                "value": r["value"], "unit": UNIT, "ms_per_step": r["ms_per_step"],
                "e2e": r["e2e"]["value"], "roofline": r["roofline"], "tile": r["config"]["tile"],
                "stages_per_step": r["config"]["stages_per_step"], "clocks": r["clocks"]}
    extras = [] if args.extras in ("", "none") else args.extras.split(",")
    for name in extras:  # the batched and differentiation workloads, same process
        fn = {"batched": run_batched, "adjoint": run_adjoint}[name]
        ln = fn(args, rank, world, local_rank, emit=False)
        if isinstance(ln, dict):
            others[ln["config"]["workload"]] = {
                k: ln[k] for k in ("value", "unit", "ms_per_step", "e2e", "roofline", "config",
                                   "gpu_launches", "clocks", "scaling")}
    r = measure_solve(args, args.workload, rank, world, local_rank, "main")
    if rank != 0:
        return 0
    spec = r["spec"]
    cpu = cpu_baseline_of(spec, r["phi0"], r["g"]) if args.cpu_baseline else None
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": spec["dtype"], "data": "synthetic",
        "config": r["config"], "e2e": r["e2e"], "gpu_launches": r["gpu_launches"],
        "roofline": r["roofline"], "cpu_baseline": cpu, "clocks": r["clocks"],
    }
    if others:
        line["also"] = others
    print(json.dumps(line), flush=True)
    return 0


def run_batched(args, rank: int, world: int, local_rank: int, emit: bool = True):
    """The batched workload: 256 problems (half 2-D normal speed, half 3-D
    air3d, seeded sizes/speeds/radii) in one batched solve per benchmark
    step; ranks split the problems by estimated cost (sharding.shard, no
    exchange).  The
    single-problem path (one lsp_hj_solve per problem, in turn) is timed
    beside it on the same problems."""
    import numpy as np
    import torch

    from paper_2411_03501_gb300 import binding as B
    from paper_2411_03501_gb300 import build as BLD
    from paper_2411_03501_gb300 import workloads as W

    torch.cuda.set_device(local_rank)
    if rank == 0 or not os.path.exists(BLD.LIB):
        BLD.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2411_03501_gb300.sharding import estimated_cost, shard
    allp = W.batched(256)
    parts = shard([estimated_cost(p[0]) for p in allp], world)
    mine = [allp[i] for i in parts[rank]]
    specs = [m[0] for m in mine]
    persistent = bool(args.persistent)
    Bt = B.Batch(specs, use_graph=True, persistent=persistent, chunk=args.batch_chunk)
    Balt = B.Batch(specs, use_graph=True, persistent=not persistent, chunk=args.batch_chunk)
    h_phi0 = [torch.as_tensor(m[1], dtype=torch.float32).pin_memory() for m in mine]
    h_g = [torch.as_tensor(m[2], dtype=torch.float32).pin_memory() for m in mine]
    d_phi0 = [t.cuda() for t in h_phi0]
    d_g = [t.cuda() for t in h_g]
    phis = [torch.empty_like(t) for t in d_phi0]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def reset():
        for a, b in zip(phis, d_phi0):
            a.copy_(b)

    # tile shape per problem dimension, timed on this batch (both launch forms
    # use the choice made for the timed one)
    tiles = Bt.autotune(d_phi0, d_g) if args.autotune else 0
    Bt.opts.batch_tiles = tiles
    Balt.opts.batch_tiles = tiles
    for _ in range(args.warmup):
        reset()
        stats = Bt.solve(phis, d_g)
    torch.cuda.synchronize()
    units_rank = sum(int(np.prod(sp["n"])) * st["stages"] for sp, st in zip(specs, stats))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clk = ClockSampler(local_rank, os.path.join(args.outdir, f"clocks_rank{rank}.csv"))
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with clk:
        for i in range(args.steps):
            reset()
            flush.zero_()
            ev[i][0].record(stream)
            Bt.solve(phis, d_g)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    t = torch.tensor([ms, float(units_rank)], dtype=torch.float64, device="cuda")
    tu = t.clone()
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.all_reduce(tu, op=torch.distributed.ReduceOp.SUM)
    ms = float(t[0].item())
    units = float(tu[1].item()) * args.steps
    value = units / (ms / 1e3)

    # end to end: pinned host fields in, batched solve, fields out
    h_out = [torch.empty_like(x).pin_memory() for x in h_phi0]
    d_g2 = [torch.empty_like(x) for x in d_g]

    def e2e():
        for a, b in zip(phis, h_phi0):
            a.copy_(b, non_blocking=True)
        for a, b in zip(d_g2, h_g):
            a.copy_(b, non_blocking=True)
        Bt.solve(phis, d_g2)
        for a, b in zip(h_out, phis):
            a.copy_(b, non_blocking=True)

    e2e()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e()
    e1.record(stream)
    torch.cuda.synchronize()
    t2 = torch.tensor([e0.elapsed_time(e1)], dtype=torch.float64, device="cuda")
    if world > 1:
        torch.distributed.all_reduce(t2, op=torch.distributed.ReduceOp.MAX)
    e2e_value = units / (float(t2.item()) / 1e3)
    bi = sum(x.numel() * 4 for x in h_phi0) + sum(x.numel() * 4 for x in h_g)
    bo = sum(x.numel() * 4 for x in h_out)

    # the other batched variant (persistent vs stage-synchronous), same timing
    for _ in range(2):
        reset()
        Balt.solve(phis, d_g)
    torch.cuda.synchronize()
    alt_ms = 0.0
    for i in range(args.steps):
        reset()
        flush.zero_()
        ev[i][0].record(stream)
        Balt.solve(phis, d_g)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    alt_ms = sum(a.elapsed_time(b) for a, b in ev)
    alt_value = float(units_rank) * args.steps / (alt_ms / 1e3)

    # the single-problem path on the same problems, one solve after another
    singles = [B.Problem(sp) for sp in specs]
    reset()
    for P, a, g in zip(singles, phis, d_g):  # warm-up
        P.solve(a, g)
    reset()
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for P, a, g in zip(singles, phis, d_g):
        P.solve(a, g)
    s1.record(stream)
    torch.cuda.synchronize()
    single_value = float(units_rank) / (s0.elapsed_time(s1) / 1e3)
    if rank != 0:
        return 0
    # one launch per stage, or one cooperative launch per solve
    launches = 1 if persistent else max(st["steps"] for st in stats) * specs[0]["rk"]
    # roofline of the batched stage kernel (the only kernel of the solve):
    # this rank's algorithmic work per solve over the solve time, averaged
    # over its launches the same way
    tot_f = tot_b = 0.0
    for sp, st in zip(specs, stats):
        bpn, fpn = algorithmic(sp)
        nst = float(np.prod(sp["n"])) * st["stages"]
        tot_f += fpn * nst
        tot_b += bpn * nst
    roof = roofline_of(tot_f / launches, tot_b / launches, (ms / 1e3) / args.steps / launches,
                       None)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "batched_256_weno5_rk3_f32", "problems": len(allp),
                   "points": sum(int(np.prod(p[0]["n"])) for p in allp),
                   "parallelism": "problems split across ranks" if world > 1 else "single",
                   "l2": "flushed (512 MB write) between timed solves",
                   "launch": "persistent" if persistent else "stage-synchronous (graph)",
                   "batch_chunk": args.batch_chunk or 128,
                   "batch_tiles": {f"{d}-D": ["16x16", "32x8", "64x4"][(tiles >> (2 * (d - 2))) & 3]
                                   for d in (2, 3, 4)},
                   ("stage_synchronous_value" if persistent else "persistent_value"): alt_value,
                   "single_problem_path_value": single_value},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": bi,
                "d2h_bytes_per_step": bo},
        "gpu_launches": launches * args.steps,
        "roofline": roof, "cpu_baseline": None, "clocks": clk.summary(),
    }
    if not emit:
        return line
    print(json.dumps(line), flush=True)
    return 0


def run_adjoint(args, rank: int, world: int, local_rank: int, emit: bool = True):
    """The differentiation workload: the air3d tube at 129^3 in FP32 over 200
    fixed RK3 steps; loss = smoothed volume of {phi <= 0} + phi at 1024 seeded
    query states.  One benchmark step = forward solve keeping every state and
    stage input (--ncheck -1, 5.2 GB; --ncheck 0: sqrt(N) checkpoints and a
    recomputation per segment), loss, reverse sweep: gradients with respect
    to v_e, v_p, the shared turn-rate bound, the target radius (and phi0 =
    target).  The metric counts the forward's point-stages per second of the
    whole gradient evaluation; the plain forward (same 200 steps) and the
    other checkpoint form are timed beside it.  Replicas under torchrun."""
    import numpy as np
    import torch

    from paper_2411_03501_gb300 import binding as B
    from paper_2411_03501_gb300 import build as BLD
    from paper_2411_03501_gb300 import workloads as W
    from paper_2411_03501_gb300.autograd import HJTube

    torch.cuda.set_device(local_rank)
    if rank == 0 or not os.path.exists(BLD.LIB):
        BLD.build()
    if world > 1:
        torch.distributed.barrier()
    n, nsteps = 129, 200
    spec = W.air3d(n=n)[0]
    npts = n ** 3
    h_sdf = torch.as_tensor(W.circle_sdf(spec, 0.0), dtype=torch.float32).pin_memory()
    rng = np.random.default_rng(20241106)
    h_q = torch.as_tensor(np.stack([rng.uniform(spec["lo"][k], spec["hi"][k], 1024)
                                    for k in range(3)], 1), dtype=torch.float32).pin_memory()
    sdf, q = h_sdf.cuda(), h_q.cuda()
    tube = HJTube(spec, nsteps=nsteps, ncheck=args.ncheck)
    other = HJTube(spec, nsteps=nsteps, ncheck=0 if args.ncheck < 0 else -1)
    stream = torch.cuda.current_stream()
    if args.tile:  # a fixed tile (the capture commands use the autotuner's choice)
        tile = tuple(int(v) for v in args.tile.split(","))
        B.lsp_set_tile(tube.grid, *tile)
    else:
        tile = tube.autotune(sdf - 5.0) if args.autotune else None
    if tile is not None:
        B.lsp_set_tile(other.grid, *tile)

    def grad_step(sdf_d, q_d, tube=tube):
        base = torch.tensor([5.0, 5.0, 1.0], dtype=torch.float64, requires_grad=True)
        r = torch.tensor(5.0, dtype=torch.float64, requires_grad=True)
        params = torch.stack([base[0], base[1], base[2], base[2]])
        target = sdf_d - r.to("cuda").float()
        loss = tube.loss(tube(target, target, params), q_d)
        loss.backward()
        return torch.cat([base.grad, r.grad.reshape(1)])

    for _ in range(args.warmup):
        g = grad_step(sdf, q)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clk = ClockSampler(local_rank, os.path.join(args.outdir, f"clocks_rank{rank}.csv"))
    if world > 1:
        torch.distributed.barrier()
    with clk:
        for i in range(args.steps):
            ev[i][0].record(stream)
            g = grad_step(sdf, q)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    # the other checkpoint form on the same tile
    for _ in range(2):
        grad_step(sdf, q, other)
    torch.cuda.synchronize()
    o0, o1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    o0.record(stream)
    for _ in range(args.steps):
        grad_step(sdf, q, other)
    o1.record(stream)
    torch.cuda.synchronize()
    other_ms = o0.elapsed_time(o1) / args.steps
    # plain forward of the same 200 steps (one checkpoint: a single copy)
    plain = HJTube(spec, nsteps=nsteps, ncheck=1)
    if tile is not None:
        B.lsp_set_tile(plain.grid, *tile)
    params = torch.tensor(spec["params"], dtype=torch.float64)
    tgt = sdf - 5.0
    with torch.no_grad():
        for _ in range(2):
            plain(tgt, tgt, params)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            plain(tgt, tgt, params)
        f1.record(stream)
        torch.cuda.synchronize()
    fwd_ms = f0.elapsed_time(f1)
    # end to end: the SDF and queries from pinned host memory, gradients back
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        g = grad_step(h_sdf.cuda(non_blocking=True), h_q.cuda(non_blocking=True)).cpu()
    e1.record(stream)
    torch.cuda.synchronize()
    t = torch.tensor([ms, e0.elapsed_time(e1), fwd_ms], dtype=torch.float64, device="cuda")
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    ms, e2e_ms, fwd_ms = (float(v) for v in t.tolist())
    units = world * npts * nsteps * 3 * args.steps
    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": units / (ms / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "adjoint_air3d_129^3_200xrk3_f32", "points": npts,
                   "rk_steps": nsteps,
                   "checkpoints": ("every state and stage input" if tube.ncheck < 0
                                   else tube.ncheck or int(np.ceil(np.sqrt(nsteps)))),
                   "other_checkpoints": ("every state and stage input" if other.ncheck < 0
                                         else int(np.ceil(np.sqrt(nsteps)))),
                   "other_checkpoints_ms_per_step": other_ms,
                   "workspace_bytes": int(B.lsp_adjoint_workspace_size(tube.grid, tube.opts,
                                                                       nsteps, tube.ncheck)),
                   "tile": list(tile) if tile is not None else None,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "fields (8.6 MB each) partly L2-resident; no flush",
                   "plain_forward_value": units / (fwd_ms / 1e3),
                   "gradient_over_forward_time": ms / fwd_ms,
                   "grads[v_e, v_p, w, r]": [float(v) for v in g.tolist()]},
        "e2e": {"value": units / (e2e_ms / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": h_sdf.numel() * 4 + h_q.numel() * 4,
                "d2h_bytes_per_step": 4 * 8},
        "gpu_launches": adjoint_launches(nsteps, 3, tube.ncheck) * args.steps, "roofline": None,
        "cpu_baseline": None, "clocks": clk.summary(),
    }
    if not emit:
        return line
    print(json.dumps(line), flush=True)
    return 0


def run_shapes(args, rank: int, world: int, local_rank: int):
    """Implicit surfaces on the device (Sec. III-C, III-D): one benchmark step
    builds a target on the air3d 201^3 grid -- a cylinder, a box and their
    union -- i.e. two primitive kernels (4 B written per node each) and one
    set operation (8 B read, 4 B written per node).  Metric: node values
    produced per second; HBM roofline of the step's algorithmic bytes."""
    import numpy as np
    import torch

    from paper_2411_03501_gb300 import binding as B
    from paper_2411_03501_gb300 import build as BLD
    from paper_2411_03501_gb300 import workloads as W

    torch.cuda.set_device(local_rank)
    if rank == 0 or not os.path.exists(BLD.LIB):
        BLD.build()
    spec = W.air3d(n=201)[0]
    npts = int(np.prod(spec["n"]))
    g = B.lsp_grid_create(3, spec["lo"], spec["hi"], spec["n"],
                          ["periodic" if p else "extrapolate" for p in spec["periodic"]])
    a = torch.empty(spec["n"], dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    out = torch.empty_like(a)
    stream = torch.cuda.current_stream()

    def step():
        B.lsp_shape_sphere(g, a, [0.0, 0.0, 0.0], 5.0, ignore=(2,))
        B.lsp_shape_box(g, b, [2.0, -3.0, 0.0], [12.0, 3.0, 6.0], ignore=(2,))
        B.lsp_shape_op("union", a, b, out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = ClockSampler(local_rank, os.path.join(args.outdir, f"clocks_rank{rank}.csv"))
    with clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    ms = float(t.item())
    value = 3.0 * npts * args.steps * world / (ms / 1e3)
    # the three kernels together: 4 + 4 + 12 algorithmic bytes per node
    roof = roofline_of(0.0, 20.0 * npts, (ms / 1e3) / args.steps, None)
    if rank != 0:
        return 0
    h_out = torch.empty(spec["n"], dtype=torch.float32).pin_memory()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for _ in range(args.steps):
        step()
        h_out.copy_(out, non_blocking=True)
    e3.record(stream)
    torch.cuda.synchronize()
    e2e_value = 3.0 * npts * args.steps / (e2.elapsed_time(e3) / 1e3)
    line = {
        "metric": "implicit-surface node values/s", "value": value, "unit": "values/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "shapes_cylinder_box_union_201^3", "points": npts,
                   "kernels_per_step": 3, "parallelism": "replicas" if world > 1 else "single",
                   "l2": "fields of 32.5 MB, three per step (partly L2-resident); no flush"},
        "e2e": {"value": e2e_value, "unit": "values/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": npts * 4},
        "gpu_launches": 3 * args.steps, "roofline": roof, "cpu_baseline": None,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def adjoint_launches(nsteps: int, rk: int, ncheck: int = 0) -> int:
    """Kernels of one gradient evaluation: forward stages, the segment
    recomputation from sqrt(N) checkpoints (which keeps every step's stage
    inputs; the last step of a segment computes its stage inputs alone) --
    none when every stage input is kept (ncheck < 0) --, one adjoint kernel
    per stage (each stage's first pass fused with the previous stage's
    gather) and one closing gather, the GLF argmax, two loss kernels."""
    import math
    recompute = 0
    if ncheck >= 0:
        C = min(ncheck or math.ceil(math.sqrt(nsteps)), nsteps)
        K = math.ceil(nsteps / C)
        nseg = math.ceil(nsteps / K)
        recompute = (nsteps - nseg) * rk + nseg * (rk - 1)
    return nsteps * rk + recompute + rk * nsteps + 1 + 1 + 2


def run_steps(args):
    """Profiling mode: `warmup` then `steps` single RK steps of the workload
    (3 stage launches each for RK3), timed with events; for ncu captures."""
    import numpy as np
    import torch

    from paper_2411_03501_gb300 import binding as B
    from paper_2411_03501_gb300 import build as BLD
    BLD.build()
    spec, phi0, g = workload_for(args)
    P = B.Problem(spec)
    phi = torch.as_tensor(phi0).to("cuda", P.torch_dtype).contiguous()
    gd = torch.as_tensor(g).to("cuda", P.torch_dtype).contiguous() if g is not None else None
    if args.tile:
        P.set_tile(*[int(v) for v in args.tile.split(",")])
        tile = P.tile()
    else:
        tile = P.autotune(phi) if args.autotune else P.tile()
    dt = B.lsp_cfl_dt(P.grid, P.opts, 0.0, spec["t_final"])
    for _ in range(args.warmup):
        P.step(phi, gd, 0.0, dt)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        P.step(phi, gd, 0.0, dt)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    print(json.dumps({"mode": "steps", "workload": spec["name"], "rk_steps": args.steps,
                      "tile": tile,
                      "ms_per_stage": ms / (args.steps * spec["rk"]),
                      "points": int(np.prod(spec["n"]))}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="car4d_81")
    ap.add_argument("--also", default="auto",
                    help="comma-separated solve workloads measured before the main one and "
                         "reported inside its line (auto: air3d_201 with the default workload)")
    ap.add_argument("--extras", default="auto",
                    help="comma-separated workloads among batched, adjoint measured before the "
                         "main one and reported under 'also' (auto: both with the default "
                         "workload)")
    ap.add_argument("--graph", type=int, default=0)
    ap.add_argument("--cpu-baseline", type=int, default=1)
    ap.add_argument("--outdir", default=os.path.join(ROOT, "bench_out"),
                    help="where the clock samples of the timed region are written")
    ap.add_argument("--mode", default="solve", choices=["solve", "steps"])
    ap.add_argument("--autotune", type=int, default=1)
    ap.add_argument("--tile", default="", help="tb,ta,ch,minb: fixed tile instead of autotuning")
    ap.add_argument("--print-kernel-hash", action="store_true")
    ap.add_argument("--diss", default="glf", choices=["glf", "llf", "lllf"],
                    help="dissipation coefficients of the solve workloads")
    ap.add_argument("--varform", type=int, default=0,
                    help="1: the variational form of the tube PDE instead of the min with the target")
    ap.add_argument("--batch-chunk", type=int, default=0,
                    help="batched workload: planes per CTA along the march (0 = the library's 128)")
    ap.add_argument("--ncheck", type=int, default=-1,
                    help="adjoint workload: checkpoints (0 = sqrt(N), -1 = keep every state and "
                         "stage input)")
    ap.add_argument("--persistent", type=int, default=1,
                    help="batched workload: time the persistent launch (1) or the "
                         "stage-synchronous graph (0); the other is timed beside it")
    args = ap.parse_args()
    if args.print_kernel_hash:
        print(kernel_hash())
        return 0
    if args.mode == "steps":
        return run_steps(args)
    if args.warmup < 3:
        args.warmup = 3
    os.makedirs(args.outdir, exist_ok=True)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.also == "auto":
        args.also = "air3d_201" if args.workload == "car4d_81" and args.mode == "solve" else ""
    if args.extras == "auto":
        args.extras = ("batched,adjoint" if args.workload == "car4d_81" and args.mode == "solve"
                       else "")
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        if args.workload == "batched":
            return run_batched(args, rank, world, local_rank)
        if args.workload == "adjoint":
            return run_adjoint(args, rank, world, local_rank)
        if args.workload == "shapes":
            return run_shapes(args, rank, world, local_rank)
        return run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
