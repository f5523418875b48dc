"""The benchmark's accounting, on the CPU: the algorithmic bytes and FLOPs
per node and stage that the roofline fractions divide by, the roofline
object, and the DRAM-traffic lines of the committed profile summaries."""
import glob
import os
import re

import pytest

import bench
from paper_2411_03501_gb300 import workloads as W


def _spec(rk, tube, dtype="f32", scheme="weno5", dyn="air3d"):
    if dyn == "air3d":
        spec = W.air3d(n=9)[0]
    else:
        spec = W.car4d(n=9)[0]
    spec.update(rk=rk, tube=tube, dtype=dtype, scheme=scheme)
    return spec


@pytest.mark.parametrize("rk,tube,words", [
    # fields read and written per node over the stages of one step, per stage:
    # RK1 phi -> W1 (+ g); RK2 phi -> W1, (W1, phi [, g]) -> phi;
    # RK3 phi -> W1, (W1, phi) -> W2, (W2, phi [, g]) -> phi
    (1, False, 2.0), (1, True, 3.0),
    (2, False, (2 + 3) / 2), (2, True, (2 + 4) / 2),
    (3, False, (2 + 3 + 3) / 3), (3, True, (2 + 3 + 4) / 3),
])
@pytest.mark.parametrize("dtype,word", [("f32", 4), ("f64", 8)])
def test_algorithmic_bytes_per_node_and_stage(rk, tube, words, dtype, word):
    nbytes, _ = bench.algorithmic(_spec(rk, tube, dtype))
    assert nbytes == pytest.approx(words * word, rel=1e-12)


def test_algorithmic_flops_of_the_benchmark_stages():
    # per axis both one-sided derivatives + 5 LF terms, the Hamiltonian, the
    # combination: air3d WENO5 in 3-D and car4d ENO3 in 4-D
    assert bench.algorithmic(_spec(3, True))[1] == 3 * (156 + 5) + 15 + 7 == 505
    assert bench.algorithmic(_spec(3, True, scheme="eno3", dyn="car4d"))[1] == \
        4 * (32 + 5) + 10 + 7 == 165


def test_roofline_object_picks_the_binding_roof():
    peaks, _ = bench._peaks()
    alu_peak = bench.sm_count() * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    # compute-heavy: 505 FLOP and 12 B per node, 8.12 M nodes in 126 us
    n = 8120601
    r = bench.roofline_of(505.0 * n, 12.0 * n, 126e-6, 68.7e6)
    assert r["bound"] == "alu" and r["other"]["bound"] == "hbm"
    assert r["achieved"] == pytest.approx(505.0 * n / 126e-6 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / alu_peak)
    assert r["other"]["frac"] == pytest.approx(12.0 * n / 126e-6 / 1e9 / float(peaks["hbm_gbs"]))
    assert r["traffic"] == 68.7e6
    # byte-heavy: 20 B and no FLOPs per value
    r = bench.roofline_of(0.0, 20.0 * n, 50e-6, None)
    assert r["bound"] == "hbm" and r["other"]["frac"] == 0.0


def test_profile_traffic_lines_parse():
    """Every traffic line of the committed summaries names a workload, a
    positive byte count, a 16-hex-digit kernel hash and the stage-kernel
    variant (the benchmark reports the figure only while the kernel sources
    hash to it and that variant ran)."""
    pat = re.compile(r"^traffic_bytes_per_launch\[([^\]]+)\]: (\d+) kernel_hash=([0-9a-f]{16}) "
                     r"pair=\d$")
    found = 0
    for f in glob.glob(os.path.join(bench.ROOT, "profiles", "*.md")):
        for ln in open(f):
            if ln.startswith("traffic_bytes_per_launch"):
                m = pat.match(ln.strip())
                assert m, (f, ln)
                assert int(m.group(2)) > 0
                found += 1
    assert found >= 2
    assert re.fullmatch(r"[0-9a-f]{16}", bench.kernel_hash())


def test_launch_accounting_of_fused_rk2_tiles():
    """A fused-RK2 tile (pair 5) counts one launch per step doing both
    stages: phi and the target in, phi' out (12 B per node in FP32 with the
    tube), twice the stage FLOPs; any other tile one launch per stage with
    the per-stage averages."""
    spec = W.rockets(n=9)[0]
    stats = {"steps": 7, "stages": 14}
    n = 9 ** 3
    bpn, fpn = bench.algorithmic(spec)
    launches, f, b, fused = bench.launch_accounting(spec, (16, 16, 4, 2, 5), stats)
    assert (launches, fused) == (7, True)
    assert f == pytest.approx(2 * fpn * n) and b == pytest.approx(12 * n)
    launches, f, b, fused = bench.launch_accounting(spec, (16, 16, 4, 2, 0), stats)
    assert (launches, fused) == (14, False)
    assert f == pytest.approx(fpn * n) and b == pytest.approx(bpn * n)
    spec3 = dict(spec, rk=3)  # pair 5 fuses RK2 steps only
    assert bench.launch_accounting(spec3, (16, 16, 4, 2, 5), {"steps": 7, "stages": 21})[3] is False
