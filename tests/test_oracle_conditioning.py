"""Conditioning of the discretisation itself (no GPU): rounding the FP64
oracle's field to FP32 once per step, the air3d tube departs from the
unrounded run by less than 1e-4 max|phi| away from the extrapolated
boundaries, but by more inside the 6-cell layer next to them.  This is why
the FP32 precision bar of the GPU tests is stated on the interior, with a
looser bound on that layer."""
import numpy as np
import pytest

from paper_2411_03501_gb300 import workloads as W


@pytest.mark.slow
def test_extrapolated_boundary_layer_amplifies_rounding(orc):
    spec, phi0, g = W.air3d(n=41)
    phi0 = phi0.astype(np.float32).astype(np.float64)
    g = g.astype(np.float32).astype(np.float64)
    ref, st = orc.solve(spec, phi0, 2.8, 3, 0.75, target=g)
    a = orc.alpha(spec, phi0)
    p, t = phi0.copy(), 0.0
    for _ in range(st["steps"]):
        dt = orc.cfl_dt(spec, a, 0.75, t, 2.8)
        p = orc.step(spec, p, dt, 3, target=g).astype(np.float32).astype(np.float64)
        t += dt
    d = np.abs(p - ref)
    scale = np.abs(ref).max()
    inner = (slice(6, -6), slice(6, -6), slice(None))
    assert d[inner].max() < 1e-4 * scale
    assert d.max() > 1e-4 * scale  # the layer is worse than the bar ...
    assert d.max() < 3e-3 * scale  # ... and within the bound the GPU tests use
