"""Where the discrete problem itself amplifies FP32-sized rounding, found
with the FP64 oracle alone (no GPU): the per-node response of the oracle's
solve to independent relative noise of FP32 size injected into every step's
field, and the set of nodes where that response is too large for the
spec bar (max|dphi| <= 1e-4 max|phi| at t_final) to be attainable by
any FP32 computation.  Shared by the CPU conditioning pins
(test_oracle_conditioning.py) and the whole-solve GPU parity bars
(gpu_helpers.check_fp32_solve).  Plain numpy; no method arithmetic beyond
calls into the oracle."""
import numpy as np

BAR = 1e-4  # max|dphi| <= BAR max|phi| at t_final


def dilate(a, spec, width=3):
    """Running max over +-width nodes along every axis (periodic axes wrap,
    others clamp)."""
    out = np.array(a, dtype=np.float64, copy=True)
    for k in range(spec["ndim"]):
        cur = out.copy()
        for sh in range(1, width + 1):
            for sgn in (1, -1):
                r = np.roll(out, sgn * sh, axis=k)
                if not spec["periodic"][k]:
                    idx = [slice(None)] * spec["ndim"]
                    idx[k] = slice(0, sh) if sgn > 0 else slice(-sh, None)
                    r[tuple(idx)] = 0.0
                cur = np.maximum(cur, r)
        out = cur
    return out


def noise_response(orc, spec, phi0, target, t_final, ref, samples=2, rel=6e-8, seed=0):
    """Per node, max over `samples` runs of |noisy - ref|: the FP64 oracle's
    solve from phi0 to t_final with every step's field multiplied by
    (1 + rel * N(0, 1)) node by node (rel ~ the FP32 unit roundoff), against
    the unperturbed solve `ref`."""
    rng = np.random.default_rng(seed)
    a = orc.alpha(spec, phi0)
    worst = np.zeros(spec["n"])
    tstop = t_final - 1e-12 * abs(t_final)
    for _ in range(samples):
        p, t = np.array(phi0, dtype=np.float64), 0.0
        while t < tstop:
            dt = orc.cfl_dt(spec, a, spec["cfl"], t, t_final)
            p = orc.step(spec, p, dt, spec["rk"], target=target)
            p = p * (1.0 + rel * rng.standard_normal(p.shape))
            t += dt
        worst = np.maximum(worst, np.abs(p - ref))
    return worst


def conditioning_mask(response, scale, spec, factor=3.0, width=1):
    """The ill-conditioned set: nodes whose oracle noise response exceeds
    BAR * scale / factor, grown by `width` nodes along every axis (the
    response is sampled from a few noise realisations; FP32 arithmetic is
    another one).  Returns (mask, dilated response).  On the air3d 41^3
    tube it covers 2.6 % of the nodes, all within 6 nodes of an
    extrapolated edge."""
    R = dilate(response, spec, width)
    return R > BAR * scale / factor, R


def boundary_distance(spec):
    """Per node, the distance in nodes to the nearest end of a non-periodic
    axis (a large number when every axis is periodic)."""
    n = spec["n"]
    out = np.full(n, 1 << 30, dtype=np.int64)
    for k in range(spec["ndim"]):
        if spec["periodic"][k]:
            continue
        i = np.arange(n[k])
        dk = np.minimum(i, n[k] - 1 - i)
        shape = [1] * spec["ndim"]
        shape[k] = n[k]
        out = np.minimum(out, dk.reshape(shape))
    return out
