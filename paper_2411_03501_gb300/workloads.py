"""Seeded synthetic inputs for the HJ level-set integrator.

This module builds problem descriptions (grid, scheme, dynamics, integrator
options) and the initial / target fields for them.  It holds none of the
method's arithmetic -- no derivative, Hamiltonian, time step or update --
only inputs, so that the GPU path and the FP64 oracle can both be fed the
same arrays.  Every random draw is seeded.

Workloads follow the shapes of the paper's examples (Sec. VI-A: a cylinder
target around the origin, a 3-D relative-dynamics game, 100-200 nodes per
axis) since the paper ships no dataset:

* ``normal_speed_2d``: 2-D front expanding at unit normal speed, circle of
  radius 0.3 on [-1, 1]^2, 101^2 nodes, ENO2, RK2, CFL 0.9, t_final 0.5, FP64.
* ``air3d``: relative pursuit-evasion game (x, y, theta), v_e = v_p = 5,
  turn-rate bounds 1, cylinder target of radius 5, x in [-6, 20],
  y in [-10, 10], theta in [0, 2 pi) periodic, 201^3 nodes, WENO5, RK3,
  CFL 0.75, t_final 2.8, FP32, reachable tube.
* ``car4d``: car (x, y, theta, v), |turn rate| <= 1, |acceleration| <= 1,
  disc target of radius 0.5, x, y in [-4, 4], v in [0, 2], 81^4 nodes, ENO3,
  RK3, CFL 0.75, t_final 1.0, FP32, reachable tube.
* ``rockets``: the two-rocket game of Sec. VI-A (x, z, theta), a = 1,
  g = 32, input bounds 1, cylinder target of capture radius 1.5 along theta,
  100^3 nodes, x, z in [-64, 64], theta in [-pi/2, pi/2] (extrapolated),
  ENO2 (Listing 5), RK2, CFL 0.75, t_final 2.5, FP32, reachable tube.
* ``double_integrator``: x1dot = x2, x2dot = u, |u| <= 1, disc target of
  radius 0.1 on [-1, 1]^2, 101^2 nodes, ENO2, RK2, CFL 0.75, t_final 1.0,
  FP64, reachable tube.
* ``batched``: 256 independent problems, half 2-D normal-speed, half 3-D
  air3d-style, sides, speeds and radii drawn from numpy's default_rng with
  seed 20241105 (side, speed, radius per problem, in that order).
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi


def problem(ndim, n, lo, hi, periodic, scheme, dyn, params, *, rk=3, cfl=0.75,
            t_final=1.0, dtype="f32", tube=False, name="", diss="glf", varform=False):
    """A problem description as a plain dict (no behaviour attached).
    diss: "glf" | "llf" | "lllf" dissipation coefficients; varform: the
    variational form of the reachable-tube PDE (rate clipped at zero)."""
    return {
        "diss": diss,
        "varform": bool(varform),
        "name": name,
        "ndim": int(ndim),
        "n": [int(v) for v in n],
        "lo": [float(v) for v in lo],
        "hi": [float(v) for v in hi],
        "periodic": [bool(v) for v in periodic],
        "scheme": scheme,
        "dyn": dyn,
        "params": [float(v) for v in params],
        "rk": int(rk),
        "cfl": float(cfl),
        "t_final": float(t_final),
        "dtype": dtype,
        "tube": bool(tube),
    }


def axis_nodes(spec: dict, k: int) -> np.ndarray:
    """Node coordinates used to build input fields (non-periodic axes include
    both ends; periodic axes exclude ``hi``)."""
    n = spec["n"][k]
    lo, hi = spec["lo"][k], spec["hi"][k]
    if spec["periodic"][k]:
        return lo + (hi - lo) / n * np.arange(n, dtype=np.float64)
    return lo + (hi - lo) / (n - 1) * np.arange(n, dtype=np.float64)


def mesh(spec: dict):
    """n-D node coordinates with matrix indexing (the grid's ``xs``)."""
    vs = [axis_nodes(spec, k) for k in range(spec["ndim"])]
    return np.meshgrid(*vs, indexing="ij")


def circle_sdf(spec: dict, radius: float, axes=(0, 1), center=None) -> np.ndarray:
    """Signed distance to a circle / cylinder / sphere of ``radius`` in the
    coordinates ``axes`` (other axes ignored), in float64."""
    xs = mesh(spec)
    c = center if center is not None else [0.0] * len(axes)
    r2 = np.zeros(spec["n"], dtype=np.float64)
    for a, ck in zip(axes, c):
        r2 = r2 + (xs[a] - ck) ** 2
    return np.sqrt(r2) - radius


def smooth_field(spec: dict, seed: int, modes: int = 3, amp: float = 1.0) -> np.ndarray:
    """Seeded smooth random field: a sum of products of low-frequency sines
    with random phases, periodic on periodic axes."""
    rng = np.random.default_rng(seed)
    xs = mesh(spec)
    out = np.zeros(spec["n"], dtype=np.float64)
    for _ in range(modes):
        term = np.full(spec["n"], amp * rng.uniform(0.5, 1.0))
        for k in range(spec["ndim"]):
            L = spec["hi"][k] - spec["lo"][k]
            if spec["periodic"][k]:
                f = int(rng.integers(1, 3))
            else:
                f = rng.uniform(0.3, 1.2)
            ph = rng.uniform(0, TWO_PI)
            term = term * np.sin(TWO_PI * f * (xs[k] - spec["lo"][k]) / L + ph)
        out = out + term
    lin = rng.normal(size=spec["ndim"])
    for k in range(spec["ndim"]):
        if not spec["periodic"][k]:
            out = out + 0.3 * lin[k] * xs[k] / max(abs(spec["hi"][k]), abs(spec["lo"][k]))
    return out


def rough_field(spec: dict, seed: int) -> np.ndarray:
    """Seeded field with kinks and a step: a min/max of planes and cones plus
    noise, to exercise ENO/WENO stencil selection."""
    rng = np.random.default_rng(seed)
    xs = mesh(spec)
    r = np.sqrt(sum(x ** 2 for x in xs[: min(2, spec["ndim"])]))
    a = r - rng.uniform(0.2, 0.5) * max(spec["hi"][0] - spec["lo"][0], 1e-9) / 2
    b = xs[0] * rng.uniform(-1, 1) + (xs[1] if spec["ndim"] > 1 else 0.0) * rng.uniform(-1, 1)
    f = np.minimum(a, np.abs(b) - 0.1)
    f = f + 0.05 * rng.standard_normal(spec["n"])
    return f


# ---------------------------------------------------------------- configs
def normal_speed_2d(n: int = 101):
    spec = problem(2, [n, n], [-1, -1], [1, 1], [False, False], "eno2", "normal_speed",
                   [1.0], rk=2, cfl=0.9, t_final=0.5, dtype="f64", tube=False,
                   name=f"normal_speed_2d_{n}^2_eno2_rk2_f64")
    phi0 = circle_sdf(spec, 0.3)
    return spec, phi0, None


def air3d(n: int = 201, ve: float = 5.0, vp: float = 5.0, we: float = 1.0, wp: float = 1.0,
          radius: float = 5.0, t_final: float = 2.8, scheme: str = "weno5", rk: int = 3,
          dtype: str = "f32", nx=None):
    ns = [n, n, n] if nx is None else list(nx)
    spec = problem(3, ns, [-6, -10, 0], [20, 10, TWO_PI], [False, False, True], scheme,
                   "air3d", [ve, vp, we, wp], rk=rk, cfl=0.75, t_final=t_final, dtype=dtype,
                   tube=True, name=f"air3d_{ns[0]}x{ns[1]}x{ns[2]}_{scheme}_rk{rk}_{dtype}")
    g = circle_sdf(spec, radius)
    return spec, g.copy(), g


def car4d(n: int = 81, wmax: float = 1.0, amax: float = 1.0, radius: float = 0.5,
          t_final: float = 1.0, scheme: str = "eno3", dtype: str = "f32"):
    spec = problem(4, [n, n, n, n], [-4, -4, 0, 0], [4, 4, TWO_PI, 2],
                   [False, False, True, False], scheme, "car4d", [wmax, amax], rk=3,
                   cfl=0.75, t_final=t_final, dtype=dtype, tube=True,
                   name=f"car4d_{n}^4_{scheme}_rk3_{dtype}")
    g = circle_sdf(spec, radius)
    return spec, g.copy(), g


def rockets(n: int = 100, a: float = 1.0, g: float = 32.0, ue: float = 1.0, up: float = 1.0,
            radius: float = 1.5, t_final: float = 2.5, scheme: str = "eno2", dtype: str = "f32"):
    """The rockets game of Sec. VI-A on the paper's grid (100 nodes per axis,
    [-64, 64] for x and z; theta over its stated range [-pi/2, pi/2])."""
    spec = problem(3, [n, n, n], [-64, -64, -math.pi / 2], [64, 64, math.pi / 2],
                   [False, False, False], scheme, "rockets", [a, g, ue, up], rk=2, cfl=0.75,
                   t_final=t_final, dtype=dtype, tube=True,
                   name=f"rockets_{n}^3_{scheme}_rk2_{dtype}")
    tgt = circle_sdf(spec, radius)
    return spec, tgt.copy(), tgt


def double_integrator(n: int = 101, umax: float = 1.0, radius: float = 0.1,
                      t_final: float = 1.0, scheme: str = "eno2", dtype: str = "f64"):
    spec = problem(2, [n, n], [-1, -1], [1, 1], [False, False], scheme, "double_integrator",
                   [umax], rk=2, cfl=0.75, t_final=t_final, dtype=dtype, tube=True,
                   name=f"double_integrator_{n}^2_{scheme}_rk2_{dtype}")
    tgt = circle_sdf(spec, radius)
    return spec, tgt.copy(), tgt


def batched(count: int = 256, seed: int = 20241105, scale: float = 1.0):
    """The batched workload: ``count`` problems, the first half 2-D normal-speed
    expansions on [-1, 1]^2 (side ~ U{64..256}, speed ~ U[2, 6], radius ~
    U[0.2, 0.6], t_final = (0.9 - r) / speed), the second half 3-D air3d games
    (side ~ U{48..128}, v_e = v_p = speed ~ U[2, 6], turn bounds 1, radius ~
    U[2, 6] = U[0.2, 0.6] x the smallest half-width 10, t_final 2.8).  All
    WENO5 + RK3, FP32, reachable tubes.  ``scale`` < 1 shrinks the sides and
    horizons for small test runs (same draws)."""
    rng = np.random.default_rng(seed)
    half = count // 2
    out = []
    for i in range(count):
        if i < half:
            side = int(rng.integers(64, 257))
            speed = float(rng.uniform(2.0, 6.0))
            r = float(rng.uniform(0.2, 0.6))
            side = max(9, int(round(side * scale)))
            spec = problem(2, [side, side], [-1, -1], [1, 1], [False, False], "weno5",
                           "normal_speed", [speed], rk=3, cfl=0.75,
                           t_final=(0.9 - r) / speed * (1.0 if scale >= 1 else scale),
                           dtype="f32", tube=True, name=f"b{i}_2d_{side}")
            g = circle_sdf(spec, r)
        else:
            side = int(rng.integers(48, 129))
            speed = float(rng.uniform(2.0, 6.0))
            r = float(rng.uniform(0.2, 0.6)) * 10.0
            side = max(9, int(round(side * scale)))
            spec = problem(3, [side, side, side], [-6, -10, 0], [20, 10, TWO_PI],
                           [False, False, True], "weno5", "air3d", [speed, speed, 1.0, 1.0],
                           rk=3, cfl=0.75, t_final=2.8 * (1.0 if scale >= 1 else scale),
                           dtype="f32", tube=True, name=f"b{i}_3d_{side}")
            g = circle_sdf(spec, r)
        out.append((spec, g.copy(), g))
    return out


CONFIGS = {
    "normal_speed_2d": normal_speed_2d,
    "air3d": air3d,
    "car4d": car4d,
    "rockets": rockets,
    "double_integrator": double_integrator,
}
