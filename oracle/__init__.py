"""FP64 CPU oracle for the HJ level-set hot path (LevelSetPy, arXiv 2411.03501).

TEST INFRASTRUCTURE ONLY.  This package is what the GPU path is checked
against.  Only the tests, the smoke check and the CPU-baseline leg of the
benchmark may import it; the product package never does, and the two share
no code.  The arithmetic lives in ``lsp_oracle.c`` (plain C, one point at a
time, double precision); this module compiles it with gcc and wraps it with
ctypes so that tests can hand it numpy arrays.

Problem description (a plain dict, produced by the seeded input generators):

    {"ndim": d, "n": [...], "lo": [...], "hi": [...], "periodic": [...],
     "scheme": "upwind1" | "eno2" | "eno3" | "weno5",
     "dyn": "normal_speed" | "translate" | "quadratic" | "air3d" | "car4d" |
            "rockets" | "double_integrator",
     "params": [...],
     "diss": "glf" | "llf" | "lllf"   (optional, default "glf"),
     "varform": bool                   (optional: the variational BRT form)}

Function-level citations are in the C source; each wrapper below names the
passage of the paper its C function follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lsp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_lib", "liblsp_oracle.so")

SCHEMES = {"upwind1": 0, "eno2": 1, "eno3": 2, "weno5": 3}
DYNAMICS = {"normal_speed": 0, "translate": 1, "quadratic": 2, "air3d": 3, "car4d": 4,
            "rockets": 5, "double_integrator": 6}


DISSIPATION = {"glf": 0, "llf": 1, "lllf": 2}


class _Problem(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("scheme", ctypes.c_int),
        ("dyn", ctypes.c_int),
        ("diss", ctypes.c_int),
        ("n", ctypes.c_int64 * 4),
        ("lo", ctypes.c_double * 4),
        ("hi", ctypes.c_double * 4),
        ("periodic", ctypes.c_int * 4),
        ("prm", ctypes.c_double * 8),
        ("varform", ctypes.c_int),
        ("pad_", ctypes.c_int),
    ]


class _Stats(ctypes.Structure):
    _fields_ = [
        ("steps", ctypes.c_int64),
        ("stages", ctypes.c_int64),
        ("dt_min", ctypes.c_double),
        ("dt_max", ctypes.c_double),
        ("t_end", ctypes.c_double),
    ]


def build(force: bool = False, openmp: bool = True) -> str:
    """Compile lsp_oracle.c into a shared library (gcc, -O2, OpenMP if the
    compiler supports it).  Returns the library path."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    cc = os.environ.get("CC", "gcc")
    base = [cc, "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", _LIB_PATH + ".tmp", "-lm"]
    cmds = [base[:2] + ["-fopenmp"] + base[2:]] if openmp else []
    cmds.append(base)
    err = None
    for cmd in cmds:
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
            return _LIB_PATH
        err = r.stderr
    raise RuntimeError("oracle build failed:\n" + (err or ""))


_lib = None


def lib():
    global _lib
    if _lib is None:
        # LSP_ORACLE_LIB lets a test point at a separately built copy (used to
        # check that the pins catch mistakes planted in the oracle source).
        path = os.environ.get("LSP_ORACLE_LIB") or build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER(_Problem)
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_dx.argtypes = [P, ctypes.c_int]
        L.orc_dx.restype = ctypes.c_double
        L.orc_derivs.argtypes = [P, dp, ctypes.c_int, dp, dp, dp]
        L.orc_derivs.restype = ctypes.c_int
        L.orc_rate.argtypes = [P, dp, dp, dp, dp]
        L.orc_rate.restype = ctypes.c_int
        L.orc_alpha.argtypes = [P, dp, dp]
        L.orc_alpha.restype = ctypes.c_int
        L.orc_cfl_dt.argtypes = [P, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.orc_cfl_dt.restype = ctypes.c_double
        L.orc_step.argtypes = [P, dp, dp, ctypes.c_int, ctypes.c_double]
        L.orc_step.restype = ctypes.c_int
        L.orc_solve.argtypes = [P, dp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_int64, ctypes.POINTER(_Stats)]
        L.orc_solve.restype = ctypes.c_int
        L.orc_ham.argtypes = [P, dp, dp]
        L.orc_ham.restype = ctypes.c_double
        L.orc_partial_bound.argtypes = [P, dp, ctypes.c_int]
        L.orc_partial_bound.restype = ctypes.c_double
        L.orc_solve_steps.argtypes = [P, dp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_int64]
        L.orc_solve_steps.restype = ctypes.c_int
        L.orc_adjoint.argtypes = [P, dp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_int64, dp, dp,
                                  dp, dp, dp]
        L.orc_adjoint.restype = ctypes.c_int
        L.orc_threads.argtypes = []
        L.orc_threads.restype = ctypes.c_int
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_set_threads.restype = None
        _lib = L
    return _lib


def threads() -> int:
    """OpenMP threads the oracle uses (1 if built without OpenMP)."""
    return int(lib().orc_threads())


def set_threads(n: int) -> None:
    """Use n OpenMP threads in later calls (for timing on one core)."""
    lib().orc_set_threads(int(n))


def _problem(spec: dict) -> _Problem:
    p = _Problem()
    d = int(spec["ndim"])
    p.ndim = d
    p.scheme = SCHEMES[spec["scheme"]]
    p.dyn = DYNAMICS[spec["dyn"]]
    p.diss = DISSIPATION[spec.get("diss", "glf")]
    p.varform = 1 if spec.get("varform", False) else 0
    for k in range(d):
        p.n[k] = int(spec["n"][k])
        p.lo[k] = float(spec["lo"][k])
        p.hi[k] = float(spec["hi"][k])
        p.periodic[k] = 1 if spec["periodic"][k] else 0
    for i, v in enumerate(spec.get("params", [])):
        p.prm[i] = float(v)
    return p


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def dx(spec: dict) -> np.ndarray:
    """Grid spacing per axis (Sec. III-B; periodic axes exclude hi)."""
    p = _problem(spec)
    return np.array([lib().orc_dx(ctypes.byref(p), k) for k in range(spec["ndim"])])


def nodes(spec: dict, k: int) -> np.ndarray:
    """Node coordinates of axis k (Sec. III-B, the grid's 1-D vectors ``vs``)."""
    h = dx(spec)[k]
    return float(spec["lo"][k]) + h * np.arange(int(spec["n"][k]), dtype=np.float64)


def derivs(spec: dict, phi, axis: int, with_ties: bool = False):
    """Left/right derivatives along ``axis`` (Sec. IV-A..IV-C).  Returns
    (p_minus, p_plus) or (p_minus, p_plus, flip) where flip is the change a
    near-tied ENO selection would cause if taken the other way."""
    p = _problem(spec)
    phi = _f64(phi).reshape(spec["n"])
    pm = np.empty_like(phi)
    pp = np.empty_like(phi)
    tie = np.empty_like(phi)
    _check(lib().orc_derivs(ctypes.byref(p), _ptr(phi), axis, _ptr(pm), _ptr(pp), _ptr(tie)),
           "derivs")
    return (pm, pp, tie) if with_ties else (pm, pp)


def alpha(spec: dict, phi) -> np.ndarray:
    """GLF coefficients per axis for this field (Listing 4, dissFunc)."""
    p = _problem(spec)
    phi = _f64(phi).reshape(spec["n"])
    a = np.zeros(4)
    _check(lib().orc_alpha(ctypes.byref(p), _ptr(phi), _ptr(a)), "alpha")
    return a[: spec["ndim"]].copy()


def rate(spec: dict, phi, alpha_in=None):
    """Method-of-lines rate L = -Hhat (Sec. IV-D, Sec. V-A).  Returns
    (L, alpha_used)."""
    p = _problem(spec)
    phi = _f64(phi).reshape(spec["n"])
    out = np.empty_like(phi)
    a_out = np.zeros(4)
    a_in = None
    if alpha_in is not None:
        a_in = np.zeros(4)
        a_in[: spec["ndim"]] = alpha_in
    _check(lib().orc_rate(ctypes.byref(p), _ptr(phi), _ptr(a_in) if a_in is not None else None,
                          _ptr(a_out), _ptr(out)), "rate")
    return out, a_out[: spec["ndim"]].copy()


def ham(spec: dict, x, p) -> float:
    """Hamiltonian H(x, p) of the dynamics in ``spec`` (Sec. VI-A pattern,
    Eqs. 31-32: closed form of -max_u min_d p.f)."""
    P = _problem(spec)
    xa = np.zeros(4)
    pa = np.zeros(4)
    xa[: spec["ndim"]] = x
    pa[: spec["ndim"]] = p
    return float(lib().orc_ham(ctypes.byref(P), _ptr(xa), _ptr(pa)))


def partial_bound(spec: dict, x, k: int) -> float:
    """Per-node bound on |dH/dp_k| (partialFunc, Listing 4)."""
    P = _problem(spec)
    xa = np.zeros(4)
    xa[: spec["ndim"]] = x
    return float(lib().orc_partial_bound(ctypes.byref(P), _ptr(xa), int(k)))


def cfl_dt(spec: dict, alpha_v, cfl: float, t: float, t_final: float) -> float:
    """CFL-limited step (Sec. IV-D, Sec. V-A)."""
    p = _problem(spec)
    a = np.zeros(4)
    a[: spec["ndim"]] = alpha_v
    return float(lib().orc_cfl_dt(ctypes.byref(p), _ptr(a), cfl, t, t_final))


def step(spec: dict, phi, dt: float, rk_order: int, target=None) -> np.ndarray:
    """One TVD-RK step (Sec. V-A) plus, if ``target`` is given, the min with
    the target (Sec. VI-A).  Returns the new field."""
    p = _problem(spec)
    out = _f64(phi).reshape(spec["n"]).copy()
    g = None if target is None else _f64(target).reshape(spec["n"])
    _check(lib().orc_step(ctypes.byref(p), _ptr(out), _ptr(g) if g is not None else None,
                          int(rk_order), float(dt)), "step")
    return out


def solve(spec: dict, phi0, t_final: float, rk_order: int, cfl: float, target=None,
          t0: float = 0.0, max_steps: int = 0):
    """Integrate to t_final (odeCFLx, Listing 3).  Returns (phi, stats dict)."""
    p = _problem(spec)
    out = _f64(phi0).reshape(spec["n"]).copy()
    g = None if target is None else _f64(target).reshape(spec["n"])
    st = _Stats()
    _check(lib().orc_solve(ctypes.byref(p), _ptr(out), _ptr(g) if g is not None else None,
                           int(rk_order), float(cfl), float(t0), float(t_final),
                           int(max_steps), ctypes.byref(st)), "solve")
    return out, {"steps": st.steps, "stages": st.stages, "dt_min": st.dt_min,
                 "dt_max": st.dt_max, "t_end": st.t_end}


def solve_steps(spec: dict, phi0, nsteps: int, rk_order: int, cfl: float, target=None):
    """Fixed number of steps with the CFL step of the state-only GLF bounds
    (no shortened last step): the forward map the adjoint reverses."""
    p = _problem(spec)
    out = _f64(phi0).reshape(spec["n"]).copy()
    g = None if target is None else _f64(target).reshape(spec["n"])
    _check(lib().orc_solve_steps(ctypes.byref(p), _ptr(out), _ptr(g) if g is not None else None,
                                 int(rk_order), float(cfl), int(nsteps)), "solve_steps")
    return out


def adjoint(spec: dict, phi0, nsteps: int, rk_order: int, cfl: float, lamT, target=None):
    """Discrete adjoint of solve_steps.  Returns (dL/dphi0, dL/dtarget or
    None, dL/dparams (8), phi_T) for dL/dphi_T = lamT."""
    p = _problem(spec)
    phi0 = _f64(phi0).reshape(spec["n"])
    lamT = _f64(lamT).reshape(spec["n"])
    g = None if target is None else _f64(target).reshape(spec["n"])
    lam0 = np.empty_like(phi0)
    lamg = np.empty_like(phi0) if g is not None else None
    dprm = np.zeros(8)
    phiT = np.empty_like(phi0)
    _check(lib().orc_adjoint(ctypes.byref(p), _ptr(phi0), _ptr(g) if g is not None else None,
                             int(rk_order), float(cfl), int(nsteps), _ptr(lamT), _ptr(lam0),
                             _ptr(lamg) if lamg is not None else None, _ptr(dprm), _ptr(phiT)),
           "adjoint")
    return lam0, lamg, dprm, phiT


# ---------------------------------------------------------------- losses
# The scalar losses of the differentiation workload (they are not in the
# paper; plain numpy, FP64): a smoothed volume of {phi <= 0} and the sum of
# phi at query states by multilinear interpolation.
def _interp_weights(spec: dict, q):
    """For each query row, the 2^d (flat node index, weight) pairs of
    multilinear interpolation; periodic axes wrap, others clamp."""
    d = spec["ndim"]
    h = dx(spec)
    idx = []
    frac = []
    for k in range(d):
        t = (q[:, k] - spec["lo"][k]) / h[k]
        n = spec["n"][k]
        if spec["periodic"][k]:
            i0 = np.floor(t).astype(np.int64)
            f = t - i0
            i0 = np.mod(i0, n)
            i1 = np.mod(i0 + 1, n)
        else:
            t = np.clip(t, 0.0, n - 1.0)
            i0 = np.minimum(np.floor(t).astype(np.int64), n - 2)
            f = t - i0
            i1 = i0 + 1
        idx.append((i0, i1))
        frac.append(f)
    out = []
    for corner in range(2 ** d):
        w = np.ones(len(q))
        flat = np.zeros(len(q), dtype=np.int64)
        for k in range(d):
            b = (corner >> (d - 1 - k)) & 1
            w = w * (frac[k] if b else 1.0 - frac[k])
            flat = flat * spec["n"][k] + idx[k][b]
        out.append((flat, w))
    return out


def loss(spec: dict, phi, queries):
    """sum_i H_eps(-phi_i) dV + sum_q phi(x_q), H_eps(s) = 1/(1+exp(-s/eps)),
    eps = max dx, dV = prod dx."""
    h = dx(spec)
    eps = float(h.max())
    dV = float(np.prod(h))
    f = _f64(phi).ravel()
    vol = np.sum(1.0 / (1.0 + np.exp(f / eps))) * dV
    val = 0.0
    for flat, w in _interp_weights(spec, np.asarray(queries, dtype=np.float64)):
        val += np.sum(w * f[flat])
    return float(vol + val)


def loss_grad(spec: dict, phi, queries):
    """d loss / d phi (same shape as phi)."""
    h = dx(spec)
    eps = float(h.max())
    dV = float(np.prod(h))
    f = _f64(phi).ravel()
    Hs = 1.0 / (1.0 + np.exp(f / eps))  # H_eps(-phi)
    g = -Hs * (1.0 - Hs) / eps * dV
    for flat, w in _interp_weights(spec, np.asarray(queries, dtype=np.float64)):
        np.add.at(g, flat, w)
    return g.reshape(spec["n"])


if __name__ == "__main__":  # pragma: no cover - manual build entry
    print(build(force="--force" in sys.argv))
