"""Thin ctypes binding of the C ABI in ``include/lsp.h``.

Functions keep the C names and only marshal arguments: torch tensors become
device pointers, the current torch CUDA stream becomes the ``stream``
argument, and a non-OK status raises :class:`LspError` with the library's
error text.  Every step of the computation runs in the CUDA library; if it
has not been built, the first call raises (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "liblsp.so")

LSP_OK, LSP_EINVAL, LSP_ENOMEM, LSP_ECUDA, LSP_EUNSUPPORTED, LSP_ENONFINITE, LSP_ETIMEOUT = range(7)
BC = {"extrapolate": 0, "periodic": 1}
SCHEMES = {"upwind1": 0, "eno2": 1, "eno3": 2, "weno5": 3}
DYNAMICS = {"normal_speed": 0, "translate": 1, "quadratic": 2, "air3d": 3, "car4d": 4,
            "rockets": 5, "double_integrator": 6}
DTYPES = {"f32": 0, "f64": 1}
DISSIPATION = {"glf": 0, "llf": 1, "lllf": 2}

# Every symbol the header declares (checked by the ABI test).
EXPORTS = [
    "lsp_version", "lsp_status_string", "lsp_last_error", "lsp_grid_create", "lsp_grid_destroy",
    "lsp_set_dynamics", "lsp_get_alpha", "lsp_workspace_size", "lsp_cfl_dt", "lsp_hj_rate",
    "lsp_hj_step", "lsp_hj_solve", "lsp_check_status", "lsp_hj_solve_noalloc",
    "lsp_set_tile", "lsp_get_tile", "lsp_autotune", "lsp_batched_workspace_size",
    "lsp_hj_solve_batched", "lsp_batched_autotune", "lsp_adjoint_workspace_size", "lsp_hj_solve_ckpt", "lsp_hj_adjoint",
    "lsp_loss_tube", "lsp_debug_stall_problem", "lsp_shape_sphere", "lsp_shape_box",
    "lsp_shape_quadric", "lsp_shape_halfspace", "lsp_shape_op",
]
SHAPE_OPS = {"union": 0, "intersect": 1, "complement": 2, "difference": 3}


class LspError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"lsp status {status}: {msg}")
        self.status = status


class lsp_solve_opts(ctypes.Structure):
    _fields_ = [
        ("rk_order", ctypes.c_int),
        ("scheme", ctypes.c_int),
        ("dtype", ctypes.c_int),
        ("tube", ctypes.c_int),
        ("cfl", ctypes.c_double),
        ("check_finite", ctypes.c_int),
        ("use_graph", ctypes.c_int),
        ("batch_chunk", ctypes.c_int),
        ("batch_persistent", ctypes.c_int),
        ("batch_wait_ms", ctypes.c_int),
        ("diss", ctypes.c_int),
        ("varform", ctypes.c_int),
        ("batch_tiles", ctypes.c_int),
    ]


class lsp_solve_stats(ctypes.Structure):
    _fields_ = [
        ("steps", ctypes.c_int64),
        ("stages", ctypes.c_int64),
        ("dt_min", ctypes.c_double),
        ("dt_max", ctypes.c_double),
        ("t_end", ctypes.c_double),
    ]


_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load liblsp.so (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(path)
    vp, sz = ctypes.c_void_p, ctypes.c_size_t
    dp = ctypes.POINTER(ctypes.c_double)
    op = ctypes.POINTER(lsp_solve_opts)
    L.lsp_version.restype = ctypes.c_int
    L.lsp_status_string.argtypes = [ctypes.c_int]
    L.lsp_status_string.restype = ctypes.c_char_p
    L.lsp_last_error.restype = ctypes.c_char_p
    L.lsp_grid_create.argtypes = [ctypes.c_int, dp, dp, ctypes.POINTER(ctypes.c_int64),
                                  ctypes.POINTER(ctypes.c_int), ctypes.POINTER(vp)]
    L.lsp_grid_destroy.argtypes = [vp]
    L.lsp_grid_destroy.restype = None
    L.lsp_set_dynamics.argtypes = [vp, ctypes.c_int, dp, ctypes.c_int]
    L.lsp_get_alpha.argtypes = [vp, dp]
    L.lsp_workspace_size.argtypes = [vp, op, ctypes.POINTER(sz)]
    L.lsp_cfl_dt.argtypes = [vp, op, ctypes.c_double, ctypes.c_double, dp]
    L.lsp_hj_rate.argtypes = [vp, op, vp, vp, vp, sz, vp]
    L.lsp_hj_step.argtypes = [vp, op, vp, vp, ctypes.c_double, dp, vp, sz, vp]
    L.lsp_hj_solve.argtypes = [vp, op, vp, vp, ctypes.c_double, ctypes.c_double, vp, sz,
                               ctypes.POINTER(lsp_solve_stats), vp]
    L.lsp_check_status.argtypes = [vp, vp]
    ui = ctypes.c_uint
    L.lsp_shape_sphere.argtypes = [vp, ctypes.c_int, dp, ctypes.c_double, ui, vp, vp]
    L.lsp_shape_box.argtypes = [vp, ctypes.c_int, dp, dp, ui, vp, vp]
    L.lsp_shape_quadric.argtypes = [vp, ctypes.c_int, dp, dp, ctypes.c_double, ui, vp, vp]
    L.lsp_shape_halfspace.argtypes = [vp, ctypes.c_int, dp, dp, ui, vp, vp]
    L.lsp_shape_op.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp, ctypes.c_int64, vp]
    L.lsp_debug_stall_problem.argtypes = [ctypes.c_int]
    L.lsp_debug_stall_problem.restype = ctypes.c_int
    L.lsp_hj_solve_noalloc.argtypes = [vp, op, vp, vp, ctypes.c_double, ctypes.c_double,
                                       ctypes.POINTER(lsp_solve_stats), vp]
    ip = ctypes.POINTER(ctypes.c_int)
    L.lsp_set_tile.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               ctypes.c_int]
    L.lsp_get_tile.argtypes = [vp, op, ip, ip, ip, ip, ip]
    L.lsp_autotune.argtypes = [vp, op, vp, vp, sz, vp, ip, ip, ip, ip, ip]
    pp = ctypes.POINTER(vp)
    L.lsp_batched_workspace_size.argtypes = [ctypes.c_int, pp, op, ctypes.POINTER(sz)]
    L.lsp_hj_solve_batched.argtypes = [ctypes.c_int, pp, op, pp, pp, dp, vp, sz,
                                       ctypes.POINTER(lsp_solve_stats), vp]
    L.lsp_batched_autotune.argtypes = [ctypes.c_int, pp, op, pp, pp, dp, vp, sz, vp, ip]
    ci = ctypes.c_int
    L.lsp_adjoint_workspace_size.argtypes = [vp, op, ci, ci, ctypes.POINTER(sz)]
    L.lsp_hj_solve_ckpt.argtypes = [vp, op, vp, vp, ci, ci, vp, sz, vp]
    L.lsp_hj_adjoint.argtypes = [vp, op, vp, ci, ci, vp, vp, vp, dp, vp, sz, vp]
    L.lsp_loss_tube.argtypes = [vp, ci, vp, vp, ci, vp, vp, vp]
    for name in ("lsp_set_tile", "lsp_get_tile", "lsp_autotune", "lsp_batched_workspace_size",
                 "lsp_hj_solve_batched", "lsp_batched_autotune", "lsp_adjoint_workspace_size", "lsp_hj_solve_ckpt",
                 "lsp_hj_adjoint", "lsp_loss_tube"):
        getattr(L, name).restype = ctypes.c_int
    for name in ("lsp_grid_create", "lsp_set_dynamics", "lsp_get_alpha", "lsp_workspace_size",
                 "lsp_cfl_dt", "lsp_hj_rate", "lsp_hj_step", "lsp_hj_solve", "lsp_check_status",
                 "lsp_hj_solve_noalloc"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(status: int):
    if status != LSP_OK:
        raise LspError(status, load().lsp_last_error().decode())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _nbytes(t) -> int:
    return t.numel() * t.element_size()


class Grid:
    """Owning wrapper of an ``lsp_grid*`` (destroyed with the object)."""

    def __init__(self, handle: int):
        self.handle = ctypes.c_void_p(handle)

    def __del__(self):
        if getattr(self, "handle", None) and self.handle.value and _lib is not None:
            _lib.lsp_grid_destroy(self.handle)
            self.handle = ctypes.c_void_p(0)


def lsp_version() -> int:
    return int(load().lsp_version())


def lsp_grid_create(ndim, gmin, gmax, n, bc) -> Grid:
    D = ctypes.c_double * ndim
    out = ctypes.c_void_p()
    bcs = [BC[b] if isinstance(b, str) else int(b) for b in bc]
    _check(load().lsp_grid_create(ndim, D(*gmin), D(*gmax), (ctypes.c_int64 * ndim)(*n),
                                  (ctypes.c_int * ndim)(*bcs), ctypes.byref(out)))
    return Grid(out.value)


def lsp_set_dynamics(grid: Grid, dyn, params):
    d = DYNAMICS[dyn] if isinstance(dyn, str) else int(dyn)
    arr = (ctypes.c_double * max(1, len(params)))(*params)
    _check(load().lsp_set_dynamics(grid.handle, d, arr, len(params)))


def lsp_get_alpha(grid: Grid, ndim: int):
    a = (ctypes.c_double * 4)()
    _check(load().lsp_get_alpha(grid.handle, a))
    return [a[k] for k in range(ndim)]


def make_opts(rk_order=3, scheme="weno5", dtype="f32", tube=False, cfl=0.75, check_finite=False,
              use_graph=False, diss="glf", varform=False) -> lsp_solve_opts:
    o = lsp_solve_opts()
    o.diss = DISSIPATION[diss] if isinstance(diss, str) else int(diss)
    o.varform = 1 if varform else 0
    o.rk_order = int(rk_order)
    o.scheme = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    o.dtype = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    o.tube = 1 if tube else 0
    o.cfl = float(cfl)
    o.check_finite = 1 if check_finite else 0
    o.use_graph = 1 if use_graph else 0
    return o


def lsp_workspace_size(grid: Grid, opts: lsp_solve_opts) -> int:
    b = ctypes.c_size_t()
    _check(load().lsp_workspace_size(grid.handle, ctypes.byref(opts), ctypes.byref(b)))
    return int(b.value)


def lsp_cfl_dt(grid: Grid, opts: lsp_solve_opts, t: float, t_final: float) -> float:
    dt = ctypes.c_double()
    _check(load().lsp_cfl_dt(grid.handle, ctypes.byref(opts), t, t_final, ctypes.byref(dt)))
    return dt.value


def lsp_hj_rate(grid: Grid, opts, phi, rate, workspace, stream=None):
    _check(load().lsp_hj_rate(grid.handle, ctypes.byref(opts), _ptr(phi), _ptr(rate),
                              _ptr(workspace), _nbytes(workspace), _stream(stream)))


def lsp_hj_step(grid: Grid, opts, phi, target, t, dt, workspace, stream=None) -> float:
    d = ctypes.c_double(dt)
    _check(load().lsp_hj_step(grid.handle, ctypes.byref(opts), _ptr(phi), _ptr(target), t,
                              ctypes.byref(d), _ptr(workspace), _nbytes(workspace),
                              _stream(stream)))
    return d.value


def lsp_hj_solve(grid: Grid, opts, phi, target, t0, t_final, workspace, stream=None) -> dict:
    st = lsp_solve_stats()
    _check(load().lsp_hj_solve(grid.handle, ctypes.byref(opts), _ptr(phi), _ptr(target), t0,
                               t_final, _ptr(workspace), _nbytes(workspace), ctypes.byref(st),
                               _stream(stream)))
    return {"steps": st.steps, "stages": st.stages, "dt_min": st.dt_min, "dt_max": st.dt_max,
            "t_end": st.t_end}


def lsp_hj_solve_noalloc(grid: Grid, opts, phi, target, t0, t_final, stream=None) -> dict:
    st = lsp_solve_stats()
    _check(load().lsp_hj_solve_noalloc(grid.handle, ctypes.byref(opts), _ptr(phi), _ptr(target),
                                       t0, t_final, ctypes.byref(st), _stream(stream)))
    return {"steps": st.steps, "stages": st.stages, "dt_min": st.dt_min, "dt_max": st.dt_max,
            "t_end": st.t_end}


def lsp_set_tile(grid: Grid, tb: int, ta: int, ch: int, minb: int = 3, pair: int = 0):
    _check(load().lsp_set_tile(grid.handle, tb, ta, ch, minb, pair))


def lsp_get_tile(grid: Grid, opts) -> tuple:
    v = [ctypes.c_int() for _ in range(5)]
    _check(load().lsp_get_tile(grid.handle, ctypes.byref(opts), *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def lsp_autotune(grid: Grid, opts, phi, workspace, stream=None) -> tuple:
    v = [ctypes.c_int() for _ in range(5)]
    _check(load().lsp_autotune(grid.handle, ctypes.byref(opts), _ptr(phi), _ptr(workspace),
                               _nbytes(workspace), _stream(stream),
                               *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def _handles(grids):
    arr = (ctypes.c_void_p * len(grids))()
    for i, g in enumerate(grids):
        arr[i] = g.handle.value
    return arr


def lsp_batched_workspace_size(grids, opts) -> int:
    b = ctypes.c_size_t()
    _check(load().lsp_batched_workspace_size(len(grids), _handles(grids), ctypes.byref(opts),
                                             ctypes.byref(b)))
    return int(b.value)


def lsp_hj_solve_batched(grids, opts, phis, targets, t_final, workspace, stream=None) -> list:
    n = len(grids)
    P = (ctypes.c_void_p * n)(*[t.data_ptr() for t in phis])
    T = (ctypes.c_void_p * n)(*[t.data_ptr() for t in targets]) if targets is not None else None
    tf = (ctypes.c_double * n)(*[float(v) for v in t_final])
    st = (lsp_solve_stats * n)()
    _check(load().lsp_hj_solve_batched(n, _handles(grids), ctypes.byref(opts), P, T, tf,
                                       _ptr(workspace), _nbytes(workspace), st, _stream(stream)))
    return [{"steps": s.steps, "stages": s.stages, "dt_min": s.dt_min, "dt_max": s.dt_max,
             "t_end": s.t_end} for s in st]


def lsp_batched_autotune(grids, opts, phis, targets, t_final, workspace, stream=None) -> int:
    """The batch_tiles value (tile shape per problem dimension) that ran the
    batched solve of these problems fastest over a short horizon; phis are
    not modified."""
    n = len(grids)
    P = (ctypes.c_void_p * n)(*[t.data_ptr() for t in phis])
    T = (ctypes.c_void_p * n)(*[t.data_ptr() for t in targets]) if targets is not None else None
    tf = (ctypes.c_double * n)(*[float(v) for v in t_final])
    out = ctypes.c_int(0)
    _check(load().lsp_batched_autotune(n, _handles(grids), ctypes.byref(opts), P, T, tf,
                                       _ptr(workspace), _nbytes(workspace), _stream(stream),
                                       ctypes.byref(out)))
    return int(out.value)


def lsp_adjoint_workspace_size(grid: Grid, opts, nsteps: int, ncheck: int = 0) -> int:
    b = ctypes.c_size_t()
    _check(load().lsp_adjoint_workspace_size(grid.handle, ctypes.byref(opts), int(nsteps),
                                             int(ncheck), ctypes.byref(b)))
    return int(b.value)


def lsp_hj_solve_ckpt(grid: Grid, opts, phi, target, nsteps, ncheck, workspace, stream=None):
    _check(load().lsp_hj_solve_ckpt(grid.handle, ctypes.byref(opts), _ptr(phi), _ptr(target),
                                    int(nsteps), int(ncheck), _ptr(workspace),
                                    _nbytes(workspace), _stream(stream)))


def lsp_hj_adjoint(grid: Grid, opts, target, nsteps, ncheck, lamT, lam0, lam_target, workspace,
                   stream=None) -> list:
    d = (ctypes.c_double * 8)()
    _check(load().lsp_hj_adjoint(grid.handle, ctypes.byref(opts), _ptr(target), int(nsteps),
                                 int(ncheck), _ptr(lamT), _ptr(lam0), _ptr(lam_target), d,
                                 _ptr(workspace), _nbytes(workspace), _stream(stream)))
    return [d[i] for i in range(8)]


def lsp_loss_tube(grid: Grid, dtype, phi, queries, value_dev, grad=None, stream=None):
    dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    nq = 0 if queries is None else queries.shape[0]
    _check(load().lsp_loss_tube(grid.handle, dt, _ptr(phi), _ptr(queries), nq, _ptr(value_dev),
                                _ptr(grad), _stream(stream)))


class Batch:
    """Batched solve of several problem descriptions (dicts of
    :mod:`workloads`) sharing scheme, RK order, CFL and tube."""

    def __init__(self, specs, device="cuda", check_finite=False, use_graph=True, chunk=0,
                 persistent=False, wait_ms=0, tiles=0):
        import torch
        self.specs = specs
        self.grids = []
        for sp in specs:
            g = lsp_grid_create(sp["ndim"], sp["lo"], sp["hi"], sp["n"],
                                ["periodic" if p else "extrapolate" for p in sp["periodic"]])
            lsp_set_dynamics(g, sp["dyn"], sp["params"])
            self.grids.append(g)
        s0 = specs[0]
        self.opts = make_opts(s0.get("rk", 3), s0["scheme"], "f32", s0.get("tube", False),
                              s0.get("cfl", 0.75), check_finite, use_graph,
                              s0.get("diss", "glf"), s0.get("varform", False))
        self.opts.batch_chunk = int(chunk)
        self.opts.batch_persistent = 1 if persistent else 0
        self.opts.batch_wait_ms = int(wait_ms)
        self.opts.batch_tiles = int(tiles)
        nbytes = lsp_batched_workspace_size(self.grids, self.opts)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)

    def solve(self, phis, targets=None, t_final=None, stream=None):
        tf = [sp["t_final"] for sp in self.specs] if t_final is None else t_final
        return lsp_hj_solve_batched(self.grids, self.opts, phis, targets, tf, self.workspace,
                                    stream)

    def autotune(self, phis, targets=None, t_final=None, stream=None) -> int:
        """Pick the tile shape per problem dimension (lsp_batched_autotune)
        and keep it for later solves; returns the batch_tiles value."""
        tf = [sp["t_final"] for sp in self.specs] if t_final is None else t_final
        self.opts.batch_tiles = lsp_batched_autotune(self.grids, self.opts, phis, targets, tf,
                                                     self.workspace, stream)
        return self.opts.batch_tiles


def lsp_check_status(workspace, stream=None):
    _check(load().lsp_check_status(_ptr(workspace), _stream(stream)))


def _darr(v, d=4):
    a = (ctypes.c_double * d)()
    for i, x in enumerate(v):
        a[i] = float(x)
    return a


def _mask(ignore) -> int:
    m = 0
    for k in ignore or ():
        m |= 1 << int(k)
    return m


def _dtype_of(t) -> int:
    import torch
    if t.dtype == torch.float64:
        return DTYPES["f64"]
    if t.dtype == torch.float32:
        return DTYPES["f32"]
    raise TypeError("shape fields are float32 or float64 tensors")


def lsp_shape_sphere(grid: Grid, out, center, radius, ignore=(), stream=None):
    """Signed distance to a sphere (a cylinder along the ignored dims)."""
    _check(load().lsp_shape_sphere(grid.handle, _dtype_of(out), _darr(center), float(radius),
                                   _mask(ignore), _ptr(out), _stream(stream)))
    return out


def lsp_shape_box(grid: Grid, out, lo, hi, ignore=(), stream=None):
    _check(load().lsp_shape_box(grid.handle, _dtype_of(out), _darr(lo), _darr(hi), _mask(ignore),
                                _ptr(out), _stream(stream)))
    return out


def lsp_shape_quadric(grid: Grid, out, center, weights, offset, ignore=(), stream=None):
    _check(load().lsp_shape_quadric(grid.handle, _dtype_of(out), _darr(center), _darr(weights),
                                    float(offset), _mask(ignore), _ptr(out), _stream(stream)))
    return out


def lsp_shape_halfspace(grid: Grid, out, normal, point, ignore=(), stream=None):
    _check(load().lsp_shape_halfspace(grid.handle, _dtype_of(out), _darr(normal), _darr(point),
                                      _mask(ignore), _ptr(out), _stream(stream)))
    return out


def lsp_shape_op(op, a, b, out, stream=None):
    """union / intersect / complement / difference of implicit fields."""
    code = SHAPE_OPS[op] if isinstance(op, str) else int(op)
    _check(load().lsp_shape_op(code, _dtype_of(a), _ptr(a), _ptr(b), _ptr(out), int(a.numel()),
                               _stream(stream)))
    return out


def lsp_debug_stall_problem(problem: int) -> int:
    """Testing aid: the persistent batched launch never counts problem
    `problem` done (-1: off), so its bounded waits run out."""
    return int(load().lsp_debug_stall_problem(int(problem)))


# ----------------------------------------------------------------- helpers
class Problem:
    """Grid + dynamics + options built from a problem description dict (the
    format of :mod:`workloads`), with a workspace tensor of the right size."""

    def __init__(self, spec: dict, device="cuda", check_finite=False, use_graph=False):
        import torch
        self.spec = spec
        d = spec["ndim"]
        self.grid = lsp_grid_create(d, spec["lo"], spec["hi"], spec["n"],
                                    ["periodic" if p else "extrapolate" for p in spec["periodic"]])
        lsp_set_dynamics(self.grid, spec["dyn"], spec["params"])
        self.opts = make_opts(spec.get("rk", 3), spec["scheme"], spec.get("dtype", "f32"),
                              spec.get("tube", False), spec.get("cfl", 0.75), check_finite,
                              use_graph, spec.get("diss", "glf"), spec.get("varform", False))
        self.torch_dtype = torch.float64 if spec.get("dtype", "f32") == "f64" else torch.float32
        nbytes = lsp_workspace_size(self.grid, self.opts)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)

    def tensor(self, arr, device="cuda"):
        import torch
        return torch.as_tensor(arr).to(device=device, dtype=self.torch_dtype).contiguous()

    def solve(self, phi, target=None, t0=0.0, t_final=None, stream=None):
        tf = self.spec["t_final"] if t_final is None else t_final
        return lsp_hj_solve(self.grid, self.opts, phi, target, t0, tf, self.workspace, stream)

    def step(self, phi, target=None, t=0.0, dt=0.0, stream=None):
        return lsp_hj_step(self.grid, self.opts, phi, target, t, dt, self.workspace, stream)

    def rate(self, phi, out, stream=None):
        lsp_hj_rate(self.grid, self.opts, phi, out, self.workspace, stream)
        return out

    def alpha(self):
        return lsp_get_alpha(self.grid, self.spec["ndim"])

    def set_tile(self, tb, ta=0, ch=0, minb=3, pair=0):
        lsp_set_tile(self.grid, tb, ta, ch, minb, pair)

    def tile(self):
        return lsp_get_tile(self.grid, self.opts)

    def autotune(self, phi, stream=None):
        return lsp_autotune(self.grid, self.opts, phi, self.workspace, stream)
