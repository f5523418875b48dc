"""The C-ABI library loads, exports every function include/lsp.h declares,
and validates arguments on the host (no GPU needed: nothing here launches a
kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lsp.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lsp_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2411_03501_gb300 import build, binding
    build.build()
    return binding.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2411_03501_gb300 import binding
    names = _declared()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), f"{n} declared in lsp.h but not exported"
    assert sorted(binding.EXPORTS) == sorted(names)


def test_status_strings_and_version(lib):
    from paper_2411_03501_gb300 import binding
    assert binding.lsp_version() >= 100
    for s in range(7):
        assert lib.lsp_status_string(s)
    assert lib.lsp_status_string(99) == b"unknown status"


def test_grid_validation_on_host(lib):
    from paper_2411_03501_gb300 import binding as B
    with pytest.raises(B.LspError) as e:
        B.lsp_grid_create(5, [0] * 5, [1] * 5, [8] * 5, ["periodic"] * 5)
    assert e.value.status == B.LSP_EINVAL
    with pytest.raises(B.LspError):
        B.lsp_grid_create(2, [0, 0], [1, -1], [8, 8], ["periodic"] * 2)
    with pytest.raises(B.LspError):
        B.lsp_grid_create(2, [0, 0], [1, 1], [8, 3], ["periodic"] * 2)
    with pytest.raises(B.LspError):
        B.lsp_grid_create(2, [0, float("nan")], [1, 1], [8, 8], ["periodic"] * 2)
    with pytest.raises(B.LspError):
        B.lsp_grid_create(3, [0] * 3, [1] * 3, [2000] * 3, ["periodic"] * 3)  # > 2^31 nodes
    g = B.lsp_grid_create(2, [0, 0], [1, 1], [9, 11], ["periodic", "extrapolate"])
    with pytest.raises(B.LspError):
        B.lsp_set_dynamics(g, "air3d", [5, 5, 1, 1])  # needs 3-D
    with pytest.raises(B.LspError):
        B.lsp_set_dynamics(g, "normal_speed", [1.0, 2.0])  # wrong count
    with pytest.raises(B.LspError):
        B.lsp_set_dynamics(g, "normal_speed", [float("inf")])
    # QUADRATIC needs no device work at set-up
    B.lsp_set_dynamics(g, "quadratic", [])
    o = B.make_opts(rk_order=3, scheme="weno5", dtype="f32", cfl=0.5)
    n = B.lsp_workspace_size(g, o)
    assert n == 256 + 2 * ((9 * 11 * 4 + 255) // 256 * 256)
    o2 = B.make_opts(rk_order=2, scheme="eno2", dtype="f64", cfl=0.5)
    assert B.lsp_workspace_size(g, o2) == 256 + (9 * 11 * 8 + 255) // 256 * 256
    with pytest.raises(B.LspError):
        B.lsp_workspace_size(g, B.make_opts(rk_order=4))
    with pytest.raises(B.LspError):
        B.lsp_workspace_size(g, B.make_opts(cfl=1.5))
    with pytest.raises(B.LspError) as e:
        B.lsp_get_alpha(g, 2)
    assert e.value.status == B.LSP_EUNSUPPORTED
    # a 7-node axis cannot hold a WENO5 stencil... it can (2*3+1);
    g7 = B.lsp_grid_create(1, [0], [1], [7], ["extrapolate"])
    B.lsp_set_dynamics(g7, "quadratic", [])
    B.lsp_workspace_size(g7, B.make_opts(scheme="weno5"))
    # null / misaligned pointers are rejected before any device work
    ws = ctypes.create_string_buffer(4096)
    with pytest.raises(B.LspError) as e:
        lib_ = B.load()
        st = lib_.lsp_hj_rate(g.handle, ctypes.byref(o), None, None, ctypes.c_void_p(0), 0, None)
        B._check(st)
    assert e.value.status == B.LSP_EINVAL


def test_product_path_fails_loudly_without_library(tmp_path):
    """The binding has no fallback: a missing library is an error."""
    from paper_2411_03501_gb300 import binding as B
    saved = B._lib
    try:
        B._lib = None
        with pytest.raises(RuntimeError):
            B.load(str(tmp_path / "missing.so"))
    finally:
        B._lib = saved


def test_fused_rk2_tile_validation_on_host(lib):
    """Tile variant 5 (both RK2 stages in one launch): accepted on 3-D grids
    when the tile with a 4-node halo fits 4 staged values per thread and with
    a 2-node halo 3 (ENO2's halo); a scheme with a wider halo that does not
    fit runs the generic kernel (reported as all -1); refused on 4-D grids
    and for tiles of more than 256 threads."""
    from paper_2411_03501_gb300 import binding as B
    g = B.lsp_grid_create(3, [0] * 3, [1] * 3, [37, 29, 45], ["extrapolate"] * 3)
    B.lsp_set_dynamics(g, "quadratic", [])  # no device work
    eno2 = B.make_opts(rk_order=2, scheme="eno2", dtype="f32")
    eno3 = B.make_opts(rk_order=2, scheme="eno3", dtype="f32")
    B.lsp_set_tile(g, 32, 8, 5, 3, 5)
    assert B.lsp_get_tile(g, eno2) == (32, 8, 5, 3, 5)
    assert B.lsp_get_tile(g, eno3) == (32, 8, 5, 3, 5)  # (14 x 38, 20 x 44 fit)
    B.lsp_set_tile(g, 64, 4, 5, 3, 5)
    assert B.lsp_get_tile(g, eno2) == (64, 4, 5, 3, 5)
    assert B.lsp_get_tile(g, eno3) == (-1, -1, -1, -1, -1)  # 16 x 76 > 4 x 256
    for bad in [(8, 4, 5, 3, 5), (32, 16, 5, 3, 5), (32, 8, 5, 5, 5), (32, 8, 0, 3, 5)]:
        with pytest.raises(B.LspError):
            B.lsp_set_tile(g, *bad)
    g4 = B.lsp_grid_create(4, [0] * 4, [1] * 4, [9, 8, 10, 11], ["extrapolate"] * 4)
    B.lsp_set_dynamics(g4, "quadratic", [])
    with pytest.raises(B.LspError):
        B.lsp_set_tile(g4, 16, 8, 5, 3, 5)


def test_adjoint_refuses_costate_dependent_bounds(lib):
    """The discrete adjoint reverses the GLF form with state-only bounds: for
    H = |p|^2/2 (whose LF bound depends on the costate) it is refused on the
    host, before any device work."""
    from paper_2411_03501_gb300 import binding as B
    g = B.lsp_grid_create(3, [0] * 3, [1] * 3, [9, 8, 10], ["extrapolate"] * 3)
    B.lsp_set_dynamics(g, "quadratic", [])
    with pytest.raises(B.LspError) as e:
        B.lsp_adjoint_workspace_size(g, B.make_opts(rk_order=3, scheme="weno5"), 4, 0)
    assert e.value.status == B.LSP_EUNSUPPORTED
