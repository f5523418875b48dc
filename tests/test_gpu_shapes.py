"""Implicit surfaces on the device (through the C ABI) against the oracle's
definitions, node by node, in FP64 and FP32 arithmetic, on ragged 2-D to 4-D
grids; set operations bit for bit."""
import numpy as np
import pytest
import torch

from oracle import shapes as S
from paper_2411_03501_gb300 import binding as B
from paper_2411_03501_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SPECS = {
    1: W.problem(1, [53], [-3], [2], [False], "eno2", "normal_speed", [1.0]),
    2: W.problem(2, [37, 29], [-2, -1], [2, 1.5], [False, True], "eno2", "normal_speed", [1.0]),
    3: W.problem(3, [21, 17, 19], [-6, -10, 0], [20, 10, 2 * np.pi], [False, False, True], "eno2",
                 "normal_speed", [1.0]),
    4: W.problem(4, [9, 11, 8, 7], [-4, -4, 0, 0], [4, 4, 2 * np.pi, 2], [False, False, True, False],
                 "eno2", "normal_speed", [1.0]),
}


def _grid(spec):
    g = B.lsp_grid_create(spec["ndim"], spec["lo"], spec["hi"], spec["n"],
                          ["periodic" if p else "extrapolate" for p in spec["periodic"]])
    return g


def _check(got, want, dtype, scale):
    """scale: the largest magnitude entering the primitive's arithmetic (the
    coordinates, centre and radius; the weighted squares of a quadric); FP32
    arithmetic is held to 32 units of 2^-24 of it, FP64 to 1e-12."""
    got = got.double().cpu().numpy()
    if dtype == torch.float64:
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * scale)
    else:
        err = np.abs(got - want).max()
        assert err <= 32 * 2.0 ** -24 * scale, (err, scale)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("ndim", [1, 2, 3, 4])
def test_primitives_match_oracle(ndim, dtype):
    spec = SPECS[ndim]
    g = _grid(spec)
    out = torch.empty(spec["n"], dtype=dtype, device="cuda")
    c = [0.3, -0.4, 1.0, 0.5][:ndim]
    X = max(max(abs(v) for v in spec["lo"]), max(abs(v) for v in spec["hi"]))
    lin = np.sqrt(ndim) * (X + 1.0) + 2.0  # distances, coordinates, centre, radius
    B.lsp_shape_sphere(g, out, c, 1.7)
    _check(out, S.sphere(spec, c, 1.7), dtype, lin)
    if ndim > 1:  # (ignoring the only dimension of a 1-D grid leaves no distance)
        B.lsp_shape_sphere(g, out, c, 1.2, ignore=(ndim - 1,))
        _check(out, S.sphere(spec, c, 1.2, ignore=(ndim - 1,)), dtype, lin)
    lo, hi = [-1.0, -0.5, 0.5, 0.2][:ndim], [1.5, 0.8, 3.0, 1.1][:ndim]
    B.lsp_shape_box(g, out, lo, hi)
    _check(out, S.box(spec, lo, hi), dtype, lin)
    if ndim > 1:
        B.lsp_shape_box(g, out, lo, hi, ignore=(0,))
        _check(out, S.box(spec, lo, hi, ignore=(0,)), dtype, lin)
    w = [1.0, 4.0, 9.0, 2.0][:ndim]
    B.lsp_shape_quadric(g, out, c, w, 2.5)
    _check(out, S.quadric(spec, c, w, 2.5), dtype, sum(w) * (X + 1.0) ** 2 + 2.5)
    nrm = [1.0, -2.0, 0.5, 0.3][:ndim]
    B.lsp_shape_halfspace(g, out, nrm, c)
    _check(out, S.halfspace(spec, nrm, c), dtype, 4.0 * lin)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_set_operations_are_exact(dtype):
    spec = SPECS[3]
    g = _grid(spec)
    a = torch.empty(spec["n"], dtype=dtype, device="cuda")
    b = torch.empty_like(a)
    B.lsp_shape_sphere(g, a, [2.0, 0.0, 0.0], 6.0, ignore=(2,))
    B.lsp_shape_box(g, b, [-2.0, -3.0, 1.0], [8.0, 3.0, 4.0])
    ah, bh = a.double().cpu().numpy(), b.double().cpu().numpy()
    out = torch.empty_like(a)
    for op, fn in (("union", S.union), ("intersect", S.intersect),
                   ("difference", S.difference)):
        B.lsp_shape_op(op, a, b, out)
        assert np.array_equal(out.double().cpu().numpy(), fn(ah, bh)), op
    B.lsp_shape_op("complement", a, None, out)
    assert np.array_equal(out.double().cpu().numpy(), S.complement(ah))
    B.lsp_shape_op("union", a, b, a)  # in place
    assert np.array_equal(a.double().cpu().numpy(), S.union(ah, bh))


def test_shape_argument_errors():
    spec = SPECS[2]
    g = _grid(spec)
    out = torch.empty(spec["n"], dtype=torch.float32, device="cuda")
    for call in (lambda: B.lsp_shape_sphere(g, out, [0, 0], -1.0),
                 lambda: B.lsp_shape_sphere(g, out, [0, 0], 1.0, ignore=(0, 1)),
                 lambda: B.lsp_shape_box(g, out, [1, 0], [0, 1]),
                 lambda: B.lsp_shape_halfspace(g, out, [0, 0], [0, 0])):
        with pytest.raises(B.LspError) as e:
            call()
        assert e.value.status == B.LSP_EINVAL


def test_large_grid_node_coordinates():
    """A 3-D grid of 16.6 M nodes (indices above 2^24, ragged axis lengths):
    the node index split by the axis lengths (multiply-high division) gives
    every node's coordinates, checked through a sphere in FP32 against the
    oracle at every node."""
    spec = W.problem(3, [257, 255, 253], [-6, -10, 0], [20, 10, 2 * np.pi], [False, False, True],
                     "eno2", "normal_speed", [1.0])
    g = _grid(spec)
    out = torch.empty(tuple(spec["n"]), dtype=torch.float32, device="cuda")
    c = [0.3, -0.4, 1.0]
    B.lsp_shape_sphere(g, out, c, 1.2)
    _check(out, S.sphere(spec, c, 1.2), torch.float32, np.sqrt(3) * 21.0 + 2.0)

