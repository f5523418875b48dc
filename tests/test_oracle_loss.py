"""Pins of the differentiation workload's loss in the oracle (oracle.loss,
oracle.loss_grad): the smoothed volume of {phi <= 0} and its gradient
against closed forms for a cylinder, and the multilinear interpolation at
query states against values worked out by hand on fields whose
interpolant is known (a sawtooth along the periodic axis, linear fields at
clamped edges).

The loss is  sum_i H_eps(-phi_i) dV + sum_q phi(x_q)  with
H_eps(s) = 1/(1 + exp(-s/eps)), eps = max_k dx_k, dV = prod_k dx_k.

Closed form of the smoothed volume of a cylinder of radius r (signed
distance s = |(x, y) - c| - r, constant along theta in [0, 2 pi)):
integrating over level sets of s, whose perimeter in the (x, y) plane is
2 pi (r + s),
    int H_eps(-s) 2 pi (r + s) ds = pi r^2 + 2 pi int s (H_eps(-s) - [s <= 0]) ds
and s (H_eps(-s) - [s <= 0]) is even with int_0^inf s/(1 + e^(s/eps)) ds =
eps^2 pi^2 / 12, so the smoothed area is pi r^2 + pi^3 eps^2 / 3, times the
2 pi of the theta axis.  Its derivative under phi -> phi - delta (the
cylinder grows by delta) is the lateral area 2 pi r x 2 pi.
"""
import numpy as np
import pytest

from paper_2411_03501_gb300 import workloads as W


def _cylinder(orc, n=81, r=4.0, c=(7.0, 0.0)):
    spec = W.air3d(n=n)[0]
    phi = W.circle_sdf(spec, r, center=list(c))
    return spec, phi, float(orc.dx(spec).max())


def test_smoothed_volume_of_a_cylinder_matches_closed_form(orc):
    """Far from the domain edges (>= 6 units, 18 eps) the grid sum equals the
    closed form to the quadrature error of a smooth function resolved on
    ~1.3 nodes per eps (measured 6e-8 relative at 81^3); the sharp volume
    (no curvature term) is 2 % away, the volume of {phi >= 0} (an exponent
    with the wrong sign) is 10 times larger."""
    spec, phi, eps = _cylinder(orc)
    r = 4.0
    got = orc.loss(spec, phi, np.zeros((0, 3)))
    want = 2 * np.pi * (np.pi * r ** 2 + np.pi ** 3 * eps ** 2 / 3)
    assert abs(got - want) <= 1e-6 * want, (got, want)
    sharp = 2 * np.pi * np.pi * r ** 2
    assert abs(got - sharp) > 20e-3 * want  # the pin resolves the curvature term


def test_smoothed_volume_converges_under_refinement(orc):
    """With eps tied to the grid, the smoothed volume tends to the sharp
    one as the grid is refined (error ~ eps^2)."""
    r = 4.0
    sharp = 2 * np.pi * np.pi * r ** 2
    errs = []
    for n in (41, 81, 161):
        spec, phi, eps = _cylinder(orc, n=n, r=r)
        errs.append(abs(orc.loss(spec, phi, np.zeros((0, 3))) - sharp))
    assert errs[0] > 3.0 * errs[1] > 9.0 * errs[2]


def test_volume_gradient_is_minus_the_lateral_area(orc):
    """Shifting phi down by delta grows the cylinder by delta: d vol/d delta
    = -sum_i dloss/dphi_i = 2 pi r x 2 pi; every entry is <= 0 (raising phi
    anywhere can only shrink {phi <= 0})."""
    spec, phi, eps = _cylinder(orc)
    r = 4.0
    g = orc.loss_grad(spec, phi, np.zeros((0, 3)))
    assert np.all(g <= 0.0)
    want = 2 * np.pi * r * 2 * np.pi
    assert abs(-g.sum() - want) <= 1e-5 * want, (-g.sum(), want)


def test_query_interpolation_wraps_the_periodic_axis(orc):
    """phi = theta node index k (a sawtooth 0..n-1 along the periodic axis,
    constant in x and y).  Multilinear interpolation between node n-1 and
    node 0 (the image of node n) across the seam: at theta = 2 pi - dth/2
    the value is (n-1)/2; at 2 pi + dth/4 (wrapped to dth/4) it is 1/4; at
    -dth/4 (wrapped to 2 pi - dth/4) it is (n-1)/4; at 6 pi + 2.5 dth it is
    2.5.  Clamping instead of wrapping would give n-1, n-1 (or 0), 0 and
    n-1."""
    spec = W.air3d(nx=[9, 8, 12])[0]
    n = spec["n"][2]
    dth = 2 * np.pi / n
    phi = np.broadcast_to(np.arange(n, dtype=np.float64), spec["n"]).copy()
    th = np.array([2 * np.pi - dth / 2, 2 * np.pi + dth / 4, -dth / 4, 6 * np.pi + 2.5 * dth])
    want = np.array([(n - 1) / 2, 0.25, (n - 1) / 4, 2.5])
    for i in range(len(th)):
        q = np.array([[3.3, -1.7, th[i]]])
        got = sum(np.sum(w * phi.ravel()[f]) for f, w in orc._interp_weights(spec, q))
        assert abs(got - want[i]) < 1e-9, (i, got, want[i])
    # the loss's query term is the sum of these values (the volume term is
    # zero for a positive field up to exp(-min phi / eps) ~ 1)
    q = np.stack([np.full(4, 3.3), np.full(4, -1.7), th], 1)
    vol = orc.loss(spec, phi + 1e3, np.zeros((0, 3)))
    assert vol < 1e-100
    assert abs(orc.loss(spec, phi + 1e3, q) - (want.sum() + 4e3)) < 1e-8


def test_query_interpolation_clamps_extrapolated_axes(orc):
    """phi = 2 x - 3 y: queries beyond the x or y range take the value at
    the nearest edge (clamped coordinates), inside they are exact."""
    spec = W.air3d(nx=[9, 8, 12])[0]
    xs = W.mesh(spec)
    phi = 2.0 * xs[0] - 3.0 * xs[1]
    q = np.array([[25.0, 1.0, 0.4], [-8.0, 1.0, 0.4], [4.0, 12.5, 1.0], [4.0, -11.0, 1.0],
                  [-7.0, -12.0, 5.0], [0.7, 0.3, 2.0]])
    want = [2 * 20 - 3, 2 * -6 - 3, 8 - 30, 8 + 30, -12 + 30, 1.4 - 0.9]
    for i in range(len(q)):
        got = sum(np.sum(w * phi.ravel()[f]) for f, w in orc._interp_weights(spec, q[i:i + 1]))
        assert abs(got - want[i]) < 1e-9, (i, got, want[i])


def test_query_gradient_scatters_the_interpolation_weights(orc):
    """The query term's gradient puts each query's 2^d weights on its 2^d
    nodes: for a far-positive field (no volume term) one query strictly
    inside a cell gives 8 entries summing to 1, one on the seam wraps onto
    theta node 0."""
    spec = W.air3d(nx=[9, 8, 12])[0]
    n = spec["n"][2]
    phi = np.full(spec["n"], 1e3)
    dth = 2 * np.pi / n
    g = orc.loss_grad(spec, phi, np.array([[3.3, -1.7, 2 * np.pi - dth / 2]]))
    nz = np.argwhere(g > 1e-12)
    assert len(nz) == 8
    assert abs(g.sum() - 1.0) < 1e-12
    assert set(nz[:, 2]) == {0, n - 1}
    np.testing.assert_allclose(g[:, :, 0].sum(), 0.5, atol=1e-12)


@pytest.mark.parametrize("scale", [0.5, 2.0])
def test_loss_is_additive_in_the_volume_and_query_terms(orc, scale):
    """loss(phi, q) = loss(phi, none) + sum_q interp(phi, q) (the two terms
    are independent), for a cylinder scaled in value."""
    spec, phi, eps = _cylinder(orc, n=41)
    rng = np.random.default_rng(20241106)
    q = np.stack([rng.uniform(spec["lo"][k], spec["hi"][k], 32) for k in range(3)], 1)
    f = scale * phi
    interp = sum(np.sum(w * f.ravel()[fl]) for fl, w in orc._interp_weights(spec, q))
    assert abs(orc.loss(spec, f, q) - orc.loss(spec, f, np.zeros((0, 3))) - interp) < 1e-9
