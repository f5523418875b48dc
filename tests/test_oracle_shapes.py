"""Pins of the oracle's implicit surfaces (Sec. III-C, III-D) against brute
force and geometry: distances to densely sampled surfaces, invariance along
ignored dimensions and along a plane, exact zeros on nodes that lie on a
surface, and the set-operation truth tables of the signs."""
import numpy as np
import pytest

from oracle import shapes as S
from paper_2411_03501_gb300 import workloads as W


def _grid3(n=(13, 11, 9)):
    return W.problem(3, list(n), [-2.0, -1.5, -1.0], [2.0, 1.5, 1.0], [False, False, False],
                     "eno2", "normal_speed", [1.0])


def _nodes(spec):
    import oracle
    xs = np.meshgrid(*[oracle.nodes(spec, k) for k in range(spec["ndim"])], indexing="ij")
    return np.stack([x.ravel() for x in xs], 1)


def test_sphere_is_the_distance_to_sampled_surface():
    spec = _grid3()
    c, r = np.array([0.3, -0.2, 0.1]), 0.8
    phi = S.sphere(spec, c, r).ravel()
    u, v = np.meshgrid(np.linspace(0, np.pi, 181), np.linspace(0, 2 * np.pi, 361), indexing="ij")
    surf = c + r * np.stack([np.sin(u) * np.cos(v), np.sin(u) * np.sin(v), np.cos(u)], -1).reshape(-1, 3)
    X = _nodes(spec)
    dist = np.sqrt(((X[:, None, :] - surf[None, :, :]) ** 2).sum(-1)).min(1)
    inside = ((X - c) ** 2).sum(1) < r * r
    brute = np.where(inside, -dist, dist)
    assert np.abs(phi - brute).max() < 0.02  # sampling step r * pi / 180


def test_cylinder_ignores_its_axis():
    spec = _grid3()
    phi = S.sphere(spec, [0.1, 0.2, 99.0], 0.5, ignore=(2,))
    assert np.array_equal(phi, np.repeat(phi[:, :, :1], spec["n"][2], axis=2))
    x0 = np.linspace(-2, 2, 13)[:, None]
    y0 = np.linspace(-1.5, 1.5, 11)[None, :]
    np.testing.assert_allclose(phi[:, :, 0], np.hypot(x0 - 0.1, y0 - 0.2) - 0.5, atol=1e-15)


def test_box_is_the_distance_to_sampled_surface():
    spec = _grid3((15, 13, 11))
    lo, hi = np.array([-0.7, -0.4, -0.5]), np.array([0.9, 0.6, 0.3])
    phi = S.box(spec, lo, hi).ravel()
    t = np.linspace(0, 1, 81)
    faces = []
    for k in range(3):
        a, b = [j for j in range(3) if j != k]
        A, Bv = np.meshgrid(lo[a] + t * (hi[a] - lo[a]), lo[b] + t * (hi[b] - lo[b]), indexing="ij")
        for side in (lo[k], hi[k]):
            P = np.zeros(A.shape + (3,))
            P[..., k] = side
            P[..., a] = A
            P[..., b] = Bv
            faces.append(P.reshape(-1, 3))
    surf = np.concatenate(faces)
    X = _nodes(spec)
    dist = np.sqrt(((X[:, None, :] - surf[None, :, :]) ** 2).sum(-1)).min(1)
    inside = np.all((X > lo) & (X < hi), axis=1)
    brute = np.where(inside, -dist, dist)
    assert np.abs(phi - brute).max() < 0.02


def test_quadric_zero_on_the_paper_ellipsoid():
    """The ellipsoid of Sec. III-C, x^2 + 4 y^2 + 9 z^2 - r: zero at the
    nodes (+-sqrt r, 0, 0) and (0, +-sqrt(r)/2, 0), negative at the centre,
    and equal to the weighted sum at every node."""
    spec = W.problem(3, [9, 9, 7], [-1, -0.5, -1 / 3], [1, 0.5, 1 / 3], [False] * 3, "eno2",
                     "normal_speed", [1.0])
    q = S.quadric(spec, [0, 0, 0], [1, 4, 9], 1.0)
    assert q[0, 4, 3] == 0.0 and q[8, 4, 3] == 0.0
    assert q[4, 0, 3] == 0.0 and q[4, 8, 3] == 0.0
    assert abs(q[4, 4, 0]) < 1e-15
    assert q[4, 4, 3] == -1.0


def test_halfspace_geometry():
    spec = _grid3()
    n, p = np.array([1.0, -2.0, 0.5]), np.array([0.2, 0.1, -0.3])
    phi = S.halfspace(spec, n, p).ravel()
    X = _nodes(spec)
    # moving along the unit normal by s changes the value by s; moving
    # within the plane does not
    u = n / np.linalg.norm(n)
    foot = X - phi[:, None] * u
    np.testing.assert_allclose((foot - p) @ n, 0.0, atol=1e-12)
    assert np.all(np.sign(phi) == np.sign((X - p) @ n))
    ax = S.halfspace(spec, [0, 1, 0], [0, 0.25, 0])
    np.testing.assert_allclose(ax, np.broadcast_to(np.linspace(-1.5, 1.5, 11)[None, :, None] - 0.25,
                                                   ax.shape), atol=1e-15)


def test_set_operations_truth_tables():
    """Sec. III-D: union = min, intersection = max, complement = -phi,
    difference = max(a, -b), read off the signs of two overlapping spheres."""
    spec = _grid3((21, 17, 15))
    a = S.sphere(spec, [-0.4, 0, 0], 0.9)
    b = S.sphere(spec, [0.5, 0.1, 0], 0.8)
    ina, inb = a < 0, b < 0
    assert np.array_equal(S.union(a, b) < 0, ina | inb)
    assert np.array_equal(S.intersect(a, b) < 0, ina & inb)
    assert np.array_equal(S.complement(a) < 0, a > 0)
    assert np.array_equal(S.difference(a, b) < 0, ina & (b > 0))
    assert (ina & inb).any() and (ina & ~inb).any()
