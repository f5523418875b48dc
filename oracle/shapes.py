"""Implicit surfaces for the oracle (TEST INFRASTRUCTURE ONLY): plain FP64
numpy definitions of the signed-distance primitives of Sec. III-C and the
calculus on implicit functions of Sec. III-D, evaluated at the grid nodes
(coordinates lo + i dx, the oracle's grid of Sec. III-B).

Each primitive measures distance in the dimensions not listed in `ignore`
(extruding the shape along the ignored ones); periodic axes are not wrapped.
"""
from __future__ import annotations

import numpy as np

from . import nodes


def _coords(spec):
    return np.meshgrid(*[nodes(spec, k) for k in range(spec["ndim"])], indexing="ij")


def _used(spec, ignore):
    return [k for k in range(spec["ndim"]) if k not in set(ignore)]


def sphere(spec, center, radius, ignore=()):
    """Sec. III-C: the signed distance |x - c| - r (negative inside)."""
    xs = _coords(spec)
    q = sum((xs[k] - center[k]) ** 2 for k in _used(spec, ignore))
    return np.sqrt(q) - radius


def box(spec, lo, hi, ignore=()):
    """Signed distance to the axis-aligned box [lo, hi]: outside, the distance
    to the nearest point of the box (the node clamped into it); inside, minus
    the distance to the nearest face."""
    xs = _coords(spec)
    used = _used(spec, ignore)
    out2 = sum((xs[k] - np.clip(xs[k], lo[k], hi[k])) ** 2 for k in used)
    inside_depth = np.min([np.minimum(xs[k] - lo[k], hi[k] - xs[k]) for k in used], axis=0)
    return np.where(out2 > 0, np.sqrt(out2), -inside_depth)


def quadric(spec, center, weights, offset, ignore=()):
    """The ellipsoid form of Sec. III-C: sum_k w_k (x_k - c_k)^2 - offset."""
    xs = _coords(spec)
    return sum(weights[k] * (xs[k] - center[k]) ** 2 for k in _used(spec, ignore)) - offset


def halfspace(spec, normal, point, ignore=()):
    """Signed distance to the plane through `point` with normal `normal`,
    negative on the side the normal points away from."""
    xs = _coords(spec)
    used = _used(spec, ignore)
    nrm = np.sqrt(sum(normal[k] ** 2 for k in used))
    return sum(normal[k] * (xs[k] - point[k]) for k in used) / nrm


def union(a, b):
    """Sec. III-D: interior of either shape, min(a, b)."""
    return np.minimum(a, b)


def intersect(a, b):
    """Sec. III-D: interior of both shapes, max(a, b)."""
    return np.maximum(a, b)


def complement(a):
    """Sec. III-D: the complement, -a."""
    return -np.asarray(a)


def difference(a, b):
    """Sec. III-D: the interior of a outside b, max(a, -b)."""
    return np.maximum(a, -np.asarray(b))
