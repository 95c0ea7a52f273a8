"""Analytic signed distance functions used to pin the tracer.

Each SDF is callable as ``f(p, shape)`` -> (n,) and offers ``grad(p, shape)``
-> (f, df/dp, df/dtheta) where theta is the SDF's own parameter vector (it
plays the role of the latent code z in gradient pins).
"""

from __future__ import annotations

import numpy as np


class SphereSDF:
    """f(p) = |p - centre| - r.  Parameters theta = [r, cx, cy, cz]."""

    def __init__(self, r=0.6, centre=(0.0, 0.0, 0.0)):
        self.theta = np.array([r, *centre], dtype=np.float64)

    def __call__(self, p, shape=None):
        q = np.atleast_2d(p) - self.theta[1:]
        return np.linalg.norm(q, axis=1) - self.theta[0]

    def grad(self, p, shape=None):
        q = np.atleast_2d(p) - self.theta[1:]
        nq = np.linalg.norm(q, axis=1)
        f = nq - self.theta[0]
        gp = q / nq[:, None]
        gth = np.concatenate([-np.ones((len(f), 1)), -gp], axis=1)
        return f, gp, gth


class BoxSDF:
    """Exact SDF of an axis-aligned box with half extents ``b``
    (Quilez's published formula: |max(q,0)| + min(max(q_x,q_y,q_z),0), q = |p|-b)."""

    def __init__(self, b=(0.4, 0.3, 0.2)):
        self.b = np.asarray(b, dtype=np.float64)

    def __call__(self, p, shape=None):
        q = np.abs(np.atleast_2d(p)) - self.b
        outside = np.linalg.norm(np.maximum(q, 0.0), axis=1)
        inside = np.minimum(q.max(axis=1), 0.0)
        return outside + inside


class PlaneSDF:
    """f(p) = n . p - offset, with unit normal n."""

    def __init__(self, n=(0.0, 0.0, 1.0), offset=0.0):
        n = np.asarray(n, dtype=np.float64)
        self.n = n / np.linalg.norm(n)
        self.offset = float(offset)

    def __call__(self, p, shape=None):
        return np.atleast_2d(p) @ self.n - self.offset


class SlabSDF:
    """Thin slab |n . p - offset| - half_thickness (exact SDF)."""

    def __init__(self, n=(0.0, 0.0, 1.0), offset=0.0, half_thickness=1e-3):
        n = np.asarray(n, dtype=np.float64)
        self.n = n / np.linalg.norm(n)
        self.offset = float(offset)
        self.h = float(half_thickness)

    def __call__(self, p, shape=None):
        return np.abs(np.atleast_2d(p) @ self.n - self.offset) - self.h


class MLPSDF:
    """The decoder evaluated with latent ``Z[shape]`` for each point."""

    def __init__(self, decoder, Z):
        self.dec = decoder
        self.Z = np.atleast_2d(np.asarray(Z, dtype=np.float64))

    def __call__(self, p, shape):
        return self.dec.forward(p, self.Z[np.asarray(shape)])

    def grad(self, p, shape):
        return self.dec.grad(p, self.Z[np.asarray(shape)])
