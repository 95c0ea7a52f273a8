"""Dense fixed-step first-root search along each ray (float64).

Used to pin the tracer: for a 1-Lipschitz SDF, classic sphere tracing
(alpha = 1, Alg. 1) never steps over a root, so it must stop at the first
zero crossing along the ray inside the bounding sphere.  This search walks
[t_in, t_out] with a fixed step, takes the first sign change from + to -
(or an exact zero), and bisects it to ``tol``.
"""

from __future__ import annotations

import numpy as np


def first_root(f, c, v, shape, t_in, t_out, enters, step=1e-4, tol=1e-12):
    """Return the first root distance per ray (inf where none is found)."""
    n = v.shape[0]
    c = np.broadcast_to(np.asarray(c, dtype=np.float64), (n, 3))
    root = np.full(n, np.inf)
    for i in np.nonzero(enters)[0]:
        ts = np.arange(t_in[i], t_out[i] + step, step)
        ts[-1] = min(ts[-1], t_out[i])
        vals = f(c[i] + ts[:, None] * v[i], np.full(ts.size, shape[i]))
        cross = np.nonzero((vals[:-1] > 0.0) & (vals[1:] <= 0.0))[0]
        if vals[0] <= 0.0:
            root[i] = ts[0]
            continue
        if cross.size == 0:
            continue
        lo, hi = ts[cross[0]], ts[cross[0] + 1]
        while hi - lo > tol:
            mid = 0.5 * (lo + hi)
            if f((c[i] + mid * v[i])[None], np.array([shape[i]]))[0] > 0.0:
                lo = mid
            else:
                hi = mid
        root[i] = 0.5 * (lo + hi)
    return root
