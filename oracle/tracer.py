"""Sphere tracing of an SDF, step by step, in float64.

The algorithm follows the paper's order:

1. Initialisation (Sec. 3.2): each ray starts at its entry point into the
   unit sphere that bounds every DeepSDF shape; rays that do not meet the
   sphere are background with infinite depth.
2. Marching (Alg. 1 with the aggressive update of Sec. 3.2): query
   b = f(p), then d <- d + alpha * b, p = c + d v.
3. Convergence (Sec. 3.2 "Convergence Criteria", Sec. A.2): a ray stops when
   |f| < eps.  A ray also stops, as background, when it leaves the unit sphere
   (Sec. B.2) or when the step budget runs out (Sec. A.2: unconverged pixels
   are background).
4. Ray distance (Eq. 1): d = alpha * sum_{n<N} f(p_n) + (1 - alpha) f(p_{N-1}),
   i.e. the last query is applied as a unit step.
5. Observations (Sec. 3.3): depth z_c = d / sqrt(x~^2+y~^2+1); normal = the
   normalised SDF gradient (analytic, or the paper's central differences with
   step delta); soft silhouette = min_n |f(p_n)| - eps, and for rays that miss
   the unit sphere the distance from the origin to the ray minus 1 (Sec. A.3).

Readings where the paper is silent (each listed in the design notes):
  * the march starts at d = t_in (Eq. 1 writes the sum from the entry point);
  * |f| < eps is strict and is tested before the step; the converging query
    counts as a step; ``max_steps`` is the number of queries per ray;
  * leaving the sphere is tested on the ray distance: d > t_out or d < t_in;
  * a tangent ray (discriminant <= 0) misses the sphere;
  * ties in min |f| keep the earlier sample;
  * the distance from the origin to a ray that points away from it is |c|.

Everything is vectorised over rays; the loop is over march steps, which is
the paper's own batched "dynamic synchronized inference" (Sec. 3.2, B.2) and
gives every ray exactly the result of its own scalar loop.
"""

from __future__ import annotations

import numpy as np

from .camera import pixel_rays, depth_from_distance

INIT_MISS, HIT, LEFT_SPHERE, MAX_STEPS = 0, 1, 2, 3


def unit_sphere_init(c, v, radius=1.0):
    """Entry/exit ray distances into the bounding sphere (Sec. 3.2).

    ``c`` is (3,) or (n, 3), ``v`` (n, 3) unit directions.  Returns
    (enters (n,) bool, t_in, t_out, distance from the origin to the ray)."""
    c = np.broadcast_to(np.asarray(c, dtype=np.float64), v.shape)
    b = np.einsum("ij,ij->i", v, c)
    cc = np.einsum("ij,ij->i", c, c)
    disc = b * b - (cc - radius * radius)
    sq = np.sqrt(np.maximum(disc, 0.0))
    t_in, t_out = -b - sq, -b + sq
    enters = (disc > 0.0) & (t_out > 0.0)
    # distance from the origin to the half-line c + t v, t >= 0
    dist = np.where(b < 0.0, np.sqrt(np.maximum(cc - b * b, 0.0)), np.sqrt(cc))
    return enters, t_in, t_out, dist


def march(f, c, v, shape, t_in, t_out, enters, max_steps, eps, alpha, k_min=1,
          record=False):
    """Sphere-trace every ray (vectorised over rays, looped over steps).

    ``c`` is (3,) or (n, 3); ``f(p, shape)`` returns the SDF for points p.
    Returns a dict of per-ray arrays; with ``record`` also every sample's
    ray distance and f as (n, max_steps) arrays (NaN past the last query)."""
    n = v.shape[0]
    c = np.broadcast_to(np.asarray(c, dtype=np.float64), (n, 3))
    d = np.where(enters, t_in, 0.0).astype(np.float64)
    active = enters.copy()
    status = np.where(enters, MAX_STEPS, INIT_MISS).astype(np.int32)
    steps = np.zeros(n, dtype=np.int32)
    d_hit = np.full(n, np.inf)
    f_last = np.full(n, np.nan)
    d_last = np.full(n, np.nan)
    topk_f = np.full((n, k_min), np.inf)      # |f| of the k smallest samples
    topk_d = np.full((n, k_min), np.nan)      # their ray distances
    topk_s = np.full((n, k_min), np.nan)      # their signed f
    rec_d = np.full((n, max_steps), np.nan) if record else None
    rec_f = np.full((n, max_steps), np.nan) if record else None
    for it in range(max_steps):
        idx = np.nonzero(active)[0]
        if idx.size == 0:
            break
        p = c[idx] + d[idx, None] * v[idx]
        s = np.asarray(f(p, shape[idx]), dtype=np.float64)
        if record:
            rec_d[idx, it] = d[idx]
            rec_f[idx, it] = s
        steps[idx] += 1
        f_last[idx] = s
        d_last[idx] = d[idx]
        a = np.abs(s)
        # keep the k samples with the smallest |f|, sorted ascending; a new
        # sample goes before the first kept one it is strictly smaller than
        # (ties keep the earlier sample)
        placed = np.zeros(idx.size, dtype=bool)
        for j in range(k_min):
            ins = (~placed) & (a < topk_f[idx, j])
            bi = idx[ins]
            if bi.size:
                topk_f[bi, j + 1:] = topk_f[bi, j:-1].copy()
                topk_d[bi, j + 1:] = topk_d[bi, j:-1].copy()
                topk_s[bi, j + 1:] = topk_s[bi, j:-1].copy()
                topk_f[bi, j] = a[ins]
                topk_d[bi, j] = d[bi]
                topk_s[bi, j] = s[ins]
            placed |= ins
        conv = np.abs(s) < eps
        ci = idx[conv]
        d_hit[ci] = d[ci] + s[conv]          # unit final step (Eq. 1)
        status[ci] = HIT
        active[ci] = False
        ri = idx[~conv]
        d[ri] = d[ri] + alpha * s[~conv]     # aggressive step (Sec. 3.2)
        left = (d[ri] > t_out[ri]) | (d[ri] < t_in[ri])
        status[ri[left]] = LEFT_SPHERE
        active[ri[left]] = False
    return {
        "status": status, "steps": steps, "d_hit": d_hit, "d_end": d,
        "f_last": f_last, "d_last": d_last,
        "min_abs_f": topk_f[:, 0], "d_at_min": topk_d[:, 0], "f_at_min": topk_s[:, 0],
        "topk_f": topk_f, "topk_d": topk_d, "topk_s": topk_s,
        "rec_d": rec_d, "rec_f": rec_f,
    }


def render(sdf, cams, max_steps=50, eps=5e-5, alpha=1.5, normal_delta=0.0,
           k_min=1, radius=1.0, with_normals=True, record=False):
    """Trace all pixels of all cameras; outputs are concatenated in camera
    order, each camera's pixels row-major.  ``cam["shape"]`` selects the
    latent (the SDF's ``shape`` argument)."""
    cs, vs, invn, shapes = [], [], [], []
    for cam in cams:
        c, v, inv = pixel_rays(cam)
        n = v.shape[0]
        if float(c @ c) <= radius * radius:
            raise ValueError("camera inside the bounding sphere")
        cs.append(np.broadcast_to(c, (n, 3)))
        vs.append(v)
        invn.append(inv)
        shapes.append(np.full(n, int(cam.get("shape", 0))))
    c = np.concatenate(cs)
    v = np.concatenate(vs)
    inv_norm = np.concatenate(invn)
    shape = np.concatenate(shapes)
    enters, t_in, t_out, dist = unit_sphere_init(c, v, radius)

    out = march(sdf, c, v, shape, t_in, t_out, enters, max_steps, eps, alpha, k_min, record)
    hit = out["status"] == HIT
    depth = np.where(hit, depth_from_distance(out["d_hit"], inv_norm), np.inf)
    sil = np.where(enters, out["min_abs_f"] - eps, dist - radius)
    p_hit = c + np.where(hit, out["d_hit"], 0.0)[:, None] * v
    out.update({
        "mask": hit, "depth": depth, "sil": sil, "enters": enters,
        "t_in": t_in, "t_out": t_out, "c": c, "v": v, "inv_norm": inv_norm,
        "shape": shape, "p_hit": p_hit, "eps": eps, "alpha": alpha,
    })
    if with_normals:
        out["normal"] = normals(sdf, p_hit, shape, hit, normal_delta)
    return out


def normals(sdf, p, shape, hit, delta=0.0):
    """Unit surface normals at ``p`` for ``hit`` rays (Sec. 3.3).

    delta = 0: the normalised analytic gradient of f.
    delta > 0: the paper's central differences with step delta."""
    n = np.zeros_like(p)
    idx = np.nonzero(hit)[0]
    if idx.size == 0:
        return n
    q = p[idx]
    if delta == 0.0:
        _, g, _ = sdf.grad(q, shape[idx])
    else:
        g = np.zeros_like(q)
        for a in range(3):
            e = np.zeros(3); e[a] = delta
            g[:, a] = (sdf(q + e, shape[idx]) - sdf(q - e, shape[idx])) / (2.0 * delta)
    n[idx] = g / np.linalg.norm(g, axis=1, keepdims=True)
    return n
