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


def _new_state(n, t_in, enters, k_min, max_steps, record):
    """Per-ray march state before the first query (Sec. 3.2 initialisation)."""
    return {
        "d": np.where(enters, t_in, 0.0).astype(np.float64),
        "active": enters.copy(),
        "status": np.where(enters, MAX_STEPS, INIT_MISS).astype(np.int32),
        "steps": np.zeros(n, dtype=np.int32),
        "d_hit": np.full(n, np.inf),
        "f_last": np.full(n, np.nan),
        "d_last": np.full(n, np.nan),
        "topk_f": np.full((n, k_min), np.inf),      # |f| of the k smallest samples
        "topk_d": np.full((n, k_min), np.nan),      # their ray distances
        "topk_s": np.full((n, k_min), np.nan),      # their signed f
        "rec_d": np.full((n, max_steps), np.nan) if record else None,
        "rec_f": np.full((n, max_steps), np.nan) if record else None,
        # distance of each step's new d from t_in / t_out (exit-test margin)
        "rec_x": np.full((n, max_steps), np.inf) if record else None,
    }


def _step(S, idx, s, it, t_in, t_out, eps, alpha):
    """One march iteration for the active rays ``idx`` with SDF values ``s``
    at their current points (Alg. 1, Sec. 3.2, Eq. 1)."""
    d = S["d"]
    if S["rec_d"] is not None:
        S["rec_d"][idx, it] = d[idx]
        S["rec_f"][idx, it] = s
    S["steps"][idx] += 1
    S["f_last"][idx] = s
    S["d_last"][idx] = d[idx]
    a = np.abs(s)
    topk_f, topk_d, topk_s = S["topk_f"], S["topk_d"], S["topk_s"]
    # keep the k samples with the smallest |f|, sorted ascending; a new
    # sample goes before the first kept one it is strictly smaller than
    # (ties keep the earlier sample)
    placed = np.zeros(idx.size, dtype=bool)
    for j in range(topk_f.shape[1]):
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
    S["d_hit"][ci] = d[ci] + s[conv]          # unit final step (Eq. 1)
    S["status"][ci] = HIT
    S["active"][ci] = False
    ri = idx[~conv]
    d[ri] = d[ri] + alpha * s[~conv]          # aggressive step (Sec. 3.2)
    left = (d[ri] > t_out[ri]) | (d[ri] < t_in[ri])
    S["status"][ri[left]] = LEFT_SPHERE
    S["active"][ri[left]] = False
    if S["rec_x"] is not None:
        S["rec_x"][ri, it] = np.minimum(np.abs(d[ri] - t_out[ri]), np.abs(d[ri] - t_in[ri]))


def _result(S):
    return {
        "status": S["status"], "steps": S["steps"], "d_hit": S["d_hit"], "d_end": S["d"],
        "f_last": S["f_last"], "d_last": S["d_last"],
        "min_abs_f": S["topk_f"][:, 0], "d_at_min": S["topk_d"][:, 0],
        "f_at_min": S["topk_s"][:, 0],
        "topk_f": S["topk_f"], "topk_d": S["topk_d"], "topk_s": S["topk_s"],
        "rec_d": S["rec_d"], "rec_f": S["rec_f"], "rec_x": S["rec_x"],
    }


def march(f, c, v, shape, t_in, t_out, enters, max_steps, eps, alpha, k_min=1,
          record=False):
    """Sphere-trace every ray (vectorised over rays, looped over steps).

    ``c`` is (3,) or (n, 3); ``f(p, shape)`` returns the SDF for points p.
    Returns a dict of per-ray arrays; with ``record`` also every sample's
    ray distance and f as (n, max_steps) arrays (NaN past the last query)."""
    n = v.shape[0]
    c = np.broadcast_to(np.asarray(c, dtype=np.float64), (n, 3))
    S = _new_state(n, t_in, enters, k_min, max_steps, record)
    for it in range(max_steps):
        idx = np.nonzero(S["active"])[0]
        if idx.size == 0:
            break
        p = c[idx] + S["d"][idx, None] * v[idx]
        s = np.asarray(f(p, shape[idx]), dtype=np.float64)
        _step(S, idx, s, it, t_in, t_out, eps, alpha)
    return _result(S)


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


# -- coarse-to-fine tracing (Sec. 3.2 "Coarse-to-fine Strategy") ---------------
#
# The trace starts on an image 2^levels times coarser per side (the paper's
# "1/4 of the resolution" read per side: two doublings after six steps reach
# full resolution) and splits every ray into its four children after every
# ``split_every`` march iterations.  The paper does not say what a child
# inherits; the readings applied here (and on the GPU) are:
#   * coarse ray (X, Y) of level l passes through the image point
#     ((X + 1/2) 2^l, (Y + 1/2) 2^l), the centre of its 2^l x 2^l pixel block;
#     its children are (2X + i, 2Y + j), i, j in {0, 1};
#   * a child has its own direction and its own unit-sphere interval; a child
#     whose ray misses the sphere is background like any such pixel;
#   * a child of a parent that missed the sphere starts afresh at its own
#     entry point;
#   * otherwise it inherits the parent's ray distance d (raised to its own
#     t_in; beyond its own t_out it has left the sphere), the parent's query
#     count, and the parent's k smallest-|f| samples with |f| floored at eps
#     (a parent's sample is not on the child's ray, so it cannot make the
#     child's silhouette negative);
#   * a child of a still-marching or converged parent marches on from d (a
#     converged parent's d is its converging sample); a child of a parent
#     that left the sphere or ran out of queries ends the same way.

def _level_camera(cam, level):
    """The camera of the 2^level-coarser image.  Scaling fx, fy, cx, cy by
    2^-level is exact in binary floating point, so pixel (X, Y) of it gives
    x~ = ((X + 1/2) 2^level - cx) / fx as on the full image."""
    k = float(2 ** level)
    return {**cam, "H": int(cam["H"]) >> level, "W": int(cam["W"]) >> level,
            "fx": cam["fx"] / k, "fy": cam["fy"] / k, "cx": cam["cx"] / k,
            "cy": cam["cy"] / k}


def _split(S, Hl, Wl, enters_c, t_in_c, t_out_c, eps, graze_c):
    """Children state of the level-l rays S (Hl x Wl, row-major): each ray's
    four children on the 2 Hl x 2 Wl grid, by the readings above."""
    def up(a):
        g = a.reshape((Hl, Wl) + a.shape[1:])
        return np.repeat(np.repeat(g, 2, axis=0), 2, axis=1).reshape((4 * Hl * Wl,) + a.shape[1:])

    n = 4 * Hl * Wl
    status_p, active_p = up(S["status"]), up(S["active"])
    d_p = up(S["d"])
    fresh = enters_c & (status_p == INIT_MISS)
    inherit = enters_c & (status_p != INIT_MISS)
    C = _new_state(n, t_in_c, enters_c, S["topk_f"].shape[1], 0, False)
    for k in ("rec_d", "rec_f", "rec_x"):
        C[k] = up(S[k]) if S[k] is not None else None
    # margins of the decisions taken here and by the ancestors (test aid):
    # entry into the bounding sphere, and the inherited d against t_out
    C["graze"] = np.minimum(up(S["graze"]), graze_c)
    C["split_x"] = up(S["split_x"]).copy()
    # inherited steps, samples and last query
    tf = up(S["topk_f"])
    C["topk_f"][inherit] = np.maximum(tf[inherit], eps)
    C["topk_s"][inherit] = np.copysign(C["topk_f"][inherit], up(S["topk_s"])[inherit])
    C["topk_d"][inherit] = up(S["topk_d"])[inherit]
    C["steps"][inherit] = up(S["steps"])[inherit]
    C["f_last"][inherit] = up(S["f_last"])[inherit]
    C["d_last"][inherit] = up(S["d_last"])[inherit]
    marching = inherit & (active_p | (status_p == HIT))
    ended = inherit & ~marching
    C["status"][ended] = status_p[ended]
    C["active"][ended] = False
    d = np.maximum(d_p, t_in_c)
    C["split_x"][marching] = np.minimum(C["split_x"][marching],
                                        np.abs(d[marching] - t_out_c[marching]))
    out = marching & (d > t_out_c)
    C["d"][marching] = d[marching]
    C["status"][marching] = MAX_STEPS
    C["active"][marching] = True
    C["status"][out] = LEFT_SPHERE
    C["active"][out] = False
    C["d"][fresh] = t_in_c[fresh]
    return C


def _graze(c, v, radius):
    """| squared distance from the origin to the ray - radius^2 |: where it is
    tiny, FP32 and FP64 may disagree on entering the bounding sphere."""
    b = v @ c
    return np.abs(float(c @ c) - b * b - radius * radius)


def render_coarse_to_fine(sdf, cams, levels=2, split_every=3, max_steps=50, eps=5e-5,
                          alpha=1.5, normal_delta=0.0, k_min=1, radius=1.0,
                          with_normals=True, record=False):
    """``render`` with the coarse-to-fine strategy of Sec. 3.2 (readings
    above).  Every camera's H and W must be multiples of 2^levels.  Returns
    the same per-pixel fields, plus ``queries``: the number of SDF queries
    made (Tab. 1 counts these).  With ``record``, each pixel's samples along
    its chain of ancestors (``rec_d``, ``rec_f``, ``rec_x``) and the margins
    of the chain's entry and split decisions (``graze``, ``split_x``)."""
    parts, queries = [], 0
    for cam in cams:
        H, W = int(cam["H"]), int(cam["W"])
        if H % (1 << levels) or W % (1 << levels):
            raise ValueError("image size not a multiple of 2^levels")
        shape_id = int(cam.get("shape", 0))
        level = levels
        c, v, inv = pixel_rays(_level_camera(cam, level))
        if float(c @ c) <= radius * radius:
            raise ValueError("camera inside the bounding sphere")
        enters, t_in, t_out, dist = unit_sphere_init(c, v, radius)
        S = _new_state(v.shape[0], t_in, enters, k_min, max_steps, record)
        S["graze"] = _graze(c, v, radius)
        S["split_x"] = np.full(v.shape[0], np.inf)
        for it in range(max_steps):
            if level > 0 and it == split_every * (levels - level + 1):
                Hl, Wl = H >> level, W >> level
                level -= 1
                c, v, inv = pixel_rays(_level_camera(cam, level))
                enters, t_in, t_out, dist = unit_sphere_init(c, v, radius)
                S = _split(S, Hl, Wl, enters, t_in, t_out, eps, _graze(c, v, radius))
            idx = np.nonzero(S["active"])[0]
            if idx.size == 0:
                if level == 0:
                    break
                continue
            p = c + S["d"][idx, None] * v[idx]
            s = np.asarray(sdf(p, np.full(idx.size, shape_id)), dtype=np.float64)
            queries += idx.size
            _step(S, idx, s, it, t_in, t_out, eps, alpha)
        while level > 0:   # max_steps shorter than the coarse phase
            # rays still marching have run out of queries (status MAX_STEPS):
            # their children end the same way
            S["active"][:] = False
            Hl, Wl = H >> level, W >> level
            level -= 1
            c, v, inv = pixel_rays(_level_camera(cam, level))
            enters, t_in, t_out, dist = unit_sphere_init(c, v, radius)
            S = _split(S, Hl, Wl, enters, t_in, t_out, eps, _graze(c, v, radius))
            S["status"][S["active"]] = MAX_STEPS
            S["active"][:] = False
        out = _result(S)
        hit = out["status"] == HIT
        out.update({
            "mask": hit, "depth": np.where(hit, depth_from_distance(out["d_hit"], inv), np.inf),
            "sil": np.where(enters, out["min_abs_f"] - eps, dist - radius),
            "enters": enters, "t_in": t_in, "t_out": t_out,
            "c": np.broadcast_to(c, v.shape), "v": v, "inv_norm": inv,
            "shape": np.full(v.shape[0], shape_id),
            "p_hit": c + np.where(hit, out["d_hit"], 0.0)[:, None] * v,
            "graze": S["graze"], "split_x": S["split_x"],
        })
        parts.append(out)
    keys = [k for k in parts[0] if parts[0][k] is not None]
    res = {k: np.concatenate([p[k] for p in parts]) for k in keys}
    res.update({"eps": eps, "alpha": alpha, "queries": queries})
    if with_normals:
        res["normal"] = normals(sdf, res["p_hit"], res["shape"], res["mask"], normal_delta)
    return res
