"""Pins for the oracle's camera-extrinsic gradients (no GPU).

The camera enters every ray through its centre c and the direction
v = R v_cam / |R v_cam|.  Pinned:

* depth: the implicit derivative at the traced hit against the closed-form
  derivative of a ray/sphere intersection with respect to c and the nine
  entries of R (R treated as a free matrix, v renormalised);
* depth: the full traced L1 depth loss of an MLP shape against central
  finite differences of the whole oracle pipeline in c and R (tight eps,
  frozen mask);
* silhouette of rays that miss the bounding sphere: the exact derivative of
  the distance from the origin to the ray (Sec. A.3) against central
  differences of that distance;
* silhouette of rays that enter: the first-term rule (sample distance held
  fixed) against central differences of |f| at the moving sample point.
"""

import numpy as np

import synth
from oracle import tracer
from oracle.camera import pixel_rays
from oracle.grad import camera_vjp
from oracle.loss import loss_terms
from oracle.mlp import from_synth
from oracle.sdf import MLPSDF, SphereSDF


def _with(cam, c=None, R=None):
    out = dict(cam)
    if c is not None:
        out["c"] = np.asarray(c, dtype=np.float64)
    if R is not None:
        out["R"] = np.asarray(R, dtype=np.float64)
    return out


def _sphere_depth(cam, r, C):
    """Closed-form first intersection depth (inf on misses) per pixel."""
    c, v, inv = pixel_rays(cam)
    oc = c - C
    b = v @ oc
    disc = b * b - oc @ oc + r * r
    t = -b - np.sqrt(np.maximum(disc, 0.0))
    return np.where(disc > 0, t * inv, np.inf)


def test_depth_grad_sphere_closed_form():
    r, C = 0.55, np.array([0.05, -0.1, 0.08])
    sdf = SphereSDF(r, C)
    cam = synth.look_at_camera((0.4, 0.3, 2.3), 17, 17)
    cam = _with(cam, c=cam["c"], R=cam["R"])
    out = tracer.render(sdf, [cam], max_steps=300, eps=1e-12, alpha=1.0, with_normals=False)
    m = out["mask"]
    rng = np.random.default_rng(3)
    g = np.where(m, rng.normal(size=m.size), 0.0)
    # keep away from the silhouette: the closed form must stay a hit
    b = out["v"] @ (np.asarray(cam["c"]) - C)
    disc = b * b - (np.asarray(cam["c"]) - C) @ (np.asarray(cam["c"]) - C) + r * r
    g[disc < 0.02] = 0.0
    Gc, GR = camera_vjp(sdf, out, [cam], g_depth=g)
    h = 1e-6
    L = lambda cm: float(np.sum(np.where(g != 0, _sphere_depth(cm, r, C), 0.0) * g))
    fd_c = np.zeros(3)
    for a in range(3):
        e = np.zeros(3); e[a] = h
        fd_c[a] = (L(_with(cam, c=cam["c"] + e)) - L(_with(cam, c=cam["c"] - e))) / (2 * h)
    fd_R = np.zeros((3, 3))
    for a in range(3):
        for bb in range(3):
            E = np.zeros((3, 3)); E[a, bb] = h
            fd_R[a, bb] = (L(_with(cam, R=cam["R"] + E)) - L(_with(cam, R=cam["R"] - E))) / (2 * h)
    np.testing.assert_allclose(Gc[0], fd_c, rtol=1e-5, atol=1e-6 * np.abs(fd_c).max())
    np.testing.assert_allclose(GR[0], fd_R, rtol=1e-5, atol=1e-6 * np.abs(fd_R).max())


def test_init_miss_silhouette_grad():
    cam = synth.look_at_camera((0.2, 0.1, 2.5), 24, 24)
    sdf = SphereSDF(0.6)
    out = tracer.render(sdf, [cam], max_steps=50, with_normals=False)
    miss = ~out["enters"]
    assert miss.sum() > 20
    rng = np.random.default_rng(4)
    g = np.where(miss, rng.normal(size=miss.size), 0.0)
    Gc, GR = camera_vjp(sdf, out, [cam], g_sil=g)

    def L(cm):
        c, v, _ = pixel_rays(cm)
        b = v @ c
        cc = c @ c
        dist = np.where(b < 0, np.sqrt(np.maximum(cc - b * b, 0)), np.sqrt(cc))
        return float(np.sum(g * (dist - 1.0)))
    h = 1e-6
    for a in range(3):
        e = np.zeros(3); e[a] = h
        fd = (L(_with(cam, c=cam["c"] + e)) - L(_with(cam, c=cam["c"] - e))) / (2 * h)
        assert abs(Gc[0, a] - fd) <= 1e-6 * max(1.0, abs(fd))
    for a in range(3):
        for bb in range(3):
            E = np.zeros((3, 3)); E[a, bb] = h
            fd = (L(_with(cam, R=cam["R"] + E)) - L(_with(cam, R=cam["R"] - E))) / (2 * h)
            assert abs(GR[0, a, bb] - fd) <= 1e-6 * max(1.0, abs(fd))


def test_entering_silhouette_first_term():
    spec = synth.SMALL_SPEC
    Ws, bs = synth.make_decoder(spec, seed=2)
    sdf = MLPSDF(from_synth(Ws, bs, spec), synth.make_latents(spec, 1, seed=2))
    cam = synth.look_at_camera((0.3, -0.4, 2.4), 16, 16)
    out = tracer.render(sdf, [cam], max_steps=60, with_normals=False)
    ent = out["enters"] & ~out["mask"]
    assert ent.sum() > 10
    rng = np.random.default_rng(5)
    g = np.where(ent, rng.normal(size=ent.size), 0.0)
    Gc, GR = camera_vjp(sdf, out, [cam], g_sil=g)
    dmin = out["d_at_min"]

    def L(cm):
        # |f| at the fixed sample distances along the moved rays
        c, v, _ = pixel_rays(cm)
        idx = np.nonzero(g != 0)[0]
        p = c + dmin[idx, None] * v[idx]
        f = sdf(p, np.zeros(idx.size, dtype=int))
        return float(np.sum(g[idx] * np.abs(f)))
    h = 1e-6
    for a in range(3):
        e = np.zeros(3); e[a] = h
        fd = (L(_with(cam, c=cam["c"] + e)) - L(_with(cam, c=cam["c"] - e))) / (2 * h)
        assert abs(Gc[0, a] - fd) <= 1e-5 * max(1.0, abs(fd))
    E = np.zeros((3, 3)); E[1, 2] = h
    fd = (L(_with(cam, R=cam["R"] + E)) - L(_with(cam, R=cam["R"] - E))) / (2 * h)
    assert abs(GR[0, 1, 2] - fd) <= 1e-5 * max(1.0, abs(fd))


def test_depth_loss_grad_vs_finite_differences_mlp():
    spec = synth.SMALL_SPEC
    Ws, bs = synth.make_decoder(spec, seed=1)
    dec = from_synth(Ws, bs, spec)
    Z = synth.make_latents(spec, 1, seed=1).astype(np.float64)
    sdf = MLPSDF(dec, Z)
    cam = synth.look_at_camera((0.3, 0.5, 2.4), 20, 20)
    tcam = _with(cam, c=np.asarray(cam["c"]) + np.array([0.03, -0.02, 0.01]))
    kw = dict(max_steps=3000, eps=1e-12, alpha=1.5, with_normals=False)
    tgt = tracer.render(sdf, [tcam], **kw)
    base = tracer.render(sdf, [cam], **kw)
    _, gd, _, _ = loss_terms(base, {"depth": tgt["depth"]})
    Gc, GR = camera_vjp(sdf, base, [cam], g_depth=gd)
    M0 = base["mask"] & np.isfinite(tgt["depth"])
    h = 1e-6

    def L(cm):
        o = tracer.render(sdf, [cm], **kw)
        assert np.array_equal(o["mask"][M0], base["mask"][M0])
        return np.abs(o["depth"][M0] - tgt["depth"][M0]).sum() / M0.sum()
    fd, an = [], []
    for a in range(3):
        e = np.zeros(3); e[a] = h
        fd.append((L(_with(cam, c=cam["c"] + e)) - L(_with(cam, c=cam["c"] - e))) / (2 * h))
        an.append(Gc[0, a])
    for (a, bb) in [(0, 0), (1, 2), (2, 1)]:
        E = np.zeros((3, 3)); E[a, bb] = h
        fd.append((L(_with(cam, R=cam["R"] + E)) - L(_with(cam, R=cam["R"] - E))) / (2 * h))
        an.append(GR[0, a, bb])
    fd, an = np.array(fd), np.array(an)
    assert np.linalg.norm(an - fd) <= 1e-4 * np.linalg.norm(fd), (an, fd)
