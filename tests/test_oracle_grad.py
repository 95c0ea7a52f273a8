"""Pins for the oracle's latent gradients and losses (no GPU).

* exact depth gradient vs the closed-form derivative of a ray/sphere
  intersection with respect to radius and centre;
* exact depth gradient of the full traced L1 depth loss vs central finite
  differences of the whole oracle pipeline (tight eps, frozen mask);
* the paper's first-term gradient (Eq. 2, Sec. 3.4) and the silhouette
  gradient (Sec. A.3) on an SDF whose df/dr is -1 everywhere;
* the central-difference normal's vector-Jacobian product vs finite
  differences with the hit points held fixed;
* loss values on hand-made arrays (Sec. A.3 Eq. 4, Sec. B.3).
"""

import numpy as np
import pytest

import synth
from oracle import tracer
from oracle.camera import pixel_rays
from oracle.grad import latent_vjp
from oracle.loss import loss_terms, regulariser
from oracle.mlp import from_synth
from oracle.sdf import MLPSDF, SphereSDF


class _SphereLatent(SphereSDF):
    """Sphere whose parameter vector [r, cx, cy, cz] plays the latent."""


def test_exact_depth_grad_sphere_closed_form():
    r, C = 0.55, np.array([0.05, -0.1, 0.08])
    sdf = _SphereLatent(r, C)
    cam = synth.look_at_camera((0.4, 0.3, 2.3), 21, 21)
    out = tracer.render(sdf, [cam], max_steps=300, eps=1e-12, alpha=1.0)
    c, v, inv = pixel_rays(cam)
    m = out["mask"]
    for i in np.nonzero(m)[0][::7]:
        g = np.zeros(len(m)); g[i] = 1.0
        G = latent_vjp(sdf, out, 1, 4, g_depth=g, mode="exact")[0]
        oc = c - C
        b = v[i] @ oc
        disc = b * b - oc @ oc + r * r
        dt_dr = -r / np.sqrt(disc)
        dt_dC = v[i] + (b * v[i] - oc) / np.sqrt(disc)
        expect = inv[i] * np.concatenate([[dt_dr], dt_dC])
        np.testing.assert_allclose(G, expect, rtol=1e-7, atol=1e-10)


def test_exact_loss_grad_vs_finite_differences_small_mlp():
    spec = synth.SMALL_SPEC
    Ws, bs = synth.make_decoder(spec, seed=1)
    dec = from_synth(Ws, bs, spec)
    Z = synth.make_latents(spec, 2, seed=1).astype(np.float64)
    cam = synth.look_at_camera((0.3, 0.5, 2.4), 20, 20)
    kw = dict(max_steps=3000, eps=1e-12, alpha=1.5, with_normals=False)
    tgt = tracer.render(MLPSDF(dec, Z[1:2]), [cam], **kw)
    z0 = Z[0].copy()
    base = tracer.render(MLPSDF(dec, z0[None]), [cam], **kw)
    _, gd, _, _ = loss_terms(base, {"depth": tgt["depth"]})
    G = latent_vjp(MLPSDF(dec, z0[None]), base, 1, spec.latent_dim, g_depth=gd)[0]
    h = 1e-6
    dims = np.random.default_rng(0).choice(spec.latent_dim, 16, replace=False)
    M0 = base["mask"] & np.isfinite(tgt["depth"])
    fd = []
    for j in dims:
        vals = []
        for sgn in (1, -1):
            z = z0.copy(); z[j] += sgn * h
            o = tracer.render(MLPSDF(dec, z[None]), [cam], **kw)
            assert np.array_equal(o["mask"][M0], base["mask"][M0])
            vals.append(np.abs(o["depth"][M0] - tgt["depth"][M0]).sum() / M0.sum())
        fd.append((vals[0] - vals[1]) / (2 * h))
    fd = np.array(fd)
    an = G[dims]
    assert np.linalg.norm(an - fd) <= 1e-4 * np.linalg.norm(fd)


def test_paper_mode_first_term_on_sphere():
    # df/dr = -1 at every point, so the first-term gradient of Eq. 2 summed
    # over the K smallest-|f| samples is -alpha * K along the ray.
    sdf = _SphereLatent(0.6)
    cam = synth.look_at_camera((0.0, 0.0, 2.5), 15, 15)
    for K in (1, 3):
        out = tracer.render(sdf, [cam], max_steps=50, eps=5e-5, alpha=1.5, k_min=K)
        m = out["mask"] & (out["steps"] >= K)
        i = np.nonzero(m)[0][len(np.nonzero(m)[0]) // 2]
        g = np.zeros(len(m)); g[i] = 1.0
        G = latent_vjp(sdf, out, 1, 4, g_depth=g, mode="paper")[0]
        assert abs(G[0] - out["inv_norm"][i] * (-1.5 * K)) < 1e-12


def test_silhouette_grad_on_sphere():
    sdf = _SphereLatent(0.6)
    cam = synth.look_at_camera((0.0, 0.0, 2.5), 31, 31)
    out = tracer.render(sdf, [cam], max_steps=50)
    miss_in = out["enters"] & ~out["mask"]
    assert miss_in.sum() > 10
    g = miss_in.astype(float)
    G = latent_vjp(sdf, out, 1, 4, g_sil=g)[0]
    # S = (distance from the centre to the ray) - r - eps for a miss: dS/dr = -1
    assert abs(G[0] - (-miss_in.sum())) < 1e-12


def test_fd_normal_vjp_vs_finite_differences():
    spec = synth.SMALL_SPEC
    Ws, bs = synth.make_decoder(spec, seed=2)
    dec = from_synth(Ws, bs, spec)
    z0 = synth.make_latents(spec, 1, seed=2)[0].astype(np.float64)
    cam = synth.look_at_camera((0.2, -0.3, 2.5), 12, 12)
    delta = 1e-3
    out = tracer.render(MLPSDF(dec, z0[None]), [cam], max_steps=100, normal_delta=delta)
    m = out["mask"]
    rng = np.random.default_rng(3)
    n_gt = rng.standard_normal((len(m), 3))
    n_gt /= np.linalg.norm(n_gt, axis=1, keepdims=True)
    _, _, gn, _ = loss_terms(out, {"depth": out["depth"], "normal": n_gt},
                             w_depth=0.0, w_normal=1.0)
    G = latent_vjp(MLPSDF(dec, z0[None]), out, 1, spec.latent_dim, g_normal=gn,
                   normal_delta=delta)[0]

    def Ln(z):
        nrm = tracer.normals(MLPSDF(dec, z[None]), out["p_hit"], out["shape"], m, delta)
        return -(np.einsum("ij,ij->i", nrm, n_gt)[m]).sum() / m.sum()

    h = 1e-6
    for j in [0, 5, 33, 63]:
        e = np.zeros_like(z0); e[j] = h
        fd = (Ln(z0 + e) - Ln(z0 - e)) / (2 * h)
        assert abs(G[j] - fd) <= 1e-6 * max(1.0, abs(fd))


def test_loss_values_hand_arrays():
    out = {
        "depth": np.array([1.0, 2.0, np.inf, 1.5]),
        "mask": np.array([True, True, False, True]),
        "sil": np.array([-0.1, -0.2, 0.3, -0.05]),
        "normal": np.array([[0, 0, 1.0], [0, 1.0, 0], [0, 0, 0], [1.0, 0, 0]]),
    }
    tgt = {
        "depth": np.array([1.5, 1.0, 2.0, np.inf]),
        "normal": np.array([[0, 0, 1.0], [0, 0, 1.0], [0, 0, 1.0], [0, 0, 1.0]]),
        "sil": np.array([1.0, 0.0, 1.0, 1.0]),
    }
    L, gd, gn, gs = loss_terms(out, tgt, w_depth=1.0)
    assert L == pytest.approx((0.5 + 1.0) / 2)          # pixels 0,1 in the region
    np.testing.assert_array_equal(gd, [-0.5, 0.5, 0.0, 0.0])
    L, _, gn, _ = loss_terms(out, tgt, w_depth=0.0, w_normal=1.0)
    assert L == pytest.approx(-(1.0 + 0.0) / 2)
    L, _, _, gs = loss_terms(out, tgt, w_depth=0.0, w_sil=1.0)
    # S_gt max(0,S) + (1 - S_gt) max(0,-S): 0, 0.2, 0.3, 0
    assert L == pytest.approx(0.5 / 4)
    np.testing.assert_allclose(gs, [0.0, -0.25, 0.25, 0.0])
    R, gR = regulariser(np.array([[1.0, -2.0]]), 0.5)
    assert R == pytest.approx(2.5) and np.allclose(gR, [[1.0, -2.0]])
