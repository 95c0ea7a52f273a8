"""Pins for the oracle's sphere tracer (no GPU).

Closed forms: plane contraction (Sec. A.1, Eq. 5-6), ray/sphere and ray/box
intersections, a fronto-parallel plane's constant depth (Sec. 3.3 depth
formula), the camera-derived threshold (Sec. A.2), the thin-surface hole of
aggressive marching (Sec. A.4), silhouette sign invariants (Sec. 3.3, A.3) and
a dense brute-force first-root search.
"""

import json
import math
import os

import numpy as np
import pytest

import synth
from oracle import tracer
from oracle.brute import first_root
from oracle.camera import epsilon_from_camera, pixel_rays
from oracle.mlp import from_synth
from oracle.sdf import BoxSDF, MLPSDF, PlaneSDF, SlabSDF, SphereSDF

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                   "paper_worked_numbers.json")))


def _cam(n=33, eye=(0.0, 0.0, 2.5)):
    return synth.look_at_camera(eye, n, n)


# -- worked numbers printed in the paper --------------------------------------

def test_min_steps_worked_example():
    g = GOLD["min_steps"]
    th = math.radians(g["theta_deg"])
    for alpha, key in [(1.0, "k_min_alpha_1.0"), (1.5, "k_min_alpha_1.5")]:
        kmin = (math.log(g["eps"]) - math.log(g["d"])) / math.log(abs(1 - alpha * math.sin(th)))
        assert math.ceil(kmin) == g[key]


def test_epsilon_from_camera_geometry():
    g = GOLD["epsilon_from_camera"]
    eps = epsilon_from_camera(g["d_min_m"], g["sensor_m"], g["focal_m"], g["resolution"])
    assert abs(eps - g["eps_approx"]) / g["eps_approx"] < g["eps_rel_tol"]
    # twice eps is the neighbouring-pixel spacing of Sec. 3.2
    sp = GOLD["neighbour_spacing"]["spacing_approx_m"]
    assert abs(2 * eps - sp) / sp < 0.05


# -- marching on an exact plane: geometric contraction -------------------------

@pytest.mark.parametrize("alpha", [1.0, 1.5])
@pytest.mark.parametrize("theta_deg", [10.0, 30.0, 75.0])
def test_plane_contraction_and_step_count(alpha, theta_deg):
    th = math.radians(theta_deg)
    D0, eps = 1.0, 5e-5
    v = np.array([[math.cos(th), 0.0, math.sin(th)]])
    plane = PlaneSDF(n=(0.0, 0.0, -1.0), offset=-D0 * math.sin(th))
    seen = []

    def f(p, shape):
        seen.append(p[0].copy())
        return plane(p)

    out = tracer.march(f, np.zeros(3), v, np.zeros(1, int), np.zeros(1),
                       np.full(1, 100.0), np.ones(1, bool), 10_000, eps, alpha)
    # distance along the ray to the plane after k steps is D0 (1 - alpha sin)^k
    q = 1.0 - alpha * math.sin(th)
    for k, p in enumerate(seen):
        along = D0 - float(p @ v[0])
        assert abs(along - D0 * q ** k) <= 1e-12 * max(1.0, k)
    # first k with |f_k| = D0 sin(th) |q|^k < eps, plus the converging query
    k_star = 0
    while D0 * math.sin(th) * abs(q) ** k_star >= eps:
        k_star += 1
    assert out["status"][0] == tracer.HIT
    assert out["steps"][0] == k_star + 1


def test_head_on_sphere_alpha1_converges_in_two_queries():
    cam = _cam(33)
    sph = SphereSDF(0.6)
    out = tracer.render(sph, [cam], max_steps=50, eps=5e-5, alpha=1.0)
    centre = 16 * 33 + 16                 # pixel centre on the optical axis
    assert out["steps"][centre] == 2      # f = 0.4 at entry, then ~0
    assert abs(out["depth"][centre] - 1.9) < 1e-12


# -- analytic shapes: depth vs closed-form intersections ------------------------

@pytest.mark.parametrize("alpha", [1.0, 1.5])
def test_sphere_depth_closed_form(alpha):
    r, eps = 0.6, 5e-5
    cam = _cam(33, eye=(0.3, -0.4, 2.4))
    out = tracer.render(SphereSDF(r), [cam], max_steps=200, eps=eps, alpha=alpha)
    c, v, inv = pixel_rays(cam)
    b = v @ c
    disc = b * b - (c @ c - r * r)
    exact_hit = disc > 0
    t = -b - np.sqrt(np.maximum(disc, 0))
    grazing = np.abs(np.sqrt(np.maximum(c @ c - b * b, 0)) - r) < 2e-3
    assert np.array_equal(out["mask"][~grazing], exact_hit[~grazing])
    m = out["mask"]
    cos_inc = np.sqrt(np.maximum(disc, 0)) / r
    bound = 2 * eps / np.maximum(cos_inc, 1e-3)
    assert np.all(np.abs(out["d_hit"][m] - t[m]) <= bound[m])
    assert np.all(np.abs(out["depth"][m] - t[m] * inv[m]) <= bound[m])


def test_box_depth_closed_form():
    eps = 5e-5
    half = np.array([0.4, 0.3, 0.2])
    cam = _cam(31, eye=(1.2, 0.9, 2.0))
    out = tracer.render(BoxSDF(half), [cam], max_steps=400, eps=eps, alpha=1.0,
                        with_normals=False)
    c, v, inv = pixel_rays(cam)
    with np.errstate(divide="ignore", invalid="ignore"):
        t1 = (-half - c) / v
        t2 = (half - c) / v
    tn = np.minimum(t1, t2).max(axis=1)
    tf = np.maximum(t1, t2).min(axis=1)
    exact_hit = (tn <= tf) & (tf > 0)
    # which face is entered, and how obliquely
    face = np.argmax(np.minimum(t1, t2), axis=1)
    cos_inc = np.abs(v[np.arange(len(v)), face])
    margin = tf - tn                      # short chords are near an edge
    clear = (~exact_hit) | ((margin > 0.05) & (cos_inc > 0.1))
    m = out["mask"]
    assert np.array_equal(m[clear & exact_hit], exact_hit[clear & exact_hit])
    sel = m & clear
    assert sel.sum() > 50
    assert np.all(np.abs(out["d_hit"][sel] - tn[sel]) <= 2 * eps / cos_inc[sel])


def test_fronto_parallel_plane_constant_depth():
    eps = 5e-5
    cam = _cam(25)
    out = tracer.render(PlaneSDF(n=(0, 0, 1), offset=0.0), [cam], max_steps=200,
                        eps=eps, alpha=1.5, with_normals=False)
    m = out["mask"]
    assert m.sum() > 100
    assert np.all(np.abs(out["depth"][m] - 2.5) < eps)


def test_thin_slab_hole_with_aggressive_marching():
    cam = _cam(33)
    slab = SlabSDF(n=(0, 0, 1), offset=0.0, half_thickness=1e-3)
    centre = 16 * 33 + 16
    o1 = tracer.render(slab, [cam], max_steps=100, alpha=1.0, with_normals=False)
    o15 = tracer.render(slab, [cam], max_steps=100, alpha=1.5, with_normals=False)
    assert o1["mask"][centre] and abs(o1["depth"][centre] - (2.5 - 1e-3)) < 1e-9
    assert not o15["mask"][centre]       # stepped over both faces (Sec. A.4)
    assert o15["status"][centre] == tracer.LEFT_SPHERE


# -- silhouette -----------------------------------------------------------------

def test_silhouette_sign_and_init_miss_value():
    spec = synth.SMALL_SPEC
    Ws, bs = synth.make_decoder(spec, seed=0)
    Z = synth.make_latents(spec, 1)
    sdf = MLPSDF(from_synth(Ws, bs, spec), Z)
    cam = _cam(32)
    out = tracer.render(sdf, [cam], max_steps=50)
    assert np.array_equal(out["sil"] < 0, out["mask"])
    c, v, _ = pixel_rays(cam)
    b = v @ c
    miss = ~out["enters"]
    assert miss.sum() > 0
    np.testing.assert_allclose(out["sil"][miss], np.sqrt(c @ c - b[miss] ** 2) - 1.0,
                               rtol=0, atol=1e-14)
    assert np.all(out["sil"][miss] > 0)
    assert np.all(np.isinf(out["depth"][~out["mask"]]))


# -- brute force first root ------------------------------------------------------

def test_alpha1_finds_first_root_analytic():
    # union of a sphere and a box (exact SDF outside both: min of exact SDFs)
    sph, box = SphereSDF(0.35, (0.3, 0.0, 0.0)), BoxSDF((0.2, 0.45, 0.2))
    f = lambda p, s=None: np.minimum(sph(p), box(p + np.array([0.35, 0.0, 0.0])))
    cam = _cam(16, eye=(0.5, 0.6, 2.3))
    out = tracer.render(f, [cam], max_steps=400, eps=1e-7, alpha=1.0, with_normals=False)
    root = first_root(f, out["c"], out["v"], out["shape"], out["t_in"], out["t_out"],
                      out["enters"], step=2e-4)
    both = out["mask"] & np.isfinite(root)
    assert both.sum() > 20
    assert np.max(np.abs(out["d_hit"][both] - root[both])) < 1e-4
    # a traced miss has no root, except grazing rays the step budget cut off
    assert np.sum(out["mask"] != np.isfinite(root)) <= 2


def test_mlp_hits_land_on_a_root():
    spec = synth.DEEPSDF_SPEC
    Ws, bs = synth.make_decoder(spec, seed=0)
    Z = synth.make_latents(spec, 1)
    dec = from_synth(Ws, bs, spec)
    sdf = MLPSDF(dec, Z)
    cam = _cam(16)
    for alpha in (1.0, 1.5):
        out = tracer.render(sdf, [cam], max_steps=100, alpha=alpha, with_normals=False)
        m = out["mask"]
        assert m.sum() > 10
        f_hit = sdf(out["p_hit"][m], out["shape"][m])
        assert np.all(np.abs(f_hit) < 2 * out["eps"])
        if alpha == 1.0:
            root = first_root(sdf, out["c"], out["v"], out["shape"], out["t_in"],
                              out["t_out"], out["enters"], step=5e-3)
            ok = np.isfinite(root) & m
            # never past the first root (the decoder is close to 1-Lipschitz)
            assert np.all(out["d_hit"][ok] <= root[ok] + 1e-6)
            # and on it, except near-tangent rays that reach |f| < eps early
            _, g, _ = sdf.grad(out["p_hit"][ok], out["shape"][ok])
            cos_inc = np.abs(np.einsum("ij,ij->i", g, out["v"][ok])) / np.linalg.norm(g, axis=1)
            steep = cos_inc > 0.3
            assert steep.sum() > 20
            assert np.all(np.abs(out["d_hit"][ok][steep] - root[ok][steep]) < 1e-4)
