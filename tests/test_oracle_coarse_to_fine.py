"""Pins for the oracle's coarse-to-fine tracing (Sec. 3.2 "Coarse-to-fine
Strategy"; no GPU).

What a child ray inherits is not stated in the paper, so the agreement of the
strategy with the paper's own images is parity unpinned.  What is pinned:
the vectorised grid code against a scalar per-pixel restatement of the same
readings (each pixel traced through its chain of ancestors), the reduction to
the plain tracer with no coarse level, the closed-form depth of an exact
sphere, the convergence and silhouette invariants, and the query saving the
strategy exists for (Tab. 1).
"""

import math

import numpy as np
import pytest

import synth
from oracle import tracer
from oracle.camera import pixel_rays
from oracle.mlp import from_synth
from oracle.sdf import MLPSDF, SphereSDF

EPS, ALPHA = 5e-5, 1.5


def _mlp_sdf():
    spec = synth.DEEPSDF_SPEC
    Ws, bs = synth.make_decoder(spec, seed=0)
    Z = synth.make_latents(spec, 1)
    return MLPSDF(from_synth(Ws, bs, spec), Z)


def _scalar_ray(cam, level, X, Y):
    """Direction of coarse ray (X, Y) of level `level`, written out:
    through the image point ((X + 1/2) 2^l, (Y + 1/2) 2^l)."""
    k = 2.0 ** level
    xt = ((X + 0.5) * k - cam["cx"]) / cam["fx"]
    yt = ((Y + 0.5) * k - cam["cy"]) / cam["fy"]
    nrm = math.sqrt(xt * xt + yt * yt + 1.0)
    vc = np.array([xt, yt, 1.0]) / nrm
    v = np.asarray(cam["R"], dtype=np.float64) @ vc
    return v / np.linalg.norm(v), 1.0 / nrm


def _scalar_pixel(sdf, cam, x, y, levels, split_every, max_steps, k_min):
    """One pixel's result by tracing its ancestors one after the other."""
    c = np.asarray(cam["c"], dtype=np.float64)
    state = None
    it = 0
    for level in range(levels, -1, -1):
        v, inv = _scalar_ray(cam, level, x >> level, y >> level)
        b = float(v @ c)
        cc = float(c @ c)
        disc = b * b - (cc - 1.0)
        sq = math.sqrt(max(disc, 0.0))
        t_in, t_out = -b - sq, -b + sq
        enters = disc > 0.0 and t_out > 0.0
        if not enters:
            state = {"st": "miss", "steps": 0, "samples": [],
                     "sil": (math.sqrt(max(cc - b * b, 0.0)) if b < 0 else math.sqrt(cc)) - 1.0}
        elif state is None or state["st"] == "miss":
            state = {"st": "run", "d": t_in, "steps": 0, "samples": []}
        else:
            if it >= max_steps and state["st"] == "run":
                state["st"] = "max"          # the parent ran out of queries
            smp = [(max(a, EPS), dd, math.copysign(max(a, EPS), s))
                   for (a, dd, s) in state["samples"]]
            state = dict(state, samples=smp)
            if state["st"] in ("run", "hit"):
                d = max(state["d"], t_in)
                state.update(d=d, st="left" if d > t_out else "run")
        end = max_steps if level == 0 else min(max_steps, split_every * (levels - level + 1))
        while it < end:
            if state["st"] == "run":
                d = state["d"]
                s = float(sdf((c + d * v)[None, :], np.zeros(1, dtype=int))[0])
                state["steps"] += 1
                smp = state["samples"]
                a = abs(s)
                pos = next((j for j, q in enumerate(smp) if a < q[0]), len(smp))
                if pos < k_min:
                    smp.insert(pos, (a, d, s))
                    del smp[k_min:]
                if a < EPS:
                    state.update(st="hit", d_hit=d + s)
                else:
                    d = d + ALPHA * s
                    state["d"] = d
                    if d > t_out or d < t_in:
                        state["st"] = "left"
            it += 1
        if level > 0 and it < split_every * (levels - level + 1):
            pass   # max_steps ended inside the coarse phase
    st = state["st"]
    status = {"miss": tracer.INIT_MISS, "hit": tracer.HIT, "left": tracer.LEFT_SPHERE,
              "run": tracer.MAX_STEPS, "max": tracer.MAX_STEPS}[st]
    if st == "miss":
        sil = state["sil"]
    else:
        sil = (state["samples"][0][0] if state["samples"] else math.inf) - EPS
    depth = state["d_hit"] * inv if st == "hit" else math.inf
    return status, state["steps"], depth, sil


@pytest.mark.parametrize("k_min,max_steps", [(1, 30), (3, 30), (1, 4), (2, 2)])
def test_grid_code_matches_scalar_ancestor_chains(k_min, max_steps):
    sdf = _mlp_sdf()
    cam = synth.look_at_camera((0.3, 0.4, 2.4), 16, 16)
    out = tracer.render_coarse_to_fine(sdf, [cam], levels=2, split_every=3,
                                       max_steps=max_steps, eps=EPS, alpha=ALPHA, k_min=k_min,
                                       with_normals=False)
    for y in range(16):
        for x in range(16):
            i = y * 16 + x
            status, steps, depth, sil = _scalar_pixel(sdf, cam, x, y, 2, 3, max_steps, k_min)
            assert out["status"][i] == status, (x, y)
            assert out["steps"][i] == steps, (x, y)
            # the two compute the ray direction in a different summation
            # order (a few ulp)
            assert out["depth"][i] == pytest.approx(depth, abs=1e-12), (x, y)
            assert out["sil"][i] == pytest.approx(sil, abs=1e-12), (x, y)
    if max_steps > 6:
        assert out["mask"].sum() > 20 and (~out["mask"]).sum() > 20


def test_no_coarse_level_is_the_plain_tracer():
    sdf = _mlp_sdf()
    cam = synth.look_at_camera((0.0, 0.0, 2.5), 16, 16)
    a = tracer.render(sdf, [cam], with_normals=False, k_min=2)
    b = tracer.render_coarse_to_fine(sdf, [cam], levels=0, with_normals=False, k_min=2)
    for k in ("status", "steps", "depth", "sil", "d_hit", "topk_f", "topk_d"):
        np.testing.assert_array_equal(a[k], b[k])
    assert b["queries"] == a["steps"].sum()


def test_exact_sphere_depth_and_invariants():
    cam = synth.look_at_camera((0.2, -0.1, 2.5), 64, 64)
    sph = SphereSDF(0.6)
    out = tracer.render_coarse_to_fine(sph, [cam], eps=EPS, alpha=ALPHA, with_normals=True)
    c, v, inv = pixel_rays(cam)
    b = v @ c
    disc = b * b - (c @ c - 0.36)
    hit_true = disc > 0
    t_true = -b - np.sqrt(np.maximum(disc, 0.0))
    m = out["mask"]
    # only rays that graze the sphere may disagree with the closed form
    graze = np.abs(disc) < 0.05
    assert np.all(m[~graze] == hit_true[~graze])
    cosi = np.abs(np.einsum("ij,ij->i", out["normal"], v))
    both = m & hit_true
    err = np.abs(out["d_hit"][both] - t_true[both])
    assert np.all(err <= 1.01 * EPS / np.maximum(cosi[both], 1e-3) + 1e-12)
    # |f| < eps at every hit (the converging query is the child's own)
    assert np.all(np.abs(out["f_last"][m]) < EPS)
    assert np.array_equal(out["sil"] < 0, m)
    np.testing.assert_allclose(out["depth"][m], out["d_hit"][m] * inv[m], rtol=0, atol=0)


def test_queries_saved_and_first_iterations_coarse():
    sdf = _mlp_sdf()
    cam = synth.look_at_camera((0.0, 0.0, 2.5), 64, 64)
    plain = tracer.render(sdf, [cam], with_normals=False)
    c2f = tracer.render_coarse_to_fine(sdf, [cam], with_normals=False)
    assert c2f["queries"] < 0.8 * plain["steps"].sum()
    # three iterations on 1/16 of the rays at most, three on 1/4
    short = tracer.render_coarse_to_fine(sdf, [cam], max_steps=3, with_normals=False)
    assert short["queries"] <= 3 * 64 * 64 // 16
    mid = tracer.render_coarse_to_fine(sdf, [cam], max_steps=6, with_normals=False)
    assert mid["queries"] - short["queries"] <= 3 * 64 * 64 // 4
    assert np.all(mid["status"][mid["enters"]] != tracer.INIT_MISS)


def test_image_size_must_divide():
    cam = synth.look_at_camera((0.0, 0.0, 2.5), 18, 16)
    with pytest.raises(ValueError):
        tracer.render_coarse_to_fine(SphereSDF(0.6), [cam], levels=2)


def test_child_starts_no_earlier_than_its_own_entry():
    # a sphere just inside the bounding sphere: a ray converges on its first
    # query at its own entry point.  Where every ancestor of a pixel enters
    # the sphere no later than its child, each level converges on one query
    # only if the child is moved up to its own t_in.
    sph = SphereSDF(1.0 - 1e-5)
    cam = synth.look_at_camera((0.0, 0.0, 2.5), 32, 32)
    out = tracer.render_coarse_to_fine(sph, [cam], eps=EPS, alpha=ALPHA, with_normals=False)
    c = np.asarray(cam["c"], dtype=np.float64)

    def t_in(level, x, y):
        v, _ = _scalar_ray(cam, level, x >> level, y >> level)
        b = float(v @ c)
        disc = b * b - (float(c @ c) - 1.0)
        return -b - math.sqrt(disc) if disc > 0 else math.nan

    checked = 0
    for y in range(32):
        for x in range(32):
            t = [t_in(l, x, y) for l in (2, 1, 0)]
            if not all(np.isfinite(t)) or not (t[0] <= t[1] <= t[2]):
                continue
            i = y * 32 + x
            assert out["mask"][i] and out["steps"][i] == 3, (x, y)
            assert abs(out["d_hit"][i] - t[2]) < 2e-5
            checked += 1
    assert checked > 50
