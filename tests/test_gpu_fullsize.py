"""The configurations at their full sizes, in the launch configuration the
benchmark times, checked on sampled pixels that the oracle traces one ray at
a time, and by properties that hold at any size.

* 512 x 512 forward+backward (the benchmark step): BF16 and FP32 depth on
  sampled rays, BF16 vs FP32 latent gradient of the whole loss, and the
  latent gradient of the sampled pixels' depth against the oracle's;
* 256 x 256 x 5 views: FP32 and BF16 depth on sampled rays of every view;
* 32 shapes x 8 views x 224 x 224 in one call (12.8 M rays): one inverse
  optimisation step (depth + central-difference normal losses), sampled depth,
  and a finite, per-shape latent gradient."""

import numpy as np
import pytest
import torch

import synth
from oracle import tracer
from oracle.camera import pixel_rays
from oracle.grad import latent_vjp
from tests.helpers import (SDF_MARGIN, ShiftedSDF, ambiguous_rays, gpu_decoder, oracle_sdf,
                           silhouette_rays, to_np, workload)

pytestmark = pytest.mark.gpu


def _oracle_sample(sdf, cams, picks, max_steps=50, eps=5e-5, alpha=1.5, margin=True):
    """Trace the picked pixels (global indices over the concatenated cameras)
    with the oracle: a dict like tracer.render's for those rays only, and
    (margin) under "shifted" the same rays' traces of f -/+ 1e-3."""
    cs, vs, invs, shapes = [], [], [], []
    offs = np.cumsum([0] + [int(c["H"]) * int(c["W"]) for c in cams])
    for k, cam in enumerate(cams):
        sel = picks[(picks >= offs[k]) & (picks < offs[k + 1])] - offs[k]
        if sel.size == 0:
            continue
        c, v, inv = pixel_rays(cam)
        cs.append(np.broadcast_to(c, (sel.size, 3)))
        vs.append(v[sel]); invs.append(inv[sel])
        shapes.append(np.full(sel.size, int(cam.get("shape", 0))))
    c = np.concatenate(cs); v = np.concatenate(vs); inv = np.concatenate(invs)
    shape = np.concatenate(shapes)
    enters, t_in, t_out, dist = tracer.unit_sphere_init(c, v)
    out = tracer.march(sdf, c, v, shape, t_in, t_out, enters, max_steps, eps, alpha, record=True)
    hit = out["status"] == tracer.HIT
    p_hit = c + np.where(hit, out["d_hit"], 0.0)[:, None] * v
    out.update({"mask": hit, "depth": np.where(hit, out["d_hit"] * inv, np.inf),
                "enters": enters, "t_in": t_in, "t_out": t_out, "c": c, "v": v, "eps": eps,
                "alpha": alpha, "shape": shape, "inv_norm": inv, "p_hit": p_hit})
    out["normal"] = tracer.normals(sdf, p_hit, shape, hit)
    if margin:
        out["shifted"] = [tracer.march(f, c, v, shape, t_in, t_out, enters, max_steps, eps, alpha)
                          for f in (ShiftedSDF(sdf, -SDF_MARGIN), ShiftedSDF(sdf, SDF_MARGIN))]
        for o in out["shifted"]:
            o["mask"] = o["status"] == tracer.HIT
    return out


def _picks(n, k, rng):
    return np.sort(rng.choice(n, size=min(k, n), replace=False))


def _check(res, orc, picks, precision):
    mask = to_np(res.mask).astype(bool)[picks]
    depth = to_np(res.depth)[picks]
    if precision == "fp32":
        amb = ambiguous_rays(orc, tol_f=1e-5, max_steps=50, normals=orc["normal"])
        ok = ~amb
        assert np.array_equal(mask[ok], orc["mask"][ok])
        assert np.array_equal(to_np(res.steps)[picks][ok], orc["steps"][ok])
        h = ok & orc["mask"]
        assert np.max(np.abs(depth[h] - orc["depth"][h])) < 1e-5
    else:
        # hit/miss identical away from silhouette rays at the 1e-3 |SDF| margin
        ok = ~silhouette_rays(orc, orc["shifted"])
        assert np.array_equal(mask[ok], orc["mask"][ok])
        h = ok & orc["mask"]
        assert np.max(np.abs(depth[h] - orc["depth"][h])) < 2e-3
    assert (ok & orc["mask"]).sum() >= 20
    return ok


def test_benchmark_step_512(cuda_device):
    from paper_1911_13225_b300 import api
    spec = synth.DEEPSDF_SPEC
    Ws, bs, Z = workload(spec, seed=0, n_shapes=2)
    dec = gpu_decoder(spec, Ws, bs)
    cam = synth.look_at_camera(synth.random_viewpoints(5, seed=0)[0], 512, 512, shape=0)
    z = torch.from_numpy(Z).to(cuda_device)
    ws = api.Workspace(512 * 512, 50)
    p16, p32 = api.TraceParams(precision="bf16"), api.TraceParams(precision="fp32")
    tgt = api.trace(dec, z, [dict(cam, shape=1)], p16, ws).depth.clone()
    sdf = oracle_sdf(spec, Ws, bs, Z)
    rng = np.random.default_rng(0)
    fg = np.nonzero(np.isfinite(to_np(tgt)))[0]
    picks = np.unique(np.concatenate([rng.choice(fg, 250, replace=False),
                                      _picks(512 * 512, 150, rng)]))
    orc = _oracle_sample(sdf, [cam], picks)
    grads = {}
    for name, p in (("bf16", p16), ("fp32", p32)):
        res = api.trace(dec, z, [cam], p, ws)
        _check(res, orc, picks, name)
        L, gd, _, _, dz = api.loss(res, {"depth": tgt}, z, ws)
        grads[name] = (float(L), api.backward(dec, z, [cam], p, ws, res, g_depth=gd, dz=dz).clone())
    assert dec.device_error() == 0
    a, b = to_np(grads["bf16"][1]).ravel(), to_np(grads["fp32"][1]).ravel()
    assert np.linalg.norm(a - b) <= 2e-2 * np.linalg.norm(b)
    # the gradient of the sampled pixels alone (the rest of the upstream
    # gradient zeroed) against the oracle's on its trace of those rays
    ok = ~ambiguous_rays(orc, tol_f=1e-5, max_steps=50, normals=orc["normal"], near_miss=1e-3)
    gs = np.zeros(512 * 512, dtype=np.float32)
    w = np.random.default_rng(5).normal(size=picks.size).astype(np.float32)
    sel = ok & orc["mask"]
    gs[picks[sel]] = w[sel]
    g_ref = latent_vjp(sdf, orc, 2, spec.latent_dim, g_depth=np.where(sel, w, 0.0).astype(np.float64))
    # (FP32 only: a few hundred rays do not average out the BF16 adjoint's
    # per-ray rounding; the BF16 bar applies to the whole loss, above)
    for name, p, tol in (("fp32", p32, 1e-3),):
        res = api.trace(dec, z, [cam], p, ws)
        dz = api.backward(dec, z, [cam], p, ws, res, g_depth=torch.from_numpy(gs).to(cuda_device))
        a = to_np(dz).astype(np.float64).ravel()
        assert np.linalg.norm(a - g_ref.ravel()) <= tol * np.linalg.norm(g_ref), name


@pytest.mark.parametrize("precision,eps_mid,tol", [("bf16", 2e-4, 2e-2), ("bf16", 0.0, 2e-2),
                                                  ("fp32", 0.0, 1e-3)])
def test_benchmark_step_512_latent_gradient_vs_oracle(cuda_device, precision, eps_mid, tol):
    """The benchmark step's latent gradient (512 x 512, the BF16 march with
    its FP16 stage and the BF16 adjoint as timed, without the FP16 stage, or
    FP32) against the FP64 oracle on 4,000 sampled
    foreground pixels: the gradient of the sum of their depths, each ray's
    Jacobian entering with weight 1, so the per-ray rounding of the 16-bit
    adjoint averages out as it does in the benchmark's loss over ~50 K hits
    (a random-sign weighting would keep it).  Pixels on silhouette rays at
    the 1e-3 |SDF| margin are left out."""
    from paper_1911_13225_b300 import api
    spec = synth.DEEPSDF_SPEC
    Ws, bs, Z = workload(spec, seed=0, n_shapes=2)
    dec = gpu_decoder(spec, Ws, bs)
    cam = synth.look_at_camera(synth.random_viewpoints(5, seed=0)[0], 512, 512, shape=0)
    z = torch.from_numpy(Z).to(cuda_device)
    ws = api.Workspace(512 * 512, 50)
    p = api.TraceParams(precision=precision, eps_mid=eps_mid)
    res = api.trace(dec, z, [cam], p, ws)
    m = to_np(res.mask).astype(bool)
    rng = np.random.default_rng(17)
    picks = np.sort(rng.choice(np.nonzero(m)[0], 4000, replace=False))
    sdf = oracle_sdf(spec, Ws, bs, Z)
    orc = _oracle_sample(sdf, [cam], picks)
    # (a ray whose convergence test sits near eps may stop one query earlier
    # or later, which moves its hit by less than eps: no effect on the bar)
    sel = ~silhouette_rays(orc, orc["shifted"], tol_f=0.0) & orc["mask"] & m[picks]
    assert sel.sum() > 3500
    gs = np.zeros(512 * 512, dtype=np.float32)
    gs[picks[sel]] = 1.0
    dz = api.backward(dec, z, [cam], p, ws, res, g_depth=torch.from_numpy(gs).to(cuda_device))
    assert dec.device_error() == 0
    g_ref = latent_vjp(sdf, orc, 2, spec.latent_dim, g_depth=sel.astype(np.float64))
    a = to_np(dz).astype(np.float64).ravel()
    assert np.linalg.norm(g_ref) > 0
    err = np.linalg.norm(a - g_ref.ravel()) / np.linalg.norm(g_ref)
    assert err <= tol, err


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_five_views_256(cuda_device, precision):
    from paper_1911_13225_b300 import api
    spec = synth.DEEPSDF_SPEC
    Ws, bs, Z = workload(spec, seed=0, n_shapes=1)
    dec = gpu_decoder(spec, Ws, bs)
    cams = [synth.look_at_camera(vp, 256, 256) for vp in synth.random_viewpoints(5, seed=0)]
    z = torch.from_numpy(Z).to(cuda_device)
    ws = api.Workspace(api.n_pixels(cams), 50)
    res = api.trace(dec, z, cams, api.TraceParams(precision=precision), ws)
    assert dec.device_error() == 0
    rng = np.random.default_rng(1)
    n = 256 * 256
    picks = []
    for k in range(5):
        m = np.nonzero(to_np(res.mask)[k * n:(k + 1) * n])[0]
        picks.append(k * n + rng.choice(m, 60, replace=False))
        picks.append(k * n + _picks(n, 30, rng))
    picks = np.unique(np.concatenate(picks))
    orc = _oracle_sample(oracle_sdf(spec, Ws, bs, Z), cams, picks)
    _check(res, orc, picks, precision)


def test_inverse_batch_32_shapes_8_views_224(cuda_device):
    from paper_1911_13225_b300 import api
    spec = synth.DEEPSDF_SPEC
    Ws, bs, Zt = workload(spec, seed=0, n_shapes=32, latent_seed=3)
    dec = gpu_decoder(spec, Ws, bs)
    ring = synth.ring_viewpoints(8)
    cams = [synth.look_at_camera(ring[v], 224, 224, shape=s) for s in range(32) for v in range(8)]
    n = api.n_pixels(cams)
    assert n == 12_845_056
    ws = api.Workspace(n, 50)
    p = api.TraceParams(precision="bf16", normal_delta=1e-3)
    z_true = torch.from_numpy(Zt).to(cuda_device)
    tgt = api.trace(dec, z_true, cams, p, ws, normals=True)
    tgt_depth, tgt_normal = tgt.depth.clone(), tgt.normal.clone()
    z = torch.zeros_like(z_true)
    res = api.trace(dec, z, cams, p, ws, normals=True)
    L, gd, gn, _, dz = api.loss(res, {"depth": tgt_depth, "normal": tgt_normal}, z, ws,
                                w_depth=10.0, w_normal=1.0)
    dz = api.backward(dec, z, cams, p, ws, res, g_depth=gd, g_normal=gn, dz=dz)
    assert dec.device_error() == 0
    g = to_np(dz)
    assert np.all(np.isfinite(g)) and np.all(np.linalg.norm(g, axis=1) > 0)
    # the normal term is a negative dot product: between -1 and 1 per pixel
    assert np.isfinite(float(L)) and float(L) > -1.0
    # sampled depth of the mean shape (z = 0) against the oracle
    rng = np.random.default_rng(2)
    per = 224 * 224
    picks = []
    for k in rng.choice(len(cams), 12, replace=False):
        m = np.nonzero(to_np(res.mask)[k * per:(k + 1) * per])[0]
        picks.append(k * per + rng.choice(m, 10, replace=False))
    picks = np.unique(np.concatenate(picks))
    orc = _oracle_sample(oracle_sdf(spec, Ws, bs, np.zeros_like(Zt)), cams, picks)
    _check(res, orc, picks, "bf16")
