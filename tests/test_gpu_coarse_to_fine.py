"""Coarse-to-fine tracing on the GPU (Sec. 3.2; dist_trace_params
coarse_levels / coarse_every) against the oracle's render_coarse_to_fine,
element by element, and the latent gradient through it.

Away from rays whose discrete decisions (of the pixel or of any of its
ancestors) sit within rounding of a threshold, the FP32 path's masks, step
counts and outcomes are identical to the oracle's and depth / silhouette are
within 1e-5; the BF16 path's depth is within 2e-3 on hits away from the
silhouette."""

import numpy as np
import pytest
import torch

import synth
from oracle import tracer
from oracle.grad import latent_vjp
from tests.helpers import (FP32_CLASS_TOL, gpu_decoder, oracle_sdf, shifted_traces, to_np,
                           workload)

pytestmark = pytest.mark.gpu


def _ambiguous(orc, tol_f, tol_d, max_steps, grazing=0.05, near_miss=0.0, budget=True):
    eps = orc["eps"]
    with np.errstate(invalid="ignore"):
        amb = np.any(np.abs(np.abs(orc["rec_f"]) - eps) < tol_f, axis=1)
    amb |= np.any(orc["rec_x"] < tol_d, axis=1)
    amb |= orc["split_x"] < max(tol_d, 1e-6)
    amb |= orc["graze"] < 1e-5
    if budget:
        amb |= orc["steps"] >= max_steps - 2
    nv = np.abs(np.einsum("ij,ij->i", orc["normal"], orc["v"]))
    amb |= orc["mask"] & (nv < grazing)
    if near_miss > 0:
        amb |= orc["enters"] & ~orc["mask"] & (orc["min_abs_f"] < near_miss)
    return amb


def _trace(cuda_device, spec, cams, n_shapes=1, seed=0, **kw):
    from paper_1911_13225_b300 import api
    Ws, bs, Z = workload(spec, seed=seed, n_shapes=n_shapes)
    dec = gpu_decoder(spec, Ws, bs)
    params = api.TraceParams(**kw)
    ws = api.Workspace(api.n_pixels(cams), params.max_steps)
    z = torch.from_numpy(Z).to(cuda_device)
    res = api.trace(dec, z, cams, params, ws)
    torch.cuda.synchronize()
    assert dec.device_error() == 0
    sdf = oracle_sdf(spec, Ws, bs, Z)
    orc = tracer.render_coarse_to_fine(
        sdf, cams, levels=params.coarse_levels, split_every=params.coarse_every,
        max_steps=params.max_steps, alpha=params.alpha, k_min=params.k_min, record=True)
    return api, dec, ws, z, params, res, orc, sdf


def _compare_fp32(res, orc, max_steps, tol_f, budget=True):
    # a short step budget ends most rays as MAX_STEPS: then only the
    # per-sample margins decide which rays are ambiguous
    ok = ~_ambiguous(orc, tol_f=tol_f, tol_d=1e-5, max_steps=max_steps, budget=budget)
    assert ok.mean() > 0.9
    mask = to_np(res.mask).astype(bool)
    assert np.array_equal(mask[ok], orc["mask"][ok])
    assert np.array_equal(to_np(res.steps)[ok], orc["steps"][ok])
    assert np.array_equal(to_np(res.status)[ok], orc["status"][ok])
    hit = ok & orc["mask"]
    assert hit.sum() > 0 or not budget
    if hit.sum():
        assert np.max(np.abs(to_np(res.depth)[hit] - orc["depth"][hit])) < 1e-5
    assert np.all(np.isinf(to_np(res.depth)[ok & ~orc["mask"]]))
    sil = to_np(res.sil)
    fin = ok & np.isfinite(orc["sil"])
    assert np.max(np.abs(sil[fin] - orc["sil"][fin])) < 1e-5
    assert np.array_equal(np.isinf(sil[ok]), np.isinf(orc["sil"][ok]))
    assert np.array_equal(sil < 0, mask)
    return ok


@pytest.mark.parametrize("levels,every", [(2, 3), (1, 3), (3, 2)])
def test_fp32_deepsdf_matches_oracle(cuda_device, levels, every):
    vps = synth.random_viewpoints(2, seed=21)
    cams = [synth.look_at_camera(vps[0], 64, 64), synth.look_at_camera(vps[1], 40, 56)]
    _, _, _, _, _, res, orc, _ = _trace(cuda_device, synth.DEEPSDF_SPEC, cams,
                                        coarse_levels=levels, coarse_every=every)
    _compare_fp32(res, orc, 50, tol_f=1e-5)
    q = to_np(res.queries)
    assert q[1] == orc["queries"] or abs(int(q[1]) - orc["queries"]) < 0.01 * orc["queries"]


@pytest.mark.parametrize("alpha,k_min,max_steps", [(1.5, 3, 50), (1.0, 1, 50), (1.5, 1, 5),
                                                    (1.5, 2, 2)])
def test_fp32_small_decoder_multi_shape(cuda_device, alpha, k_min, max_steps):
    """Small decoder, two latents, k = 3 samples; step budgets that end inside
    the coarse phase (the remaining splits run with no query left)."""
    vps = synth.random_viewpoints(2, seed=5)
    cams = [synth.look_at_camera(vps[0], 32, 32, shape=1),
            synth.look_at_camera(vps[1], 16, 24, shape=0)]
    _, _, _, _, _, res, orc, _ = _trace(cuda_device, synth.SMALL_SPEC, cams, n_shapes=2,
                                        alpha=alpha, k_min=k_min, max_steps=max_steps,
                                        coarse_levels=2)
    ok = _compare_fp32(res, orc, max_steps, tol_f=4e-6, budget=max_steps > 6)
    if max_steps <= 6:
        assert ok.mean() > 0.9
        assert np.all(to_np(res.steps) <= max_steps)
        return
    ent = ok & orc["enters"]
    dmin, fmin = to_np(res.d_min), to_np(res.f_min)
    have = np.isfinite(orc["topk_d"][ent])
    np.testing.assert_array_equal(np.isfinite(dmin[ent]), have)
    assert np.max(np.abs(dmin[ent][have] - orc["topk_d"][ent][have])) < 1e-5
    assert np.max(np.abs(fmin[ent][have] - orc["topk_s"][ent][have])) < 1e-5


@pytest.mark.parametrize("precision", ["bf16", "fp16", "fp32_tc"])
def test_tensor_core_march_depth_within_2e3(cuda_device, precision):
    cam = synth.look_at_camera(synth.random_viewpoints(1, seed=3)[0], 96, 96)
    _, _, _, _, params, res, orc, sdf = _trace(cuda_device, synth.DEEPSDF_SPEC, [cam],
                                               precision=precision, coarse_levels=2)
    # hit/miss identical away from silhouette rays at the 1e-3 |SDF| margin
    # (of the pixel or any ancestor: the shifted traces are coarse-to-fine too)
    shifted = shifted_traces(lambda f: tracer.render_coarse_to_fine(
        f, [cam], levels=2, split_every=params.coarse_every, max_steps=50, with_normals=False), sdf)
    amb = _ambiguous(orc, tol_f=FP32_CLASS_TOL, tol_d=0.0, max_steps=50, grazing=0.0)
    for o in shifted:
        amb |= (o["mask"] != orc["mask"]) | (o["steps"] >= 48)
    ok = ~amb
    mask = to_np(res.mask).astype(bool)
    assert (mask == orc["mask"]).mean() > 0.99
    assert np.array_equal(mask[ok], orc["mask"][ok])
    hit = ok & orc["mask"]
    assert hit.sum() > 100
    err = np.abs(to_np(res.depth)[hit] - orc["depth"][hit])
    assert np.max(err) < (1e-4 if precision == "fp32_tc" else 2e-3)
    assert np.array_equal(to_np(res.sil) < 0, mask)


def test_fewer_queries_than_the_plain_trace(cuda_device):
    from paper_1911_13225_b300 import api
    spec = synth.DEEPSDF_SPEC
    Ws, bs, Z = workload(spec)
    dec = gpu_decoder(spec, Ws, bs)
    cam = synth.look_at_camera((0.0, 0.3, 2.5), 128, 128)
    ws = api.Workspace(128 * 128, 50)
    z = torch.from_numpy(Z).to(cuda_device)
    q = {}
    for lv in (0, 2):
        res = api.trace(dec, z, [cam], api.TraceParams(precision="bf16", coarse_levels=lv), ws)
        q[lv] = float(to_np(res.queries).sum())
    assert q[2] < 0.75 * q[0], q


def test_latent_gradient_through_coarse_to_fine(cuda_device):
    """dist_trace_bwd on a coarse-to-fine trace: the exact implicit gradient at
    the GPU's hits against the oracle's on its own coarse-to-fine trace, with
    the same upstream gradients (zeroed on ambiguous rays): 1e-3 relative."""
    spec = synth.DEEPSDF_SPEC
    vps = synth.random_viewpoints(1, seed=11)
    cams = [synth.look_at_camera(vps[0], 48, 48, shape=0)]
    api, dec, ws, z, params, res, orc, sdf = _trace(cuda_device, spec, cams, n_shapes=2, seed=7,
                                                    max_steps=60, coarse_levels=2)
    tgt = api.trace(dec, z, [dict(cams[0], shape=1)], params, ws)
    _, gd, _, _, _ = api.loss(res, {"depth": tgt.depth}, z, ws)
    amb = _ambiguous(orc, tol_f=1e-5, tol_d=1e-5, max_steps=60, near_miss=1e-3)
    g = to_np(gd).astype(np.float64)
    g[amb] = 0.0
    dz = api.backward(dec, z, cams, params, ws, res,
                      g_depth=torch.from_numpy(g.astype(np.float32)).to(cuda_device))
    ref = latent_vjp(sdf, orc, 2, spec.latent_dim, g_depth=g.astype(np.float32).astype(np.float64))
    a = to_np(dz).astype(np.float64).ravel()
    b = ref.ravel()
    assert np.linalg.norm(b) > 0
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-3


def test_invalid_coarse_arguments(cuda_device):
    from paper_1911_13225_b300 import api
    from paper_1911_13225_b300._abi import DistError
    spec = synth.DEEPSDF_SPEC
    Ws, bs, Z = workload(spec)
    dec = gpu_decoder(spec, Ws, bs)
    ws = api.Workspace(64 * 64, 50)
    z = torch.from_numpy(Z).to(cuda_device)
    cam = synth.look_at_camera((0.0, 0.0, 2.5), 30, 32)   # 30 not a multiple of 4
    for kw in (dict(coarse_levels=2), dict(coarse_levels=5), dict(coarse_levels=1, coarse_every=0),
               dict(coarse_levels=1, precision="bf16", refine_steps=1)):
        with pytest.raises(DistError):
            c = cam if kw.get("coarse_levels") == 2 else synth.look_at_camera((0, 0, 2.5), 32, 32)
            api.trace(dec, z, [c], api.TraceParams(**kw), ws)
