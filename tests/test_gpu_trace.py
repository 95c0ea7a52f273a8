"""FP32 CUDA sphere tracer vs the FP64 oracle, element by element
(dist_trace_fwd / dist_render_normals through the C ABI).

Away from rays whose discrete decisions sit within rounding of a threshold
(tests/helpers.ambiguous_rays), masks, step counts and outcome codes must be
identical and depth / silhouette within 1e-5 in scene units."""

import functools

import numpy as np
import pytest
import torch

import synth
from oracle import tracer
from tests.helpers import (ambiguous_rays, gpu_decoder, oracle_sdf, shifted_traces,
                           silhouette_rays, to_np, workload)

pytestmark = pytest.mark.gpu

DEPTH_TOL = 1e-5


def _run(cuda_device, spec, cams, n_shapes=1, alpha=1.5, max_steps=50, k_min=1, seed=0,
         normals=False, delta=0.0, precision="fp32"):
    from paper_1911_13225_b300 import api
    Ws, bs, Z = workload(spec, seed=seed, n_shapes=n_shapes)
    dec = gpu_decoder(spec, Ws, bs)
    n = api.n_pixels(cams)
    ws = api.Workspace(n, max_steps)
    params = api.TraceParams(max_steps=max_steps, alpha=alpha, k_min=k_min, normal_delta=delta,
                             precision=precision)
    res = api.trace(dec, torch.from_numpy(Z).to(cuda_device), cams, params, ws, normals=normals)
    torch.cuda.synchronize()
    sdf = oracle_sdf(spec, Ws, bs, Z)
    orc = tracer.render(sdf, cams, max_steps=max_steps, alpha=alpha, k_min=k_min,
                        with_normals=True, record=True)
    return res, orc, sdf


def _compare(res, orc, max_steps, tol_f, tol_d=1e-5, depth_tol=DEPTH_TOL, min_ok=0.9,
             step_slack=0):
    amb = ambiguous_rays(orc, tol_f=tol_f, tol_d=tol_d, max_steps=max_steps,
                         normals=orc["normal"])
    ok = ~amb
    assert ok.mean() > min_ok, f"too many ambiguous rays: {amb.mean():.3f}"
    mask = to_np(res.mask).astype(bool)
    assert np.array_equal(mask[ok], orc["mask"][ok])
    if step_slack == 0:
        assert np.array_equal(to_np(res.steps)[ok], orc["steps"][ok])
    else:
        ds = np.abs(to_np(res.steps)[ok].astype(np.int64) - orc["steps"][ok])
        assert np.max(ds) <= step_slack and np.mean(ds > 0) < 0.01
    assert np.array_equal(to_np(res.status)[ok], orc["status"][ok])
    hit = ok & orc["mask"]
    assert hit.sum() > 0
    assert np.max(np.abs(to_np(res.depth)[hit] - orc["depth"][hit])) < depth_tol
    assert np.all(np.isinf(to_np(res.depth)[ok & ~orc["mask"]]))
    assert np.max(np.abs(to_np(res.sil)[ok] - orc["sil"][ok])) < depth_tol
    # invariant on every ray: S < 0 <=> hit
    assert np.array_equal(to_np(res.sil) < 0, mask)
    return ok


@pytest.mark.parametrize("alpha", [1.5, 1.0])
def test_small_decoder_32x32(cuda_device, alpha):
    cam = synth.look_at_camera((0, 0, 2.5), 32, 32)
    res, orc, _ = _run(cuda_device, synth.SMALL_SPEC, [cam], alpha=alpha)
    _compare(res, orc, 50, tol_f=4e-6)


def test_deepsdf_decoder_ragged_tiles(cuda_device):
    cam = synth.look_at_camera(synth.random_viewpoints(1, seed=3)[0], 45, 37)
    res, orc, _ = _run(cuda_device, synth.DEEPSDF_SPEC, [cam])
    _compare(res, orc, 50, tol_f=1e-5)


# FP32-class tensor-core queries (two-term FP16 split): f within ~2e-6 of the
# FP64 decoder (the tensor core's FP32 accumulation truncates), so over ~20
# steps of 1.5 f the sample positions drift by up to ~6e-5 from the oracle's;
# the exit and convergence margins and the depth bar are set from that
# (depth 1e-4 = 2 eps), not from the FP32 CUDA-core bar.  A drifted sample
# can meet |f| < eps one step earlier or later than the oracle's: step counts
# may differ by one on at most 1% of the rays.
FP32TC = dict(tol_f=2e-5, tol_d=6e-5, depth_tol=1e-4, min_ok=0.75, step_slack=1)


@pytest.mark.parametrize("alpha", [1.5, 1.0])
def test_deepsdf_fp32_tc_trace(cuda_device, alpha):
    vps = synth.random_viewpoints(2, seed=11)
    cams = [synth.look_at_camera(vps[0], 64, 64), synth.look_at_camera(vps[1], 33, 50),
            synth.look_at_camera(synth.random_viewpoints(1, seed=3)[0], 45, 37)]
    res, orc, _ = _run(cuda_device, synth.DEEPSDF_SPEC, cams, alpha=alpha, precision="fp32_tc")
    _compare(res, orc, 50, **FP32TC)


def test_multi_camera_multi_shape_topk(cuda_device):
    vps = synth.random_viewpoints(3, seed=5)
    cams = [synth.look_at_camera(vps[0], 24, 20, shape=1),
            synth.look_at_camera(vps[1], 16, 16, shape=0),
            synth.look_at_camera(vps[2], 9, 31, shape=1)]
    res, orc, _ = _run(cuda_device, synth.SMALL_SPEC, cams, n_shapes=2, k_min=3)
    ok = _compare(res, orc, 50, tol_f=4e-6)
    dmin, fmin = to_np(res.d_min), to_np(res.f_min)
    ent = ok & orc["enters"]
    have = np.isfinite(orc["topk_d"][ent])
    np.testing.assert_array_equal(np.isfinite(dmin[ent]), have)
    assert np.max(np.abs(dmin[ent][have] - orc["topk_d"][ent][have])) < DEPTH_TOL
    assert np.max(np.abs(fmin[ent][have] - orc["topk_s"][ent][have])) < DEPTH_TOL


@pytest.mark.parametrize("delta,precision", [(0.0, "fp32"), (1e-3, "fp32"), (1e-3, "bf16"),
                                             (1e-3, "fp32_tc")])
def test_normals_at_gpu_hits(cuda_device, delta, precision):
    """Normals at the GPU's hits against the oracle's at the same points:
    analytic (FP32 adjoint) or the paper's central differences with step
    delta, whose queries are FP32 (CUDA cores) or FP32-class (tensor cores,
    after a tensor-core march)."""
    cam = synth.look_at_camera((0.4, 0.7, 2.3), 40, 40)
    spec = synth.DEEPSDF_SPEC
    res, orc, sdf = _run(cuda_device, spec, [cam], normals=True, delta=delta, precision=precision)
    m = to_np(res.mask).astype(bool)
    c, v = orc["c"], orc["v"]
    p = c[m] + to_np(res.d_hit)[m].astype(np.float64)[:, None] * v[m]
    n_ref = tracer.normals(sdf, p, orc["shape"][m], np.ones(m.sum(), bool), delta)
    err = np.linalg.norm(to_np(res.normal)[m] - n_ref, axis=1)
    tol = 1e-4 if delta == 0.0 else 3e-3
    assert np.quantile(err, 0.99) < tol and np.max(err) < 10 * tol
    assert np.all(to_np(res.normal)[~m] == 0)


@functools.lru_cache(maxsize=None)
def _oracle_view(size, vp_seed):
    """The oracle's trace of the DeepSDF decoder (seed 0) from viewpoint
    vp_seed, and its traces shifted by -1e-3 and +1e-3 (cached: every
    precision mode compares against the same oracle)."""
    spec = synth.DEEPSDF_SPEC
    Ws, bs, Z = workload(spec, seed=0, n_shapes=1)
    cam = synth.look_at_camera(synth.random_viewpoints(1, seed=vp_seed)[0], size, size)
    sdf = oracle_sdf(spec, Ws, bs, Z)
    orc = tracer.render(sdf, [cam], record=True)
    return orc, shifted_traces(lambda f: tracer.render(f, [cam], with_normals=False), sdf)


@pytest.mark.parametrize("precision,eps_lo,refine,alpha_r,engine,rule", [
    ("bf16", 1e-3, 0, 0.0, "tc", "march"), ("fp16", 1e-3, 0, 0.0, "tc", "march"),
    ("fp16", 1e-4, 1, 0.0, "tc", "march"), ("fp16", 2e-4, 1, 0.0, "tc", "march"),
    ("bf16", 1e-3, 0, 1.0, "tc", "march"), ("bf16", 3e-4, 0, 1.0, "tc", "march"),
    ("fp16", 1e-4, 1, 1.0, "tc", "march"), ("bf16", 1e-3, 0, 0.0, "simt", "march"),
    ("fp16", 1e-4, 1, 0.0, "simt", "march"), ("bf16", 1e-3, 0, 0.0, "tc", "secant"),
    ("fp16", 1e-3, 0, 0.0, "tc", "secant"), ("bf16", 3e-3, 0, 0.0, "tc", "secant"),
    ("bf16", 1e-3, 0, 0.0, "simt", "secant")])
@pytest.mark.parametrize("size,vp_seed", [(64, 3), (96, 8)])
def test_tensor_core_trace_depth_within_2e3(cuda_device, size, vp_seed, precision, eps_lo, refine,
                                            alpha_r, engine, rule):
    """Tensor-core marching (BF16 or FP16 operands) until |f| < eps_lo, then
    FP32-class queries (tensor-core split or CUDA-core FP32; aggressive or
    secant steps): converge to eps = 5e-5 (refine = 0) or accept after
    `refine` FP32 queries within 4 eps_lo (unit final step).  Depth within
    2e-3 of the FP64 oracle on hits away from the silhouette; masks agree
    except on silhouette rays at the 1e-3 |SDF| margin."""
    from paper_1911_13225_b300 import api
    spec = synth.DEEPSDF_SPEC
    Ws, bs, Z = workload(spec, seed=0, n_shapes=1)
    dec = gpu_decoder(spec, Ws, bs)
    cam = synth.look_at_camera(synth.random_viewpoints(1, seed=vp_seed)[0], size, size)
    ws = api.Workspace(size * size, 50)
    params = api.TraceParams(precision=precision, eps_bf16=eps_lo, refine_steps=refine,
                             alpha_refine=alpha_r, refine_engine=engine, refine_rule=rule)
    res = api.trace(dec, torch.from_numpy(Z).to(cuda_device), [cam], params, ws)
    assert dec.device_error() == 0
    orc, shifted = _oracle_view(size, vp_seed)
    # 16-bit queries move the march's samples, so hit/miss may differ only on
    # silhouette rays at the 1e-3 |SDF| margin (tests/helpers.silhouette_rays);
    # everywhere else the masks are identical
    ok = ~silhouette_rays(orc, shifted)
    assert ok.mean() > 0.9
    mask = to_np(res.mask).astype(bool)
    assert (mask == orc["mask"]).mean() > 0.99
    assert np.array_equal(mask[ok], orc["mask"][ok])
    hit = ok & orc["mask"]
    assert hit.sum() > 100
    err = np.abs(to_np(res.depth)[hit] - orc["depth"][hit])
    assert np.max(err) < 2e-3
    assert np.array_equal(to_np(res.sil) < 0, mask)
    q = to_np(res.queries)
    assert q[0] > 0 and q[1] > 0


@pytest.mark.parametrize("eps_mid", [2e-4, 4e-4])
@pytest.mark.parametrize("size,vp_seed", [(64, 3), (96, 8)])
def test_bf16_march_with_fp16_stage(cuda_device, size, vp_seed, eps_mid):
    """BF16 march, FP16 queries once the BF16 |f| < 1e-3, FP32-class
    queries once the FP16 |f| < eps_mid, convergence at eps = 5e-5: the same
    bars as the two-stage march (masks bit-exact away from the silhouette
    rays at the 1e-3 |SDF| margin, depth within 2e-3), with fewer
    FP32-class queries than without the FP16 stage."""
    from paper_1911_13225_b300 import api
    spec = synth.DEEPSDF_SPEC
    Ws, bs, Z = workload(spec, seed=0, n_shapes=1)
    dec = gpu_decoder(spec, Ws, bs)
    cam = synth.look_at_camera(synth.random_viewpoints(1, seed=vp_seed)[0], size, size)
    ws = api.Workspace(size * size, 50)
    z = torch.from_numpy(Z).to(cuda_device)
    res = api.trace(dec, z, [cam], api.TraceParams(precision="bf16", eps_mid=eps_mid), ws)
    two = api.trace(dec, z, [cam], api.TraceParams(precision="bf16"), ws)
    assert dec.device_error() == 0
    orc, shifted = _oracle_view(size, vp_seed)
    ok = ~silhouette_rays(orc, shifted)
    mask = to_np(res.mask).astype(bool)
    assert np.array_equal(mask[ok], orc["mask"][ok])
    hit = ok & orc["mask"]
    assert hit.sum() > 100
    assert np.max(np.abs(to_np(res.depth)[hit] - orc["depth"][hit])) < 2e-3
    assert np.array_equal(to_np(res.sil) < 0, mask)
    q, q2 = to_np(res.queries), to_np(two.queries)
    assert q[1] < q2[1], (q, q2)


def test_fp16_stage_arguments(cuda_device):
    from paper_1911_13225_b300 import api
    from paper_1911_13225_b300._abi import DistError
    spec = synth.DEEPSDF_SPEC
    Ws, bs, Z = workload(spec)
    dec = gpu_decoder(spec, Ws, bs)
    ws = api.Workspace(64 * 64, 50)
    z = torch.from_numpy(Z).to(cuda_device)
    cam = synth.look_at_camera((0.0, 0.0, 2.5), 64, 64)
    for kw in (dict(eps_mid=1e-3), dict(eps_mid=2e-3), dict(eps_mid=-1e-4),
               dict(eps_mid=2e-4, coarse_levels=2), dict(eps_mid=2e-4, refine_steps=1),
               dict(eps_mid=2e-4, refine_engine="simt"), dict(eps_mid=2e-4, refine_rule="secant")):
        with pytest.raises(DistError):
            api.trace(dec, z, [cam], api.TraceParams(precision="bf16", **kw), ws)
    # other precisions ignore it
    api.trace(dec, z, [cam], api.TraceParams(precision="fp16", eps_mid=2e-4), ws)
    assert dec.device_error() == 0


def test_all_rays_miss_the_sphere(cuda_device):
    from paper_1911_13225_b300 import api
    spec = synth.SMALL_SPEC
    Ws, bs, Z = workload(spec)
    dec = gpu_decoder(spec, Ws, bs)
    cam = synth.look_at_camera((0, 0, 2.5), 8, 8)
    cam["R"] = -cam["R"]            # looking away from the origin
    cam["R"][:, 0] *= -1            # keep a proper rotation
    ws = api.Workspace(64)
    res = api.trace(dec, torch.from_numpy(Z).to(cuda_device), [cam], api.TraceParams(), ws)
    torch.cuda.synchronize()
    assert not to_np(res.mask).any()
    assert np.all(np.isinf(to_np(res.depth)))
    assert np.all(to_np(res.sil) > 0)
    assert np.all(to_np(res.steps) == 0)
    assert int(res.queries.sum()) == 0


def test_one_pixel_and_invalid_arguments(cuda_device):
    from paper_1911_13225_b300 import api
    from paper_1911_13225_b300._abi import DistError, DIST_E_INVALID
    spec = synth.SMALL_SPEC
    Ws, bs, Z = workload(spec)
    dec = gpu_decoder(spec, Ws, bs)
    ws = api.Workspace(16, 50)
    z = torch.from_numpy(Z).to(cuda_device)
    cam = synth.look_at_camera((0, 0, 2.5), 1, 1)
    res = api.trace(dec, z, [cam], api.TraceParams(), ws)
    torch.cuda.synchronize()
    orc = tracer.render(oracle_sdf(spec, Ws, bs, Z), [cam], with_normals=False)
    assert bool(to_np(res.mask)[0]) == bool(orc["mask"][0])
    inside = synth.look_at_camera((0, 0, 0.5), 4, 4)
    with pytest.raises(DistError) as e:
        api.trace(dec, z, [inside], api.TraceParams(), ws)
    assert e.value.status == DIST_E_INVALID
    with pytest.raises(DistError):
        api.trace(dec, z, [cam], api.TraceParams(k_min=4), ws)
    with pytest.raises(DistError):
        api.trace(dec, z, [synth.look_at_camera((0, 0, 2.5), 5, 5)], api.TraceParams(), ws)
    with pytest.raises(DistError):
        api.trace(dec, z, [cam], api.TraceParams(max_steps=51), ws)
    bad_shape = dict(cam, shape=3)
    with pytest.raises(DistError):
        api.trace(dec, z, [bad_shape], api.TraceParams(), ws)
