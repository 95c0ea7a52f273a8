"""Latency mode of the fused tensor-core march (dist_trace_params
latency_mode): a step whose lists fit in a few tiles is decoded with each
tile spread over a four-SM cluster.  Every output column is accumulated in
the same order and the head adds the same chunk sums in the same order as in
the one-tile-per-SM kernel, so a trace must come out bit for bit the same
with the mode on and off; on a small image every step runs in the latency
mode, and the result still meets the oracle."""

import numpy as np
import pytest
import torch

import synth
from oracle import tracer
from tests.helpers import (gpu_decoder, oracle_sdf, shifted_traces, silhouette_rays, to_np,
                           workload)

pytestmark = pytest.mark.gpu

FIELDS = ("depth", "sil", "mask", "steps", "status", "d_hit", "d_min", "f_min", "queries")


def _run(cuda_device, spec, cams, n_shapes=1, seed=0, **kw):
    from paper_1911_13225_b300 import api
    Ws, bs, Z = workload(spec, seed=seed, n_shapes=n_shapes)
    dec = gpu_decoder(spec, Ws, bs)
    z = torch.from_numpy(Z).to(cuda_device)
    out = {}
    for mode in (1, 0):
        params = api.TraceParams(latency_mode=mode, **kw)
        ws = api.Workspace(api.n_pixels(cams), params.max_steps)
        res = api.trace(dec, z, cams, params, ws)
        torch.cuda.synchronize()
        assert dec.device_error() == 0
        out[mode] = {f: to_np(getattr(res, f)) for f in FIELDS}
    return out, (Ws, bs, Z)


def _assert_identical(out):
    for f in FIELDS:
        a, b = out[1][f], out[0][f]
        assert a.dtype == b.dtype and a.shape == b.shape, f
        # bit patterns (depth holds +inf on misses, d_min / f_min NaN-free)
        assert np.array_equal(a.view(np.uint8), b.view(np.uint8)), f


def test_bitwise_same_trace_with_fp16_stage(cuda_device):
    """The BF16 march with an FP16 stage (three row lists in both decoder
    kernels): identical results with and without the latency mode."""
    vps = synth.random_viewpoints(2, seed=17)
    cams = [synth.look_at_camera(vps[0], 96, 96, shape=0),
            synth.look_at_camera(vps[1], 64, 48, shape=1)]
    out, _ = _run(cuda_device, synth.DEEPSDF_SPEC, cams, n_shapes=2, precision="bf16",
                  eps_mid=2e-4, k_min=3)
    assert out[1]["mask"].sum() > 500
    _assert_identical(out)


@pytest.mark.parametrize("precision", ["bf16", "fp16", "fp32_tc"])
@pytest.mark.parametrize("levels", [0, 2])
def test_bitwise_same_trace_with_and_without(cuda_device, precision, levels):
    """96 x 96 and 64 x 48 views of two shapes: the first steps run on the
    one-tile-per-SM kernel, the shrinking tail in the latency mode."""
    vps = synth.random_viewpoints(2, seed=17)
    cams = [synth.look_at_camera(vps[0], 96, 96, shape=0),
            synth.look_at_camera(vps[1], 64, 48, shape=1)]
    out, _ = _run(cuda_device, synth.DEEPSDF_SPEC, cams, n_shapes=2, precision=precision,
                  coarse_levels=levels, k_min=3)
    assert out[1]["mask"].sum() > 500
    _assert_identical(out)


def test_split_steps_bitwise_benchmark_view(cuda_device):
    """The 512 x 512 benchmark view with the FP16 stage: its middle steps
    (about 16..24) fit their FP32-class tiles on the latency-mode clusters
    and their 16-bit tiles on the SMs left over, so the two decoder kernels
    decode them side by side.  Identical results (query counts included:
    only one of the two kernels counts a step's queries) with the mode on
    and off."""
    spec = synth.DEEPSDF_SPEC
    cam = synth.look_at_camera(synth.random_viewpoints(5, seed=0)[0], 512, 512, shape=0)
    out, _ = _run(cuda_device, spec, [cam], n_shapes=2, precision="bf16", eps_mid=2e-4)
    assert out[1]["mask"].sum() > 40000
    _assert_identical(out)


@pytest.mark.parametrize("kw", [dict(precision="fp16", eps_bf16=2e-4),
                                dict(precision="bf16", coarse_levels=2),
                                dict(precision="bf16", eps_mid=2e-4, k_min=3)],
                         ids=["fp16", "bf16-coarse-to-fine", "bf16-fp16-stage-k3"])
def test_split_steps_bitwise_other_marches(cuda_device, kw):
    """Other marches whose middle steps the two decoder kernels may share (a
    second 512 x 512 viewpoint, two shapes in one call): identical results
    with the latency mode on and off."""
    spec = synth.DEEPSDF_SPEC
    vps = synth.random_viewpoints(5, seed=0)
    cams = [synth.look_at_camera(vps[1], 512, 512, shape=0),
            synth.look_at_camera(vps[2], 256, 256, shape=1)]
    out, _ = _run(cuda_device, spec, cams, n_shapes=2, **kw)
    assert out[1]["mask"].sum() > 20000
    _assert_identical(out)


@pytest.mark.parametrize("precision", ["bf16", "fp32_tc"])
def test_benchmark_view_bitwise(cuda_device, precision):
    """One 256 x 256 view of the benchmark's kind (its tail is where the
    latency mode takes over): identical results."""
    cam = synth.look_at_camera(synth.random_viewpoints(1, seed=2)[0], 256, 256)
    out, _ = _run(cuda_device, synth.DEEPSDF_SPEC, [cam], precision=precision)
    _assert_identical(out)


@pytest.mark.parametrize("precision", ["bf16", "fp32_tc"])
def test_small_image_all_steps_in_latency_mode(cuda_device, precision):
    """16 x 16 and 12 x 20 views (at most two tiles per step: every step in the
    latency mode, both tile kinds): bitwise the same as the one-tile-per-SM
    kernel, and the depth within 1e-4 (FP32-class) or 2e-3 (BF16 march) of
    the oracle's away from the silhouette."""
    spec = synth.DEEPSDF_SPEC
    cams = [synth.look_at_camera((0.0, 0.4, 2.2), 16, 16),
            synth.look_at_camera((1.5, -0.3, 1.6), 12, 20)]
    out, (Ws, bs, Z) = _run(cuda_device, spec, cams, precision=precision)
    _assert_identical(out)
    sdf = oracle_sdf(spec, Ws, bs, Z)
    orc = tracer.render(sdf, cams, record=True)
    shifted = shifted_traces(lambda f: tracer.render(f, cams, with_normals=False), sdf)
    # hit/miss identical away from silhouette rays at the 1e-3 |SDF| margin
    ok = ~silhouette_rays(orc, shifted)
    assert ok.mean() > 0.8
    mask = out[1]["mask"].astype(bool)
    assert np.array_equal(mask[ok], orc["mask"][ok])
    hit = ok & orc["mask"]
    assert hit.sum() > 20
    err = np.abs(out[1]["depth"][hit] - orc["depth"][hit])
    assert np.max(err) < (1e-4 if precision == "fp32_tc" else 2e-3)


def test_empty_and_single_ray_launches(cuda_device):
    """A view that misses the sphere (empty lists from the first step) and a
    1 x 1 view: the same in both modes."""
    cams = [synth.look_at_camera((0.0, 0.0, 2.5), 1, 1)]
    out, _ = _run(cuda_device, synth.DEEPSDF_SPEC, cams, precision="bf16")
    _assert_identical(out)
    away = synth.look_at_camera((0.0, 0.0, 2.5), 8, 8)
    away = dict(away)
    away["R"] = (np.asarray(away["R"]) * np.array([1.0, -1.0, -1.0])[None, :]).astype(np.float32)
    out, _ = _run(cuda_device, synth.DEEPSDF_SPEC, [away], precision="bf16")
    _assert_identical(out)


def test_invalid_latency_mode(cuda_device):
    from paper_1911_13225_b300 import api
    from paper_1911_13225_b300._abi import DistError
    spec = synth.DEEPSDF_SPEC
    Ws, bs, Z = workload(spec)
    dec = gpu_decoder(spec, Ws, bs)
    ws = api.Workspace(64, 50)
    z = torch.from_numpy(Z).to(cuda_device)
    cam = synth.look_at_camera((0.0, 0.0, 2.5), 8, 8)
    with pytest.raises(DistError):
        api.trace(dec, z, [cam], api.TraceParams(precision="bf16", latency_mode=2), ws)
