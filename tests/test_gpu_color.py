"""Texture re-rendering on the GPU (dist_render_color, Sec. B.1): the colour
decoder evaluated at the traced hits, against the oracle's texture network at
the same points."""

import numpy as np
import pytest
import torch

import synth
from oracle.camera import pixel_rays
from oracle.mlp import OracleDecoder
from tests.helpers import gpu_decoder, to_np, workload

pytestmark = pytest.mark.gpu


def _setup(cuda_device):
    from paper_1911_13225_b300 import api
    spec = synth.DEEPSDF_SPEC
    Ws, bs, Z = workload(spec, seed=0, n_shapes=2)
    dec = gpu_decoder(spec, Ws, bs)
    Wc, bc = synth.make_color_decoder(spec, latent_dim0=512, out_dim=3, seed=1)
    tex = api.Decoder(Wc, bc, spec.latent_dim, spec.skip, latent_dim0=512, out_dim=3)
    zt = np.random.default_rng(2).normal(0.0, 0.3, (2, 256)).astype(np.float32)
    codes = np.concatenate([Z, zt], axis=1)
    vps = synth.random_viewpoints(2, seed=9)
    cams = [synth.look_at_camera(vps[0], 48, 48, shape=0), synth.look_at_camera(vps[1], 40, 56, shape=1)]
    ws = api.Workspace(api.n_pixels(cams), 50)
    z = torch.from_numpy(Z).to(cuda_device)
    oracle = OracleDecoder(Wc, bc, spec.latent_dim, spec.skip, latent_dim0=512, out_dim=3)
    return api, dec, tex, z, torch.from_numpy(codes).to(cuda_device), codes, cams, ws, oracle


def _oracle_rgb(oracle, codes, cams, d_hit, mask):
    out, off = [], 0
    for cam in cams:
        n = int(cam["H"]) * int(cam["W"])
        c, v, _ = pixel_rays(cam)
        m = mask[off:off + n]
        rgb = np.zeros((n, 3))
        if m.any():
            P = c + d_hit[off:off + n][m, None].astype(np.float64) * v[m]
            rgb[m] = oracle(P, codes[int(cam["shape"])].astype(np.float64))
        out.append(rgb)
        off += n
    return np.concatenate(out)


@pytest.mark.parametrize("precision,tol_q99,tol_max", [("fp32", 2e-6, 2e-6), ("bf16", 1.5e-2, 4e-2),
                                                        ("fp16", 3e-3, 1e-2)])
def test_color_at_hits_matches_oracle(cuda_device, precision, tol_q99, tol_max):
    api, dec, tex, z, codes_t, codes, cams, ws, oracle = _setup(cuda_device)
    res = api.trace(dec, z, cams, api.TraceParams(precision="fp32"), ws)
    rgb = to_np(api.render_color(tex, codes_t, cams, res, ws, precision=precision))
    assert dec.device_error() == 0 and tex.device_error() == 0
    mask = to_np(res.mask).astype(bool)
    assert mask.sum() > 200
    ref = _oracle_rgb(oracle, codes, cams, to_np(res.d_hit), mask)
    assert np.all(rgb[~mask] == 0.0)
    err = np.abs(rgb[mask] - ref[mask]).ravel()
    assert np.std(ref[mask]) > 0.05          # the colours vary over the surface
    assert np.quantile(err, 0.99) < tol_q99 and err.max() < tol_max, (np.quantile(err, 0.99), err.max())


def test_color_decoder_rejected_by_tracing_and_sdf_by_color(cuda_device):
    from paper_1911_13225_b300._abi import DistError
    api, dec, tex, z, codes_t, codes, cams, ws, oracle = _setup(cuda_device)
    with pytest.raises(DistError):
        api.trace(tex, codes_t, cams, api.TraceParams(), ws)
    res = api.trace(dec, z, cams, api.TraceParams(), ws)
    with pytest.raises(DistError):
        api.render_color(dec, z, cams, res, ws)
