"""Inverse optimisation through the differentiable renderer (Sec. 4.2: shape
from depth by optimising the latent code with Adam, Sec. B.4), a reduced
copy of the 32-shape x 8-view x 224^2 batch: 2 shapes x 4 ring views at 48^2
in one call per Adam step, L1 depth loss, z0 = 0 (Adam lr 2e-3: the synthetic
latents are N(0, 0.01^2)).

The gradient path is the torch.autograd.Function (dist_trace_fwd /
dist_trace_bwd).  Checked: the loss falls, the recovered depth maps approach
the targets, and every Adam step's dL/dz agrees with the FP32 path's."""

import numpy as np
import pytest
import torch

import synth
from tests.helpers import gpu_decoder, to_np, workload

pytestmark = pytest.mark.gpu

SIDE = 48


def _views(n_shapes, n_views):
    vps = synth.ring_viewpoints(n_views)
    return [synth.look_at_camera(vps[v], SIDE, SIDE, shape=s)
            for s in range(n_shapes) for v in range(n_views)]


@pytest.mark.parametrize("precision", ["bf16", "fp32"])
def test_adam_recovers_depth_of_target_latents(cuda_device, precision):
    from paper_1911_13225_b300 import api
    spec = synth.DEEPSDF_SPEC
    Ws, bs, _ = workload(spec)
    dec = gpu_decoder(spec, Ws, bs)
    n_shapes, n_views = 2, 4
    cams = _views(n_shapes, n_views)
    z_true = torch.from_numpy(synth.make_latents(spec, n_shapes, seed=3)).to(cuda_device)
    params = api.TraceParams(precision=precision)
    ws = api.Workspace(api.n_pixels(cams), params.max_steps)
    with torch.no_grad():
        tgt = api.trace(dec, z_true, cams, params, ws).depth.clone()
    fg = torch.isfinite(tgt)
    assert fg.float().mean() > 0.1

    z = torch.zeros_like(z_true, requires_grad=True)
    opt = torch.optim.Adam([z], lr=2e-3)

    def l1(depth):
        m = fg & torch.isfinite(depth)
        return (depth[m] - tgt[m]).abs().mean(), m

    losses = []
    for it in range(60):
        opt.zero_grad()
        depth, sil, mask = api.render(z, dec, cams, params, ws)
        loss, _ = l1(depth)
        loss.backward()
        assert torch.isfinite(z.grad).all()
        opt.step()
        losses.append(float(loss.detach()))
    assert dec.device_error() == 0
    assert min(losses[-5:]) < 0.5 * losses[0], losses[::8]
    with torch.no_grad():
        d0 = api.trace(dec, torch.zeros_like(z_true), cams, params, ws).depth
        d1 = api.trace(dec, z.detach(), cams, params, ws).depth
    e0, _ = l1(d0)
    e1, _ = l1(d1)
    assert float(e1) < 0.5 * float(e0)


def test_bf16_latent_gradient_tracks_fp32_along_the_descent(cuda_device):
    """At several points of an Adam descent the BF16 path's dL/dz is within the
    BF16 gradient bar (2e-2 relative, l2) of the FP32 path's."""
    from paper_1911_13225_b300 import api
    spec = synth.DEEPSDF_SPEC
    Ws, bs, _ = workload(spec)
    dec = gpu_decoder(spec, Ws, bs)
    cams = _views(2, 4)
    z_true = torch.from_numpy(synth.make_latents(spec, 2, seed=3)).to(cuda_device)
    p16, p32 = api.TraceParams(precision="bf16"), api.TraceParams(precision="fp32")
    ws = api.Workspace(api.n_pixels(cams), 50)
    with torch.no_grad():
        tgt = api.trace(dec, z_true, cams, p32, ws).depth.clone()
    target = {"depth": tgt}
    z = torch.zeros_like(z_true)
    rel = []
    for it in range(8):
        grads = {}
        for name, p in (("bf16", p16), ("fp32", p32)):
            res = api.trace(dec, z, cams, p, ws)
            _, gd, _, _, dz = api.loss(res, target, z, ws)
            grads[name] = api.backward(dec, z, cams, p, ws, res, g_depth=gd, dz=dz)
        a, b = to_np(grads["bf16"]).ravel(), to_np(grads["fp32"]).ravel()
        rel.append(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))
        z = z - 2e-3 * torch.sign(grads["fp32"])
    assert dec.device_error() == 0
    assert np.median(rel) < 2e-2 and max(rel) < 5e-2, rel
