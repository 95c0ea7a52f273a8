"""Central finite differences of the 512 x 512 forward+backward workload's
loss on the DeepSDF decoder (8 x 512, latent 256, skip at layer 4): the
latent gradient that the autograd wrapper (torch.autograd.Function over
dist_trace_fwd / dist_trace_bwd) returns, in FP32 and with the BF16 march and
BF16 adjoint, against central differences with h = 1e-3 on 16 seeded latent
dimensions (Sec. 3.4 / Eq. 2: the gradient of a depth loss through the
converged sphere-tracing root; here its exact implicit form).

The loss is the L1 depth loss against a depth map rendered from a second
latent, as in the benchmark step, restricted to a set of pixels on which it
is smooth in z: the rendered foreground eroded by one pixel (no pixel
crosses the silhouette under the perturbations), without pixels within
2e-3 of the target depth (no pixel crosses the L1 kink: a 1e-3 change of one
latent entry moves the depth by ~1e-4 here).  The differences are taken on
FP32 traces converged to |f| < 1e-6 (200 queries per ray), so a difference
of two renders is the change of the root, not of where the march stopped.
The gradients come from those same traces (FP32) and from the benchmark's
own settings (|f| < 5e-5, 50 queries, alpha 1.5; FP32, and the BF16 march
with the BF16 adjoint).  Bars: relative l2 error over the 16 entries 1e-3
(FP32), 2e-3 (FP32 at eps 5e-5) and 2e-2 (BF16), against the differences
with their O(h^2) truncation error removed by Richardson's combination of
h = 1e-3 and h = 5e-4 (with h = 1e-3 alone that error is about 1e-3 here,
the size of the FP32 bar; the plain differences are checked too, the bar
widened by the measured truncation error)."""

import numpy as np
import pytest
import torch

import synth
from tests.helpers import gpu_decoder, to_np, workload

pytestmark = pytest.mark.gpu

SIZE = 512
H_FD = 1e-3


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.fixture(scope="module")
def fd_setup(cuda_device):
    from paper_1911_13225_b300 import api
    spec = synth.DEEPSDF_SPEC
    Ws, bs, Z = workload(spec, seed=0, n_shapes=2)
    dec = gpu_decoder(spec, Ws, bs)
    cam = synth.look_at_camera(synth.random_viewpoints(5, seed=0)[0], SIZE, SIZE, shape=0)
    z_all = torch.from_numpy(Z).to(cuda_device)
    ws = api.Workspace(SIZE * SIZE, 200)
    tight = api.TraceParams(max_steps=200, eps=1e-6)
    tgt = api.trace(dec, z_all, [dict(cam, shape=1)], api.TraceParams(precision="bf16"), ws)
    tgt_depth = tgt.depth.clone()
    base = api.trace(dec, z_all, [cam], tight, ws)
    m = (to_np(base.mask) > 0).reshape(SIZE, SIZE)
    er = m.copy()
    er[1:, :] &= m[:-1, :]; er[:-1, :] &= m[1:, :]; er[:, 1:] &= m[:, :-1]; er[:, :-1] &= m[:, 1:]
    er = er.reshape(-1) & np.isfinite(to_np(tgt_depth))
    with np.errstate(invalid="ignore"):
        er &= np.abs(to_np(base.depth) - to_np(tgt_depth)) > 2e-3
    assert er.sum() > 10000
    dims = np.random.default_rng(1).choice(spec.latent_dim, 16, replace=False)
    depths = {}
    keep = er.copy()
    for h in (H_FD, H_FD / 2):
        for i, j in enumerate(dims):
            for sgn in (1, -1):
                zp = z_all.clone()
                zp[0, j] += sgn * h
                r = api.trace(dec, zp, [cam], tight, ws)
                depths[h, i, sgn] = r.depth.clone()
                keep &= to_np(r.mask) > 0
    for kw in (dict(precision="fp32"), dict(precision="bf16"),
               dict(precision="bf16", eps_mid=2e-4)):      # the traces the gradients come from
        keep &= to_np(api.trace(dec, z_all, [cam], api.TraceParams(**kw), ws).mask) > 0
    keep &= to_np(base.mask) > 0
    # the mask is frozen: a pixel that any of these traces does not converge
    # on is left out of the finite differences and of the autograd loss alike
    assert keep.sum() > 0.99 * er.sum(), (int(keep.sum()), int(er.sum()))
    sel = torch.from_numpy(keep).to(cuda_device)

    def loss_of(depth):
        return float((depth[sel].double() - tgt_depth[sel].double()).abs().mean())

    def central(h):
        return np.array([(loss_of(depths[h, i, 1]) - loss_of(depths[h, i, -1])) / (2 * h)
                         for i in range(len(dims))])

    fd, fd2 = central(H_FD), central(H_FD / 2)
    # the central difference's error is h^2/6 L''' + O(h^4): the two step sizes give it
    # (fd - fd2 = 3/4 of fd's) and Richardson's combination cancels it
    rich = (4.0 * fd2 - fd) / 3.0
    return dict(api=api, dec=dec, cam=cam, z_all=z_all, ws=ws, tgt=tgt_depth, sel=sel,
                dims=dims, fd=fd, rich=rich, trunc=4.0 / 3.0 * (fd - fd2))


@pytest.mark.parametrize("precision,tight,tol,eps_mid", [("fp32", True, 1e-3, 0.0),
                                                         ("fp32", False, 2e-3, 0.0),
                                                         ("bf16", False, 2e-2, 0.0),
                                                         ("bf16", False, 2e-2, 2e-4)])
def test_latent_gradient_matches_central_differences(fd_setup, precision, tight, tol, eps_mid):
    """FP32 through the traces the differences are taken on (|f| < 1e-6):
    1e-3.  At the benchmark's settings (|f| < 5e-5) the hit points sit up to
    eps / |grad f . v| from the converged root the differences see: bar
    2e-3.  BF16 march (with and without its FP16 stage) and BF16 adjoint at
    the benchmark's settings: 2e-2.
    The bars apply to the central differences with their O(h^2) truncation
    error removed (Richardson's combination of h = 1e-3 and 5e-4); against
    the plain h = 1e-3 differences the bar is widened by that truncation
    error, which is measured, not assumed."""
    S = fd_setup
    api = S["api"]
    params = (api.TraceParams(precision=precision, max_steps=200, eps=1e-6) if tight
              else api.TraceParams(precision=precision, eps_mid=eps_mid))
    z = S["z_all"].clone().requires_grad_(True)
    depth, _, mask = api.render(z, S["dec"], [S["cam"]], params, S["ws"])
    sel = S["sel"]
    assert bool((mask[sel] > 0).all())
    loss = (depth[sel] - S["tgt"][sel]).abs().mean()
    (gz,) = torch.autograd.grad(loss, z)
    assert S["dec"].device_error() == 0
    g = to_np(gz)[0, S["dims"]].astype(np.float64)
    assert np.abs(S["fd"]).max() > 0
    trunc = _rel(S["fd"], S["rich"])
    assert trunc < 5e-3, trunc            # h = 1e-3 is small enough for the latents' scale
    err = _rel(g, S["rich"])
    assert err < tol, (precision, err, g, S["rich"])
    assert _rel(g, S["fd"]) < tol + 1.5 * trunc, (precision, _rel(g, S["fd"]), trunc)
