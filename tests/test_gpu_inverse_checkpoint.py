"""The inverse-optimisation loop (Sec. 4.2: latent codes from depth and
normal maps through the renderer, optimised with Adam; Sec. B.4: lr 1e-2,
z0 = 0) as the library runs it: dist_adam_step against the oracle's Adam,
and a checkpointed run (z, Adam moments, step count saved to .npz and
loaded into a fresh problem) that continues bit for bit like the
uninterrupted run."""

from ctypes import c_void_p

import numpy as np
import pytest
import torch

import synth
from oracle.optim import adam_step as oracle_adam
from tests.helpers import gpu_decoder, to_np, workload

pytestmark = pytest.mark.gpu


def test_adam_step_matches_oracle(cuda_device):
    from paper_1911_13225_b300.inverse import adam_step
    rng = np.random.default_rng(0)
    n = 32 * 256 + 77                      # several blocks and a ragged tail
    z0 = rng.normal(0, 0.01, n).astype(np.float32)
    z, m, v = (torch.from_numpy(a).to(cuda_device) for a in
               (z0.copy(), np.zeros(n, np.float32), np.zeros(n, np.float32)))
    zo, mo, vo = z0.astype(np.float64), np.zeros(n), np.zeros(n)
    for t in range(1, 13):
        g = (rng.normal(0, 1, n) * 10.0 ** rng.integers(-4, 1, n)).astype(np.float32)
        adam_step(z, torch.from_numpy(g).to(cuda_device), m, v, t, lr=1e-2)
        zo, mo, vo = oracle_adam(zo, g.astype(np.float64), mo, vo, t, lr=1e-2)
    torch.cuda.synchronize()
    # FP32 element-wise arithmetic: each step is within ~1e-6 of its size
    # (1e-2); the moments within FP32 rounding of their running sums, whose
    # terms reach |g| ~ 1 (m) and g^2 ~ 1 (v)
    assert np.max(np.abs(to_np(z) - zo)) < 2e-7
    np.testing.assert_allclose(to_np(m), mo, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(to_np(v), vo, rtol=1e-5, atol=1e-7)


def test_adam_step_rejects_bad_arguments(cuda_device):
    from paper_1911_13225_b300 import _abi
    x = torch.zeros(8, device=cuda_device)
    L = _abi.lib()
    p = c_void_p(x.data_ptr())
    s = c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.dist_adam_step(p, p, p, p, 8, 0, 1e-2, 0.9, 0.999, 1e-8, s) == _abi.DIST_E_INVALID
    assert L.dist_adam_step(p, p, p, p, 0, 1, 1e-2, 0.9, 0.999, 1e-8, s) == _abi.DIST_E_INVALID
    assert L.dist_adam_step(p, p, p, p, 8, 1, 1e-2, 1.0, 0.999, 1e-8, s) == _abi.DIST_E_INVALID
    assert L.dist_adam_step(None, p, p, p, 8, 1, 1e-2, 0.9, 0.999, 1e-8, s) == _abi.DIST_E_INVALID


def _problem(cuda_device, dec, cams, tgt_depth, tgt_normal, params):
    from paper_1911_13225_b300.inverse import InverseProblem
    # lr 2e-3: the synthetic latents are N(0, 0.01^2), so the paper's 1e-2
    # would overshoot them in a few steps
    return InverseProblem(dec, cams, 2, tgt_depth, tgt_normal, params=params, lr=2e-3,
                          w_depth=10.0, w_normal=1.0)


def test_checkpointed_run_resumes_bit_for_bit(cuda_device, tmp_path):
    """A reduced copy of the 32-shape x 8-view x 224^2 batch (2 shapes x 4
    ring views at 48^2, BF16 march, depth + central-difference normal
    losses): 6 Adam steps in one go against 3 steps, a checkpoint, a fresh
    problem loaded from it, and 3 more steps."""
    from paper_1911_13225_b300 import api
    spec = synth.DEEPSDF_SPEC
    Ws, bs, _ = workload(spec)
    dec = gpu_decoder(spec, Ws, bs)
    ring = synth.ring_viewpoints(4)
    cams = [synth.look_at_camera(ring[v], 48, 48, shape=s) for s in range(2) for v in range(4)]
    params = api.TraceParams(precision="bf16", normal_delta=1e-3)
    z_true = torch.from_numpy(synth.make_latents(spec, 2, seed=3)).to(cuda_device)
    ws = api.Workspace(api.n_pixels(cams), params.max_steps)
    tgt = api.trace(dec, z_true, cams, params, ws, normals=True)
    tgt_depth, tgt_normal = tgt.depth.clone(), tgt.normal.clone()

    full = _problem(cuda_device, dec, cams, tgt_depth, tgt_normal, params)
    losses = [float(full.step()) for _ in range(6)]
    ref = full.state_dict()

    first = _problem(cuda_device, dec, cams, tgt_depth, tgt_normal, params)
    for _ in range(3):
        first.step()
    path = str(tmp_path / "inverse.npz")
    first.save(path)
    resumed = _problem(cuda_device, dec, cams, tgt_depth, tgt_normal, params)
    resumed.load(path)
    assert resumed.t == 3
    for _ in range(3):
        resumed.step()
    got = resumed.state_dict()
    assert dec.device_error() == 0
    assert int(got["t"]) == 6
    for k in ("z", "m", "v"):
        np.testing.assert_array_equal(got[k], ref[k])
    assert np.all(np.isfinite(losses)) and losses[-1] < losses[0]
    # a checkpoint of a problem with other loss weights is refused
    other = _problem(cuda_device, dec, cams, tgt_depth, None,
                     api.TraceParams(precision="bf16"))
    with pytest.raises(ValueError):
        other.load(path)
