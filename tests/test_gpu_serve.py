"""Continuous-batching server (dist_serve_*): mixed render and
render+backward requests of several sizes and latents give the same results
in the mix as alone and as dist_trace_fwd / the backward entry points;
admission errors are reported."""

import numpy as np
import pytest
import torch

import synth
from tests.helpers import gpu_decoder, to_np, workload

pytestmark = pytest.mark.gpu


def _requests(spec, n_req, seed=0):
    rng = np.random.default_rng(seed)
    Z = synth.make_latents(spec, n_req + 1, seed=seed + 1)
    vps = synth.random_viewpoints(n_req, seed=seed + 2)
    reqs = []
    for i in range(n_req):
        s = int(rng.choice([16, 24, 32, 48]))
        cam = synth.look_at_camera(vps[i], s, s)
        kind = "backward" if rng.random() < 0.3 else "render"
        reqs.append((cam, Z[i], kind))
    return reqs, Z[-1]


def _target(api, dec, cam, z_tgt, ws, params, dev):
    z = torch.from_numpy(z_tgt[None]).to(dev)
    return to_np(api.trace(dec, z, [dict(cam, shape=0)], params, ws).depth)


@pytest.mark.parametrize("precision,latency_mode,eps_mid", [("fp32", 1, 0.0), ("bf16", 1, 0.0),
                                                           ("bf16", 0, 0.0), ("bf16", 1, 2e-4)])
def test_mixed_load_equals_alone_and_direct_calls(cuda_device, precision, latency_mode, eps_mid):
    """(With latency_mode 0 the server decodes every step one tile per SM, the
    direct calls use the default latency mode: the results still agree bit
    for bit.  eps_mid: the BF16 march with its FP16 stage, in the server and
    in the direct calls.)"""
    from paper_1911_13225_b300 import api
    from paper_1911_13225_b300.serve import Server
    spec = synth.DEEPSDF_SPEC if precision == "bf16" else synth.SMALL_SPEC
    Ws, bs, _ = workload(spec)
    dec = gpu_decoder(spec, Ws, bs)
    params = api.TraceParams(precision=precision, eps_mid=eps_mid)
    srv_params = api.TraceParams(precision=precision, latency_mode=latency_mode, eps_mid=eps_mid)
    reqs, z_tgt = _requests(spec, 12)
    ws = api.Workspace(48 * 48, 50)
    tgts = [_target(api, dec, c, z_tgt, ws, params, cuda_device) if k == "backward" else None
            for c, _, k in reqs]
    srv = Server(dec, srv_params, max_rays=8192, mem_budget=1 << 30, max_requests=8)
    # all at once: requests join and leave the running batch
    mixed = [srv.submit(c, z, k, t) for (c, z, k), t in zip(reqs, tgts)]
    for t in mixed:
        srv.wait(t)
    # one at a time
    alone = []
    for (c, z, k), t in zip(reqs, tgts):
        alone.append(srv.wait(srv.submit(c, z, k, t)))
    srv.close()
    for (cam, z, kind), a, b, tgt in zip(reqs, mixed, alone, tgts):
        np.testing.assert_array_equal(a.depth, b.depth)
        np.testing.assert_array_equal(a.sil, b.sil)
        np.testing.assert_array_equal(a.mask, b.mask)
        # and the same as the direct entry points
        zt = torch.from_numpy(z[None]).to(cuda_device)
        ref = api.trace(dec, zt, [dict(cam, shape=0)], params, ws)
        np.testing.assert_array_equal(a.depth, to_np(ref.depth))
        np.testing.assert_array_equal(a.mask, to_np(ref.mask))
        if kind == "backward":
            L, gd, _, _, dz = api.loss(ref, {"depth": torch.from_numpy(tgt).to(cuda_device)}, zt, ws)
            dz = api.backward(dec, zt, [dict(cam, shape=0)], params, ws, ref, g_depth=gd, dz=dz)
            assert abs(a.loss[0] - b.loss[0]) <= 1e-12 * max(1.0, abs(b.loss[0]))
            assert abs(a.loss[0] - float(L.item())) <= 1e-9 * max(1.0, abs(a.loss[0]))
            for x in (a.dz, b.dz):
                assert np.linalg.norm(x - to_np(dz)[0]) <= 1e-5 * max(np.linalg.norm(to_np(dz)), 1e-12)
    if precision == "bf16":
        assert dec.device_error() == 0


def test_admission_by_memory_and_errors(cuda_device):
    from paper_1911_13225_b300 import api
    from paper_1911_13225_b300._abi import DistError, DIST_E_INVALID, DIST_E_NOMEM
    from paper_1911_13225_b300.serve import Server
    spec = synth.SMALL_SPEC
    Ws, bs, Z = workload(spec, n_shapes=4)
    dec = gpu_decoder(spec, Ws, bs)
    # the pool holds two 32x32 requests at a time; eight must all complete
    srv = Server(dec, api.TraceParams(), max_rays=2048, mem_budget=1 << 30, max_requests=4)
    cams = [synth.look_at_camera(v, 32, 32) for v in synth.random_viewpoints(8, seed=4)]
    ts = [srv.submit(c, Z[i % 4]) for i, c in enumerate(cams)]
    for t in ts:
        srv.wait(t)
        assert np.isfinite(t.depth).any() or np.isinf(t.depth).all()
    with pytest.raises(DistError) as e:
        srv.submit(synth.look_at_camera((0, 0, 2.5), 64, 64), Z[0])
    assert e.value.status == DIST_E_NOMEM
    with pytest.raises(DistError) as e:
        srv.submit(synth.look_at_camera((0, 0, 0.5), 8, 8), Z[0])
    assert e.value.status == DIST_E_INVALID
    with pytest.raises(DistError) as e:
        srv.submit(cams[0], Z[0], kind="backward", tgt_depth=None)
    assert e.value.status == DIST_E_INVALID
    srv.close()
    tiny = Server(dec, api.TraceParams(), max_rays=4096, mem_budget=4096, max_requests=4)
    with pytest.raises(DistError) as e:
        tiny.submit(cams[0], Z[0])
    assert e.value.status == DIST_E_NOMEM
    tiny.close()
