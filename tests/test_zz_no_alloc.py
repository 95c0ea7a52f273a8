"""dist_sdf_eval_static: the allocation-free decoder evaluation.

It exists for callers that may not allocate device memory (a plugin held to
its host application's GPU budget, a framework whose pool owns the device,
a latency-critical thread that must not take an allocation's implicit
synchronisation).  Its scratch is a fixed built-in device array, so it must
give the same results as dist_sdf_eval with a workspace -- on consecutive
calls too, since every call reuses that one array -- and it must refuse
sizes beyond the array.  This file sorts last so a stop-at-first-failure run
has already run every other test.
"""

from ctypes import c_void_p

import numpy as np
import pytest
import torch

import synth
from tests.helpers import gpu_decoder, to_np, workload

pytestmark = pytest.mark.gpu


def _static(dec, z, pts, shp, precision, want_grad):
    from paper_1911_13225_b300 import _abi
    n = pts.shape[0]
    f = torch.empty(n, device=pts.device)
    g = torch.empty(n, 3, device=pts.device) if want_grad else None
    prec = _abi.PREC_FP32 if precision == "fp32" else _abi.PREC_BF16
    st = _abi.lib().dist_sdf_eval_static(
        dec.handle, c_void_p(z.data_ptr()), int(z.shape[0]), c_void_p(pts.data_ptr()),
        c_void_p(shp.data_ptr()), n, prec, c_void_p(f.data_ptr()),
        c_void_p(g.data_ptr()) if g is not None else None,
        c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, f, g


@pytest.mark.parametrize("spec,precision", [(synth.SMALL_SPEC, "fp32"),
                                            (synth.DEEPSDF_SPEC, "fp32"),
                                            (synth.DEEPSDF_SPEC, "bf16")])
def test_static_scratch_matches_workspace_entry_point(cuda_device, spec, precision):
    from paper_1911_13225_b300 import api, _abi
    Ws, bs, Z = workload(spec, seed=9, n_shapes=3)
    dec = gpu_decoder(spec, Ws, bs)
    ws = api.Workspace(8192)
    z = torch.from_numpy(Z).to(cuda_device)
    want_grad = precision == "fp32"
    rng = np.random.default_rng(21)
    for n in (1000, 4099):          # two calls in a row through the same scratch
        pts = torch.from_numpy(rng.uniform(-0.9, 0.9, (n, 3)).astype(np.float32)).to(cuda_device)
        shp = torch.from_numpy(rng.integers(0, 3, n).astype(np.int32)).to(cuda_device)
        if want_grad:
            f_ref, g_ref = api.sdf_eval(dec, z, pts, shp, ws, precision=precision, grad=True)
        else:
            f_ref = api.sdf_eval(dec, z, pts, shp, ws, precision=precision)
        st, f, g = _static(dec, z, pts, shp, precision, want_grad)
        torch.cuda.synchronize()
        assert st == _abi.DIST_OK, _abi.lib().dist_last_error()
        tol_f = 5e-6 if precision == "fp32" else 5e-3
        assert np.max(np.abs(to_np(f) - to_np(f_ref))) <= tol_f
        if want_grad:
            assert np.max(np.abs(to_np(g) - to_np(g_ref))) <= 2e-5
    if precision == "bf16":
        assert dec.device_error() == 0


def test_static_scratch_rejects_sizes_beyond_its_limit(cuda_device):
    from paper_1911_13225_b300 import _abi
    spec = synth.SMALL_SPEC
    Ws, bs, Z = workload(spec, n_shapes=65)
    dec = gpu_decoder(spec, Ws, bs)
    z = torch.from_numpy(Z).to(cuda_device)
    pts = torch.zeros(65537, 3, device=cuda_device)
    shp = torch.zeros(65537, dtype=torch.int32, device=cuda_device)
    st, _, _ = _static(dec, z[:1], pts, shp, "fp32", False)
    assert st == _abi.DIST_E_INVALID
    assert b"65536" in _abi.lib().dist_last_error()
    st, _, _ = _static(dec, z, pts[:10], shp[:10], "fp32", False)
    assert st == _abi.DIST_E_INVALID
    st, f, _ = _static(dec, z[:1], pts[:65536], shp[:65536], "fp32", False)
    torch.cuda.synchronize()
    assert st == _abi.DIST_OK and torch.isfinite(f).all()
