"""dist_sdf_eval_static: the allocation-free decoder evaluation.

It exists for callers that may not allocate device memory (a plugin held to
its host application's GPU budget, a framework whose pool owns the device,
a latency-critical thread that must not take an allocation's implicit
synchronisation).  Its scratch is a fixed built-in device array; it runs the
same kernels as dist_sdf_eval with a workspace, so its results must be the
same bits -- on consecutive calls too, since every call reuses that one
array -- and within the decoder bars of the FP64 oracle; it must refuse
sizes beyond the array.  This file sorts last so a stop-at-first-failure run
has already run every other test."""

from ctypes import c_void_p

import numpy as np
import pytest
import torch

import synth
from tests.helpers import gpu_decoder, oracle_sdf, to_np, workload

pytestmark = pytest.mark.gpu


def _static(dec, z, pts, shp, precision, want_grad):
    from paper_1911_13225_b300 import _abi
    n = pts.shape[0]
    f = torch.full((n,), float("nan"), device=pts.device)
    g = torch.full((n, 3), float("nan"), device=pts.device) if want_grad else None
    st = _abi.lib().dist_sdf_eval_static(
        dec.handle, c_void_p(z.data_ptr()), int(z.shape[0]), c_void_p(pts.data_ptr()),
        c_void_p(shp.data_ptr()), n, _abi.PRECISIONS[precision], c_void_p(f.data_ptr()),
        c_void_p(g.data_ptr()) if g is not None else None,
        c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, f, g


def _oracle_bar(spec, precision, f, fo):
    """The decoder bars of the parity tests against the FP64 oracle: FP32
    and FP32-class within 5e-6 at every point; 16-bit operands within 5e-3
    (BF16) or 6.25e-4 (FP16) at every point and 1e-3 / 1.25e-4 on average."""
    d = np.abs(f.astype(np.float64) - fo)
    if precision in ("fp32", "fp32_tc"):
        assert np.max(d) < (2e-6 if spec is synth.SMALL_SPEC else 5e-6)
    else:
        scale = 1.0 if precision == "bf16" else 0.125
        assert np.max(d) < 5e-3 * scale and np.mean(d) < 1e-3 * scale


@pytest.mark.parametrize("spec,precision", [(synth.SMALL_SPEC, "fp32"),
                                            (synth.DEEPSDF_SPEC, "fp32"),
                                            (synth.DEEPSDF_SPEC, "bf16"),
                                            (synth.DEEPSDF_SPEC, "fp16"),
                                            (synth.DEEPSDF_SPEC, "fp32_tc")])
def test_static_scratch_matches_workspace_entry_point(cuda_device, spec, precision):
    from paper_1911_13225_b300 import api, _abi
    Ws, bs, Z = workload(spec, seed=9, n_shapes=3)
    dec = gpu_decoder(spec, Ws, bs)
    ws = api.Workspace(8192)
    z = torch.from_numpy(Z).to(cuda_device)
    want_grad = precision == "fp32"
    rng = np.random.default_rng(21)
    sdf = oracle_sdf(spec, Ws, bs, Z)
    for n in (1000, 4099):          # two calls in a row through the same scratch
        pts_np = rng.uniform(-0.9, 0.9, (n, 3)).astype(np.float32)
        shp_np = rng.integers(0, 3, n).astype(np.int32)
        pts, shp = torch.from_numpy(pts_np).to(cuda_device), torch.from_numpy(shp_np).to(cuda_device)
        if want_grad:
            f_ref, g_ref = api.sdf_eval(dec, z, pts, shp, ws, precision=precision, grad=True)
        else:
            f_ref = api.sdf_eval(dec, z, pts, shp, ws, precision=precision)
        st, f, g = _static(dec, z, pts, shp, precision, want_grad)
        torch.cuda.synchronize()
        assert st == _abi.DIST_OK, _abi.lib().dist_last_error()
        # the same kernels on the same inputs: the same bits
        np.testing.assert_array_equal(to_np(f), to_np(f_ref))
        if want_grad:
            np.testing.assert_array_equal(to_np(g), to_np(g_ref))
        _oracle_bar(spec, precision, to_np(f), sdf(pts_np.astype(np.float64), shp_np))
    if precision != "fp32":
        assert dec.device_error() == 0


def test_static_scratch_at_full_capacity(cuda_device):
    """n = 65536 points and n_shapes = 64 codes, the array's limits: the last
    packed-point, output and bias-table entries are written and read (FP32
    with gradient writes the staging region too); same bits as the workspace
    entry point, shape indices covering 0..63."""
    from paper_1911_13225_b300 import api, _abi
    spec = synth.DEEPSDF_SPEC
    Ws, bs, Z = workload(spec, seed=2, n_shapes=64)
    dec = gpu_decoder(spec, Ws, bs)
    ws = api.Workspace(8192)                 # 81,920 points
    z = torch.from_numpy(Z).to(cuda_device)
    n = 65536
    rng = np.random.default_rng(3)
    pts_np = rng.uniform(-0.9, 0.9, (n, 3)).astype(np.float32)
    shp_np = (np.arange(n) % 64).astype(np.int32)
    rng.shuffle(shp_np[:-64])                # the last 64 points keep codes 0..63 in order
    pts, shp = torch.from_numpy(pts_np).to(cuda_device), torch.from_numpy(shp_np).to(cuda_device)
    f_ref, g_ref = api.sdf_eval(dec, z, pts, shp, ws, precision="fp32", grad=True)
    st, f, g = _static(dec, z, pts, shp, "fp32", True)
    torch.cuda.synchronize()
    assert st == _abi.DIST_OK, _abi.lib().dist_last_error()
    np.testing.assert_array_equal(to_np(f), to_np(f_ref))
    np.testing.assert_array_equal(to_np(g), to_np(g_ref))
    for prec in ("bf16", "fp32_tc"):
        r = api.sdf_eval(dec, z, pts, shp, ws, precision=prec)
        st, f, _ = _static(dec, z, pts, shp, prec, False)
        torch.cuda.synchronize()
        assert st == _abi.DIST_OK, _abi.lib().dist_last_error()
        np.testing.assert_array_equal(to_np(f), to_np(r))
    assert dec.device_error() == 0
    # the tail (last code, last slot) against the oracle
    tail = slice(n - 256, n)
    fo = oracle_sdf(spec, Ws, bs, Z)(pts_np[tail].astype(np.float64), shp_np[tail])
    assert np.max(np.abs(to_np(f_ref)[tail] - fo)) < 5e-6


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
    assert b"64" in _abi.lib().dist_last_error()
    # the static entry gives gradients in FP32 only; the small decoder has no
    # tensor-core path
    deep = synth.DEEPSDF_SPEC
    Wd, bd, Zd = workload(deep, n_shapes=1)
    ddec = gpu_decoder(deep, Wd, bd)
    zd = torch.from_numpy(Zd).to(cuda_device)
    for prec in ("bf16", "fp16", "fp32_tc"):
        st, _, _ = _static(ddec, zd, pts[:10], shp[:10], prec, True)
        assert st == _abi.DIST_E_INVALID
    st, _, _ = _static(dec, z[:1], pts[:10], shp[:10], "bf16", False)
    assert st == _abi.DIST_E_UNSUPPORTED
