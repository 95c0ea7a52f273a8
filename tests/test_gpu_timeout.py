"""Failure detection without a GPU fault: every device-side wait of the
tensor-core kernels is bounded, and a wait that runs out makes the kernel
set the decoder's error word, drain, free its tensor memory and return, so
the context stays usable.

The wait is made to run out by a flag that nothing sets: with
withhold_copies the forward kernel's weight loader issues no copies, so the
MMA issuer's wait for the first weight stage never completes; with a 1 ms
limit it gives up, the other roles see the abort flag, and the C ABI then
reports DIST_E_TIMEOUT.  Afterwards the same decoder traces normally, bit
for bit like before."""

from ctypes import byref, c_int32

import numpy as np
import pytest
import torch

import synth
from tests.helpers import gpu_decoder, to_np, workload

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_the_gpu_keeps_working(cuda_device):
    from paper_1911_13225_b300 import api, _abi
    spec = synth.DEEPSDF_SPEC
    Ws, bs, Z = workload(spec)
    dec = gpu_decoder(spec, Ws, bs)
    cam = synth.look_at_camera(synth.random_viewpoints(1, seed=3)[0], 64, 64)
    ws = api.Workspace(64 * 64, 50)
    z = torch.from_numpy(Z).to(cuda_device)
    # latency mode off: every step is decoded by the kernel whose loader is withheld
    params = api.TraceParams(precision="bf16", latency_mode=0)
    before = api.trace(dec, z, [cam], params, ws)
    assert dec.device_error() == 0

    dec.set_wait_limit(1_000_000, withhold_copies=True)      # 1 ms
    api.trace(dec, z, [cam], params, ws)
    pts = torch.zeros(300, 3, device=cuda_device)
    api.sdf_eval(dec, z, pts, torch.zeros(300, dtype=torch.int32, device=cuda_device), ws,
                 precision="bf16")
    code = c_int32(0)
    st = _abi.lib().dist_decoder_device_error(dec.handle, byref(code))
    assert st == _abi.DIST_E_TIMEOUT
    assert code.value & 2, code.value          # the MMA issuer's wait ran out
    assert code.value & 4, code.value          # the epilogue saw the abort
    assert not code.value & 64
    # the word was cleared by the read
    assert dec.device_error() == 0

    dec.set_wait_limit(1_000_000_000, withhold_copies=False)
    after = api.trace(dec, z, [cam], params, ws)
    torch.cuda.synchronize()
    assert dec.device_error() == 0
    for k in ("depth", "sil", "mask", "steps", "status"):
        np.testing.assert_array_equal(to_np(getattr(after, k)), to_np(getattr(before, k)))


def test_wait_limit_arguments(cuda_device):
    from paper_1911_13225_b300 import _abi
    from paper_1911_13225_b300._abi import DistError
    spec = synth.DEEPSDF_SPEC
    Ws, bs, _ = workload(spec)
    dec = gpu_decoder(spec, Ws, bs)
    for bad in (0, 9_999, 10_000_000_001):
        with pytest.raises(DistError):
            dec.set_wait_limit(bad)
    small = gpu_decoder(synth.SMALL_SPEC, *workload(synth.SMALL_SPEC)[:2])
    assert _abi.lib().dist_decoder_set_wait_limit(small.handle, 10**6, 0) == \
        _abi.DIST_E_UNSUPPORTED
