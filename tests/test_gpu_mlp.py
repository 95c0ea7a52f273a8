"""GPU decoder kernels vs the FP64 oracle decoder at random points
(dist_sdf_eval through the C ABI): values and gradients, several tiles and a
ragged tail, several latent codes."""

import numpy as np
import pytest
import torch

import synth
from tests.helpers import gpu_decoder, lowp_decoder_reference, oracle_sdf, to_np, workload

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [1, 127, 128 * 3 + 5, 148 * 128 + 77])
@pytest.mark.parametrize("precision", ["bf16", "fp16"])
def test_tensor_core_decoder(cuda_device, n, precision):
    """tcgen05 decoder (dist_sdf_eval, precision BF16 or FP16): against the
    same arithmetic emulated in fp64 (16-bit-rounded weights and activations)
    and against the FP64 oracle."""
    from paper_1911_13225_b300 import api
    spec = synth.DEEPSDF_SPEC
    Ws, bs, Z = workload(spec, seed=4, n_shapes=3)
    dec = gpu_decoder(spec, Ws, bs)
    assert dec.has_bf16
    ws = api.Workspace(max(n, 1024))
    rng = np.random.default_rng(n)
    pts = rng.uniform(-0.9, 0.9, (n, 3)).astype(np.float32)
    shp = rng.integers(0, 3, n).astype(np.int32)
    f = api.sdf_eval(dec, torch.from_numpy(Z).to(cuda_device), torch.from_numpy(pts).to(cuda_device),
                     torch.from_numpy(shp).to(cuda_device), ws, precision=precision)
    f = to_np(f).astype(np.float64)
    assert dec.device_error() == 0
    emu = lowp_decoder_reference(Ws, bs, Z, pts, shp, precision)
    d_emu = np.abs(f - emu)
    # identical arithmetic up to FP32 summation order; an activation whose
    # FP32 value sits at a rounding midpoint may round the other way and move
    # f by up to ~1e-3 (bf16), so the bound is on the typical point
    scale = 1.0 if precision == "bf16" else 0.125
    # fp16's 8x finer grid puts more activations near a rounding midpoint;
    # the median is a statement about many points
    if n >= 100:
        assert np.median(d_emu) < (1e-5 if precision == "bf16" else 5e-5)
    # (the skip layer's GEMM also takes the rounded ray point, one more place
    # where an FP32-order difference can flip a rounding: up to one 16-bit
    # ulp of an activation times a weight, ~2e-4 for fp16)
    q99 = 1e-3 if precision == "bf16" else 2.5e-4
    assert np.quantile(d_emu, 0.99) < q99 and np.max(d_emu) < 5e-3 * scale
    fo = oracle_sdf(spec, Ws, bs, Z)(pts.astype(np.float64), shp)
    d_or = np.abs(f - fo)
    assert np.max(d_or) < 5e-3 * scale and np.mean(d_or) < 1e-3 * scale


@pytest.mark.parametrize("n", [1, 200, 128 * 3 + 5, 148 * 128 + 77, 148 * 128 * 3 + 300])
def test_a_rows_value_does_not_depend_on_its_batch(cuda_device, n):
    """The tensor-core forward accumulates every output in the same K order
    and adds the head's chunk sums in one fixed order, whatever tile, CTA or
    launch a row lands in: the same point gives the same bits alone, in a
    shuffled batch and in a batch of another size, for 16-bit and FP32-class
    rows."""
    from paper_1911_13225_b300 import api
    spec = synth.DEEPSDF_SPEC
    Ws, bs, Z = workload(spec, seed=6, n_shapes=2)
    dec = gpu_decoder(spec, Ws, bs)
    ws = api.Workspace(max(n, 1024))
    rng = np.random.default_rng(n + 5)
    pts = torch.from_numpy(rng.uniform(-0.9, 0.9, (n, 3)).astype(np.float32)).to(cuda_device)
    shp = torch.from_numpy(rng.integers(0, 2, n).astype(np.int32)).to(cuda_device)
    zt = torch.from_numpy(Z).to(cuda_device)
    perm = torch.from_numpy(rng.permutation(n)).to(cuda_device)
    half = max(1, n // 2)
    for prec in ("bf16", "fp16", "fp32_tc"):
        full = to_np(api.sdf_eval(dec, zt, pts, shp, ws, precision=prec))
        shuf = to_np(api.sdf_eval(dec, zt, pts[perm], shp[perm], ws, precision=prec))
        part = to_np(api.sdf_eval(dec, zt, pts[:half], shp[:half], ws, precision=prec))
        np.testing.assert_array_equal(shuf, full[to_np(perm)])
        np.testing.assert_array_equal(part, full[:half])
        assert np.all(np.isfinite(full))
    assert dec.device_error() == 0


@pytest.mark.parametrize("n", [1, 63, 64 * 5 + 7, 148 * 64 + 33, 148 * 64 * 3 + 5])
def test_fp32_class_tensor_core_decoder(cuda_device, n):
    """Two-term FP16 split on the tensor cores (precision FP32_TC).  The split
    arithmetic is FP32-accurate; the tensor core's FP32 accumulation, which
    does not round to nearest, leaves ~2e-6 (measured on B300).  Bound: the
    FP32 SIMT kernel's bound against the FP64 oracle, 5e-6, at every point,
    and at least 10x closer to the oracle than the FP16 kernel."""
    from paper_1911_13225_b300 import api
    spec = synth.DEEPSDF_SPEC
    Ws, bs, Z = workload(spec, seed=4, n_shapes=3)
    dec = gpu_decoder(spec, Ws, bs)
    ws = api.Workspace(max(n, 1024))
    rng = np.random.default_rng(n + 1)
    pts = rng.uniform(-1, 1, (n, 3)).astype(np.float32)
    shp = rng.integers(0, 3, n).astype(np.int32)
    zt = torch.from_numpy(Z).to(cuda_device)
    pt, st = torch.from_numpy(pts).to(cuda_device), torch.from_numpy(shp).to(cuda_device)
    f_tc = to_np(api.sdf_eval(dec, zt, pt, st, ws, precision="fp32_tc")).astype(np.float64)
    f_32 = to_np(api.sdf_eval(dec, zt, pt, st, ws, precision="fp32")).astype(np.float64)
    f_16 = to_np(api.sdf_eval(dec, zt, pt, st, ws, precision="fp16")).astype(np.float64)
    assert dec.device_error() == 0
    fo = oracle_sdf(spec, Ws, bs, Z)(pts.astype(np.float64), shp)
    e_tc, e_16 = np.abs(f_tc - fo), np.abs(f_16 - fo)
    assert np.max(e_tc) < 5e-6
    assert np.max(np.abs(f_tc - f_32)) < 5e-6
    if n >= 64:
        assert np.median(e_tc) * 10 < np.median(e_16)


@pytest.mark.parametrize("spec,tol_f,tol_g", [(synth.SMALL_SPEC, 2e-6, 1e-5),
                                              (synth.DEEPSDF_SPEC, 5e-6, 2e-5)])
@pytest.mark.parametrize("n", [1, 63, 64 * 5 + 7, 4099])
def test_fp32_values_and_gradients(cuda_device, spec, tol_f, tol_g, n):
    from paper_1911_13225_b300 import api
    Ws, bs, Z = workload(spec, seed=4, n_shapes=3)
    dec = gpu_decoder(spec, Ws, bs)
    ws = api.Workspace(4096)
    rng = np.random.default_rng(n)
    pts = rng.uniform(-1, 1, (n, 3)).astype(np.float32)
    shp = rng.integers(0, 3, n).astype(np.int32)
    zt = torch.from_numpy(Z).to(cuda_device)
    f, g = api.sdf_eval(dec, zt, torch.from_numpy(pts).to(cuda_device),
                        torch.from_numpy(shp).to(cuda_device), ws, grad=True)
    f_only = api.sdf_eval(dec, zt, torch.from_numpy(pts).to(cuda_device),
                          torch.from_numpy(shp).to(cuda_device), ws)
    torch.cuda.synchronize()
    sdf = oracle_sdf(spec, Ws, bs, Z)
    fo, go, _ = sdf.grad(pts.astype(np.float64), shp)
    assert np.max(np.abs(to_np(f) - fo)) < tol_f
    assert np.max(np.abs(to_np(f_only) - fo)) < tol_f
    # the gradient is piecewise constant: a pre-activation within FP32
    # rounding of 0 may flip one ReLU; those points are compared loosely
    _, (_, pre, _) = sdf.dec.forward(pts.astype(np.float64), sdf.Z[shp], keep=True)
    kink = np.min(np.concatenate([np.abs(a) for a in pre], axis=1), axis=1) < 1e-5
    assert kink.mean() < 0.5
    err = np.max(np.abs(to_np(g) - go), axis=1)
    assert np.max(err[~kink]) < tol_g
    assert np.max(err) < 0.05


@pytest.mark.parametrize("n", [1, 63, 64 * 5 + 7, 148 * 64 + 33, 148 * 64 * 3 + 5])
def test_fp32_class_adjoint_values_and_gradients(cuda_device, n):
    """FP32-class tensor-core adjoint (dist_sdf_eval, FP32_TC with grad): f
    and grad_p f against the FP64 oracle at the FP32 SIMT kernel's bars
    (5e-6, 2e-5 away from ReLU kinks), one and several tiles per CTA and a
    ragged tail, three latent codes."""
    from paper_1911_13225_b300 import api
    spec = synth.DEEPSDF_SPEC
    Ws, bs, Z = workload(spec, seed=4, n_shapes=3)
    dec = gpu_decoder(spec, Ws, bs)
    ws = api.Workspace(max(n, 1024))
    rng = np.random.default_rng(n + 2)
    pts = rng.uniform(-1, 1, (n, 3)).astype(np.float32)
    shp = rng.integers(0, 3, n).astype(np.int32)
    zt = torch.from_numpy(Z).to(cuda_device)
    pt, st = torch.from_numpy(pts).to(cuda_device), torch.from_numpy(shp).to(cuda_device)
    f, g = api.sdf_eval(dec, zt, pt, st, ws, precision="fp32_tc", grad=True)
    f32, g32 = api.sdf_eval(dec, zt, pt, st, ws, precision="fp32", grad=True)
    torch.cuda.synchronize()
    assert dec.device_error() == 0
    sdf = oracle_sdf(spec, Ws, bs, Z)
    fo, go, _ = sdf.grad(pts.astype(np.float64), shp)
    f, g = to_np(f).astype(np.float64), to_np(g).astype(np.float64)
    assert np.max(np.abs(f - fo)) < 5e-6
    _, (_, pre, _) = sdf.dec.forward(pts.astype(np.float64), sdf.Z[shp], keep=True)
    kink = np.min(np.concatenate([np.abs(a) for a in pre], axis=1), axis=1) < 1e-5
    err = np.max(np.abs(g - go), axis=1)
    assert np.max(err) < 0.05
    if (~kink).any():
        assert np.max(err[~kink]) < 2e-5
        # and as close to the oracle as the FP32 SIMT adjoint, to within 2e-5
        err32 = np.max(np.abs(to_np(g32).astype(np.float64) - go), axis=1)
        assert np.max(err[~kink]) < np.max(err32[~kink]) + 2e-5
