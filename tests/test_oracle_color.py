"""Pins for the oracle's texture network (Sec. B.1 texture re-rendering; no GPU).

Reading: the colour network has the geometry network's layer widths; layer 0
reads [shape code, texture code, xyz], the skip layer [h, texture code, xyz]
(the last ``latent_dim`` code entries), and the head has three tanh outputs.
Pinned against a scalar restatement with explicit loops on a tiny network,
and against the SDF decoder when the code is just the skip code and one
output."""

import math

import numpy as np

import synth
from oracle.mlp import OracleDecoder


def _scalar(Ws, bs, p, code, L, skip):
    """The network written out with loops over neurons."""
    x_in = list(code) + list(p)
    x_skip = list(code[len(code) - L:]) + list(p)
    h = x_in
    for l in range(len(Ws) - 1):
        if l == skip:
            h = h + x_skip
        W, b = Ws[l], bs[l]
        h = [max(0.0, sum(float(W[o][i]) * h[i] for i in range(len(h))) + float(b[o]))
             for o in range(W.shape[0])]
    W, b = Ws[-1], bs[-1]
    return [math.tanh(sum(float(W[o][i]) * h[i] for i in range(len(h))) + float(b[o]))
            for o in range(W.shape[0])]


def test_texture_network_matches_scalar_loops():
    spec = synth.DecoderSpec(latent_dim=2, width=8, n_hidden=3, skip=2)
    Ws, bs = synth.make_color_decoder(spec, latent_dim0=5, out_dim=3, seed=4)
    assert Ws[0].shape == (8, 8) and Ws[2].shape == (8, 8) and Ws[1].shape == (3, 8)
    dec = OracleDecoder(Ws, bs, spec.latent_dim, spec.skip, latent_dim0=5, out_dim=3)
    rng = np.random.default_rng(0)
    P = rng.uniform(-0.6, 0.6, (7, 3))
    code = rng.normal(0, 0.5, 5)
    out = dec(P, code)
    assert out.shape == (7, 3)
    for k in range(7):
        ref = _scalar(Ws, bs, P[k], code, spec.latent_dim, spec.skip)
        np.testing.assert_allclose(out[k], ref, rtol=0, atol=1e-13)


def test_one_output_with_skip_code_is_the_sdf_decoder():
    spec = synth.SMALL_SPEC._replace(skip=2) if hasattr(synth.SMALL_SPEC, "_replace") else \
        synth.DecoderSpec(latent_dim=64, width=128, n_hidden=4, skip=2)
    Ws, bs = synth.make_color_decoder(spec, latent_dim0=spec.latent_dim, out_dim=1, seed=1)
    a = OracleDecoder(Ws, bs, spec.latent_dim, spec.skip)
    b = OracleDecoder(Ws, bs, spec.latent_dim, spec.skip, latent_dim0=spec.latent_dim, out_dim=1)
    rng = np.random.default_rng(1)
    P = rng.uniform(-0.6, 0.6, (50, 3))
    z = rng.normal(0, 0.1, spec.latent_dim)
    np.testing.assert_array_equal(a(P, z), b(P, z))
