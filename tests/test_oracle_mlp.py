"""Pins for the oracle's DeepSDF decoder (no GPU).

The decoder definition (input [z, p], skip input [h, z, p], ReLU, tanh head;
Sec. B.1) is pinned by weights that make it compute closed forms, and its
hand-written chain rule by central finite differences.
"""

import numpy as np
import pytest

import synth
from oracle.mlp import OracleDecoder, from_synth



def _abs_net(L=2, r=0.3):
    # layer 0 reads [z0, z1, x, y, z] and emits relu(+-x), relu(+-y), relu(+-z), relu(+-z0)
    W0 = np.zeros((8, L + 3))
    for k, col in enumerate([L, L + 1, L + 2, 0]):
        W0[2 * k, col] = 1.0
        W0[2 * k + 1, col] = -1.0
    W1 = np.eye(8)
    Wh = np.ones((1, 8))
    return OracleDecoder([W0, W1, Wh], [np.zeros(8), np.zeros(8), np.array([-r])], L, -1)


def test_forward_closed_form_no_skip():
    dec = _abs_net()
    rng = np.random.default_rng(0)
    p = rng.uniform(-1, 1, (50, 3))
    z = np.array([0.2, -7.0])
    f = dec.forward(p, z)
    expect = np.tanh(np.abs(p).sum(1) + 0.2 - 0.3)
    np.testing.assert_allclose(f, expect, rtol=0, atol=1e-15)


def test_forward_closed_form_skip():
    # L = 1, width 6, skip at layer 2: layer 1 outputs 6 - 1 - 3 = 2 values,
    # layer 2 reads [h(2), z0, x, y, z] and must route x (column 3) through.
    L = 1
    W0 = np.zeros((6, 4)); W0[0, 1] = 1.0          # h0 = relu(x)
    b0 = np.zeros(6)
    W1 = np.zeros((2, 6)); W1[0, 0] = 2.0          # h1 = [relu(2 relu(x)), 0]
    b1 = np.zeros(2)
    W2 = np.zeros((6, 6))
    W2[0, 0] = 1.0    # relu(2 relu(x))
    W2[1, 3] = -1.0   # relu(-x) via the skip copy of x
    W2[2, 5] = 1.0    # relu(z_coord) via the skip copy
    W2[3, 2] = 1.0    # relu(z0) via the skip copy of the latent
    b2 = np.zeros(6)
    Wh = np.array([[1.0, 1.0, 10.0, 100.0, 0.0, 0.0]])
    dec = OracleDecoder([W0, W1, W2, Wh], [b0, b1, b2, np.array([0.0])], L, 2)
    p = np.array([[0.3, 0.1, -0.2], [-0.4, 0.5, 0.25]])
    z = np.array([0.001])
    f = dec.forward(p, z)
    x, zc = p[:, 0], p[:, 2]
    s = 2 * np.maximum(x, 0) + np.maximum(-x, 0) + 10 * np.maximum(zc, 0) + 100 * 0.001
    np.testing.assert_allclose(f, np.tanh(s), rtol=0, atol=1e-15)


@pytest.mark.parametrize("spec", [synth.SMALL_SPEC, synth.DEEPSDF_SPEC])
def test_chain_rule_vs_central_differences(spec):
    Ws, bs = synth.make_decoder(spec, seed=3)
    dec = from_synth(Ws, bs, spec)
    z = synth.make_latents(spec, 1, seed=3)[0].astype(np.float64)
    rng = np.random.default_rng(5)
    p = rng.uniform(-0.7, 0.7, (6, 3))
    f, gp, gz = dec.grad(p, z)
    h = 1e-6
    for a in range(3):
        e = np.zeros(3); e[a] = h
        fd = (dec.forward(p + e, z) - dec.forward(p - e, z)) / (2 * h)
        np.testing.assert_allclose(gp[:, a], fd, rtol=1e-6, atol=1e-9)
    for j in [0, 1, spec.latent_dim // 2, spec.latent_dim - 1]:
        e = np.zeros(spec.latent_dim); e[j] = h
        fd = (dec.forward(p, z + e) - dec.forward(p, z - e)) / (2 * h)
        np.testing.assert_allclose(gz[:, j], fd, rtol=1e-6, atol=1e-9)


def test_synth_decoder_shapes():
    spec = synth.DEEPSDF_SPEC
    Ws, bs = synth.make_decoder(spec)
    shapes = [W.shape for W in Ws]
    assert shapes == [(512, 259), (512, 512), (512, 512), (253, 512), (512, 512),
                      (512, 512), (512, 512), (512, 512), (1, 512)]
    assert all(W.dtype == np.float32 for W in Ws)
    # deterministic from the seed
    Ws2, _ = synth.make_decoder(spec)
    assert all(np.array_equal(a, b) for a, b in zip(Ws, Ws2))
