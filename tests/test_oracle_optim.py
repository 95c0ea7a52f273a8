"""Pins of the oracle's Adam step (oracle/optim.py), the optimiser of the
inverse problem (Sec. 4.2, Sec. B.4), against a library implementation and
against closed forms of the first steps."""

import numpy as np
import torch

from oracle.optim import adam_step


def test_matches_torch_adam_over_many_steps():
    rng = np.random.default_rng(0)
    z0 = rng.normal(0, 0.01, (4, 16))
    z, m, v = z0.copy(), np.zeros_like(z0), np.zeros_like(z0)
    p = torch.tensor(z0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    for t in range(1, 31):
        g = rng.normal(0, 1, z0.shape) * (1 + t % 3)
        z, m, v = adam_step(z, g, m, v, t)
        p.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        np.testing.assert_allclose(z, p.detach().numpy(), rtol=0, atol=1e-13)


def test_first_step_moves_each_entry_by_lr_times_sign():
    # t = 1: m_hat = g and v_hat = g^2, so the step is lr g / (|g| + eps)
    g = np.array([3.0, -0.5, 1e-3, -7.0])
    z, m, v = adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.1, eps=1e-8)
    np.testing.assert_allclose(z, -0.1 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-12)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-12)


def test_constant_gradient_gives_constant_step():
    # with g constant, m_hat = g and v_hat = g^2 at every t: steps of lr
    z, m, v = np.zeros(2), np.zeros(2), np.zeros(2)
    g = np.array([2.0, -4.0])
    for t in range(1, 11):
        z, m, v = adam_step(z, g, m, v, t, lr=1e-2, eps=0.0)
        np.testing.assert_allclose(z, -1e-2 * t * np.sign(g), rtol=1e-12)
