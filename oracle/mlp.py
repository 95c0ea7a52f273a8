"""DeepSDF decoder f(p, z) in float64 with its hand-derived chain rule.

The paper renders the conditional SDF f_theta(p, z) of DeepSDF (Sec. 3.4,
"Approximated Gradient Back-Propagation") with the DeepSDF architecture: nine
fully connected layers, hidden width 512, latent 256 (Sec. B.1).  The input is
the concatenation [z, p]; the skip layer reads [h, z, p]; hidden layers use
ReLU and the head uses tanh.  This module evaluates that definition directly,
unfolded (the latent is concatenated, not folded into a bias), one matrix
product per layer.
"""

from __future__ import annotations

import numpy as np


class OracleDecoder:
    """f(p, z) for weights ``Ws[l]`` ([out, in]) and biases ``bs[l]``.

    ``latent_dim0`` > ``latent_dim`` gives the texture network of Sec. B.1
    (reading: layer 0 reads the whole code, e.g. [shape code, texture code],
    and the skip layer its last ``latent_dim`` entries, the texture code);
    ``out_dim`` > 1 gives that many tanh outputs (colour)."""

    def __init__(self, Ws, bs, latent_dim: int, skip: int, latent_dim0: int = 0,
                 out_dim: int = 1):
        self.Ws = [np.asarray(W, dtype=np.float64) for W in Ws]
        self.bs = [np.asarray(b, dtype=np.float64) for b in bs]
        self.L = int(latent_dim)
        self.L0 = int(latent_dim0) if latent_dim0 else self.L
        self.out_dim = int(out_dim)
        self.skip = int(skip)
        self.n_hidden = len(self.Ws) - 1

    # -- forward ---------------------------------------------------------
    def _inputs(self, p, z):
        p = np.atleast_2d(np.asarray(p, dtype=np.float64))
        z = np.asarray(z, dtype=np.float64)
        if z.ndim == 1:
            z = np.broadcast_to(z, (p.shape[0], z.shape[0]))
        return np.concatenate([z, p], axis=1)

    def forward(self, p, z, keep=False):
        """Return f (n,) (or (n, out_dim) for out_dim > 1) and, with ``keep``,
        the per-layer pre-activations."""
        x_in = self._inputs(p, z)
        # the skip layer's input tail: [last latent_dim code entries, p]
        x_skip = x_in[:, self.L0 - self.L:]
        h = x_in
        pre = []
        for l in range(self.n_hidden):
            if l == self.skip:
                h = np.concatenate([h, x_skip], axis=1)
            a = h @ self.Ws[l].T + self.bs[l]
            pre.append(a)
            h = np.maximum(a, 0.0)
        s = h @ self.Ws[-1].T + self.bs[-1]
        if self.out_dim > 1:
            return np.tanh(s)
        f = np.tanh(s[:, 0])
        if keep:
            return f, (x_in, pre, s[:, 0])
        return f

    __call__ = forward

    # -- reverse-mode chain rule ------------------------------------------
    def grad(self, p, z):
        """Return (f, df/dp (n,3), df/dz (n,L)).

        Written out by the chain rule: df/ds = 1 - tanh(s)^2; each hidden layer
        passes g -> (W^T g) * 1[a > 0]; the skip concatenation splits the
        gradient between the previous layer's output and the input [z, p].
        """
        assert self.out_dim == 1 and self.L0 == self.L, "gradients of the SDF decoder only"
        f, (x_in, pre, s) = self.forward(p, z, keep=True)
        n = x_in.shape[0]
        g_x = np.zeros_like(x_in)               # gradient w.r.t. [z, p]
        g = (1.0 - f * f)[:, None] * self.Ws[-1]  # d f / d h_last  (n, width)
        for l in range(self.n_hidden - 1, -1, -1):
            g = g * (pre[l] > 0.0)              # through ReLU
            g_in = g @ self.Ws[l]               # d f / d (layer-l input)
            if l == self.skip:
                k = g_in.shape[1] - x_in.shape[1]
                g_x += g_in[:, k:]
                g = g_in[:, :k]
            elif l == 0:
                g_x += g_in
            else:
                g = g_in
        assert g_x.shape == (n, self.L + 3)
        return f, g_x[:, self.L:], g_x[:, :self.L]


def from_synth(Ws, bs, spec):
    """Build an ``OracleDecoder`` from ``synth.make_decoder`` output."""
    return OracleDecoder(Ws, bs, spec.latent_dim, spec.skip)
