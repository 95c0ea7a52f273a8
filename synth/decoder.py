"""Seeded DeepSDF-shaped decoder weights and latent codes.

Layer convention (shared by every consumer of these arrays):

* ``W[l]`` has shape ``[out_l, in_l]`` (row-major, float32), ``b[l]`` shape ``[out_l]``.
* Layer 0 reads ``[z (latent_dim), x, y, z_coord]`` -- latent first, then xyz,
  the DeepSDF input order.
* The skip layer ``spec.skip`` reads ``[h (out of layer skip-1), z, xyz]``;
  layer ``skip-1`` therefore outputs ``width - latent_dim - 3`` values so the
  concatenation is ``width`` wide.
* Hidden layers 0..n_hidden-1 are followed by ReLU; layer ``n_hidden`` is the
  head (``width -> 1``) followed by tanh.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class DecoderSpec:
    latent_dim: int
    width: int
    n_hidden: int
    skip: int  # -1: no skip concatenation

    def in_dim(self, l: int) -> int:
        if l == 0:
            return self.latent_dim + 3
        if l == self.n_hidden:  # head
            return self.width
        if l == self.skip:
            return self.width
        return self.width

    def out_dim(self, l: int) -> int:
        if l == self.n_hidden:
            return 1
        if self.skip > 0 and l == self.skip - 1:
            return self.width - self.latent_dim - 3
        return self.width

    @property
    def n_layers(self) -> int:
        return self.n_hidden + 1


# 9 FC layers, hidden 512, latent 256, skip at layer 4 (DeepSDF shape).
DEEPSDF_SPEC = DecoderSpec(latent_dim=256, width=512, n_hidden=8, skip=4)
# Small correctness decoder: latent 64, 4 hidden layers of 128, no skip.
SMALL_SPEC = DecoderSpec(latent_dim=64, width=128, n_hidden=4, skip=-1)


def make_decoder(spec: DecoderSpec, seed: int = 0, radius: float = 0.6,
                 perturb: float = 0.25, hidden_bias: float = 0.002):
    """Return ``(Ws, bs)`` lists of float32 arrays for ``spec``.

    Hidden weights ~ N(0, 2/out) with a seeded multiplicative perturbation of
    relative size ``perturb`` (renormalised to keep the variance), small
    seeded hidden biases, head weights sqrt(pi)/sqrt(in) and head bias
    ``-radius`` (geometric initialisation: the pre-tanh output approximates
    |p| - radius, and the finite width makes the surface bumpy).  The skip
    layer's weights are scaled by 1/sqrt(2) so the concatenation does not
    double the signal variance.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    Ws, bs = [], []
    for l in range(spec.n_layers):
        fan_in, fan_out = spec.in_dim(l), spec.out_dim(l)
        if l < spec.n_hidden:
            W = rng.normal(0.0, np.sqrt(2.0 / fan_out), size=(fan_out, fan_in))
            W *= (1.0 + perturb * rng.standard_normal(size=W.shape)) / np.sqrt(1.0 + perturb ** 2)
            if l == spec.skip:
                W *= 1.0 / np.sqrt(2.0)
            b = hidden_bias * rng.standard_normal(size=fan_out)
        else:
            W = np.full((1, fan_in), np.sqrt(np.pi) / np.sqrt(fan_in))
            W += 1e-4 * rng.standard_normal(size=W.shape)
            b = np.array([-radius])
        Ws.append(np.ascontiguousarray(W, dtype=np.float32))
        bs.append(np.ascontiguousarray(b, dtype=np.float32))
    return Ws, bs


def make_latents(spec: DecoderSpec, n: int, seed: int = 0, sigma: float = 0.01):
    """``n`` latent codes z ~ N(0, sigma^2) of length ``spec.latent_dim`` (float32)."""
    rng = np.random.Generator(np.random.PCG64(10_000 + seed))
    return np.ascontiguousarray(
        rng.normal(0.0, sigma, size=(n, spec.latent_dim)), dtype=np.float32)


def make_color_decoder(spec: DecoderSpec, latent_dim0: int, out_dim: int = 3, seed: int = 0):
    """Weights of a texture network with the layer widths of ``spec``: layer 0
    reads ``[code (latent_dim0), xyz]``, the skip layer ``[h, last
    spec.latent_dim code entries, xyz]``, the head has ``out_dim`` rows
    (tanh outputs).  Hidden weights ~ N(0, 2/out); head ~ N(0, 1/in)."""
    rng = np.random.Generator(np.random.PCG64(50_000 + seed))
    Ws, bs = [], []
    for l in range(spec.n_layers):
        fan_in = latent_dim0 + 3 if l == 0 else spec.in_dim(l)
        fan_out = out_dim if l == spec.n_hidden else spec.out_dim(l)
        if l < spec.n_hidden:
            W = rng.normal(0.0, np.sqrt(2.0 / fan_out), size=(fan_out, fan_in))
            if l == spec.skip:
                W *= 1.0 / np.sqrt(2.0)
            b = 0.002 * rng.standard_normal(size=fan_out)
        else:
            W = rng.normal(0.0, np.sqrt(1.0 / fan_in), size=(fan_out, fan_in))
            b = np.zeros(fan_out)
        Ws.append(np.ascontiguousarray(W, dtype=np.float32))
        bs.append(np.ascontiguousarray(b, dtype=np.float32))
    return Ws, bs
