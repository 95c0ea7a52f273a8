"""Shared helpers for the GPU parity tests: seeded workloads and the
classification of rays whose discrete decisions are within rounding of a
threshold (so FP32 and FP64 may legitimately take different branches)."""

from __future__ import annotations

import numpy as np

import synth
from oracle import tracer
from oracle.mlp import from_synth
from oracle.sdf import MLPSDF


def workload(spec, seed=0, n_shapes=1, latent_seed=0):
    Ws, bs = synth.make_decoder(spec, seed=seed)
    Z = synth.make_latents(spec, n_shapes, seed=latent_seed)
    return Ws, bs, Z


def oracle_sdf(spec, Ws, bs, Z):
    return MLPSDF(from_synth(Ws, bs, spec), Z.astype(np.float64))


def gpu_decoder(spec, Ws, bs):
    from paper_1911_13225_b300 import api
    return api.Decoder.from_spec(spec, Ws, bs)


def to_np(t):
    return t.detach().cpu().numpy()


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    a = ((a + 0x7FFF + ((a >> 16) & 1)) >> 16) << 16
    return a.astype(np.uint32).view(np.float32).astype(np.float64)


def fp16_round(x):
    """Round to the nearest IEEE half (ties to even), returned as float64."""
    return np.asarray(x, dtype=np.float32).astype(np.float16).astype(np.float64)


def e4m3_round(x):
    """Round to the nearest FP8 E4M3 value (3 mantissa bits, ties to even;
    saturating at 448, subnormals down to 2^-9), returned as float64."""
    x = np.asarray(x, dtype=np.float64)
    a = np.minimum(np.abs(x), 448.0)
    e = np.maximum(np.floor(np.log2(np.maximum(a, 2.0 ** -9))), -6.0)
    q = 2.0 ** (e - 3)
    return np.sign(x) * np.minimum(np.round(a / q) * q, 448.0)


def fp8_decoder_reference(Ws, bs, Z, pts, shape, act_scale, latent=256, skip=4):
    """The DeepSDF decoder as an FP8 (E4M3) tensor-core kernel would run it:
    GEMM layers 1..7 with E4M3 activations (per-layer scale ``act_scale[l]``)
    and E4M3 weights (per-output-row scale), exact accumulation; layer 0, the
    folded latent biases, the skip layer's xyz term and the head in full
    precision."""
    W = [np.asarray(w, dtype=np.float64) for w in Ws]
    b = [np.asarray(v, dtype=np.float64) for v in bs]
    z = np.asarray(Z, dtype=np.float64)[shape]
    p = np.asarray(pts, dtype=np.float64)
    hk = W[skip].shape[1] - latent - 3
    b0 = z @ W[0][:, :latent].T + b[0]
    bsk = z @ W[skip][:, hk:hk + latent].T + b[skip]
    h = np.maximum(p @ W[0][:, latent:].T + b0, 0.0)
    maxima = []
    for l in range(1, len(W) - 1):
        Wl = W[l][:, :hk] if l == skip else W[l]
        maxima.append(float(np.max(h)))
        sa = act_scale[l - 1] if act_scale is not None else max(np.max(h), 1e-30) / 448.0
        sw = np.maximum(np.max(np.abs(Wl), axis=1, keepdims=True), 1e-30) / 448.0
        a = (e4m3_round(h / sa) * sa) @ (e4m3_round(Wl / sw) * sw).T
        a = a + (p @ W[l][:, hk + latent:].T + bsk if l == skip else b[l])
        h = np.maximum(a, 0.0)
    return np.tanh(h @ W[-1].T + b[-1])[:, 0], maxima


def lowp_decoder_reference(Ws, bs, Z, pts, shape, precision, latent=256, skip=4):
    rnd = bf16_round if precision == "bf16" else fp16_round
    return bf16_decoder_reference(Ws, bs, Z, pts, shape, latent, skip, rnd=rnd)


def bf16_decoder_reference(Ws, bs, Z, pts, shape, latent=256, skip=4, rnd=None):
    """The DeepSDF decoder evaluated the way the BF16 tensor-core kernel does:
    GEMM layers 1..7 with bf16-rounded weights and bf16-rounded input
    activations (fp64 accumulation; the skip layer's xyz term through the
    same rounded GEMM), layer 0, the folded latent biases and the head in
    full precision.  ``rnd`` replaces the bf16 rounding (e.g. by fp16)."""
    bf16_round_ = rnd or bf16_round
    W = [np.asarray(w, dtype=np.float64) for w in Ws]
    b = [np.asarray(v, dtype=np.float64) for v in bs]
    z = np.asarray(Z, dtype=np.float64)[shape]
    p = np.asarray(pts, dtype=np.float64)
    hk = W[skip].shape[1] - latent - 3
    b0 = (z @ W[0][:, :latent].T + b[0]).astype(np.float32).astype(np.float64)
    bs_ = (z @ W[skip][:, hk:hk + latent].T + b[skip]).astype(np.float32).astype(np.float64)
    h = np.maximum(p @ W[0][:, latent:].T + b0, 0.0)
    for l in range(1, len(W) - 1):
        hb = bf16_round_(h)
        if l == skip:
            # the kernel's skip-layer GEMM also runs over the point (the
            # operand's padding columns), rounded like the activations
            a = hb @ bf16_round_(W[l][:, :hk]).T + \
                bf16_round_(p) @ bf16_round_(W[l][:, hk + latent:]).T + bs_
        else:
            a = hb @ bf16_round_(W[l]).T + b[l]
        h = np.maximum(a, 0.0)
    return np.tanh(h @ W[-1].T + b[-1])[:, 0]


def ambiguous_rays(orc, tol_f, tol_d=1e-5, max_steps=50, grazing=0.05, near_miss=0.0,
                   normals=None):
    """Rays whose FP32 trace may take a different branch than FP64.

    * some sample has | |f| - eps | < tol_f  (convergence test);
    * some stepped distance lands within tol_d of t_in / t_out (exit test);
    * the ray used (almost) its whole step budget;
    * hits at grazing incidence (|n . v| < grazing) -- the silhouette;
    * misses whose min |f| < near_miss.
    """
    eps, alpha = orc["eps"], orc["alpha"]
    rf, rd = orc["rec_f"], orc["rec_d"]
    with np.errstate(invalid="ignore"):
        a = np.abs(np.abs(rf) - eps) < tol_f
        stepped = rd + alpha * rf
        ex = (np.abs(stepped - orc["t_out"][:, None]) < tol_d) | \
             (np.abs(stepped - orc["t_in"][:, None]) < tol_d)
    amb = np.any(a, axis=1) | np.any(ex, axis=1)
    amb |= orc["steps"] >= max_steps - 2
    if normals is not None:
        nv = np.abs(np.einsum("ij,ij->i", normals, orc["v"]))
        amb |= orc["mask"] & (nv < grazing)
    if near_miss > 0:
        amb |= orc["enters"] & ~orc["mask"] & (orc["min_abs_f"] < near_miss)
    # rays grazing the bounding sphere: FP32 and FP64 may disagree on entry
    b = np.einsum("ij,ij->i", orc["v"], orc["c"])
    qq = np.einsum("ij,ij->i", orc["c"], orc["c"]) - b * b
    amb |= np.abs(qq - 1.0) < 1e-5
    return amb


# -------------------------------------------- silhouette rays at an |SDF| margin

SDF_MARGIN = 1e-3       # the |SDF| margin of the mask contract (hit/miss bit-exact beyond it)
FP32_CLASS_TOL = 5e-6   # bound on |f| error of the GPU's FP32 / FP32-class queries vs FP64


class ShiftedSDF:
    """f + delta: the zero level set moved by about delta along the normal
    (outwards for delta < 0).  Same gradient as f."""

    def __init__(self, sdf, delta):
        self.sdf, self.delta = sdf, float(delta)

    def __call__(self, p, shape=None):
        return self.sdf(p, shape) + self.delta

    def grad(self, p, shape=None):
        f, gp, gz = self.sdf.grad(p, shape)
        return f + self.delta, gp, gz


def shifted_traces(trace, sdf, margin=SDF_MARGIN):
    """The oracle trace ``trace(sdf')`` of the decoder shifted by -margin and
    +margin (trace is a function of an SDF, e.g. a partial of tracer.render)."""
    return [trace(ShiftedSDF(sdf, d)) for d in (-margin, margin)]


def silhouette_rays(orc, shifted, max_steps=50, tol_f=FP32_CLASS_TOL):
    """Rays excluded from the bit-exact hit/miss comparison of a 16-bit march
    against the oracle: rays within the |SDF| margin of the silhouette, read
    as "the oracle's hit/miss outcome changes when f is shifted by -margin
    or +margin" (the surface moved out or in by the margin: near-miss rays
    and barely-penetrating grazing hits); rays that use (almost) their whole
    step budget in any of the three traces (the budget is a count of
    queries, not a distance); rays whose convergence test the oracle passed
    or failed within the FP32-class query error (tol_f) of eps; and rays
    grazing the bounding sphere.  ``orc`` is the recorded oracle trace and
    ``shifted`` its two shifted traces (shifted_traces)."""
    amb = ambiguous_rays(orc, tol_f=tol_f, tol_d=0.0, max_steps=max_steps)
    for o in shifted:
        amb |= o["mask"] != orc["mask"]
        amb |= o["steps"] >= max_steps - 2
    return amb
