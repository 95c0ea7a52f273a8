"""Seeded synthetic inputs for the DIST sphere tracer.

This package is the only code that both the FP64 oracle (``oracle/``) and the
CUDA path (``paper_1911_13225_b300``) use.  It draws decoder weights, latent
codes and camera poses from numpy's PCG64 generator and holds none of the
method's arithmetic: no ray generation, no MLP evaluation, no marching.

DeepSDF's trained weights are not available, so the decoder is a seeded
geometric initialisation (f(p) ~ |p| - r, after Atzmon & Lipman, "SAL",
CVPR 2020) plus a seeded perturbation, with the DeepSDF layer shapes
(9 fully connected layers, hidden width 512, latent 256, skip concatenation
of [latent, xyz] at layer 4; Sec. B.1 "Network Architecture").
"""

from .decoder import (DecoderSpec, DEEPSDF_SPEC, SMALL_SPEC, make_color_decoder, make_decoder,
                      make_latents)
from .camera import look_at_camera, random_viewpoints, ring_viewpoints

__all__ = [
    "DecoderSpec",
    "DEEPSDF_SPEC",
    "SMALL_SPEC",
    "make_color_decoder",
    "make_decoder",
    "make_latents",
    "look_at_camera",
    "random_viewpoints",
    "ring_viewpoints",
]
