"""ctypes mirror of include/dist.h.  Marshalling only: no computation here.

The shared library is loaded from this package directory; if it is missing
the import fails loudly (there is no CPU fallback).
"""

from __future__ import annotations

import ctypes
import os
from ctypes import (POINTER, Structure, c_char_p, c_double, c_float, c_int, c_int64,
                    c_size_t, c_uint64, c_void_p)

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdist.so")

DIST_OK, DIST_E_INVALID, DIST_E_NOMEM, DIST_E_CUDA, DIST_E_TIMEOUT, DIST_E_BUSY, \
    DIST_E_UNSUPPORTED = range(7)
STATUS_NAMES = {0: "DIST_OK", 1: "DIST_E_INVALID", 2: "DIST_E_NOMEM", 3: "DIST_E_CUDA",
                4: "DIST_E_TIMEOUT", 5: "DIST_E_BUSY", 6: "DIST_E_UNSUPPORTED"}
PREC_FP32, PREC_BF16, PREC_FP16, PREC_FP32_TC = 0, 1, 2, 3
PRECISIONS = {"fp32": PREC_FP32, "bf16": PREC_BF16, "fp16": PREC_FP16, "fp32_tc": PREC_FP32_TC}
REFINE_ENGINES = {"tc": 0, "simt": 1}
REFINE_RULES = {"march": 0, "secant": 1}
GRAD_EXACT, GRAD_PAPER = 0, 1
RAY_INIT_MISS, RAY_HIT, RAY_LEFT, RAY_MAX_STEPS = 0, 1, 2, 3
REQ_RENDER, REQ_RENDER_BACKWARD = 0, 1

# every entry point include/dist.h declares
EXPORTS = [
    "dist_decoder_create", "dist_decoder_destroy", "dist_decoder_has_bf16",
    "dist_decoder_device_error", "dist_profile_enable",
    "dist_profile_read",
    "dist_trace_params_default", "dist_workspace_create", "dist_workspace_destroy",
    "dist_trace_fwd", "dist_render_normals", "dist_sdf_eval", "dist_loss", "dist_trace_bwd",
    "dist_trace_bwd_camera", "dist_photo_loss", "dist_render_color",
    "dist_serve_create", "dist_serve_submit", "dist_serve_poll", "dist_serve_destroy",
    "dist_last_error", "dist_version", "dist_sdf_eval_static", "dist_adam_step",
    "dist_decoder_set_wait_limit",
]


class DecoderDesc(Structure):
    _fields_ = [("latent_dim", c_int), ("width", c_int), ("n_hidden", c_int), ("skip", c_int),
                ("latent_dim0", c_int), ("out_dim", c_int)]


class Camera(Structure):
    _fields_ = [("fx", c_float), ("fy", c_float), ("cx", c_float), ("cy", c_float),
                ("R", c_float * 9), ("c", c_float * 3), ("H", c_int), ("W", c_int),
                ("shape", c_int)]


class TraceParams(Structure):
    _fields_ = [("max_steps", c_int), ("eps", c_float), ("alpha", c_float), ("k_min", c_int),
                ("normal_delta", c_float), ("grad_mode", c_int), ("precision", c_int),
                ("eps_bf16", c_float), ("radius", c_float), ("refine_steps", c_int),
                ("alpha_refine", c_float), ("refine_engine", c_int), ("refine_rule", c_int),
                ("coarse_levels", c_int), ("coarse_every", c_int), ("latency_mode", c_int),
                ("eps_mid", c_float)]


class TraceOut(Structure):
    _fields_ = [("depth", c_void_p), ("sil", c_void_p), ("mask", c_void_p),
                ("steps", c_void_p), ("status", c_void_p), ("d_hit", c_void_p),
                ("d_min", c_void_p), ("f_min", c_void_p), ("normal", c_void_p),
                ("queries", c_void_p), ("grad_len", c_void_p)]


class LossWeights(Structure):
    _fields_ = [("w_depth", c_float), ("w_normal", c_float), ("w_sil", c_float),
                ("w_reg", c_float)]


class Request(Structure):
    _fields_ = [("kind", c_int), ("cam", Camera), ("z", c_void_p), ("tgt_depth", c_void_p),
                ("depth", c_void_p), ("sil", c_void_p), ("mask", c_void_p), ("dz", c_void_p),
                ("loss", c_void_p)]


_lib = None


def lib():
    """Load libdist.so (built by ``paper_1911_13225_b300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"{LIB_PATH} is missing: build it with `python -m paper_1911_13225_b300.build` "
            "(the CUDA library is required; there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "dist_decoder_create": (c_int, [POINTER(DecoderDesc), POINTER(c_void_p),
                                        POINTER(c_void_p), POINTER(c_void_p)]),
        "dist_decoder_destroy": (c_int, [c_void_p]),
        "dist_decoder_has_bf16": (c_int, [c_void_p]),
        "dist_decoder_device_error": (c_int, [c_void_p, POINTER(ctypes.c_int32)]),
        "dist_decoder_set_wait_limit": (c_int, [c_void_p, c_uint64, c_int]),
        "dist_profile_enable": (c_int, [c_int]),
        "dist_profile_read": (c_int, [POINTER(c_double), POINTER(c_int64), POINTER(c_int64)]),
        "dist_trace_params_default": (None, [POINTER(TraceParams)]),
        "dist_workspace_create": (c_int, [c_int64, c_int, POINTER(c_void_p)]),
        "dist_workspace_destroy": (c_int, [c_void_p]),
        "dist_trace_fwd": (c_int, [c_void_p, c_void_p, c_int, POINTER(Camera), c_int,
                                   POINTER(TraceParams), POINTER(TraceOut), c_void_p, c_void_p]),
        "dist_render_normals": (c_int, [c_void_p, c_void_p, c_int, POINTER(Camera), c_int,
                                        POINTER(TraceParams), POINTER(TraceOut), c_void_p,
                                        c_void_p, c_void_p]),
        "dist_sdf_eval": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_int64, c_int,
                                  c_void_p, c_void_p, c_void_p, c_void_p]),
        "dist_loss": (c_int, [c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                              c_void_p, c_void_p, c_void_p, c_int, c_int, POINTER(LossWeights),
                              c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                              c_void_p]),
        "dist_trace_bwd": (c_int, [c_void_p, c_void_p, c_int, POINTER(Camera), c_int,
                                   POINTER(TraceParams), POINTER(TraceOut), c_void_p, c_void_p,
                                   c_void_p, c_void_p, c_void_p, c_void_p]),
        "dist_trace_bwd_camera": (c_int, [c_void_p, c_void_p, c_int, POINTER(Camera), c_int,
                                          POINTER(TraceParams), POINTER(TraceOut), c_void_p,
                                          c_void_p, c_void_p, c_void_p, c_void_p]),
        "dist_render_color": (c_int, [c_void_p, c_void_p, c_int, POINTER(Camera), c_int,
                                      POINTER(TraceOut), c_int, c_void_p, c_void_p, c_void_p]),
        "dist_photo_loss": (c_int, [POINTER(Camera), c_int, c_void_p, c_void_p, c_int, c_void_p,
                                    c_int, c_float, c_void_p, c_void_p, c_void_p, c_void_p]),
        "dist_serve_create": (c_int, [c_void_p, POINTER(TraceParams), c_int64, c_size_t, c_int,
                                      POINTER(c_void_p)]),
        "dist_serve_submit": (c_int, [c_void_p, POINTER(Request), POINTER(c_uint64)]),
        "dist_serve_poll": (c_int, [c_void_p, c_uint64, POINTER(c_int)]),
        "dist_serve_destroy": (c_int, [c_void_p]),
        "dist_last_error": (c_char_p, []),
        "dist_version": (c_char_p, []),
        "dist_sdf_eval_static": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_int64,
                                         c_int, c_void_p, c_void_p, c_void_p]),
        "dist_adam_step": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int,
                                   c_float, c_float, c_float, c_float, c_void_p]),
    }
    for name, (res, args) in sig.items():
        if not hasattr(L, name):
            continue        # tests/test_abi.py requires every declared symbol
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


class DistError(RuntimeError):
    def __init__(self, status, where):
        msg = lib().dist_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status, where):
    if status != DIST_OK:
        raise DistError(status, where)
