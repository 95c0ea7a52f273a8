"""Python binding of libdist: torch tensors in, C-ABI calls out.

Every computation runs in the CUDA library; this module only allocates the
caller-owned output tensors, marshals pointers and checks status codes.
"""

from __future__ import annotations

import ctypes
from ctypes import byref, c_void_p
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np
import torch

from . import _abi
from ._abi import check, lib


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    return c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return c_void_p(s.cuda_stream)


@dataclass
class TraceParams:
    """Mirror of dist_trace_params with the paper's defaults (Sec. 3.2, B.4)."""
    max_steps: int = 50
    eps: float = 5e-5
    alpha: float = 1.5
    k_min: int = 1
    normal_delta: float = 0.0
    grad_mode: str = "exact"      # "exact" | "paper"
    precision: str = "fp32"       # "fp32" | "bf16" | "fp16" | "fp32_tc"
    eps_bf16: float = 1e-3        # low-precision phase threshold (BF16 / FP16)
    radius: float = 1.0
    refine_steps: int = 0         # 0: FP32 convergence; n: accept after n FP32 queries
    alpha_refine: float = 0.0     # step factor of the FP32 phase (0: alpha)
    refine_engine: str = "tc"     # FP32-class queries after the hand-over: "tc" | "simt"
    refine_rule: str = "march"    # their step rule: "march" (alpha) | "secant"
    coarse_levels: int = 0        # coarse-to-fine tracing (Sec. 3.2): 0 off, 2 the paper's
    coarse_every: int = 3         # march iterations per coarse level
    latency_mode: int = 1         # 1: small steps spread each tile over a four-SM cluster
    eps_mid: float = 0.0          # BF16 march: > 0 = an FP16 stage before the FP32-class queries

    def c(self) -> _abi.TraceParams:
        return _abi.TraceParams(
            int(self.max_steps), float(self.eps), float(self.alpha), int(self.k_min),
            float(self.normal_delta),
            _abi.GRAD_EXACT if self.grad_mode == "exact" else _abi.GRAD_PAPER,
            _abi.PRECISIONS[self.precision], float(self.eps_bf16), float(self.radius),
            int(self.refine_steps), float(self.alpha_refine),
            _abi.REFINE_ENGINES[self.refine_engine], _abi.REFINE_RULES[self.refine_rule],
            int(self.coarse_levels), int(self.coarse_every), int(self.latency_mode),
            float(self.eps_mid))


def camera_struct(cam) -> _abi.Camera:
    """A synth-style camera dict -> dist_camera."""
    R = np.asarray(cam["R"], dtype=np.float32).reshape(9)
    c = np.asarray(cam["c"], dtype=np.float32).reshape(3)
    return _abi.Camera(float(cam["fx"]), float(cam["fy"]), float(cam["cx"]), float(cam["cy"]),
                       (ctypes.c_float * 9)(*R.tolist()), (ctypes.c_float * 3)(*c.tolist()),
                       int(cam["H"]), int(cam["W"]), int(cam.get("shape", 0)))


def camera_array(cams: Sequence[dict]):
    arr = (_abi.Camera * len(cams))()
    for i, cam in enumerate(cams):
        arr[i] = camera_struct(cam)
    return arr


class Decoder:
    """Decoder weights uploaded to the device (dist_decoder_create)."""

    def __init__(self, Ws, bs, latent_dim: int, skip: int, latent_dim0: int = 0,
                 out_dim: int = 1):
        Ws = [np.ascontiguousarray(W, dtype=np.float32) for W in Ws]
        bs = [np.ascontiguousarray(b, dtype=np.float32) for b in bs]
        self.latent_dim = int(latent_dim)
        self.latent_dim0 = int(latent_dim0) if latent_dim0 else self.latent_dim
        self.out_dim = int(out_dim)
        self.width = int(Ws[0].shape[0])
        self.n_hidden = len(Ws) - 1
        self.skip = int(skip)
        desc = _abi.DecoderDesc(self.latent_dim, self.width, self.n_hidden, self.skip,
                                self.latent_dim0, self.out_dim)
        Wp = (c_void_p * len(Ws))(*[W.ctypes.data for W in Ws])
        bp = (c_void_p * len(bs))(*[b.ctypes.data for b in bs])
        h = c_void_p()
        check(lib().dist_decoder_create(byref(desc), Wp, bp, byref(h)), "dist_decoder_create")
        self._keep = (Ws, bs)
        self.handle = h

    @classmethod
    def from_spec(cls, spec, Ws, bs):
        return cls(Ws, bs, spec.latent_dim, spec.skip)

    @property
    def has_bf16(self) -> bool:
        return bool(lib().dist_decoder_has_bf16(self.handle))

    def device_error(self) -> int:
        """Synchronise and return (then clear) the tensor-core kernels' error
        word (0: no wait ran out and no FP16 overflow since the last call)."""
        code = ctypes.c_int32(0)
        st = lib().dist_decoder_device_error(self.handle, byref(code))
        if st != _abi.DIST_E_TIMEOUT:
            check(st, "dist_decoder_device_error")
        return int(code.value)

    def set_wait_limit(self, wait_ns: int = 1_000_000_000, withhold_copies: bool = False) -> None:
        """Limit of the tensor-core forward kernel's waits; withhold_copies
        (tests of the failure path) makes its weight loader issue nothing."""
        check(lib().dist_decoder_set_wait_limit(self.handle, int(wait_ns), int(bool(withhold_copies))),
              "dist_decoder_set_wait_limit")

    def close(self):
        if self.handle:
            lib().dist_decoder_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Workspace:
    """Device scratch for up to ``max_rays`` pixels (dist_workspace_create)."""

    def __init__(self, max_rays: int, max_steps: int = 100):
        h = c_void_p()
        check(lib().dist_workspace_create(int(max_rays), int(max_steps), byref(h)),
              "dist_workspace_create")
        self.handle = h
        self.max_rays = int(max_rays)
        self.max_steps = int(max_steps)

    def close(self):
        if self.handle:
            lib().dist_workspace_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class TraceResult:
    depth: torch.Tensor
    sil: torch.Tensor
    mask: torch.Tensor
    steps: torch.Tensor
    status: torch.Tensor
    d_hit: torch.Tensor
    d_min: torch.Tensor
    f_min: torch.Tensor
    normal: Optional[torch.Tensor]
    queries: torch.Tensor
    grad_len: Optional[torch.Tensor] = None   # |central-difference gradient| beside `normal`
    _c: _abi.TraceOut = field(default=None, repr=False)

    def c(self) -> _abi.TraceOut:
        return _abi.TraceOut(_ptr(self.depth), _ptr(self.sil), _ptr(self.mask), _ptr(self.steps),
                             _ptr(self.status), _ptr(self.d_hit), _ptr(self.d_min),
                             _ptr(self.f_min), _ptr(self.normal), _ptr(self.queries),
                             _ptr(self.grad_len))


def n_pixels(cams) -> int:
    return int(sum(int(c["H"]) * int(c["W"]) for c in cams))


def alloc_result(n: int, k_min: int, device, normals: bool) -> TraceResult:
    f = dict(device=device, dtype=torch.float32)
    return TraceResult(
        depth=torch.empty(n, **f), sil=torch.empty(n, **f),
        mask=torch.empty(n, device=device, dtype=torch.uint8),
        steps=torch.empty(n, device=device, dtype=torch.int32),
        status=torch.empty(n, device=device, dtype=torch.int32),
        d_hit=torch.empty(n, **f), d_min=torch.empty(n, k_min, **f),
        f_min=torch.empty(n, k_min, **f),
        normal=torch.empty(n, 3, **f) if normals else None,
        queries=torch.zeros(2, device=device, dtype=torch.int64),
        grad_len=torch.empty(n, **f) if normals else None)


def trace(dec: Decoder, z: torch.Tensor, cams, params: TraceParams, ws: Workspace,
          normals: bool = False, out: Optional[TraceResult] = None, stream=None,
          cam_c=None) -> TraceResult:
    """dist_trace_fwd: render depth / silhouette / mask (and normals)."""
    z = z.contiguous()
    assert z.dtype == torch.float32 and z.is_cuda
    n = n_pixels(cams)
    if out is None:
        out = alloc_result(n, params.k_min, z.device, normals)
    cam_c = cam_c if cam_c is not None else camera_array(cams)
    p = params.c()
    o = out.c()
    check(lib().dist_trace_fwd(dec.handle, _ptr(z), int(z.shape[0]), cam_c, len(cams),
                               byref(p), byref(o), ws.handle, _stream(stream)),
          "dist_trace_fwd")
    return out


def sdf_eval(dec: Decoder, z: torch.Tensor, pts: torch.Tensor, shape: torch.Tensor,
             ws: Workspace, precision: str = "fp32", grad: bool = False, stream=None):
    """dist_sdf_eval: f (and grad_p f) at points ``pts`` [n, 3] with latent ``shape`` [n]."""
    pts = pts.contiguous().float()
    shape = shape.contiguous().to(torch.int32)
    n = pts.shape[0]
    f = torch.empty(n, device=pts.device, dtype=torch.float32)
    g = torch.empty(n, 3, device=pts.device, dtype=torch.float32) if grad else None
    prec = _abi.PRECISIONS[precision]
    check(lib().dist_sdf_eval(dec.handle, _ptr(z.contiguous()), int(z.shape[0]), _ptr(pts),
                              _ptr(shape), n, prec, _ptr(f), _ptr(g), ws.handle, _stream(stream)),
          "dist_sdf_eval")
    return (f, g) if grad else f


def render_normals(dec: Decoder, z: torch.Tensor, cams, params: TraceParams, ws: Workspace,
                   fwd: TraceResult, stream=None) -> torch.Tensor:
    n = n_pixels(cams)
    normal = torch.empty(n, 3, device=z.device, dtype=torch.float32)
    p = params.c()
    o = fwd.c()
    check(lib().dist_render_normals(dec.handle, _ptr(z.contiguous()), int(z.shape[0]),
                                    camera_array(cams), len(cams), byref(p), byref(o), _ptr(normal),
                                    ws.handle, _stream(stream)), "dist_render_normals")
    return normal


def loss(fwd: TraceResult, target: dict, z: torch.Tensor, ws: Workspace, w_depth=1.0,
         w_normal=0.0, w_sil=0.0, w_reg=0.0, stream=None):
    """dist_loss: returns (loss (float64 device scalar), g_depth, g_normal, g_sil, dz)."""
    n = fwd.depth.shape[0]
    dev = fwd.depth.device
    g_depth = torch.empty(n, device=dev, dtype=torch.float32)
    g_normal = torch.empty(n, 3, device=dev, dtype=torch.float32) if w_normal else None
    g_sil = torch.empty(n, device=dev, dtype=torch.float32) if w_sil else None
    dz = torch.zeros_like(z)
    L = torch.empty(1, device=dev, dtype=torch.float64)
    w = _abi.LossWeights(float(w_depth), float(w_normal), float(w_sil), float(w_reg))
    check(lib().dist_loss(n, _ptr(fwd.depth), _ptr(fwd.mask), _ptr(fwd.sil), _ptr(fwd.normal),
                          _ptr(target["depth"]), _ptr(target.get("normal")),
                          _ptr(target.get("sil")), _ptr(z), int(z.shape[0]), int(z.shape[1]),
                          byref(w), _ptr(L), _ptr(g_depth), _ptr(g_normal), _ptr(g_sil),
                          _ptr(dz), ws.handle, _stream(stream)), "dist_loss")
    return L, g_depth, g_normal, g_sil, dz


def backward(dec: Decoder, z: torch.Tensor, cams, params: TraceParams, ws: Workspace,
             fwd: TraceResult, g_depth=None, g_normal=None, g_sil=None,
             dz: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """dist_trace_bwd: dL/dz accumulated into ``dz`` (zeros if None)."""
    z = z.contiguous()
    if dz is None:
        dz = torch.zeros_like(z)
    p = params.c()
    o = fwd.c()
    check(lib().dist_trace_bwd(dec.handle, _ptr(z), int(z.shape[0]), camera_array(cams),
                               len(cams), byref(p), byref(o), _ptr(g_depth), _ptr(g_normal),
                               _ptr(g_sil), _ptr(dz), ws.handle, _stream(stream)),
          "dist_trace_bwd")
    return dz


def backward_camera(dec: Decoder, z: torch.Tensor, cams, params: TraceParams, ws: Workspace,
                    fwd: TraceResult, g_depth=None, g_sil=None, stream=None) -> torch.Tensor:
    """dist_trace_bwd_camera: [n_cams, 12] = dL/dc (3) and dL/dR row-major (9)."""
    z = z.contiguous()
    out = torch.empty(len(cams), 12, device=z.device, dtype=torch.float32)
    p = params.c()
    o = fwd.c()
    check(lib().dist_trace_bwd_camera(dec.handle, _ptr(z), int(z.shape[0]), camera_array(cams),
                                      len(cams), byref(p), byref(o), _ptr(g_depth), _ptr(g_sil),
                                      _ptr(out), ws.handle, _stream(stream)),
          "dist_trace_bwd_camera")
    return out


def photo_loss(cams, depth: torch.Tensor, images: torch.Tensor, pairs, ws: Workspace,
               w: float = 1.0, stream=None):
    """dist_photo_loss: (loss (float64 device scalar), g_depth [n])."""
    depth = depth.contiguous().float()
    images = images.contiguous().float()
    n = depth.shape[0]
    channels = images.numel() // n
    pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    loss = torch.empty(1, device=depth.device, dtype=torch.float64)
    g = torch.empty(n, device=depth.device, dtype=torch.float32)
    check(lib().dist_photo_loss(camera_array(cams), len(cams), _ptr(depth), _ptr(images),
                                int(channels), pr.ctypes.data_as(ctypes.c_void_p), int(pr.shape[0]),
                                float(w), _ptr(loss), _ptr(g), ws.handle, _stream(stream)),
          "dist_photo_loss")
    return loss, g


def render_color(tex: Decoder, codes: torch.Tensor, cams, fwd: "TraceResult", ws: Workspace,
                 precision: str = "bf16", stream=None) -> torch.Tensor:
    """dist_render_color: [n, 3] colour of the hit pixels of ``fwd`` (0 elsewhere)."""
    codes = codes.contiguous().float()
    n = fwd.depth.shape[0]
    rgb = torch.empty(n, 3, device=codes.device, dtype=torch.float32)
    o = fwd.c()
    check(lib().dist_render_color(tex.handle, _ptr(codes), int(codes.shape[0]), camera_array(cams),
                                  len(cams), byref(o), _abi.PRECISIONS[precision], _ptr(rgb),
                                  ws.handle, _stream(stream)),
          "dist_render_color")
    return rgb


class DistRender(torch.autograd.Function):
    """Differentiable render: z -> (depth, silhouette[, normal]).

    Forward is dist_trace_fwd (normals when ``params.normal_delta`` is used
    by the caller's loss); backward is dist_trace_bwd with the incoming
    gradients."""

    @staticmethod
    def forward(ctx, z, dec, cams, params, ws, with_normals=False):
        res = trace(dec, z, cams, params, ws, normals=with_normals)
        ctx.save_for_backward(z)
        ctx.res, ctx.dec, ctx.cams, ctx.params, ctx.ws = res, dec, cams, params, ws
        ctx.mark_non_differentiable(res.mask)
        outs = (res.depth, res.sil, res.mask)
        if with_normals:
            outs = outs + (res.normal,)
        return outs

    @staticmethod
    def backward(ctx, g_depth, g_sil, _g_mask, g_normal=None):
        (z,) = ctx.saved_tensors
        gd = None if g_depth is None else torch.nan_to_num(g_depth.contiguous(), 0.0, 0.0, 0.0)
        gs = None if g_sil is None else g_sil.contiguous()
        gn = None if g_normal is None else g_normal.contiguous()
        if gn is not None and ctx.params.normal_delta <= 0:
            gn = None
        dz = backward(ctx.dec, z, ctx.cams, ctx.params, ctx.ws, ctx.res, gd, gn, gs)
        return dz, None, None, None, None, None


def render(z, dec, cams, params, ws, with_normals=False):
    return DistRender.apply(z, dec, cams, params, ws, with_normals)
