"""Inverse optimisation of latent codes through the renderer (Sec. 4.2: shape
from depth (and normal) maps by optimising z with Adam; Sec. B.4: lr 1e-2,
z initialised to 0; Sec. B.3: depth and normal losses over the rendered
foreground).

One step runs every shape and view of the batch through the library once:
dist_trace_fwd (with central-difference normals when the normal loss is on),
dist_loss, dist_trace_bwd and dist_adam_step, all stream-ordered on the
device with preallocated buffers (no host synchronisation inside a step).

The optimiser state (z, Adam moments m and v, step count t, hyper-
parameters) saves to and loads from an .npz file; the step is a function of
that state and the fixed inputs alone, so a run resumed from a checkpoint
continues bit for bit like the uninterrupted run.  Marshalling only: every
computation is in libdist.
"""

from __future__ import annotations

from ctypes import byref, c_void_p
from typing import Optional, Sequence

import numpy as np
import torch

from . import _abi, api
from ._abi import check, lib


def _p(t):
    return None if t is None else c_void_p(t.data_ptr())


def adam_step(z: torch.Tensor, dz: torch.Tensor, m: torch.Tensor, v: torch.Tensor, t: int,
              lr: float = 1e-2, betas=(0.9, 0.999), eps: float = 1e-8, stream=None) -> None:
    """dist_adam_step: z, m, v updated in place (step number t, from 1)."""
    for x in (z, dz, m, v):
        assert x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()
    s = stream if stream is not None else torch.cuda.current_stream()
    check(lib().dist_adam_step(_p(z), _p(dz), _p(m), _p(v), int(z.numel()), int(t), float(lr),
                               float(betas[0]), float(betas[1]), float(eps),
                               c_void_p(s.cuda_stream)), "dist_adam_step")


class InverseProblem:
    """Latent codes of ``n_shapes`` shapes from target depth (and normal) maps
    of their views.  ``cams`` are synth-style camera dicts (each names its
    shape); targets are device tensors over the concatenated pixels."""

    STATE_KEYS = ("z", "m", "v", "t", "lr", "beta1", "beta2", "eps", "w_depth", "w_normal")

    def __init__(self, dec: api.Decoder, cams: Sequence[dict], n_shapes: int,
                 tgt_depth: torch.Tensor, tgt_normal: Optional[torch.Tensor] = None,
                 params: Optional[api.TraceParams] = None, ws: Optional[api.Workspace] = None,
                 lr: float = 1e-2, betas=(0.9, 0.999), eps: float = 1e-8,
                 w_depth: float = 10.0, w_normal: float = 1.0, z0: Optional[torch.Tensor] = None):
        self.dec, self.cams = dec, list(cams)
        self.params = params if params is not None else api.TraceParams(precision="bf16")
        self.w_depth = float(w_depth)
        self.w_normal = float(w_normal) if tgt_normal is not None else 0.0
        if self.w_normal and self.params.normal_delta <= 0:
            raise ValueError("a normal loss needs central-difference normals (normal_delta > 0)")
        n = api.n_pixels(self.cams)
        self.ws = ws if ws is not None else api.Workspace(n, self.params.max_steps)
        dev = tgt_depth.device
        L = dec.latent_dim
        self.z = (z0.clone().float().contiguous() if z0 is not None
                  else torch.zeros(n_shapes, L, device=dev, dtype=torch.float32))
        self.m = torch.zeros_like(self.z)
        self.v = torch.zeros_like(self.z)
        self.t = 0
        self.lr, self.beta1, self.beta2, self.eps = float(lr), float(betas[0]), float(betas[1]), \
            float(eps)
        self.tgt_depth = tgt_depth.contiguous().float()
        self.tgt_normal = tgt_normal.contiguous().float() if tgt_normal is not None else None
        # preallocated per-step buffers and C structs
        self.res = api.alloc_result(n, self.params.k_min, dev, normals=self.w_normal > 0)
        self.g_depth = torch.empty(n, device=dev, dtype=torch.float32)
        self.g_normal = torch.empty(n, 3, device=dev, dtype=torch.float32) \
            if self.w_normal else None
        self.dz = torch.zeros_like(self.z)
        self.loss = torch.zeros(1, device=dev, dtype=torch.float64)
        self._cams = api.camera_array(self.cams)
        self._p = self.params.c()
        self._o = self.res.c()
        self._w = _abi.LossWeights(self.w_depth, self.w_normal, 0.0, 0.0)
        self.n = n

    def step(self, stream=None) -> torch.Tensor:
        """One Adam step; returns the loss before the update (device float64 [1])."""
        L = lib()
        s = stream if stream is not None else torch.cuda.current_stream()
        sp = c_void_p(s.cuda_stream)
        ns = int(self.z.shape[0])
        check(L.dist_trace_fwd(self.dec.handle, _p(self.z), ns, self._cams, len(self.cams),
                               byref(self._p), byref(self._o), self.ws.handle, sp),
              "dist_trace_fwd")
        check(L.dist_loss(self.n, _p(self.res.depth), _p(self.res.mask), _p(self.res.sil),
                          _p(self.res.normal), _p(self.tgt_depth), _p(self.tgt_normal), None,
                          _p(self.z), ns, int(self.z.shape[1]), byref(self._w), _p(self.loss),
                          _p(self.g_depth), _p(self.g_normal), None, _p(self.dz),
                          self.ws.handle, sp), "dist_loss")
        check(L.dist_trace_bwd(self.dec.handle, _p(self.z), ns, self._cams, len(self.cams),
                               byref(self._p), byref(self._o), _p(self.g_depth),
                               _p(self.g_normal), None, _p(self.dz), self.ws.handle, sp),
              "dist_trace_bwd")
        self.t += 1
        adam_step(self.z, self.dz, self.m, self.v, self.t, self.lr, (self.beta1, self.beta2),
                  self.eps, stream=s)
        return self.loss

    # -------------------------------------------------------- checkpoint

    def state_dict(self) -> dict:
        torch.cuda.current_stream().synchronize()
        return {"z": self.z.cpu().numpy(), "m": self.m.cpu().numpy(), "v": self.v.cpu().numpy(),
                "t": np.int64(self.t), "lr": np.float64(self.lr),
                "beta1": np.float64(self.beta1), "beta2": np.float64(self.beta2),
                "eps": np.float64(self.eps), "w_depth": np.float64(self.w_depth),
                "w_normal": np.float64(self.w_normal)}

    def load_state_dict(self, st: dict) -> None:
        z = np.asarray(st["z"], dtype=np.float32)
        if z.shape != tuple(self.z.shape):
            raise ValueError(f"checkpoint z has shape {z.shape}, problem has {tuple(self.z.shape)}")
        if float(st["w_depth"]) != self.w_depth or float(st["w_normal"]) != self.w_normal:
            raise ValueError("checkpoint loss weights differ from this problem's")
        dev = self.z.device
        self.z.copy_(torch.from_numpy(z).to(dev))
        self.m.copy_(torch.from_numpy(np.asarray(st["m"], dtype=np.float32)).to(dev))
        self.v.copy_(torch.from_numpy(np.asarray(st["v"], dtype=np.float32)).to(dev))
        self.t = int(st["t"])
        self.lr, self.beta1, self.beta2, self.eps = (float(st["lr"]), float(st["beta1"]),
                                                     float(st["beta2"]), float(st["eps"]))
        torch.cuda.current_stream().synchronize()

    def save(self, path: str) -> None:
        np.savez(path, **self.state_dict())

    def load(self, path: str) -> None:
        with np.load(path) as f:
            self.load_state_dict({k: f[k] for k in self.STATE_KEYS})
