"""Python binding of the continuous-batching render server (dist_serve_*).

Marshalling only: the server loop, batching and all compute live in
libdist.so.  Result buffers are numpy arrays owned by the Ticket until the
request is polled done.
"""

from __future__ import annotations

import ctypes
import time
from ctypes import byref, c_int, c_uint64, c_void_p

import numpy as np

from . import _abi
from ._abi import check, lib
from .api import camera_struct


class Ticket:
    def __init__(self, ticket, cam, kind, z, tgt, L):
        n = int(cam["H"]) * int(cam["W"])
        self.id = ticket
        self.kind = kind
        self.n = n
        self.z = np.ascontiguousarray(z, dtype=np.float32)
        self.tgt = None if tgt is None else np.ascontiguousarray(tgt, dtype=np.float32)
        self.depth = np.empty(n, dtype=np.float32)
        self.sil = np.empty(n, dtype=np.float32)
        self.mask = np.empty(n, dtype=np.uint8)
        self.dz = np.zeros(L, dtype=np.float32)
        self.loss = np.zeros(1, dtype=np.float64)
        self.t_submit = time.perf_counter()
        self.t_done = None
        self.done = False


class Server:
    """dist_serve_create / submit / poll / destroy."""

    def __init__(self, dec, params, max_rays: int, mem_budget: int, max_requests: int = 64):
        self.dec = dec
        self.L = dec.latent_dim
        h = c_void_p()
        p = params.c()
        check(lib().dist_serve_create(dec.handle, byref(p), int(max_rays), int(mem_budget),
                                      int(max_requests), byref(h)), "dist_serve_create")
        self.handle = h
        self.live = {}

    def submit(self, cam, z, kind: str = "render", tgt_depth=None) -> Ticket:
        k = _abi.REQ_RENDER if kind == "render" else _abi.REQ_RENDER_BACKWARD
        t = Ticket(0, cam, k, z, tgt_depth, self.L)
        req = _abi.Request()
        req.kind = k
        req.cam = camera_struct(cam)
        req.z = t.z.ctypes.data
        req.tgt_depth = t.tgt.ctypes.data if t.tgt is not None else None
        req.depth = t.depth.ctypes.data
        req.sil = t.sil.ctypes.data
        req.mask = t.mask.ctypes.data
        req.dz = t.dz.ctypes.data if k == _abi.REQ_RENDER_BACKWARD else None
        req.loss = t.loss.ctypes.data if k == _abi.REQ_RENDER_BACKWARD else None
        tid = c_uint64()
        check(lib().dist_serve_submit(self.handle, byref(req), byref(tid)), "dist_serve_submit")
        t.id = tid.value
        self.live[t.id] = t
        return t

    def poll(self, t: Ticket) -> bool:
        if t.done:
            return True
        d = c_int(0)
        check(lib().dist_serve_poll(self.handle, c_uint64(t.id), byref(d)), "dist_serve_poll")
        if d.value:
            t.done = True
            t.t_done = time.perf_counter()
            self.live.pop(t.id, None)
        return t.done

    def wait(self, t: Ticket, timeout: float = 60.0, sleep: float = 2e-4) -> Ticket:
        t0 = time.perf_counter()
        while not self.poll(t):
            if time.perf_counter() - t0 > timeout:
                raise TimeoutError(f"request {t.id} not done after {timeout} s")
            time.sleep(sleep)
        return t

    def close(self):
        if self.handle:
            check(lib().dist_serve_destroy(self.handle), "dist_serve_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
