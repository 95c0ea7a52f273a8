"""Seeded pinhole cameras looking at the origin.

A camera is a plain dict:
``{"fx","fy","cx","cy": float, "R": 3x3 camera-to-world rotation (columns are
the camera's x-right, y-down, z-forward axes in world coordinates, OpenCV
convention), "c": camera centre (3,), "H","W": image size, "shape": latent
index}``.  All floats are float64 numbers that are exactly representable in
float32, so the oracle and the CUDA path see bit-identical cameras.
"""

from __future__ import annotations

import numpy as np


def _f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def look_at_camera(eye, H: int, W: int, fov_deg: float = 50.0, shape: int = 0):
    eye = np.asarray(eye, dtype=np.float64)
    fwd = -eye / np.linalg.norm(eye)
    up = np.array([0.0, 1.0, 0.0])
    if abs(float(fwd @ up)) > 0.99:
        up = np.array([0.0, 0.0, 1.0])
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd], axis=1)
    f = (W / 2.0) / np.tan(np.deg2rad(fov_deg) / 2.0)
    fy = (H / 2.0) / np.tan(np.deg2rad(fov_deg) / 2.0)
    return {
        "fx": float(_f32(f)), "fy": float(_f32(fy)),
        "cx": float(_f32(W / 2.0)), "cy": float(_f32(H / 2.0)),
        "R": _f32(R), "c": _f32(eye), "H": int(H), "W": int(W), "shape": int(shape),
    }


def random_viewpoints(n: int, radius: float = 2.5, seed: int = 0):
    """``n`` camera centres uniform on the sphere of ``radius`` (seeded)."""
    rng = np.random.Generator(np.random.PCG64(20_000 + seed))
    v = rng.standard_normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v * radius


def ring_viewpoints(n: int, radius: float = 2.5, elevation_deg: float = 20.0):
    """``n`` centres at azimuth k*360/n and a fixed elevation."""
    el = np.deg2rad(elevation_deg)
    out = []
    for k in range(n):
        az = 2.0 * np.pi * k / n
        out.append([radius * np.cos(el) * np.sin(az), -radius * np.sin(el),
                    radius * np.cos(el) * np.cos(az)])
    return np.asarray(out)
