"""Pixel-centre camera rays and the depth conversion (float64).

* One ray per pixel, shot through the pixel centre (Sec. A.4 "Drawbacks"
  names the single pixel-centre ray as the source of aliasing), so pixel
  (x, y) uses image coordinates (x + 0.5, y + 0.5).
* (x~, y~, 1)^T = K^{-1} (x, y, 1)^T is the normalised homogeneous coordinate
  and the depth of a point at ray distance d is z_c = d / sqrt(x~^2 + y~^2 + 1)
  (Sec. 3.3, "Depth and Surface Normal").
* The ray direction is the unit vector along (x~, y~, 1) rotated to world
  coordinates by the camera-to-world rotation R and renormalised (R arrives
  rounded to float32, so it is orthonormal only to ~1e-8); the ray is
  c + d v with d the Euclidean distance from c (Alg. 1).
"""

from __future__ import annotations

import numpy as np


def pixel_rays(cam):
    """Return (c (3,), v (H*W, 3) world unit directions, inv_norm (H*W,)).

    ``inv_norm`` = 1 / sqrt(x~^2 + y~^2 + 1), so depth = d * inv_norm.
    Pixels are ordered row-major: index = y * W + x.
    """
    H, W = int(cam["H"]), int(cam["W"])
    ys, xs = np.meshgrid(np.arange(H, dtype=np.float64),
                         np.arange(W, dtype=np.float64), indexing="ij")
    xt = (xs.ravel() + 0.5 - cam["cx"]) / cam["fx"]
    yt = (ys.ravel() + 0.5 - cam["cy"]) / cam["fy"]
    norm = np.sqrt(xt * xt + yt * yt + 1.0)
    v_cam = np.stack([xt, yt, np.ones_like(xt)], axis=1) / norm[:, None]
    R = np.asarray(cam["R"], dtype=np.float64)
    v = v_cam @ R.T
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return np.asarray(cam["c"], dtype=np.float64), v, 1.0 / norm


def depth_from_distance(d, inv_norm):
    """z_c = d / sqrt(x~^2 + y~^2 + 1) (Sec. 3.3)."""
    return d * inv_norm


def epsilon_from_camera(d_min, sensor, focal, resolution, theta=0.0):
    """Convergence threshold from camera geometry (Sec. A.2):
    eps = d_min * S * cos^2(theta) / (2 f R)."""
    return d_min * sensor * np.cos(theta) ** 2 / (2.0 * focal * resolution)
