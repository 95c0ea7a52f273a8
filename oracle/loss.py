"""Image-plane losses and their per-pixel upstream gradients (float64).

* Depth: L1 over the foreground region given by the rendered silhouette
  (Sec. B.3; Sec. 4.2.1 uses L1 for depth), intersected with the target's
  foreground so that the target depth is finite.
* Normal: negative dot product with the target normal over the same region
  (Sec. B.3).
* Silhouette: L_s = S_gt max(0, S_r) + (1 - S_gt) max(0, -S_r) per pixel
  (Sec. A.3), averaged over all pixels.
* Latent regulariser: ||z||^2 (Sec. B.4, weight 1.0 there).

Reading: each image term is a mean over its region (the paper does not say
mean or sum).  The total is w_d L_d + w_n L_n + w_s L_s + w_r sum ||z||^2.
"""

from __future__ import annotations

import numpy as np


def loss_terms(out, target, w_depth=1.0, w_normal=0.0, w_sil=0.0):
    """Return (loss, g_depth, g_normal (n,3), g_sil) for a rendered ``out``.

    ``target`` holds ``depth`` (inf = background), optional ``normal`` and
    ``sil`` (1 = foreground, 0 = background)."""
    depth, mask = out["depth"], out["mask"]
    n = depth.shape[0]
    gt_d = np.asarray(target["depth"], dtype=np.float64)
    M = mask & np.isfinite(gt_d)
    nM = max(int(M.sum()), 1)
    g_depth = np.zeros(n)
    g_normal = np.zeros((n, 3))
    g_sil = np.zeros(n)
    loss = 0.0
    if w_depth != 0.0:
        r = np.where(M, depth - np.where(M, gt_d, 0.0), 0.0)
        loss += w_depth * np.abs(r).sum() / nM
        g_depth = w_depth * np.sign(r) / nM
    if w_normal != 0.0:
        gt_n = np.asarray(target["normal"], dtype=np.float64)
        dots = np.einsum("ij,ij->i", out["normal"], gt_n)
        loss += w_normal * (-(dots[M]).sum()) / nM
        g_normal = np.where(M[:, None], -w_normal * gt_n / nM, 0.0)
    if w_sil != 0.0:
        S = out["sil"]
        S_gt = np.asarray(target["sil"], dtype=np.float64)
        per = S_gt * np.maximum(0.0, S) + (1.0 - S_gt) * np.maximum(0.0, -S)
        loss += w_sil * per.sum() / n
        g_sil = w_sil * (S_gt * (S > 0) - (1.0 - S_gt) * (S < 0)) / n
    return loss, g_depth, g_normal, g_sil


def regulariser(Z, w_reg):
    """w_r * sum ||z||^2 and its gradient 2 w_r z (Sec. B.4)."""
    Z = np.asarray(Z, dtype=np.float64)
    return w_reg * float((Z * Z).sum()), 2.0 * w_reg * Z
