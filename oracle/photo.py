"""Multi-view photometric loss (Sec. 4.2 multi-view reconstruction, Sec. B.3
visibility), float64.

For each ordered pair (i, j) of views, every pixel x of view i that the
renderer hit is lifted to the world point P = c_i + d v_i(x) with d its ray
distance (depth / inv_norm), projected into view j, and image j is sampled
there bilinearly: I_{j->i}(x).  The loss is the L1 colour difference
|I_i(x) - I_{j->i}(x)| (summed over the colour channels) over the pixels
visible in both views.  Visibility (Sec. B.3): the depth of P in view j
against view j's rendered depth interpolated at the projection, visible when
the squared difference is below 1e-3.

Readings (the paper gives the equation and the threshold only):
  * pixel centres at (x + 1/2, y + 1/2) (as for the rays); bilinear
    interpolation between the four neighbouring pixel centres, and a
    projection whose four neighbours are not all inside the image, or not all
    hit in view j, is not visible;
  * the loss is the mean over the visible pixels of all pairs (the other
    image losses are means too); with no visible pixel it is 0;
  * the visibility test and the rendered depth of view j are constants of the
    derivative; the gradient flows into view i's depth through the projection
    (bilinear interpolation is differentiated within its cell).
"""

from __future__ import annotations

import numpy as np

from .camera import pixel_rays

VIS_THRESH = 1e-3


def _bilinear(img, u, v):
    """Sample img [H, W, C] at image coordinates (u, v) (pixel centres at
    k + 1/2): values [n, C], derivatives d/du and d/dv [n, C], and validity."""
    H, W = img.shape[:2]
    x = u - 0.5
    y = v - 0.5
    x0 = np.floor(x).astype(np.int64)
    y0 = np.floor(y).astype(np.int64)
    ok = (x0 >= 0) & (y0 >= 0) & (x0 <= W - 2) & (y0 <= H - 2)
    x0c = np.clip(x0, 0, W - 2)
    y0c = np.clip(y0, 0, H - 2)
    fx = (x - x0c)[:, None]
    fy = (y - y0c)[:, None]
    i00 = img[y0c, x0c]
    i01 = img[y0c, x0c + 1]
    i10 = img[y0c + 1, x0c]
    i11 = img[y0c + 1, x0c + 1]
    val = (1 - fy) * ((1 - fx) * i00 + fx * i01) + fy * ((1 - fx) * i10 + fx * i11)
    du = (1 - fy) * (i01 - i00) + fy * (i11 - i10)
    dv = (1 - fx) * (i10 - i00) + fx * (i11 - i01)
    return val, du, dv, ok


def warp_loss(cams, depths, images, pairs, w=1.0, vis_thresh=VIS_THRESH):
    """Return (loss, [g_depth per view], [visible mask per pair]).

    ``depths[i]`` is view i's rendered depth (H*W, inf = background),
    ``images[i]`` its colour image (H, W, C), ``pairs`` a list of (i, j)."""
    rays = [pixel_rays(cam) for cam in cams]
    g = [np.zeros_like(np.asarray(d, dtype=np.float64)) for d in depths]
    terms, vis_all = [], []
    total = 0
    for (i, j) in pairs:
        ci, vi, invi = rays[i]
        cj = np.asarray(cams[j]["c"], dtype=np.float64)
        Rj = np.asarray(cams[j]["R"], dtype=np.float64)
        Di = np.asarray(depths[i], dtype=np.float64)
        hit = np.isfinite(Di)
        idx = np.nonzero(hit)[0]
        d = Di[idx] / invi[idx]
        P = ci + d[:, None] * vi[idx]
        pc = (P - cj) @ Rj                    # R^T (P - c_j), row vectors
        q = vi[idx] @ Rj                      # dp/dd
        front = pc[:, 2] > 1e-9
        pz = np.where(front, pc[:, 2], 1.0)
        fx_, fy_, cx_, cy_ = (float(cams[j][k]) for k in ("fx", "fy", "cx", "cy"))
        u = fx_ * pc[:, 0] / pz + cx_
        v = fy_ * pc[:, 1] / pz + cy_
        Hj, Wj = int(cams[j]["H"]), int(cams[j]["W"])
        Dj = np.asarray(depths[j], dtype=np.float64).reshape(Hj, Wj, 1)
        Ij = np.asarray(images[j], dtype=np.float64)
        Ii = np.asarray(images[i], dtype=np.float64).reshape(-1, Ij.shape[2])
        # clip the sample points so that the lookups stay inside (masked below)
        us = np.where(front, u, 0.0)
        vs = np.where(front, v, 0.0)
        dval, _, _, okd = _bilinear(np.where(np.isfinite(Dj), Dj, 0.0), us, vs)
        # all four neighbours hit in view j
        yy = np.clip(np.floor(vs - 0.5).astype(np.int64), 0, Hj - 2)
        xx = np.clip(np.floor(us - 0.5).astype(np.int64), 0, Wj - 2)
        fin = np.isfinite(Dj[..., 0])
        allfin = fin[yy, xx] & fin[yy, xx + 1] & fin[yy + 1, xx] & fin[yy + 1, xx + 1]
        vis = front & okd & allfin & ((pc[:, 2] - dval[:, 0]) ** 2 < vis_thresh)
        val, du, dv, _ = _bilinear(Ij, us, vs)
        r = Ii[idx] - val
        terms.append(np.where(vis, np.abs(r).sum(axis=1), 0.0))
        total += int(vis.sum())
        # d(loss term)/dd = sum_c sign(r_c) * -(dI/du du/dd + dI/dv dv/dd)
        dudd = fx_ * (q[:, 0] * pz - pc[:, 0] * q[:, 2]) / (pz * pz)
        dvdd = fy_ * (q[:, 1] * pz - pc[:, 1] * q[:, 2]) / (pz * pz)
        dterm = -(np.sign(r) * (du * dudd[:, None] + dv * dvdd[:, None])).sum(axis=1)
        gi = np.zeros_like(Di)
        gi[idx] = np.where(vis, dterm / invi[idx], 0.0)   # d(term)/d depth_i
        g[i] = g[i] + gi
        vmask = np.zeros(Di.shape, dtype=bool)
        vmask[idx] = vis
        vis_all.append(vmask)
    if total == 0:
        return 0.0, [np.zeros_like(x) for x in g], vis_all
    loss = w * float(sum(t.sum() for t in terms)) / total
    g = [w * x / total for x in g]
    return loss, g, vis_all
