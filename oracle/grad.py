"""Latent-code and camera gradients of the rendered observations (float64).

Given per-pixel upstream gradients (dL/d depth, dL/d normal, dL/d silhouette),
return dL/dz for every latent code.

Depth, two modes:

* ``exact`` (default): implicit differentiation at the hit point
  p = c + d v, where f(p(z), z) = 0 defines d(z):
  dd/dz = -(df/dz) / (grad_p f . v), and dz_c/dz = dd/dz / sqrt(x~^2+y~^2+1)
  (Sec. 3.3 depth formula).  This is the derivative of the converged root; it
  differs from the traced distance only by the convergence residual (|f| <
  eps).  Rays whose |grad_p f . v| < 1e-3 |grad_p f| (grazing) get zero
  gradient (reading: the implicit form is singular there).
* ``paper``: the approximation of Sec. 3.4 -- keep only the first term of
  Eq. 2, drop the residual e of Eq. 1, and sum over the K samples of the ray
  with the smallest |f| (Sec. B.2, K in Sec. B.4):
  dd/dz ~= alpha * sum_k df(p_k, z)/dz with p_k held fixed.
  Parity unpinned as an approximation (no reference values exist); its
  arithmetic is pinned on an analytic SDF.

Silhouette (Sec. A.3): S = min_n |f(p_n)| - eps, so dS/dz = sign(f(p_min))
df(p_min, z)/dz with p_min held fixed (the first-term rule of Sec. 3.4).  Rays
that miss the bounding sphere have S = dist - 1, independent of z.

Normal (Sec. 3.3): with the central-difference normal of step delta > 0,
n = g/|g|, g_a = (f(p + delta e_a) - f(p - delta e_a)) / (2 delta), and the
vector-Jacobian product is taken with the hit point p held fixed.  With the
analytic normal (delta = 0) of a ReLU decoder, the normalised gradient is
piecewise constant in z, so its gradient is zero almost everywhere.
"""

from __future__ import annotations

import numpy as np


def _accumulate(out_shape_grad, shapes, weights, jac):
    for s in np.unique(shapes):
        sel = shapes == s
        out_shape_grad[s] += (weights[sel, None] * jac[sel]).sum(axis=0)


def latent_vjp(sdf, out, n_shapes, latent_dim, g_depth=None, g_normal=None,
               g_sil=None, mode="exact", normal_delta=0.0, grazing=1e-3):
    """dL/dz (n_shapes, latent_dim) from per-pixel upstream gradients."""
    G = np.zeros((n_shapes, latent_dim))
    shape = out["shape"]
    v = out["v"]
    c = out["c"]
    hit = out["mask"]
    if g_depth is not None and np.any(g_depth[hit] != 0.0):
        idx = np.nonzero(hit & (g_depth != 0.0))[0]
        if mode == "exact":
            p = out["p_hit"][idx]
            _, gp, gz = sdf.grad(p, shape[idx])
            gv = np.einsum("ij,ij->i", gp, v[idx])
            ok = np.abs(gv) >= grazing * np.linalg.norm(gp, axis=1)
            dd_dz = np.where(ok[:, None], -gz / np.where(ok, gv, 1.0)[:, None], 0.0)
        elif mode == "paper":
            alpha = out["alpha"]
            dd_dz = np.zeros((idx.size, latent_dim))
            K = out["topk_d"].shape[1]
            for k in range(K):
                dk = out["topk_d"][idx, k]
                have = np.isfinite(dk)
                if not np.any(have):
                    continue
                p = c[idx[have]] + dk[have, None] * v[idx[have]]
                _, _, gz = sdf.grad(p, shape[idx[have]])
                dd_dz[have] += alpha * gz
        else:
            raise ValueError(mode)
        jac = out["inv_norm"][idx, None] * dd_dz
        _accumulate(G, shape[idx], g_depth[idx], jac)
    if g_sil is not None and np.any(g_sil[out["enters"]] != 0.0):
        idx = np.nonzero(out["enters"] & (g_sil != 0.0))[0]
        p = c[idx] + out["d_at_min"][idx, None] * v[idx]
        _, _, gz = sdf.grad(p, shape[idx])
        jac = np.sign(out["f_at_min"][idx])[:, None] * gz
        _accumulate(G, shape[idx], g_sil[idx], jac)
    if g_normal is not None and normal_delta > 0.0 and np.any(g_normal[hit] != 0.0):
        idx = np.nonzero(hit & np.any(g_normal != 0.0, axis=1))[0]
        p = out["p_hit"][idx]
        fp = np.zeros((idx.size, 3)); fm = np.zeros((idx.size, 3))
        jp = []; jm = []
        for a in range(3):
            e = np.zeros(3); e[a] = normal_delta
            f1, _, z1 = sdf.grad(p + e, shape[idx])
            f2, _, z2 = sdf.grad(p - e, shape[idx])
            fp[:, a] = f1; fm[:, a] = f2
            jp.append(z1); jm.append(z2)
        g = (fp - fm) / (2.0 * normal_delta)
        gn = np.linalg.norm(g, axis=1, keepdims=True)
        nrm = g / gn
        up = g_normal[idx]
        dL_dg = (up - nrm * np.einsum("ij,ij->i", nrm, up)[:, None]) / gn
        for a in range(3):
            jac = (jp[a] - jm[a]) / (2.0 * normal_delta)
            _accumulate(G, shape[idx], dL_dg[:, a], jac)
    return G


# -- camera extrinsics -----------------------------------------------------------
#
# The paper optimises the camera pose through the renderer with the shape
# fixed, from a depth map and a binary silhouette (Sec. 4.2 "Back-Propagation
# Effectiveness").  The camera enters each ray through its centre c and its
# direction v = u / |u|, u = R v_cam (v_cam the unit pixel direction in the
# camera frame, fixed by the intrinsics).  Readings:
#   * depth: the exact implicit derivative of the converged root,
#     f(c + d v) = 0  =>  dd = -(grad_p f . (dc + d dv)) / (grad_p f . v),
#     z_c = d / sqrt(x~^2 + y~^2 + 1); grazing rays (|grad f . v| <
#     1e-3 |grad f|) get zero gradient, as for the latent;
#   * silhouette of a ray that entered the bounding sphere: S = |f(p_min)| -
#     eps with the sample's ray distance d_min held fixed and the point moving
#     with the camera (the first-term rule of Sec. 3.4):
#     dS = sign(f_min) grad_p f(p_min) . (dc + d_min dv);
#   * silhouette of a ray that misses the sphere: S = dist(origin, ray) -
#     radius, differentiated exactly (Sec. A.3);
#   * R is treated as a free 3 x 3 matrix: dL/du = (I - v v^T) dL/dv / |u|,
#     dL/dR = dL/du v_cam^T.

def camera_vjp(sdf, out, cams, g_depth=None, g_sil=None, grazing=1e-3, radius=1.0):
    """dL/dc (n_cams, 3) and dL/dR (n_cams, 3, 3) from per-pixel upstream
    gradients of depth and silhouette (pixels in camera order, row-major)."""
    n_cams = len(cams)
    Gc = np.zeros((n_cams, 3))
    GR = np.zeros((n_cams, 3, 3))
    off = 0
    for ci, cam in enumerate(cams):
        H, W = int(cam["H"]), int(cam["W"])
        sl = slice(off, off + H * W)
        off += H * W
        ys, xs = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64),
                             indexing="ij")
        xt = (xs.ravel() + 0.5 - cam["cx"]) / cam["fx"]
        yt = (ys.ravel() + 0.5 - cam["cy"]) / cam["fy"]
        nrm = np.sqrt(xt * xt + yt * yt + 1.0)
        v_cam = np.stack([xt, yt, np.ones_like(xt)], axis=1) / nrm[:, None]
        R = np.asarray(cam["R"], dtype=np.float64)
        u = v_cam @ R.T
        un = np.linalg.norm(u, axis=1)
        v = u / un[:, None]
        c = np.asarray(cam["c"], dtype=np.float64)
        shape = out["shape"][sl]
        dLdc = np.zeros((H * W, 3))
        dLdv = np.zeros((H * W, 3))
        if g_depth is not None:
            gd = np.asarray(g_depth, dtype=np.float64)[sl]
            idx = np.nonzero(out["mask"][sl] & (gd != 0.0))[0]
            if idx.size:
                d = out["d_hit"][sl][idx]
                p = c + d[:, None] * v[idx]
                _, gp, _ = sdf.grad(p, shape[idx])
                gv = np.einsum("ij,ij->i", gp, v[idx])
                ok = np.abs(gv) >= grazing * np.linalg.norm(gp, axis=1)
                w = np.where(ok, gd[idx] / nrm[idx] / np.where(ok, gv, 1.0), 0.0)
                dLdc[idx] += -w[:, None] * gp
                dLdv[idx] += -(w * d)[:, None] * gp
        if g_sil is not None:
            gs = np.asarray(g_sil, dtype=np.float64)[sl]
            ent = out["enters"][sl]
            idx = np.nonzero(ent & (gs != 0.0) & np.isfinite(out["d_at_min"][sl]))[0]
            if idx.size:
                d = out["d_at_min"][sl][idx]
                p = c + d[:, None] * v[idx]
                _, gp, _ = sdf.grad(p, shape[idx])
                s = np.sign(out["f_at_min"][sl][idx]) * gs[idx]
                dLdc[idx] += s[:, None] * gp
                dLdv[idx] += (s * d)[:, None] * gp
            idx = np.nonzero(~ent & (gs != 0.0))[0]
            if idx.size:
                b = v[idx] @ c
                cc = float(c @ c)
                away = b >= 0.0
                dist = np.where(away, np.sqrt(cc), np.sqrt(np.maximum(cc - b * b, 0.0)))
                g = gs[idx] / dist
                dLdc[idx] += g[:, None] * np.where(away[:, None], c[None, :], c[None, :] - b[:, None] * v[idx])
                dLdv[idx] += np.where(away[:, None], 0.0, -(g * b)[:, None] * c[None, :])
        Gc[ci] = dLdc.sum(axis=0)
        proj = dLdv - v * np.einsum("ij,ij->i", v, dLdv)[:, None]
        dLdu = proj / un[:, None]
        GR[ci] = dLdu.T @ v_cam
    return Gc, GR
