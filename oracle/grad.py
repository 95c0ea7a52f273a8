"""Latent-code gradients of the rendered observations (float64).

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
