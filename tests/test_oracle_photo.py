"""Pins for the oracle's multi-view photometric loss (no GPU).

* a view warped onto itself reproduces itself: loss 0;
* the gradient with respect to the rendered depth against central
  differences of the loss (pixels away from the L1 kink, the bilinear cell
  edges and the visibility threshold);
* a texture linear in image coordinates is reproduced exactly by bilinear
  sampling, so the warped image of a plane seen by a translated camera has a
  closed form;
* points hidden in the other view (an occluder in its depth map) are not
  visible and do not contribute.
"""

import numpy as np

import synth
from oracle import photo, tracer
from oracle.camera import pixel_rays
from oracle.sdf import SphereSDF


def _texture(cam, depth, seed=0):
    """Colour from the world point of each hit: smooth, three channels."""
    c, v, inv = pixel_rays(cam)
    d = np.where(np.isfinite(depth), depth / inv, 0.0)
    P = c + d[:, None] * v
    k = np.random.default_rng(seed).normal(size=(3, 3)) * 4.0
    img = 0.5 + 0.5 * np.sin(P @ k.T + np.array([0.3, 1.1, 2.0]))
    img[~np.isfinite(depth)] = 0.0
    return img.reshape(int(cam["H"]), int(cam["W"]), 3)


def _scene(n=32):
    sph = SphereSDF(0.6)
    vps = synth.ring_viewpoints(8)
    cams = [synth.look_at_camera(vps[k], n, n) for k in (0, 1)]
    outs = [tracer.render(sph, [c], max_steps=200, eps=1e-10, alpha=1.0, with_normals=False)
            for c in cams]
    depths = [o["depth"] for o in outs]
    images = [_texture(c, d) for c, d in zip(cams, depths)]
    return cams, depths, images


def test_self_warp_is_identity():
    cams, depths, images = _scene()
    loss, g, vis = photo.warp_loss(cams, depths, images, [(0, 0), (1, 1)])
    assert vis[0].sum() > 50
    # the camera rotations arrive rounded to float32 (orthonormal to ~1e-8),
    # so the round trip lands within ~1e-7 pixel of the centre
    assert loss < 1e-6


def test_depth_gradient_vs_finite_differences():
    cams, depths, images = _scene()
    pairs = [(0, 1), (1, 0)]
    loss, g, vis = photo.warp_loss(cams, depths, images, pairs)
    assert loss > 1e-4
    rng = np.random.default_rng(1)
    cand = np.nonzero(vis[0])[0]
    checked = 0
    for i in rng.permutation(cand)[:60]:
        h = 1e-7
        dp = [d.copy() for d in depths]; dm = [d.copy() for d in depths]
        dp[0][i] += h; dm[0][i] -= h
        lp, _, vp = photo.warp_loss(cams, dp, images, pairs)
        lm, _, vm = photo.warp_loss(cams, dm, images, pairs)
        if not (np.array_equal(vp[0], vis[0]) and np.array_equal(vm[0], vis[0])):
            continue
        fd = (lp - lm) / (2 * h)
        # skip samples whose finite difference crosses a kink (L1 or cell edge)
        if abs(fd - g[0][i]) > 1e-4 * max(1e-3, abs(fd)):
            h2 = 1e-8
            dp[0][i] = depths[0][i] + h2; dm[0][i] = depths[0][i] - h2
            fd2 = (photo.warp_loss(cams, dp, images, pairs)[0] -
                   photo.warp_loss(cams, dm, images, pairs)[0]) / (2 * h2)
            if abs(fd2 - fd) > 1e-3 * max(1e-3, abs(fd)):
                continue          # a kink inside [d - h, d + h]
        assert abs(fd - g[0][i]) <= 1e-4 * max(1e-3, abs(fd)), (i, fd, g[0][i])
        checked += 1
    assert checked > 30


def test_linear_texture_plane_closed_form():
    # fronto-parallel plane z = 0 seen from two cameras translated along x
    n = 24
    cam0 = synth.look_at_camera((0.0, 0.0, 2.5), n, n)
    cam1 = dict(cam0, c=np.asarray(cam0["c"], dtype=np.float64) + np.array([0.1, 0.0, 0.0]))
    depths = []
    for cam in (cam0, cam1):
        c, v, inv = pixel_rays(cam)
        t = -c[2] / v[:, 2]                      # hit of z = 0
        depths.append(t * inv)
    a, b, k = 0.013, -0.007, 0.4
    H = W = n
    ys, xs = np.meshgrid(np.arange(H) + 0.5, np.arange(W) + 0.5, indexing="ij")
    img1 = (a * xs + b * ys + k)[..., None].repeat(3, axis=2)
    img0 = np.zeros((H, W, 3))
    loss, g, vis = photo.warp_loss([cam0, cam1], depths, [img0, img1], [(0, 1)])
    # the analytic warp: project each hit of view 0 into view 1
    c0, v0, inv0 = pixel_rays(cam0)
    P = c0 + (depths[0] / inv0)[:, None] * v0
    R1 = np.asarray(cam1["R"]); c1 = np.asarray(cam1["c"])
    pc = (P - c1) @ R1
    u = cam1["fx"] * pc[:, 0] / pc[:, 2] + cam1["cx"]
    v = cam1["fy"] * pc[:, 1] / pc[:, 2] + cam1["cy"]
    warped = a * u + b * v + k
    m = vis[0]
    assert m.sum() > 100
    expect = 3 * np.abs(warped[m]).sum() / m.sum()
    assert abs(loss - expect) < 1e-12 * max(1.0, expect)


def test_occluded_points_are_not_visible():
    cams, depths, images = _scene()
    _, _, vis = photo.warp_loss(cams, depths, images, [(0, 1)])
    occl = [depths[0], depths[1].copy()]
    fin = np.isfinite(occl[1])
    occl[1][fin] -= 0.5                       # something 0.5 in front everywhere
    loss, g, vis2 = photo.warp_loss(cams, occl, images, [(0, 1)])
    assert vis[0].sum() > 50 and vis2[0].sum() == 0 and loss == 0.0
    assert not np.any(g[0])


def test_visibility_threshold():
    # view 1's depth moved by delta: visible while delta^2 < 1e-3 (Sec. B.3)
    cams, depths, images = _scene()
    _, _, vis = photo.warp_loss(cams, depths, images, [(0, 1)])
    base = vis[0].sum()
    counts = {}
    for delta in (0.025, 0.04):
        d1 = depths[1].copy()
        fin = np.isfinite(d1)
        d1[fin] -= delta
        _, _, v = photo.warp_loss(cams, [depths[0], d1], images, [(0, 1)])
        counts[delta] = v[0].sum()
    assert counts[0.025] >= 0.9 * base and counts[0.04] <= 0.1 * base, (base, counts)
