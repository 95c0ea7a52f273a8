"""Pins of the oracle's camera model (oracle/camera.py: pixel_rays) that do
not go through pixel_rays' own arithmetic.

Sec. 3.3 defines the depth of a point at ray distance d as
z_c = d / sqrt(x~^2 + y~^2 + 1) with (x~, y~, 1) = K^-1 (u, v, 1), i.e. the
pinhole model in a camera frame with z forward; the cameras here use OpenCV
axes (x right, y down, z forward) and R is camera-to-world (its columns are
those axes in world coordinates).  The checks build the camera frame from
the look-at geometry itself (forward towards the target, right horizontal,
down = forward x right), project world points with x~ = X_c / Z_c, and
require that pixel_rays' ray through the resulting pixel passes through the
point.  An off-axis camera makes R non-symmetric, so a transposed R (world-
to-camera used as camera-to-world) fails every one of them."""

import numpy as np
import pytest

import synth
from oracle.camera import depth_from_distance, pixel_rays

EYES = [(1.3, -0.7, 1.9), (-2.0, 1.1, -0.9), (0.4, 2.2, 1.0)]


def _frame(eye):
    """Camera axes of a camera at `eye` looking at the origin with world up
    +y: forward towards the origin, right perpendicular to forward and up,
    down completing a right-handed (x right, y down, z forward) frame."""
    eye = np.asarray(eye, dtype=np.float64)
    fwd = -eye / np.linalg.norm(eye)
    right = np.cross(fwd, [0.0, 1.0, 0.0])
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    return right, down, fwd


def _projection_error(cam, pts):
    """Largest distance between each world point and the ray that
    pixel_rays shoots through the pixel position the pinhole model assigns
    to it (the point is put on a pixel centre by shifting the principal
    point), plus the depth error of that point."""
    right, down, fwd = _frame(cam["c"])
    worst = 0.0
    for P in pts:
        rel = np.asarray(P, dtype=np.float64) - np.asarray(cam["c"], dtype=np.float64)
        X, Y, Z = rel @ right, rel @ down, rel @ fwd
        assert Z > 0
        u, v = cam["fx"] * X / Z + cam["cx"], cam["fy"] * Y / Z + cam["cy"]
        # move the principal point so (u, v) is the centre of pixel (x0, y0)
        x0, y0 = int(np.floor(u)), int(np.floor(v))
        shifted = dict(cam, cx=cam["cx"] - (u - x0 - 0.5), cy=cam["cy"] - (v - y0 - 0.5))
        c, dirs, inv = pixel_rays(shifted)
        k = y0 * int(cam["W"]) + x0
        t = float(rel @ dirs[k])
        worst = max(worst, float(np.linalg.norm(c + t * dirs[k] - P)))
        worst = max(worst, abs(float(depth_from_distance(t, inv[k])) - Z))
    return worst


@pytest.mark.parametrize("eye", EYES)
def test_centre_ray_passes_through_the_look_at_target(eye):
    cam = synth.look_at_camera(eye, 33, 41)        # odd sizes: a pixel centre on the axis
    c, v, inv = pixel_rays(cam)
    k = 16 * 41 + 20                               # (x, y) = (20, 16): x~ = y~ = 0
    assert inv[k] == 1.0
    dist = np.linalg.norm(c)
    assert np.linalg.norm(c + dist * v[k]) < 1e-6   # float32-rounded camera
    bad = dict(cam, R=cam["R"].T)
    _, vb, _ = pixel_rays(bad)
    assert np.linalg.norm(c + dist * vb[k]) > 1e-2


@pytest.mark.parametrize("eye", EYES)
def test_world_points_project_to_their_closed_form_pixels(eye):
    cam = synth.look_at_camera(eye, 64, 48)
    pts = np.array([[0.2, 0.1, -0.3], [-0.35, 0.4, 0.25], [0.0, -0.5, 0.1], [0.3, 0.3, 0.3]])
    assert _projection_error(cam, pts) < 1e-6
    # the same check fails with the rotation transposed
    assert _projection_error(dict(cam, R=cam["R"].T), pts) > 1e-2


@pytest.mark.parametrize("eye", EYES)
def test_camera_to_world_axes_and_camera_frame_point(eye):
    """R's columns are the camera's right, down and forward axes (OpenCV);
    R^T (P - c) is a point's camera-frame position, which for a point on
    pixel (x, y)'s ray at depth Z is Z (x~, y~, 1)."""
    cam = synth.look_at_camera(eye, 30, 20)      # H = 30, W = 20
    R = np.asarray(cam["R"], dtype=np.float64)
    right, down, fwd = _frame(eye)
    np.testing.assert_allclose(R[:, 0], right, atol=1e-7)
    np.testing.assert_allclose(R[:, 1], down, atol=1e-7)
    np.testing.assert_allclose(R[:, 2], fwd, atol=1e-7)
    np.testing.assert_allclose(np.cross(R[:, 0], R[:, 1]), R[:, 2], atol=1e-6)
    c, v, inv = pixel_rays(cam)
    for (x, y) in [(0, 0), (19, 29), (7, 21), (13, 2)]:
        k = y * 20 + x
        d = 1.7
        P = c + d * v[k]
        Xc = R.T @ (P - c)
        Z = d * inv[k]
        want = Z * np.array([(x + 0.5 - cam["cx"]) / cam["fx"], (y + 0.5 - cam["cy"]) / cam["fy"], 1.0])
        np.testing.assert_allclose(Xc, want, atol=1e-6)
        # image x grows to the camera's right, image y downwards
        assert np.sign(Xc[0]) == np.sign(x + 0.5 - cam["cx"])
        assert np.sign(Xc[1]) == np.sign(y + 0.5 - cam["cy"])
