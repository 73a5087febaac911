"""Pins of the oracle's spotlight shadow and distance falloff (Sec. 5
"Spotlight Lighting": an alpha map rendered from a camera at the light,
reversed, low-pass filtered and projected onto the ground; brightness falling
off with the distance to the light, from the depth map).

* The blur is scipy's Gaussian filter (mode 'nearest', truncate 3) over the
  two image axes, and keeps constant images constant.
* Projecting into the light camera inverts the light camera's own rays: the
  ground point a light pixel's ray reaches samples exactly that pixel's texel.
* Bilinear sampling reproduces a linear map exactly.
* With no occluder the ground below the light gets albedo * r_ref^2 / h^2; a
  fully opaque light map darkens the ground completely; the performer's colour
  is scaled by r_ref^2 / |X - L|^2 at its depth point; rays that miss the
  ground keep the performer's colour.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2202_06088_gb300 import inputs as I

scipy_ndimage = pytest.importorskip("scipy.ndimage")


@pytest.mark.parametrize("sigma", [0.6, 1.5, 2.2])
def test_blur_is_the_gaussian_filter(sigma):
    rng = np.random.default_rng(1)
    img = rng.uniform(0, 1, (2, 23, 31))
    ref = scipy_ndimage.gaussian_filter(img, sigma=(0, sigma, sigma), mode="nearest", truncate=3.0)
    np.testing.assert_allclose(oracle.gaussian_blur(img, sigma), ref, rtol=0, atol=1e-12)
    np.testing.assert_allclose(oracle.gaussian_blur(np.full((1, 9, 7), 0.3), sigma), 0.3, rtol=0, atol=1e-15)


def _light(W=24, H=16):
    return I.look_at(np.array([0.9, 0.2, 3.0]), np.array([0.5, 0.5, 0.0]), W, H, fov_y_deg=50.0)


def _ground_hits(light, ground_z):
    rays, pix = I.camera_rays(light, 0.0, tiled=False)
    o = rays.origins.astype(np.float64)
    d = rays.dirs.astype(np.float64)
    s = (ground_z - o[2]) / d[2]
    return o + s * d, pix


def test_projection_inverts_the_light_camera():
    light = _light()
    rng = np.random.default_rng(2)
    Al = rng.uniform(0, 1, (light.height, light.width))
    P, pix = _ground_hits(light, 0.0)
    n = P.shape[1]
    # viewer rays straight down onto those ground points, nothing in front
    o = P + np.array([[0.0], [0.0], [5.0]])
    d = np.tile(np.array([[0.0], [0.0], [-1.0]]), (1, n))
    out = oracle.spotlight(o, d, np.zeros((n, 3)), np.zeros(n), np.full(n, np.inf), light, Al, 0.0,
                           [1.0, 1.0, 1.0], 1.0)
    py, px = np.divmod(pix, light.width)
    f = 1.0 / np.sum((P - light.eye[:, None]) ** 2, axis=0)
    # the light camera's rays are FP32: ground points sit within ~1e-7 pixel of
    # the pixel centres, a convention error (half-pixel shift, flipped axis)
    # would move them by half a pixel or more
    np.testing.assert_allclose(out[:, 0], (1 - Al[py, px]) * f, rtol=1e-4, atol=0)


def test_bilinear_is_exact_on_a_linear_map():
    light = _light(40, 30)
    x = np.arange(40, dtype=np.float64)
    Al = np.tile(0.01 * x, (30, 1))                     # alpha = 0.01 * (pixel x coordinate)
    P, pix = _ground_hits(light, 0.0)
    # points half-way between horizontally adjacent pixel rays' ground hits do
    # not project to half-way pixels; use a finer light camera's hits instead
    fine = I.look_at(light.eye, light.eye + light.forward, 80, 60, fov_y_deg=light.fov_y_deg)
    Pf, pf = _ground_hits(fine, 0.0)
    keep = (pf % 80 > 1) & (pf % 80 < 78) & (pf // 80 > 1) & (pf // 80 < 58)
    Pf = Pf[:, keep]
    pf = pf[keep]
    n = Pf.shape[1]
    o = Pf + np.array([[0.0], [0.0], [1.0]])
    d = np.tile(np.array([[0.0], [0.0], [-1.0]]), (1, n))
    out = oracle.spotlight(o, d, np.zeros((n, 3)), np.zeros(n), np.full(n, np.inf), light, Al, 0.0,
                           [1.0, 1.0, 1.0], 1.0)
    # fine pixel centre (i + 0.5) / 80 of the width is coarse coordinate (i + 0.5) / 2 - 0.5
    xc = ((pf % 80) + 0.5) / 2.0 - 0.5
    f = 1.0 / np.sum((Pf - light.eye[:, None]) ** 2, axis=0)
    np.testing.assert_allclose(out[:, 1] / f, 1 - 0.01 * xc, rtol=0, atol=1e-6)


def test_closed_forms():
    light = I.Camera(np.array([0.5, 0.5, 4.0]), np.array([1.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0]),
                     np.array([0.0, 0.0, -1.0]), 8, 8, 60.0)
    o = np.array([[0.5, 0.7], [0.5, 0.4], [2.0, 2.0]])
    d = np.array([[0.0, 0.0], [0.0, 0.0], [-1.0, -1.0]])
    clear = np.zeros((8, 8))
    out = oracle.spotlight(o, d, np.zeros((2, 3)), np.zeros(2), np.full(2, np.inf), light, clear, 0.0,
                           [0.5, 0.6, 0.7], 2.0)
    np.testing.assert_allclose(out[0], np.array([0.5, 0.6, 0.7]) * 4.0 / 16.0, rtol=1e-14)
    opaque = np.ones((8, 8))
    out = oracle.spotlight(o, d, np.zeros((2, 3)), np.zeros(2), np.full(2, np.inf), light, opaque, 0.0,
                           [0.5, 0.6, 0.7], 2.0)
    assert np.all(out == 0.0)
    # performer in front: colour scaled by the falloff at its depth point, the
    # ground weighted by 1 - alpha
    rgb = np.array([[0.2, 0.3, 0.4], [0.1, 0.1, 0.1]])
    out = oracle.spotlight(o, d, rgb, np.array([0.75, 0.0]), np.array([1.0, np.inf]), light, clear, 0.0,
                           [0.5, 0.6, 0.7], 2.0)
    X = o[:, 0] + 1.0 * d[:, 0]
    fX = 4.0 / np.sum((X - light.eye) ** 2)
    np.testing.assert_allclose(out[0], rgb[0] * fX + 0.25 * np.array([0.5, 0.6, 0.7]) * 4.0 / 16.0, rtol=1e-14)
    # a ray going up never meets the ground
    out = oracle.spotlight(o, -d, rgb, np.zeros(2), np.full(2, np.inf), light, clear, 0.0, [1, 1, 1], 2.0)
    np.testing.assert_array_equal(out, rgb)
