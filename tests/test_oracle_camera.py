"""Pins of the oracle's pinhole camera rays (Sec. 4.3 "Rendering": a ray
through the centre of every pixel of a view) to facts other than its own
formula: the pixel order against the seeded generator's independent
lexsort-based tile order and against tile geometry, unit directions, the
centre pixel looking along the optical axis, the tangents of each ray's angles
against the image-plane coordinates of its pixel, the symmetry of mirrored
pixels, and the vertical field of view spanned by the outermost pixel rows."""
import math
from types import SimpleNamespace

import numpy as np
import pytest

import oracle
from paper_2202_06088_gb300 import inputs as I


def _cam(W, H, fov=40.0, eye=(0.5, 0.5, 3.0), seed=0):
    rng = np.random.default_rng(seed)
    target = np.array([0.5, 0.5, 0.5]) + rng.normal(0, 0.1, 3)
    return I.look_at(np.asarray(eye, float) + rng.normal(0, 0.2, 3), target, W, H, fov_y_deg=fov)


@pytest.mark.parametrize("W,H", [(53, 37), (8, 4), (1, 1), (40, 1), (1, 40), (33, 9), (64, 48)])
@pytest.mark.parametrize("tiled", [True, False, (4, 8), (16, 2)])
def test_pixel_order(W, H, tiled):
    r = oracle.camera_rays(_cam(W, H), 0.3, tiled)
    pix = r["pixel"]
    assert sorted(pix.tolist()) == list(range(W * H))          # every pixel once
    tw, th = (8, 4) if tiled is True else (tiled if tiled else (0, 0))
    ref = I.tile_order(W, H, tw, th) if tiled else np.arange(W * H)   # built by sorting keys, not by loops
    np.testing.assert_array_equal(pix, ref)
    if tiled and H >= th:
        # the first band's full tiles: 32 consecutive rays fill each one
        py, px = np.divmod(pix, W)
        for k in range(W // tw):
            sl = slice(32 * k, 32 * k + 32)
            assert (px[sl].min(), px[sl].max(), py[sl].min(), py[sl].max()) == (tw * k, tw * k + tw - 1, 0, th - 1)


@pytest.mark.parametrize("fov", [20.0, 40.0, 90.0])
def test_directions_follow_the_pinhole(fov):
    W, H = 31, 17                                             # odd: one pixel on the optical axis
    cam = _cam(W, H, fov)
    r = oracle.camera_rays(cam, 0.0, tiled=False)
    d = r["dirs"]
    np.testing.assert_allclose(np.linalg.norm(d, axis=0), 1.0, atol=1e-14)
    centre = (H // 2) * W + W // 2
    np.testing.assert_allclose(d[:, r["pixel"] == centre][:, 0], cam.forward, atol=1e-14)
    py, px = np.divmod(r["pixel"], W)
    th = math.tan(math.radians(fov) / 2)
    # tangents of the angles to the optical axis = image-plane coordinates
    along = cam.forward @ d
    np.testing.assert_allclose((cam.right @ d) / along, (2 * (px + 0.5) / W - 1) * th * W / H, atol=1e-12)
    np.testing.assert_allclose((cam.up @ d) / along, (1 - 2 * (py + 0.5) / H) * th, atol=1e-12)
    # row 0 looks up, column 0 looks left; mirrored pixels mirror the ray
    assert (cam.up @ d[:, py == 0] > 0).all() and (cam.right @ d[:, px == 0] < 0).all()
    a = d[:, (py == 3) & (px == 5)][:, 0]
    b = d[:, (py == H - 1 - 3) & (px == W - 1 - 5)][:, 0]
    np.testing.assert_allclose(cam.forward @ a, cam.forward @ b, atol=1e-14)
    np.testing.assert_allclose(cam.right @ a, -(cam.right @ b), atol=1e-14)
    np.testing.assert_allclose(cam.up @ a, -(cam.up @ b), atol=1e-14)


def test_vertical_field_of_view():
    # the pixel rows at the edges span the field of view less half a pixel on each side
    H, fov = 1000, 50.0
    cam = _cam(3, H, fov)
    r = oracle.camera_rays(cam, 0.0, tiled=False)
    py, px = np.divmod(r["pixel"], 3)
    top = r["dirs"][:, (py == 0) & (px == 1)][:, 0]
    bottom = r["dirs"][:, (py == H - 1) & (px == 1)][:, 0]
    angle = math.degrees(math.acos(float(top @ bottom)))
    expected = 2 * math.degrees(math.atan((1 - 1 / H) * math.tan(math.radians(fov / 2))))
    assert abs(angle - expected) < 1e-9
    assert fov - 0.2 < angle < fov


def test_agrees_with_the_generator():
    # the seeded generator's rays (computed there independently, then rounded
    # to FP32) equal the oracle's up to that rounding
    cam = _cam(53, 37, seed=3)
    got, pix = I.camera_rays(cam, 0.625)
    r = oracle.camera_rays(cam, 0.625)
    np.testing.assert_array_equal(pix, r["pixel"])
    np.testing.assert_allclose(got.dirs, r["dirs"], atol=1e-7)
    np.testing.assert_allclose(got.origins, r["origins"], atol=1e-7)
    np.testing.assert_array_equal(got.times, np.float32(r["times"]))


def test_times_and_origins():
    cam = SimpleNamespace(eye=(1.0, -2.0, 0.25), right=(1.0, 0.0, 0.0), up=(0.0, 0.0, 1.0), forward=(0.0, 1.0, 0.0),
                          fov_y_deg=60.0, width=5, height=3)
    r = oracle.camera_rays(cam, 0.75, tiled=True)
    assert (r["times"] == 0.75).all()
    np.testing.assert_array_equal(r["origins"], np.repeat(np.array([[1.0], [-2.0], [0.25]]), 15, axis=1))
    # the middle pixel of a 5x3 image looks straight ahead
    np.testing.assert_allclose(r["dirs"][:, r["pixel"] == 7][:, 0], [0.0, 1.0, 0.0], atol=1e-15)
