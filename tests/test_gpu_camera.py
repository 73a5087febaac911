"""GPU parity of the ray setup (Sec. 4.3 "Rendering": a pinhole ray through
the centre of every pixel of each view) through the C ABI against the FP64
oracle: pixel ids, origins and times exactly, unit directions within 1e-6
(FP32 arithmetic on FP32 camera vectors), for cameras of ragged sizes (single
pixels, single rows and columns, partial 8x4 tiles), both orders, more than
one launch's worth of cameras, and the 8 views of the 1080p training
workload."""
from types import SimpleNamespace

import numpy as np
import pytest
import torch

import oracle
from paper_2202_06088_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(cuda_lib):
    from paper_2202_06088_gb300 import binding
    return binding


def _f32_cam(cam):
    # the camera the library sees: its vectors rounded to FP32
    r = lambda v: np.asarray(v, np.float32).astype(np.float64)
    return SimpleNamespace(eye=r(cam.eye), right=r(cam.right), up=r(cam.up), forward=r(cam.forward),
                           fov_y_deg=float(np.float32(cam.fov_y_deg)), width=cam.width, height=cam.height)


def _check(B, cams, times, tiled):
    cams = [_f32_cam(c) for c in cams]
    times = [float(np.float32(t)) for t in times]
    n = sum(c.width * c.height for c in cams)
    pix = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    got = B.neuvv_camera_rays(cams, times, tiled=tiled, pixel_of_ray=pix)
    shape = B.TILE_SHAPES[int(tiled)] if tiled else False
    parts = [oracle.camera_rays(c, t, shape) for c, t in zip(cams, times)]
    cat = lambda k, ax: np.concatenate([p[k] for p in parts], axis=ax)
    np.testing.assert_array_equal(pix.cpu().numpy(), cat("pixel", 0))
    np.testing.assert_array_equal(got.o.cpu().numpy().astype(np.float64), cat("origins", 1))
    np.testing.assert_array_equal(got.t.cpu().numpy().astype(np.float64), cat("times", 0))
    err = np.abs(got.d.cpu().numpy().astype(np.float64) - cat("dirs", 1)).max()
    assert err <= 1e-6, err


@pytest.mark.parametrize("tiled", [1, 2, 3, 0])
def test_ragged_cameras_match_oracle(B, tiled):
    sizes = [(53, 37), (8, 4), (1, 1), (40, 1), (1, 40), (33, 9), (17, 5)]
    cams = [I.look_at(np.array([0.5, 0.5, 0.5]) + 2.5 * np.array([np.cos(k), np.sin(k), 0.3]),
                      np.array([0.5, 0.5, 0.5]), w, h, fov_y_deg=30.0 + 8 * k) for k, (w, h) in enumerate(sizes)]
    _check(B, cams, np.linspace(0.0, 1.0, len(cams)), tiled)


def test_more_cameras_than_one_launch(B):
    cams = I.sphere_cameras(5, 40, 2.5, 13, 6)
    _check(B, cams, np.random.default_rng(5).uniform(0, 1, 40), True)


def test_training_views_at_1080p(B):
    _, _, cams, ts = I.config2_rays(n_views=8)
    _check(B, cams, ts, True)


def test_device_rays_render_like_host_rays(B):
    # the renderer sees the same rays (to FP32 rounding) either way
    tree = I.config1_tree()
    cam = I.look_at(np.array([0.5, -2.0, 1.0]), np.array([0.5, 0.5, 0.5]), 128, 128)
    host, _ = I.camera_rays(cam, 0.4)
    tree_d = B.Tree(tree, "f32")
    a = B.neuvv_render(tree_d, B.neuvv_camera_rays([cam], [0.4]), kernel="packet")["rgb"].cpu().numpy()
    b = B.neuvv_render(tree_d, B.DeviceRays.from_host(host), kernel="packet")["rgb"].cpu().numpy()
    diff = np.abs(a - b).max(axis=1)
    assert (diff <= 1e-4).mean() >= 0.999
    assert tree_d.status() == 0
