"""GPU parity of the spotlight shadow and distance falloff (Sec. 5
"Spotlight Lighting") through the C ABI against the FP64 oracle: the shadow
map's Gaussian filter within 1e-6, and the lit image within 1e-5 relative,
given the same renders (the renders themselves are covered by the render
tests).  The pipeline: alpha map rendered from a camera at the light, filtered,
projected onto the ground under the viewer's render of the five-ellipsoid
VOctree, with the falloff from the viewer's depth map."""
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


@pytest.mark.parametrize("sigma", [0.8, 1.5, 3.0])
def test_blur_matches_oracle(B, sigma):
    rng = np.random.default_rng(12)
    img = rng.uniform(0, 1, (2, 37, 53)).astype(np.float32)
    got = B.neuvv_gaussian_blur(torch.from_numpy(img).cuda(), sigma).cpu().numpy()
    ref = oracle.gaussian_blur(img.astype(np.float64), sigma)
    assert np.abs(got - ref).max() <= 1e-6


def test_spotlight_matches_oracle(B):
    tree = I.config1_tree()
    tree_d = B.Tree(tree, "f32")
    viewer = I.look_at(np.array([2.2, -1.6, 1.4]), np.array([0.5, 0.5, 0.3]), 160, 120)
    vr, _ = I.camera_rays(viewer, 0.4)
    light = I.look_at(np.array([0.6, 0.4, 3.0]), np.array([0.5, 0.5, 0.3]), 64, 64, fov_y_deg=45.0)
    lr, lpix = I.camera_rays(light, 0.4)
    dv = B.DeviceRays.from_host(vr)
    render = B.neuvv_render(tree_d, dv, kernel="packet")
    lrender = B.neuvv_render(tree_d, B.DeviceRays.from_host(lr), kernel="packet")
    # the light's alpha map in image layout, then filtered
    amap = torch.zeros(64 * 64, device="cuda")
    amap[torch.from_numpy(lpix).cuda()] = lrender["alpha"]
    blurred = B.neuvv_gaussian_blur(amap.view(1, 64, 64), 1.5)[0]
    albedo, r_ref = [0.8, 0.75, 0.7], 3.0
    got = B.neuvv_spotlight(dv, render, light, blurred, 0.0, albedo, r_ref).cpu().numpy()
    cpu = {k: v.cpu().numpy().astype(np.float64) for k, v in render.items() if isinstance(v, torch.Tensor)}
    ref = oracle.spotlight(vr.origins, vr.dirs, cpu["rgb"], cpu["alpha"], cpu["depth"], light,
                           blurred.cpu().numpy().astype(np.float64), 0.0, albedo, r_ref)
    assert np.abs(got - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())
    # the ground under the performer is shadowed: some lit ground pixels see the
    # light map at alpha > 0.5, and they are darker than unshadowed ground
    assert (blurred.cpu().numpy() > 0.5).any()
    ground = (cpu["alpha"] < 1e-3) & (vr.dirs[2] < 0)
    assert ground.mean() > 0.2
