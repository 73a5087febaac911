"""GPU parity of the density-only render (Sec. 5 "Spotlight Lighting": the
shadow map is the VOctree's alpha seen from the light) through the C ABI:
alpha, depth, optical depth and segment counts bit-identical to the full
packet render (the same walk and compositing on the same densities), and
alpha within 1e-4 of the FP64 oracle, for FP32, BF16 and FP8 storage at both
record shapes (K 8 with degree 2, K 16 with degree 3); ragged ray counts;
run on a second stream beside a full render of the same tree."""
import numpy as np
import pytest
import torch

import oracle
from paper_2202_06088_gb300 import inputs as I

from test_gpu_render import _ambiguous_stop

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(cuda_lib):
    from paper_2202_06088_gb300 import binding
    return binding


def _tree(K, T, deg):
    st, rng, _ = I.solid_scene_structure(1235, 6)
    return I.make_coefficients(rng, st, K=K, T=T, hh_degree=deg)


@pytest.fixture(scope="module", params=[(8, 30, 2), (16, 150, 3)], ids=["k8d2", "k16d3"])
def tree(request):
    return _tree(*request.param)


@pytest.fixture(scope="module")
def rays():
    r, _ = I.config1_rays()
    return r.subset(np.arange(r.n - 77))                   # a ragged last packet


@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
def test_alpha_equals_full_render(B, tree, rays, dtype):
    tree_d = B.Tree(tree, dtype)
    dr = B.DeviceRays.from_host(rays)
    full = {k: v.cpu().numpy() for k, v in B.neuvv_render(tree_d, dr, kernel="packet").items()}
    got = {k: v.cpu().numpy() for k, v in B.neuvv_render_alpha(tree_d, dr).items()}
    for k in ("alpha", "depth", "tau", "nseg"):
        np.testing.assert_array_equal(got[k], full[k], err_msg=k)
    assert (full["alpha"] > 0.5).mean() > 0.05
    assert tree_d.status() == 0


def test_alpha_matches_oracle(B, tree, rays):
    tree_d = B.Tree(tree, "f32")
    got = B.neuvv_render_alpha(tree_d, B.DeviceRays.from_host(rays))["alpha"].cpu().numpy()
    ref = oracle.render(tree, rays)
    ok = ~_ambiguous_stop(ref)
    assert ok.mean() > 0.99
    assert np.abs(got[ok] - ref["alpha"][ok]).max() <= 1e-4


def test_alpha_beside_a_full_render(B, tree, rays):
    # no shared work counter: a second stream may run it beside neuvv_render
    tree_d = B.Tree(tree, "bf16")
    dr = B.DeviceRays.from_host(rays)
    ref_full = B.neuvv_render(tree_d, dr, kernel="packet")
    ref_a = ref_full["alpha"].clone()
    ref_rgb = ref_full["rgb"].clone()
    side = torch.cuda.Stream()
    main = torch.cuda.current_stream()
    side.wait_stream(main)
    for _ in range(5):
        with torch.cuda.stream(side):
            a = B.neuvv_render_alpha(tree_d, dr)
        f = B.neuvv_render(tree_d, dr, kernel="packet")
        main.wait_stream(side)
        torch.cuda.synchronize()
        assert torch.equal(a["alpha"], ref_a)
        assert torch.equal(f["rgb"], ref_rgb)
    assert tree_d.status() == 0
