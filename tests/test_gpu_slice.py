"""GPU parity of the time slice (Sec. 7; the caption of the HH-colour figure)
through the C ABI: neuvv_slice against the FP64 oracle's slice, and
neuvv_render_slice against the oracle's render of that slice, which its own
pins tie to the HH render at the same time.

Tolerances: slice entries within 1e-5 relative (FP32 sums of at most 16
products of O(1) terms; density within 1e-5 of its magnitude); renders at
the FP32 bar of 1e-4, with the early-stop and near-tie exemptions of the
render tests.  BF16 and FP8 trees are compared with the oracle on their
rounded coefficients.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2202_06088_gb300 import inputs as I

from helpers import psnr
from test_gpu_render import _check_render

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(cuda_lib):
    from paper_2202_06088_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def c1():
    return I.config1_tree()


def _rounded(tree, dtype):
    if dtype == "f32":
        return tree
    if dtype == "bf16":
        return tree.with_coeffs(oracle.round_bf16(tree.w_sigma), oracle.round_bf16(tree.w_gamma),
                                oracle.round_bf16(tree.w_hh))
    return oracle.quantize_fp8_tree(tree)[0]


def _check_slice(got, ref, deg):
    ny = (deg + 1) ** 2
    sig = got[:, 0].astype(np.float64)
    assert np.all(got[:, 1:4] == 0)
    assert np.abs(sig - ref["sigma"]).max() <= 1e-5 * max(1.0, np.abs(ref["sigma"]).max())
    sh = got[:, 4:4 + 3 * ny].reshape(-1, 3, ny).astype(np.float64)
    err = np.abs(sh - ref["sh"])
    assert (err <= 1e-5 * (1 + np.abs(ref["sh"]))).all(), err.max()


@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
@pytest.mark.parametrize("t", [0.0, 0.37, 1.0])
def test_slice_matches_oracle(B, c1, dtype, t):
    tree_d = B.Tree(c1, dtype)
    got = B.neuvv_slice(tree_d, t).cpu().numpy()
    ref = oracle.slice_at(_rounded(c1, dtype), t)
    assert got.shape == (c1.n_leaves, B.slice_stride(c1.hh_degree))
    _check_slice(got, ref, c1.hh_degree)
    assert tree_d.status() == 0


@pytest.mark.parametrize("K,deg", [(4, 1), (16, 3)])
def test_slice_other_shapes_and_padded_stride(B, K, deg):
    rng = np.random.default_rng(70 + K)
    st = I.random_mixed_tree(5, 70 + K, p_leaf=0.3, p_empty=0.2)
    tree = I.make_coefficients(rng, st, K=K, T=9, hh_degree=deg, signed_density=True)
    tree_d = B.Tree(tree, "f32")
    stride = B.slice_stride(deg) + 8
    buf = torch.full((tree.n_leaves, stride), 7.0, device="cuda")
    got = B.neuvv_slice(tree_d, 0.55, out=buf).cpu().numpy()
    _check_slice(got, oracle.slice_at(tree, 0.55), deg)
    assert np.all(got[:, B.slice_stride(deg):] == 7.0)          # the rest of each row is untouched


def test_slice_rejects_bad_arguments(B, c1):
    tree_d = B.Tree(c1, "f32")
    from paper_2202_06088_gb300.binding import NeuvvError
    buf = torch.zeros(c1.n_leaves, 32, device="cuda")
    with pytest.raises(NeuvvError):
        B.neuvv_slice(tree_d, 0.5, out=torch.zeros(c1.n_leaves, 30, device="cuda"))   # stride below 4 + 27
    with pytest.raises(NeuvvError):
        B.neuvv_slice(tree_d, 1.5, out=buf)                                             # t outside [0, 1]
    with pytest.raises(NeuvvError):
        B.neuvv_slice(tree_d, 0.5, out=buf.view(-1)[1:1 + c1.n_leaves * 28].view(c1.n_leaves, 28))  # misaligned


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_render_slice_matches_oracle_and_hh_render(B, c1, dtype):
    rays, _ = I.config1_rays()
    t = float(np.float32(0.37))
    rays.times[:] = np.float32(t)
    tree_d = B.Tree(c1, dtype)
    sl = B.neuvv_slice(tree_d, t)
    dr = B.DeviceRays.from_host(rays)
    got = {k: v.cpu().numpy() for k, v in B.neuvv_render_slice(tree_d, sl, dr).items()}
    src = _rounded(c1, dtype)
    ref = oracle.render_slice(src, oracle.slice_at(src, t), rays)
    ref_hh = oracle.render(src, rays)
    assert np.abs(ref["rgb"] - ref_hh["rgb"]).max() <= 1e-12
    _check_render(ref_hh, got, 1e-4, src)
    # the same frame through the HH path of the library
    hh = {k: v.cpu().numpy() for k, v in B.neuvv_render(tree_d, dr, kernel="packet").items()}
    assert np.abs(hh["rgb"] - got["rgb"]).max() <= 1e-4
    assert psnr(got["rgb"], hh["rgb"]) >= 80.0
    assert tree_d.status() == 0
