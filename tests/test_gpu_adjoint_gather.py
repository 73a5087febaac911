"""GPU parity of the leaf-major adjoint (neuvv_tree_reserve_adjoint): a count
over the segment log gives each leaf's samples, the replayed samples leave
their gradient factors at the next position of their leaf's run, and one
thread per leaf sums its run into its gradient record.  Checked against the FP64 oracle's analytic gradient at the
adjoint's bar (per leaf record, relative 1e-4 plus 1e-6 of the largest), and
against the atomic scatter on the same inputs: every gradient entry within
1e-5 of its plane's largest entry (FP32 summation order is all that differs),
the touched bitmap identical.  Covers FP32, BF16 and FP8 storage, both record
shapes, a reservation smaller than the log (chunks past it take the atomic
path), repeated calls (each call counts and lays out the runs afresh) and
the full-size training workload."""
import numpy as np
import pytest
import torch

import oracle
from paper_2202_06088_gb300 import inputs as I

from test_gpu_backward import _record_planes, _rel_err, _setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(cuda_lib):
    from paper_2202_06088_gb300 import binding
    return binding


def _bits(touched, n):
    b = touched.cpu().numpy().view(np.uint32)
    return ((b[np.arange(n) >> 5] >> (np.arange(n) & 31)) & 1).astype(bool)


def _both(B, tree_d, dr, g, ga, slots, act="sigmoid", repeat=1):
    """Gradients of the atomic path and of the leaf-major path (same forward)."""
    out = B.alloc_out(dr.n, log_bytes_per_ray=64)
    B.neuvv_render(tree_d, dr, act=act, kernel="packet", out=out)
    res = []
    for reserve in (0, slots):
        tree_d.reserve_adjoint(reserve)
        grad, touched = tree_d.new_grad(), tree_d.new_touched()
        for _ in range(repeat):
            B.neuvv_render_backward(tree_d, dr, out, g, ga, grad=grad, touched=touched, act=act, kernel="packet")
        torch.cuda.synchronize()
        res.append((grad.clone(), touched.clone()))
    tree_d.reserve_adjoint(0)
    return res


def _close(ga_, gb_):
    a, b = ga_.cpu().numpy().astype(np.float64), gb_.cpu().numpy().astype(np.float64)
    scale = np.abs(a).max(axis=0, keepdims=True) + 1e-30
    return (np.abs(a - b) / scale).max()


@pytest.mark.parametrize("K,deg,depth,act,signed", [
    (8, 2, 5, "sigmoid", True),
    (16, 3, 5, "identity", False),
])
def test_gather_matches_oracle_and_atomic_path(B, K, deg, depth, act, signed):
    tree, rays, g, ga = _setup(50 + K + depth, K, deg, depth, 4096 + 3, signed=signed)
    ref_out = oracle.render(tree, rays, act=act)
    keep = ref_out["stop_margin"] > 1e-3
    rays = rays.subset(np.nonzero(keep)[0])
    g, ga = g[keep], ga[keep]
    ref = oracle.render_grad(tree, rays, g, ga, act=act)
    tree_d = B.Tree(tree, "f32")
    dr = B.DeviceRays.from_host(rays)
    gt, gat = torch.from_numpy(g).cuda(), torch.from_numpy(ga).cuda()
    (g_atom, t_atom), (g_gath, t_gath) = _both(B, tree_d, dr, gt, gat, 1 << 22, act=act)
    num, den = _rel_err(_record_planes(tree_d, g_gath), ref)
    assert np.all(num <= 1e-4 * den + 1e-6 * den.max()), (num / np.maximum(den, 1e-30)).max()
    assert _close(g_atom, g_gath) <= 1e-5
    assert torch.equal(t_atom, t_gath)
    assert _bits(t_gath, tree.n_leaves)[den > 0].all()
    assert tree_d.status() == 0


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
@pytest.mark.parametrize("shape", [(8, 30, 2), (16, 150, 3)], ids=["k8d2", "k16d3"])
def test_gather_storage_types(B, dtype, shape):
    K, T, deg = shape
    st, rng, _ = I.solid_scene_structure(1235, 6)
    tree = I.make_coefficients(rng, st, K=K, T=T, hh_degree=deg)
    rays, _ = I.config1_rays()
    g = torch.from_numpy(np.random.default_rng(3).standard_normal((rays.n, 3)).astype(np.float32)).cuda()
    tree_d = B.Tree(tree, dtype)
    dr = B.DeviceRays.from_host(rays)
    (g_atom, t_atom), (g_gath, t_gath) = _both(B, tree_d, dr, g, None, 1 << 22)
    assert _close(g_atom, g_gath) <= 1e-5
    assert torch.equal(t_atom, t_gath)
    assert t_gath.any()
    assert tree_d.status() == 0


def test_small_reservation_and_repeated_calls(B):
    # a reservation of 3 log chunks: the rest of the log takes the atomic
    # path; three calls accumulate three times the gradient
    tree, rays, g, ga = _setup(71, 8, 2, 5, 4096 + 3)
    tree_d = B.Tree(tree, "f32")
    dr = B.DeviceRays.from_host(rays)
    gt = torch.from_numpy(g).cuda()
    (g_atom, t_atom), (g_gath, t_gath) = _both(B, tree_d, dr, gt, None, 3 * 256, repeat=3)
    assert _close(g_atom, g_gath) <= 1e-5
    assert torch.equal(t_atom, t_gath)
    (g1, _), (g1g, _) = _both(B, tree_d, dr, gt, None, 1 << 22, repeat=1)
    assert _close(3 * g1g, g_gath) <= 1e-5
    assert tree_d.status() == 0


def test_gather_at_full_training_size(B):
    tree = I.config2_tree()
    rays = I.config2_rays(n_views=8)[0]
    tree_d = B.Tree(tree, "bf16")
    dr = B.DeviceRays.from_host(rays)
    g = torch.from_numpy(np.random.default_rng(9).standard_normal((rays.n, 3)).astype(np.float32) * 1e-3).cuda()
    (g_atom, t_atom), (g_gath, t_gath) = _both(B, tree_d, dr, g, None, 1 << 27)
    assert _close(g_atom, g_gath) <= 1e-5
    assert torch.equal(t_atom, t_gath)
    assert tree_d.status() == 0
