"""The differentiable-render workload at full size: the five-ellipsoid scene at
depth 8 (1,281,162 leaves), 262,144 rays drawn from 16 cameras x 16 time
stamps, MSE loss against target images rendered (by the oracle) from the same
tree with every coefficient perturbed by N(0, 0.05).

* The loss through the torch.autograd.Function matches the oracle's loss.
* The fused adjoint over all 262,144 rays, given the oracle's dL/dC, matches
  the oracle's analytic gradient: relative 1e-4 in L2 over all leaves, every
  entry within 1e-4 of its plane's largest entry.
* On the leaves of one depth-4 subtree, the GPU gradient matches FP64 central
  differences of the oracle's loss within relative 1e-3 (Sec. 4.3
  "Optimization": the coefficients are fitted by gradient descent).
"""
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


@pytest.fixture(scope="module")
def case():
    tree = I.config3_tree()
    rays = I.config3_rays()
    target = oracle.render(I.perturbed(tree, seed=3000), rays)["rgb"]
    return tree, rays, target


def _planes(tree_d, g):
    info = tree_d.info
    K, Kp, Nh = info.K, info.K_pad, info.N_h
    g = g.cpu().numpy().astype(np.float64)
    return {"w_sigma": g[:, :K].T, "w_gamma": g[:, Kp:Kp + K].T,
            "w_hh": g[:, 2 * Kp:2 * Kp + 3 * Nh].T.reshape(3, Nh, -1)}


def test_workload_size(case):
    tree, rays, _ = case
    assert tree.depth == 8 and tree.n_leaves == 1_281_162 and rays.n == 262_144


def test_loss_and_adjoint_over_the_batch(B, case):
    tree, rays, target = case
    n = rays.n
    tree_d = B.Tree(tree, "f32", with_optimizer=True)
    dr = B.DeviceRays.from_host(rays)
    tgt = torch.from_numpy(target.astype(np.float32)).cuda()
    coeffs = tree_d.master().clone().requires_grad_(True)
    rgb, alpha, _ = B.render_differentiable(coeffs, tree_d, dr)
    loss = ((rgb - tgt) ** 2).sum() / n
    loss.backward()
    ref = oracle.render(tree, rays)
    ref_loss = float(((ref["rgb"] - target) ** 2).sum() / n)
    assert abs(loss.item() - ref_loss) <= 1e-4 * ref_loss
    # the adjoint, fed the oracle's dL/dC (rays at the early-stop threshold excluded)
    g = 2.0 * (ref["rgb"] - target) / n
    keep = ref["stop_margin"] > 1e-3
    assert keep.mean() > 0.99
    g[~keep] = 0.0
    out = B.neuvv_render(tree_d, dr, kernel="packet")
    grad = B.neuvv_render_backward(tree_d, dr, out, torch.from_numpy(g.astype(np.float32)).cuda(), kernel="packet")
    got = _planes(tree_d, grad)
    want = oracle.render_grad(tree, rays, g)
    for k in ("w_sigma", "w_gamma", "w_hh"):
        a, b = got[k].ravel(), want[k].ravel()
        assert np.linalg.norm(a - b) <= 1e-4 * np.linalg.norm(b), k
        assert np.abs(a - b).max() <= 1e-4 * np.abs(b).max(), k
    # the autograd gradient is the same adjoint (its dL/dC is the GPU's own)
    assert torch.count_nonzero(coeffs.grad).item() > 0
    assert tree_d.status() == 0


def _rays_through_box(rays, lo, hi):
    """Rays whose line meets the box [lo, hi] in front of the origin (slab test)."""
    o = rays.origins.astype(np.float64)
    d = rays.dirs.astype(np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        t0 = (lo[:, None] - o) * inv
        t1 = (hi[:, None] - o) * inv
    tmin = np.nanmax(np.minimum(t0, t1), 0)
    tmax = np.nanmin(np.maximum(t0, t1), 0)
    return np.nonzero(tmax >= np.maximum(tmin, 0.0))[0]


def test_gradient_matches_central_differences_on_a_depth4_subtree(B, case):
    tree, rays, target = case
    n = rays.n
    st = tree.structure
    # the level-4 node whose subtree (4 levels under it) holds the most leaves
    lvl, xyz = st.leaf_level, st.leaf_coords
    deep = lvl >= 4
    anc = xyz[deep] >> (lvl[deep] - 4)[:, None]
    keys, counts = np.unique(anc[:, 0] * 256 + anc[:, 1] * 16 + anc[:, 2], return_counts=True)
    key = keys[np.argmax(counts)]
    cell = np.array([key // 256, (key // 16) % 16, key % 16])
    in_sub = np.nonzero(deep)[0][np.all(anc == cell, 1)]
    assert in_sub.size >= 50
    lo = np.asarray(tree.aabb_min, np.float64) + cell / 16.0
    sub = _rays_through_box(rays, lo, lo + 1.0 / 16.0)
    assert sub.size >= 100
    r_sub = rays.subset(sub)
    # no early stop: the loss is smooth in every coefficient
    base = oracle.render(tree, rays, t_stop=0.0)
    g = 2.0 * (base["rgb"] - target) / n
    tree_d = B.Tree(tree, "f32")
    dr = B.DeviceRays.from_host(rays)
    out = B.neuvv_render(tree_d, dr, t_stop=0.0, kernel="packet")
    grad = B.neuvv_render_backward(tree_d, dr, out, torch.from_numpy(g.astype(np.float32)).cuda(), t_stop=0.0,
                                   kernel="packet")
    got = _planes(tree_d, grad)
    ws, wg, wh = (tree.w_sigma.astype(np.float64), tree.w_gamma.astype(np.float64), tree.w_hh.astype(np.float64))
    arrs = {"w_sigma": ws, "w_gamma": wg, "w_hh": wh}
    t_sub = target[sub]

    def L_sub():
        o = oracle.render(tree, r_sub, t_stop=0.0, otree=oracle.OracleTree(tree, ws, wg, wh))
        return float(((o["rgb"] - t_sub) ** 2).sum() / n)

    # the subtree's leaves with the largest oracle gradient
    an = oracle.render_grad(tree, r_sub, g[sub], t_stop=0.0)
    mag = np.abs(an["w_hh"][:, :, in_sub]).sum((0, 1)) + np.abs(an["w_sigma"][:, in_sub]).sum(0)
    leaves = in_sub[np.argsort(-mag)[:4]]
    h = 1e-6
    worst = 0.0
    for leaf in leaves:
        for name, idx in [("w_sigma", (0, leaf)), ("w_sigma", (5, leaf)), ("w_gamma", (2, leaf)),
                          ("w_hh", (0, 0, leaf)), ("w_hh", (1, 7, leaf)), ("w_hh", (2, 12, leaf))]:
            b0 = arrs[name][idx]
            arrs[name][idx] = b0 + h
            lp = L_sub()
            arrs[name][idx] = b0 - h
            lm = L_sub()
            arrs[name][idx] = b0
            fd = (lp - lm) / (2 * h)
            scale = max(abs(fd), 1e-3 * np.abs(got[name][..., leaf]).max(), 1e-12)
            worst = max(worst, abs(got[name][idx] - fd) / scale)
    assert worst <= 1e-3, worst
