"""Pin for the oracle's analytic gradient (Sec. 4.3 "Optimization"): FP64
central finite differences of the oracle's forward render, which uses none of
the adjoint formulas, on a depth-4 tree."""
import numpy as np
import pytest

import oracle
from paper_2202_06088_gb300 import inputs as I

from test_oracle_render import _random_rays


def _loss(tree, rays, g, ga, ws, wg, wh, t_stop, act):
    ot = oracle.OracleTree(tree, ws, wg, wh)
    out = oracle.render(tree, rays, t_stop=t_stop, act=act, otree=ot)
    return float((out["rgb"] * g).sum() + (out["alpha"] * ga).sum()), out


@pytest.mark.parametrize("act,signed,t_stop", [("sigmoid", False, 0.0), ("identity", True, 0.0),
                                               ("sigmoid", True, 1e-4)])
def test_gradient_matches_central_differences(act, signed, t_stop):
    rng = np.random.default_rng(20)
    st = I.random_mixed_tree(4, 21, p_leaf=0.25, p_empty=0.2)
    tree = I.make_coefficients(rng, st, K=4, T=5, hh_degree=3, mean_sigma=8.0, signed_density=signed)
    rays = _random_rays(rng, 48)
    rays.times[:] = np.float32(0.4)
    ws = tree.w_sigma.astype(np.float64)
    wg = tree.w_gamma.astype(np.float64)
    wh = tree.w_hh.astype(np.float64)
    g = rng.standard_normal((rays.n, 3))
    ga = rng.standard_normal(rays.n)
    L0, out0 = _loss(tree, rays, g, ga, ws, wg, wh, t_stop, act)
    if t_stop > 0:
        # keep rays whose early-stop decision is not within reach of the step
        keep = out0["stop_margin"] > 1e-3
        rays = rays.subset(np.nonzero(keep)[0])
        g, ga = g[keep], ga[keep]
    an = oracle.render_grad(tree, rays, g, ga, t_stop=t_stop, act=act,
                            otree=oracle.OracleTree(tree, ws, wg, wh))
    touched = np.nonzero(np.abs(an["w_hh"]).sum((0, 1)) > 0)[0]
    assert touched.size > 5
    # pre-activation of the density at t = 0.4 (to stay clear of the ReLU kink)
    u = np.float32(0.4) * (tree.T - 1)
    f0 = int(np.floor(u))
    fr = float(u) - f0
    a_row = (1 - fr) * tree.basis_A[f0].astype(np.float64) + fr * tree.basis_A[f0 + 1].astype(np.float64)
    pre = a_row @ ws
    h = 1e-6
    checked = 0
    for leaf in rng.choice(touched, size=min(12, touched.size), replace=False):
        if abs(pre[leaf]) < 1e-3:
            continue
        picks = [("w_sigma", (k, leaf)) for k in range(tree.K)] + [("w_gamma", (k, leaf)) for k in range(tree.K)]
        picks += [("w_hh", (ch, int(j), leaf)) for ch in range(3) for j in rng.choice(tree.N_h, 4, replace=False)]
        for name, idx in picks:
            arrs = {"w_sigma": ws, "w_gamma": wg, "w_hh": wh}
            base = arrs[name][idx]
            arrs[name][idx] = base + h
            Lp, _ = _loss(tree, rays, g, ga, ws, wg, wh, t_stop, act)
            arrs[name][idx] = base - h
            Lm, _ = _loss(tree, rays, g, ga, ws, wg, wh, t_stop, act)
            arrs[name][idx] = base
            fd = (Lp - Lm) / (2 * h)
            a = an[name][idx]
            assert abs(fd - a) <= 1e-6 * abs(a) + 2e-9, (name, idx, fd, a)
            checked += 1
    assert checked > 50


def test_gradient_is_zero_for_untouched_leaves_and_linear_in_upstream():
    rng = np.random.default_rng(22)
    st = I.random_mixed_tree(4, 23)
    tree = I.make_coefficients(rng, st, K=3, T=4, hh_degree=2)
    rays = _random_rays(rng, 32)
    g = rng.standard_normal((rays.n, 3))
    a1 = oracle.render_grad(tree, rays, g)
    a2 = oracle.render_grad(tree, rays, 2.5 * g)
    for k in a1:
        assert np.allclose(a2[k], 2.5 * a1[k], rtol=1e-12, atol=1e-15)
    tr = oracle.trace(tree, rays, max_out=128)
    hit = np.zeros(tree.n_leaves, bool)
    for i in range(rays.n):
        hit[tr["leaf"][i, :tr["count"][i]]] = True
    assert np.all(a1["w_hh"][:, :, ~hit] == 0) and np.all(a1["w_sigma"][:, ~hit] == 0)
