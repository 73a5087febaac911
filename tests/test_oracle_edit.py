"""Pins of the oracle's appearance edits (Sec. 5 "Appearance editing": the
terminating voxel where a ray's accumulated alpha passes a threshold, 0.99 in
the paper; per-voxel target colour c_d, density sigma_d and times t_d blended
into the render).

* Picking on a constant density sigma0: the alpha 1 - exp(-sigma0 s) passes the
  threshold at s* = ln(1 / (1 - threshold)) / sigma0 from the entry, so the
  picked leaf is the one holding the point at s* on the ray (brute force over
  the leaf boxes); rays whose box chord is shorter pick nothing.
* With no active edit (beta = 0 and no density, or ray times before t_d) the
  edited render is the render.
* Editing every voxel (t_d = 0, beta = 1, constant sigma_d and c_d) gives the
  closed form alpha = 1 - exp(-sigma_d L), rgb = alpha c_d over the box chord L.
* Painting gives each picked leaf the mean colour of the rays that picked it.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2202_06088_gb300 import inputs as I

from test_oracle_render import _box_chord, _const_tree, _random_rays


def test_pick_on_constant_density():
    sigma0 = float(np.float32(12.0))
    tree = _const_tree(3, sigma0)
    rng = np.random.default_rng(21)
    rays = _random_rays(rng, 400)
    thr = 0.99
    got = oracle.pick(tree, rays, thr, t_stop=0.0)
    tr = oracle.trace(tree, rays, max_out=64)
    s_star = math.log(1.0 / (1.0 - thr)) / sigma0
    for i in range(rays.n):
        o = rays.origins[:, i].astype(np.float64)
        d = rays.dirs[:, i].astype(np.float64)
        L = _box_chord(o, d)
        if L < s_star - 1e-9:
            assert got[i] == -1
            continue
        # the leaf whose segment holds the point at s* past the entry
        c = tr["count"][i]
        entry = tr["t0"][i, 0]
        k = np.searchsorted(tr["t1"][i, :c] - entry, s_star - 1e-12)
        assert got[i] == tr["leaf"][i, k], i
    assert (got >= 0).mean() > 0.2


def test_no_active_edit_is_the_render():
    rng = np.random.default_rng(22)
    st = I.random_mixed_tree(4, 22, p_leaf=0.3, p_empty=0.2)
    tree = I.make_coefficients(rng, st, K=4, T=5, hh_degree=2, mean_sigma=8.0)
    rays = _random_rays(rng, 300)
    rays.times[:] = np.float32(0.3)
    ref = oracle.render(tree, rays)
    e = np.tile([0.9, 0.1, 0.4, -1.0, 0.0], (tree.n_leaves, 1))
    got = oracle.render_edit(tree, rays, e, beta=0.0)
    for k in ("rgb", "alpha", "tau"):
        np.testing.assert_array_equal(got[k], ref[k])
    np.testing.assert_allclose(got["depth"], ref["depth"], rtol=1e-14)   # midpoint summed in another order
    e[:, 3] = 50.0
    e[:, 4] = 0.31                                  # after the rays' time
    got = oracle.render_edit(tree, rays, e, beta=1.0)
    for k in ("rgb", "alpha", "tau"):
        np.testing.assert_array_equal(got[k], ref[k])
    np.testing.assert_allclose(got["depth"], ref["depth"], rtol=1e-14)


def test_editing_every_voxel_closed_form():
    tree = _const_tree(3, 2.0)
    rng = np.random.default_rng(23)
    rays = _random_rays(rng, 300)
    sd = float(np.float32(1.3))
    cd = np.array([0.2, 0.5, 0.9])
    e = np.tile(np.concatenate([cd, [sd, 0.0]]), (tree.n_leaves, 1))
    got = oracle.render_edit(tree, rays, e, beta=1.0, t_stop=0.0)
    L = np.array([_box_chord(rays.origins[:, i].astype(np.float64), rays.dirs[:, i].astype(np.float64))
                  for i in range(rays.n)])
    a = 1.0 - np.exp(-sd * L)
    np.testing.assert_allclose(got["alpha"], a, rtol=0, atol=1e-12)
    np.testing.assert_allclose(got["rgb"], a[:, None] * cd[None, :], rtol=0, atol=1e-12)


def test_paint_means():
    leaves = np.array([3, 3, -1, 7, 3, 7])
    cols = np.array([[0.1, 0.2, 0.3], [0.3, 0.2, 0.1], [1, 1, 1], [0.5, 0.5, 0.5], [0.2, 0.2, 0.2], [0.0, 0.0, 1.0]])
    e = oracle.paint(10, leaves, cols, 4.0, 0.25)
    np.testing.assert_allclose(e[3], [0.2, 0.2, 0.2, 4.0, 0.25])
    np.testing.assert_allclose(e[7], [0.25, 0.25, 0.75, 4.0, 0.25])
    assert np.all(e[[0, 1, 2, 4, 5, 6, 8, 9], 4] == 2.0)     # untouched leaves stay inactive
