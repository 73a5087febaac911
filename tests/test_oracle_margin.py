"""Pins for the oracle's traversal decision margin (reading A8: leaf sequences
are compared exactly except on rays whose two nearest order-deciding plane
crossings are closer than the traversals' rounding).

The margin of a ray is the smallest distance along it between two crossings
of planes of different axes whose order decides which occupied leaves the
ray visits.  It is pinned by what it promises: moving every plane crossing
of a ray by less than half its margin -- a shifted and slightly turned line --
leaves the visited leaves unchanged (checked against a brute-force slab test
of every leaf box), and by hand-built rays through cell edges.
"""
import numpy as np
import pytest

import oracle
from paper_2202_06088_gb300 import inputs as I

from test_oracle_render import _brute_force


def _rays(o, d):
    o = np.asarray(o, np.float64).reshape(3, -1)
    d = np.asarray(d, np.float64).reshape(3, -1)
    return I.Rays(o, d, np.full(o.shape[1], 0.5))


def _full(depth):
    rng = np.random.default_rng(3)
    return I.make_coefficients(rng, I.full_tree(depth), K=2, T=3, hh_degree=1)


def test_ray_through_an_edge_between_leaves_has_zero_margin():
    """N = 4 cells per axis, every finest cell its own leaf.  The diagonal ray
    in the plane z = 0.3 through (0.5, 0.5) crosses x = k/4 and y = k/4 at the
    same instants: the cells on either side of each edge are different
    leaves, so the order of the two crossings decides the sequence."""
    tree = _full(2)
    d = np.array([1.0, 1.0, 0.0]) / np.sqrt(2.0)
    o = np.array([0.5, 0.5, 0.3]) - 3.0 * d
    tr = oracle.trace(tree, _rays(o, d), max_out=32)
    assert tr["margin"][0] == 0.0


def test_axis_ray_through_cell_centres_has_no_margin():
    """A ray along +x through the centres of cells crosses planes of one
    axis only: no order to decide."""
    tree = _full(3)
    tr = oracle.trace(tree, _rays([-1.0, 0.3125, 0.5625], [1.0, 0.0, 0.0]), max_out=32)
    assert tr["count"][0] == 8
    assert np.isinf(tr["margin"][0])


def test_margin_is_the_gap_between_the_two_crossings():
    """The diagonal ray of the first test, moved back along x by g d_x: every
    crossing of a plane x = k/4 now comes a distance g (along the unit
    direction) after the crossing of y = k/4, and each such pair decides the
    sequence, so the margin is g, reported in finest cells of 1/4."""
    tree = _full(2)
    d = np.array([1.0, 1.0, 0.0]) / np.sqrt(2.0)
    g = 2e-4
    o = np.array([0.5, 0.5, 0.3]) - 3.0 * d - np.array([g * d[0], 0.0, 0.0])
    tr = oracle.trace(tree, _rays(o, d), max_out=32)
    assert abs(tr["margin"][0] - g / 0.25) < 1e-9


def test_margin_ignores_near_ties_whose_order_does_not_matter():
    """Eight leaves of level 1 (each 2 x 2 x 2 finest cells).  The ray
    y = 2x + 1/4 in the plane z = 0.3 enters through x = 0 exactly where it
    crosses y = 1/4 and later crosses x = 1/4 exactly where it crosses
    y = 3/4: both ties lie inside one leaf, so neither order decides
    anything.  The pairs that do decide are the crossing of y = 1/2 (between
    the two leaves, at x = 1/8) and the x crossings next to it, at x = 0 and
    x = 1/4: the margin is (1/8) sqrt(5) along the ray, in cells of 1/4."""
    rng = np.random.default_rng(5)
    g = np.stack(np.meshgrid(np.arange(2), np.arange(2), np.arange(2), indexing="ij"), -1).reshape(-1, 3)
    eight = I.make_coefficients(rng, I.build_tree(2, np.full(8, 1), g), K=2, T=3, hh_degree=1)
    d = np.array([1.0, 2.0, 0.0]) / np.sqrt(5.0)
    o = np.array([0.25, 0.75, 0.3]) - 3.0 * d
    tr = oracle.trace(eight, _rays(o, d), max_out=8)
    assert tr["count"][0] == 2
    assert abs(tr["margin"][0] - 0.125 * np.sqrt(5.0) / 0.25) < 1e-9


def _edge_rays(rng, n, depth):
    """Rays through points within 1e-3 cells of random cell edges, so that
    many have small margins; a third of the edges lie on the root box's faces
    (near-ties at the entry or the exit)."""
    N = 1 << depth
    o = np.empty((3, n))
    d = np.empty((3, n))
    for i in range(n):
        p = rng.uniform(0.0, 1.0, 3)
        ax = rng.choice(3, 2, replace=False)
        for a in ax:
            p[a] = rng.integers(1, N) / N + rng.uniform(-1e-3, 1e-3) / N
        if rng.random() < 1.0 / 3.0:
            p[ax[0]] = float(rng.integers(0, 2))
        v = rng.standard_normal(3)
        v /= np.linalg.norm(v)
        o[:, i] = p - 2.5 * v
        d[:, i] = v
    return o, d


def _perturbed(rng, o, d, delta, t_max):
    """A line whose plane crossings each move by less than delta (along the
    original unit direction): origin shifted by at most delta/2 |d_a| per
    axis, each direction component scaled by at most delta / (2 t_max)."""
    u = rng.uniform(-1.0, 1.0, 3)
    v = rng.uniform(-1.0, 1.0, 3)
    return o + u * 0.45 * delta * np.abs(d), d * (1.0 + v * 0.45 * delta / t_max)


@pytest.mark.parametrize("seed,depth", [(11, 3), (12, 4), (13, 3)])
def test_crossings_moved_within_half_the_margin_keep_the_leaves(seed, depth):
    rng = np.random.default_rng(seed)
    tree = I.make_coefficients(rng, I.random_mixed_tree(depth, seed, 0.35, 0.25), K=2, T=3, hh_degree=1)
    o, d = _edge_rays(rng, 150, depth)
    tr = oracle.trace(tree, _rays(o, d), max_out=4 * (1 << depth))
    cell = 1.0 / (1 << depth)
    small = 0
    for i in range(o.shape[1]):
        ids = tr["leaf"][i, :tr["count"][i]]
        assert np.array_equal(ids, _brute_force(tree, o[:, i], d[:, i])[0])
        m = tr["margin"][i] * cell
        small += m < 1e-2 * cell
        delta = 0.5 * min(m, 0.05 * cell)
        if delta == 0.0:
            continue
        for _ in range(4):
            po, pd = _perturbed(rng, o[:, i], d[:, i], delta, 4.5)
            assert np.array_equal(_brute_force(tree, po, pd)[0], ids), (i, tr["margin"][i])
    assert small >= 5        # the rays do come close to order-deciding edges


def test_few_rays_of_the_render_workload_have_small_margins():
    """On the 128x128 view of the depth-6 tree, below 0.1 % of the rays have
    a decision margin under 1e-4 finest cells (exact ties are not typical),
    and the margins up to the early stop are never smaller than over the
    whole ray (and larger on some rays: pairs behind the stop are left out)."""
    tree = I.config1_tree()
    rays, _ = I.config1_rays()
    ref = oracle.render(tree, rays)
    tr = oracle.trace(tree, rays, max_out=256)
    assert (ref["trace_margin"] < 1e-4).mean() < 1e-3
    assert np.all(ref["trace_margin"] >= tr["margin"])
    assert (ref["trace_margin"] > tr["margin"]).any()
    assert np.isfinite(ref["trace_margin"]).any()
