"""Pins of the oracle's time slice (Sec. 7; the caption of the HH-colour
figure: at a fixed time t the hyper angle gamma(t) is constant and the 4D
harmonics reduce to 3D spherical harmonics with coefficients
s_lm = sum_{n >= l} w_nlm R_nl(gamma(t))).

* Rendering the slice (plain SH colour, the slice's density) reproduces the
  HH render at time t: the two regroup one double sum, so they agree to
  rounding (1e-12) on every output, for sigmoid and identity colour and for
  signed densities.
* At gamma = pi/2 (w_gamma = 0) the Gegenbauer values at 0 are known
  (C^1_0 = 1, C^1_2 = -1, C^2_0 = 1, C^2_2 = -2, C^{l+1}_0 = 1), so each
  coefficient is one or two terms of the leaf's w_HH.
* The slice's density is the density the render composites: with colour
  fixed to one channel value the render's alpha equals that of the slice.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2202_06088_gb300 import inputs as I

from test_oracle_render import _random_rays


def _tree(seed, K, deg, depth, signed=False):
    rng = np.random.default_rng(seed)
    st = I.random_mixed_tree(depth, seed, p_leaf=0.3, p_empty=0.2)
    return rng, I.make_coefficients(rng, st, K=K, T=7, hh_degree=deg, mean_sigma=8.0, signed_density=signed)


@pytest.mark.parametrize("K,deg,depth,act,signed,t", [
    (4, 1, 3, "sigmoid", False, 0.0),
    (8, 2, 4, "sigmoid", True, 0.37),
    (16, 3, 4, "identity", False, 0.81),
    (5, 3, 3, "sigmoid", True, 1.0),
])
def test_slice_render_equals_hh_render(K, deg, depth, act, signed, t):
    rng, tree = _tree(100 + K + deg, K, deg, depth, signed)
    rays = _random_rays(rng, 600)
    rays.times[:] = np.float32(t)
    ref = oracle.render(tree, rays, act=act)
    sl = oracle.slice_at(tree, float(np.float32(t)))
    got = oracle.render_slice(tree, sl, rays, act=act)
    assert (ref["alpha"] > 0.01).mean() > 0.2
    for k in ("rgb", "alpha", "tau"):
        assert np.abs(got[k] - ref[k]).max() <= 1e-12, k
    fin = np.isfinite(ref["depth"])
    assert np.array_equal(fin, np.isfinite(got["depth"]))
    assert np.abs(got["depth"][fin] - ref["depth"][fin]).max() <= 1e-12
    assert np.array_equal(got["nseg"], ref["nseg"])


def test_slice_at_right_angle_hyper_angle():
    """w_gamma = 0 gives gamma = pi sigmoid(0) = pi/2: cos = 0, sin = 1."""
    rng, tree = _tree(7, 6, 3, 3)
    tree = tree.with_coeffs(w_gamma=np.zeros_like(tree.w_gamma))
    sl = oracle.slice_at(tree, 0.4)
    L = oracle.lib()
    A = lambda n, l: L.or_hh_norm(n, l)
    w = tree.w_hh.astype(np.float64)                       # [3][N_h][leaf]
    ix = oracle.hh_index
    for ch in range(3):
        for m in (0,):
            np.testing.assert_allclose(sl["sh"][:, ch, 0], A(0, 0) * w[ch, ix(0, 0, 0)] - A(2, 0) * w[ch, ix(2, 0, 0)],
                                       rtol=0, atol=1e-12)
        for m in (-1, 0, 1):
            np.testing.assert_allclose(sl["sh"][:, ch, 2 + m],
                                       A(1, 1) * w[ch, ix(1, 1, m)] - 2.0 * A(3, 1) * w[ch, ix(3, 1, m)],
                                       rtol=0, atol=1e-12)
        for l in (2, 3):
            for m in range(-l, l + 1):
                np.testing.assert_allclose(sl["sh"][:, ch, l * l + l + m], A(l, l) * w[ch, ix(l, l, m)],
                                           rtol=0, atol=1e-12)


def test_slice_density_is_the_basis_projection():
    """sigma = ReLU(a(u) . w_sigma) with a(u) lerped between frames (A6)."""
    _, tree = _tree(11, 5, 2, 3, signed=True)
    t = 0.6
    u = t * (tree.T - 1)
    f0 = int(math.floor(u))
    fr = u - f0
    a = (1 - fr) * tree.basis_A[f0].astype(np.float64) + fr * tree.basis_A[f0 + 1].astype(np.float64)
    pre = a @ tree.w_sigma.astype(np.float64)
    sl = oracle.slice_at(tree, t)
    np.testing.assert_allclose(sl["sigma"], np.maximum(pre, 0.0), rtol=0, atol=1e-12)
    assert (pre < 0).any() and (pre > 0).any()
