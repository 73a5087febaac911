"""Pins for the oracle's traversal and compositing (Sec. 4.3 "Rendering",
Eq. volume-rendering, Eq. project-sigma, Eq. project-gamma).

Traversal is checked against brute force (slab test of every leaf box, sorted
by entry); compositing against closed forms and identities.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2202_06088_gb300 import inputs as I


def _leaf_boxes(tree):
    st = tree.structure
    D = st.depth
    lo = st.leaf_coords.astype(np.float64) * (2.0 ** (D - st.leaf_level))[:, None]
    hi = lo + (2.0 ** (D - st.leaf_level))[:, None]
    N = float(1 << D)
    bmin, bmax = np.array(tree.aabb_min), np.array(tree.aabb_max)
    return bmin + lo / N * (bmax - bmin), bmin + hi / N * (bmax - bmin)


def _brute_force(tree, o, d):
    """Every leaf box intersected with the ray by the slab method; positive
    chords sorted by entry distance."""
    d = d / np.linalg.norm(d)
    lo, hi = _leaf_boxes(tree)
    with np.errstate(divide="ignore", invalid="ignore"):
        t0 = (lo - o) / d
        t1 = (hi - o) / d
    tmin = np.where(d == 0, np.where((o >= lo) & (o <= hi), -np.inf, np.inf), np.minimum(t0, t1))
    tmax = np.where(d == 0, np.where((o >= lo) & (o <= hi), np.inf, -np.inf), np.maximum(t0, t1))
    a = np.maximum(tmin.max(1), 0.0)
    b = tmax.min(1)
    keep = b > a
    idx = np.nonzero(keep)[0]
    order = np.argsort(a[idx])
    return idx[order], a[idx][order], b[idx][order]


def _random_rays(rng, n, center=0.5, radius=2.0, inside_frac=0.2):
    o = np.empty((3, n))
    d = np.empty((3, n))
    for i in range(n):
        if rng.random() < inside_frac:
            p = rng.uniform(0.0, 1.0, 3)
        else:
            v = rng.standard_normal(3)
            p = center + radius * v / np.linalg.norm(v)
        tgt = rng.uniform(0.0, 1.0, 3)
        dd = tgt - p if np.linalg.norm(tgt - p) > 1e-3 else rng.standard_normal(3)
        o[:, i] = p
        d[:, i] = dd / np.linalg.norm(dd)
    return I.Rays(o.astype(np.float32), d.astype(np.float32), np.full(n, 0.5, np.float32))


@pytest.mark.parametrize("seed,depth", [(0, 3), (1, 4), (2, 5), (3, 4)])
def test_trace_matches_brute_force(seed, depth):
    rng = np.random.default_rng(seed)
    st = I.random_mixed_tree(depth, seed)
    tree = I.make_coefficients(rng, st, K=2, T=3, hh_degree=1)
    rays = _random_rays(rng, 300)
    tr = oracle.trace(tree, rays, max_out=4 * (1 << depth))
    for i in range(rays.n):
        o = rays.origins[:, i].astype(np.float64)
        d = rays.dirs[:, i].astype(np.float64)
        ids, a, b = _brute_force(tree, o, d)
        c = tr["count"][i]
        assert c == ids.size, (i, c, ids.size)
        assert np.array_equal(tr["leaf"][i, :c], ids)
        assert np.allclose(tr["t0"][i, :c], a, atol=1e-12)
        assert np.allclose(tr["t1"][i, :c], b, atol=1e-12)


def test_trace_on_non_unit_box():
    rng = np.random.default_rng(7)
    st = I.random_mixed_tree(4, 7)
    tree = I.make_coefficients(rng, st, K=2, T=3, hh_degree=1, aabb_min=(-1.0, 0.5, 2.0), aabb_max=(3.0, 1.5, 4.0))
    n = 200
    o = np.empty((3, n))
    d = np.empty((3, n))
    c = np.array([1.0, 1.0, 3.0])
    for i in range(n):
        v = rng.standard_normal(3)
        o[:, i] = c + 6.0 * v / np.linalg.norm(v)
        tgt = rng.uniform([-1.0, 0.5, 2.0], [3.0, 1.5, 4.0])
        d[:, i] = (tgt - o[:, i]) / np.linalg.norm(tgt - o[:, i])
    rays = I.Rays(o.astype(np.float32), d.astype(np.float32), np.zeros(n, np.float32))
    tr = oracle.trace(tree, rays, max_out=64)
    for i in range(n):
        ids, a, b = _brute_force(tree, rays.origins[:, i].astype(np.float64), rays.dirs[:, i].astype(np.float64))
        assert np.array_equal(tr["leaf"][i, :tr["count"][i]], ids)
        assert np.allclose(tr["t1"][i, :ids.size] - tr["t0"][i, :ids.size], b - a, atol=1e-12)


def _const_tree(depth, sigma0, K=1, T=2, degree=1, full=True, seed=0):
    st = I.full_tree(depth) if full else I.random_mixed_tree(depth, seed)
    tree = I.make_coefficients(np.random.default_rng(seed), st, K=K, T=T, hh_degree=degree)
    A = np.zeros((T, K), np.float32)
    A[:, 0] = sigma0
    ws = np.zeros((K, st.n_leaves), np.float32)
    ws[0] = 1.0
    t2 = tree.with_coeffs(w_sigma=ws)
    t2.basis_A = A
    return t2


def _box_chord(o, d):
    d = d / np.linalg.norm(d)
    with np.errstate(divide="ignore"):
        t0 = (0.0 - o) / d
        t1 = (1.0 - o) / d
    a = max(np.minimum(t0, t1).max(), 0.0)
    b = np.maximum(t0, t1).min()
    return max(b - a, 0.0)


def test_constant_density_transmittance_closed_form():
    """Constant sigma0 everywhere: tau = sigma0 * L and alpha = 1 - exp(-sigma0 L)."""
    sigma0 = float(np.float32(1.7))   # the basis table is float32
    tree = _const_tree(3, sigma0)
    rng = np.random.default_rng(8)
    rays = _random_rays(rng, 200)
    out = oracle.render(tree, rays, t_stop=0.0)
    for i in range(rays.n):
        L = _box_chord(rays.origins[:, i].astype(np.float64), rays.dirs[:, i].astype(np.float64))
        assert abs(out["tau"][i] - sigma0 * L) < 1e-12
        assert abs(out["alpha"][i] - (1.0 - math.exp(-sigma0 * L))) < 1e-12


def test_weights_plus_transmittance_is_one():
    tree = I.config1_tree()
    rays, _ = I.config1_rays()
    out = oracle.render(tree, rays)
    assert np.abs(out["alpha"] + np.exp(-out["tau"]) - 1.0).max() < 1e-12


def test_early_stop_after_threshold_crossing():
    """The ray stops after the first segment that brings T below t_stop."""
    sigma0 = 40.0
    tree = _const_tree(4, sigma0)
    rays = I.Rays(np.array([[-1.0], [0.53], [0.47]], np.float32), np.array([[1.0], [0.0], [0.0]], np.float32),
                  np.zeros(1, np.float32))
    full = oracle.trace(tree, rays, max_out=64)
    out = oracle.render(tree, rays, t_stop=1e-4)
    chords = full["t1"][0, :full["count"][0]] - full["t0"][0, :full["count"][0]]
    tau = np.cumsum(sigma0 * chords)
    expected = int(np.argmax(np.exp(-tau) < 1e-4)) + 1
    assert out["nseg"][0] == expected
    assert abs(out["tau"][0] - tau[expected - 1]) < 1e-12


def test_single_voxel_premultiplied_colour_and_depth():
    """One occupied leaf, only w_000 non-zero: c = sigmoid(w / (pi sqrt 2)) for every
    direction and time; C = (1 - exp(-sigma delta)) c; depth = chord midpoint."""
    st = I.build_tree(2, np.array([2]), np.array([[1, 2, 1]]))
    rng = np.random.default_rng(9)
    tree = I.make_coefficients(rng, st, K=3, T=4, hh_degree=2)
    wh = np.zeros_like(tree.w_hh)
    wh[:, 0, 0] = [0.7, -1.3, 2.1]
    tree = tree.with_coeffs(w_hh=wh)
    rays = _random_rays(rng, 100)
    rays.times[:] = rng.uniform(0, 1, rays.n).astype(np.float32)
    out = oracle.render(tree, rays, t_stop=0.0)
    tr = oracle.trace(tree, rays)
    c = 1.0 / (1.0 + np.exp(-wh[:, 0, 0].astype(np.float64) / (math.pi * math.sqrt(2))))
    for i in range(rays.n):
        if tr["count"][i] == 0:
            assert out["alpha"][i] == 0.0 and np.all(out["rgb"][i] == 0.0)
            continue
        a = 1.0 - math.exp(-out["tau"][i])
        assert np.allclose(out["rgb"][i], a * c, atol=1e-14)
        assert abs(out["depth"][i] - 0.5 * (tr["t0"][i, 0] + tr["t1"][i, 0])) < 1e-12 or a < 1e-4


def test_one_hot_density_reproduces_basis_curve():
    """w_sigma = e_k: sigma(t) = A[u, k] at frames u = t (T-1), linear in between."""
    st = I.build_tree(1, np.array([1]), np.array([[0, 0, 0]]))
    rng = np.random.default_rng(10)
    K, T = 4, 7
    tree = I.make_coefficients(rng, st, K=K, T=T, hh_degree=1)
    o = np.array([[-1.0], [0.25], [0.25]], np.float32)
    d = np.array([[1.0], [0.0], [0.0]], np.float32)
    for k in range(K):
        ws = np.zeros((K, 1), np.float32)
        ws[k, 0] = 1.0
        tk = tree.with_coeffs(w_sigma=ws)
        for u in [0.0, 1.0, 2.5, 3.25, 6.0]:
            rays = I.Rays(o, d, np.array([u / (T - 1)], np.float32))
            out = oracle.render(tk, rays, t_stop=0.0)
            f0 = int(math.floor(u))
            f1 = min(f0 + 1, T - 1)
            fr = float(np.float32(u / (T - 1))) * (T - 1) - f0
            ref = (1 - fr) * float(tree.basis_A[f0, k]) + fr * float(tree.basis_A[f1, k])
            assert abs(out["tau"][0] / 0.5 - max(ref, 0.0)) < 1e-12


def test_relu_clamps_negative_density():
    st = I.build_tree(1, np.array([1]), np.array([[0, 0, 0]]))
    tree = I.make_coefficients(np.random.default_rng(11), st, K=2, T=3, hh_degree=1)
    tree = tree.with_coeffs(w_sigma=-np.abs(tree.w_sigma) - 1.0)
    tree.basis_A = np.abs(tree.basis_A) + 0.1
    rays = I.Rays(np.array([[-1.0], [0.25], [0.25]], np.float32), np.array([[1.0], [0.0], [0.0]], np.float32),
                  np.array([0.3], np.float32))
    out = oracle.render(tree, rays)
    assert out["tau"][0] == 0.0 and out["alpha"][0] == 0.0 and out["nseg"][0] == 1


def test_gamma_linear_in_time_changes_colour_through_hh():
    """A leaf with only the (n=1, l=0) harmonic: H_100 = Abar_10 * 2 cos(gamma) * Y_00,
    so the colour is sigmoid(w * Abar_10 * 2 cos(gamma) / (2 sqrt pi)) with
    gamma = pi * sigmoid(b(t) . w_gamma)."""
    st = I.build_tree(1, np.array([1]), np.array([[0, 0, 0]]))
    tree = I.make_coefficients(np.random.default_rng(12), st, K=2, T=3, hh_degree=1)
    wh = np.zeros_like(tree.w_hh)
    wh[:, oracle.hh_index(1, 0, 0), 0] = [1.5, -0.5, 0.25]
    tree = tree.with_coeffs(w_hh=wh)
    rays = I.Rays(np.array([[-1.0], [0.25], [0.25]], np.float32), np.array([[1.0], [0.0], [0.0]], np.float32),
                  np.array([0.0], np.float32))
    out = oracle.render(tree, rays, t_stop=0.0)
    pre = float(tree.basis_B[0] @ tree.w_gamma[:, 0].astype(np.float64))
    gamma = math.pi / (1 + math.exp(-pre))
    abar10 = 2.0 * math.sqrt(2.0 * 2.0 * 1.0 / (math.pi * 2.0))   # (2*0)!! sqrt(2(n+1)(n-l)!/(pi (n+l+1)!)) with n=1,l=0
    h = abar10 * 2.0 * math.cos(gamma) * 0.5 / math.sqrt(math.pi) / 2.0
    c = 1.0 / (1.0 + np.exp(-wh[:, oracle.hh_index(1, 0, 0), 0] * h))
    a = 1.0 - math.exp(-out["tau"][0])
    assert np.allclose(out["rgb"][0], a * c, atol=1e-14)
