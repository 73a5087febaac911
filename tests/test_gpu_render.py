"""GPU parity of the forward path through the C ABI: trace (visited leaves),
render in FP32 (plain and packet kernels) and BF16, against the FP64 oracle
on the same seeded inputs.

Tolerances (from the task's numerical bar): FP32 colour/alpha within 1e-4 max
abs on a [0, 1] scale; BF16-stored coefficients within 4e-3 max abs and
>= 50 dB PSNR against the oracle on the unrounded coefficients, and within
1e-4 against the oracle on the BF16-rounded coefficients.  Leaf sequences
must match exactly, except on rays whose oracle decision margin is below the
rounding of an FP32 traversal (reading A8; fewer than 0.1 % of the rays).
"""
import numpy as np
import pytest

import oracle
from paper_2202_06088_gb300 import inputs as I

from helpers import MAX_EXEMPT_FRACTION, compare_traces, exempt_fraction, nseg_differences_unexplained, psnr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(cuda_lib):
    from paper_2202_06088_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def c1():
    return I.config1_tree()


@pytest.fixture(scope="module")
def c1_rays():
    return I.config1_rays()[0]


def _gpu_trace(B, tree_d, rays, max_out):
    dr = B.DeviceRays.from_host(rays)
    tr = B.neuvv_trace(tree_d, dr, max_out)
    return {k: v.cpu().numpy() for k, v in tr.items()}


def _render(B, tree_d, rays, kernel, t_stop=1e-4, act="sigmoid"):
    dr = B.DeviceRays.from_host(rays)
    out = B.neuvv_render(tree_d, dr, t_stop=t_stop, act=act, kernel=kernel)
    return {k: v.cpu().numpy() for k, v in out.items()}


def _ambiguous_stop(ref):
    """Rays whose optical depth passes the early-stop threshold within 1e-3."""
    return ref["stop_margin"] < 1e-3


def _check_render(ref, got, tol, tree):
    """Colour and alpha within tol everywhere; depth within 1e-3 where the
    oracle's alpha is above 1e-3; composited-segment counts equal except on
    rays where the oracle marks the early stop or the traversal ambiguous
    (few of them)."""
    assert np.abs(got["rgb"] - ref["rgb"]).max() <= tol, np.abs(got["rgb"] - ref["rgb"]).max()
    assert np.abs(got["alpha"] - ref["alpha"]).max() <= tol
    fin = np.isfinite(ref["depth"]) & (ref["alpha"] > 1e-3)
    assert np.all(np.isfinite(got["depth"][fin]))
    assert np.abs(got["depth"][fin] - ref["depth"][fin]).max() <= 1e-3
    bad = nseg_differences_unexplained(ref, got, tree)
    assert len(bad) == 0, bad[:10]
    assert exempt_fraction(ref, tree) < MAX_EXEMPT_FRACTION


def test_trace_matches_oracle_c1(B, c1, c1_rays):
    tree_d = B.Tree(c1, "f32")
    ref = oracle.trace(c1, c1_rays, max_out=96)
    got = _gpu_trace(B, tree_d, c1_rays, 96)
    exempt, bad = compare_traces(c1, ref, got, 96)
    assert bad == [], bad[:10]
    print(f"exempt rays: {len(exempt)} of {c1_rays.n}")
    assert len(exempt) < MAX_EXEMPT_FRACTION * c1_rays.n
    assert tree_d.status() == 0


@pytest.mark.parametrize("seed,depth", [(1, 4), (2, 5), (5, 6)])
def test_trace_matches_oracle_mixed_trees(B, seed, depth):
    rng = np.random.default_rng(seed)
    st = I.random_mixed_tree(depth, seed)
    tree = I.make_coefficients(rng, st, K=2, T=3, hh_degree=1)
    from test_oracle_render import _random_rays
    rays = _random_rays(rng, 3000 + 17)   # several tiles and a ragged tail
    tree_d = B.Tree(tree, "f32")
    mo = 4 * (1 << depth)
    ref = oracle.trace(tree, rays, max_out=mo)
    got = _gpu_trace(B, tree_d, rays, mo)
    exempt, bad = compare_traces(tree, ref, got, mo)
    assert bad == [], bad[:10]
    assert len(exempt) < MAX_EXEMPT_FRACTION * rays.n + 1


@pytest.mark.parametrize("kernel", ["plain", "packet"])
def test_render_fp32_matches_oracle_c1(B, c1, c1_rays, kernel):
    tree_d = B.Tree(c1, "f32")
    ref = oracle.render(c1, c1_rays)
    got = _render(B, tree_d, c1_rays, kernel)
    _check_render(ref, got, 1e-4, c1)
    assert tree_d.status() == 0


def test_render_bf16_against_unrounded_and_rounded_oracle(B, c1, c1_rays):
    tree_d = B.Tree(c1, "bf16")
    got = _render(B, tree_d, c1_rays, "packet")
    ref = oracle.render(c1, c1_rays)
    err = np.abs(got["rgb"] - ref["rgb"]).max()
    assert err <= 4e-3, err
    assert psnr(got["rgb"], ref["rgb"]) >= 50.0
    rounded = c1.with_coeffs(oracle.round_bf16(c1.w_sigma), oracle.round_bf16(c1.w_gamma), oracle.round_bf16(c1.w_hh))
    ref_q = oracle.render(rounded, c1_rays)
    _check_render(ref_q, got, 1e-4, rounded)


@pytest.mark.parametrize("K,deg", [(4, 1), (16, 3), (31, 2)])
def test_render_other_shapes_and_identity_activation(B, K, deg):
    rng = np.random.default_rng(40 + K)
    st = I.random_mixed_tree(5, 40 + K, p_leaf=0.2, p_empty=0.2)
    tree = I.make_coefficients(rng, st, K=K, T=7, hh_degree=deg, mean_sigma=12.0, signed_density=True)
    from test_oracle_render import _random_rays
    rays = _random_rays(rng, 2048 + 5)
    rays.times[:] = rng.uniform(0, 1, rays.n).astype(np.float32)
    for act in ("sigmoid", "identity"):
        ref = oracle.render(tree, rays, act=act)
        for kernel in ("plain", "packet"):
            td = B.Tree(tree, "f32")
            got = _render(B, td, rays, kernel, act=act)
            _check_render(ref, got, 1e-4 if act == "sigmoid" else 3e-4, tree)


def test_render_edge_cases(B, c1):
    tree_d = B.Tree(c1, "f32")
    # empty batch
    empty = I.Rays(np.zeros((3, 0), np.float32), np.zeros((3, 0), np.float32), np.zeros(0, np.float32))
    out = _render(B, tree_d, empty, "packet")
    assert out["rgb"].shape == (0, 3)
    # rays that miss, start inside, run along axes, and a zero direction
    o = np.array([[5, 0.5, 0.5], [0.5, 0.5, 0.5], [-1, 0.5, 0.5], [0.5, -1, 0.5], [0.5, 0.5, 2.0], [0.3, 0.3, 0.3]],
                 np.float32).T
    d = np.array([[1, 0, 0], [0.3, -0.2, 0.9], [1, 0, 0], [0, 1, 0], [0, 0, -1], [0, 0, 0]], np.float32).T
    rays = I.Rays(np.ascontiguousarray(o), np.ascontiguousarray(d), np.full(6, 0.5, np.float32))
    good = rays.subset(np.arange(5))
    ref = oracle.render(c1, good)
    got = _render(B, tree_d, rays, "packet")
    assert np.abs(got["rgb"][:5] - ref["rgb"]).max() <= 1e-4
    assert got["alpha"][0] == 0.0 and got["alpha"][5] == 0.0 and np.all(got["rgb"][5] == 0.0)
    assert tree_d.status() == 0


def test_render_stops_early_and_respects_t_stop_zero(B, c1, c1_rays):
    tree_d = B.Tree(c1, "f32")
    ref0 = oracle.render(c1, c1_rays, t_stop=0.0)
    got0 = _render(B, tree_d, c1_rays, "packet", t_stop=0.0)
    _check_render(ref0, got0, 1e-4, c1)
    got = _render(B, tree_d, c1_rays, "packet")
    assert (got["nseg"] <= got0["nseg"]).all() and (got["nseg"] < got0["nseg"]).any()
