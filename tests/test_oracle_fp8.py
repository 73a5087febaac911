"""Pins for the oracle's FP8 E4M3 storage rounding (the storage ablation).

E4M3 is fixed by its definition: 1 sign bit, 4 exponent bits with bias 7, 3
fraction bits, subnormals (exponent field 0) worth m/8 * 2^-6, largest finite
magnitude 448 (the all-ones exponent with fraction 111 is NaN, the only
non-finite code).  The checks below decode every code from that definition,
compare with torch's float8_e4m3fn cast (a library routine), and check the
per-leaf scales by their defining property."""
import numpy as np
import pytest
import torch

import oracle
from paper_2202_06088_gb300 import inputs as I


def e4m3_codes():
    """All finite non-negative E4M3 values, in code order, decoded from the
    definition."""
    vals = []
    for code in range(0x7F):                      # 0x7F is NaN
        e, m = code >> 3, code & 7
        vals.append(m / 8 * 2.0 ** -6 if e == 0 else (1 + m / 8) * 2.0 ** (e - 7))
    return np.array(vals)


def test_definition_gives_448_and_subnormal_spacing():
    v = e4m3_codes()
    assert v[-1] == 448.0 and v[1] == 2.0 ** -9 and np.all(np.diff(v) > 0)
    assert v.size == 127


def test_every_code_is_a_fixed_point():
    v = e4m3_codes()
    both = np.concatenate([v, -v])
    assert np.array_equal(oracle.round_e4m3(both), both)


def test_midpoints_round_to_the_even_code():
    v = e4m3_codes()
    mid = 0.5 * (v[:-1] + v[1:])
    got = oracle.round_e4m3(mid)
    codes = np.arange(v.size)
    even = np.where(codes[:-1] % 2 == 0, v[:-1], v[1:])
    assert np.array_equal(got, even)
    assert np.array_equal(oracle.round_e4m3(-mid), -even)
    # just off the midpoint goes to the nearer code
    assert np.array_equal(oracle.round_e4m3(np.nextafter(mid, np.inf)), v[1:])
    assert np.array_equal(oracle.round_e4m3(np.nextafter(mid, -np.inf)), v[:-1])


def test_matches_torch_float8_cast_on_random_float32():
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.uniform(-448, 448, 20000), rng.standard_normal(20000) * 1e-2,
                        rng.standard_normal(20000) * 1e-3]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(oracle.round_e4m3(x.astype(np.float64)), ref)


def test_saturates_above_448():
    x = np.array([448.0, 460.0, 464.0, 1e6, -1e6])
    assert np.array_equal(oracle.round_e4m3(x), [448, 448, 448, 448, -448])


def test_group_scale_is_the_smallest_fitting_power_of_two():
    rng = np.random.default_rng(6)
    w = (rng.standard_normal((500, 16)) * np.exp(rng.uniform(-12, 8, (500, 1)))).astype(np.float32)
    w[0] = 0
    w[1, :] = 0
    w[1, 3] = 448.0                                  # exactly 448 * 2^0
    w[2, :] = 0
    w[2, 5] = -896.0                                 # exactly 448 * 2^1
    deq, s = oracle.quantize_fp8_groups(w)
    mx = np.abs(w.astype(np.float64)).max(1)
    assert s[0] == 1.0 and np.all(deq[0] == 0)
    assert s[1] == 1.0 and s[2] == 2.0
    e = np.log2(s)
    assert np.array_equal(e, np.round(e))
    nz = mx > 0
    assert np.all(mx[nz] <= 448 * s[nz])
    assert np.all(mx[nz] > 448 * s[nz] / 2)          # half the scale would not fit
    # dequantised / scale is an E4M3 value, the nearest one to w / scale
    q = deq / s[:, None]
    assert np.array_equal(oracle.round_e4m3(q.ravel()), q.ravel())
    assert np.array_equal(q, oracle.round_e4m3((w.astype(np.float64) / s[:, None]).ravel()).reshape(w.shape))
    # relative error of the largest entry within half a spacing (2^-4)
    i = np.arange(w.shape[0])[nz]
    j = np.abs(w).argmax(1)[nz]
    assert np.all(np.abs(deq[i, j] - w[i, j]) <= 2.0 ** -4 * np.abs(w[i, j]))


def test_tree_quantisation_uses_one_scale_per_leaf_and_group():
    tree = I.config1_tree()
    q, scales = oracle.quantize_fp8_tree(tree)
    assert scales.shape == (tree.n_leaves, 3)
    L = tree.n_leaves
    for arr, src, g in ((q.w_sigma.reshape(-1, L), tree.w_sigma.reshape(-1, L), 0),
                        (q.w_gamma.reshape(-1, L), tree.w_gamma.reshape(-1, L), 1),
                        (q.w_hh.reshape(-1, L), tree.w_hh.reshape(-1, L), 2)):
        s = scales[:, g]
        assert np.all(np.abs(src).max(0) <= 448 * s)
        r = arr.astype(np.float64) / s[None, :]
        assert np.array_equal(oracle.round_e4m3(r.ravel()), r.ravel())
    # coarse, but the image survives: FP8 storage changes colours by a few percent at most
    rays = I.config1_rays()[0].subset(np.arange(0, 16384, 7))
    a = oracle.render(tree, rays)
    b = oracle.render(q, rays)
    assert np.abs(a["rgb"] - b["rgb"]).max() < 0.1
