"""Pins of the oracle's image-gradient regulariser L_grad (Sec. 4.3
"Optimization": lambda * sum ||grad |I - I_hat|||^2 over the training views).

* Its gradient matches FP64 central differences of its loss (random images
  away from the |.| kink).
* A constant error image has no gradient: loss and gradient are zero.
* A horizontal ramp |I - I_hat| = a x has (width-1) height unit steps of
  size a per channel: loss = lam 3 a^2 (width-1) height.
* Pixels without a ray (-1) take part in no difference.
* The ray order does not matter: permuting the rays (and the map with them)
  permutes the gradient.
"""
import numpy as np

import oracle


def _setup(rng, V, H, W, holes=0.0):
    n = V * H * W
    perm = rng.permutation(n)
    m = perm.reshape(V, H, W).copy()
    if holes:
        m[rng.uniform(size=m.shape) < holes] = -1
    return n, m


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    n, m = _setup(rng, 2, 5, 7, holes=0.1)
    rgb = rng.uniform(0, 1, (n, 3))
    tgt = rng.uniform(0, 1, (n, 3))
    out = oracle.grad_loss(rgb, tgt, m, 7, 5, 0.1)
    for k in rng.choice(n * 3, 40, replace=False):
        i, c = divmod(int(k), 3)
        h = 1e-6
        rp = rgb.copy(); rp[i, c] += h
        rm = rgb.copy(); rm[i, c] -= h
        fd = (oracle.grad_loss(rp, tgt, m, 7, 5, 0.1)["loss"] - oracle.grad_loss(rm, tgt, m, 7, 5, 0.1)["loss"]) / (2 * h)
        assert abs(fd - out["grad"][i, c]) <= 1e-7 * max(1.0, abs(fd)), (i, c, fd, out["grad"][i, c])


def test_constant_error_has_no_gradient():
    rng = np.random.default_rng(4)
    n, m = _setup(rng, 3, 4, 6)
    tgt = rng.integers(0, 64, (n, 3)) / 64.0        # exact binary fractions: the error is exactly 0.25
    rgb = tgt + 0.25
    out = oracle.grad_loss(rgb, tgt, m, 6, 4, 0.1)
    assert out["loss"] == 0.0
    assert np.all(out["grad"] == 0.0)


def test_horizontal_ramp_closed_form():
    V, H, W, a, lam = 2, 3, 5, 0.03, 0.1
    m = np.arange(V * H * W).reshape(V, H, W)
    x = np.tile(np.arange(W), V * H).astype(np.float64)
    tgt = np.zeros((V * H * W, 3))
    rgb = (a * x)[:, None] * np.ones((1, 3))
    out = oracle.grad_loss(rgb, tgt, m, W, H, lam)
    assert abs(out["loss"] - lam * 3 * a * a * (W - 1) * H * V) <= 1e-15
    # interior pixels: a step in from the left and a step out to the right cancel
    g = out["grad"].reshape(V, H, W, 3)
    assert np.all(g[:, :, 1:-1] == 0.0)
    np.testing.assert_allclose(g[:, :, -1], lam * 2 * a, rtol=1e-12)


def test_pixels_without_rays_take_no_part():
    rng = np.random.default_rng(5)
    n, m = _setup(rng, 1, 4, 4)
    rgb = rng.uniform(0, 1, (n, 3))
    tgt = rng.uniform(0, 1, (n, 3))
    full = oracle.grad_loss(rgb, tgt, m, 4, 4, 1.0)
    m2 = m.copy()
    gone = m2[0, 1, 2]
    m2[0, 1, 2] = -1
    part = oracle.grad_loss(rgb, tgt, m2, 4, 4, 1.0)
    assert np.all(part["grad"][gone] == 0.0)
    E = np.abs(tgt - rgb)
    lost = sum(float(((E[gone] - E[m[0, y, x]]) ** 2).sum()) for y, x in ((1, 1), (1, 3), (0, 2), (2, 2)))
    assert abs(full["loss"] - part["loss"] - lost) <= 1e-12


def test_ray_order_does_not_matter():
    rng = np.random.default_rng(6)
    n, m = _setup(rng, 2, 3, 4)
    rgb = rng.uniform(0, 1, (n, 3))
    tgt = rng.uniform(0, 1, (n, 3))
    ref = oracle.grad_loss(rgb, tgt, m, 4, 3, 0.1)
    p = rng.permutation(n)                      # new ray i is old ray p[i]
    inv = np.argsort(p)
    got = oracle.grad_loss(rgb[p], tgt[p], inv[m], 4, 3, 0.1)
    assert abs(got["loss"] - ref["loss"]) <= 1e-15
    np.testing.assert_array_equal(got["grad"], ref["grad"][p])
