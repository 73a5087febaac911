"""GPU parity of the image-gradient regulariser L_grad (Sec. 4.3
"Optimization") through the C ABI against the FP64 oracle: the loss within
relative 1e-5 (FP32 sums over all pixel pairs), the gradient within 1e-6 of
its scale (plus the rounding of the FP32 gradient it is added to), on images with missing pixels, in tile ray order (the bench's
camera rays) and in a random ray order; at the bench size on the 8 views of
the depth-9 workload."""
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


def _check(B, rgb, tgt, m, lam, W, H):
    ref = oracle.grad_loss(rgb, tgt, m, W, H, lam)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    base = np.random.default_rng(1).standard_normal(rgb.shape).astype(np.float32)
    grad = dev(base)                                   # accumulates into an existing gradient
    loss = torch.zeros(1, device="cuda")
    B.neuvv_grad_loss(dev(rgb), dev(tgt), torch.from_numpy(m.astype(np.int32)).cuda(), lam, grad, loss)
    got = grad.cpu().numpy().astype(np.float64) - base
    assert abs(loss.item() - ref["loss"]) <= 1e-5 * abs(ref["loss"]) + 1e-9
    scale = np.abs(ref["grad"]).max()
    # the sum into an FP32 gradient of magnitude |base| rounds to half an ulp of it
    tol = 1e-6 * max(scale, 1e-3) + 2.0 ** -24 * (np.abs(base).max() + scale)
    assert np.abs(got - ref["grad"]).max() <= tol


@pytest.mark.parametrize("order", ["tiles", "random"])
def test_grad_loss_matches_oracle(B, order):
    rng = np.random.default_rng(8)
    V, H, W = 3, 37, 53                                # ragged against the 8x4 tiles
    per = H * W
    if order == "tiles":
        pix = I.tile_order(W, H)
    else:
        pix = rng.permutation(per)
    m = np.full((V, H, W), -1, np.int64)
    for v in range(V):
        m.reshape(V, -1)[v, pix] = v * per + np.arange(per)
    m[rng.uniform(size=m.shape) < 0.05] = -1           # pixels without a ray
    n = V * per
    rgb = rng.uniform(0, 1, (n, 3)).astype(np.float32).astype(np.float64)
    tgt = rng.uniform(0, 1, (n, 3)).astype(np.float32).astype(np.float64)
    tgt[::17] = rgb[::17]                              # exact ties: zero subgradient
    _check(B, rgb, tgt, m, 0.1, W, H)


def test_grad_loss_at_bench_size(B):
    rays, pix, cams, _ = I.config2_rays(n_views=8)
    V, H, W = 8, 1080, 1920
    m = np.empty((V, H * W), np.int64)
    for v in range(V):
        m[v, pix[v]] = v * H * W + np.arange(H * W)
    rng = np.random.default_rng(9)
    n = rays.n
    rgb = rng.uniform(0, 1, (n, 3)).astype(np.float32).astype(np.float64)
    tgt = np.clip(rgb + rng.normal(0, 0.05, (n, 3)), 0, 1).astype(np.float32).astype(np.float64)
    _check(B, rgb, tgt, m.reshape(V, H, W), 0.1, W, H)


@pytest.mark.parametrize("H,W", [(1, 1), (1, 40), (40, 1), (9, 33), (8, 32)])
def test_grad_loss_degenerate_shapes(B, H, W):
    # single pixels, single rows and columns (no vertical or horizontal
    # pairs), one pixel past a 32x8 tile, and exactly one tile
    rng = np.random.default_rng(H * 1000 + W)
    V = 2
    n = V * H * W
    m = rng.permutation(n).reshape(V, H, W)
    rgb = rng.uniform(0, 1, (n, 3)).astype(np.float32).astype(np.float64)
    tgt = rng.uniform(0, 1, (n, 3)).astype(np.float32).astype(np.float64)
    _check(B, rgb, tgt, m, 0.1, W, H)
