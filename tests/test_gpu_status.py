"""Failure detection on the device, exercised without a fault: the limits of
neuvv_tree_set_limits make the error paths run on ordinary inputs.

- A walk-step cap of 2 ends every ray after two steps: NEUVV_STATUS_SEGMENT_CAP
  is raised, the rays end with at most two segments, the kernels return.
- A poll limit of 0 makes the time slice's wait on its copy give up at once:
  NEUVV_STATUS_TIMEOUT is raised, the blocks wait for their copies to land
  and return, and the next call with the default limit is correct again.
- A segment log replayed against a tree with fewer leaves than the log's
  entries: NEUVV_STATUS_BAD_INDEX, the entries are skipped.
Nothing traps and no wait is unbounded; the context stays usable (each test
ends with a correct call on the same tree)."""
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
def c1():
    return I.config1_tree()


@pytest.mark.parametrize("kernel", ["plain", "packet"])
def test_step_cap_raises_its_flag_and_ends_rays(B, c1, kernel):
    rays, _ = I.config1_rays()
    tree_d = B.Tree(c1, "f32")
    dr = B.DeviceRays.from_host(rays)
    tree_d.set_limits(step_cap=2)
    out = B.neuvv_render(tree_d, dr, kernel=kernel)
    torch.cuda.synchronize()
    flags = tree_d.status()
    assert flags & B.STATUS_SEGMENT_CAP
    assert not flags & B.STATUS_TIMEOUT
    assert (out["nseg"] <= 2).all().item()
    assert torch.isfinite(out["rgb"]).all().item()
    tree_d.set_limits()                       # back to the default: correct again
    out = B.neuvv_render(tree_d, dr, kernel=kernel)
    ref = oracle.render(c1, rays)
    assert np.abs(out["rgb"].cpu().numpy() - ref["rgb"]).max() <= 1e-4
    assert tree_d.status() == 0


def test_slice_wait_limit_raises_timeout_and_returns(B, c1):
    tree_d = B.Tree(c1, "bf16")
    tree_d.set_limits(wait_polls=0)
    sl = torch.full((c1.n_leaves, B.slice_stride(c1.hh_degree)), 7.0, device="cuda")
    B.neuvv_slice(tree_d, 0.37, out=sl)
    torch.cuda.synchronize()                  # every block returned
    flags = tree_d.status()
    assert flags & B.STATUS_TIMEOUT
    assert not flags & B.STATUS_SEGMENT_CAP
    assert (sl == 7.0).all().item()           # no tile was processed
    tree_d.set_limits()
    B.neuvv_slice(tree_d, 0.37, out=sl)
    got = sl.cpu().numpy()
    rounded = c1.with_coeffs(oracle.round_bf16(c1.w_sigma), oracle.round_bf16(c1.w_gamma),
                             oracle.round_bf16(c1.w_hh))
    ref = oracle.slice_at(rounded, 0.37)
    assert np.abs(got[:, 0] - ref["sigma"]).max() <= 1e-5 * max(1.0, np.abs(ref["sigma"]).max())
    assert tree_d.status() == 0


def test_log_of_another_tree_raises_bad_index(B, c1):
    rays, _ = I.config1_rays()
    big = B.Tree(c1, "f32")
    dr = B.DeviceRays.from_host(rays)
    out = B.alloc_out(dr.n, dr.o.device, log_bytes_per_ray=64)
    B.neuvv_render(big, dr, kernel="packet", out=out)
    rng = np.random.default_rng(3)
    small_tree = I.make_coefficients(rng, I.random_mixed_tree(3, 3), K=8, T=30, hh_degree=2)
    small = B.Tree(small_tree, "f32")
    assert small.n_leaves < int(out["nseg"].sum().item())
    g = torch.randn(dr.n, 3, device="cuda")
    grad = B.neuvv_render_backward(small, dr, out, g, kernel="packet")
    torch.cuda.synchronize()
    assert small.status() & B.STATUS_BAD_INDEX
    assert torch.isfinite(grad).all().item()
    # the same call on the tree that wrote the log is clean
    B.neuvv_render_backward(big, dr, out, g, kernel="packet")
    torch.cuda.synchronize()
    assert big.status() == 0


def test_set_limits_rejects_negative_values(B, c1):
    tree_d = B.Tree(c1, "f32")
    with pytest.raises(B.NeuvvError, match="step_cap"):
        tree_d.set_limits(step_cap=-1)
    with pytest.raises(B.NeuvvError, match="wait_polls"):
        tree_d.set_limits(wait_polls=-1)
