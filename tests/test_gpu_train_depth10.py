"""The training-step workload at full size: a depth-10 shell VOctree of
7,999,994 leaves (K=16, T=300, HH degree 3) stored in BF16 with an FP32
master, 1,048,576 rays per step drawn from 32 views x 32 time stamps.  One
step = forward, MSE gradient, fused adjoint, Adam on the touched leaves
(Sec. 4.3 "Optimization").

The oracle checks a seeded sample of rays one by one (forward within the BF16
bar, adjoint within relative 1e-4 on the BF16-rounded coefficients), and Adam
on the touched leaves of that sample.  Step times are printed.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2202_06088_gb300 import inputs as I

from helpers import psnr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(cuda_lib):
    from paper_2202_06088_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def c5():
    tree = I.config5_tree()
    rays = I.config5_rays()
    rounded = tree.with_coeffs(oracle.round_bf16(tree.w_sigma), oracle.round_bf16(tree.w_gamma),
                               oracle.round_bf16(tree.w_hh))
    return tree, rays, rounded


def _sample(n, k, seed):
    return np.sort(np.random.default_rng(seed).choice(n, size=k, replace=False))


def test_workload_size(c5):
    tree, rays, _ = c5
    assert tree.depth == 10 and tree.n_leaves == 7_999_994 and rays.n == 1_048_576
    assert tree.K == 16 and tree.T == 300 and tree.hh_degree == 3


def test_training_step_sampled_parity(B, c5):
    tree, rays, rounded = c5
    n = rays.n
    tree_d = B.Tree(tree, "bf16", with_optimizer=True)
    dr = B.DeviceRays.from_host(rays)
    B.neuvv_autotune(tree_d, dr)
    out = B.neuvv_render(tree_d, dr, kernel="packet")
    assert tree_d.status() == 0
    assert (out["alpha"] - (1 - torch.exp(-out["tau"]))).abs().max().item() <= 2e-5
    assert (out["alpha"] > 0).float().mean().item() > 0.02
    # forward: BF16 bar against the unrounded oracle, 1e-4 against the rounded one
    idx = _sample(n, 3000, 11)
    sub = rays.subset(idx)
    got = {k: v[torch.from_numpy(idx).cuda()].cpu().numpy() for k, v in out.items()}
    ref = oracle.render(tree, sub)
    assert np.abs(got["rgb"] - ref["rgb"]).max() <= 4e-3
    assert psnr(got["rgb"], ref["rgb"]) >= 50.0
    ref_q = oracle.render(rounded, sub)
    ok = ref_q["stop_margin"] > 1e-3
    assert np.abs(got["rgb"] - ref_q["rgb"])[ok].max() <= 1e-4
    # adjoint over all rays, dL/dC non-zero on the sample only
    keep = idx[ok]
    rng = np.random.default_rng(12)
    g_sub = rng.standard_normal((keep.size, 3)).astype(np.float32)
    g = torch.zeros(n, 3, device="cuda")
    g[torch.from_numpy(keep).cuda()] = torch.from_numpy(g_sub).cuda()
    grad = tree_d.new_grad()
    touched = tree_d.new_touched()
    B.neuvv_render_backward(tree_d, dr, out, g, None, grad, touched, kernel="packet")
    sub_k = rays.subset(keep)
    want = oracle.render_grad(rounded, sub_k, g_sub)
    info = tree_d.info
    K, Kp, Nh = info.K, info.K_pad, info.N_h
    G = grad.cpu().numpy().astype(np.float64)
    hit = np.nonzero((np.abs(want["w_hh"]).sum((0, 1)) + np.abs(want["w_sigma"]).sum(0)) > 0)[0]
    assert hit.size > 1000
    for got_, ref_ in ((G[hit, 2 * Kp:2 * Kp + 3 * Nh], want["w_hh"][:, :, hit].reshape(3 * Nh, -1).T),
                       (G[hit, :K], want["w_sigma"][:, hit].T), (G[hit, Kp:Kp + K], want["w_gamma"][:, hit].T)):
        assert np.linalg.norm(got_ - ref_) <= 1e-4 * np.linalg.norm(ref_)
        assert np.abs(got_ - ref_).max() <= 1e-4 * np.abs(ref_).max()
    # the touched bitmap holds exactly the leaves the sampled rays composited
    bits = touched.cpu().numpy().view(np.uint32)
    flags = ((bits[:, None] >> np.arange(32, dtype=np.uint32)) & 1).ravel()[:tree.n_leaves].astype(bool)
    assert np.all(flags[hit])
    assert np.abs(G[~flags]).max() == 0.0
    # Adam on the touched leaves, fed the oracle's gradient (one step from the initial master)
    S = info.rec_stride_f32
    gref = np.zeros((hit.size, S), np.float32)
    gref[:, :K] = want["w_sigma"][:, hit].T
    gref[:, Kp:Kp + K] = want["w_gamma"][:, hit].T
    gref[:, 2 * Kp:2 * Kp + 3 * Nh] = want["w_hh"][:, :, hit].reshape(3 * Nh, -1).T
    grad.zero_()
    grad[torch.from_numpy(hit).cuda()] = torch.from_numpy(gref).cuda()
    w0 = np.zeros((hit.size, S), np.float64)
    w0[:, :K] = tree.w_sigma[:, hit].T
    w0[:, Kp:Kp + K] = tree.w_gamma[:, hit].T
    w0[:, 2 * Kp:2 * Kp + 3 * Nh] = tree.w_hh[:, :, hit].reshape(3 * Nh, -1).T
    before = tree_d.master()[torch.from_numpy(hit).cuda()].cpu().numpy()
    assert np.array_equal(before.astype(np.float64), w0)
    B.neuvv_adam_step(tree_d, grad, touched, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, step=1)
    m = np.zeros_like(w0)
    v = np.zeros_like(w0)
    oracle.adam(w0, m, v, gref.astype(np.float64), np.ones(hit.size, np.uint8), 1e-3, 0.9, 0.999, 1e-8, 1)
    after = tree_d.master()[torch.from_numpy(hit).cuda()].cpu().numpy()
    assert np.abs(after - w0).max() <= 1e-6
    # untouched leaves did not move (a sample of them)
    others = np.setdiff1d(_sample(tree.n_leaves, 20000, 13), np.nonzero(flags)[0])
    m_o = tree_d.master()[torch.from_numpy(others).cuda()].cpu().numpy()
    assert np.array_equal(m_o[:, :K], tree.w_sigma[:, others].T)
    assert tree_d.status() == 0


def test_ray_order_on_the_training_batch(B, c5):
    """The batch of rays from 32 views x 32 times in random order, with the
    library's ray order (packets re-formed from the sorted rays): the same
    outputs as rays in the given order, the adjoint replayed through the
    permuted log the same gradient; forward times printed."""
    tree, rays, _ = c5
    n = rays.n
    tree_d = B.Tree(tree, "bf16")
    dr = B.DeviceRays.from_host(rays)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    res = {}
    for order in (B.ORDER_AS_GIVEN, B.ORDER_BY_RAY):
        tree_d.set_packet_order(order)
        out = B.alloc_out(n, dr.o.device, log_bytes_per_ray=64)
        B.neuvv_render(tree_d, dr, kernel="packet", out=out)
        ev[0].record()
        B.neuvv_render(tree_d, dr, kernel="packet", out=out)
        ev[1].record()
        torch.cuda.synchronize()
        res[order] = (out, ev[0].elapsed_time(ev[1]))
    a, b = res[B.ORDER_AS_GIVEN][0], res[B.ORDER_BY_RAY][0]
    for k in ("rgb", "alpha", "depth", "tau", "nseg"):
        assert torch.equal(a[k], b[k]), k
    g = torch.randn(n, 3, device="cuda")
    tree_d.set_packet_order(B.ORDER_AS_GIVEN)
    ga = B.neuvv_render_backward(tree_d, dr, a, g, kernel="packet")
    gb = B.neuvv_render_backward(tree_d, dr, b, g, kernel="packet")
    assert (ga - gb).abs().max().item() <= 1e-5 * ga.abs().max().item()
    print(f"depth-10 batch forward: rays as given {res[0][1]:.3f} ms, ray order {res[2][1]:.3f} ms")
    assert tree_d.status() == 0


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_training_step_time(B, c5, dtype):
    """Forward + MSE + adjoint + Adam over the 1,048,576 rays (times printed)."""
    tree, rays, _ = c5
    n = rays.n
    tree_d = B.Tree(tree, dtype, with_optimizer=True)
    dr = B.DeviceRays.from_host(rays)
    B.neuvv_autotune(tree_d, dr)
    target = torch.full((n, 3), 0.25, device="cuda")
    out = B.alloc_out(n)
    grad_rgb = torch.empty(n, 3, device="cuda")
    grad = tree_d.new_grad()
    touched = tree_d.new_touched()
    loss = torch.zeros(1, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    times = []
    for k in range(1, 7):
        ev[0].record()
        B.neuvv_render(tree_d, dr, kernel="packet", out=out)
        ev[1].record()
        loss.zero_()
        B.neuvv_mse_grad(out["rgb"], target, scale=1.0 / n, grad=grad_rgb, loss=loss)
        ev[2].record()
        B.neuvv_render_backward(tree_d, dr, out, grad_rgb, None, grad, touched, kernel="packet")
        ev[3].record()
        B.neuvv_adam_step(tree_d, grad, touched, lr=1e-3, step=k)
        ev[4].record()
        torch.cuda.synchronize()
        if k > 3:
            times.append([ev[i].elapsed_time(ev[i + 1]) for i in range(4)])
    t = np.mean(times, 0)
    samples = int(out["nseg"].sum().item())
    print(f"depth-10 step {dtype}: fwd {t[0]:.3f} mse {t[1]:.3f} bwd {t[2]:.3f} adam {t[3]:.3f} ms; "
          f"{samples} samples, {samples / (t.sum() / 1e3) / 1e6:.0f} Msamples/s")
    assert np.isfinite(loss.item())
    assert tree_d.status() == 0
