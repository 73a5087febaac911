"""neuvv_render_backward_adam: the adjoint and the Adam step of Sec. 4.3
"Optimization" in one call, fused into the per-leaf reduction on the
leaf-major path.  It must leave the tree exactly as neuvv_render_backward
followed by neuvv_adam_step leaves it: the same FP32 master, Adam moments
and storage records (up to FP32 rounding of identical formulas), the
gradient rows zero and the touched bitmap clear.  Checked with the whole
batch in the reservation (every leaf fused), with a partial reservation
(samples beyond it go through the atomic scatter into grad, whose rows the
fused step then reads), without a reservation (the two steps run apart), and
against the oracle's gradient and Adam."""
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


def _case(seed=300, K=8, deg=2, depth=5, n=2048):
    rng = np.random.default_rng(seed)
    tree = I.make_coefficients(rng, I.random_mixed_tree(depth, seed, 0.3, 0.2), K=K, T=6, hh_degree=deg,
                               mean_sigma=10.0)
    cams = I.sphere_cameras(seed, 4, 2.5, 32, 16)
    parts = [I.camera_rays(c, float(t))[0] for c, t in zip(cams, (0.1, 0.4, 0.4, 0.9))]
    rays = I.Rays.concat(parts)
    g = rng.standard_normal((rays.n, 3)).astype(np.float32)
    return tree, rays, g


def _state(tree_d):
    m, v = tree_d.adam_state()
    st = tree_d.storage()
    st = st.view(torch.int16) if st.dtype == torch.bfloat16 else st
    return {"master": tree_d.master().clone(), "m": m.clone(), "v": v.clone(), "storage": st.clone()}


def _prepare(B, tree, dtype, rays, reserve):
    tree_d = B.Tree(tree, dtype, with_optimizer=True)
    dr = B.DeviceRays.from_host(rays)
    out = B.alloc_out(rays.n, dr.o.device, log_bytes_per_ray=4096)
    B.neuvv_render(tree_d, dr, kernel="packet", out=out)
    torch.cuda.synchronize()
    used = int(out["log"][0].item())
    if reserve == "all":
        tree_d.reserve_adjoint((used + 1) * 256)
    elif reserve == "part":
        tree_d.reserve_adjoint(max(1, used // 3) * 256)
    return tree_d, dr, out, used


@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
@pytest.mark.parametrize("reserve", ["all", "part", "none"])
def test_fused_step_equals_backward_then_adam(B, dtype, reserve):
    tree, rays, g = _case()
    gt = torch.from_numpy(g).cuda()
    a, dr, out_a, used = _prepare(B, tree, dtype, rays, reserve)
    b, _, out_b, _ = _prepare(B, tree, dtype, rays, reserve)
    assert used > 3
    for step in (1, 2):
        grad_a, touched_a = a.new_grad(), a.new_touched()
        B.neuvv_render_backward(a, dr, out_a, gt, None, grad_a, touched_a, kernel="packet")
        B.neuvv_adam_step(a, grad_a, touched_a, lr=0.01, step=step)
        grad_b, touched_b = b.new_grad(), b.new_touched()
        B.neuvv_render_backward_adam(b, dr, out_b, gt, None, grad_b, touched_b, lr=0.01, step=step)
        torch.cuda.synchronize()
        sa, sb = _state(a), _state(b)
        for k in ("master", "m", "v"):
            d = (sa[k] - sb[k]).abs().max().item()
            assert d <= 1e-6 * max(1.0, sa[k].abs().max().item()), (k, d)
        assert torch.count_nonzero(sa["m"]).item() > 0
        if dtype == "fp8":
            # codes may differ only where the masters differ in the last bit
            assert (sa["storage"] != sb["storage"]).float().mean().item() < 1e-3
        else:
            assert (sa["storage"].int() - sb["storage"].int()).abs().max().item() <= 1
        assert torch.count_nonzero(grad_b).item() == 0 and torch.count_nonzero(touched_b).item() == 0
        assert torch.count_nonzero(grad_a).item() == 0
        # the next step renders the updated storage
        B.neuvv_render(a, dr, kernel="packet", out=out_a)
        B.neuvv_render(b, dr, kernel="packet", out=out_b)
    assert a.status() == 0 and b.status() == 0


def test_fused_step_matches_the_oracle(B):
    """One fused step from the initial state against the oracle's analytic
    gradient of the same batch followed by its Adam (pinned to
    torch.optim.Adam): the master within the Adam test's tolerance."""
    tree, rays, g = _case(seed=301)
    tree_d, dr, out, _ = _prepare(B, tree, "f32", rays, "all")
    info = tree_d.info
    K, Kp, Nh, S = info.K, info.K_pad, info.N_h, info.rec_stride_f32
    ref_out = oracle.render(tree, rays)
    keep = ref_out["stop_margin"] > 1e-3
    g = np.where(keep[:, None], g, 0.0).astype(np.float32)
    w0 = tree_d.master().cpu().numpy().astype(np.float64)
    grad, touched = tree_d.new_grad(), tree_d.new_touched()
    B.neuvv_render_backward_adam(tree_d, dr, out, torch.from_numpy(g).cuda(), None, grad, touched, lr=0.01,
                                 beta1=0.9, beta2=0.99, eps=1e-8, step=1)
    got = tree_d.master().cpu().numpy().astype(np.float64)
    rg = oracle.render_grad(tree, rays, g)
    G = np.zeros_like(w0)
    G[:, :K] = rg["w_sigma"].T
    G[:, Kp:Kp + K] = rg["w_gamma"].T
    G[:, 2 * Kp:2 * Kp + 3 * Nh] = rg["w_hh"].reshape(3 * Nh, -1).T
    hit = np.abs(G).sum(1) > 0
    w, m, v = w0.copy(), np.zeros_like(w0), np.zeros_like(w0)
    oracle.adam(w, m, v, G, hit, 0.01, 0.9, 0.99, 1e-8, 1)
    # Adam's first step moves every touched entry by about lr sign(g): compare
    # the steps where the gradient is not at FP32 noise level
    big = np.abs(G) > 1e-4 * np.abs(G).max()
    assert big.sum() > 100
    assert np.abs((got - w0)[big] - (w - w0)[big]).max() <= 1e-4
    assert np.array_equal(got[~hit], w0[~hit])
    assert S == w0.shape[1]
