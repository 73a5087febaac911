"""GPU parity of the fused adjoint, the loss and the sparse Adam step through
the C ABI, against the FP64 oracle's analytic gradient (itself pinned to
finite differences) and against FP64 central differences directly.

Gradient tolerance: relative 1e-4 of the oracle's analytic gradient, measured
per leaf record as ||g_gpu - g_ref|| <= 1e-4 ||g_ref|| + 1e-6 max||g_ref||
(FP32 atomics sum in any order); relative 1e-3 against finite differences.
"""
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


def _record_planes(tree_d, g):
    """Splits a [n_leaves, rec_stride_f32] gradient into the oracle's planes."""
    info = tree_d.info
    K, Kp, Nh = info.K, info.K_pad, info.N_h
    g = g.cpu().numpy().astype(np.float64)
    return {"w_sigma": g[:, :K].T, "w_gamma": g[:, Kp:Kp + K].T,
            "w_hh": g[:, 2 * Kp:2 * Kp + 3 * Nh].T.reshape(3, Nh, -1)}


def _rel_err(got, ref):
    num = sum(((got[k] - ref[k]) ** 2).sum(0) for k in ref if k != "w_hh") + ((got["w_hh"] - ref["w_hh"]) ** 2).sum((0, 1))
    den = sum((ref[k] ** 2).sum(0) for k in ref if k != "w_hh") + (ref["w_hh"] ** 2).sum((0, 1))
    num, den = np.sqrt(num), np.sqrt(den)
    return num, den


def _setup(seed, K, deg, depth, n_rays, dtype="f32", signed=False):
    rng = np.random.default_rng(seed)
    st = I.random_mixed_tree(depth, seed, p_leaf=0.25, p_empty=0.2)
    tree = I.make_coefficients(rng, st, K=K, T=6, hh_degree=deg, mean_sigma=10.0, signed_density=signed)
    from test_oracle_render import _random_rays
    rays = _random_rays(rng, n_rays)
    rays.times[:] = rng.uniform(0, 1, rays.n).astype(np.float32)
    g = rng.standard_normal((rays.n, 3)).astype(np.float32)
    ga = rng.standard_normal(rays.n).astype(np.float32)
    return tree, rays, g, ga


@pytest.mark.parametrize("K,deg,depth,act,signed,kernel", [
    (8, 2, 4, "sigmoid", False, "plain"),
    (8, 2, 5, "sigmoid", True, "packet"),
    (16, 3, 5, "identity", False, "packet"),
    (4, 1, 4, "sigmoid", True, "plain"),
])
def test_adjoint_matches_oracle_gradient(B, K, deg, depth, act, signed, kernel):
    tree, rays, g, ga = _setup(50 + K + depth, K, deg, depth, 4096 + 3, signed=signed)
    ref_out = oracle.render(tree, rays, act=act)
    keep = ref_out["stop_margin"] > 1e-3       # stop decision far from the threshold
    rays = rays.subset(np.nonzero(keep)[0])
    g, ga = g[keep], ga[keep]
    ref = oracle.render_grad(tree, rays, g, ga, act=act)
    tree_d = B.Tree(tree, "f32")
    dr = B.DeviceRays.from_host(rays)
    out = B.neuvv_render(tree_d, dr, act=act, kernel=kernel)
    touched = tree_d.new_touched()
    grad = B.neuvv_render_backward(tree_d, dr, out, torch.from_numpy(g).cuda(), torch.from_numpy(ga).cuda(),
                                   touched=touched, act=act, kernel=kernel)
    got = _record_planes(tree_d, grad)
    num, den = _rel_err(got, ref)
    scale = den.max()
    assert np.all(num <= 1e-4 * den + 1e-6 * scale), (num / np.maximum(den, 1e-30)).max()
    # touched bitmap = leaves with a non-zero reference gradient (plus any with exact zeros)
    bits = touched.cpu().numpy().view(np.uint32)
    tb = ((bits[np.arange(tree.n_leaves) >> 5] >> (np.arange(tree.n_leaves) & 31)) & 1).astype(bool)
    assert np.all(tb[den > 0])
    assert tree_d.status() == 0


def test_adjoint_bf16_storage_matches_oracle_on_rounded_coefficients(B):
    tree, rays, g, ga = _setup(61, 16, 3, 5, 2048)
    tree_d = B.Tree(tree, "bf16")
    rounded = tree.with_coeffs(oracle.round_bf16(tree.w_sigma), oracle.round_bf16(tree.w_gamma),
                               oracle.round_bf16(tree.w_hh))
    ref_out = oracle.render(rounded, rays)
    keep = ref_out["stop_margin"] > 1e-3
    rays = rays.subset(np.nonzero(keep)[0])
    g, ga = g[keep], ga[keep]
    ref = oracle.render_grad(rounded, rays, g, ga)
    dr = B.DeviceRays.from_host(rays)
    out = B.neuvv_render(tree_d, dr)
    grad = B.neuvv_render_backward(tree_d, dr, out, torch.from_numpy(g).cuda(), torch.from_numpy(ga).cuda())
    num, den = _rel_err(_record_planes(tree_d, grad), ref)
    assert np.all(num <= 1e-4 * den + 1e-6 * den.max())


def test_adjoint_matches_fp64_finite_differences(B):
    """GPU gradient of L = sum g.C + ga.alpha against central differences of the
    FP64 oracle forward (h = 1e-6 on float64 coefficients)."""
    tree, rays, g, ga = _setup(70, 8, 2, 4, 64)
    ref_out = oracle.render(tree, rays, t_stop=0.0)
    tree_d = B.Tree(tree, "f32")
    dr = B.DeviceRays.from_host(rays)
    out = B.neuvv_render(tree_d, dr, t_stop=0.0)
    grad = B.neuvv_render_backward(tree_d, dr, out, torch.from_numpy(g).cuda(), torch.from_numpy(ga).cuda(),
                                   t_stop=0.0)
    got = _record_planes(tree_d, grad)
    ws, wg, wh = (tree.w_sigma.astype(np.float64), tree.w_gamma.astype(np.float64), tree.w_hh.astype(np.float64))
    arrs = {"w_sigma": ws, "w_gamma": wg, "w_hh": wh}

    def L():
        o = oracle.render(tree, rays, t_stop=0.0, otree=oracle.OracleTree(tree, ws, wg, wh))
        return float((o["rgb"] * g).sum() + (o["alpha"] * ga).sum())

    rng = np.random.default_rng(71)
    hit = np.nonzero(np.abs(got["w_hh"]).sum((0, 1)) > 0)[0]
    h = 1e-6
    worst = 0.0
    for leaf in rng.choice(hit, size=min(6, hit.size), replace=False):
        for name, idx in [("w_sigma", (0, leaf)), ("w_gamma", (1, leaf)), ("w_hh", (0, 0, leaf)),
                          ("w_hh", (2, 5, leaf)), ("w_hh", (1, 9, leaf))]:
            base = arrs[name][idx]
            arrs[name][idx] = base + h
            lp = L()
            arrs[name][idx] = base - h
            lm = L()
            arrs[name][idx] = base
            fd = (lp - lm) / (2 * h)
            err = abs(got[name][idx] - fd) / max(abs(fd), 1e-3)
            worst = max(worst, err)
    assert worst <= 1e-3, worst


def test_autograd_function_matches_direct_calls(B):
    tree, rays, g, ga = _setup(80, 8, 2, 4, 1024)
    tree_d = B.Tree(tree, "f32", with_optimizer=True)
    dr = B.DeviceRays.from_host(rays)
    coeffs = tree_d.master().clone().requires_grad_(True)
    rgb, alpha, depth = B.render_differentiable(coeffs, tree_d, dr)
    loss = (rgb * torch.from_numpy(g).cuda()).sum() + (alpha * torch.from_numpy(ga).cuda()).sum()
    loss.backward()
    out = B.neuvv_render(tree_d, dr)
    direct = B.neuvv_render_backward(tree_d, dr, out, torch.from_numpy(g).cuda(), torch.from_numpy(ga).cuda())
    # the same adjoint; FP32 atomic sums in another order: within 1e-5 of the largest entry
    assert (coeffs.grad - direct).abs().max().item() <= 1e-5 * direct.abs().max().item()


@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
def test_autograd_function_renders_from_its_input(B, dtype):
    """VOctreeRender renders the coefficients it is given: perturbed records
    passed as ``coeffs`` give the image of a tree built from those
    coefficients (bit for bit: the same storage rounding), and a torch
    optimiser step on ``coeffs`` changes the next render accordingly."""
    tree, rays, g, ga = _setup(81, 8, 2, 4, 1024)
    tree_d = B.Tree(tree, dtype, with_optimizer=True)
    dr = B.DeviceRays.from_host(rays)
    info = tree_d.info
    K, Kp, Nh = info.K, info.K_pad, info.N_h
    pert = I.perturbed(tree, seed=5, std=0.2)
    rec = np.zeros((tree.n_leaves, info.rec_stride_f32), np.float32)
    rec[:, :K] = pert.w_sigma.T
    rec[:, Kp:Kp + K] = pert.w_gamma.T
    rec[:, 2 * Kp:2 * Kp + 3 * Nh] = pert.w_hh.reshape(3 * Nh, -1).T
    coeffs = torch.from_numpy(rec).cuda().requires_grad_(True)
    rgb, alpha, _ = B.render_differentiable(coeffs, tree_d, dr)
    fresh = B.neuvv_render(B.Tree(pert, dtype), dr)
    assert torch.equal(rgb, fresh["rgb"]) and torch.equal(alpha, fresh["alpha"])
    # one SGD step on coeffs, then the next render is that of the stepped records
    loss = (rgb * torch.from_numpy(g).cuda()).sum()
    loss.backward()
    opt = torch.optim.SGD([coeffs], lr=0.05)
    opt.step()
    rgb2, _, _ = B.render_differentiable(coeffs, tree_d, dr)
    stepped = coeffs.detach().cpu().numpy()
    again = pert.with_coeffs(np.ascontiguousarray(stepped[:, :K].T), np.ascontiguousarray(stepped[:, Kp:Kp + K].T),
                             np.ascontiguousarray(stepped[:, 2 * Kp:2 * Kp + 3 * Nh].T.reshape(3, Nh, -1)))
    assert torch.equal(rgb2, B.neuvv_render(B.Tree(again, dtype), dr)["rgb"])
    assert not torch.equal(rgb2, rgb)
    # the tree's own master copy as coeffs: nothing is written, the storage renders
    own = tree_d.master()
    r3, _, _ = B.render_differentiable(own, tree_d, dr)
    assert torch.equal(r3, rgb2)


def test_mse_grad_matches_numpy(B):
    rng = np.random.default_rng(90)
    n = 10007
    a = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    b = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    loss = torch.zeros(1, device="cuda")
    grad = B.neuvv_mse_grad(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), scale=1.0 / n, loss=loss)
    assert np.allclose(grad.cpu().numpy(), 2.0 / n * (a - b), rtol=1e-6, atol=1e-9)
    ref = ((a.astype(np.float64) - b) ** 2).sum() / n
    assert abs(loss.item() - ref) <= 1e-5 * ref


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_sparse_adam_matches_oracle(B, dtype):
    rng = np.random.default_rng(91)
    st = I.random_mixed_tree(4, 91)
    tree = I.make_coefficients(rng, st, K=8, T=4, hh_degree=2)
    tree_d = B.Tree(tree, dtype, with_optimizer=True)
    info = tree_d.info
    L, S = tree.n_leaves, info.rec_stride_f32
    w = tree_d.master().cpu().numpy().astype(np.float64)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    for step in range(1, 4):
        gnp = np.zeros((L, S), np.float32)
        touched = rng.random(L) < 0.6
        gnp[touched, :info.rec_len] = rng.standard_normal((touched.sum(), info.rec_len)).astype(np.float32)
        bits = np.zeros((L + 31) // 32, np.uint32)
        for l in np.nonzero(touched)[0]:
            bits[l >> 5] |= np.uint32(1 << (l & 31))
        grad = torch.from_numpy(gnp).cuda()
        tb = torch.from_numpy(bits.view(np.int32)).cuda()
        B.neuvv_adam_step(tree_d, grad, tb, lr=0.01, beta1=0.9, beta2=0.99, eps=1e-8, step=step)
        oracle.adam(w, m, v, gnp.astype(np.float64), touched.astype(np.uint8), 0.01, 0.9, 0.99, 1e-8, step)
        assert torch.count_nonzero(grad).item() == 0
        assert torch.count_nonzero(tb).item() == 0
    got = tree_d.master().cpu().numpy()
    assert np.abs(got - w).max() <= 1e-5
    ma, va = tree_d.adam_state()
    assert np.abs(ma.cpu().numpy() - m).max() <= 1e-6
    if dtype == "bf16":
        st_ = tree_d.storage().float().cpu().numpy()[:, :info.rec_len]
        # the storage is its own master rounded to nearest even (torch's cast) ...
        own = torch.from_numpy(got[:, :info.rec_len]).to(torch.bfloat16).float().numpy()
        assert np.array_equal(st_, own)
        # ... and within half a BF16 spacing (plus the master's error) of the oracle's weights
        wo = w[:, :info.rec_len]
        assert np.all(np.abs(st_ - wo) <= 2.0 ** -8 * np.abs(wo) + 2e-5)


def test_adjoint_from_the_segment_log_matches_the_walk(B):
    """The packet forward's segment log lets the adjoint replay each packet's
    shading rounds without walking; any log size, including one too small for
    most packets (those are walked), and a log written for other rays (ignored)
    give the same gradient."""
    rng = np.random.default_rng(95)
    st = I.random_mixed_tree(6, 95, p_leaf=0.3, p_empty=0.2)
    tree = I.make_coefficients(rng, st, K=16, T=9, hh_degree=3, mean_sigma=8.0)
    from test_oracle_render import _random_rays
    rays = _random_rays(rng, 4096 + 7)
    rays.times[:] = rng.uniform(0, 1, rays.n).astype(np.float32)
    g = torch.from_numpy(rng.standard_normal((rays.n, 3)).astype(np.float32)).cuda()
    tree_d = B.Tree(tree, "bf16")
    dr = B.DeviceRays.from_host(rays)
    walk = B.neuvv_render_backward(tree_d, dr, B.neuvv_render(tree_d, dr, kernel="packet"), g, kernel="packet")
    ref = walk.cpu().numpy().astype(np.float64)
    scale = np.abs(ref).max()
    for per_ray in (64, 24, 2):      # ample, room for a few packets only (the others are walked), none
        out = B.neuvv_render(tree_d, dr, kernel="packet", out=B.alloc_out(rays.n, log_bytes_per_ray=per_ray))
        if per_ray == 24:
            held = B.neuvv_log_read(out, rays.n, 8)["count"] >= 0
            assert held.any().item() and (~held & (out["nseg"] > 0)).any().item()
        got = B.neuvv_render_backward(tree_d, dr, out, g, kernel="packet").cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-5 * scale, per_ray
        assert np.linalg.norm(got - ref) <= 1e-6 * np.linalg.norm(ref)
    # a log filled for a different batch is not used
    other = rays.subset(np.arange(rays.n - 40))
    out_o = B.neuvv_render(tree_d, B.DeviceRays.from_host(other), kernel="packet",
                           out=B.alloc_out(rays.n, log_bytes_per_ray=64))
    out = B.neuvv_render(tree_d, dr, kernel="packet")
    out["log"] = out_o["log"]
    got = B.neuvv_render_backward(tree_d, dr, out, g, kernel="packet").cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-5 * scale
    # the plain forward marks a log empty
    out_p = B.alloc_out(rays.n, log_bytes_per_ray=64)
    B.neuvv_render(tree_d, dr, kernel="packet", out=out_p)
    B.neuvv_render(tree_d, dr, kernel="plain", out=out_p)
    got = B.neuvv_render_backward(tree_d, dr, out_p, g, kernel="packet").cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-5 * scale
    assert tree_d.status() == 0
