"""FP8 E4M3 coefficient storage with per-leaf power-of-two scales (the storage
ablation) through the C ABI.

* The records tree_create writes hold exactly the oracle's quantisation of
  the seeded coefficients: the same scales, the same codes.
* Render, adjoint and composition on FP8 storage match the oracle on the
  dequantised coefficients within the FP32 tolerances (1e-4 colour, relative
  1e-4 gradient).  The error against the unquantised oracle is the price of the
  format; it is reported and only bounded loosely.
* Adam on an FP8 tree updates the FP32 master like the oracle's Adam, and
  re-encodes each touched record from its own master under the same rule.
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
def c1():
    return I.config1_tree()


def _decode(tree_d):
    """Entries and scales of FP8 records, read back as raw bytes; codes decoded
    by torch's float8_e4m3fn view."""
    info = tree_d.info
    raw = tree_d.storage().cpu().numpy()
    assert raw.dtype == np.uint8 and raw.shape[1] == info.rec_stride
    scales = raw[:, :12].copy().view(np.float32).astype(np.float64)
    codes = torch.from_numpy(raw[:, 16:16 + info.rec_len].copy()).view(torch.float8_e4m3fn)
    vals = codes.to(torch.float64).numpy()
    j = np.arange(info.rec_len)
    grp = np.where(j < info.K_pad, 0, np.where(j < 2 * info.K_pad, 1, 2))
    return vals * scales[:, grp], scales, raw


def _planes(tree, rec, K_pad):
    """Record entries [L, rec_len] -> (w_sigma [K, L], w_gamma [K, L], w_hh [3, N_h, L])."""
    K = tree.K
    return rec[:, :K].T, rec[:, K_pad:K_pad + K].T, rec[:, 2 * K_pad:].T.reshape(tree.w_hh.shape)


@pytest.mark.parametrize("which", ["c1", "shell16"])
def test_records_hold_the_oracle_quantisation(B, c1, which):
    if which == "c1":
        tree = c1
    else:  # the K=16, degree-3 record shape of the large workloads, small tree
        rng = np.random.default_rng(17)
        tree = I.make_coefficients(rng, I.random_mixed_tree(5, 17, p_leaf=0.3, p_empty=0.2), K=16, T=9,
                                   hh_degree=3)
    tree_d = B.Tree(tree, "fp8")
    vals, scales, raw = _decode(tree_d)
    q, s_ref = oracle.quantize_fp8_tree(tree)
    assert np.array_equal(scales, s_ref)
    ws, wg, wh = _planes(tree, vals, tree_d.info.K_pad)
    assert np.array_equal(ws, q.w_sigma.astype(np.float64))
    assert np.array_equal(wg, q.w_gamma.astype(np.float64))
    assert np.array_equal(wh, q.w_hh.astype(np.float64))
    # K_pad entries past K, the header's fourth word and the tail padding are zero
    K, Kp = tree.K, tree_d.info.K_pad
    assert np.all(vals[:, K:Kp] == 0) and np.all(vals[:, Kp + K:2 * Kp] == 0)
    assert np.all(raw[:, 12:16] == 0) and np.all(raw[:, 16 + tree_d.info.rec_len:] == 0)


def test_render_on_fp8_storage(B, c1):
    rays = I.config1_rays()[0]
    tree_d = B.Tree(c1, "fp8")
    dr = B.DeviceRays.from_host(rays)
    q, _ = oracle.quantize_fp8_tree(c1)
    ref_q = oracle.render(q, rays)
    ok = ref_q["stop_margin"] > 1e-3
    assert ok.mean() > 0.99
    for kernel in ("plain", "packet"):
        got = {k: v.cpu().numpy() for k, v in B.neuvv_render(tree_d, dr, kernel=kernel).items()}
        assert np.abs(got["rgb"][ok] - ref_q["rgb"][ok]).max() <= 1e-4
        assert np.abs(got["alpha"][ok] - ref_q["alpha"][ok]).max() <= 1e-4
    assert tree_d.status() == 0
    # the ablation's cost against the unquantised coefficients (reported; loose floor)
    ref = oracle.render(c1, rays)
    err = np.abs(got["rgb"] - ref["rgb"]).max()
    p = psnr(got["rgb"], ref["rgb"])
    print(f"FP8 storage vs unquantised oracle: max abs {err:.3e}, PSNR {p:.1f} dB")
    assert p >= 30.0


def test_adjoint_on_fp8_storage(B, c1):
    rng = np.random.default_rng(23)
    rays = I.config1_rays()[0].subset(np.arange(0, 16384, 3))
    tree_d = B.Tree(c1, "fp8")
    dr = B.DeviceRays.from_host(rays)
    out = B.neuvv_render(tree_d, dr, kernel="packet")
    g = rng.standard_normal((rays.n, 3))
    q, _ = oracle.quantize_fp8_tree(c1)
    ref_out = oracle.render(q, rays)
    keep = ref_out["stop_margin"] > 1e-3
    g[~keep] = 0.0
    grad = B.neuvv_render_backward(tree_d, dr, out, torch.from_numpy(g.astype(np.float32)).cuda(), kernel="packet")
    ref = oracle.render_grad(q, rays, g)
    G = grad.cpu().numpy().astype(np.float64)
    info = tree_d.info
    K, Kp, Nh = info.K, info.K_pad, info.N_h
    got_s, ref_s = G[:, :K].T, ref["w_sigma"]
    got_g, ref_g = G[:, Kp:Kp + K].T, ref["w_gamma"]
    got_h, ref_h = G[:, 2 * Kp:2 * Kp + 3 * Nh].T.reshape(ref["w_hh"].shape), ref["w_hh"]
    for got_, ref_ in ((got_s, ref_s), (got_g, ref_g), (got_h, ref_h)):
        assert np.linalg.norm(got_ - ref_) <= 1e-4 * np.linalg.norm(ref_)
        assert np.abs(got_ - ref_).max() <= 1e-4 * np.abs(ref_).max()


def test_adam_reencodes_fp8_records(B):
    rng = np.random.default_rng(93)
    tree = I.make_coefficients(rng, I.random_mixed_tree(4, 93), K=8, T=4, hh_degree=2)
    tree_d = B.Tree(tree, "fp8", with_optimizer=True)
    info = tree_d.info
    L, S = tree.n_leaves, info.rec_stride_f32
    w = tree_d.master().cpu().numpy().astype(np.float64)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    ever = np.zeros(L, bool)
    before = tree_d.storage().cpu().numpy().copy()
    for step in range(1, 4):
        gnp = np.zeros((L, S), np.float32)
        touched = rng.random(L) < 0.6
        ever |= touched
        gnp[touched, :info.rec_len] = rng.standard_normal((touched.sum(), info.rec_len)).astype(np.float32)
        bits = np.zeros((L + 31) // 32, np.uint32)
        for l in np.nonzero(touched)[0]:
            bits[l >> 5] |= np.uint32(1 << (l & 31))
        grad = torch.from_numpy(gnp).cuda()
        tb = torch.from_numpy(bits.view(np.int32)).cuda()
        B.neuvv_adam_step(tree_d, grad, tb, lr=0.01, beta1=0.9, beta2=0.99, eps=1e-8, step=step)
        oracle.adam(w, m, v, gnp.astype(np.float64), touched.astype(np.uint8), 0.01, 0.9, 0.99, 1e-8, step)
        assert torch.count_nonzero(grad).item() == 0
    got = tree_d.master().cpu().numpy()
    assert np.abs(got - w).max() <= 1e-5
    vals, scales, raw = _decode(tree_d)
    # untouched leaves keep their records byte for byte
    assert np.array_equal(raw[~ever], before[~ever])
    # touched records: each group's scale is the smallest power of two that
    # fits its master, and the codes are the nearest E4M3 values (torch's cast)
    j = np.arange(info.rec_len)
    grp = np.where(j < info.K_pad, 0, np.where(j < 2 * info.K_pad, 1, 2))
    gm = got[:, :info.rec_len].astype(np.float64)
    for g in range(3):
        mx = np.abs(gm[ever][:, grp == g]).max(1)
        s = scales[ever, g]
        nz = mx > 0
        assert np.all(mx[nz] <= 448 * s[nz]) and np.all(mx[nz] > 224 * s[nz])
        assert np.all(s[~nz] == 1.0)
    own = torch.from_numpy((gm / scales[:, grp]).astype(np.float32)).to(torch.float8_e4m3fn).to(torch.float64)
    assert np.array_equal(vals[ever], (own.numpy() * scales[:, grp])[ever])
    # and they are within half an FP8 spacing (plus the master's error) of the oracle's weights
    mag = np.maximum(np.abs(w[:, :info.rec_len]), np.abs(gm))
    spacing = 2.0 ** (np.floor(np.log2(np.maximum(mag, 1e-30))) - 3)
    spacing = np.maximum(spacing, 2.0 ** -9 * scales[:, grp])
    assert np.all(np.abs(vals - w[:, :info.rec_len])[ever] <= (0.5 * spacing + 2e-5)[ever])


def test_compose_on_fp8_storage(B, c1):
    prims = I.config4_primitives(8, T=c1.T)
    rays, _, _ = I.config4_rays(64, 64)
    tree_d = B.Tree(c1, "fp8")
    P = len(prims)
    xf = np.ascontiguousarray(np.asarray([p.transform for p in prims], np.float32).reshape(P, 12))
    off = np.ascontiguousarray(np.asarray([p.time_offset for p in prims], np.float32))
    tint = np.ascontiguousarray(np.asarray([p.tint for p in prims], np.float32).reshape(P, 3))
    got = {k: v.cpu().numpy() for k, v in B.neuvv_compose([tree_d] * P, xf, off, tint,
                                                           B.DeviceRays.from_host(rays)).items()}
    q, _ = oracle.quantize_fp8_tree(c1)
    ref = oracle.compose([q] * P, [p.transform for p in prims], [p.time_offset for p in prims],
                         [p.tint for p in prims], rays)
    ok = ref["stop_margin"] > 1e-3
    d_rgb = np.abs(got["rgb"] - ref["rgb"]).max(1)[ok]
    d_a = np.abs(got["alpha"] - ref["alpha"])[ok]
    # the compose allowance: at most 0.1 % of pixels above 1e-4 (grazing face
    # crossings in a primitive's frame), none above 2e-3
    assert (d_rgb > 1e-4).mean() <= 1e-3 and (d_a > 1e-4).mean() <= 1e-3
    assert d_rgb.max() <= 2e-3 and d_a.max() <= 2e-3
