"""Pins for the oracle's composition (Eq. st_composite_affine, Algorithm 1),
its sparse Adam (Sec. 4.3 "Optimization") and its BF16 rounding.

Composition is pinned by reductions (identity transform = plain render,
disjoint primitives = union, scale invariance, looping re-time), by the
two-layer case worked by hand and by three layers in Algorithm 1's literal
mode, where the sequential merge depends on the layers' order; Adam and BF16
by library routines."""
import math

import numpy as np
import pytest

import oracle
from paper_2202_06088_gb300 import inputs as I


@pytest.fixture(scope="module")
def c1():
    return I.config1_tree()


def _identity():
    return np.concatenate([np.eye(3), np.zeros((3, 1))], 1)


def test_single_identity_primitive_equals_render(c1):
    rays, _ = I.config1_rays()
    r = oracle.render(c1, rays)
    c = oracle.compose([c1], [_identity()], [0.0], [[1.0, 1.0, 1.0]], rays)
    assert np.abs(c["rgb"] - r["rgb"]).max() < 1e-12
    assert np.abs(c["alpha"] - r["alpha"]).max() < 1e-12
    fin = np.isfinite(r["depth"])
    assert np.array_equal(fin, np.isfinite(c["depth"]))
    assert np.abs(c["depth"][fin] - r["depth"][fin]).max() < 1e-12


def test_time_offset_loops_and_tint_scales(c1):
    rays, _ = I.config1_rays()
    T = c1.T
    # offset of a whole period maps every frame to itself
    a = oracle.compose([c1], [_identity()], [0.0], [[1, 1, 1]], rays)
    b = oracle.compose([c1], [_identity()], [float(T - 1)], [[1, 1, 1]], rays)
    assert np.abs(a["rgb"] - b["rgb"]).max() < 1e-12
    # offset of k frames equals rendering at t + k/(T-1) (no wrap at t=0.37, k=3)
    k = 3.0
    shifted = I.Rays(rays.origins, rays.dirs, (rays.times.astype(np.float64) + k / (T - 1)).astype(np.float64))
    c = oracle.compose([c1], [_identity()], [k], [[1, 1, 1]], rays)
    r = oracle.render(c1, shifted)
    assert np.abs(c["rgb"] - r["rgb"]).max() < 1e-9
    tint = [0.5, 0.75, 0.25]
    d = oracle.compose([c1], [_identity()], [0.0], [tint], rays)
    assert np.abs(d["rgb"] - a["rgb"] * np.array(tint)).max() < 1e-14
    assert np.abs(d["alpha"] - a["alpha"]).max() == 0.0


def test_scale_invariance(c1):
    """Scaling a primitive by s about its centre and the camera distance by s
    gives the same image (optical depth integrates over local length), with
    depth scaled by s."""
    cam = I.sphere_cameras(43, 1, 2.5, 48, 48)[0]
    rays, _ = I.camera_rays(cam, 0.37)
    s = 1.7
    M = np.concatenate([s * np.eye(3), (np.array([0.5, 0.5, 0.5]) * (1 - s))[:, None]], 1)
    # the same rays, origins moved away from the centre by s (in float64)
    rays2 = I.Rays(0.5 + s * (rays.origins.astype(np.float64) - 0.5), rays.dirs.astype(np.float64), rays.times)
    a = oracle.compose([c1], [_identity()], [0.0], [[1, 1, 1]], rays)
    b = oracle.compose([c1], [M], [0.0], [[1, 1, 1]], rays2)
    assert np.abs(a["rgb"] - b["rgb"]).max() < 1e-12
    fin = np.isfinite(a["depth"])
    assert np.abs(b["depth"][fin] - s * a["depth"][fin]).max() < 1e-11


def test_rotation_is_the_inverse_view(c1):
    """Rotating the primitive by R equals viewing the original with the camera
    rotated by R^-1 about the primitive's centre."""
    rng = np.random.default_rng(30)
    R = I._random_rotations(rng, 1)[0]
    ctr = np.array([0.5, 0.5, 0.5])
    M = np.concatenate([R, (ctr - R @ ctr)[:, None]], 1)
    rays = I.config1_rays()[0].subset(np.arange(0, 16384, 7))
    a = oracle.compose([c1], [M], [0.0], [[1, 1, 1]], rays)
    o2 = (R.T @ (rays.origins.astype(np.float64) - ctr[:, None])) + ctr[:, None]
    d2 = R.T @ rays.dirs.astype(np.float64)
    b = oracle.render(c1, I.Rays(o2, d2, rays.times))
    assert np.abs(a["rgb"] - b["rgb"]).max() < 1e-9


def test_disjoint_primitives_give_the_union(c1):
    cam = I.look_at(np.array([0.0, -6.0, 0.5]), np.array([0.0, 0.0, 0.5]), 64, 32)
    rays, _ = I.camera_rays(cam, 0.2)
    left = np.concatenate([np.eye(3), np.array([[-1.6], [-0.5], [0.0]])], 1)
    right = np.concatenate([np.eye(3), np.array([[0.6], [-0.5], [0.0]])], 1)
    both = oracle.compose([c1, c1], [left, right], [0.0, 5.0], [[1, 1, 1], [1, 0.5, 0.5]], rays)
    l = oracle.compose([c1], [left], [0.0], [[1, 1, 1]], rays)
    r = oracle.compose([c1], [right], [5.0], [[1, 0.5, 0.5]], rays)
    assert (l["alpha"] > 0).any() and (r["alpha"] > 0).any()
    assert not ((l["alpha"] > 0) & (r["alpha"] > 0)).any()
    assert np.abs(both["rgb"] - (l["rgb"] + r["rgb"])).max() < 1e-14
    assert np.abs(both["alpha"] - (l["alpha"] + r["alpha"])).max() < 1e-14


def test_two_layers_by_hand(c1):
    """L = 2, worked out by hand: the nearer layer f goes over the farther b,
    I = P_f + (1 - A_f) P_b, A = A_f + (1 - A_f) A_b, D = D_f; Algorithm 1 read
    on premultiplied colour gives the same (sequential order irrelevant at L = 2)."""
    cam = I.look_at(np.array([0.5, -4.0, 0.5]), np.array([0.5, 0.5, 0.5]), 40, 40)
    rays, _ = I.camera_rays(cam, 0.6)
    near = np.concatenate([0.8 * np.eye(3), np.array([[0.1], [-0.2], [0.1]])], 1)
    far = _identity()
    lay = [oracle.compose([c1], [M], [o], [t], rays) for M, o, t in
           ((near, 2.0, [1, 1, 1]), (far, 9.0, [0.6, 0.9, 1.0]))]
    for order in ((0, 1), (1, 0)):
        prims = [(near, 2.0, [1, 1, 1]), (far, 9.0, [0.6, 0.9, 1.0])]
        ps = [prims[i] for i in order]
        for mode in ("sorted", "alg1"):
            out = oracle.compose([c1, c1], [p[0] for p in ps], [p[1] for p in ps], [p[2] for p in ps], rays, mode=mode)
            for i in range(rays.n):
                D = [lay[0]["depth"][i], lay[1]["depth"][i]]
                f, b = (0, 1) if D[0] <= D[1] else (1, 0)
                if D[0] == D[1] and order == (1, 0):
                    f, b = b, f
                I_ = lay[f]["rgb"][i] + (1 - lay[f]["alpha"][i]) * lay[b]["rgb"][i]
                A_ = lay[f]["alpha"][i] + (1 - lay[f]["alpha"][i]) * lay[b]["alpha"][i]
                assert np.allclose(out["rgb"][i], I_, atol=1e-14)
                assert abs(out["alpha"][i] - A_) < 1e-14
                assert out["depth"][i] == min(D)


def _three_layers(c1, n=64):
    """Three half-size copies of the depth-6 tree behind one another as seen
    from a camera on the -y side, shifted sideways so that they overlap in
    part: near, mid and far."""
    cam = I.look_at(np.array([0.5, -4.0, 0.5]), np.array([0.5, 0.5, 0.5]), n, n, fov_y_deg=12.0)
    rays, _ = I.camera_rays(cam, 0.6)
    prims = {}
    for name, dy, dx in (("near", -0.6, -0.03), ("mid", 0.0, 0.0), ("far", 0.6, 0.03)):
        prims[name] = (np.concatenate([0.6 * np.eye(3), np.array([[0.2 + dx], [0.2 + dy], [0.2]])], 1),
                       {"near": 2.0, "mid": 5.0, "far": 11.0}[name],
                       {"near": [1.0, 0.8, 0.6], "mid": [0.5, 1.0, 0.7], "far": [0.9, 0.9, 1.0]}[name])
    layers = {k: oracle.compose([c1], [M], [o], [t], rays) for k, (M, o, t) in prims.items()}
    return rays, prims, layers


@pytest.mark.parametrize("order", [("near", "far", "mid"), ("far", "near", "mid"), ("mid", "near", "far")])
def test_algorithm1_three_layers_by_hand(c1, order):
    """Algorithm 1 taken literally on three premultiplied layers, worked by
    hand for pixels where all three are present with depths near < mid < far:
      (near, far, mid): far goes behind near (D_f > D_n); mid is not nearer
        than the running depth D_n, so it goes behind everything so far:
        I = P_n + (1-A_n) P_f + (1-A_n)(1-A_f) P_m;
      (far, near, mid): near goes in front (D_n <= D_f), mid behind:
        the same I as above;
      (mid, near, far): near in front of mid, far behind: the depth-sorted
        result I = P_n + (1-A_n) P_m + (1-A_n)(1-A_m) P_f.
    Alpha is 1 - (1-A_n)(1-A_m)(1-A_f) and depth D_n in every order.  In the
    first two orders the literal algorithm differs from the sorted mode, which
    always gives the last formula."""
    rays, prims, L = _three_layers(c1)
    ps = [prims[k] for k in order]
    out = oracle.compose([c1] * 3, [p[0] for p in ps], [p[1] for p in ps], [p[2] for p in ps], rays, mode="alg1")
    srt = oracle.compose([c1] * 3, [p[0] for p in ps], [p[1] for p in ps], [p[2] for p in ps], rays, mode="sorted")
    n, m, f = L["near"], L["mid"], L["far"]
    sel = ((n["alpha"] > 0.05) & (m["alpha"] > 0.05) & (f["alpha"] > 0.05)
           & (n["depth"] < m["depth"]) & (m["depth"] < f["depth"]))
    assert sel.sum() >= 20
    An, Am, Af = (x["alpha"][sel, None] for x in (n, m, f))
    Pn, Pm, Pf = (x["rgb"][sel] for x in (n, m, f))
    sorted_I = Pn + (1 - An) * Pm + (1 - An) * (1 - Am) * Pf
    mid_last_I = Pn + (1 - An) * Pf + (1 - An) * (1 - Af) * Pm
    want = mid_last_I if order[2] == "mid" else sorted_I
    assert np.abs(out["rgb"][sel] - want).max() < 1e-13
    assert np.abs(srt["rgb"][sel] - sorted_I).max() < 1e-13
    assert np.abs(out["alpha"][sel] - (1 - (1 - An) * (1 - Am) * (1 - Af))[:, 0]).max() < 1e-13
    assert np.array_equal(out["depth"][sel], n["depth"][sel])
    if order[2] == "mid":
        assert np.abs(mid_last_I - sorted_I).max() > 1e-3


def test_adam_matches_torch_on_touched_rows():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(31)
    n, rec = 40, 7
    w = rng.standard_normal((n, rec))
    touched = rng.random(n) < 0.5
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    wt = torch.tensor(w[touched].copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([wt], lr=0.01, betas=(0.9, 0.99), eps=1e-8)
    w0 = w.copy()
    for step in range(1, 6):
        g = rng.standard_normal((n, rec))
        oracle.adam(w, m, v, g, touched, 0.01, 0.9, 0.99, 1e-8, step)
        opt.zero_grad()
        wt.grad = torch.tensor(g[touched])
        opt.step()
    assert np.abs(w[touched] - wt.detach().numpy()).max() < 1e-13
    assert np.array_equal(w[~touched], w0[~touched])


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(32)
    x = np.concatenate([rng.standard_normal(10000).astype(np.float32) * 10.0 ** rng.integers(-8, 8, 10000),
                        np.array([0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.4e38, -3.4e38, 1e-40, np.inf, -np.inf],
                                 np.float32)]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(oracle.round_bf16(x).view(np.uint32), ref.view(np.uint32))
