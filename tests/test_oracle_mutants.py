"""The oracle's pins are strong enough to catch plausible mistakes.

Each case plants one mistake (a dropped term, a wrong sign, index, constant
or operand order) in a copy of the oracle's C source, compiles it with gcc,
and runs a battery of the pins against it on the CPU: at least one pin must
fail.  The unmodified source must pass the same battery."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2202_06088_gb300 import inputs as I

MUTANTS = {
    "printed_A_nl_factorial": ("fact(n - l) / (M_PI * fact(n + l + 1))", "fact(n - l + 1) / (M_PI * fact(n + l + 1))"),
    "gegenbauer_lambda_n_plus_l": ("or_hh_norm(n, l) * pow(sin(gamma), l) * or_gegenbauer(n - l, l + 1.0, cos(gamma))",
                                   "or_hh_norm(n, l) * pow(sin(gamma), l) * or_gegenbauer(n - l, n + l, cos(gamma))"),
    "missing_sqrt2_m_pos": ("if (m > 0) return sqrt(2.0) * K * P * cos(am * phi);", "if (m > 0) return K * P * cos(am * phi);"),
    "legendre_recurrence_sign": ("(ll + m - 1.0) * pmm) / (ll - m)", "(ll - m - 1.0) * pmm) / (ll - m)"),
    "transmittance_off_by_one": ("double T = exp(-tau);", "double T = exp(-(tau + e.sigma * delta));"),
    "child_slot_xz_swapped": ("(int)(((cell[0] >> bit) & 1) * 4 + ((cell[1] >> bit) & 1) * 2 + ((cell[2] >> bit) & 1))",
                              "(int)(((cell[2] >> bit) & 1) * 4 + ((cell[1] >> bit) & 1) * 2 + ((cell[0] >> bit) & 1))"),
    "basis_lerp_weights_swapped": ("a[k] = (1.0 - fr) * tr->A[f0 * tr->K + k] + fr * tr->A[f1 * tr->K + k];",
                                   "a[k] = fr * tr->A[f0 * tr->K + k] + (1.0 - fr) * tr->A[f1 * tr->K + k];"),
    "depth_uses_entry_not_midpoint": ("dnum += w * 0.5 * (segs[i].t0 + segs[i].t1);", "dnum += w * segs[i].t0;"),
    "grad_suffix_sign": ("(Tn * s->e.c[ch] - suffix[4 * (i + 1) + ch])", "(Tn * s->e.c[ch] + suffix[4 * (i + 1) + ch])"),
    "grad_drops_alpha_term": ("dsig += gA * s->delta * (Tn - suffix[4 * (i + 1) + 3]);", ""),
    "grad_drops_sigmoid_slope": ("dc * s->e.c[ch] * (1.0 - s->e.c[ch])", "dc * s->e.c[ch]"),
    "grad_gamma_missing_pi": ("dgamma * M_PI * sg * (1.0 - sg)", "dgamma * sg * (1.0 - sg)"),
    "radial_derivative_sign": ("return or_hh_norm(n, l) * (t1 - t2);", "return or_hh_norm(n, l) * (t1 + t2);"),
    "compose_over_without_transmittance": ("for (int ch = 0; ch < 3; ++ch) I[ch] += (1.0 - A) * LC[3 * j + ch];",
                                           "for (int ch = 0; ch < 3; ++ch) I[ch] += LC[3 * j + ch];"),
    "compose_scale_not_applied_to_depth": ("LD[j] = isinf(out.depth) ? INFINITY : out.depth / inv_s;",
                                           "LD[j] = out.depth;"),
    "early_stop_one_segment_late": ("if (exp(-tau) < op->t_stop) break;",
                                    "if (exp(-(tau - e.sigma * delta)) < op->t_stop) break;"),
    "e4m3_subnormal_spacing_halved": ("if (binade < -6) binade = -6;", "if (binade < -7) binade = -7;"),
    "e4m3_ties_away_from_zero": ("return copysign(nearbyint(a / spacing) * spacing, x);",
                                 "return copysign(round(a / spacing) * spacing, x);"),
    "fp8_scale_search_starts_too_high": ("int p = e - 10;", "int p = e - 8;"),
    "fp8_scale_not_smallest_at_exact_fit": ("while (ldexp(448.0, p) < mx) ++p;", "while (ldexp(448.0, p) <= mx) ++p;"),
    "edit_blend_weights_swapped": ("e.c[ch] = (1.0 - c->beta) * e.c[ch] + c->beta * E[ch];",
                                   "e.c[ch] = c->beta * e.c[ch] + (1.0 - c->beta) * E[ch];"),
    "pick_uses_transmittance": ("if (1.0 - exp(-optical) >= c->threshold) {", "if (exp(-optical) >= c->threshold) {"),
    "slice_gamma_missing_pi": ("const double gamma = M_PI * sigmoid(pg);", "const double gamma = sigmoid(pg);"),
    "slice_m_index_mirrored": ("sh[(leaf * 3 + ch) * NY + l * l + l + m] = acc;", "sh[(leaf * 3 + ch) * NY + l * l + l - m] = acc;"),
    "slice_radial_l_for_n": ("* or_hh_radial(n, l, gamma);\n          sh[", "* or_hh_radial(l, l, gamma);\n          sh["),
    "alg1_compares_first_depth": ("if (LD[i] <= D) {", "if (LD[i] <= LD[0]) {"),
    "margin_skips_entry_crossings": (
        "if (ahead - tin < *margin && order_matters(tr, c_out, ax_in, si, x, sx)) *margin = ahead - tin;", ""),
    "margin_plane_behind_on_wrong_side": ("c_prev[x] -= sx;", "c_prev[x] += sx;"),
    "margin_counts_every_near_tie": (
        "if (gap < *margin && order_matters(tr, cell, ax, sa, x, gd[x] > 0.0 ? 1 : -1)) *margin = gap;",
        "if (gap < *margin) *margin = gap;"),
    "margin_gap_from_segment_start": ("double gap = tnext[x] - tnext[ax];", "double gap = tnext[x] - t_cur;"),
    "margin_past_the_early_stop": ("if (margin && tnext[ax] <= t_limit) {", "if (margin) {"),
}


def _battery():
    """Quick versions of the pins; returns the names of those that fail."""
    failed = []
    rng = np.random.default_rng(0)
    # orthonormality (degree 2, exact quadrature)
    xg, wg = np.polynomial.legendre.leggauss(16)
    gam = (xg + 1) * math.pi / 2
    wg = wg * math.pi / 2 * np.sin(gam) ** 2
    xt, wt = np.polynomial.legendre.leggauss(8)
    phis = np.arange(8) * 2 * math.pi / 8
    G = np.zeros((14, 14))
    for g, w1 in zip(gam, wg):
        for ct, w2 in zip(xt, wt):
            st = math.sqrt(1 - ct * ct)
            for ph in phis:
                h = oracle.hh_all(2, g, np.array([st * math.cos(ph), st * math.sin(ph), ct]))
                G += w1 * w2 * (2 * math.pi / 8) * np.outer(h, h)
    if np.abs(G - np.eye(14)).max() > 1e-9:
        failed.append("orthonormal")
    # addition theorem up to degree 3
    for _ in range(5):
        v = rng.standard_normal(3)
        v /= np.linalg.norm(v)
        h = oracle.hh_all(3, rng.uniform(0, math.pi), v)
        for n in range(4):
            s_ = sum(h[oracle.hh_index(n, l, m)] ** 2 for l in range(n + 1) for m in range(-l, l + 1))
            if abs(s_ - (n + 1) ** 2 / (2 * math.pi ** 2)) > 1e-12:
                failed.append("addition")
                break
    # harmonic derivative vs finite difference
    d = np.array([0.36, 0.48, 0.8])
    fd = (oracle.hh_all(3, 1.0 + 1e-6, d) - oracle.hh_all(3, 1.0 - 1e-6, d)) / 2e-6
    if np.abs(oracle.hh_all_dgamma(3, 1.0, d) - fd).max() > 1e-7:
        failed.append("dgamma")
    # traversal against brute force
    from test_oracle_render import _brute_force, _random_rays, _const_tree
    st = I.random_mixed_tree(4, 3)
    tree = I.make_coefficients(rng, st, K=2, T=3, hh_degree=1)
    rays = _random_rays(rng, 60)
    tr = oracle.trace(tree, rays, max_out=64)
    for i in range(rays.n):
        ids, a, b = _brute_force(tree, rays.origins[:, i].astype(np.float64), rays.dirs[:, i].astype(np.float64))
        if not np.array_equal(tr["leaf"][i, :tr["count"][i]], ids):
            failed.append("trace")
            break
    # constant density closed form, weights + T = 1, early stop
    ct = _const_tree(3, float(np.float32(1.7)))
    out = oracle.render(ct, rays, t_stop=0.0)
    from test_oracle_render import _box_chord
    L = np.array([_box_chord(rays.origins[:, i].astype(np.float64), rays.dirs[:, i].astype(np.float64))
                  for i in range(rays.n)])
    if np.abs(out["alpha"] - (1 - np.exp(-float(np.float32(1.7)) * L))).max() > 1e-12:
        failed.append("closed_form")
    c1 = I.config1_tree()
    r1 = I.config1_rays()[0].subset(np.arange(0, 16384, 97))
    o1 = oracle.render(c1, r1)
    if np.abs(o1["alpha"] + np.exp(-o1["tau"]) - 1).max() > 1e-12:
        failed.append("sum_to_one")
    deep = _const_tree(4, 40.0)
    r = I.Rays(np.array([[-1.0], [0.53], [0.47]], np.float32), np.array([[1.0], [0.0], [0.0]], np.float32),
               np.zeros(1, np.float32))
    f = oracle.trace(deep, r, max_out=64)
    tau = np.cumsum(40.0 * (f["t1"][0, :f["count"][0]] - f["t0"][0, :f["count"][0]]))
    if oracle.render(deep, r)["nseg"][0] != int(np.argmax(np.exp(-tau) < 1e-4)) + 1:
        failed.append("early_stop")
    # single voxel: colour closed form and depth at the chord midpoint
    sv = I.make_coefficients(rng, I.build_tree(2, np.array([2]), np.array([[1, 2, 1]])), K=3, T=4, hh_degree=2)
    wh = np.zeros_like(sv.w_hh)
    wh[:, 0, 0] = [0.7, -1.3, 2.1]
    sv = sv.with_coeffs(w_hh=wh)
    o = oracle.render(sv, rays, t_stop=0.0)
    tsv = oracle.trace(sv, rays)
    hit = tsv["count"] > 0
    cc = 1 / (1 + np.exp(-wh[:, 0, 0].astype(np.float64) / (math.pi * math.sqrt(2))))
    a = 1 - np.exp(-o["tau"][hit])
    if np.abs(o["rgb"][hit] - a[:, None] * cc).max() > 1e-13 or \
            np.abs(o["depth"][hit] - 0.5 * (tsv["t0"][hit, 0] + tsv["t1"][hit, 0]))[a > 1e-4].max() > 1e-12:
        failed.append("single_voxel")
    # one-hot density reproduces the basis at a fractional frame
    one = I.make_coefficients(rng, I.build_tree(1, np.array([1]), np.array([[0, 0, 0]])), K=3, T=5, hh_degree=1)
    ws = np.zeros((3, 1), np.float32)
    ws[1, 0] = 1
    one = one.with_coeffs(w_sigma=ws)
    rr = I.Rays(np.array([[-1.0], [0.25], [0.25]], np.float32), np.array([[1.0], [0.0], [0.0]], np.float32),
                np.array([0.5625], np.float32))
    u = 0.5625 * 4
    ref = (1 - (u - 2)) * float(one.basis_A[2, 1]) + (u - 2) * float(one.basis_A[3, 1])
    if abs(oracle.render(one, rr, t_stop=0.0)["tau"][0] / 0.5 - ref) > 1e-12:
        failed.append("one_hot")
    # gradient vs central differences
    from test_oracle_grad import _loss
    gt = I.make_coefficients(rng, I.random_mixed_tree(3, 21, 0.3, 0.2), K=3, T=4, hh_degree=2, mean_sigma=6.0)
    gr = _random_rays(rng, 24)
    g = rng.standard_normal((gr.n, 3))
    ga = rng.standard_normal(gr.n)
    ws, wgm, whh = (gt.w_sigma.astype(np.float64), gt.w_gamma.astype(np.float64), gt.w_hh.astype(np.float64))
    an = oracle.render_grad(gt, gr, g, ga, t_stop=0.0, otree=oracle.OracleTree(gt, ws, wgm, whh))
    leaf = int(np.argmax(np.abs(an["w_hh"]).sum((0, 1))))
    for name, idx in (("w_sigma", (0, leaf)), ("w_gamma", (1, leaf)), ("w_hh", (1, 3, leaf)), ("w_hh", (0, 0, leaf))):
        arr = {"w_sigma": ws, "w_gamma": wgm, "w_hh": whh}[name]
        b0 = arr[idx]
        arr[idx] = b0 + 1e-6
        lp, _ = _loss(gt, gr, g, ga, ws, wgm, whh, 0.0, "sigmoid")
        arr[idx] = b0 - 1e-6
        lm, _ = _loss(gt, gr, g, ga, ws, wgm, whh, 0.0, "sigmoid")
        arr[idx] = b0
        fdv = (lp - lm) / 2e-6
        if abs(fdv - an[name][idx]) > 1e-6 * abs(an[name][idx]) + 1e-8:
            failed.append("fd_" + name)
            break
    # compose: two layers by hand and scale invariance
    eye = np.concatenate([np.eye(3), np.zeros((3, 1))], 1)
    cam = I.look_at(np.array([0.5, -4.0, 0.5]), np.array([0.5, 0.5, 0.5]), 12, 12)
    cr, _ = I.camera_rays(cam, 0.6)
    near = np.concatenate([0.8 * np.eye(3), np.array([[0.1], [-0.2], [0.1]])], 1)
    l0 = oracle.compose([c1], [near], [2.0], [[1, 1, 1]], cr)
    l1 = oracle.compose([c1], [eye], [9.0], [[0.6, 0.9, 1.0]], cr)
    both = oracle.compose([c1, c1], [near, eye], [2.0, 9.0], [[1, 1, 1], [0.6, 0.9, 1.0]], cr)
    front = l0["depth"] <= l1["depth"]
    Pf = np.where(front[:, None], l0["rgb"], l1["rgb"])
    Pb = np.where(front[:, None], l1["rgb"], l0["rgb"])
    Af = np.where(front, l0["alpha"], l1["alpha"])
    if np.abs(both["rgb"] - (Pf + (1 - Af)[:, None] * Pb)).max() > 1e-13:
        failed.append("compose_by_hand")
    s = 1.7
    M = np.concatenate([s * np.eye(3), (np.array([0.5, 0.5, 0.5]) * (1 - s))[:, None]], 1)
    cr2 = I.Rays(0.5 + s * (cr.origins.astype(np.float64) - 0.5), cr.dirs.astype(np.float64), cr.times)
    a0 = oracle.compose([c1], [eye], [0.0], [[1, 1, 1]], cr)
    a1 = oracle.compose([c1], [M], [0.0], [[1, 1, 1]], cr2)
    fin = np.isfinite(a0["depth"])
    if np.abs(a1["depth"][fin] - s * a0["depth"][fin]).max() > 1e-10:
        failed.append("compose_scale")
    # time slice: rendering it reproduces the HH render at its time
    sr = _random_rays(rng, 80)
    sr.times[:] = np.float32(0.45)
    if np.abs(oracle.render_slice(gt, oracle.slice_at(gt, float(np.float32(0.45))), sr)["rgb"]
              - oracle.render(gt, sr)["rgb"]).max() > 1e-12:
        failed.append("slice")
    # appearance edits: every voxel edited gives the constant-slab closed form;
    # the pick on a constant density lands where alpha passes the threshold
    et = _const_tree(3, 2.0)
    e_all = np.tile([0.2, 0.5, 0.9, 1.5, 0.0], (et.n_leaves, 1))
    eo = oracle.render_edit(et, rays, e_all, beta=1.0, t_stop=0.0)
    if np.abs(eo["rgb"][:, 2] - 0.9 * (1 - np.exp(-1.5 * L))).max() > 1e-12:
        failed.append("edit")
    pt = _const_tree(3, float(np.float32(12.0)))
    pk = oracle.pick(pt, rays, 0.99, t_stop=0.0)
    ptr = oracle.trace(pt, rays, max_out=64)
    s_star = math.log(100.0) / float(np.float32(12.0))
    for i in range(rays.n):
        if L[i] < s_star + 1e-6:
            if pk[i] != -1:
                failed.append("pick")
                break
            continue
        k = np.searchsorted(ptr["t1"][i, :ptr["count"][i]] - ptr["t0"][i, 0], s_star - 1e-12)
        if pk[i] != ptr["leaf"][i, k]:
            failed.append("pick")
            break
    # Algorithm 1 literally on three layers (near, far, mid): mid goes behind
    import test_oracle_compose as toc
    try:
        toc.test_algorithm1_three_layers_by_hand(c1, ("far", "near", "mid"))
    except AssertionError:
        failed.append("alg1_three_layers")
    # decision margins: the hand-built edge rays, moved crossings, the workload
    import test_oracle_margin as tom
    for fn in (tom.test_ray_through_an_edge_between_leaves_has_zero_margin,
               tom.test_margin_is_the_gap_between_the_two_crossings,
               tom.test_margin_ignores_near_ties_whose_order_does_not_matter,
               tom.test_few_rays_of_the_render_workload_have_small_margins,
               lambda: tom.test_crossings_moved_within_half_the_margin_keep_the_leaves(11, 3)):
        try:
            fn()
        except AssertionError:
            failed.append("margin")
            break
    # FP8 E4M3: midpoints go to the even code; per-group scales are minimal
    from test_oracle_fp8 import e4m3_codes
    v = e4m3_codes()
    mid = 0.5 * (v[:-1] + v[1:])
    even = np.where(np.arange(v.size - 1) % 2 == 0, v[:-1], v[1:])
    if not np.array_equal(oracle.round_e4m3(mid), even):
        failed.append("fp8_ties")
    _, sq = oracle.quantize_fp8_groups(np.array([[448.0, 1.0], [300.0, -1.0], [0.0, 0.0]], np.float32))
    if not np.array_equal(sq, [1.0, 1.0, 1.0]):
        failed.append("fp8_scale")
    return failed


@pytest.fixture(scope="module")
def swap():
    saved = oracle._lib

    def use(L):
        oracle._lib = L

    yield use
    oracle._lib = saved


def test_unmodified_oracle_passes_the_battery():
    assert _battery() == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, swap, tmp_path):
    old, new = MUTANTS[name]
    src = oracle.source()
    assert src.count(old) == 1, f"pattern for {name} not found exactly once"
    L = oracle.compile_variant(src.replace(old, new), str(tmp_path / f"mut_{name}.so"))
    swap(L)
    failed = _battery()
    assert failed, f"no pin caught the planted mistake {name}"
