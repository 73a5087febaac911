"""Comparison helpers shared by the GPU parity tests."""
import numpy as np


def align_sequences(a_ids, a_len, b_ids, b_len, eps):
    """Matches two leaf sequences of one ray.  Equal ids pair up in order; a
    segment present on one side only is allowed when its chord is below eps
    (the extra cell that a near-tie between two crossing planes puts on the
    ray, with a chord no longer than the tie's width).  Returns (ok, pairs)."""
    i = j = 0
    pairs = []
    na, nb = len(a_ids), len(b_ids)
    while i < na or j < nb:
        if i < na and j < nb and a_ids[i] == b_ids[j]:
            pairs.append((i, j))
            i += 1
            j += 1
        elif i < na and a_len[i] < eps:
            i += 1
        elif j < nb and b_len[j] < eps:
            j += 1
        else:
            return False, pairs
    return True, pairs


def psnr(a, b, peak=1.0):
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10.0 * np.log10(peak * peak / mse)


def finest_cell(tree):
    return min((tree.aabb_max[k] - tree.aabb_min[k]) for k in range(3)) / (1 << tree.depth)


def compare_traces(tree, ref, gpu, max_out, eps_rel=1e-3, chord_tol_rel=5e-3):
    """Per-ray leaf sequences: ids must align exactly (tiny near-tie cells
    excepted), chords agree within chord_tol_rel of a finest cell.  Returns
    counts (n_ok, n_bad, bad_rays)."""
    cell = finest_cell(tree)
    eps = eps_rel * cell
    bad = []
    n = ref["count"].shape[0]
    for r in range(n):
        ca, cb = int(ref["count"][r]), int(gpu["count"][r])
        if ca > max_out or cb > max_out:
            bad.append((r, "overflow"))
            continue
        a_ids = ref["leaf"][r, :ca]
        b_ids = gpu["leaf"][r, :cb]
        a_len = ref["t1"][r, :ca] - ref["t0"][r, :ca]
        b_len = gpu["t1"][r, :cb] - gpu["t0"][r, :cb]
        ok, pairs = align_sequences(a_ids, a_len, b_ids, b_len, eps)
        if ok:
            for i, j in pairs:
                if abs(a_len[i] - b_len[j]) > chord_tol_rel * cell:
                    ok = False
                    break
        if not ok:
            bad.append((r, "mismatch"))
    return n - len(bad), len(bad), bad


def nseg_mismatch_explained(B, tree, tree_d, rays, idx, max_out=None):
    """For rays whose composited-segment counts differ between the GPU and the
    oracle, checks that their leaf sequences still align under the tiny-cell
    rule (the difference is a near-tie cell with a chord below 1e-3 of a
    finest cell).  Returns the indices that are not explained."""
    import oracle
    if len(idx) == 0:
        return []
    sub = rays.subset(np.asarray(idx))
    mo = max_out or 4 * (1 << tree.depth)
    ref = oracle.trace(tree, sub, max_out=mo)
    dr = B.DeviceRays.from_host(sub)
    got = {k: v.cpu().numpy() for k, v in B.neuvv_trace(tree_d, dr, mo).items()}
    _, _, bad = compare_traces(tree, ref, got, mo)
    bad_rows = {r for r, _ in bad}
    # aligned sequences of equal length cannot explain a different count
    bad_rows |= {r for r in range(len(idx)) if int(ref["count"][r]) == int(got["count"][r])}
    return [int(np.asarray(idx)[r]) for r in sorted(bad_rows)]
