"""Comparison helpers shared by the GPU parity tests.

Leaf sequences (reading A8) are compared exactly, except on rays whose
oracle decision margin -- the smallest distance along the ray between two
plane crossings whose order decides which leaves are visited -- is below the
rounding of an FP32 traversal: ``decision_eps_cells``.  Those rays are counted
and must stay below 0.1 % of a batch."""
import numpy as np

U32 = 2.0 ** -24           # FP32 unit roundoff
MAX_EXEMPT_FRACTION = 1e-3


def psnr(a, b, peak=1.0):
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10.0 * np.log10(peak * peak / mse)


def finest_cell(tree):
    return min((tree.aabb_max[k] - tree.aabb_min[k]) for k in range(3)) / (1 << tree.depth)


def decision_eps_cells(tree):
    """Decision margin, in finest cells, below which an FP32 traversal may
    order two crossings differently from the FP64 oracle: 8 unit roundoffs of
    the root box's diagonal (the longest distance a crossing is measured
    over from the ray's entry).  Each crossing distance of the FP32 walk is
    within about two roundings of its value, so a margin above this bound
    decides the same order on both sides."""
    diag = float(np.linalg.norm(np.asarray(tree.aabb_max, np.float64) - np.asarray(tree.aabb_min, np.float64)))
    return 8.0 * U32 * diag / finest_cell(tree)


def compare_sequences(tree, ref_leaf, ref_chord, ref_count, got_leaf, got_chord, got_count, margin,
                      chord_tol_cells=1e-3):
    """Per ray: leaf ids equal exactly and chords within chord_tol_cells
    finest cells, unless the ray's oracle margin is below decision_eps_cells
    (exempt).  Counts are compared as given (callers cut both sides to the
    segments they composite).  Returns (exempt ray indices, failing ray
    indices with a reason)."""
    eps = decision_eps_cells(tree)
    cell = finest_cell(tree)
    exempt, bad = [], []
    for r in range(len(ref_count)):
        if margin[r] < eps:
            exempt.append(r)
            continue
        ca, cb = int(ref_count[r]), int(got_count[r])
        if ca != cb:
            bad.append((r, f"count {cb} != {ca}"))
            continue
        if not np.array_equal(np.asarray(ref_leaf[r, :ca], np.int64), np.asarray(got_leaf[r, :cb], np.int64)):
            bad.append((r, "leaf ids"))
            continue
        if ca and np.abs(np.asarray(ref_chord[r, :ca], np.float64) - got_chord[r, :cb]).max() > chord_tol_cells * cell:
            bad.append((r, "chord"))
    return exempt, bad


def compare_traces(tree, ref, gpu, max_out, chord_tol_cells=1e-3):
    """Whole-ray traces (neuvv_trace against oracle.trace, which carries the
    margin over the whole ray)."""
    n = ref["count"].shape[0]
    over = [r for r in range(n) if ref["count"][r] > max_out or gpu["count"][r] > max_out]
    assert not over, over[:10]
    return compare_sequences(tree, ref["leaf"], ref["t1"] - ref["t0"], ref["count"], gpu["leaf"],
                             gpu["t1"] - gpu["t0"], gpu["count"], ref["margin"], chord_tol_cells)


def nseg_differences_unexplained(ref, got, tree, stop_eps=1e-3):
    """Rays whose composited-segment counts differ although neither the early
    stop (oracle stop margin below stop_eps) nor the traversal (oracle
    decision margin below decision_eps_cells) is ambiguous on them."""
    diff = got["nseg"] != ref["nseg"]
    diff &= ref["stop_margin"] >= stop_eps
    diff &= ref["trace_margin"] >= decision_eps_cells(tree)
    return np.nonzero(diff)[0]


def exempt_fraction(ref, tree):
    return float((ref["trace_margin"] < decision_eps_cells(tree)).mean())
