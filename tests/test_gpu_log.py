"""The timed kernel's own leaf sequences (Sec. 4.3 "Rendering": the voxels
each ray crosses and the lengths of its segments inside them).

The packet forward -- the kernel the bench times, in the launch the
autotuner picks -- records every segment it composites in its segment log;
neuvv_log_read decodes that log per ray.  Each ray's logged (leaf, chord)
list must equal the oracle's traversal up to the composited count: leaf ids
exactly, chords within 1e-3 of a finest cell.  Exempt are only rays the
oracle itself marks ambiguous: a traversal decision margin below the FP32
rounding of the crossings (reading A8), counted and below 0.1 % of the rays,
and, for where the composited prefix ends, an early-stop margin below 1e-3
(then the common prefix is compared).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2202_06088_gb300 import inputs as I

from helpers import MAX_EXEMPT_FRACTION, compare_sequences

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(cuda_lib):
    from paper_2202_06088_gb300 import binding
    return binding


def _rounded(tree, dtype):
    if dtype == "bf16":
        return tree.with_coeffs(oracle.round_bf16(tree.w_sigma), oracle.round_bf16(tree.w_gamma),
                                oracle.round_bf16(tree.w_hh))
    return tree


def _check_log(tree, ref, tr, got_leaf, got_chord, got_count, nseg):
    """ref: oracle.render (nseg, margins); tr: oracle.trace; got_*: the log."""
    assert (got_count >= 0).all(), "a packet is missing from the log"
    assert np.array_equal(got_count, nseg)
    stop_amb = ref["stop_margin"] < 1e-3
    n_ref = np.where(stop_amb, np.minimum(ref["nseg"], nseg), ref["nseg"])
    n_got = np.where(stop_amb, n_ref, nseg)
    exempt, bad = compare_sequences(tree, tr["leaf"], tr["t1"] - tr["t0"], n_ref, got_leaf, got_chord, n_got,
                                    ref["trace_margin"])
    assert bad == [], bad[:10]
    assert len(exempt) < MAX_EXEMPT_FRACTION * len(nseg) + 1, len(exempt)
    return exempt


def _render_and_read(B, tree_d, dr, max_out, log_bytes_per_ray=64):
    out = B.alloc_out(dr.n, dr.o.device, log_bytes_per_ray=log_bytes_per_ray)
    B.neuvv_render(tree_d, dr, kernel="packet", out=out)
    log = B.neuvv_log_read(out, dr.n, max_out)
    return out, log


@pytest.mark.parametrize("dtype,order", [("f32", None), ("bf16", None), ("f32", 2)])
def test_packet_log_matches_oracle_c1(B, dtype, order):
    """The autotuned launch, and the packets re-formed by the library's ray
    order on the same view's rays shuffled (the log then lists packets of
    sorted rays; each ray's segments are read back at its own index)."""
    tree = I.config1_tree()
    rays, _ = I.config1_rays()
    if order is not None:
        rays = rays.subset(np.random.default_rng(4).permutation(rays.n))
    tree_d = B.Tree(tree, dtype)
    dr = B.DeviceRays.from_host(rays)
    B.neuvv_autotune(tree_d, dr)
    if order is not None:
        tree_d.set_packet_order(order)
    mo = 4 * (1 << tree.depth)
    out, log = _render_and_read(B, tree_d, dr, mo)
    src = _rounded(tree, dtype)
    ref = oracle.render(src, rays)
    tr = oracle.trace(src, rays, max_out=mo)
    exempt = _check_log(tree, ref, tr, log["leaf"].cpu().numpy(), log["chord"].cpu().numpy(),
                        log["count"].cpu().numpy(), out["nseg"].cpu().numpy())
    print(f"exempt rays: {len(exempt)} of {rays.n}")
    assert tree_d.status() == 0


@pytest.mark.parametrize("seed,depth,bricks", [(1, 4, True), (2, 5, True), (5, 6, False), (6, 7, True)])
def test_packet_log_matches_oracle_mixed_trees(B, seed, depth, bricks):
    """Leaves at every level, empty nodes, origins inside the box; with the
    brick map (depth >= 3) and without bricks (descents from the lowest common
    ancestor)."""
    rng = np.random.default_rng(seed)
    tree = I.make_coefficients(rng, I.random_mixed_tree(depth, seed), K=3, T=5, hh_degree=2, mean_sigma=8.0)
    from test_oracle_render import _random_rays
    rays = _random_rays(rng, 3000 + 17)     # several packets and a ragged tail
    rays.times[:] = rng.uniform(0, 1, rays.n).astype(np.float32)
    tree_d = B.Tree(tree, "f32", bricks=bricks)
    dr = B.DeviceRays.from_host(rays)
    mo = 4 * (1 << depth)
    # incoherent rays shade few lanes per round: a log of 4 KB per ray holds them all
    out, log = _render_and_read(B, tree_d, dr, mo, log_bytes_per_ray=4096)
    ref = oracle.render(tree, rays)
    tr = oracle.trace(tree, rays, max_out=mo)
    _check_log(tree, ref, tr, log["leaf"].cpu().numpy(), log["chord"].cpu().numpy(), log["count"].cpu().numpy(),
               out["nseg"].cpu().numpy())
    assert tree_d.status() == 0


def test_packet_log_full_size_sampled(B):
    """The bench's workload and launch (8 x 1080p views of the depth-9 shell
    tree, BF16 storage, autotuned packet kernel, 64 log bytes per ray): the
    log of every ray is decoded and 4000 seeded rays are compared with the
    oracle on the BF16-rounded coefficients."""
    tree = I.config2_tree()
    rays = I.config2_rays()[0]
    tree_d = B.Tree(tree, "bf16")
    dr = B.DeviceRays.from_host(rays)
    B.neuvv_autotune(tree_d, dr)
    mo = 96
    out, log = _render_and_read(B, tree_d, dr, mo)
    cnt = log["count"]
    assert (cnt >= 0).all().item()                      # 64 B per ray holds every packet
    assert torch.equal(cnt, out["nseg"])
    idx = np.sort(np.random.default_rng(77).choice(rays.n, size=4000, replace=False))
    it = torch.from_numpy(idx).cuda()
    sub = rays.subset(idx)
    src = _rounded(tree, "bf16")
    ref = oracle.render(src, sub)
    tr = oracle.trace(src, sub, max_out=512)
    nseg = out["nseg"][it].cpu().numpy()
    keep = nseg <= mo                                   # rays with more segments than max_out: not decoded whole
    assert keep.mean() > 0.999
    sel = np.nonzero(keep)[0]
    refk = {k: v[sel] for k, v in ref.items()}
    trk = {k: v[sel] for k, v in tr.items()}
    exempt = _check_log(tree, refk, trk, log["leaf"][it].cpu().numpy()[sel], log["chord"][it].cpu().numpy()[sel],
                        cnt[it].cpu().numpy()[sel], nseg[sel])
    print(f"exempt rays: {len(exempt)} of {sel.size}")
    assert tree_d.status() == 0


def test_log_read_marks_rays_without_a_log(B):
    tree = I.config1_tree()
    rays, _ = I.config1_rays()
    tree_d = B.Tree(tree, "f32")
    dr = B.DeviceRays.from_host(rays)
    out = B.alloc_out(dr.n, dr.o.device, log_bytes_per_ray=64)
    B.neuvv_render(tree_d, dr, kernel="plain", out=out)          # the plain kernel marks the log empty
    log = B.neuvv_log_read(out, dr.n, 8)
    assert (log["count"] == -1).all().item()
    B.neuvv_render(tree_d, dr, kernel="packet", out=out)
    sub = B.neuvv_log_read(out, dr.n - 32, 8)                    # a log written for other rays
    assert (sub["count"] == -1).all().item()
    tiny = B.alloc_out(dr.n, dr.o.device, log_bytes_per_ray=8)   # room for few packets: the rest walk
    B.neuvv_render(tree_d, dr, kernel="packet", out=tiny)
    t = B.neuvv_log_read(tiny, dr.n, 64)
    c, ns = t["count"], tiny["nseg"]
    logged = c >= 0
    assert torch.equal(c[logged], ns[logged])
    assert ((c == -1) | logged).all().item() and (~logged).any().item() and logged.any().item()


def _log_leaf_slots(log, n_rays):
    """The leaf entries of the chunks the forward handed out, from the log's
    layout (64-byte header; heads, keys and order per packet, the ray
    permutation, the sort bins, next links; then leaf and chord per slot)."""
    words = log.cpu().numpy().view(np.uint32)
    used = int(words[0]) | (int(words[1]) << 32)
    n_chunks = int(words[2])
    n_packets = (n_rays + 31) // 32
    pk_bytes = (4 * n_packets + 15) // 16 * 16
    perm_bytes = (4 * n_rays + 15) // 16 * 16
    fixed = 64 + 3 * pk_bytes + perm_bytes + 4 * 4096
    leaf_off = (fixed + 4 * n_chunks + 15) // 16 * 16
    chunks = min(used, n_chunks)
    return words[leaf_off // 4: leaf_off // 4 + chunks * 8 * 32], words[16: 16 + n_packets]


@pytest.mark.parametrize("n", [4096 + 3, 32 * 40])
def test_log_slots_without_a_segment_read_empty(B, n):
    """Every slot of a chunk the forward handed out holds a segment or kEmpty,
    so that the adjoint can count each leaf's samples slot by slot: the rounds
    of a packet's last chunk after its end and the lanes past the last ray are
    written empty.  The log starts out as zeros (leaf 0, a real leaf), so a
    slot left unwritten would add samples of leaf 0."""
    tree = I.config1_tree()
    rays, _ = I.config1_rays()
    rays = rays.subset(np.arange(n) + 6000)             # rows through the middle of the view
    tree_d = B.Tree(tree, "bf16")
    dr = B.DeviceRays.from_host(rays)
    # every ray of these rows crosses the object: 4 KB per ray holds every packet
    out = B.alloc_out(dr.n, dr.o.device, log_bytes_per_ray=4096)
    out["log"].zero_()
    B.neuvv_render(tree_d, dr, kernel="packet", out=out)
    torch.cuda.synchronize()
    leaf, heads = _log_leaf_slots(out["log"], dr.n)
    nseg = out["nseg"].cpu().numpy()
    logged = np.repeat(heads != 0xFFFFFFFF, 32)[:dr.n]
    assert logged.any()
    assert (nseg[~logged] == 0).all(), np.nonzero(nseg[~logged])[0][:8]   # packets without a chunk shaded nothing
    full = int((leaf != 0xFFFFFFFF).sum())
    assert full == int(nseg.sum()), (full, int(nseg.sum()), leaf.size)
    dec = B.neuvv_log_read(out, dr.n, 256)
    assert torch.equal(dec["count"], out["nseg"])
    assert int((leaf == 0).sum()) == int(np.count_nonzero(dec["leaf"].cpu().numpy() == 0))
    assert tree_d.status() == 0
