"""The autotuner of the packet kernels (batching: ray-packet launch and
packet order chosen by timing, not fixed): it keeps the fastest of the
candidates it timed, keeps that choice for trees of the same shape on the
same device without timing again, and its choice changes how fast the
kernels run, not what they compute."""
import numpy as np
import pytest
import torch

from paper_2202_06088_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(cuda_lib):
    from paper_2202_06088_gb300 import binding
    return binding


def _chosen(tree_d):
    i = tree_d.info
    return (i.packet_block, i.packet_queue, i.packet_ready, i.packet_order)


def test_autotune_keeps_the_fastest_and_reuses_it(B):
    B.neuvv_autotune_clear_cache()
    tree = I.config1_tree()
    rays, _ = I.config1_rays()
    dr = B.DeviceRays.from_host(rays)
    a = B.Tree(tree, "bf16")
    default = B.neuvv_render(a, dr, kernel="packet")
    best_ms = B.neuvv_autotune(a, dr)
    rows, cached = B.neuvv_autotune_report(a)
    assert not cached
    assert len(rows) >= 10 and {r["order"] for r in rows} == {B.ORDER_AS_GIVEN, B.ORDER_BY_REGION, B.ORDER_BY_RAY}
    fastest = min(rows, key=lambda r: r["ms"])
    assert _chosen(a) == (fastest["block"], fastest["queue"], fastest["ready"], fastest["order"])
    assert abs(best_ms - fastest["ms"]) < 1e-6
    # a second tree of the same shape: the kept choice, nothing timed again
    b = B.Tree(tree, "bf16")
    assert B.neuvv_autotune(b, dr) == best_ms
    rows_b, cached_b = B.neuvv_autotune_report(b)
    assert cached_b and rows_b == rows and _chosen(b) == _chosen(a)
    # another storage type is another key: timed afresh
    c = B.Tree(tree, "f32")
    B.neuvv_autotune(c, dr)
    assert not B.neuvv_autotune_report(c)[1]
    # the launch changes the speed, not the image (rays are independent)
    out = B.alloc_out(dr.n, dr.o.device, log_bytes_per_ray=64)
    B.neuvv_render(a, dr, kernel="packet", out=out)
    for k in ("rgb", "alpha", "nseg"):
        assert torch.equal(out[k], default[k]), k
    B.neuvv_autotune_clear_cache()
    d = B.Tree(tree, "bf16")
    B.neuvv_autotune(d, dr)
    assert not B.neuvv_autotune_report(d)[1]


@pytest.mark.parametrize("order", [0, 1, 2])
@pytest.mark.parametrize("batch", ["view", "shuffled"])
def test_packet_order_does_not_change_results(B, order, batch):
    """Every packet order computes the same rays: the region-ordered schedule
    runs the same packets, the ray order re-forms them, and outputs, segment
    counts and the adjoint that replays the log are those of ray order; on a
    view and on the same rays shuffled."""
    tree = I.config1_tree()
    rays, _ = I.config1_rays()
    if batch == "shuffled":
        rays = rays.subset(np.random.default_rng(9).permutation(rays.n))
    dr = B.DeviceRays.from_host(rays)
    t = B.Tree(tree, "f32")
    t.set_packet_order(0)
    ref = B.alloc_out(dr.n, dr.o.device, log_bytes_per_ray=64)
    B.neuvv_render(t, dr, kernel="packet", out=ref)
    g = torch.randn(dr.n, 3, device="cuda")
    g_ref = B.neuvv_render_backward(t, dr, ref, g, kernel="packet")
    t.set_packet_order(order)
    out = B.alloc_out(dr.n, dr.o.device, log_bytes_per_ray=64)
    B.neuvv_render(t, dr, kernel="packet", out=out)
    for k in ("rgb", "alpha", "depth", "tau", "nseg"):
        assert torch.equal(out[k], ref[k]), k
    g_out = B.neuvv_render_backward(t, dr, out, g, kernel="packet")
    assert (g_out - g_ref).abs().max().item() <= 1e-5 * g_ref.abs().max().item()
    assert t.status() == 0
    with pytest.raises(B.NeuvvError, match="order"):
        t.set_packet_order(7)
