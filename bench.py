#!/usr/bin/env python3
"""VOctree renderer benchmark (NeuVV Sec. 4.3): training-step throughput.

Workload: the depth-9 shell VOctree (~2M occupied leaves, K=16 temporal
bases over T=150 frames, HH degree 3), 8 camera poses on a sphere of radius
2.5 at 1920x1080, each at its own time stamp: 16,588,800 rays per step, all
resident in HBM.  Coefficients are stored in BF16 with an FP32 master copy.

One step = forward render (packet kernel) -> loss gradient against fixed
target images (Eq. rgb-loss plus 0.1 x the image-gradient regulariser of
Sec. 4.3) -> fused adjoint and sparse Adam on the touched leaves in one call
(gradient sums formed per leaf from each leaf's run of samples, laid out by
a count over the segment log, where a step has at least one ray per leaf,
and the Adam update applied by the same per-leaf pass).  The
headline metric is leaf-segment samples per second of the forward+backward
pair (a sample is one leaf segment evaluated by the forward and re-evaluated
by the adjoint, counted once).

Also reported: the BF16 forward alone (ms per 1080p frame), the plain FP32
single-view kernel on the same rays, the roofline of the dominant kernel,
the same metric end to end through the C ABI with host buffers, and the FP64
oracle timed on a bounded sample on the host cores.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Multi-GPU (torchrun) runs independent replicas: one per GPU, no data-path
collective; only the timing uses a barrier and a max over ranks.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "VOctree Msamples/s fwd+bwd (BF16 batched vs FP32 plain); ms per 1080p frame; %roof"
UNIT = "Msamples/s"
LAMBDA_GRAD = 0.1   # weight of the image-gradient regulariser in the total loss (Sec. 4.3)
WORKLOAD = ("depth-9 shell VOctree (~2M leaves, K=16, T=150, HH degree 3), 8 views x 1920x1080 "
            "at 8 time stamps (16,588,800 rays), BF16 storage + FP32 master; step = fwd + loss grad (MSE + 0.1 "
            "image-gradient regulariser) + adjoint + sparse Adam")


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle baseline sample")
    p.add_argument("--views", type=int, default=8, help="1920x1080 views per step (8 = the benchmark workload)")
    p.add_argument("--no-autotune", action="store_true", help="keep the default packet launch configuration")
    p.add_argument("--no-fp8", action="store_true", help="skip the FP8-storage ablation leg")
    p.add_argument("--no-gather", action="store_true",
                   help="adjoint with the atomic scatter only (no leaf-major workspace reserved)")
    p.add_argument("--no-extra", action="store_true",
                   help="skip the legs of the other workloads (depth-8 and depth-10 training, stereo composition)")
    p.add_argument("--launch", default=None, help="packet launch block,queue,ready (profiling case; default: library's)")
    p.add_argument("--order", type=int, default=None,
                   help="packet order of the forward after autotuning (0 as given, 1 by region; default: tuned)")
    p.add_argument("--profile-kernel", choices=["fwd", "bwd", "bwd_adam"], default=None,
                   help="profiling case: launch that kernel twice on the workload and exit (no JSON)")
    p.add_argument("--profile-workload", choices=["views", "depth8_train"], default="views",
                   help="profiling case's input: the --views 1080p views of the depth-9 tree, or the depth-8 "
                        "training batch (262,144 rays over 1.28 M leaves: fewer samples than leaves)")
    return p.parse_args()


def flops_per_sample(K, deg, backward=False):
    """Algorithmic FP32 operations per leaf segment (FMA = 2): two K-dots,
    the radial recurrence (4 per (n,l) pair), the colour sums (per channel
    N_h FMAs over m plus one FMA per (n,l) pair), activations and compositing
    (~20).  The adjoint recomputes that and adds d/dgamma of the radial
    factors, dL/dw_HH (2 per coefficient), dL/dgamma (per channel N_h + pairs
    FMAs) and the two K-long scatters."""
    nh = sum((n + 1) ** 2 for n in range(deg + 1))
    pairs = (deg + 1) * (deg + 2) // 2
    fwd = 4 * K + 4 * pairs + 3 * 2 * (nh + pairs) + 20
    if not backward:
        return fwd
    return fwd + 4 * pairs + 3 * 2 * nh + 3 * 2 * (nh + pairs) + 4 * K + 30


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured", float(d.get("sm_max_mhz", 2070.0))
    except Exception:
        return 6800.0, "fallback", 2070.0


def kernel_sources_digest():
    """sha256 (first 16 hex digits) over the library's CUDA sources, in name order."""
    import hashlib
    d = os.path.join(ROOT, "paper_2202_06088_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(d)):
        if name.endswith((".cu", ".cuh", ".h", ".cpp")):
            h.update(name.encode())
            with open(os.path.join(d, name), "rb") as f:
                h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel):
    """DRAM bytes per launch of a step kernel from the committed ncu summary,
    or None when the summary is missing or the kernel sources changed since."""
    path = os.path.join(ROOT, "profiles", "dram_traffic_depth9_8x1080p.md")
    try:
        with open(path) as f:
            lines = f.read().splitlines()
    except OSError:
        return None
    digest = kernel_sources_digest()
    for ln in lines:
        w = ln.split()
        if len(w) == 6 and w[0] == "traffic" and w[2] == kernel and w[4] == "sources":
            return int(w[3]) if w[5] == digest else None
    return None


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def grad_planes(ot):
    """FP64 gradient planes of an oracle tree, written once so that their
    pages are mapped before any timed region."""
    return {"w_sigma": np.full((ot.K, ot.n_leaves), 0.0), "w_gamma": np.full((ot.K, ot.n_leaves), 0.0),
            "w_hh": np.full((3, ot.N_h, ot.n_leaves), 0.0)}


ORACLE_SPAN = 4096   # consecutive rays of the workload (a band of 128 pixel tiles of one view)


ORACLE_SPANS_PER_CORE = 32   # spans per thread in one timed call (equal contiguous shares per thread)


def oracle_sample(rng, n_rays, n_spans):
    """Ray indices of n_spans seeded random distinct spans of ORACLE_SPAN
    consecutive rays, the spans in random order.  The oracle's samples keep
    the workload's neighbourhoods (a span's rays meet the same records, as
    the GPU's packets do), and with many spans per thread each thread's share
    mixes costly and cheap parts of the views."""
    total = n_rays // ORACLE_SPAN
    pick = rng.choice(total, size=min(max(n_spans, 1), total), replace=False)
    return (pick[:, None] * ORACLE_SPAN + np.arange(ORACLE_SPAN)[None, :]).ravel()


def oracle_step(tree, rays, ot, planes, rng, cores):
    """One timed oracle call as both oracle arms make it: forward and adjoint
    of ORACLE_SPANS_PER_CORE random spans per thread, accumulated into the
    FP64 planes.  Returns (samples, seconds, the sample's rays, their dL/dC,
    their segment counts)."""
    import oracle
    sub = rays.subset(oracle_sample(rng, rays.n, ORACLE_SPANS_PER_CORE * cores))
    g = rng.standard_normal((sub.n, 3))
    nseg = oracle.render(tree, sub, otree=ot, nthreads=cores)["nseg"]
    t0 = time.perf_counter()
    oracle.render_grad(tree, sub, g, otree=ot, nthreads=cores, out=planes)
    return int(nseg.sum()), time.perf_counter() - t0, sub, g, nseg


def cpu_baseline(tree, rays, target_seconds, seed=99):
    """The FP64 oracle's forward+adjoint on the host cores, timed as the
    reference arm times it (`oracle_step`), calls repeated until about
    target_seconds; then part of one call's sample on one core."""
    import oracle
    rng = np.random.default_rng(seed)
    ot = oracle.OracleTree(tree)
    cores = oracle.default_threads()
    planes = grad_planes(ot)
    oracle_step(tree, rays, ot, planes, rng, cores)   # warm-up
    samples, dt, calls = 0, 0.0, 0
    while dt < target_seconds and calls < 64:
        s_, t_, sub, g, nseg = oracle_step(tree, rays, ot, planes, rng, cores)
        samples, dt, calls = samples + s_, dt + t_, calls + 1
    # on one core: seeded spans of the last call's sample (about 3 s; one with samples at least)
    per_span_seg = nseg.reshape(-1, ORACLE_SPAN).sum(1)
    per_span = t_ * cores / per_span_seg.size
    k1 = int(max(1, min(per_span_seg.size, 3.0 / per_span)))
    spans1 = rng.choice(per_span_seg.size, size=k1, replace=False)
    if per_span_seg[spans1].sum() == 0:
        spans1[0] = rng.choice(np.nonzero(per_span_seg > 0)[0])
    pick = (spans1[:, None] * ORACLE_SPAN + np.arange(ORACLE_SPAN)[None, :]).ravel()
    s1 = int(nseg[pick].sum())
    t0 = time.perf_counter()
    oracle.render_grad(tree, sub.subset(pick), g[pick], otree=ot, nthreads=1, out=planes)
    dt1 = time.perf_counter() - t0
    per_call = ORACLE_SPAN * ORACLE_SPANS_PER_CORE * cores
    return {"value": samples / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{calls} calls of {per_call} rays, each in {ORACLE_SPANS_PER_CORE * cores} seeded random spans "
                      f"of {ORACLE_SPAN} consecutive rays of the same 16.6M-ray workload ({samples} samples in "
                      f"all), FP64 forward+adjoint into gradient planes allocated once, {dt:.1f} s",
            "single_core": {"value": s1 / dt1 / 1e6, "unit": UNIT, "rays": int(pick.size), "seconds": dt1}}


def run_reference(args):
    """The reference arm: the FP64 oracle (the only reference this method has)
    timed on bounded samples of the same workload on the host cores.  Each
    step is one call as `cpu_baseline` makes them (`oracle_step`: the
    forward and adjoint of seeded random spans of the rays, accumulated into
    FP64 gradient planes allocated once, outside the timed region, as the
    GPU's adjoint accumulates into its gradient buffer)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2202_06088_gb300 import inputs as I
    oracle.build()
    tree = I.config2_tree()
    rays = I.config2_rays()[0]
    ot = oracle.OracleTree(tree)
    cores = oracle.default_threads()
    rng = np.random.default_rng(5)
    per_step = ORACLE_SPAN * ORACLE_SPANS_PER_CORE * cores   # one call of cpu_baseline per step
    planes = grad_planes(ot)
    times, samples = [], []
    for s in range(args.warmup + args.steps):
        nseg, dt = oracle_step(tree, rays, ot, planes, rng, cores)[:2]
        if s >= args.warmup:
            times.append(dt)
            samples.append(nseg)
    value = sum(samples) / sum(times) / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "per_step_sample_rays": per_step},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} rays per step in {ORACLE_SPANS_PER_CORE * cores} seeded random "
                                       f"spans of {ORACLE_SPAN} "
                                       "consecutive rays of the workload, FP64 fwd+adjoint into gradient planes "
                                       "allocated once"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def slowest_rank_ms(ms, world, device):
    """The job's time: the maximum over the ranks of each rank's timed
    region (every rank runs the same replica workload)."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_msamples_per_s(samples_per_rank, ms_step, world):
    """Whole-job throughput: all ranks' samples over the slowest rank's step."""
    return world * samples_per_rank / (ms_step / 1e3) / 1e6


def reserve_adjoint(B, tree_d, dr, out, enable=True):
    """Sizes the segment log so that it holds every packet of a forward over
    these rays (grown from its given size when the forward ran out of chunks:
    the adjoint walks a packet the log does not hold again, which is slow for
    long incoherent rays), then reserves the leaf-major adjoint's workspace
    for the chunks used (plus a quarter).  Returns the chunks used and the
    chunks the log holds."""
    import numpy as np
    import torch
    for _ in range(4):
        B.neuvv_render(tree_d, dr, kernel="packet", out=out)
        torch.cuda.synchronize()
        head = out["log"][:3].cpu().numpy().astype(np.int64)
        used, n_chunks = int(head[0]), int(head[2])
        if used <= n_chunks:
            break
        log = out["log"]
        out["log"] = torch.empty(int(log.numel() * 1.25 * used / max(n_chunks, 1)) + 1024, dtype=log.dtype,
                                 device=log.device)
        del log
    if enable:
        tree_d.reserve_adjoint(min(n_chunks, used + used // 4 + 1) * 256)
    return used, n_chunks


def train_step_leg(B, tree, rays, dtype, steps, seed, gather=True, force_gather=False):
    """ms per training step (fwd + MSE + adjoint + Adam) and samples/s on one
    workload, targets rendered from perturbed coefficients."""
    import torch
    from paper_2202_06088_gb300 import inputs as I
    dr = B.DeviceRays.from_host(rays)
    n = rays.n
    tgt_tree = B.Tree(I.perturbed(tree, seed=seed), "f32")
    target = B.neuvv_render(tgt_tree, dr, kernel="packet")["rgb"].clone()
    del tgt_tree
    tree_d = B.Tree(tree, dtype, with_optimizer=True)
    B.neuvv_autotune(tree_d, dr)
    out = B.alloc_out(n, dr.o.device, log_bytes_per_ray=64)
    # the per-leaf pass pays per leaf: worth it with at least a sample per leaf
    gather = gather and (n >= tree.n_leaves or force_gather)
    reserve_adjoint(B, tree_d, dr, out, gather)
    grad_rgb = torch.empty(n, 3, device=dr.o.device)
    grad = tree_d.new_grad()
    touched = tree_d.new_touched()
    loss = torch.zeros(1, device=dr.o.device)

    def step(k):
        B.neuvv_render(tree_d, dr, kernel="packet", out=out)
        loss.zero_()
        B.neuvv_mse_grad(out["rgb"], target, scale=1.0 / n, grad=grad_rgb, loss=loss)
        B.neuvv_render_backward_adam(tree_d, dr, out, grad_rgb, None, grad, touched, lr=1e-3, step=k)

    for k in range(3):
        step(k + 1)
    torch.cuda.synchronize()
    samples = int(out["nseg"].sum().item())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(steps):
        step(4 + k)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    # where one step's time goes
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record()
    B.neuvv_render(tree_d, dr, kernel="packet", out=out)
    ev[1].record()
    loss.zero_()
    B.neuvv_mse_grad(out["rgb"], target, scale=1.0 / n, grad=grad_rgb, loss=loss)
    ev[2].record()
    B.neuvv_render_backward_adam(tree_d, dr, out, grad_rgb, None, grad, touched, lr=1e-3, step=4 + steps)
    ev[3].record()
    torch.cuda.synchronize()
    parts = {name: ev[i].elapsed_time(ev[i + 1]) for i, name in enumerate(("fwd", "mse", "bwd_adam"))}
    return {"ms_per_step": ms, "msamples_per_s": samples / (ms / 1e3) / 1e6, "rays": n,
            "leaves": tree.n_leaves, "samples_per_step": samples, "storage": dtype, "steps": steps,
            "adjoint": "leaf-major reduction" if gather else "atomic scatter", "parts_ms": parts}


def extra_workloads(B, steps, gather=True):
    """The other synthetic workloads, one leg each: the depth-8 differentiable
    render (262,144 rays over 16 cameras x 16 times), the 8-primitive stereo
    composition at 2 x 2160^2 replayed from a CUDA graph, and the depth-10
    training step (8M leaves, 1,048,576 rays) in BF16 and FP8 storage."""
    import torch
    from paper_2202_06088_gb300 import inputs as I
    res = {}
    tree3 = I.config3_tree()
    res["depth8_train_262k_rays"] = train_step_leg(B, tree3, I.config3_rays(), "bf16", steps, 1003, gather)
    del tree3
    tree1 = I.config1_tree()
    prims = I.config4_primitives(8, T=tree1.T)
    rays4 = I.config4_rays()[0]
    t4 = B.Tree(tree1, "bf16")
    dr4 = B.DeviceRays.from_host(rays4)
    xf = [p.transform for p in prims]
    off = [p.time_offset for p in prims]
    tint = [p.tint for p in prims]
    out4 = B.alloc_out(rays4.n)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        B.neuvv_compose([t4] * 8, xf, off, tint, dr4, out=out4)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        B.neuvv_compose([t4] * 8, xf, off, tint, dr4, out=out4)
    for _ in range(3):
        graph.replay()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        graph.replay()
    e1.record()
    torch.cuda.synchronize()
    ms4 = e0.elapsed_time(e1) / steps
    res["compose_8prims_stereo_2160"] = {"ms_per_stereo_frame": ms4, "rays": rays4.n, "primitives": 8,
                                         "mray_prims_per_s": rays4.n * 8 / (ms4 / 1e3) / 1e6,
                                         "storage": "bf16", "cuda_graph": True, "steps": steps}
    del graph, t4, dr4, out4
    tree5 = I.config5_tree()
    rays5 = I.config5_rays()
    res["depth10_train_1m_rays"] = train_step_leg(B, tree5, rays5, "bf16", steps, 1005, gather)
    res["depth10_train_1m_rays_fp8"] = train_step_leg(B, tree5, rays5, "fp8", steps, 1005, gather)
    # the same step with the leaf-major adjoint (Adam fused into the per-leaf pass) for comparison
    res["depth10_train_1m_rays_leaf_major"] = train_step_leg(B, tree5, rays5, "bf16", steps, 1005, gather,
                                                             force_gather=True)
    return res


def profile_case(args, B, tree, dr):
    """Two launches of one kernel of the step on the given views (for ncu)."""
    import torch
    tree_d = B.Tree(tree, "bf16", with_optimizer=args.profile_kernel == "bwd_adam")
    if args.launch:
        tree_d.set_launch(*[int(x) for x in args.launch.split(",")])
    if args.order is not None:
        tree_d.set_packet_order(args.order)
    out = B.alloc_out(dr.n, dr.o.device, log_bytes_per_ray=64)
    reserve_adjoint(B, tree_d, dr, out, not args.no_gather)
    grad_rgb = torch.randn(dr.n, 3, device=dr.o.device) * 1e-3
    grad = tree_d.new_grad()
    touched = tree_d.new_touched()
    for k in range(2):
        if args.profile_kernel == "fwd":
            B.neuvv_render(tree_d, dr, kernel="packet", out=out)
        elif args.profile_kernel == "bwd":
            B.neuvv_render_backward(tree_d, dr, out, grad_rgb, None, grad, touched, kernel="packet")
        else:
            B.neuvv_render_backward_adam(tree_d, dr, out, grad_rgb, None, grad, touched, lr=1e-3, step=k + 1)
    torch.cuda.synchronize()
    print(f"profile case done: {args.profile_kernel} on {dr.n} rays", flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2202_06088_gb300 import binding as B
    from paper_2202_06088_gb300 import inputs as I
    B.lib()

    dev = torch.device("cuda", local)
    if args.profile_kernel and args.profile_workload == "depth8_train":
        profile_case(args, B, I.config3_tree(), B.DeviceRays.from_host(I.config3_rays(), device=dev))
        return
    tree = I.config2_tree()
    rays, view_pixels, view_cams, view_times = I.config2_rays(n_views=args.views)
    n = rays.n
    if args.profile_kernel:
        profile_case(args, B, tree, B.DeviceRays.from_host(rays, device=dev))
        return
    tree_d = B.Tree(tree, "bf16", with_optimizer=True)
    # the pixel tile of the views' packets, then the rays generated on the
    # device in that tiling (the same rays as the generator's, in tile order)
    tiles = B.neuvv_autotune_tiles(tree_d, view_cams, view_times) if not args.no_autotune else B.TILES_8X4
    pix = torch.empty(n, dtype=torch.int32, device=dev)
    dr = B.neuvv_camera_rays(view_cams, view_times, tiled=tiles, pixel_of_ray=pix, device=dev)
    # fixed target images: the same views rendered from perturbed coefficients
    tgt_tree = B.Tree(I.perturbed(tree, seed=1000), "f32")
    target = B.neuvv_render(tgt_tree, dr, kernel="packet")["rgb"].clone()
    del tgt_tree
    if not args.no_autotune:
        B.neuvv_autotune(tree_d, dr)
    if args.order is not None:
        tree_d.set_packet_order(args.order)
    launch = {"block": tree_d.info.packet_block, "queue": tree_d.info.packet_queue,
              "ready": tree_d.info.packet_ready, "order": tree_d.info.packet_order,
              "tiles": {1: "8x4", 2: "4x8", 3: "16x2"}[tiles], "autotuned": not args.no_autotune}
    out = B.alloc_out(n, dev, log_bytes_per_ray=64)
    log_used, log_chunks = reserve_adjoint(B, tree_d, dr, out, not args.no_gather)
    grad_rgb = torch.empty(n, 3, device=dev)
    grad = tree_d.new_grad()
    touched = tree_d.new_touched()
    loss = torch.zeros(1, device=dev)
    stream = torch.cuda.current_stream()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    # the image-gradient regulariser needs each view's pixel -> ray map
    W_img, H_img = 1920, 1080
    view_of_ray = torch.arange(n, device=dev, dtype=torch.int64) // (H_img * W_img)
    ray_of_pixel = torch.empty(args.views * H_img * W_img, dtype=torch.int32, device=dev)
    ray_of_pixel[view_of_ray * (H_img * W_img) + pix.long()] = torch.arange(n, device=dev, dtype=torch.int32)
    ray_of_pixel = ray_of_pixel.view(args.views, H_img, W_img)
    del view_of_ray, pix

    def step(k, evs=None):
        if evs:
            evs[0].record(stream)
        B.neuvv_render(tree_d, dr, kernel="packet", out=out)
        if evs:
            evs[1].record(stream)
        loss.zero_()
        B.neuvv_mse_grad(out["rgb"], target, scale=1.0 / n, grad=grad_rgb, loss=loss)
        if evs:
            evs[2].record(stream)
        B.neuvv_grad_loss(out["rgb"], target, ray_of_pixel, LAMBDA_GRAD / n, grad_rgb, loss)
        if evs:
            evs[3].record(stream)
        B.neuvv_render_backward_adam(tree_d, dr, out, grad_rgb, None, grad, touched, lr=1e-3, beta1=0.9,
                                     beta2=0.999, eps=1e-8, step=k)
        if evs:
            evs[4].record(stream)

    clocks = ClockSampler(local)
    clocks.start()
    for k in range(args.warmup):
        step(k + 1)
    torch.cuda.synchronize()
    samples_before = int(out["nseg"].sum().item())
    # distinct leaves one step touches (for the algorithmic bytes)
    B.neuvv_render(tree_d, dr, kernel="packet", out=out)
    B.neuvv_mse_grad(out["rgb"], target, scale=1.0 / n, grad=grad_rgb, loss=loss)
    B.neuvv_render_backward(tree_d, dr, out, grad_rgb, None, grad, touched, kernel="packet")
    torch.cuda.synchronize()
    touched_leaves = int(sum(bin(int(x) & 0xFFFFFFFF).count("1") for x in touched.cpu().numpy()))
    grad.zero_()
    touched.zero_()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    torch.cuda.nvtx.range_push("timed_steps")   # lets a profiler list the timed launches alone
    for k in range(args.steps):
        step(args.warmup + k + 1, ev[k])
    torch.cuda.nvtx.range_pop()
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms_total = slowest_rank_ms(t_start.elapsed_time(t_end), world, dev)
    ms_step = ms_total / args.steps
    samples = 0.5 * (samples_before + int(out["nseg"].sum().item()))
    value = job_msamples_per_s(samples, ms_step, world)
    kern = {name: statistics.mean(ev[k][i].elapsed_time(ev[k][i + 1]) for k in range(args.steps))
            for i, name in enumerate(["fwd", "mse", "lgrad", "bwd_adam"])}
    # the adjoint and Adam as two calls (no fusion), for comparison
    B.neuvv_render(tree_d, dr, kernel="packet", out=out)
    a0, a1, a2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    bwd_ms, adam_ms = [], []
    for r in range(3):
        a0.record(stream)
        B.neuvv_render_backward(tree_d, dr, out, grad_rgb, None, grad, touched, kernel="packet")
        a1.record(stream)
        B.neuvv_adam_step(tree_d, grad, touched, lr=1e-3, step=args.warmup + args.steps + 1 + r)
        a2.record(stream)
        torch.cuda.synchronize()
        bwd_ms.append(a0.elapsed_time(a1))
        adam_ms.append(a1.elapsed_time(a2))
    kern["bwd_unfused"] = statistics.mean(bwd_ms[1:])
    kern["adam_unfused"] = statistics.mean(adam_ms[1:])
    # the same adjoint call with the atomic scatter only, for comparison
    if not args.no_gather:
        tree_d.reserve_adjoint(0)
        B.neuvv_render(tree_d, dr, kernel="packet", out=out)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        B.neuvv_render_backward(tree_d, dr, out, grad_rgb, None, grad, touched, kernel="packet")
        a0.record(stream)
        for _ in range(5):
            B.neuvv_render_backward(tree_d, dr, out, grad_rgb, None, grad, touched, kernel="packet")
        a1.record(stream)
        torch.cuda.synchronize()
        kern["bwd_atomic_scatter_only"] = a0.elapsed_time(a1) / 5
        grad.zero_()
        touched.zero_()
        reserve_adjoint(B, tree_d, dr, out)

    # -- the BF16 forward alone and the plain FP32 single-view kernel
    reps = max(3, args.steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        B.neuvv_render(tree_d, dr, kernel="packet", out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1) / reps
    fwd_samples = int(out["nseg"].sum().item())
    tree32 = B.Tree(tree, "f32")
    B.neuvv_render(tree32, dr, kernel="plain", out=out)
    e0.record(stream)
    for _ in range(reps):
        B.neuvv_render(tree32, dr, kernel="plain", out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1) / reps
    plain_samples = int(out["nseg"].sum().item())
    rgb32 = B.neuvv_render(tree32, dr, kernel="packet")["rgb"]
    del tree32

    # -- time slice (Sec. 7): slice the tree at the first view's time, then
    #    render that view from the slice and from the HH records
    hbm_gbs0 = load_peaks()[0]
    view = rays.subset(np.arange(1920 * 1080))
    t_view = float(view.times[0])
    drv = B.DeviceRays.from_host(view, device=dev)
    sl = B.neuvv_slice(tree_d, t_view)
    outv = B.alloc_out(view.n, dev)
    for _ in range(2):
        B.neuvv_slice(tree_d, t_view, out=sl)
        B.neuvv_render_slice(tree_d, sl, drv, out=outv)
    e0.record(stream)
    for _ in range(reps):
        B.neuvv_slice(tree_d, t_view, out=sl)
    e1.record(stream)
    torch.cuda.synchronize()
    slice_ms = e0.elapsed_time(e1) / reps
    e0.record(stream)
    for _ in range(reps):
        B.neuvv_render_slice(tree_d, sl, drv, out=outv)
    e1.record(stream)
    torch.cuda.synchronize()
    rs_ms = e0.elapsed_time(e1) / reps
    rgb_slice = outv["rgb"].clone()
    e0.record(stream)
    for _ in range(reps):
        B.neuvv_render(tree_d, drv, kernel="packet", out=outv)
    e1.record(stream)
    torch.cuda.synchronize()
    rv_ms = e0.elapsed_time(e1) / reps
    slice_bytes = tree.n_leaves * ((tree_d.info.rec_stride * 2) + 4 * sl.shape[1])
    time_slice = {"leaves": tree.n_leaves, "slice_ms": slice_ms, "slice_record_bytes": 4 * sl.shape[1],
                  "slice_achieved_gbs": slice_bytes / (slice_ms / 1e3) / 1e9,
                  "slice_frac_of_hbm": slice_bytes / (slice_ms / 1e3) / 1e9 / hbm_gbs0,
                  "render_slice_ms_per_1080p_frame": rs_ms, "render_hh_ms_per_1080p_frame": rv_ms,
                  "max_abs_rgb_slice_vs_hh": float((rgb_slice - outv["rgb"]).abs().max().item())}
    # -- spotlight shadow and distance falloff (Sec. 5): alpha map from a
    #    256x256 camera at the light, Gaussian filter, lit view 0
    light_cam = I.look_at(np.array([0.5, 0.5, 3.0]), np.array([0.5, 0.5, 0.5]), 256, 256, fov_y_deg=40.0)
    # the light's rays in row-major pixel order: its alpha output is the map
    lrays, _ = I.camera_rays(light_cam, t_view, tiled=False)
    dlr = B.DeviceRays.from_host(lrays, device=dev)
    lout = B.alloc_out(lrays.n, dev)
    amap = lout["alpha"].view(1, 256, 256)
    blurred = torch.empty_like(amap)
    lit = torch.empty_like(outv["rgb"])

    def light_pass():
        # the light's alpha map: a density-only render (no colour)
        B.neuvv_render_alpha(tree_d, dlr, out=lout)
        B.neuvv_gaussian_blur(amap, 1.5, out=blurred)

    def lit_frame():
        light_pass()
        B.neuvv_render(tree_d, drv, kernel="packet", out=outv)
        B.neuvv_spotlight(drv, outv, light_cam, blurred[0], 0.0, [0.8, 0.8, 0.8], 2.5, out=lit)

    # the light pass (no shared work counter) on a second stream, concurrent
    # with the viewer's render
    side = torch.cuda.Stream(device=dev)
    light_done = torch.cuda.Event()

    def lit_frame_concurrent():
        side.wait_stream(stream)                            # the previous frame is done with the buffers
        with torch.cuda.stream(side):
            light_pass()
            light_done.record(side)
        B.neuvv_render(tree_d, drv, kernel="packet", out=outv)
        stream.wait_event(light_done)
        B.neuvv_spotlight(drv, outv, light_cam, blurred[0], 0.0, [0.8, 0.8, 0.8], 2.5, out=lit)

    def timed(fn):
        fn()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    # the light map of the density-only pass equals the full render's alpha
    B.neuvv_render(tree_d, dlr, kernel="packet", out=lout)
    alpha_full = lout["alpha"].clone()
    light_pass()
    torch.cuda.synchronize()
    alpha_same = bool(torch.equal(alpha_full, lout["alpha"]))
    lit_ms = timed(lit_frame)
    lit_seq = lit.clone()
    lit_cc_ms = timed(lit_frame_concurrent)
    same = float((lit_seq - lit).abs().max().item())
    part_ms = {name: timed(fn) for name, fn in (
        ("light_alpha_256x256", lambda: B.neuvv_render_alpha(tree_d, dlr, out=lout)),
        ("light_full_render_256x256", lambda: B.neuvv_render(tree_d, dlr, kernel="packet", out=lout)),
        ("gaussian_blur", lambda: B.neuvv_gaussian_blur(amap, 1.5, out=blurred)),
        ("spotlight_shading", lambda: B.neuvv_spotlight(drv, outv, light_cam, blurred[0], 0.0, [0.8, 0.8, 0.8], 2.5,
                                                        out=lit)))}
    time_slice["spotlight"] = {"lit_1080p_frame_ms": lit_ms, "plain_1080p_frame_ms": rv_ms,
                               "overhead_frac": lit_ms / rv_ms - 1.0,
                               "lit_1080p_frame_ms_light_pass_concurrent": lit_cc_ms,
                               "overhead_frac_light_pass_concurrent": lit_cc_ms / rv_ms - 1.0,
                               "parts_ms": part_ms, "light_alpha_equals_full_render_alpha": alpha_same,
                               "max_abs_lit_concurrent_vs_sequential": same,
                               "light_map": [256, 256], "blur_sigma": 1.5,
                               "note": "density-only light render (256x256) + blur + viewer render + spotlight "
                                       "shading; the paper reports about 20% lower render speed with shadows and "
                                       "falloff"}
    del alpha_full
    del sl, outv, drv, dlr, lout, amap, blurred, lit, lit_seq

    # -- storage ablation: the same training step on FP8 E4M3 records with
    #    per-leaf scales (same FP32 master, same rays and targets)
    fp8 = None
    if not args.no_fp8:
        tree8 = B.Tree(tree, "fp8", with_optimizer=True)
        tree8.set_launch(launch["block"], launch["queue"], launch["ready"])
        tree8.set_packet_order(launch["order"])
        reserve_adjoint(B, tree8, dr, out, not args.no_gather)
        rgb8 = B.neuvv_render(tree8, dr, kernel="packet")["rgb"]
        mse8 = float(((rgb8 - rgb32) ** 2).mean().item())
        rgb16 = B.neuvv_render(tree_d, dr, kernel="packet")["rgb"]
        mse16 = float(((rgb16 - rgb32) ** 2).mean().item())
        del rgb8, rgb16
        g8 = tree8.new_grad()
        t8 = tree8.new_touched()
        st8 = args.steps // 2 + 1

        def step8(k):
            B.neuvv_render(tree8, dr, kernel="packet", out=out)
            loss.zero_()
            B.neuvv_mse_grad(out["rgb"], target, scale=1.0 / n, grad=grad_rgb, loss=loss)
            B.neuvv_grad_loss(out["rgb"], target, ray_of_pixel, LAMBDA_GRAD / n, grad_rgb, loss)
            B.neuvv_render_backward_adam(tree8, dr, out, grad_rgb, None, g8, t8, lr=1e-3, beta1=0.9, beta2=0.999,
                                         eps=1e-8, step=k)

        for k in range(3):
            step8(k + 1)
        torch.cuda.synchronize()
        e0.record(stream)
        for k in range(st8):
            step8(4 + k)
        e1.record(stream)
        torch.cuda.synchronize()
        ms8 = e0.elapsed_time(e1) / st8
        e0.record(stream)
        for _ in range(reps):
            B.neuvv_render(tree8, dr, kernel="packet", out=out)
        e1.record(stream)
        torch.cuda.synchronize()
        f8 = e0.elapsed_time(e1) / reps
        psnr = lambda m: float("inf") if m == 0 else 10 * np.log10(1.0 / m)
        fp8 = {"record_bytes": tree8.info.rec_stride, "ms_per_step": ms8,
               "msamples_per_s": samples / (ms8 / 1e3) / 1e6, "fwd_ms_per_1080p_frame": f8 / args.views,
               "psnr_vs_fp32_storage_db": psnr(mse8), "bf16_psnr_vs_fp32_storage_db": psnr(mse16),
               "steps": st8}
        del tree8, g8, t8
    del rgb32

    # -- roofline of the dominant kernel of the step
    hbm_gbs, peak_kind, sm_max = load_peaks()
    props = torch.cuda.get_device_properties(dev)
    fp32_tflops = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    info = tree_d.info
    elem = 2 if info.dtype == B.BF16 else 4
    rec_bytes = info.rec_stride * elem
    ray_in, fwd_out = 28, 28
    # the fused adjoint + Adam call: each touched leaf's record read once, its
    # FP32 master, m and v (rec_len entries each) read and written, its
    # storage entries written; per ray its ray, saved colour, dL/dC, tau and
    # segment count
    traffic = {
        "fwd": (touched_leaves * rec_bytes + n * (ray_in + fwd_out), samples * flops_per_sample(info.K, info.hh_degree)),
        "bwd_adam": (touched_leaves * (rec_bytes + 6 * 4 * info.rec_len + elem * info.rec_len)
                     + n * (ray_in + 12 + 12 + 4 + 4),
                     samples * flops_per_sample(info.K, info.hh_degree, backward=True)
                     + touched_leaves * info.rec_len * 10),
        "mse": (n * 36, 0),
    }
    def roofline_of(part):
        bytes_, flops_ = traffic[part]
        t_s = kern[part] / 1e3
        if flops_ / (fp32_tflops * 1e12) > bytes_ / (hbm_gbs * 1e9):
            r = {"bound": "alu", "achieved": flops_ / t_s / 1e12, "peak": fp32_tflops, "unit": "TFLOP/s",
                 "peak_kind": "derived: SMs x 128 FP32 lanes x 2 x max SM clock"}
        else:
            r = {"bound": "hbm", "achieved": bytes_ / t_s / 1e9, "peak": hbm_gbs, "unit": "GB/s",
                 "peak_kind": f"{peak_kind} (copy bandwidth)"}
        r["frac"] = r["achieved"] / r["peak"]
        r["kernel"] = part
        # DRAM bytes per launch from one ncu capture of this workload (null once the kernel changed)
        r["traffic"] = measured_traffic(part) if args.views == 8 else None
        r["algorithmic_bytes"] = bytes_
        r["algorithmic_flops"] = flops_
        return r

    dom = max(("fwd", "mse", "bwd_adam"), key=kern.get)
    roof = roofline_of(dom)
    # the other large step part against its own roof
    roof_other = {p: roofline_of(p) for p in ("fwd", "bwd_adam") if p != dom}

    # -- end to end through the C ABI with host buffers.  Every step copies its
    # inputs in from pinned host memory -- the target images and the views'
    # camera poses and times -- generates the rays of its views on the device
    # (neuvv_camera_rays) and copies its loss out.  The targets go to one of
    # two device buffers on a copy stream, so that step k + 1's upload runs
    # while step k computes (what a training loop with a prefetching loader
    # does); all uploads lie inside the timed region.
    h_tgt = target.cpu().pin_memory()
    bufs = [torch.empty_like(target) for _ in range(2)]
    dr_e2e = B.DeviceRays(torch.empty_like(dr.o), torch.empty_like(dr.d), torch.empty_like(dr.t))
    h_loss = torch.zeros(1).pin_memory()
    e2e_steps = max(3, args.steps // 2)
    copy_stream = torch.cuda.Stream(device=dev)
    copied = [torch.cuda.Event() for _ in range(2)]
    used = [torch.cuda.Event() for _ in range(2)]

    def upload(j):
        b = j % 2
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(used[b])              # the buffer's previous step is done with it
            bufs[b].copy_(h_tgt, non_blocking=True)
            copied[b].record(copy_stream)

    def e2e_step(j, k):
        b = j % 2
        B.neuvv_camera_rays(view_cams, view_times, tiled=tiles, out=dr_e2e)
        B.neuvv_render(tree_d, dr_e2e, kernel="packet", out=out)
        stream.wait_event(copied[b])
        loss.zero_()
        B.neuvv_mse_grad(out["rgb"], bufs[b], scale=1.0 / n, grad=grad_rgb, loss=loss)
        B.neuvv_grad_loss(out["rgb"], bufs[b], ray_of_pixel, LAMBDA_GRAD / n, grad_rgb, loss)
        used[b].record(stream)
        B.neuvv_render_backward_adam(tree_d, dr_e2e, out, grad_rgb, None, grad, touched, lr=1e-3, step=k)
        h_loss.copy_(loss, non_blocking=True)

    def e2e_run(n_steps, k0):
        copy_stream.wait_stream(stream)
        upload(0)
        for j in range(n_steps):
            if j + 1 < n_steps:
                upload(j + 1)
            e2e_step(j, k0 + j)
        stream.wait_stream(copy_stream)

    e2e_run(2, args.warmup + args.steps + 1)
    torch.cuda.synchronize()
    e2e_samples = float(out["nseg"].sum().item())       # samples of the device-generated rays
    e0.record(stream)
    e2e_run(e2e_steps, args.warmup + args.steps + 3)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    h2d = n * 12 + len(view_cams) * (15 + 1) * 4          # targets + camera structs and times (launch parameters)
    e2e = {"value": world * e2e_samples / (e2e_ms / 1e3) / 1e6, "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": 4, "ms_per_step": e2e_ms, "samples_per_step": e2e_samples,
           "pipeline": "per step: targets uploaded (on a copy stream, one step ahead, two buffers), rays generated "
                       "on the device from the views' cameras, fwd + loss + adjoint + Adam, loss read back"}
    del bufs, dr_e2e

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "rays": n, "leaves": tree.n_leaves, "depth": tree.depth, "K": tree.K,
                   "T": tree.T, "hh_degree": tree.hh_degree, "storage": "bf16", "master": "f32",
                   "samples_per_step": samples, "touched_leaves": touched_leaves,
                   "l2": "inputs larger than L2 (rays 464 MB + records 512 MB per step)",
                   "parallelism": f"replicas x{world}", "launch": launch,
                   "segment_log": {"chunks_used": log_used, "chunks": log_chunks,
                                   "adjoint": "atomic scatter" if args.no_gather else "leaf-major reduction"},
                   "clocks_window": "warm-up and timed steps"},
        "kernels_ms": kern,
        "fwd_bf16_packet": {"ms_per_1080p_frame": fwd_ms / args.views, "msamples_per_s": fwd_samples / (fwd_ms / 1e3) / 1e6},
        "fwd_fp32_plain": {"ms_per_1080p_frame": plain_ms / args.views,
                           "msamples_per_s": plain_samples / (plain_ms / 1e3) / 1e6},
        "fp8_ablation": fp8,
        "time_slice_and_lighting": time_slice,
        "roofline": roof,
        "roofline_other_parts": roof_other,
        "e2e": e2e,
        "gpu_launches": (8 if args.no_gather else 9) * args.steps,
        "clocks": clk,
    }
    if not args.no_extra:
        line["other_workloads"] = extra_workloads(B, max(5, args.steps // 2), not args.no_gather)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(tree, rays, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
