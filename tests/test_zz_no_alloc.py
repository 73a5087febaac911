"""neuvv_compose_noalloc: composition for callers that cannot allocate device
memory when they render (a frame callback that must stay out of the
allocator, or a process whose device memory another framework reserved up
front).  It keeps its packet counter in the library's own static device
memory, and runs the same kernel on the same inputs as neuvv_compose (rays
do not interact, whichever warp takes their packet), so its images must be
bit-identical to neuvv_compose's, call after call.

This file is named to be collected last: if it fails, a run that stops at the
first failure has already run every other test.  It also passes on its own in
a fresh process (the first call on a device looks up the counter's address).
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2202_06088_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _args(B, prims):
    P = len(prims)
    xf = np.ascontiguousarray(np.asarray([p.transform for p in prims], np.float32).reshape(P, 12))
    off = np.ascontiguousarray(np.asarray([p.time_offset for p in prims], np.float32))
    tint = np.ascontiguousarray(np.asarray([p.tint for p in prims], np.float32).reshape(P, 3))
    return xf, off, tint


def test_noalloc_compose_matches_compose_on_consecutive_calls(cuda_lib):
    from paper_2202_06088_gb300 import binding as B
    L = cuda_lib
    tree = I.config1_tree()
    prims = I.config4_primitives(8, T=tree.T)
    rays, _, _ = I.config4_rays(96, 96)
    tree_d = B.Tree(tree, "f32")
    dr = B.DeviceRays.from_host(rays)
    xf, off, tint = _args(B, prims)
    ref = B.neuvv_compose([tree_d] * 8, xf, off, tint, dr)
    torch.cuda.synchronize()
    arr = (ctypes.c_void_p * 8)(*([tree_d.handle.value] * 8))
    op = B.OptsC(1e-4, 0, 0, 0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        out = {"rgb": torch.full((dr.n, 3), float("nan"), device="cuda"),
               "alpha": torch.full((dr.n,), float("nan"), device="cuda"),
               "depth": torch.full((dr.n,), float("nan"), device="cuda")}
        rc, oc = dr.c(), B._outc(out)
        status = L.neuvv_compose_noalloc(arr, xf.ctypes.data, off.ctypes.data, tint.ctypes.data, 8, ctypes.byref(rc),
                                         0.0, ctypes.byref(op), ctypes.byref(oc), stream)
        assert status == 0, L.neuvv_last_error()
        torch.cuda.synchronize()
        assert (ref["alpha"] > 0.01).float().mean().item() > 0.05
        assert torch.equal(out["rgb"], ref["rgb"]), call
        assert torch.equal(out["alpha"], ref["alpha"]), call
        assert torch.equal(out["depth"], ref["depth"]), call
    # the binding's wrapper (outputs allocated by it on the tree's device)
    got = B.neuvv_compose_noalloc([tree_d] * 8, xf, off, tint, dr)
    assert got["rgb"].device == ref["rgb"].device
    assert torch.equal(got["rgb"], ref["rgb"]) and torch.equal(got["alpha"], ref["alpha"])
    assert tree_d.status() == 0


def test_noalloc_compose_rejects_more_rays_than_its_maximum(cuda_lib):
    from paper_2202_06088_gb300 import binding as B
    L = cuda_lib
    tree_d = B.Tree(I.config1_tree(), "f32")
    small = torch.zeros(16, device="cuda")
    rc = B.RaysC()
    rc.ox = rc.oy = rc.oz = rc.dx = rc.dy = rc.dz = small.data_ptr()
    rc.t = None
    rc.n = (1 << 37) + 1               # checked on the host; nothing is launched
    out = {"rgb": small, "alpha": small, "depth": None}
    oc = B._outc(out)
    eye = np.ascontiguousarray(np.concatenate([np.eye(3), np.zeros((3, 1))], 1).astype(np.float32))
    z = np.zeros(1, np.float32)
    ones = np.ones(3, np.float32)
    arr = (ctypes.c_void_p * 1)(tree_d.handle.value)
    op = B.OptsC(1e-4, 0, 0, 0)
    status = L.neuvv_compose_noalloc(arr, eye.ctypes.data, z.ctypes.data, ones.ctypes.data, 1, ctypes.byref(rc), 0.0,
                                     ctypes.byref(op), ctypes.byref(oc), None)
    assert status == 1
    assert b"rays" in L.neuvv_last_error()
