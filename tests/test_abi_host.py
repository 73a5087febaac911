"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads,
exports every entry point that include/neuvv.h declares, and rejects bad
arguments on the host before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2202_06088_gb300 import binding
    return binding.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "neuvv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(neuvv_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary_calls():
    names = _declared()
    for must in ("neuvv_render", "neuvv_render_backward", "neuvv_compose", "neuvv_tree_create", "neuvv_tree_destroy",
                 "neuvv_adam_step", "neuvv_autotune", "neuvv_last_error", "neuvv_tree_coeff_ptrs"):
        assert must in names


def test_library_exports_every_declared_symbol(L):
    from paper_2202_06088_gb300 import binding
    for name in _declared():
        assert hasattr(L, name), name
    assert set(binding.EXPORTS) <= set(_declared())


def test_null_and_bad_arguments_are_rejected_on_the_host(L):
    from paper_2202_06088_gb300 import binding as B
    assert L.neuvv_tree_create(None, None) == 1
    assert L.neuvv_render(None, None, 0.0, None, None, None) == 1
    assert b"NULL" in L.neuvv_last_error()
    d = B.TreeDesc()
    d.depth, d.K, d.T, d.hh_degree, d.n_nodes, d.n_leaves = 0, 8, 30, 2, 1, 0
    h = ctypes.c_void_p()
    assert L.neuvv_tree_create(ctypes.byref(d), ctypes.byref(h)) == 1
    assert b"depth" in L.neuvv_last_error()
    d.depth, d.K = 3, 33
    assert L.neuvv_tree_create(ctypes.byref(d), ctypes.byref(h)) == 1
    assert b"K" in L.neuvv_last_error()


def _desc(child, n_leaves, K=2, T=3, deg=1, depth=2):
    from paper_2202_06088_gb300 import binding as B
    arrs = {"child": np.ascontiguousarray(child, np.uint32),
            "ws": np.zeros((K, n_leaves), np.float32), "wg": np.zeros((K, n_leaves), np.float32),
            "wh": np.zeros((3 * 5, n_leaves), np.float32), "A": np.ones((T, K), np.float32),
            "B": np.ones((T, K), np.float32)}
    d = B.TreeDesc()
    d.depth, d.K, d.T, d.hh_degree, d.dtype = depth, K, T, deg, 0
    d.n_nodes, d.n_leaves = arrs["child"].size // 8, n_leaves
    d.child, d.w_sigma, d.w_gamma = arrs["child"].ctypes.data, arrs["ws"].ctypes.data, arrs["wg"].ctypes.data
    d.w_hh, d.basis_A, d.basis_B = arrs["wh"].ctypes.data, arrs["A"].ctypes.data, arrs["B"].ctypes.data
    for k in range(3):
        d.aabb_min[k], d.aabb_max[k] = 0.0, 1.0
    return d, arrs


def test_malformed_child_tables_are_rejected(L):
    E = 0xFFFFFFFF
    # leaf id out of range
    d, keep = _desc([0x80000005] + [E] * 7, 1)
    h = ctypes.c_void_p()
    assert L.neuvv_tree_create(ctypes.byref(d), ctypes.byref(h)) == 1
    assert b"leaf id" in L.neuvv_last_error()
    # child pointing backwards (a cycle)
    d, keep = _desc([1] + [E] * 7 + [0] + [E] * 7, 0)
    assert L.neuvv_tree_create(ctypes.byref(d), ctypes.byref(h)) == 1
    # internal node at the finest level (depth 1 tree with a child node)
    d, keep = _desc([1] + [E] * 7 + [E] * 8, 0, depth=1)
    assert L.neuvv_tree_create(ctypes.byref(d), ctypes.byref(h)) == 1
    assert b"finest" in L.neuvv_last_error()
    # a node with two parents
    d, keep = _desc([1, 1] + [E] * 6 + [E] * 8, 0, depth=3)
    assert L.neuvv_tree_create(ctypes.byref(d), ctypes.byref(h)) == 1
    assert b"two parents" in L.neuvv_last_error()


def test_render_argument_checks_precede_any_launch(L):
    from paper_2202_06088_gb300 import binding as B
    rays = B.RaysC()
    rays.n = -1
    op = B.OptsC(1e-4, 0, 0, 0)
    # tree handle checked first
    assert L.neuvv_render(None, ctypes.byref(rays), 0.0, ctypes.byref(op), None, None) == 1
    # compose: prim count and transform validity are checked on the host
    arr = (ctypes.c_void_p * 1)(None)
    xf = np.zeros(12, np.float32)
    z = np.zeros(3, np.float32)
    assert L.neuvv_compose(arr, xf.ctypes.data, z.ctypes.data, z.ctypes.data, 0, ctypes.byref(rays), 0.0,
                           ctypes.byref(op), None, None) == 1
    assert L.neuvv_mse_grad(None, None, -1, 1.0, None, None, None) == 1


def test_camera_rays_arguments_are_checked_on_the_host(L):
    from paper_2202_06088_gb300 import binding as B
    cam = B.LightC()
    cam.forward[2], cam.right[0], cam.up[1] = 1.0, 1.0, 1.0
    cam.fov_y_deg, cam.width, cam.height = 40.0, 8, 4
    cams = (B.LightC * 1)(cam)
    t = (ctypes.c_float * 1)(0.5)
    buf = ctypes.c_void_p(16)        # never dereferenced: every call below fails its checks first
    assert L.neuvv_camera_rays(cams, t, 0, 1, buf, buf, buf, None, 32, None) == 1
    assert b"n_cams" in L.neuvv_last_error()
    assert L.neuvv_camera_rays(None, t, 1, 1, buf, buf, buf, None, 32, None) == 1
    assert L.neuvv_camera_rays(cams, t, 1, 1, buf, buf, buf, None, 31, None) == 1
    assert b"pixel count" in L.neuvv_last_error()
    assert L.neuvv_camera_rays(cams, t, 1, 1, None, buf, buf, None, 32, None) == 1
    t[0] = 1.5
    assert L.neuvv_camera_rays(cams, t, 1, 1, buf, buf, buf, None, 32, None) == 1
    assert b"time" in L.neuvv_last_error()
    t[0] = 0.5
    cams[0].fov_y_deg = 180.0
    assert L.neuvv_camera_rays(cams, t, 1, 1, buf, buf, buf, None, 32, None) == 1
    cams[0].fov_y_deg, cams[0].width = 40.0, 0
    assert L.neuvv_camera_rays(cams, t, 1, 1, buf, buf, buf, None, 0, None) == 1


def test_reserve_adjoint_arguments_are_checked_on_the_host(L):
    assert L.neuvv_tree_reserve_adjoint(None, 0) == 1
    assert b"NULL" in L.neuvv_last_error()


def test_new_entry_points_check_their_arguments_on_the_host(L):
    """Null trees, negative limits, unknown orders and tile shapes, missing
    buffers: rejected before any device work."""
    from paper_2202_06088_gb300 import binding as B
    assert L.neuvv_tree_set_limits(None, 0, 0) == 1
    assert L.neuvv_tree_set_packet_order(None, 0) == 1
    assert L.neuvv_tree_set_records(None, None, None) == 1
    n = ctypes.c_int32()
    assert L.neuvv_autotune_report(None, None, 0, ctypes.byref(n), None) == 1
    assert L.neuvv_autotune_clear_cache() == 0
    assert L.neuvv_log_read(None, 4, 8, None, None, None, None) == 1
    assert b"nseg" in L.neuvv_last_error()
    assert L.neuvv_render_backward_adam(None, None, 0.0, None, None, None, None, None, None, 1e-3, 0.9, 0.999,
                                        1e-8, 1, None) == 1
    cam = B.LightC()
    cam.fov_y_deg, cam.width, cam.height = 40.0, 8, 4
    for k in range(3):
        cam.right[k], cam.up[k], cam.forward[k] = float(k == 0), float(k == 1), float(k == 2)
    arr = (B.LightC * 1)(cam)
    ts = (ctypes.c_float * 1)(0.5)
    buf = np.zeros(7 * 32, np.float32)
    p = buf.ctypes.data
    # tile shapes 0..3 are known; 4 is rejected before the launch
    assert L.neuvv_camera_rays(arr, ts, 1, 4, p, p, p, None, 32, None) == 1
    assert b"tile" in L.neuvv_last_error()
    best = ctypes.c_int32()
    assert L.neuvv_autotune_tiles(None, arr, ts, 1, ctypes.byref(best), None, None) == 1
