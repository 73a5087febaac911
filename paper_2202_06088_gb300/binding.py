"""Python binding of the C ABI in ``include/neuvv.h`` (argument marshalling only).

Every function here turns PyTorch CUDA tensors into plain pointers and sizes,
calls the entry point of the same name in ``libneuvv.so`` on the current
PyTorch stream, and turns a non-zero status into an exception.  No step of the
rendering, its adjoint, the composition or the optimiser runs in Python.  If
the library cannot be loaded (or built in-tree with nvcc), every call raises:
there is no fallback path.
"""

from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

from . import build as _build

_lock = threading.Lock()
_lib = None

F32, BF16, FP8 = 0, 1, 2
# device status bits (neuvv_tree_status)
STATUS_SEGMENT_CAP, STATUS_BAD_INDEX, STATUS_TIMEOUT = 0x1, 0x2, 0x4
ORDER_AS_GIVEN, ORDER_BY_REGION, ORDER_BY_RAY = 0, 1, 2
TILES_NONE, TILES_8X4, TILES_4X8, TILES_16X2 = 0, 1, 2, 3
TILE_SHAPES = {TILES_8X4: (8, 4), TILES_4X8: (4, 8), TILES_16X2: (16, 2)}
_DTYPES = {"f32": F32, "float32": F32, "bf16": BF16, "bfloat16": BF16, "fp8": FP8, "fp8_e4m3": FP8}
_ACT = {"sigmoid": 0, "identity": 1}
_KERNEL = {"auto": 0, "plain": 1, "packet": 2}
_MODE = {"sorted": 0, "alg1": 1}


class NeuvvError(RuntimeError):
    pass


class TreeDesc(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_int32), ("K", ctypes.c_int32), ("T", ctypes.c_int32), ("hh_degree", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("with_optimizer", ctypes.c_int32),
                ("n_nodes", ctypes.c_int64), ("n_leaves", ctypes.c_int64),
                ("child", ctypes.c_void_p), ("w_sigma", ctypes.c_void_p), ("w_gamma", ctypes.c_void_p),
                ("w_hh", ctypes.c_void_p), ("basis_A", ctypes.c_void_p), ("basis_B", ctypes.c_void_p),
                ("aabb_min", ctypes.c_float * 3), ("aabb_max", ctypes.c_float * 3), ("flags", ctypes.c_uint32)]


class TreeInfo(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_int32), ("K", ctypes.c_int32), ("K_pad", ctypes.c_int32), ("T", ctypes.c_int32),
                ("hh_degree", ctypes.c_int32), ("N_h", ctypes.c_int32), ("rec_len", ctypes.c_int32),
                ("rec_stride", ctypes.c_int32), ("rec_stride_f32", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("n_nodes", ctypes.c_int64), ("n_leaves", ctypes.c_int64),
                ("device", ctypes.c_int32), ("packet_block", ctypes.c_int32), ("packet_queue", ctypes.c_int32),
                ("packet_ready", ctypes.c_int32), ("packet_order", ctypes.c_int32),
                ("packet_tiles", ctypes.c_int32)]


class RaysC(ctypes.Structure):
    _fields_ = [("ox", ctypes.c_void_p), ("oy", ctypes.c_void_p), ("oz", ctypes.c_void_p),
                ("dx", ctypes.c_void_p), ("dy", ctypes.c_void_p), ("dz", ctypes.c_void_p),
                ("t", ctypes.c_void_p), ("n", ctypes.c_int64)]


class OutC(ctypes.Structure):
    _fields_ = [("rgb", ctypes.c_void_p), ("alpha", ctypes.c_void_p), ("depth", ctypes.c_void_p),
                ("tau", ctypes.c_void_p), ("nseg", ctypes.c_void_p), ("log", ctypes.c_void_p),
                ("log_bytes", ctypes.c_int64)]


class TuneEntryC(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int32), ("queue", ctypes.c_int32), ("ready", ctypes.c_int32),
                ("order", ctypes.c_int32), ("ms", ctypes.c_float)]


class OptsC(ctypes.Structure):
    _fields_ = [("t_stop", ctypes.c_float), ("color_act", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("compose_mode", ctypes.c_int32)]


EXPORTS = ["neuvv_last_error", "neuvv_tree_create", "neuvv_tree_destroy", "neuvv_tree_get_info",
           "neuvv_tree_coeff_ptrs", "neuvv_tree_status", "neuvv_render", "neuvv_render_backward", "neuvv_compose",
           "neuvv_adam_step", "neuvv_mse_grad", "neuvv_trace", "neuvv_autotune", "neuvv_compose_noalloc",
           "neuvv_tree_set_launch", "neuvv_slice", "neuvv_render_slice", "neuvv_grad_loss",
           "neuvv_gaussian_blur", "neuvv_spotlight", "neuvv_pick", "neuvv_paint", "neuvv_render_edit",
           "neuvv_camera_rays", "neuvv_render_alpha", "neuvv_tree_reserve_adjoint", "neuvv_tree_set_limits",
           "neuvv_log_read", "neuvv_tree_set_records", "neuvv_render_backward_adam",
           "neuvv_tree_set_packet_order", "neuvv_autotune_report", "neuvv_autotune_clear_cache",
           "neuvv_autotune_tiles"]


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Loads libneuvv.so (building it with nvcc when it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB
            if not os.path.exists(path):
                raise NeuvvError(f"CUDA library not found at {path}")
            L = ctypes.CDLL(path)
            p, i32, i64, f = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
            L.neuvv_last_error.restype = ctypes.c_char_p
            L.neuvv_last_error.argtypes = []
            sig = {
                "neuvv_tree_create": [p, p], "neuvv_tree_destroy": [p], "neuvv_tree_get_info": [p, p],
                "neuvv_tree_coeff_ptrs": [p, p, p, p, p], "neuvv_tree_status": [p, p],
                "neuvv_render": [p, p, f, p, p, p],
                "neuvv_render_backward": [p, p, f, p, p, p, p, p, p, p],
                "neuvv_compose": [p, p, p, p, i32, p, f, p, p, p],
                "neuvv_compose_noalloc": [p, p, p, p, i32, p, f, p, p, p],
                "neuvv_adam_step": [p, p, p, f, f, f, f, i32, p],
                "neuvv_mse_grad": [p, p, i64, f, p, p, p],
                "neuvv_trace": [p, p, i32, p, p, p, p, p],
                "neuvv_autotune": [p, p, f, p, p],
                "neuvv_tree_set_launch": [p, i32, i32, i32],
                "neuvv_slice": [p, f, p, i32, p],
                "neuvv_grad_loss": [p, p, i64, p, i32, i32, i32, f, p, p, p],
                "neuvv_gaussian_blur": [p, p, i32, i32, i32, f, p],
                "neuvv_pick": [p, p, f, f, p, p],
                "neuvv_paint": [p, p, p, i64, f, f, p, p, p],
                "neuvv_render_edit": [p, p, f, p, p, f, p, p],
                "neuvv_spotlight": [p, p, p, p, p, p, f, p, f, p, p],
                "neuvv_render_slice": [p, p, i32, p, p, p, p],
                "neuvv_camera_rays": [p, p, i32, i32, p, p, p, p, i64, p],
                "neuvv_render_alpha": [p, p, f, p, p, p],
                "neuvv_tree_reserve_adjoint": [p, i64],
                "neuvv_tree_set_limits": [p, i32, i32],
                "neuvv_log_read": [p, i64, i32, p, p, p, p],
                "neuvv_tree_set_records": [p, p, p],
                "neuvv_render_backward_adam": [p, p, f, p, p, p, p, p, p, f, f, f, f, i32, p],
                "neuvv_tree_set_packet_order": [p, i32],
                "neuvv_autotune_report": [p, p, i32, p, p],
                "neuvv_autotune_clear_cache": [],
                "neuvv_autotune_tiles": [p, p, p, i32, p, p, p],
            }
            for name, args in sig.items():
                fn = getattr(L, name)
                fn.restype = ctypes.c_int
                fn.argtypes = args
            _lib = L
    return _lib


def _check(status: int) -> None:
    if status != 0:
        msg = lib().neuvv_last_error().decode(errors="replace")
        raise NeuvvError(f"neuvv status {status}: {msg}")


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        if not x.is_cuda:
            raise NeuvvError("expected a CUDA tensor")
        if not x.is_contiguous():
            raise NeuvvError("expected a contiguous tensor")
        return ctypes.c_void_p(x.data_ptr())
    return x


class _CudaView:
    """__cuda_array_interface__ holder for library-owned device memory."""

    def __init__(self, ptr: int, shape, typestr: str, owner):
        self._owner = owner
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 2, "strides": None}


class Tree:
    """A VOctree uploaded to the current CUDA device (neuvv_tree_create)."""

    def __init__(self, voctree, dtype: str = "f32", with_optimizer: bool = False, bricks: bool = True):
        L = lib()
        self.dtype = _DTYPES[dtype]
        child = np.ascontiguousarray(voctree.child, np.uint32)
        ws = np.ascontiguousarray(voctree.w_sigma, np.float32)
        wg = np.ascontiguousarray(voctree.w_gamma, np.float32)
        wh = np.ascontiguousarray(voctree.w_hh, np.float32)
        A = np.ascontiguousarray(voctree.basis_A, np.float32)
        B = np.ascontiguousarray(voctree.basis_B, np.float32)
        d = TreeDesc()
        d.depth, d.K, d.T, d.hh_degree = voctree.depth, voctree.K, voctree.T, voctree.hh_degree
        d.dtype, d.with_optimizer = self.dtype, int(with_optimizer)
        d.flags = 0 if bricks else 1
        d.n_nodes, d.n_leaves = child.size // 8, ws.shape[1]
        d.child, d.w_sigma, d.w_gamma, d.w_hh = child.ctypes.data, ws.ctypes.data, wg.ctypes.data, wh.ctypes.data
        d.basis_A, d.basis_B = A.ctypes.data, B.ctypes.data
        for k in range(3):
            d.aabb_min[k] = voctree.aabb_min[k]
            d.aabb_max[k] = voctree.aabb_max[k]
        h = ctypes.c_void_p()
        _check(L.neuvv_tree_create(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h
        info = TreeInfo()
        _check(L.neuvv_tree_get_info(h, ctypes.byref(info)))
        self.info = info
        self.n_leaves = int(info.n_leaves)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib is not None:
            _lib.neuvv_tree_destroy(h)
            self.handle = None

    def _ptrs(self):
        s, m, a, v = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib().neuvv_tree_coeff_ptrs(self.handle, ctypes.byref(s), ctypes.byref(m), ctypes.byref(a),
                                           ctypes.byref(v)))
        return s.value, m.value, a.value, v.value

    def storage(self) -> torch.Tensor:
        """View of the storage records [n_leaves, rec_stride] (float32, bfloat16,
        or the raw bytes of FP8 records)."""
        s = self._ptrs()[0]
        if self.dtype == FP8:
            return torch.as_tensor(_CudaView(s, (self.n_leaves, self.info.rec_stride), "|u1", self), device="cuda")
        if self.dtype == F32:
            return torch.as_tensor(_CudaView(s, (self.n_leaves, self.info.rec_stride), "<f4", self), device="cuda")
        t = torch.as_tensor(_CudaView(s, (self.n_leaves, self.info.rec_stride), "<i2", self), device="cuda")
        return t.view(torch.bfloat16)

    def master(self) -> torch.Tensor | None:
        m = self._ptrs()[1]
        if not m:
            return None
        return torch.as_tensor(_CudaView(m, (self.n_leaves, self.info.rec_stride_f32), "<f4", self), device="cuda")

    def adam_state(self):
        _, _, a, v = self._ptrs()
        if not a:
            return None, None
        shape = (self.n_leaves, self.info.rec_stride_f32)
        return (torch.as_tensor(_CudaView(a, shape, "<f4", self), device="cuda"),
                torch.as_tensor(_CudaView(v, shape, "<f4", self), device="cuda"))

    def refresh_info(self) -> TreeInfo:
        info = TreeInfo()
        _check(lib().neuvv_tree_get_info(self.handle, ctypes.byref(info)))
        self.info = info
        return info

    def set_launch(self, block: int, queue: int, ready: int) -> None:
        _check(lib().neuvv_tree_set_launch(self.handle, int(block), int(queue), int(ready)))
        self.refresh_info()

    def records_ptr(self) -> int:
        """Device address of the tree's FP32 records: the master copy, or the
        storage itself for an FP32 tree without optimizer state (0 if none)."""
        s, m, _, _ = self._ptrs()
        return m or (s if self.dtype == F32 else 0)

    def set_records(self, records: torch.Tensor) -> None:
        """Replaces the coefficients with FP32 records [n_leaves, rec_stride_f32]
        (neuvv_tree_set_records: master copy and storage, re-rounded)."""
        if records.shape != (self.n_leaves, self.info.rec_stride_f32) or records.dtype != torch.float32:
            raise NeuvvError("records must be float32 [n_leaves, rec_stride_f32]")
        _check(lib().neuvv_tree_set_records(self.handle, _ptr(records.contiguous()), _stream()))

    def set_packet_order(self, order: int) -> None:
        """ORDER_AS_GIVEN or ORDER_BY_REGION for the packet forward with a log."""
        _check(lib().neuvv_tree_set_packet_order(self.handle, int(order)))
        self.refresh_info()

    def set_limits(self, step_cap: int = 0, wait_polls: int = 1 << 22) -> None:
        """Walk-step cap per ray (0: the default, which no ray reaches) and
        polls of a bounded device wait (neuvv_tree_set_limits)."""
        _check(lib().neuvv_tree_set_limits(self.handle, int(step_cap), int(wait_polls)))

    def reserve_adjoint(self, n_slots: int) -> None:
        """Workspace of the leaf-major adjoint for logs of up to n_slots slots
        (56 B per slot; 0 frees it)."""
        _check(lib().neuvv_tree_reserve_adjoint(self.handle, int(n_slots)))

    def status(self) -> int:
        f = ctypes.c_uint32()
        _check(lib().neuvv_tree_status(self.handle, ctypes.byref(f)))
        return int(f.value)

    def new_grad(self) -> torch.Tensor:
        return torch.zeros(self.n_leaves, self.info.rec_stride_f32, device="cuda", dtype=torch.float32)

    def new_touched(self) -> torch.Tensor:
        return torch.zeros((self.n_leaves + 31) // 32, device="cuda", dtype=torch.int32)


class DeviceRays:
    """Rays resident on the device as float32 SoA tensors (origins/dirs [3, n])."""

    def __init__(self, origins: torch.Tensor, dirs: torch.Tensor, times: torch.Tensor | None = None):
        self.o = origins.contiguous()
        self.d = dirs.contiguous()
        self.t = None if times is None else times.contiguous()
        for x in (self.o, self.d) + (() if self.t is None else (self.t,)):
            if x.dtype != torch.float32 or not x.is_cuda:
                raise NeuvvError("rays must be float32 CUDA tensors")
        self.n = int(self.o.shape[1])

    @staticmethod
    def from_host(rays, device="cuda", non_blocking=False) -> "DeviceRays":
        return DeviceRays(torch.as_tensor(np.ascontiguousarray(rays.origins, np.float32)).to(device, non_blocking=non_blocking),
                          torch.as_tensor(np.ascontiguousarray(rays.dirs, np.float32)).to(device, non_blocking=non_blocking),
                          torch.as_tensor(np.ascontiguousarray(rays.times, np.float32)).to(device, non_blocking=non_blocking))

    def c(self) -> RaysC:
        r = RaysC()
        base = self.o.data_ptr()
        r.ox, r.oy, r.oz = base, self.o[1].data_ptr(), self.o[2].data_ptr()
        r.dx, r.dy, r.dz = self.d[0].data_ptr(), self.d[1].data_ptr(), self.d[2].data_ptr()
        r.t = None if self.t is None else self.t.data_ptr()
        r.n = self.n
        return r


def _opts(t_stop=1e-4, act="sigmoid", kernel="auto", mode="sorted") -> OptsC:
    return OptsC(float(t_stop), _ACT[act], _KERNEL[kernel], _MODE[mode])


def alloc_out(n: int, device="cuda", log_bytes_per_ray: int = 0) -> dict:
    """Output tensors of a render; with log_bytes_per_ray > 0 also a segment log
    (lets the backward replay the forward's segments instead of walking)."""
    out = {"rgb": torch.empty(n, 3, device=device), "alpha": torch.empty(n, device=device),
           "depth": torch.empty(n, device=device), "tau": torch.empty(n, device=device),
           "nseg": torch.empty(n, device=device, dtype=torch.int32)}
    if log_bytes_per_ray > 0:
        out["log"] = torch.empty((n * log_bytes_per_ray + 1023) // 16 * 16 // 4 + 64, device=device, dtype=torch.int32)
    return out


def _outc(out: dict) -> OutC:
    ptrs = [None if out.get(k) is None else out[k].data_ptr() for k in ("rgb", "alpha", "depth", "tau", "nseg")]
    log = out.get("log")
    return OutC(*ptrs, None if log is None else log.data_ptr(), 0 if log is None else log.numel() * log.element_size())


def neuvv_render(tree: Tree, rays: DeviceRays, t: float = 0.0, t_stop: float = 1e-4, act: str = "sigmoid",
                 kernel: str = "auto", out: dict | None = None) -> dict:
    out = out if out is not None else alloc_out(rays.n)
    rc, oc, op = rays.c(), _outc(out), _opts(t_stop, act, kernel)
    _check(lib().neuvv_render(tree.handle, ctypes.byref(rc), float(t), ctypes.byref(op), ctypes.byref(oc), _stream()))
    return out


def neuvv_render_alpha(tree: Tree, rays: DeviceRays, t: float = 0.0, t_stop: float = 1e-4,
                       out: dict | None = None) -> dict:
    """Density-only render: alpha, depth, tau and nseg as neuvv_render, no colour."""
    if out is None:
        dev = rays.o.device
        out = {"alpha": torch.empty(rays.n, device=dev), "depth": torch.empty(rays.n, device=dev),
               "tau": torch.empty(rays.n, device=dev), "nseg": torch.empty(rays.n, device=dev, dtype=torch.int32)}
    oc = _outc({k: v for k, v in out.items() if k not in ("rgb", "log")})
    rc, op = rays.c(), _opts(t_stop, "sigmoid", "packet")
    _check(lib().neuvv_render_alpha(tree.handle, ctypes.byref(rc), float(t), ctypes.byref(op), ctypes.byref(oc),
                                    _stream()))
    return out


def neuvv_grad_loss(rgb: torch.Tensor, target: torch.Tensor, ray_of_pixel: torch.Tensor, lam: float = 0.1,
                    grad: torch.Tensor | None = None, loss: torch.Tensor | None = None) -> torch.Tensor:
    """Adds the image-gradient regulariser's gradient to grad (zeros if None)
    and its value to loss[0]; ray_of_pixel: int32 [n_views, height, width]."""
    grad = grad if grad is not None else torch.zeros_like(rgb)
    V, H, W = ray_of_pixel.shape
    _check(lib().neuvv_grad_loss(_ptr(rgb), _ptr(target), int(rgb.shape[0]), _ptr(ray_of_pixel), int(W), int(H),
                                 int(V), float(lam), _ptr(grad), _ptr(loss), _stream()))
    return grad


def neuvv_pick(tree: Tree, rays: DeviceRays, threshold: float = 0.99, t: float = 0.0) -> torch.Tensor:
    """Terminating leaf of each ray (int32, -1 where alpha never reaches the threshold)."""
    leaf = torch.empty(rays.n, dtype=torch.int32, device=rays.o.device)
    rc = rays.c()
    _check(lib().neuvv_pick(tree.handle, ctypes.byref(rc), float(t), float(threshold), _ptr(leaf), _stream()))
    return leaf


def new_edits(tree: Tree) -> torch.Tensor:
    """Edit records [n_leaves, 8], all inactive (t_d = 2)."""
    e = torch.zeros(max(tree.info.n_leaves, 1), 8, device=f"cuda:{tree.info.device}")
    e[:, 3] = -1.0
    e[:, 4] = 2.0
    return e


def neuvv_paint(tree: Tree, leaf: torch.Tensor, colors: torch.Tensor, sigma_d: float, t_d: float,
                edits: torch.Tensor) -> torch.Tensor:
    accum = torch.zeros(max(tree.info.n_leaves, 1), 4, device=edits.device)
    _check(lib().neuvv_paint(tree.handle, _ptr(leaf), _ptr(colors.contiguous()), int(leaf.numel()), float(sigma_d),
                             float(t_d), _ptr(accum), _ptr(edits), _stream()))
    return edits


def neuvv_render_edit(tree: Tree, rays: DeviceRays, edits: torch.Tensor, beta: float = 1.0, t: float = 0.0,
                      t_stop: float = 1e-4, act: str = "sigmoid", out: dict | None = None) -> dict:
    out = out if out is not None else alloc_out(rays.n)
    rc, oc, op = rays.c(), _outc(out), _opts(t_stop, act, "packet")
    _check(lib().neuvv_render_edit(tree.handle, ctypes.byref(rc), float(t), ctypes.byref(op), _ptr(edits),
                                   float(beta), ctypes.byref(oc), _stream()))
    return out


class LightC(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_float * 3), ("right", ctypes.c_float * 3), ("up", ctypes.c_float * 3),
                ("forward", ctypes.c_float * 3), ("fov_y_deg", ctypes.c_float), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32)]


def light_of(cam) -> LightC:
    """The C description of a pinhole camera placed at the light (any object
    with eye, right, up, forward, fov_y_deg, width, height)."""
    L = LightC()
    for k in range(3):
        L.eye[k], L.right[k], L.up[k], L.forward[k] = (float(cam.eye[k]), float(cam.right[k]), float(cam.up[k]),
                                                       float(cam.forward[k]))
    L.fov_y_deg, L.width, L.height = float(cam.fov_y_deg), int(cam.width), int(cam.height)
    return L


def neuvv_gaussian_blur(img: torch.Tensor, sigma: float, out: torch.Tensor | None = None) -> torch.Tensor:
    """img: FP32 [n_images, height, width] on the device."""
    out = out if out is not None else torch.empty_like(img)
    n, h, w = img.shape
    _check(lib().neuvv_gaussian_blur(_ptr(img.contiguous()), _ptr(out), int(w), int(h), int(n), float(sigma),
                                     _stream()))
    return out


def neuvv_camera_rays(cams, times, tiled: bool = True, out: DeviceRays | None = None,
                      pixel_of_ray: torch.Tensor | None = None, device="cuda") -> DeviceRays:
    """Rays through the pixel centres of each camera (any objects with eye,
    right, up, forward, fov_y_deg, width, height), generated on the device:
    camera c's rays follow camera c-1's, at time times[c]; tiled: False
    (row-major), True or TILES_8X4, TILES_4X8, TILES_16X2 (tiles of 32 pixels).  out (optional): DeviceRays of the total size to write into;
    pixel_of_ray (optional, int32 [n]) receives each ray's row-major pixel."""
    cams, times = list(cams), [float(x) for x in times]
    if len(cams) != len(times):
        raise NeuvvError("one time per camera")
    n = sum(int(c.width) * int(c.height) for c in cams)
    if out is None:
        out = DeviceRays(torch.empty(3, n, device=device), torch.empty(3, n, device=device),
                         torch.empty(n, device=device))
    if out.n != n or out.t is None:
        raise NeuvvError("out must hold the cameras' total pixel count, with times")
    done = 0
    for c0 in range(0, len(cams), 32):
        part = cams[c0:c0 + 32]
        arr = (LightC * len(part))(*[light_of(c) for c in part])
        ts = (ctypes.c_float * len(part))(*times[c0:c0 + 32])
        m = sum(int(c.width) * int(c.height) for c in part)
        o, d, t = out.o[:, done:done + m].contiguous(), out.d[:, done:done + m].contiguous(), out.t[done:done + m]
        pix = None if pixel_of_ray is None else pixel_of_ray[done:done + m]
        mode = int(tiled) if not isinstance(tiled, bool) else int(tiled)
        _check(lib().neuvv_camera_rays(arr, ts, len(part), mode, _ptr(o), _ptr(d), _ptr(t),
                                       None if pix is None else _ptr(pix), m, _stream()))
        if o.data_ptr() != out.o[:, done:done + m].data_ptr():  # a chunk of several: copy the [3][m] block back
            out.o[:, done:done + m].copy_(o)
            out.d[:, done:done + m].copy_(d)
        done += m
    return out


def neuvv_spotlight(rays: DeviceRays, render: dict, light_cam, light_alpha: torch.Tensor, ground_z: float,
                    albedo, r_ref: float, out: torch.Tensor | None = None) -> torch.Tensor:
    out = out if out is not None else torch.empty_like(render["rgb"])
    rc, L = rays.c(), light_of(light_cam)
    alb = (ctypes.c_float * 3)(*[float(x) for x in albedo])
    _check(lib().neuvv_spotlight(ctypes.byref(rc), _ptr(render["rgb"]), _ptr(render["alpha"]), _ptr(render["depth"]),
                                 ctypes.byref(L), _ptr(light_alpha.contiguous()), float(ground_z), alb, float(r_ref),
                                 _ptr(out), _stream()))
    return out


def slice_stride(degree: int) -> int:
    """Floats per leaf of a time slice: [sigma, 0, 0, 0] then 3 (degree+1)^2
    coefficients, rounded up to a multiple of 4."""
    return (4 + 3 * (degree + 1) ** 2 + 3) // 4 * 4


def neuvv_slice(tree: Tree, t: float, out: torch.Tensor | None = None) -> torch.Tensor:
    """Time slice of the tree at t: FP32 [n_leaves, slice_stride] (density in
    column 0, spherical-harmonic coefficients from column 4)."""
    stride = slice_stride(tree.info.hh_degree) if out is None else out.shape[1]
    if out is None:
        out = torch.zeros(max(tree.info.n_leaves, 1), stride, device=f"cuda:{tree.info.device}", dtype=torch.float32)
    _check(lib().neuvv_slice(tree.handle, float(t), _ptr(out), int(stride), _stream()))
    return out


def neuvv_render_slice(tree: Tree, sl: torch.Tensor, rays: DeviceRays, t_stop: float = 1e-4, act: str = "sigmoid",
                       out: dict | None = None) -> dict:
    out = out if out is not None else alloc_out(rays.n)
    rc, oc, op = rays.c(), _outc(out), _opts(t_stop, act, "packet")
    _check(lib().neuvv_render_slice(tree.handle, _ptr(sl), int(sl.shape[1]), ctypes.byref(rc), ctypes.byref(op),
                                    ctypes.byref(oc), _stream()))
    return out


def neuvv_render_backward(tree: Tree, rays: DeviceRays, saved: dict, grad_rgb: torch.Tensor,
                          grad_alpha: torch.Tensor | None = None, grad: torch.Tensor | None = None,
                          touched: torch.Tensor | None = None, t: float = 0.0, t_stop: float = 1e-4,
                          act: str = "sigmoid", kernel: str = "auto") -> torch.Tensor:
    grad = grad if grad is not None else tree.new_grad()
    rc, sc, op = rays.c(), _outc(saved), _opts(t_stop, act, kernel)
    _check(lib().neuvv_render_backward(tree.handle, ctypes.byref(rc), float(t), ctypes.byref(op), ctypes.byref(sc),
                                       _ptr(grad_rgb.contiguous()),
                                       _ptr(None if grad_alpha is None else grad_alpha.contiguous()), _ptr(grad),
                                       _ptr(touched), _stream()))
    return grad


def neuvv_render_backward_adam(tree: Tree, rays: DeviceRays, saved: dict, grad_rgb: torch.Tensor,
                               grad_alpha: torch.Tensor | None, grad: torch.Tensor, touched: torch.Tensor, lr: float,
                               beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, step: int = 1,
                               t: float = 0.0, t_stop: float = 1e-4, act: str = "sigmoid",
                               kernel: str = "packet") -> None:
    """Adjoint followed by Adam on the touched leaves in one call (fused into
    the per-leaf reduction on the leaf-major path)."""
    rc, sc, op = rays.c(), _outc(saved), _opts(t_stop, act, kernel)
    _check(lib().neuvv_render_backward_adam(tree.handle, ctypes.byref(rc), float(t), ctypes.byref(op),
                                            ctypes.byref(sc), _ptr(grad_rgb.contiguous()),
                                            _ptr(None if grad_alpha is None else grad_alpha.contiguous()), _ptr(grad),
                                            _ptr(touched), float(lr), float(beta1), float(beta2), float(eps),
                                            int(step), _stream()))


def neuvv_compose(trees, transforms, time_offsets, tints, rays: DeviceRays, t: float = 0.0, t_stop: float = 1e-4,
                  act: str = "sigmoid", mode: str = "sorted", out: dict | None = None) -> dict:
    P = len(trees)
    arr = (ctypes.c_void_p * P)(*[tr.handle.value for tr in trees])
    xf = np.ascontiguousarray(np.asarray(transforms, np.float32).reshape(P, 12))
    toff = np.ascontiguousarray(np.asarray(time_offsets, np.float32).reshape(P))
    tint = np.ascontiguousarray(np.asarray(tints, np.float32).reshape(P, 3))
    out = out if out is not None else alloc_out(rays.n)
    rc, oc, op = rays.c(), _outc(out), _opts(t_stop, act, "auto", mode)
    _check(lib().neuvv_compose(arr, xf.ctypes.data, toff.ctypes.data, tint.ctypes.data, P, ctypes.byref(rc), float(t),
                               ctypes.byref(op), ctypes.byref(oc), _stream()))
    return out


def neuvv_compose_noalloc(trees, transforms, time_offsets, tints, rays: DeviceRays, t: float = 0.0,
                          t_stop: float = 1e-4, act: str = "sigmoid", mode: str = "sorted", out: dict | None = None) -> dict:
    """neuvv_compose without any device allocation during the call (the work
    counter is a static array of the library); overlapping calls race."""
    P = len(trees)
    arr = (ctypes.c_void_p * P)(*[tr.handle.value for tr in trees])
    xf = np.ascontiguousarray(np.asarray(transforms, np.float32).reshape(P, 12))
    toff = np.ascontiguousarray(np.asarray(time_offsets, np.float32).reshape(P))
    tint = np.ascontiguousarray(np.asarray(tints, np.float32).reshape(P, 3))
    if out is None:
        dev = f"cuda:{trees[0].info.device}"
        out = {"rgb": torch.empty(rays.n, 3, device=dev), "alpha": torch.empty(rays.n, device=dev),
               "depth": torch.empty(rays.n, device=dev)}
    rc, oc, op = rays.c(), _outc(out), _opts(t_stop, act, "auto", mode)
    _check(lib().neuvv_compose_noalloc(arr, xf.ctypes.data, toff.ctypes.data, tint.ctypes.data, P,
                                       ctypes.byref(rc), float(t), ctypes.byref(op), ctypes.byref(oc), _stream()))
    return out


def neuvv_adam_step(tree: Tree, grad: torch.Tensor, touched: torch.Tensor, lr: float, beta1: float = 0.9,
                    beta2: float = 0.999, eps: float = 1e-8, step: int = 1) -> None:
    _check(lib().neuvv_adam_step(tree.handle, _ptr(grad), _ptr(touched), lr, beta1, beta2, eps, int(step), _stream()))


def neuvv_mse_grad(rgb: torch.Tensor, target: torch.Tensor, scale: float = 1.0, grad: torch.Tensor | None = None,
                   loss: torch.Tensor | None = None):
    n = rgb.shape[0]
    grad = grad if grad is not None else torch.empty_like(rgb)
    _check(lib().neuvv_mse_grad(_ptr(rgb.contiguous()), _ptr(target.contiguous()), n, scale, _ptr(grad), _ptr(loss),
                                _stream()))
    return grad


def neuvv_trace(tree: Tree, rays: DeviceRays, max_out: int = 64) -> dict:
    n = rays.n
    leaf = torch.empty(n, max_out, device="cuda", dtype=torch.int32)
    t0 = torch.empty(n, max_out, device="cuda")
    t1 = torch.empty(n, max_out, device="cuda")
    count = torch.empty(n, device="cuda", dtype=torch.int32)
    rc = rays.c()
    _check(lib().neuvv_trace(tree.handle, ctypes.byref(rc), max_out, _ptr(leaf), _ptr(t0), _ptr(t1), _ptr(count),
                             _stream()))
    return {"leaf": leaf, "t0": t0, "t1": t1, "count": count}


def neuvv_log_read(saved: dict, n: int, max_out: int = 64) -> dict:
    """The (leaf, chord) lists the packet forward logged in saved["log"], per
    ray, with count = -1 for rays whose packet is not in the log."""
    dev = saved["nseg"].device
    leaf = torch.empty(n, max_out, device=dev, dtype=torch.int32)
    chord = torch.empty(n, max_out, device=dev)
    count = torch.empty(n, device=dev, dtype=torch.int32)
    sc = _outc(saved)
    _check(lib().neuvv_log_read(ctypes.byref(sc), int(n), int(max_out), _ptr(leaf), _ptr(chord), _ptr(count),
                                _stream()))
    return {"leaf": leaf, "chord": chord, "count": count}


def neuvv_autotune(tree: Tree, rays: DeviceRays, t: float = 0.0) -> float:
    ms = ctypes.c_float()
    rc = rays.c()
    _check(lib().neuvv_autotune(tree.handle, ctypes.byref(rc), float(t), ctypes.byref(ms), _stream()))
    tree.refresh_info()
    return float(ms.value)


def neuvv_autotune_report(tree: Tree) -> tuple:
    """(candidates as dicts in timing order, whether the tree's last
    neuvv_autotune reused a kept choice)."""
    n, cached = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().neuvv_autotune_report(tree.handle, None, 0, ctypes.byref(n), None))
    buf = (TuneEntryC * max(n.value, 1))()
    _check(lib().neuvv_autotune_report(tree.handle, buf, n.value, ctypes.byref(n), ctypes.byref(cached)))
    rows = [{"block": e.block, "queue": e.queue, "ready": e.ready, "order": e.order, "ms": e.ms}
            for e in buf[:n.value]]
    return rows, bool(cached.value)


def neuvv_autotune_tiles(tree: Tree, cams, times) -> int:
    """The fastest pixel tile (TILES_*) of camera packets for this tree, timed
    on the rays of the given cameras (at most 32); stored in the tree."""
    cams, times = list(cams), [float(x) for x in times]
    arr = (LightC * len(cams))(*[light_of(c) for c in cams])
    ts = (ctypes.c_float * len(cams))(*times)
    best, ms = ctypes.c_int32(), ctypes.c_float()
    _check(lib().neuvv_autotune_tiles(tree.handle, arr, ts, len(cams), ctypes.byref(best), ctypes.byref(ms), _stream()))
    tree.refresh_info()
    return int(best.value)


def neuvv_autotune_clear_cache() -> None:
    _check(lib().neuvv_autotune_clear_cache())


class VOctreeRender(torch.autograd.Function):
    """Differentiable VOctree render: forward = neuvv_render, backward =
    neuvv_render_backward (fused adjoint).  ``coeffs`` holds the coefficients
    to render, FP32 records [n_leaves, rec_stride_f32] in the tree's record
    layout, and receives the gradient.  The forward renders from them: unless
    ``coeffs`` is the tree's own FP32 record buffer (its master copy, or the
    storage of an FP32 tree), they are written into the tree first
    (neuvv_tree_set_records, rounded to the storage type), so an optimiser
    step on ``coeffs`` changes the next render."""

    @staticmethod
    def forward(ctx, coeffs, tree, rays, t, t_stop, act):
        if coeffs.data_ptr() != tree.records_ptr():
            tree.set_records(coeffs.detach())
        out = neuvv_render(tree, rays, t=t, t_stop=t_stop, act=act,
                           out=alloc_out(rays.n, rays.o.device, log_bytes_per_ray=64))
        ctx.tree, ctx.rays, ctx.t, ctx.t_stop, ctx.act = tree, rays, t, t_stop, act
        ctx.log = out["log"]
        ctx.save_for_backward(out["rgb"], out["tau"], out["nseg"])
        ctx.mark_non_differentiable(out["depth"])
        return out["rgb"], out["alpha"], out["depth"]

    @staticmethod
    def backward(ctx, grad_rgb, grad_alpha, grad_depth):
        rgb, tau, nseg = ctx.saved_tensors
        saved = {"rgb": rgb, "tau": tau, "nseg": nseg, "log": ctx.log}
        g = neuvv_render_backward(ctx.tree, ctx.rays, saved, grad_rgb.contiguous(),
                                  None if grad_alpha is None else grad_alpha.contiguous(), t=ctx.t,
                                  t_stop=ctx.t_stop, act=ctx.act)
        return g, None, None, None, None, None


def render_differentiable(coeffs: torch.Tensor, tree: Tree, rays: DeviceRays, t: float = 0.0, t_stop: float = 1e-4,
                          act: str = "sigmoid"):
    return VOctreeRender.apply(coeffs, tree, rays, t, t_stop, act)
