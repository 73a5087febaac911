"""FP64 CPU oracle for VOctree rendering -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (the CUDA library and its
binding) never does, and this package imports nothing from the product: both
take their inputs from the seeded generator.

The arithmetic lives in ``neuvv_oracle.c`` (plain C, double precision); this
module compiles it with gcc and marshals numpy arrays.  Each wrapper names the
passage of the paper that the C function follows.
"""

from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "neuvv_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (host code, no architecture-specific flags)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-pthread",
                               "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Tree(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_int), ("K", ctypes.c_int), ("T", ctypes.c_int), ("degree", ctypes.c_int),
                ("n_nodes", ctypes.c_int64), ("n_leaves", ctypes.c_int64),
                ("child", ctypes.c_void_p), ("w_sigma", ctypes.c_void_p), ("w_gamma", ctypes.c_void_p),
                ("w_hh", ctypes.c_void_p), ("coeff_f64", ctypes.c_int),
                ("A", ctypes.c_void_p), ("B", ctypes.c_void_p),
                ("bmin", ctypes.c_double * 3), ("bmax", ctypes.c_double * 3)]


class _Opts(ctypes.Structure):
    _fields_ = [("t_stop", ctypes.c_double), ("act", ctypes.c_int)]


def configure(L):
    """Declares the argument and result types of a loaded oracle library."""
    d = ctypes.c_double
    p = ctypes.c_void_p
    i64 = ctypes.c_int64
    ci = ctypes.c_int
    L.or_gegenbauer.restype = d
    L.or_gegenbauer.argtypes = [ci, d, d]
    L.or_legendre.restype = d
    L.or_legendre.argtypes = [ci, ci, d]
    L.or_sh_real.restype = d
    L.or_sh_real.argtypes = [ci, ci, p]
    L.or_hh_norm.restype = d
    L.or_hh_norm.argtypes = [ci, ci]
    L.or_hh_radial.restype = d
    L.or_hh_radial.argtypes = [ci, ci, d]
    L.or_hh_radial_dgamma.restype = d
    L.or_hh_radial_dgamma.argtypes = [ci, ci, d]
    L.or_hh.restype = d
    L.or_hh.argtypes = [ci, ci, ci, d, p]
    L.or_hh_all.restype = None
    L.or_hh_all.argtypes = [ci, d, p, p, p]
    L.or_n_hh.restype = ci
    L.or_n_hh.argtypes = [ci]
    L.or_hh_index.restype = ci
    L.or_hh_index.argtypes = [ci, ci, ci]
    L.or_render.restype = None
    L.or_render.argtypes = [p, p, i64, p, p, p, p, p, p, p, p, p, p, ci]
    L.or_trace_batch.restype = None
    L.or_trace_batch.argtypes = [p, i64, p, p, ci, p, p, p, p, p, ci]
    L.or_render_grad.restype = None
    L.or_render_grad.argtypes = [p, p, i64, p, p, p, p, p, p, p, p, ci]
    L.or_compose.restype = None
    L.or_compose.argtypes = [p, p, p, p, ci, ci, p, i64, p, p, p, p, p, p, p, p, p, ci]
    L.or_adam.restype = None
    L.or_adam.argtypes = [i64, ci, p, p, p, p, p, d, d, d, d, ci]
    L.or_round_bf16.restype = None
    L.or_round_bf16.argtypes = [p, p, i64]
    L.or_quantize_fp8.restype = None
    L.or_quantize_fp8.argtypes = [p, i64, ci, p, p]
    L.or_round_e4m3.restype = None
    L.or_round_e4m3.argtypes = [p, p, i64]
    L.or_slice.argtypes = [p, d, p, p]
    L.or_pick.argtypes = [p, p, i64, p, p, p, d, p, ci]
    L.or_render_edit.argtypes = [p, p, p, d, i64, p, p, p, p, p, p, p, p, ci]
    L.or_render_slice.argtypes = [p, p, p, p, i64, p, p, p, p, p, p, p, ci]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = configure(ctypes.CDLL(build()))
    return _lib


def compile_variant(src_text: str, out_path: str):
    """Compiles another version of the oracle source (the mutation tests plant
    mistakes in a copy to check that the pins catch them) and loads it."""
    c_path = out_path + ".c"
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O1", "-std=c99", "-fPIC", "-shared", "-pthread", "-fno-fast-math",
                           "-ffp-contract=off", c_path, "-o", out_path, "-lm"])
    return configure(ctypes.CDLL(out_path))


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1)


class OracleTree:
    """Holds the arrays alive while the C struct points at them.

    Coefficients may be float32 (read exactly as doubles) or float64 (for
    finite differences).  ``tree`` is any object with the generator's VOctree
    attributes (child, w_sigma, w_gamma, w_hh, basis_A, basis_B, ...).
    """

    def __init__(self, tree, w_sigma=None, w_gamma=None, w_hh=None):
        ws = tree.w_sigma if w_sigma is None else w_sigma
        wg = tree.w_gamma if w_gamma is None else w_gamma
        wh = tree.w_hh if w_hh is None else w_hh
        f64 = any(np.asarray(x).dtype == np.float64 for x in (ws, wg, wh))
        dt = np.float64 if f64 else np.float32
        self.child = np.ascontiguousarray(tree.child, np.uint32)
        self.ws = np.ascontiguousarray(ws, dt)
        self.wg = np.ascontiguousarray(wg, dt)
        self.wh = np.ascontiguousarray(wh, dt)
        self.A = np.ascontiguousarray(tree.basis_A, np.float64)
        self.B = np.ascontiguousarray(tree.basis_B, np.float64)
        self.K, self.T, self.degree, self.depth = tree.K, tree.T, tree.hh_degree, tree.depth
        self.n_leaves = int(self.ws.shape[1])
        self.N_h = lib().or_n_hh(self.degree)
        s = _Tree()
        s.depth, s.K, s.T, s.degree = self.depth, self.K, self.T, self.degree
        s.n_nodes, s.n_leaves = self.child.size // 8, self.n_leaves
        s.child, s.w_sigma, s.w_gamma, s.w_hh = (self.child.ctypes.data, self.ws.ctypes.data,
                                                 self.wg.ctypes.data, self.wh.ctypes.data)
        s.coeff_f64 = 1 if f64 else 0
        s.A, s.B = self.A.ctypes.data, self.B.ctypes.data
        for k in range(3):
            s.bmin[k] = tree.aabb_min[k]
            s.bmax[k] = tree.aabb_max[k]
        self.struct = s


def _opts(t_stop: float, act: str) -> _Opts:
    return _Opts(float(t_stop), {"sigmoid": 0, "identity": 1}[act])


def _rays64(rays):
    o = np.ascontiguousarray(rays.origins, np.float64)
    d = np.ascontiguousarray(rays.dirs, np.float64)
    t = np.ascontiguousarray(rays.times, np.float64)
    return o, d, t


def render(tree, rays, t_stop: float = 1e-4, act: str = "sigmoid", nthreads: int | None = None,
           otree: OracleTree | None = None) -> dict:
    """Eq. volume-rendering over the voxels each ray crosses (Sec. 4.3 "Rendering").

    Returns rgb [n,3] (premultiplied, black background), alpha, depth, tau
    (optical depth sum sigma*delta), nseg (composited segments),
    stop_margin (|tau_{i+1} - ln(1/t_stop)| minimum, for near-threshold checks)
    and trace_margin: the traversal's decision margin (reading A8) up to the
    early stop, in finest cells -- the smallest distance along the ray
    between two plane crossings whose order decides which leaves are visited.
    """
    ot = otree or OracleTree(tree)
    o, d, t = _rays64(rays)
    n = t.size
    out = {k: np.zeros(n) for k in ("alpha", "depth", "tau", "stop_margin", "trace_margin")}
    out["rgb"] = np.zeros((n, 3))
    out["nseg"] = np.zeros(n, np.int32)
    op = _opts(t_stop, act)
    lib().or_render(ctypes.byref(ot.struct), ctypes.byref(op), n, _ptr(o), _ptr(d), _ptr(t), _ptr(out["rgb"]),
                    _ptr(out["alpha"]), _ptr(out["depth"]), _ptr(out["tau"]), _ptr(out["nseg"]),
                    _ptr(out["stop_margin"]), _ptr(out["trace_margin"]), nthreads or default_threads())
    return out


def trace(tree, rays, max_out: int = 64, nthreads: int | None = None, otree: OracleTree | None = None) -> dict:
    """Occupied leaves each ray crosses, with entry/exit distances (Sec. 4.3
    "Rendering": voxels on the path and the lengths of the segments inside),
    and each ray's decision margin over its whole length in finest cells
    (reading A8; see ``render``)."""
    ot = otree or OracleTree(tree)
    o, d, _ = _rays64(rays)
    n = o.shape[1]
    leaf = np.full((n, max_out), -1, np.int64)
    t0 = np.zeros((n, max_out))
    t1 = np.zeros((n, max_out))
    cnt = np.zeros(n, np.int32)
    margin = np.zeros(n)
    lib().or_trace_batch(ctypes.byref(ot.struct), n, _ptr(o), _ptr(d), max_out, _ptr(leaf), _ptr(t0), _ptr(t1),
                         _ptr(cnt), _ptr(margin), nthreads or default_threads())
    return {"leaf": leaf, "t0": t0, "t1": t1, "count": cnt, "margin": margin}


def render_grad(tree, rays, grad_rgb, grad_alpha=None, t_stop: float = 1e-4, act: str = "sigmoid",
                nthreads: int | None = None, otree: OracleTree | None = None, out: dict | None = None) -> dict:
    """Analytic gradient of L(C, alpha) w.r.t. (w_sigma, w_gamma, w_hh), given
    dL/dC and dL/dalpha per ray (Sec. 4.3 "Optimization").  Planes as inputs.
    With ``out`` (float64 planes of the returned shapes) the gradient is
    added to those arrays instead of to fresh zeroed ones."""
    ot = otree or OracleTree(tree)
    o, d, t = _rays64(rays)
    n = t.size
    g = np.ascontiguousarray(grad_rgb, np.float64).reshape(n, 3)
    ga = None if grad_alpha is None else np.ascontiguousarray(grad_alpha, np.float64)
    if out is None:
        gs = np.zeros((ot.K, ot.n_leaves))
        gg = np.zeros((ot.K, ot.n_leaves))
        gh = np.zeros((3, ot.N_h, ot.n_leaves))
    else:
        gs, gg, gh = out["w_sigma"], out["w_gamma"], out["w_hh"]
        for a, shape in ((gs, (ot.K, ot.n_leaves)), (gg, (ot.K, ot.n_leaves)), (gh, (3, ot.N_h, ot.n_leaves))):
            assert a.dtype == np.float64 and a.flags.c_contiguous and a.shape == shape
    op = _opts(t_stop, act)
    lib().or_render_grad(ctypes.byref(ot.struct), ctypes.byref(op), n, _ptr(o), _ptr(d), _ptr(t), _ptr(g),
                         None if ga is None else _ptr(ga), _ptr(gs), _ptr(gg), _ptr(gh), nthreads or default_threads())
    return {"w_sigma": gs, "w_gamma": gg, "w_hh": gh}


def slice_at(tree, t: float, otree: OracleTree | None = None) -> dict:
    """Time slice (Sec. 7; caption of the HH-colour figure): at time t each
    leaf's density sigma and spherical-harmonic colour coefficients
    sh[leaf][ch][l^2 + l + m] = sum_{n >= l} w_nlm R_nl(gamma(t))."""
    ot = otree or OracleTree(tree)
    t = min(max(float(t), 0.0), 1.0)
    ny = (ot.degree + 1) ** 2
    sigma = np.zeros(ot.n_leaves)
    sh = np.zeros((ot.n_leaves, 3, ny))
    lib().or_slice(ctypes.byref(ot.struct), t * (ot.T - 1), _ptr(sigma), _ptr(sh))
    return {"sigma": sigma, "sh": sh}


def render_slice(tree, sl: dict, rays, t_stop: float = 1e-4, act: str = "sigmoid", nthreads: int | None = None,
                 otree: OracleTree | None = None) -> dict:
    """Eq. volume-rendering of a time slice: the tree's voxels and chords, the
    slice's density, colour act(sum_lm s_lm Y_lm(d)).  Ray times are unused."""
    ot = otree or OracleTree(tree)
    o, d, _ = _rays64(rays)
    n = o.shape[1]
    sigma = np.ascontiguousarray(sl["sigma"], np.float64)
    sh = np.ascontiguousarray(sl["sh"], np.float64)
    out = {k: np.zeros(n) for k in ("alpha", "depth", "tau")}
    out["rgb"] = np.zeros((n, 3))
    out["nseg"] = np.zeros(n, np.int32)
    op = _opts(t_stop, act)
    lib().or_render_slice(ctypes.byref(ot.struct), ctypes.byref(op), _ptr(sigma), _ptr(sh), n, _ptr(o), _ptr(d),
                          _ptr(out["rgb"]), _ptr(out["alpha"]), _ptr(out["depth"]), _ptr(out["tau"]),
                          _ptr(out["nseg"]), nthreads or default_threads())
    return out


def grad_loss(rgb, target, ray_of_pixel, width: int, height: int, lam: float) -> dict:
    """The image-gradient regulariser L_grad (Sec. 4.3 "Optimization", the
    equation after the RGB loss) and its gradient with respect to the
    rendered colours: lam * sum over views and pixels of ||grad |I - I_hat|||^2,
    the image gradient as forward differences between horizontally and
    vertically adjacent pixels (a pair counts when both pixels have a ray),
    summed over the three channels.  ray_of_pixel [n_views, height, width]
    holds the ray of each pixel or -1.  Returns loss (float) and grad [n, 3]
    (d|I - I_hat|/d I_hat = sign(I_hat - I), 0 where they are equal)."""
    rgb = np.asarray(rgb, np.float64)
    tgt = np.asarray(target, np.float64)
    m = np.asarray(ray_of_pixel, np.int64).reshape(-1, height, width)
    E = np.abs(tgt - rgb)                                   # [n, 3]
    loss = 0.0
    dE = np.zeros_like(E)
    for a, b in ((m[:, :, :-1], m[:, :, 1:]), (m[:, :-1, :], m[:, 1:, :])):   # (left, right), (up, down)
        ok = (a >= 0) & (b >= 0)
        ra, rb = a[ok], b[ok]
        D = E[rb] - E[ra]                                    # forward difference, per channel
        loss += float((D * D).sum())
        np.add.at(dE, rb, 2.0 * D)
        np.add.at(dE, ra, -2.0 * D)
    return {"loss": lam * loss, "grad": lam * np.sign(rgb - tgt) * dE}


def pick(tree, rays, threshold: float = 0.99, t_stop: float = 1e-4, nthreads: int | None = None,
         otree: OracleTree | None = None) -> np.ndarray:
    """Terminating voxel of each ray (Sec. 5 "Appearance editing": the voxel
    where the accumulated alpha of the NeuVV render first reaches the
    threshold, 0.99 in the paper); -1 where it never does."""
    ot = otree or OracleTree(tree)
    o, d, t = _rays64(rays)
    n = t.size
    leaf = np.full(n, -1, np.int64)
    op = _opts(t_stop, "sigmoid")
    lib().or_pick(ctypes.byref(ot.struct), ctypes.byref(op), n, _ptr(o), _ptr(d), _ptr(t), float(threshold),
                  _ptr(leaf), nthreads or default_threads())
    return leaf


def paint(n_leaves: int, leaves, colors, sigma_d: float, t_d: float, edits=None) -> np.ndarray:
    """Assigns target colours to the picked voxels (Sec. 5 "Appearance
    editing"): each leaf picked by at least one ray gets the mean colour of
    those rays, with target density sigma_d and time t_d; other leaves keep
    their edit (initially inactive: t_d = 2).  Returns edits [n_leaves, 5]."""
    e = np.array(edits, np.float64) if edits is not None else np.tile([0.0, 0.0, 0.0, -1.0, 2.0], (n_leaves, 1))
    leaves = np.asarray(leaves, np.int64)
    ok = leaves >= 0
    s = np.zeros((n_leaves, 3))
    cnt = np.zeros(n_leaves)
    np.add.at(s, leaves[ok], np.asarray(colors, np.float64)[ok])
    np.add.at(cnt, leaves[ok], 1.0)
    hit = cnt > 0
    e[hit, :3] = s[hit] / cnt[hit, None]
    e[hit, 3] = sigma_d
    e[hit, 4] = t_d
    return e


def render_edit(tree, rays, edits, beta: float = 1.0, t_stop: float = 1e-4, act: str = "sigmoid",
                nthreads: int | None = None, otree: OracleTree | None = None) -> dict:
    """Eq. volume-rendering with per-voxel edits [n_leaves, 5] = (c_d, sigma_d,
    t_d): active at ray time t >= t_d, density sigma_d when sigma_d >= 0,
    colour (1 - beta) c + beta c_d."""
    ot = otree or OracleTree(tree)
    o, d, t = _rays64(rays)
    n = t.size
    ed = np.ascontiguousarray(edits, np.float64)
    out = {k: np.zeros(n) for k in ("alpha", "depth", "tau")}
    out["rgb"] = np.zeros((n, 3))
    out["nseg"] = np.zeros(n, np.int32)
    op = _opts(t_stop, act)
    lib().or_render_edit(ctypes.byref(ot.struct), ctypes.byref(op), _ptr(ed), float(beta), n, _ptr(o), _ptr(d),
                         _ptr(t), _ptr(out["rgb"]), _ptr(out["alpha"]), _ptr(out["depth"]), _ptr(out["tau"]),
                         _ptr(out["nseg"]), nthreads or default_threads())
    return out


def camera_rays(cam, t: float, tiled=True) -> dict:
    """Pinhole camera rays through pixel centres (Sec. 4.3 "Rendering": one
    ray per pixel of a view).  cam: eye, orthonormal right/up/forward,
    fov_y_deg, width, height.  Pixel (px, py) looks along
    forward + sx right + sy up with sx = (2 (px + 1/2) / W - 1) tan(fov_y / 2) W / H
    and sy = (1 - 2 (py + 1/2) / H) tan(fov_y / 2), normalised.  The rays list
    the pixels row-major, or (tiled) tile by tile: tw x th tiles (tiled =
    True: 8 x 4; or a (tw, th) pair) in row-major order of the tiles, the
    pixels of each tile row-major, the tiles at the right and bottom edges
    cut to the image.  Returns origins and dirs [3, n], times [n] and the
    row-major pixel of each ray."""
    W, H = int(cam.width), int(cam.height)
    if tiled is not False and tiled is not None:
        tw, th_ = (8, 4) if tiled is True else (int(tiled[0]), int(tiled[1]))
        parts = []
        for y0 in range(0, H, th_):
            ys = np.arange(y0, min(y0 + th_, H))
            for x0 in range(0, W, tw):
                xs = np.arange(x0, min(x0 + tw, W))
                parts.append((ys[:, None] * W + xs[None, :]).ravel())
        pix = np.concatenate(parts)
    else:
        pix = np.arange(W * H)
    py, px = pix // W, pix % W
    th = math.tan(math.radians(float(cam.fov_y_deg)) / 2.0)
    sx = (2.0 * (px + 0.5) / W - 1.0) * th * (W / H)
    sy = (1.0 - 2.0 * (py + 0.5) / H) * th
    f, r, u = (np.asarray(x, np.float64) for x in (cam.forward, cam.right, cam.up))
    d = f[:, None] + r[:, None] * sx[None, :] + u[:, None] * sy[None, :]
    d = d / np.linalg.norm(d, axis=0, keepdims=True)
    o = np.repeat(np.asarray(cam.eye, np.float64)[:, None], pix.size, axis=1)
    return {"origins": o, "dirs": d, "times": np.full(pix.size, float(t)), "pixel": pix}


def gaussian_blur(img, sigma: float):
    """The low-pass filter of the shadow map (Sec. 5 "Spotlight Lighting":
    shadows rendered at low resolution and Gaussian-filtered against Moire
    patterns).  img [n_images, height, width]; weights exp(-k^2 / (2 sigma^2))
    for |k| <= floor(3 sigma + 0.5), normalised, applied along x then y with
    the edge pixel repeated beyond the border."""
    img = np.asarray(img, np.float64)
    r = int(3.0 * sigma + 0.5)
    k = np.arange(-r, r + 1, dtype=np.float64)
    w = np.exp(-k * k / (2.0 * sigma * sigma))
    w /= w.sum()
    out = img
    for axis in (2, 1):
        n = out.shape[axis]
        acc = np.zeros_like(out)
        for wi, ki in zip(w, k):
            idx = np.clip(np.arange(n) + int(ki), 0, n - 1)
            acc += wi * np.take(out, idx, axis=axis)
        out = acc
    return out


def spotlight(origins, dirs, rgb, alpha, depth, light, light_alpha, ground_z: float, albedo, r_ref: float):
    """Spotlight shadow and distance falloff (Sec. 5 "Spotlight Lighting").
    Per viewer ray (origins, dirs [3, n]) with its render (premultiplied rgb
    [n, 3], alpha, depth along the unit direction):
      f(r) = (r_ref / r)^2                       distance falloff from the light
      X = o + depth d;  C_lit = C f(|X - L|)     (C unchanged where depth is inf)
      ground point P = o + s d on z = ground_z (s > 0); P projected into the
      light's camera (the pinhole of `light`, pixel centres at integer + 0.5)
      samples the filtered light alpha map bilinearly (0 outside it);
      G = albedo (1 - alpha_light(P)) f(|P - L|)
      out = C_lit + (1 - alpha) G (C_lit where the ray misses the ground).
    light: an inputs.Camera at the light position; light_alpha [H_l, W_l]."""
    o = np.asarray(origins, np.float64)
    d = np.asarray(dirs, np.float64)
    d = d / np.linalg.norm(d, axis=0, keepdims=True)
    C = np.asarray(rgb, np.float64)
    A = np.asarray(alpha, np.float64)
    D = np.asarray(depth, np.float64)
    L = np.asarray(light.eye, np.float64)
    Al = np.asarray(light_alpha, np.float64)
    Hl, Wl = Al.shape
    n = C.shape[0]
    fall = lambda P: r_ref * r_ref / np.sum((P - L[:, None]) ** 2, axis=0)
    out = C.copy()
    fin = np.isfinite(D)
    X = o[:, fin] + D[fin] * d[:, fin]
    out[fin] = C[fin] * fall(X)[:, None]
    with np.errstate(divide="ignore", invalid="ignore"):
        s = (ground_z - o[2]) / d[2]
    hit = np.isfinite(s) & (s > 0)
    P = o[:, hit] + s[hit] * d[:, hit]
    v = P - L[:, None]
    zc = light.forward @ v
    th = math.tan(math.radians(light.fov_y_deg) / 2.0)
    sx = (light.right @ v) / zc
    sy = (light.up @ v) / zc
    px = (sx / (th * Wl / Hl) + 1.0) * Wl / 2.0 - 0.5      # pixel coordinate, centres at integers
    py = (1.0 - sy / th) * Hl / 2.0 - 0.5
    x0 = np.floor(px).astype(np.int64)
    y0 = np.floor(py).astype(np.int64)
    fx, fy = px - x0, py - y0
    def tex(yy, xx):
        ok = (zc > 0) & (xx >= 0) & (xx < Wl) & (yy >= 0) & (yy < Hl)
        val = np.zeros(xx.shape)
        val[ok] = Al[yy[ok], xx[ok]]
        return val
    al = ((1 - fx) * (1 - fy) * tex(y0, x0) + fx * (1 - fy) * tex(y0, x0 + 1)
          + (1 - fx) * fy * tex(y0 + 1, x0) + fx * fy * tex(y0 + 1, x0 + 1))
    G = np.asarray(albedo, np.float64)[None, :] * ((1.0 - al) * fall(P))[:, None]
    out[hit] += (1.0 - A[hit])[:, None] * G
    return out


def compose(trees, transforms, time_offsets, tints, rays, mode: str = "sorted", t_stop: float = 1e-4,
            act: str = "sigmoid", nthreads: int | None = None) -> dict:
    """Eq. st_composite_affine per primitive, then depth-aware blending
    (Algorithm 1; mode 'sorted' = stable depth sort + premultiplied over,
    'alg1' = Algorithm 1 literally on premultiplied layers).

    Besides rgb, alpha, depth and the early-stop margin, reports per pixel
    trace_margin (the smallest decision margin of the layers' traversals, in
    finest cells of each layer's tree) and depth_margin (the smallest gap
    between two layers' finite depths: below the depths' rounding error the
    blending order is not determined)."""
    ots = [t if isinstance(t, OracleTree) else OracleTree(t) for t in trees]
    P = len(ots)
    arr = (ctypes.c_void_p * P)(*[ctypes.addressof(x.struct) for x in ots])
    xf = np.ascontiguousarray(np.asarray(transforms, np.float64).reshape(P, 12))
    toff = np.ascontiguousarray(time_offsets, np.float64)
    tint = np.ascontiguousarray(np.asarray(tints, np.float64).reshape(P, 3))
    o, d, t = _rays64(rays)
    n = t.size
    rgb = np.zeros((n, 3))
    alpha = np.zeros(n)
    depth = np.zeros(n)
    margin = np.zeros(n)
    tmargin = np.zeros(n)
    dmargin = np.zeros(n)
    op = _opts(t_stop, act)
    lib().or_compose(arr, _ptr(xf), _ptr(toff), _ptr(tint), P, {"sorted": 0, "alg1": 1}[mode], ctypes.byref(op), n,
                     _ptr(o), _ptr(d), _ptr(t), _ptr(rgb), _ptr(alpha), _ptr(depth), _ptr(margin), _ptr(tmargin),
                     _ptr(dmargin), nthreads or default_threads())
    return {"rgb": rgb, "alpha": alpha, "depth": depth, "stop_margin": margin, "trace_margin": tmargin,
            "depth_margin": dmargin}


def adam(w, m, v, g, touched, lr, b1, b2, eps, step):
    """Sparse Adam, in place on float64 [n_leaves, rec] arrays."""
    for a in (w, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = np.ascontiguousarray(g, np.float64)
    tch = np.ascontiguousarray(touched, np.uint8)
    lib().or_adam(w.shape[0], w.shape[1], _ptr(w), _ptr(m), _ptr(v), _ptr(g), _ptr(tch), lr, b1, b2, eps, step)


def round_bf16(x: np.ndarray) -> np.ndarray:
    """float32 -> bfloat16 (round to nearest even) -> float32."""
    x = np.ascontiguousarray(x, np.float32)
    out = np.empty_like(x)
    lib().or_round_bf16(_ptr(x), _ptr(out), x.size)
    return out


def round_e4m3(x: np.ndarray) -> np.ndarray:
    """The nearest FP8 E4M3 value of each entry (ties to even, saturating at 448)."""
    x = np.ascontiguousarray(x, np.float64)
    out = np.empty_like(x)
    lib().or_round_e4m3(_ptr(x), _ptr(out), x.size)
    return out


def quantize_fp8_groups(w: np.ndarray):
    """[n_groups, len] float32 -> (dequantised float64 [n_groups, len], scales
    [n_groups]): each group scaled by the smallest power of two that brings its
    largest magnitude to <= 448, rounded to E4M3, scaled back."""
    w = np.ascontiguousarray(w, np.float32)
    out = np.empty(w.shape, np.float64)
    scale = np.empty(w.shape[0], np.float64)
    lib().or_quantize_fp8(_ptr(w), w.shape[0], w.shape[1], _ptr(out), _ptr(scale))
    return out, scale


def quantize_fp8_tree(tree):
    """The tree as FP8 storage holds it: per leaf, one scale for its w_sigma,
    one for its w_gamma, one for its w_hh (all three channels).  Returns the
    tree with dequantised coefficients and the scales [n_leaves, 3]."""
    L = tree.n_leaves
    ws, s_s = quantize_fp8_groups(tree.w_sigma.reshape(tree.K, L).T)
    wg, s_g = quantize_fp8_groups(tree.w_gamma.reshape(tree.K, L).T)
    wh, s_h = quantize_fp8_groups(tree.w_hh.reshape(-1, L).T)
    out = tree.with_coeffs(ws.T.astype(np.float32), wg.T.astype(np.float32),
                           wh.T.reshape(tree.w_hh.shape).astype(np.float32))
    return out, np.stack([s_s, s_g, s_h], axis=1)


# -- point evaluations for the pins -------------------------------------------

def hh_all(degree: int, gamma: float, d) -> np.ndarray:
    d = np.ascontiguousarray(d, np.float64)
    out = np.zeros(lib().or_n_hh(degree))
    lib().or_hh_all(degree, gamma, _ptr(d), _ptr(out), None)
    return out


def hh_all_dgamma(degree: int, gamma: float, d) -> np.ndarray:
    d = np.ascontiguousarray(d, np.float64)
    out = np.zeros(lib().or_n_hh(degree))
    dout = np.zeros_like(out)
    lib().or_hh_all(degree, gamma, _ptr(d), _ptr(out), _ptr(dout))
    return dout


def sh_real(l: int, m: int, d) -> float:
    d = np.ascontiguousarray(d, np.float64)
    return lib().or_sh_real(l, m, _ptr(d))


def gegenbauer(k: int, lam: float, x: float) -> float:
    return lib().or_gegenbauer(k, lam, x)


def legendre(l: int, m: int, x: float) -> float:
    return lib().or_legendre(l, m, x)


def hh_index(n: int, l: int, m: int) -> int:
    return lib().or_hh_index(n, l, m)
