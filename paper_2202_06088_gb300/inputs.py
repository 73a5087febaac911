"""Seeded synthetic inputs for VOctree rendering.

This module generates the *inputs* of the renderer and nothing else: the sparse
octree structure (Sec. 4.3, "Initialization": large empty nodes, fine occupied
voxels), the per-leaf coefficient vectors w^sigma, w^gamma, w^HH (Sec. 4.3,
"we store coefficients ... into an octree-based representation"), the shared
temporal bases A and B (Eq. project-sigma, Eq. project-gamma), pinhole cameras and
rays.  It holds none of the method's arithmetic: no density, hyper-angle,
harmonic, compositing or blending formula appears here.  Both the FP64 oracle
(through the tests and the bench) and the CUDA path consume what it returns.

Tree encoding shared by both sides (it is the input format of the C ABI):
  * nodes are numbered breadth first (root = 0, then level 1, ...), Morton order
    inside a level, so the top levels form a contiguous prefix;
  * ``child[node * 8 + c]`` with ``c = 4 * xbit + 2 * ybit + zbit`` holds
    ``EMPTY`` (0xFFFFFFFF), ``LEAF_BIT | leaf_id`` for an occupied leaf, or the
    index of an internal child node;
  * leaf ids follow the Morton order of the leaves' finest-level corners, so
    spatially close leaves are close in memory.
Coefficient planes are float32, ``w_sigma[K][n_leaves]``, ``w_gamma[K][n_leaves]``
and ``w_hh[3][N_h][n_leaves]`` (channel, then harmonic index
``idx(n, l, m) = n(n+1)(2n+1)/6 + l^2 + l + m``).
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

EMPTY = np.uint32(0xFFFFFFFF)
LEAF_BIT = np.uint32(0x80000000)

# child slot c = 4*x + 2*y + z  ->  offset (x, y, z)
CHILD_OFFSETS = np.array([[(c >> 2) & 1, (c >> 1) & 1, c & 1] for c in range(8)], dtype=np.int64)


def n_hh(degree: int) -> int:
    """Number of 4D harmonics with n <= degree: sum (n+1)^2 (14 for 2, 30 for 3)."""
    return sum((n + 1) ** 2 for n in range(degree + 1))


# ----------------------------------------------------------------------------
# Morton codes and tree assembly
# ----------------------------------------------------------------------------

def _spread3(x: np.ndarray) -> np.ndarray:
    x = x.astype(np.int64) & 0x1FFFFF
    x = (x | (x << 32)) & 0x1F00000000FFFF
    x = (x | (x << 16)) & 0x1F0000FF0000FF
    x = (x | (x << 8)) & 0x100F00F00F00F00F
    x = (x | (x << 4)) & 0x10C30C30C30C30C3
    x = (x | (x << 2)) & 0x1249249249249249
    return x


def morton3(coords: np.ndarray) -> np.ndarray:
    """Interleave (x, y, z) bits with x most significant in each triple."""
    c = np.asarray(coords, dtype=np.int64)
    return (_spread3(c[:, 0]) << 2) | (_spread3(c[:, 1]) << 1) | _spread3(c[:, 2])


@dataclasses.dataclass
class TreeStructure:
    depth: int
    child: np.ndarray        # uint32 [n_nodes * 8]
    leaf_level: np.ndarray   # int32 [n_leaves]
    leaf_coords: np.ndarray  # int32 [n_leaves, 3], at the leaf's own level

    @property
    def n_nodes(self) -> int:
        return self.child.size // 8

    @property
    def n_leaves(self) -> int:
        return self.leaf_level.size


def build_tree(depth: int, leaf_level: np.ndarray, leaf_coords: np.ndarray) -> TreeStructure:
    """Assemble the child table from a set of non-overlapping occupied cells.

    ``leaf_level[i]`` in [1, depth] and ``leaf_coords[i]`` (integer cell index at
    that level) describe occupied leaf i.  Every strict ancestor of a leaf becomes
    an internal node; every other cell is empty.
    """
    if depth < 1 or depth > 20:
        raise ValueError("depth must be in [1, 20]")
    leaf_level = np.asarray(leaf_level, dtype=np.int64)
    leaf_coords = np.asarray(leaf_coords, dtype=np.int64).reshape(-1, 3)
    if leaf_level.size and (leaf_level.min() < 1 or leaf_level.max() > depth):
        raise ValueError("leaf levels must lie in [1, depth]")
    # leaf ids: Morton order of the finest-level corner, ties (impossible for
    # non-overlapping cells) broken by level
    fine = leaf_coords << (depth - leaf_level)[:, None]
    order = np.lexsort((leaf_level, morton3(fine)))
    leaf_level = leaf_level[order]
    leaf_coords = leaf_coords[order]

    node_keys = []   # per level: sorted Morton keys of internal nodes
    for L in range(depth):
        sel = leaf_level > L
        anc = leaf_coords[sel] >> (leaf_level[sel] - L)[:, None]
        keys = np.unique(morton3(anc)) if anc.size else np.zeros(0, np.int64)
        if L == 0:
            keys = np.zeros(1, np.int64)  # the root always exists
        node_keys.append(keys)
    base = np.cumsum([0] + [k.size for k in node_keys])
    n_nodes = int(base[-1])

    leaf_keys = []   # per level: (sorted keys, leaf ids)
    leaf_ids = np.arange(leaf_level.size, dtype=np.int64)
    for L in range(depth + 1):
        sel = leaf_level == L
        k = morton3(leaf_coords[sel])
        o = np.argsort(k, kind="stable")
        leaf_keys.append((k[o], leaf_ids[sel][o]))

    child = np.full(n_nodes * 8, EMPTY, dtype=np.uint32)
    for L in range(depth):
        keys = node_keys[L]
        for c in range(8):
            # Morton key of child c of node with key k is (k << 3) | c
            ck = (keys << 3) | c
            slot = (base[L] + np.arange(keys.size)) * 8 + c
            if L + 1 < depth:
                nk = node_keys[L + 1]
                if nk.size:
                    pos_c = np.minimum(np.searchsorted(nk, ck), nk.size - 1)
                    hit = nk[pos_c] == ck
                    child[slot[hit]] = (base[L + 1] + pos_c[hit]).astype(np.uint32)
            lk, lid = leaf_keys[L + 1]
            if lk.size:
                pos = np.searchsorted(lk, ck)
                pos_c = np.minimum(pos, lk.size - 1)
                hit = lk[pos_c] == ck
                if np.any(child[slot[hit]] != EMPTY):
                    raise ValueError("a leaf overlaps an internal node")
                child[slot[hit]] = lid[pos_c[hit]].astype(np.uint32) | LEAF_BIT
    return TreeStructure(depth, child, leaf_level.astype(np.int32), leaf_coords.astype(np.int32))


def random_mixed_tree(depth: int, seed: int, p_leaf: float = 0.3, p_empty: float = 0.3) -> TreeStructure:
    """Random tree with occupied leaves at several levels (traversal tests)."""
    rng = np.random.default_rng(seed)
    levels, coords = [], []
    frontier = [(0, (0, 0, 0))]
    while frontier:
        L, c = frontier.pop()
        for off in CHILD_OFFSETS:
            cc = (2 * c[0] + int(off[0]), 2 * c[1] + int(off[1]), 2 * c[2] + int(off[2]))
            r = rng.random()
            if L + 1 == depth:
                if r < 0.5:
                    levels.append(L + 1)
                    coords.append(cc)
            elif r < p_leaf:
                levels.append(L + 1)
                coords.append(cc)
            elif r < p_leaf + p_empty:
                pass
            else:
                frontier.append((L + 1, cc))
    if not levels:
        levels, coords = [depth], [(0, 0, 0)]
    return build_tree(depth, np.array(levels), np.array(coords))


def full_tree(depth: int) -> TreeStructure:
    """Every finest-level cell occupied."""
    n = 1 << depth
    g = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 3)
    return build_tree(depth, np.full(g.shape[0], depth), g)


# ----------------------------------------------------------------------------
# Occupancy from seeded implicit shapes (replaces the paper's density-threshold
# initialisation from a trained network, which needs captured data)
# ----------------------------------------------------------------------------

def _random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


@dataclasses.dataclass
class Shape:
    centers: np.ndarray   # [E, 3]
    axes: np.ndarray      # [E, 3]
    rots: np.ndarray      # [E, 3, 3], columns = local axes in world
    noise_amp: float = 0.0
    noise_w: np.ndarray | None = None     # [M, 3]
    noise_phase: np.ndarray | None = None
    noise_a: np.ndarray | None = None

    def field(self, p: np.ndarray) -> np.ndarray:
        """Approximate signed distance to the union of ellipsoids (Lipschitz <= 1),
        displaced by smooth noise."""
        f = np.full(p.shape[0], np.inf)
        for c, a, R in zip(self.centers, self.axes, self.rots):
            loc = (p - c) @ R
            r = np.sqrt(((loc / a) ** 2).sum(1))
            f = np.minimum(f, (r - 1.0) * a.min())
        if self.noise_amp:
            f = f + self.noise_amp * self._noise(p)
        return f

    def _noise(self, p: np.ndarray) -> np.ndarray:
        s = np.zeros(p.shape[0])
        for w, ph, a in zip(self.noise_w, self.noise_phase, self.noise_a):
            s += a * np.sin(p @ w + ph)
        return s / self.noise_a.sum()

    def lipschitz(self) -> float:
        lip = 1.0
        if self.noise_amp:
            lip += self.noise_amp * float((self.noise_a * np.linalg.norm(self.noise_w, axis=1)).sum() / self.noise_a.sum())
        return lip


def make_shape(rng: np.random.Generator, n_ell: int, c_lo: float, c_hi: float, a_lo: float, a_hi: float,
               noise_amp: float = 0.0, n_waves: int = 8) -> Shape:
    centers = rng.uniform(c_lo, c_hi, (n_ell, 3))
    axes = rng.uniform(a_lo, a_hi, (n_ell, 3))
    rots = _random_rotations(rng, n_ell)
    sh = Shape(centers, axes, rots, noise_amp)
    if noise_amp:
        d = rng.standard_normal((n_waves, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        sh.noise_w = d * rng.uniform(8.0, 24.0, (n_waves, 1))
        sh.noise_phase = rng.uniform(0, 2 * np.pi, n_waves)
        sh.noise_a = rng.uniform(0.5, 1.0, n_waves)
    return sh


def occupied_cells(shape: Shape, depth: int, mode: str, h: float = 0.0, axis_scale: float = 1.0,
                   chunk: int = 1 << 22) -> np.ndarray:
    """Finest-level cells of the unit cube whose centre is occupied.

    mode 'solid': inside the union (field <= 0); mode 'shell': |field| < h.
    Nodes are refined only where the Lipschitz bound allows an occupied centre.
    """
    sh = dataclasses.replace(shape, axes=shape.axes * axis_scale)
    lip = sh.lipschitz()
    cand = np.zeros((1, 3), np.int64)
    for L in range(1, depth + 1):
        cand = (cand[:, None, :] * 2 + CHILD_OFFSETS[None]).reshape(-1, 3)
        size = 1.0 / (1 << L)
        # finest centres inside this node lie within r of its centre
        r = 0.5 * math.sqrt(3.0) * (size - 1.0 / (1 << depth))
        keep = np.zeros(cand.shape[0], bool)
        for s in range(0, cand.shape[0], chunk):
            p = (cand[s:s + chunk] + 0.5) * size
            f = sh.field(p)
            if mode == "solid":
                keep[s:s + chunk] = f - lip * r <= 0.0
            else:
                keep[s:s + chunk] = np.abs(f) - lip * r < h
        cand = cand[keep]
    return cand.astype(np.int32)


# ----------------------------------------------------------------------------
# Coefficients and temporal bases
# ----------------------------------------------------------------------------

def smooth_curves(rng: np.random.Generator, T: int, K: int) -> np.ndarray:
    """K smooth curves over T frames, each a sum of 3 sinusoids with period >= T/2,
    min-max normalised to [0, 1].  Returns [T, K] float64."""
    f = np.arange(T, dtype=np.float64)
    out = np.zeros((T, K))
    for k in range(K):
        for _ in range(3):
            period = rng.uniform(T / 2.0, 2.0 * T)
            out[:, k] += rng.uniform(0.5, 1.0) * np.sin(2 * np.pi * f / period + rng.uniform(0, 2 * np.pi))
        lo, hi = out[:, k].min(), out[:, k].max()
        out[:, k] = (out[:, k] - lo) / (hi - lo) if hi > lo else 0.5
    return out


@dataclasses.dataclass
class VOctree:
    """Host copy of a VOctree: structure + coefficient planes + shared bases."""
    structure: TreeStructure
    K: int
    T: int
    hh_degree: int
    w_sigma: np.ndarray   # float32 [K, L]
    w_gamma: np.ndarray   # float32 [K, L]
    w_hh: np.ndarray      # float32 [3, N_h, L]
    basis_A: np.ndarray   # float32 [T, K]
    basis_B: np.ndarray   # float32 [T, K]
    aabb_min: tuple = (0.0, 0.0, 0.0)
    aabb_max: tuple = (1.0, 1.0, 1.0)
    info: dict = dataclasses.field(default_factory=dict)

    @property
    def depth(self) -> int:
        return self.structure.depth

    @property
    def child(self) -> np.ndarray:
        return self.structure.child

    @property
    def n_leaves(self) -> int:
        return self.structure.n_leaves

    @property
    def n_nodes(self) -> int:
        return self.structure.n_nodes

    @property
    def N_h(self) -> int:
        return n_hh(self.hh_degree)

    def with_coeffs(self, w_sigma=None, w_gamma=None, w_hh=None) -> "VOctree":
        return dataclasses.replace(
            self,
            w_sigma=self.w_sigma if w_sigma is None else np.ascontiguousarray(w_sigma, np.float32),
            w_gamma=self.w_gamma if w_gamma is None else np.ascontiguousarray(w_gamma, np.float32),
            w_hh=self.w_hh if w_hh is None else np.ascontiguousarray(w_hh, np.float32))


# E[softplus(Z)], Z ~ N(0, 1): used only to scale the density basis so that the
# mean leaf density is about the target
_E_SOFTPLUS_STD_NORMAL = 0.8065786


def make_coefficients(rng: np.random.Generator, structure: TreeStructure, K: int, T: int, hh_degree: int,
                      mean_sigma: float = 30.0, hh_std: float = 0.3, signed_density: bool = False,
                      aabb_min=(0.0, 0.0, 0.0), aabb_max=(1.0, 1.0, 1.0)) -> VOctree:
    L = structure.n_leaves
    Nh = n_hh(hh_degree)
    z = rng.standard_normal((K, L), dtype=np.float32)
    w_sigma = np.logaddexp(np.float32(0.0), z).astype(np.float32)   # softplus
    w_gamma = rng.standard_normal((K, L), dtype=np.float32)
    w_hh = (hh_std * rng.standard_normal((3, Nh, L), dtype=np.float32)).astype(np.float32)
    curves_a = smooth_curves(rng, T, K)
    if signed_density:
        curves_a = 1.5 * curves_a - 0.5     # some frames push the pre-activation below 0
    scale = mean_sigma / (K * max(float(np.abs(curves_a).mean()), 1e-6) * _E_SOFTPLUS_STD_NORMAL)
    basis_A = (scale * curves_a).astype(np.float32)
    basis_B = ((2.0 * smooth_curves(rng, T, K) - 1.0) * (2.0 / math.sqrt(K))).astype(np.float32)
    return VOctree(structure, K, T, hh_degree, w_sigma, w_gamma, w_hh, basis_A, basis_B,
                   tuple(float(v) for v in aabb_min), tuple(float(v) for v in aabb_max))


# ----------------------------------------------------------------------------
# Cameras and rays
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Rays:
    """Structure-of-arrays rays: origins [3, n], directions [3, n], times [n]."""
    origins: np.ndarray
    dirs: np.ndarray
    times: np.ndarray

    @property
    def n(self) -> int:
        return self.times.size

    def subset(self, idx) -> "Rays":
        return Rays(np.ascontiguousarray(self.origins[:, idx]), np.ascontiguousarray(self.dirs[:, idx]),
                    np.ascontiguousarray(self.times[idx]))

    @staticmethod
    def concat(parts) -> "Rays":
        return Rays(np.ascontiguousarray(np.concatenate([p.origins for p in parts], 1)),
                    np.ascontiguousarray(np.concatenate([p.dirs for p in parts], 1)),
                    np.ascontiguousarray(np.concatenate([p.times for p in parts])))


@dataclasses.dataclass
class Camera:
    eye: np.ndarray
    right: np.ndarray
    up: np.ndarray
    forward: np.ndarray
    width: int
    height: int
    fov_y_deg: float = 40.0


def look_at(eye, target, width: int, height: int, fov_y_deg: float = 40.0, up_hint=(0.0, 0.0, 1.0)) -> Camera:
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    up_hint = np.asarray(up_hint, np.float64)
    if abs(float(fwd @ up_hint)) > 0.999:
        up_hint = np.array([0.0, 1.0, 0.0])
    right = np.cross(fwd, up_hint)
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    return Camera(eye, right, up, fwd, width, height, fov_y_deg)


def sphere_cameras(seed: int, n: int, radius: float, width: int, height: int,
                   center=(0.5, 0.5, 0.5), fov_y_deg: float = 40.0) -> list:
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    c = np.asarray(center, np.float64)
    return [look_at(c + radius * vi, c, width, height, fov_y_deg) for vi in v]


def tile_order(width: int, height: int, tw: int = 8, th: int = 4) -> np.ndarray:
    """Pixel indices (row-major ids) listed tile by tile: each run of tw*th rays
    covers one tw x th pixel tile, so a 32-ray packet is spatially coherent."""
    y, x = np.divmod(np.arange(width * height, dtype=np.int64), width)
    key = np.lexsort((x % tw, y % th, x // tw, y // th))
    return key


def camera_rays(cam: Camera, t: float, pixels: np.ndarray | None = None, tiled: bool = True) -> tuple:
    """Rays through pixel centres.  Returns (Rays, pixel_ids) where pixel_ids[i]
    is the row-major pixel of ray i."""
    W, H = cam.width, cam.height
    if pixels is None:
        pixels = tile_order(W, H) if tiled else np.arange(W * H, dtype=np.int64)
    py, px = np.divmod(pixels, W)
    th = math.tan(math.radians(cam.fov_y_deg) / 2.0)
    sx = (2.0 * (px + 0.5) / W - 1.0) * th * (W / H)
    sy = (1.0 - 2.0 * (py + 0.5) / H) * th
    d = cam.forward[:, None] + cam.right[:, None] * sx[None] + cam.up[:, None] * sy[None]
    d /= np.linalg.norm(d, axis=0, keepdims=True)
    o = np.repeat(cam.eye[:, None], pixels.size, axis=1)
    rays = Rays(np.ascontiguousarray(o, np.float32), np.ascontiguousarray(d, np.float32),
                np.full(pixels.size, t, np.float32))
    return rays, pixels


# ----------------------------------------------------------------------------
# The five workloads (scene seed 1234 + i, camera seed 42 + i)
# ----------------------------------------------------------------------------

def _calibrate_solid(shape: Shape, depth: int, target: int) -> float:
    lo, hi = 0.25, 4.0
    for _ in range(18):
        mid = math.sqrt(lo * hi)
        n = occupied_cells(shape, depth, "solid", axis_scale=mid).shape[0]
        if n < target:
            lo = mid
        else:
            hi = mid
    return math.sqrt(lo * hi)


def solid_scene_structure(seed: int, depth: int, target_at_depth6: int = 20000) -> tuple:
    """Union of 5 seeded ellipsoids (centres U[0.3,0.7]^3, semi-axes U[0.08,0.2],
    uniform rotations), axes scaled so that the depth-6 build has about
    ``target_at_depth6`` leaves; the same shape is used at any depth."""
    rng = np.random.default_rng(seed)
    shape = make_shape(rng, 5, 0.3, 0.7, 0.08, 0.2)
    s = _calibrate_solid(shape, 6, target_at_depth6)
    cells = occupied_cells(shape, depth, "solid", axis_scale=s)
    st = build_tree(depth, np.full(cells.shape[0], depth), cells)
    return st, rng, {"axis_scale": s}


def shell_scene_structure(seed: int, depth: int, n_ell: int, target: int) -> tuple:
    """Noise-displaced shell around a union of seeded ellipsoids; the half
    thickness h is set so that the leaf count is about ``target``."""
    rng = np.random.default_rng(seed)
    shape = make_shape(rng, n_ell, 0.25, 0.75, 0.08, 0.22, noise_amp=0.02)
    # occupancy grows linearly with h once h exceeds a cell: two linear steps
    h = 2.0 / (1 << depth)
    for _ in range(2):
        n = occupied_cells(shape, depth, "shell", h=h).shape[0]
        h *= target / max(n, 1)
    cells = occupied_cells(shape, depth, "shell", h=h)
    st = build_tree(depth, np.full(cells.shape[0], depth), cells)
    return st, rng, {"shell_half_thickness": h}


def config1_tree(depth: int = 6) -> VOctree:
    st, rng, info = solid_scene_structure(1235, depth)
    tree = make_coefficients(rng, st, K=8, T=30, hh_degree=2)
    tree.info.update(info, name=f"c1-solid-5ell-d{depth}")
    return tree


def config1_rays() -> tuple:
    cam = sphere_cameras(43, 1, 2.5, 128, 128)[0]
    return camera_rays(cam, 0.37)


def config2_tree(depth: int = 9, target: int = 2_000_000) -> VOctree:
    st, rng, info = shell_scene_structure(1236, depth, 12, target)
    tree = make_coefficients(rng, st, K=16, T=150, hh_degree=3)
    tree.info.update(info, name=f"c2-shell-12ell-d{depth}")
    return tree


def config2_rays(width: int = 1920, height: int = 1080, n_views: int = 8) -> tuple:
    cams = sphere_cameras(44, n_views, 2.5, width, height)
    ts = np.random.default_rng(44 + 1000).uniform(0.0, 1.0, n_views)
    parts, pix = [], []
    for cam, t in zip(cams, ts):
        r, p = camera_rays(cam, float(t))
        parts.append(r)
        pix.append(p)
    return Rays.concat(parts), pix, cams, ts


def training_rays(seed: int, n_rays: int, n_views: int, n_times: int, width: int, height: int,
                  radius: float = 2.5) -> Rays:
    """Rays drawn uniformly over (camera, time stamp, pixel), in the order
    drawn (a training batch as a data loader delivers it)."""
    cams = sphere_cameras(seed, n_views, radius, width, height)
    rng = np.random.default_rng(seed + 1000)
    times = np.linspace(0.0, 1.0, n_times).astype(np.float32)
    view = rng.integers(0, n_views, n_rays)
    tsel = rng.integers(0, n_times, n_rays)
    pix = rng.integers(0, width * height, n_rays)
    o = np.empty((3, n_rays), np.float32)
    d = np.empty((3, n_rays), np.float32)
    for v in range(n_views):
        sel = np.nonzero(view == v)[0]
        r, _ = camera_rays(cams[v], 0.0, pixels=pix[sel])
        o[:, sel] = r.origins
        d[:, sel] = r.dirs
    return Rays(o, d, times[tsel].astype(np.float32))


def config3_tree() -> VOctree:
    st, rng, info = solid_scene_structure(1235, 8)
    tree = make_coefficients(rng, st, K=8, T=30, hh_degree=2)
    tree.info.update(info, name="c3-solid-5ell-d8")
    return tree


def config3_rays(n_rays: int = 262_144) -> Rays:
    return training_rays(45, n_rays, 16, 16, 512, 512)


def perturbed(tree: VOctree, seed: int, std: float = 0.05) -> VOctree:
    """Copy of ``tree`` with every coefficient perturbed by N(0, std)."""
    rng = np.random.default_rng(seed)
    return tree.with_coeffs(
        tree.w_sigma + std * rng.standard_normal(tree.w_sigma.shape, dtype=np.float32),
        tree.w_gamma + std * rng.standard_normal(tree.w_gamma.shape, dtype=np.float32),
        tree.w_hh + std * rng.standard_normal(tree.w_hh.shape, dtype=np.float32))


@dataclasses.dataclass
class Primitive:
    transform: np.ndarray   # [3, 4] world-from-local: [s R | translation]
    time_offset: float      # frames
    tint: np.ndarray        # [3]


def config4_primitives(n: int = 8, T: int = 30, seed: int = 1238) -> list:
    """Rigid transform uniform on SO(3), scale U[0.5,1.5], centre in a 4x4x2 box,
    time offset U[0, T), tint U[0.5, 1]^3.  The local unit cube is centred first."""
    rng = np.random.default_rng(seed)
    R = _random_rotations(rng, n)
    s = rng.uniform(0.5, 1.5, n)
    c = rng.uniform([-2.0, -2.0, -1.0], [2.0, 2.0, 1.0], (n, 3))
    off = rng.uniform(0.0, T, n)
    tint = rng.uniform(0.5, 1.0, (n, 3))
    prims = []
    for i in range(n):
        M = s[i] * R[i]
        tr = c[i] - M @ np.array([0.5, 0.5, 0.5])
        prims.append(Primitive(np.concatenate([M, tr[:, None]], 1), float(off[i]), tint[i]))
    return prims


def config4_rays(width: int = 2160, height: int = 2160, eye_sep: float = 0.064, t: float = 0.5) -> tuple:
    rng = np.random.default_rng(46)
    v = rng.standard_normal(3)
    v /= np.linalg.norm(v)
    center = np.zeros(3)
    mid = center + 8.0 * v
    base = look_at(mid, center, width, height)
    parts, pix, cams = [], [], []
    for sgn in (-0.5, 0.5):
        cam = look_at(mid + sgn * eye_sep * base.right, center, width, height)
        r, p = camera_rays(cam, t)
        parts.append(r)
        pix.append(p)
        cams.append(cam)
    return Rays.concat(parts), pix, cams


def config5_tree(depth: int = 10, target: int = 8_000_000) -> VOctree:
    st, rng, info = shell_scene_structure(1239, depth, 12, target)
    tree = make_coefficients(rng, st, K=16, T=300, hh_degree=3)
    tree.info.update(info, name=f"c5-shell-12ell-d{depth}")
    return tree


def config5_rays(n_rays: int = 1_048_576) -> Rays:
    return training_rays(47, n_rays, 32, 32, 1920, 1080)
