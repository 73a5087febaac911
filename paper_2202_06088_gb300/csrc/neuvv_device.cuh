// Device building blocks of the VOctree renderer (sm_103a).
//
// Everything a ray needs, shared by the forward, adjoint, trace and compose
// kernels so that all of them walk exactly the same voxels:
//   * RayWalk   -- stackless octree walk (Sec. 4.3 "Rendering": the voxels on
//                  the ray and the chord lengths {delta_i} inside them);
//   * sh_real   -- real spherical harmonics of the view direction, l <= 3
//                  (App. A, Eq. real-SH; no Condon-Shortley phase);
//   * hh_radial -- Abar_{n,l} sin^l(gamma) C^{l+1}_{n-l}(cos gamma) and its
//                  gamma-derivative, by the Gegenbauer recurrence in registers
//                  (Eq. complex-HSH);
//   * LeafRecord-- one leaf's coefficient record fetched with 16-byte vector
//                  loads and widened to FP32.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace neuvv {

constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr uint32_t kLeafBit = 0x80000000u;
constexpr float kPi = 3.14159265358979323846f;
constexpr uint32_t kStatusSegCap = 0x1u;    // a ray reached its walk-step cap
constexpr uint32_t kStatusBadIndex = 0x2u;  // a child, brick, leaf or log index out of range
constexpr uint32_t kStatusTimeout = 0x4u;   // a bounded wait (an mbarrier poll) gave up

__host__ __device__ constexpr int n_hh(int deg) { return deg < 0 ? 0 : n_hh(deg - 1) + (deg + 1) * (deg + 1); }
__host__ __device__ constexpr int hh_index(int n, int l, int m) { return n * (n + 1) * (2 * n + 1) / 6 + l * l + l + m; }
__host__ __device__ constexpr int radial_index(int n, int l) { return n * (n + 1) / 2 + l; }

// Device view of a tree, passed to kernels by value.
struct DevTree {
  const uint32_t *child;  // [n_nodes][8]
  const void *rec;        // [n_leaves][rec_stride] storage records
  const float *A;         // [T][KP] density basis (zero padded)
  const float *B;         // [T][KP] hyper-angle basis
  uint32_t *status;       // device status word
  long long n_nodes, n_leaves;
  float bmin[3], bmax[3];
  float scale[3];         // 2^depth / (bmax - bmin)
  float hh_norm[16];      // Abar_{n,l} at [4n + l]
  int depth, T, K, rec_stride, smem_nodes;
  // Bricks: for each internal node at brick_level (nodes brick_first ..
  // brick_first + brick_count - 1), a dense table over its finest cells of
  // (level << 28 | leaf id), an id from kBrickBoxBase up for empty: the node
  // that holds each cell, so the descent below brick_level is one load (and
  // for an empty cell, when the id says so, an empty box around it larger
  // than its node).  Null when the tree has none.
  const uint32_t *bricks;
  int brick_level, brick_first, brick_count;
  // Brick map: a dense grid over the cells of level brick_level, one word per
  // cell: (0 << 28) | brick index (the cell is an internal node with a brick),
  // (L << 28) | leaf id (the cell lies in a leaf of level L <= brick_level), or
  // (kCoarseEmpty << 28) | (s << 24) | six 4-bit extents for an empty cell:
  // the box from (cell - below * 2^s) to (cell + above * 2^s) per axis, x in
  // bits 0-7, y 8-15, z 16-23 (below in the low nibble), holds no non-empty
  // cell.  Null when the tree has none; the walk then descends the octree.
  const uint32_t *coarse;
  // Limits: walk steps per ray (0: 3 * 2^depth + 8, enough for any ray) and
  // polls of a bounded wait before it gives up and flags kStatusTimeout.
  int step_cap, wait_polls;
  // Words of the per-thread descent path in a packet kernel's shared memory
  // (0 with a brick map, whose walk never descends the child table).
  int path_words;
};

constexpr uint32_t kCoarseEmpty = 15u;

constexpr uint32_t kBrickEmpty = 0x0FFFFFFFu;
// Brick entries with an id from kBrickBoxBase up are empty: kBrickEmpty, or
// kBrickBoxBase | the extents of an empty box around the cell (4 bits each,
// cells below and above it on x in bits 0-7, y 8-15, z 16-23, below in the
// low nibble).  Leaf ids stay below kBrickBoxBase.
constexpr uint32_t kBrickBoxBase = 0x0F000000u;

__device__ __forceinline__ void raise_status(const DevTree &tr, uint32_t bit) {
  if (tr.status) atomicOr(tr.status, bit);
}

// ---------------------------------------------------------------------------
// Octree walk.  Grid space: the root box is [0, N]^3, N = 2^depth, finest
// cells are unit cubes.  Positions are kept relative to the ray's entry into
// the root box so that FP32 coordinates stay below N.  Chords must be exact
// to a few FP32 ulps of the chord itself (a thin corner clip of a leaf
// weighs its gradient by its chord), so:
//   * the entry point is carried as go + lo per axis, go a multiple of
//     2^(depth-24) grid units, so that plane - go is exact for every cell
//     plane x in [0, N];
//   * a plane's distance (x - go) * inv - lo * inv is carried as an
//     unevaluated sum hi + lo: the exact product of the exact gap with inv,
//     minus the small per-axis constant lo * inv;
//   * a chord is the difference of two such sums, so its error is relative to
//     the chord, not to the distance from the entry.
// Decisions:
//   * exit axis = argmin of the three exit distances, exact ties x < y < z;
//   * the next cell is one step across the exit face on that axis, and on the
//     other axes the cell holding the exit point (a coordinate exactly on a
//     cell boundary goes to the side the ray moves towards), clamped to the
//     node just left.
// Every distance is along the unit direction, in world units.
// ---------------------------------------------------------------------------
struct RayWalk {
  float go[3];     // grid position of the entry point (a multiple of 2^(depth-24))
  float gd[3];     // grid-space direction (unit world direction * scale)
  float inv[3];    // 1 / gd (inf when gd == 0)
  float c[3];      // (exact entry - go) * inv: plane x lies at (x - go) * inv - c
  float t_base;    // world distance of the entry point from the origin
  float t_cur;     // current distance past the entry point (hi part)
  float t_lo;      // its lo part (t_cur + t_lo: see the plane distances above)
  float t_far;     // exit distance of the root box past the entry point
  int cell[3];
  int steps, max_steps;
  int restart;     // level at which the next descent may start (0 = root)
  uint32_t c_idx;  // brick-map cell of the last lookup (0xFFFFFFFF: none) ...
  uint32_t c_word; // ... and its word
  bool alive;
};

// Error-free transformations: s + e = a + b and p + e = a * b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
  p = a * b;
  e = fmaf(a, b, -p);
}

__device__ __forceinline__ int cell_of(float p, float v, int N) {
  // the cell the ray occupies just after this instant: floor(p), or
  // ceil(p) - 1 when moving towards lower coordinates (one rounding each)
  const int c = v < 0.f ? __float2int_ru(p) - 1 : __float2int_rd(p);
  return min(max(c, 0), N - 1);
}

// Intersects the line o + s d (s >= 0, d as given, not normalised) with the
// tree's box.  On a hit: the parameter interval [s_in, s_out] and the axis of
// the entry face (-1 when the origin is inside the box).
__device__ __forceinline__ bool box_interval(const DevTree &tr, const float o[3], const float d[3], float &s_in,
                                             float &s_out, int &ax_in) {
  float sn = -INFINITY, sf = INFINITY;
  int axn = -1;
  bool hit = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (d[a] == 0.f) {
      if (o[a] < tr.bmin[a] || o[a] > tr.bmax[a]) hit = false;
    } else {
      const float s0 = (tr.bmin[a] - o[a]) / d[a], s1 = (tr.bmax[a] - o[a]) / d[a];
      const float lo = fminf(s0, s1), hi = fmaxf(s0, s1);
      if (lo > sn) {
        sn = lo;
        axn = a;
      }
      sf = fminf(sf, hi);
    }
  }
  s_in = fmaxf(sn, 0.f);
  s_out = sf;
  ax_in = sn > 0.f ? axn : -1;
  return hit && s_in < s_out;
}

// Starts the walk at point p + pl of the tree's frame (inside the box; on
// the entry face when the ray comes from outside; pl the part of the point
// below p's FP32 precision) along the unit direction dn.
__device__ __forceinline__ void walk_start(const DevTree &tr, const float p[3], const float pl[3], const float dn[3],
                                           RayWalk &w) {
  const int N = 1 << tr.depth;
  const float q = ldexpf(1.f, tr.depth - 24), iq = ldexpf(1.f, 24 - tr.depth);
  float tf = INFINITY;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    // grid coordinate gh + gl = (p + pl - bmin) * scale, then split at q
    float dh, dl, gh, ge;
    two_sum(p[a], -tr.bmin[a], dh, dl);
    two_prod(dh, tr.scale[a], gh, ge);
    float gl = fmaf(dl + pl[a], tr.scale[a], ge);
    if (!(gh > 0.f)) { gh = 0.f; gl = fmaxf(gl, 0.f); }
    if (gh >= (float)N) { gh = (float)N; gl = fminf(gl, 0.f); }
    const float go = rintf(gh * iq) * q;  // x - go is exact for integer x in [0, N]
    const float lo = (gh - go) + gl;
    w.go[a] = go;
    w.gd[a] = dn[a] * tr.scale[a];
    w.inv[a] = w.gd[a] != 0.f ? 1.f / w.gd[a] : INFINITY;
    w.c[a] = w.gd[a] != 0.f ? lo * w.inv[a] : 0.f;
    // the cell the ray occupies just after the exact entry point
    int cell = cell_of(go, w.gd[a], N);
    if (go == floorf(go) && lo != 0.f) cell = (lo < 0.f ? (int)go - 1 : (int)go);
    w.cell[a] = min(max(cell, 0), N - 1);
    if (w.gd[a] != 0.f) tf = fminf(tf, ((w.gd[a] > 0.f ? (float)N : 0.f) - go) * w.inv[a] - w.c[a]);
  }
  w.t_cur = 0.f;
  w.t_lo = 0.f;
  w.t_far = tf;
  w.restart = 0;
  w.c_idx = 0xFFFFFFFFu;
  w.c_word = 0u;
  w.steps = 0;
  w.max_steps = tr.step_cap > 0 ? tr.step_cap : 3 * N + 8;
  w.alive = tf > 0.f;
}

// Ray given in the tree's own frame.  The entry point is formed from the exact
// input line with one FMA per axis and the entry face's coordinate set
// exactly, so a distant origin costs no precision inside the box.
__device__ __forceinline__ bool walk_init(const DevTree &tr, const float o[3], const float d[3], RayWalk &w,
                                          float dn[3]) {
  const float len = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  w.alive = false;
  if (!(len > 0.f)) return false;
  const float il = 1.f / len;
  dn[0] = d[0] * il;
  dn[1] = d[1] * il;
  dn[2] = d[2] * il;
  float s_in, s_out;
  int ax;
  if (!box_interval(tr, o, d, s_in, s_out, ax)) return false;
  float p[3], pl[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    p[a] = o[a];
    pl[a] = 0.f;
  }
  if (ax >= 0) {
    // entry parameter s = (face - o) / d on the entry axis as sh + sl, then
    // each other coordinate o + s d as an unevaluated sum (error-free steps)
    float f = tr.bmin[0], oa = o[0], da = d[0];
#pragma unroll
    for (int a = 1; a < 3; ++a)
      if (a == ax) { f = tr.bmin[a]; oa = o[a]; da = d[a]; }
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (a == ax && d[a] < 0.f) f = tr.bmax[a];
    float nh, nl;
    two_sum(f, -oa, nh, nl);
    const float sh = nh / da;
    const float sl = (fmaf(-sh, da, nh) + nl) / da;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a == ax) {
        p[a] = f;
      } else {
        float ph, pe, sh2, se;
        two_prod(sh, d[a], ph, pe);
        two_sum(o[a], ph, sh2, se);
        const float lo = fmaf(sl, d[a], se + pe);
        p[a] = sh2 + lo;
        pl[a] = lo - (p[a] - sh2);
      }
    }
  }
  w.t_base = s_in * len;
  walk_start(tr, p, pl, dn, w);
  return w.alive;
}

// Path of the current descent, one node per level, kept per thread in shared
// memory (entry L at path[L * stride]) so that the next descent can start at
// the lowest common ancestor of the old and the new cell instead of the root.
struct PathRef {
  uint32_t *path;
  int stride;
};

// Descends to the tree cell holding `cell`, from the root or (kPath) from the
// ancestor at level `start` recorded by the previous descent.  Returns the
// child entry found (kEmpty or kLeafBit|leaf) and its level.  The first
// smem_nodes rows of the child table may be read from shared memory.
template <bool kSmem, bool kPath>
__device__ __forceinline__ uint32_t descend(const DevTree &tr, const uint32_t *s_child, PathRef pr, const int cell[3],
                                            int start, int &level) {
  const int D = tr.depth;
  uint32_t node = 0;
  int L = 0;
  if (kPath && start > 0) {
    L = start;
    if (tr.bricks && L > tr.brick_level) L = tr.brick_level;
    node = pr.path[L * pr.stride];
  }
  for (; L < D; ++L) {
    if (kPath) pr.path[L * pr.stride] = node;
    if (tr.bricks && L == tr.brick_level) {
      // the rest of the descent is one entry of the node's brick
      const uint32_t b = node - (uint32_t)tr.brick_first;
      if (b >= (uint32_t)tr.brick_count) {
        raise_status(tr, kStatusBadIndex);
        level = L + 1;
        return kEmpty;
      }
      const int sh = D - L;
      const int m = (1 << sh) - 1;
      const uint32_t idx = (uint32_t)(((cell[0] & m) << (2 * sh)) | ((cell[1] & m) << sh) | (cell[2] & m));
      const uint32_t v = __ldg(tr.bricks + ((size_t)b << (3 * sh)) + idx);
      level = (int)(v >> 28);
      const uint32_t id = v & kBrickEmpty;
      return id >= kBrickBoxBase ? kEmpty : (kLeafBit | id);
    }
    const int bit = D - 1 - L;
    const int slot = (((cell[0] >> bit) & 1) << 2) | (((cell[1] >> bit) & 1) << 1) | ((cell[2] >> bit) & 1);
    uint32_t e;
    if (kSmem && node < (uint32_t)tr.smem_nodes)
      e = s_child[node * 8 + slot];
    else
      e = __ldg(tr.child + (size_t)node * 8 + slot);
    if (e == kEmpty || (e & kLeafBit)) {
      level = L + 1;
      if (e != kEmpty && (e & ~kLeafBit) >= (uint32_t)tr.n_leaves) {
        raise_status(tr, kStatusBadIndex);
        return kEmpty;
      }
      return e;
    }
    if (e >= (uint32_t)tr.n_nodes) {
      raise_status(tr, kStatusBadIndex);
      level = L + 1;
      return kEmpty;
    }
    node = e;
  }
  level = D;
  return kEmpty;
}

// One step of the walk: the tree cell holding the current finest cell, then
// the move across its exit face.  Returns true (with the leaf, the distance
// t0 of the segment's start past the entry point and its chord dt) when that
// cell is an occupied leaf crossed with a positive chord.  Clears w.alive when
// the ray leaves the root box or reaches its step cap.
template <bool kSmem, bool kPath = false>
__device__ __forceinline__ bool walk_step(const DevTree &tr, const uint32_t *s_child, RayWalk &w, uint32_t &leaf,
                                          float &t0, float &dt, PathRef pr = PathRef{nullptr, 0}) {
  const int N = 1 << tr.depth;
  if (++w.steps > w.max_steps) {
    raise_status(tr, kStatusSegCap);
    w.alive = false;
    return false;
  }
  // the box [lo, hi) the ray crosses next: the tree cell holding the current
  // finest cell, or with a brick map possibly a larger empty box
  uint32_t e;
  int lo[3], hi[3];
  bool fine = false;  // the box is a single finest cell
  if (tr.coarse) {
    const int cs = tr.depth - tr.brick_level, Lc = tr.brick_level;
    const int cx = w.cell[0] >> cs, cy = w.cell[1] >> cs, cz = w.cell[2] >> cs;
    const uint32_t ci = ((uint32_t)cx << (2 * Lc)) | ((uint32_t)cy << Lc) | (uint32_t)cz;
    if (ci != w.c_idx) {
      w.c_idx = ci;
      w.c_word = __ldg(tr.coarse + ci);
    }
    const uint32_t cw = w.c_word, kind = cw >> 28;
    if (kind == kCoarseEmpty) {
      // the empty box around this brick-map cell: extents below and above
      // it per axis, 4 bits each in units of 2^s cells
      const int s = (int)((cw >> 24) & 15u), Nc = 1 << Lc;
      const int cc[3] = {cx, cy, cz};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int below = (int)((cw >> (8 * a)) & 15u) << s, above = (int)((cw >> (8 * a + 4)) & 15u) << s;
        lo[a] = max(cc[a] - below, 0) << cs;
        hi[a] = min(cc[a] + above + 1, Nc) << cs;
      }
      e = kEmpty;
    } else {
      int level;
      uint32_t box = 0u;  // an empty box's code from the brick (0: none)
      if (kind == 0) {
        const uint32_t b = cw & 0x0FFFFFFFu;
        if (b >= (uint32_t)tr.brick_count) {
          raise_status(tr, kStatusBadIndex);
          w.alive = false;
          return false;
        }
        const int m = (1 << cs) - 1;
        const uint32_t idx = (uint32_t)(((w.cell[0] & m) << (2 * cs)) | ((w.cell[1] & m) << cs) | (w.cell[2] & m));
        const uint32_t v = __ldg(tr.bricks + ((size_t)b << (3 * cs)) + idx);
        level = (int)(v >> 28);
        const uint32_t id = v & kBrickEmpty;
        e = id >= kBrickBoxBase ? kEmpty : (kLeafBit | id);
        if (id >= kBrickBoxBase && id != kBrickEmpty) box = id;  // an empty box around the cell
      } else {
        level = (int)kind;
        e = kLeafBit | (cw & 0x0FFFFFFFu);
      }
      if (e != kEmpty && (e & ~kLeafBit) >= (uint32_t)tr.n_leaves) {
        raise_status(tr, kStatusBadIndex);
        e = kEmpty;
      }
      if (box) {
        // extents below and above the cell per axis, 4 bits each
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          lo[a] = w.cell[a] - (int)((box >> (8 * a)) & 15u);
          hi[a] = w.cell[a] + (int)((box >> (8 * a + 4)) & 15u) + 1;
        }
        fine = (box & 0x00FFFFFFu) == 0u;
      } else {
        const int size = 1 << (tr.depth - level);
        fine = size == 1;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          lo[a] = w.cell[a] & -size;
          hi[a] = lo[a] + size;
        }
      }
    }
  } else {
    int level;
    e = descend<kSmem, kPath>(tr, s_child, pr, w.cell, w.restart, level);
    const int size = 1 << (tr.depth - level);
    fine = size == 1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      lo[a] = w.cell[a] & -size;
      hi[a] = lo[a] + size;
    }
  }
  float gap[3], tx[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    gap[a] = (float)(w.gd[a] > 0.f ? hi[a] : lo[a]) - w.go[a];  // exact
    // the plane's distance gap * inv - c with one rounding, so that the exit
    // axis is decided on distances accurate to an ulp
    tx[a] = w.gd[a] != 0.f ? fmaf(gap[a], w.inv[a], -w.c[a]) : INFINITY;
  }
  // exit axis: first minimum (exact ties x < y < z); register-only selects
  int ax = 0;
  float t_exit = tx[0], g_ax = gap[0], i_ax = w.inv[0], c_ax = w.c[0];
  if (tx[1] < t_exit) { ax = 1; t_exit = tx[1]; g_ax = gap[1]; i_ax = w.inv[1]; c_ax = w.c[1]; }
  if (tx[2] < t_exit) { ax = 2; t_exit = tx[2]; g_ax = gap[2]; i_ax = w.inv[2]; c_ax = w.c[2]; }
  // the exit plane lies at t_exit + x_lo: x_lo = (gap * inv - t_exit) - c
  // (the product exact inside the FMA)
  const float x_lo = fmaf(g_ax, i_ax, -t_exit) - c_ax;
  const float chord = (t_exit - w.t_cur) + (x_lo - w.t_lo);
  bool found = false;
  if (e != kEmpty && chord > 0.f) {
    leaf = e & ~kLeafBit;
    t0 = w.t_cur;
    dt = chord;
    found = true;
  }
  // step to the next cell
  if (t_exit >= w.t_far) {
    w.alive = false;
  } else {
    if (chord > 0.f) {
      w.t_cur = t_exit;
      w.t_lo = x_lo;
    }
    // on the other axes the neighbour of a finest cell across the exit face
    // has the same coordinates; a larger box needs the exit point's cell.
    // The ray's coordinates move one way only, so a cell behind the current
    // one on such an axis is the exit point's rounding (at an edge the ray
    // crosses, the exit plane of one axis and a cell boundary of another at
    // one distance) and is not taken: otherwise two boxes meeting at that
    // edge could hand the walk back and forth without progress.
    if (!fine) {
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        if (b != ax) {
          const float p = fmaf(w.t_cur, w.gd[b], w.go[b]);
          const int c = min(max(cell_of(p, w.gd[b], N), lo[b]), hi[b] - 1);
          w.cell[b] = w.gd[b] > 0.f ? max(c, w.cell[b]) : (w.gd[b] < 0.f ? min(c, w.cell[b]) : c);
        }
      }
    }
    const int lo_ax = ax == 0 ? lo[0] : (ax == 1 ? lo[1] : lo[2]);
    const int hi_ax = ax == 0 ? hi[0] : (ax == 1 ? hi[1] : hi[2]);
    const float gd_ax = ax == 0 ? w.gd[0] : (ax == 1 ? w.gd[1] : w.gd[2]);
    const int nc = gd_ax > 0.f ? hi_ax : lo_ax - 1;
    const bool inside = nc >= 0 && nc < N;
#pragma unroll
    for (int b = 0; b < 3; ++b)
      if (b == ax) w.cell[b] = nc;
    // deepest level whose cell holds both the old node and the new cell
    if (kPath && inside && !tr.coarse) w.restart = tr.depth - 32 + __clz(nc ^ lo_ax);
    if (!inside) w.alive = false;
  }
  return found;
}

// Advances to the next occupied-leaf segment (see walk_step); false when the
// ray has left the root box (or hit its step cap).
template <bool kSmem, bool kPath = false>
__device__ __forceinline__ bool walk_next(const DevTree &tr, const uint32_t *s_child, RayWalk &w, uint32_t &leaf,
                                          float &t0, float &dt, PathRef pr = PathRef{nullptr, 0}) {
  while (w.alive)
    if (walk_step<kSmem, kPath>(tr, s_child, w, leaf, t0, dt, pr)) return true;
  return false;
}

// ---------------------------------------------------------------------------
// Real spherical harmonics of a unit direction, l <= DEG <= 3, index l^2+l+m.
// Y_l0 = K_l0 P_l(z); Y_l,m>0 = sqrt2 K_lm P_l^m(z) cos(m phi);
// Y_l,m<0 = sqrt2 K_l|m| P_l^|m|(z) sin(|m| phi), written as polynomials in
// (x, y, z) (sin^m(theta) e^{i m phi} = (x + i y)^m).
// ---------------------------------------------------------------------------
template <int DEG>
__device__ __forceinline__ void sh_real(const float d[3], float *Y) {
  const float x = d[0], y = d[1], z = d[2];
  Y[0] = 0.28209479177387814f;  // 1 / (2 sqrt(pi))
  if (DEG >= 1) {
    const float c1 = 0.4886025119029199f;  // sqrt(3 / (4 pi))
    Y[1] = c1 * y;
    Y[2] = c1 * z;
    Y[3] = c1 * x;
  }
  if (DEG >= 2) {
    const float c2a = 1.0925484305920792f;   // sqrt(15 / (4 pi))
    const float c20 = 0.31539156525252005f;  // sqrt(5 / (16 pi))
    const float c22 = 0.5462742152960396f;   // sqrt(15 / (16 pi))
    Y[4] = c2a * x * y;
    Y[5] = c2a * y * z;
    Y[6] = c20 * (3.f * z * z - 1.f);
    Y[7] = c2a * x * z;
    Y[8] = c22 * (x * x - y * y);
  }
  if (DEG >= 3) {
    const float c3a = 0.5900435899266435f;  // sqrt(35 / (32 pi))
    const float c3b = 2.890611442640554f;   // sqrt(105 / (4 pi))
    const float c3c = 0.4570457994644658f;  // sqrt(21 / (32 pi))
    const float c30 = 0.3731763325901154f;  // sqrt(7 / (16 pi))
    const float c32 = 1.445305721320277f;   // sqrt(105 / (16 pi))
    const float zz = z * z;
    Y[9] = c3a * y * (3.f * x * x - y * y);
    Y[10] = c3b * x * y * z;
    Y[11] = c3c * y * (5.f * zz - 1.f);
    Y[12] = c30 * z * (5.f * zz - 3.f);
    Y[13] = c3c * x * (5.f * zz - 1.f);
    Y[14] = c32 * z * (x * x - y * y);
    Y[15] = c3a * x * (x * x - 3.f * y * y);
  }
}

// ---------------------------------------------------------------------------
// Radial factors R_nl = Abar_{n,l} sin^l(g) C^{l+1}_{n-l}(cos g) for n <= DEG,
// stored at radial_index(n, l); optionally dR_nl/dg.  Gegenbauer recurrence
// k C_k = 2x(k+lam-1) C_{k-1} - (k+2lam-2) C_{k-2}, differentiated alongside.
// ---------------------------------------------------------------------------
template <int DEG, bool kDeriv>
__device__ __forceinline__ void hh_radial(float cg, float sg, const float *norm, float *R, float *dR) {
  float sl = 1.f, slm1 = 0.f;  // sin^l, sin^(l-1)
#pragma unroll
  for (int l = 0; l <= DEG; ++l) {
    const float lam = (float)(l + 1);
    float cm2 = 0.f, cm1 = 0.f, dm2 = 0.f, dm1 = 0.f;  // C_{k-2}, C_{k-1} and d/dx
#pragma unroll
    for (int k = 0; l + k <= DEG; ++k) {
      float ck, dk;
      if (k == 0) {
        ck = 1.f;
        dk = 0.f;
      } else if (k == 1) {
        ck = 2.f * lam * cg;
        dk = 2.f * lam;
      } else {
        const float a = 2.f * (k + lam - 1.f) / k, b = (k + 2.f * lam - 2.f) / k;
        ck = a * cg * cm1 - b * cm2;
        dk = a * (cm1 + cg * dm1) - b * dm2;
      }
      const int n = l + k;
      const float An = norm[4 * n + l];
      R[radial_index(n, l)] = An * sl * ck;
      if (kDeriv) {
        // d/dg [sin^l g C(cos g)] = l sin^(l-1) g cos g C - sin^(l+1) g C'
        dR[radial_index(n, l)] = An * ((float)l * slm1 * cg * ck - sl * sg * dk);
      }
      cm2 = cm1;
      cm1 = ck;
      dm2 = dm1;
      dm1 = dk;
    }
    slm1 = sl;
    sl *= sg;
  }
}

// ---------------------------------------------------------------------------
// Leaf records: [w_sigma KP][w_gamma KP][w_hh 3*NH channel-major][pad]
// ---------------------------------------------------------------------------
template <typename E>
struct Elem;
template <>
struct Elem<float> {
  static constexpr int kPerVec = 4;
  __device__ __forceinline__ static void unpack(const uint4 v, float *o) {
    o[0] = __uint_as_float(v.x);
    o[1] = __uint_as_float(v.y);
    o[2] = __uint_as_float(v.z);
    o[3] = __uint_as_float(v.w);
  }
};
template <>
struct Elem<__nv_bfloat16> {
  static constexpr int kPerVec = 8;
  __device__ __forceinline__ static void unpack(const uint4 v, float *o) {
    o[0] = __uint_as_float(v.x << 16);
    o[1] = __uint_as_float(v.x & 0xFFFF0000u);
    o[2] = __uint_as_float(v.y << 16);
    o[3] = __uint_as_float(v.y & 0xFFFF0000u);
    o[4] = __uint_as_float(v.z << 16);
    o[5] = __uint_as_float(v.z & 0xFFFF0000u);
    o[6] = __uint_as_float(v.w << 16);
    o[7] = __uint_as_float(v.w & 0xFFFF0000u);
  }
};

__device__ __forceinline__ uint4 ldg_v4(const uint4 *p) {
  uint4 r;
  asm volatile("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(p));
  return r;
}

// FP8 storage (an ablation): E4M3 codes with power-of-two scales per leaf.
// Record = 16-byte header {scale of w_sigma, of w_gamma, of w_hh, 0} as FP32,
// then one code byte per entry of the FP32 layout, zero padded to 16 bytes;
// rec_stride counts bytes.  Entry value = decoded code * scale of its group.
struct Fp8E4M3 {};

template <int KP, int DEG, typename E>
struct LeafRecord {
  static constexpr int NH = n_hh(DEG);
  static constexpr int LEN = 2 * KP + 3 * NH;
  static constexpr int PV = Elem<E>::kPerVec;
  static constexpr int NV = (LEN + PV - 1) / PV;
  float w[NV * PV];

  __device__ __forceinline__ void load(const DevTree &tr, uint32_t leaf) {
    const uint4 *p = reinterpret_cast<const uint4 *>(static_cast<const E *>(tr.rec) + (size_t)leaf * tr.rec_stride);
    uint4 raw[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) raw[i] = ldg_v4(p + i);
#pragma unroll
    for (int i = 0; i < NV; ++i) Elem<E>::unpack(raw[i], w + i * PV);
  }
  // The same record from a copy in shared memory (a staged tile).
  __device__ __forceinline__ void load_shared(const uint4 *p) {
#pragma unroll
    for (int i = 0; i < NV; ++i) Elem<E>::unpack(p[i], w + i * PV);
  }
  // Only the vectors that hold w_sigma and w_gamma.
  __device__ __forceinline__ void load_sigma_gamma(const DevTree &tr, uint32_t leaf) {
    constexpr int NS = (2 * KP + PV - 1) / PV;
    const uint4 *p = reinterpret_cast<const uint4 *>(static_cast<const E *>(tr.rec) + (size_t)leaf * tr.rec_stride);
    uint4 raw[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) raw[i] = ldg_v4(p + i);
#pragma unroll
    for (int i = 0; i < NS; ++i) Elem<E>::unpack(raw[i], w + i * PV);
  }
  // Only the vectors that hold w_gamma.
  __device__ __forceinline__ void load_gamma(const DevTree &tr, uint32_t leaf) {
    constexpr int V0 = KP / PV, V1 = (2 * KP + PV - 1) / PV;
    const uint4 *p = reinterpret_cast<const uint4 *>(static_cast<const E *>(tr.rec) + (size_t)leaf * tr.rec_stride);
#pragma unroll
    for (int i = V0; i < V1; ++i) Elem<E>::unpack(ldg_v4(p + i), w + i * PV);
  }
  // Only the vectors that hold w_sigma (a density-only pass).
  __device__ __forceinline__ void load_sigma(const DevTree &tr, uint32_t leaf) {
    constexpr int NS = (KP + PV - 1) / PV;
    const uint4 *p = reinterpret_cast<const uint4 *>(static_cast<const E *>(tr.rec) + (size_t)leaf * tr.rec_stride);
    uint4 raw[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) raw[i] = ldg_v4(p + i);
#pragma unroll
    for (int i = 0; i < NS; ++i) Elem<E>::unpack(raw[i], w + i * PV);
  }
  __device__ __forceinline__ static void prefetch_sigma_l2(const DevTree &tr, uint32_t leaf) {
    const char *p = reinterpret_cast<const char *>(static_cast<const E *>(tr.rec) + (size_t)leaf * tr.rec_stride);
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p + KP * sizeof(E) - 1));
  }
  // Asks L2 for the lines of a leaf's record ahead of its use (no registers held).
  __device__ __forceinline__ static void prefetch_l2(const DevTree &tr, uint32_t leaf) {
    const char *p = reinterpret_cast<const char *>(static_cast<const E *>(tr.rec) + (size_t)leaf * tr.rec_stride);
    constexpr int kBytes = NV * 16;
#pragma unroll
    for (int b = 0; b < kBytes; b += 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(p + b));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p + kBytes - 1));
  }
  __device__ __forceinline__ float sig(int k) const { return w[k]; }
  __device__ __forceinline__ float gam(int k) const { return w[KP + k]; }
  __device__ __forceinline__ float hh(int ch, int i) const { return w[2 * KP + ch * NH + i]; }
  __device__ __forceinline__ float scale_sigma() const { return 1.f; }
  __device__ __forceinline__ float scale_gamma() const { return 1.f; }
  __device__ __forceinline__ float scale_hh() const { return 1.f; }
};

// Exponent p of an FP8 group's scale 2^p: the smallest p with
// max |w| <= 448 * 2^p, so that w / 2^p encodes without saturating (0 for an
// all-zero group).  Host and device use this one rule.
__host__ __device__ inline int fp8_scale_exp(float maxabs) {
  if (!(maxabs > 0.f)) return 0;
  int ex;
  frexpf(maxabs, &ex);  // maxabs in [2^(ex-1), 2^ex); 448 * 2^(ex-9) = 0.875 * 2^ex
  int p = ex - 9;
  if (ldexpf(448.f, p) < maxabs) ++p;
  return p;
}

template <int KP, int DEG>
struct LeafRecord<KP, DEG, Fp8E4M3> {
  static constexpr int NH = n_hh(DEG);
  static constexpr int LEN = 2 * KP + 3 * NH;
  static constexpr int NV = (LEN + 15) / 16;
  uint4 raw[NV];  // codes, decoded where an entry is used
  float sc[3];    // group scales (powers of two)

  __device__ __forceinline__ void load(const DevTree &tr, uint32_t leaf) {
    const uint4 *p = reinterpret_cast<const uint4 *>(static_cast<const unsigned char *>(tr.rec) +
                                                     (size_t)leaf * tr.rec_stride);
    const uint4 h = ldg_v4(p);
#pragma unroll
    for (int i = 0; i < NV; ++i) raw[i] = ldg_v4(p + 1 + i);
    sc[0] = __uint_as_float(h.x);
    sc[1] = __uint_as_float(h.y);
    sc[2] = __uint_as_float(h.z);
  }
  __device__ __forceinline__ void load_shared(const uint4 *p) {
    const uint4 h = p[0];
#pragma unroll
    for (int i = 0; i < NV; ++i) raw[i] = p[1 + i];
    sc[0] = __uint_as_float(h.x);
    sc[1] = __uint_as_float(h.y);
    sc[2] = __uint_as_float(h.z);
  }
  // The header and the code vectors that hold w_sigma and w_gamma.
  __device__ __forceinline__ void load_sigma_gamma(const DevTree &tr, uint32_t leaf) {
    constexpr int NS = (2 * KP + 15) / 16;
    const uint4 *p = reinterpret_cast<const uint4 *>(static_cast<const unsigned char *>(tr.rec) +
                                                     (size_t)leaf * tr.rec_stride);
    const uint4 h = ldg_v4(p);
#pragma unroll
    for (int i = 0; i < NV; ++i) raw[i] = i < NS ? ldg_v4(p + 1 + i) : make_uint4(0u, 0u, 0u, 0u);
    sc[0] = __uint_as_float(h.x);
    sc[1] = __uint_as_float(h.y);
    sc[2] = __uint_as_float(h.z);
  }
  // The header and the code vectors that hold w_gamma.
  __device__ __forceinline__ void load_gamma(const DevTree &tr, uint32_t leaf) {
    constexpr int V0 = KP / 16, V1 = (2 * KP + 15) / 16;
    const uint4 *p = reinterpret_cast<const uint4 *>(static_cast<const unsigned char *>(tr.rec) +
                                                     (size_t)leaf * tr.rec_stride);
    const uint4 h = ldg_v4(p);
#pragma unroll
    for (int i = 0; i < NV; ++i) raw[i] = (i >= V0 && i < V1) ? ldg_v4(p + 1 + i) : make_uint4(0u, 0u, 0u, 0u);
    sc[0] = __uint_as_float(h.x);
    sc[1] = __uint_as_float(h.y);
    sc[2] = __uint_as_float(h.z);
  }
  // The header and the code vectors that hold w_sigma (a density-only pass).
  __device__ __forceinline__ void load_sigma(const DevTree &tr, uint32_t leaf) {
    constexpr int NS = (KP + 15) / 16;
    const uint4 *p = reinterpret_cast<const uint4 *>(static_cast<const unsigned char *>(tr.rec) +
                                                     (size_t)leaf * tr.rec_stride);
    const uint4 h = ldg_v4(p);
#pragma unroll
    for (int i = 0; i < NV; ++i) raw[i] = i < NS ? ldg_v4(p + 1 + i) : make_uint4(0u, 0u, 0u, 0u);
    sc[0] = __uint_as_float(h.x);
    sc[1] = __uint_as_float(h.y);
    sc[2] = __uint_as_float(h.z);
  }
  __device__ __forceinline__ static void prefetch_sigma_l2(const DevTree &tr, uint32_t leaf) {
    const char *p = reinterpret_cast<const char *>(tr.rec) + (size_t)leaf * tr.rec_stride;
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p + 16 + KP - 1));
  }
  __device__ __forceinline__ static void prefetch_l2(const DevTree &tr, uint32_t leaf) {
    const char *p = reinterpret_cast<const char *>(tr.rec) + (size_t)leaf * tr.rec_stride;
    constexpr int kBytes = 16 + NV * 16;
#pragma unroll
    for (int b = 0; b < kBytes; b += 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(p + b));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p + kBytes - 1));
  }
  // Entry j's code value, not yet scaled (j is a compile-time index once the
  // callers' loops are unrolled).
  __device__ __forceinline__ float code(int j) const {
    const uint4 v = raw[j >> 4];
    const int w = (j >> 2) & 3;
    const unsigned int word = w == 0 ? v.x : (w == 1 ? v.y : (w == 2 ? v.z : v.w));
    const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)((word >> (16 * ((j >> 1) & 1))) & 0xFFFFu),
                                                     __NV_E4M3);
    const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&h));
    return (j & 1) ? f.y : f.x;
  }
  // The scale is a power of two, so applying it to a finished dot product
  // gives the same FP32 result as scaling every entry first.
  __device__ __forceinline__ float sig(int k) const { return code(k); }
  __device__ __forceinline__ float gam(int k) const { return code(KP + k); }
  __device__ __forceinline__ float hh(int ch, int i) const { return code(2 * KP + ch * NH + i); }
  __device__ __forceinline__ float scale_sigma() const { return sc[0]; }
  __device__ __forceinline__ float scale_gamma() const { return sc[1]; }
  __device__ __forceinline__ float scale_hh() const { return sc[2]; }
};

// Per-ray constants: interpolated basis rows and the view-direction harmonics.
template <int KP, int DEG>
struct RayConst {
  float a[KP], b[KP];
  float Y[(DEG + 1) * (DEG + 1)];
};

// Frame coordinate u = t (T - 1) (t clamped to [0, 1]); rows lerped in u.
template <int KP, int DEG>
__device__ __forceinline__ void ray_const_basis(const DevTree &tr, float u, RayConst<KP, DEG> &rc) {
  const float umax = (float)(tr.T - 1);
  u = fminf(fmaxf(u, 0.f), umax);
  int f0 = min((int)floorf(u), tr.T - 1);
  const int f1 = min(f0 + 1, tr.T - 1);
  const float fr = u - (float)f0;
  const float *A0 = tr.A + (size_t)f0 * KP, *A1 = tr.A + (size_t)f1 * KP;
  const float *B0 = tr.B + (size_t)f0 * KP, *B1 = tr.B + (size_t)f1 * KP;
#pragma unroll
  for (int k = 0; k < KP; ++k) {
    rc.a[k] = (1.f - fr) * __ldg(A0 + k) + fr * __ldg(A1 + k);
    rc.b[k] = (1.f - fr) * __ldg(B0 + k) + fr * __ldg(B1 + k);
  }
}

__device__ __forceinline__ float sigmoidf_fast(float x) { return 1.f / (1.f + __expf(-x)); }

// One Adam step of one entry (Sec. 4.3 "Optimization"): moments
// m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2, then
// w <- w - lr m_hat / (sqrt(v_hat) + eps) with m_hat = m / c1 and
// v_hat = v / c2 (bias corrections c = 1 - b^step), taken as
// (lr / c1) m / (sqrt(v (1 / c2)) + eps) with one fast division.
__device__ __forceinline__ void adam_entry(float g, float b1, float b2, float lr_c1, float inv_c2, float eps, float &w,
                                           float &m, float &v) {
  m = fmaf(b1, m, (1.f - b1) * g);
  v = fmaf(b2, v, (1.f - b2) * g * g);
  w -= __fdividef(lr_c1 * m, sqrtf(v * inv_c2) + eps);
}

// float -> bfloat16 bits, round to nearest even (a NaN stays a quiet NaN).
__device__ __forceinline__ unsigned short f32_to_bf16_rne(float f) {
  unsigned int u = __float_as_uint(f);
  if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x007FFFFFu)) return (unsigned short)((u >> 16) | 0x40u);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (unsigned short)(u >> 16);
}

// Opacity of a segment of optical depth sd, 1 - exp(-sd), without the
// cancellation of 1 - expf(-sd) when sd is small (a thin or faint segment):
// there 1 - expf(-sd) carries an absolute error of an FP32 ulp of 1, which is
// a relative error of ~1e-7 / sd.  The transmittance factor exp(-sd) itself is
// accurate relative to its value and keeps using expf.
__device__ __forceinline__ float alpha_of(float sd) { return -expm1f(-sd); }

// Evaluated sample: density, hyper-angle terms and colour of one leaf.
template <int DEG>
struct Sample {
  float pre_sigma, sigma;
  float s_gamma;        // sigmoid(b . w_gamma); gamma = pi * s_gamma
  float cg, sg;         // cos, sin of gamma
  float z[3], c[3];     // pre-activation colour, colour
  float u[3];           // d z / d gamma (evaluated when the adjoint asks for it)
  float R[(DEG + 1) * (DEG + 2) / 2];
};

// Where a ray's interpolated basis rows a(u), b(u) live: registers
// (RegRows) or a per-thread column of shared memory (SmemRows, entry k at
// p[k * stride], b after a).
template <int KP>
struct RegRows {
  const float *a, *b;
  __device__ __forceinline__ float A(int k) const { return a[k]; }
  __device__ __forceinline__ float B(int k) const { return b[k]; }
};
template <int KP>
struct SmemRows {
  const float *p;
  int stride;
  __device__ __forceinline__ float A(int k) const { return p[k * stride]; }
  __device__ __forceinline__ float B(int k) const { return p[(KP + k) * stride]; }
};

// Frame coordinate u = t (T - 1), rows lerped in u, written to shared memory.
template <int KP>
__device__ __forceinline__ void rows_to_smem(const DevTree &tr, float u, float *p, int stride) {
  const float umax = (float)(tr.T - 1);
  u = fminf(fmaxf(u, 0.f), umax);
  const int f0 = min((int)floorf(u), tr.T - 1);
  const int f1 = min(f0 + 1, tr.T - 1);
  const float fr = u - (float)f0;
  const float *A0 = tr.A + (size_t)f0 * KP, *A1 = tr.A + (size_t)f1 * KP;
  const float *B0 = tr.B + (size_t)f0 * KP, *B1 = tr.B + (size_t)f1 * KP;
#pragma unroll
  for (int k = 0; k < KP; ++k) {
    p[k * stride] = (1.f - fr) * __ldg(A0 + k) + fr * __ldg(A1 + k);
    p[(KP + k) * stride] = (1.f - fr) * __ldg(B0 + k) + fr * __ldg(B1 + k);
  }
}

// Pre-activation density a(u) . w_sigma (Eq. project-sigma), four independent
// FMA chains; the slice kernel forms it with the same operations.
template <int KP, typename Rows, typename Rec>
__device__ __forceinline__ float pre_sigma_of(const Rows &rows, const Rec &r) {
  // four partial sums: independent FMA chains
  float p4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < KP; ++k) p4[k & 3] = fmaf(rows.A(k), r.sig(k), p4[k & 3]);
  return ((p4[0] + p4[1]) + (p4[2] + p4[3])) * r.scale_sigma();
}

// Eq. project-sigma, Eq. project-gamma, Eq. HH-color-2 for one leaf.  When the
// density is zero the sample cannot contribute and colour is not evaluated.
// With kDz the gamma-derivative of each channel's pre-activation is formed
// from the same inner sums sum_m w Y (the adjoint then needs no coefficient
// after this call).
template <int KP, int DEG, typename E, typename Rows, bool kDz = false>
__device__ __forceinline__ void eval_sample(const DevTree &tr, const Rows &rows, const float *Y,
                                            const LeafRecord<KP, DEG, E> &r, int act, Sample<DEG> &s) {
  const float ps = pre_sigma_of<KP>(rows, r);
  s.pre_sigma = ps;
  s.sigma = fmaxf(ps, 0.f);
  if (!(s.sigma > 0.f)) return;
  float q4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < KP; ++k) q4[k & 3] = fmaf(rows.B(k), r.gam(k), q4[k & 3]);
  const float pg = ((q4[0] + q4[1]) + (q4[2] + q4[3])) * r.scale_gamma();
  s.s_gamma = sigmoidf_fast(pg);
  sincospif(s.s_gamma, &s.sg, &s.cg);
  float dR[(DEG + 1) * (DEG + 2) / 2];
  hh_radial<DEG, kDz>(s.cg, s.sg, tr.hh_norm, s.R, dR);
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    float z = 0.f, u = 0.f;
#pragma unroll
    for (int n = 0; n <= DEG; ++n)
#pragma unroll
      for (int l = 0; l <= n; ++l) {
        float acc = 0.f;
#pragma unroll
        for (int m = -l; m <= l; ++m) acc = fmaf(r.hh(ch, hh_index(n, l, m)), Y[l * l + l + m], acc);
        z = fmaf(acc, s.R[radial_index(n, l)], z);
        if (kDz) u = fmaf(acc, dR[radial_index(n, l)], u);
      }
    z *= r.scale_hh();
    if (kDz) u *= r.scale_hh();
    s.z[ch] = z;
    s.u[ch] = u;
    s.c[ch] = act == 0 ? sigmoidf_fast(z) : z;
  }
}

template <int KP, int DEG, typename E>
__device__ __forceinline__ void eval_sample(const DevTree &tr, const RayConst<KP, DEG> &rc,
                                            const LeafRecord<KP, DEG, E> &r, int act, Sample<DEG> &s) {
  eval_sample<KP, DEG, E>(tr, RegRows<KP>{rc.a, rc.b}, rc.Y, r, act, s);
}

// ---------------------------------------------------------------------------
// Time slices (Sec. 7; the caption of the HH-colour figure): at a fixed time
// gamma(t) is a constant and the 4D harmonics reduce to 3D spherical
// harmonics.  A slice record holds [sigma, 0, 0, 0] then the coefficients
// s[ch][l^2 + l + m] = sum_{n >= l} w[ch][n,l,m] R_nl(gamma(t)), FP32.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int slice_len(int deg) { return 4 + 3 * (deg + 1) * (deg + 1); }
__host__ __device__ constexpr int slice_min_stride(int deg) { return (slice_len(deg) + 3) / 4 * 4; }

// Density and colour of one leaf of a slice seen along unit direction with
// harmonics Y.
template <int DEG>
__device__ __forceinline__ void shade_slice(const float *slice, int stride, uint32_t leaf, const float *Y, int act,
                                            float &sigma, float c[3]) {
  constexpr int NY = (DEG + 1) * (DEG + 1), NV = slice_min_stride(DEG) / 4;
  const uint4 *p = reinterpret_cast<const uint4 *>(slice + (size_t)leaf * stride);
  float v[NV * 4];
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    const uint4 q = ldg_v4(p + i);
    v[4 * i] = __uint_as_float(q.x);
    v[4 * i + 1] = __uint_as_float(q.y);
    v[4 * i + 2] = __uint_as_float(q.z);
    v[4 * i + 3] = __uint_as_float(q.w);
  }
  sigma = v[0];
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    float z = 0.f;
#pragma unroll
    for (int k = 0; k < NY; ++k) z = fmaf(v[4 + ch * NY + k], Y[k], z);
    c[ch] = act == 0 ? sigmoidf_fast(z) : z;
  }
}

__device__ __forceinline__ void slice_prefetch_l2(const float *slice, int stride, int deg, uint32_t leaf) {
  const char *p = reinterpret_cast<const char *>(slice + (size_t)leaf * stride);
  const int bytes = slice_min_stride(deg) * 4;
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p + bytes - 1));
}

// Rays in structure-of-arrays form.
struct DevRays {
  const float *ox, *oy, *oz, *dx, *dy, *dz, *t;
  long long n;
  float t_scalar;
};

// Rays are read once per launch: loads with the evict-first (streaming)
// policy leave L2 to the records and the walk's tables.
__device__ __forceinline__ void load_ray(const DevRays &r, long long i, float o[3], float d[3], float &t) {
  o[0] = __ldcs(r.ox + i);
  o[1] = __ldcs(r.oy + i);
  o[2] = __ldcs(r.oz + i);
  d[0] = __ldcs(r.dx + i);
  d[1] = __ldcs(r.dy + i);
  d[2] = __ldcs(r.dz + i);
  t = r.t ? __ldcs(r.t + i) : r.t_scalar;
  t = fminf(fmaxf(t, 0.f), 1.f);
}

struct DevOut {
  float *rgb, *alpha, *depth, *tau;
  int *nseg;
};

}  // namespace neuvv
