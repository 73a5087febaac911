// C ABI of the VOctree renderer: tree upload, argument checking, launch
// configuration and dispatch to the kernels.  See include/neuvv.h for the
// contract of every entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/neuvv.h"
#include "neuvv_kernels.h"

using namespace neuvv;

namespace {

thread_local std::string g_err;

neuvv_status fail(neuvv_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

neuvv_status cuda_fail(cudaError_t e, const char *what) {
  return fail(e == cudaErrorMemoryAllocation ? NEUVV_ERR_OOM : NEUVV_ERR_CUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

// Switches to the tree's device for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

int kpad_of(int K) { return K <= 8 ? 8 : (K <= 16 ? 16 : 32); }

// Abar_{n,l} = 2^l l! sqrt(2(n+1)(n-l)! / (pi (n+l+1)!))  (orthonormal on S^3)
double hh_norm_value(int n, int l) {
  auto fact = [](int k) {
    double r = 1.0;
    for (int i = 2; i <= k; ++i) r *= i;
    return r;
  };
  return std::ldexp(1.0, l) * fact(l) * std::sqrt(2.0 * (n + 1) * fact(n - l) / (M_PI * fact(n + l + 1)));
}

// float -> bfloat16 bits, round to nearest even (NaN kept quiet).
uint16_t bf16_bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x007FFFFFu)) return (uint16_t)((u >> 16) | 0x40u);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

constexpr int kWorkSlots = 4;  // fwd, bwd, compose, spare

}  // namespace

struct neuvv_tree {
  neuvv_tree_info info{};
  uint32_t *child = nullptr;
  uint32_t *bricks = nullptr;
  uint32_t *coarse = nullptr;
  int brick_level = 0, brick_first = 0, brick_count = 0;
  void *rec = nullptr;
  float *master = nullptr, *m = nullptr, *v = nullptr;
  float *A = nullptr, *B = nullptr;
  uint32_t *status = nullptr;
  unsigned long long *work = nullptr;
  GatherWs gws{};           // workspace of the leaf-major adjoint (neuvv_tree_reserve_adjoint)
  bool master_is_storage = false;
  float bmin[3], bmax[3], scale[3];
  float hh_norm[16];
  int num_sms = 0;
  LaunchCfg plain{128, 1, 1, 0, 0, 0};
  LaunchCfg packet{64, 8, 16, 0, 1, 0};
  LaunchCfg compose{128, 1, 1, 0, 1, 0};
  int step_cap = 0;             // walk steps per ray (0: 3 * 2^depth + 8)
  int wait_polls = 1 << 22;     // polls of a bounded device wait
  std::vector<neuvv_tune_entry> tune_table;  // candidates of the last neuvv_autotune and their times
  int tune_cached = 0;                       // 1: that call reused an earlier choice
  int packet_tiles = NEUVV_TILES_8X4;        // pixel tile of camera packets (neuvv_autotune_tiles)
};

namespace {

void free_gather(neuvv_tree *t) {
  cudaFree(t->gws.fac);
  cudaFree(t->gws.off);
  cudaFree(t->gws.cur);
  cudaFree(t->gws.part);
  t->gws = GatherWs{};
}

DevTree dev_tree(const neuvv_tree *t) {
  DevTree d;
  d.child = t->child;
  d.rec = t->rec;
  d.A = t->A;
  d.B = t->B;
  d.status = t->status;
  d.n_nodes = t->info.n_nodes;
  d.n_leaves = t->info.n_leaves;
  for (int a = 0; a < 3; ++a) {
    d.bmin[a] = t->bmin[a];
    d.bmax[a] = t->bmax[a];
    d.scale[a] = t->scale[a];
  }
  for (int k = 0; k < 16; ++k) d.hh_norm[k] = t->hh_norm[k];
  d.depth = t->info.depth;
  d.T = t->info.T;
  d.K = t->info.K;
  d.rec_stride = t->info.rec_stride;
  d.smem_nodes = 0;
  d.bricks = t->bricks;
  d.brick_level = t->brick_level;
  d.brick_first = t->brick_first;
  d.brick_count = t->brick_count;
  d.coarse = t->coarse;
  d.path_words = t->coarse ? 0 : kPathWords;
  d.step_cap = t->step_cap;
  d.wait_polls = t->wait_polls;
  return d;
}

neuvv_status check_rays(const neuvv_rays *r) {
  if (!r) return fail(NEUVV_ERR_INVALID_ARG, "rays is NULL");
  if (r->n < 0) return fail(NEUVV_ERR_INVALID_ARG, "rays->n < 0");
  if (r->n > 0 && (!r->ox || !r->oy || !r->oz || !r->dx || !r->dy || !r->dz))
    return fail(NEUVV_ERR_INVALID_ARG, "ray origin/direction pointer is NULL");
  if (r->n > ((int64_t)1 << 37)) return fail(NEUVV_ERR_INVALID_ARG, "too many rays");
  return NEUVV_OK;
}

DevRays dev_rays(const neuvv_rays *r, float t) {
  DevRays d{r->ox, r->oy, r->oz, r->dx, r->dy, r->dz, r->t, (long long)r->n, t};
  return d;
}

// Device view of a caller's segment log buffer (layout private to the
// library): 64-byte header, heads, key and order [n_packets], perm [n_rays],
// the sort bins, next [n_chunks], then leaf and chord planes of n_chunks x
// kLogRounds x 32 entries.  n_chunks = 0 when the buffer is absent or too
// small for one chunk.  *chunk_bytes (nullable) receives the bytes from the
// start of next[] to the end of the buffer (scratch for a ray order before
// the forward fills the chunks).
SampleLog log_view(void *base, int64_t bytes, int64_t n_rays, int64_t *chunk_bytes = nullptr) {
  SampleLog l;
  std::memset(&l, 0, sizeof l);
  if (chunk_bytes) *chunk_bytes = 0;
  if (!base || bytes < 64) return l;
  char *p = static_cast<char *>(base);
  l.counter = reinterpret_cast<unsigned long long *>(p);
  l.header = reinterpret_cast<uint32_t *>(p + 8);
  const int64_t n_packets = (n_rays + 31) / 32;
  const int64_t pk_bytes = (4 * n_packets + 15) / 16 * 16;
  const int64_t perm_bytes = (4 * n_rays + 15) / 16 * 16;
  const int64_t fixed = 64 + 3 * pk_bytes + perm_bytes + 4 * kSortBins;
  const int64_t per_chunk = 4 + (int64_t)kLogRounds * 32 * 8;
  const int64_t avail = bytes - fixed - 16;
  if (avail < per_chunk) return l;
  int64_t nc = avail / per_chunk;
  if (nc > (int64_t)0x7FFFFFFF) nc = 0x7FFFFFFF;
  l.heads = reinterpret_cast<uint32_t *>(p + 64);
  l.key = reinterpret_cast<uint32_t *>(p + 64 + pk_bytes);
  l.order = reinterpret_cast<uint32_t *>(p + 64 + 2 * pk_bytes);
  l.perm = reinterpret_cast<uint32_t *>(p + 64 + 3 * pk_bytes);
  l.bins = reinterpret_cast<uint32_t *>(p + 64 + 3 * pk_bytes + perm_bytes);
  l.next = reinterpret_cast<uint32_t *>(p + fixed);
  const int64_t leaf_off = (fixed + 4 * nc + 15) / 16 * 16;
  l.leaf = reinterpret_cast<uint32_t *>(p + leaf_off);
  l.dt = reinterpret_cast<float *>(p + leaf_off + nc * kLogRounds * 32 * 4);
  l.n_chunks = (uint32_t)nc;
  if (chunk_bytes) *chunk_bytes = bytes - fixed;
  return l;
}

neuvv_status check_log(const neuvv_out *out) {
  if (out && out->log && (((uintptr_t)out->log & 15) != 0 || out->log_bytes < 0))
    return fail(NEUVV_ERR_INVALID_ARG, "out->log must be 16-byte aligned with log_bytes >= 0");
  return NEUVV_OK;
}

// Marks a caller's log empty (a call that does not fill it).
cudaError_t clear_log(const neuvv_out *out, cudaStream_t st) {
  if (!out || !out->log || out->log_bytes < 64) return cudaSuccess;
  return cudaMemsetAsync(static_cast<char *>(out->log) + 8, 0, 24, st);
}

neuvv_status check_opts(const neuvv_render_opts *o) {
  if (!o) return fail(NEUVV_ERR_INVALID_ARG, "opts is NULL");
  if (!(o->t_stop >= 0.f && o->t_stop < 1.f)) return fail(NEUVV_ERR_INVALID_ARG, "t_stop must be in [0, 1)");
  if (o->color_act != NEUVV_ACT_SIGMOID && o->color_act != NEUVV_ACT_IDENTITY)
    return fail(NEUVV_ERR_INVALID_ARG, "unknown color_act %d", o->color_act);
  if (o->kernel < NEUVV_KERNEL_AUTO || o->kernel > NEUVV_KERNEL_PACKET)
    return fail(NEUVV_ERR_INVALID_ARG, "unknown kernel %d", o->kernel);
  if (o->compose_mode != NEUVV_COMPOSE_SORTED && o->compose_mode != NEUVV_COMPOSE_ALG1)
    return fail(NEUVV_ERR_INVALID_ARG, "unknown compose_mode %d", o->compose_mode);
  return NEUVV_OK;
}

neuvv_status check_time(const neuvv_rays *r, float t) {
  if (!r->t && !(t >= 0.f && t <= 1.f)) return fail(NEUVV_ERR_INVALID_ARG, "scalar t must be in [0, 1]");
  return NEUVV_OK;
}

// Writes, for the subtree of `node` (at `level`, origin o in brick-local
// finest cells), the entry (level << 28 | id) of the tree cell holding each
// finest cell of the brick (side 2^sh).
void fill_brick(const uint32_t *child, uint32_t node, int level, int depth, int sh, int ox, int oy, int oz,
                uint32_t *brick) {
  const int half = 1 << (depth - level - 1);
  for (int c = 0; c < 8; ++c) {
    const int cx = ox + ((c >> 2) & 1) * half, cy = oy + ((c >> 1) & 1) * half, cz = oz + (c & 1) * half;
    const uint32_t e = child[(size_t)node * 8 + c];
    if (e != kEmpty && !(e & kLeafBit)) {
      fill_brick(child, e, level + 1, depth, sh, cx, cy, cz, brick);
      continue;
    }
    const uint32_t id = e == kEmpty ? kBrickEmpty : (e & ~kLeafBit);
    const uint32_t v = ((uint32_t)(level + 1) << 28) | id;
    for (int x = cx; x < cx + half; ++x)
      for (int y = cy; y < cy + half; ++y)
        for (int z = cz; z < cz + half; ++z) brick[((size_t)x << (2 * sh)) | ((size_t)y << sh) | (size_t)z] = v;
  }
}

// Brick-map words of the subtree of `node` (an internal node at `level`, at
// brick-map cell (ox, oy, oz) of level Lb): leaves fill the cells they cover,
// internal nodes at level Lb are bricks, empty children are left as they are.
void fill_coarse(const uint32_t *child, uint32_t node, int level, int Lb, int ox, int oy, int oz, int64_t first,
                 uint32_t *map) {
  const int half = 1 << (Lb - level - 1);
  for (int c = 0; c < 8; ++c) {
    const int cx = ox + ((c >> 2) & 1) * half, cy = oy + ((c >> 1) & 1) * half, cz = oz + (c & 1) * half;
    const uint32_t e = child[(size_t)node * 8 + c];
    if (e == kEmpty) continue;
    if (!(e & kLeafBit)) {
      if (level + 1 == Lb) {
        map[((size_t)cx << (2 * Lb)) | ((size_t)cy << Lb) | (size_t)cz] = (uint32_t)((int64_t)e - first);
      } else {
        fill_coarse(child, e, level + 1, Lb, cx, cy, cz, first, map);
      }
      continue;
    }
    const uint32_t v = ((uint32_t)(level + 1) << 28) | (e & ~kLeafBit);
    for (int x = cx; x < cx + half; ++x)
      for (int y = cy; y < cy + half; ++y)
        for (int z = cz; z < cz + half; ++z) map[((size_t)x << (2 * Lb)) | ((size_t)y << Lb) | (size_t)z] = v;
  }
}

// Empty boxes of the brick map's empty cells.  Each starts as the cube of
// radius k-1 around the cell (k its Chebyshev distance to the nearest
// occupied cell) and grows, face by face (+x, -x, +y, -y, +z, -z, in two
// rounds, the first capped at the cube's size), as far as it stays empty; a
// box-emptiness test is O(1) on a prefix sum of the occupancy.  The word of
// an empty cell is then (kCoarseEmpty << 28) | (s << 24) | the six extents
// (cells below and above the cell on x, y, z, 4 bits each, in units of 2^s,
// rounded down): s is the smallest shift that fits the largest extent.
void coarse_empty_boxes(const std::vector<uint8_t> &occ, const std::vector<int32_t> &dist, int n,
                        std::vector<uint32_t> &map) {
  const size_t m = (size_t)n + 1;
  std::vector<int32_t> P(m * m * m, 0);
  auto pa = [m](int x, int y, int z) { return ((size_t)x * m + y) * m + z; };
  for (int x = 0; x < n; ++x)
    for (int y = 0; y < n; ++y)
      for (int z = 0; z < n; ++z)
        P[pa(x + 1, y + 1, z + 1)] = occ[((size_t)x * n + y) * n + z] + P[pa(x, y + 1, z + 1)] +
                                     P[pa(x + 1, y, z + 1)] + P[pa(x + 1, y + 1, z)] - P[pa(x, y, z + 1)] -
                                     P[pa(x, y + 1, z)] - P[pa(x + 1, y, z)] + P[pa(x, y, z)];
  // occupied cells in [lo, hi] (inclusive) per axis
  auto count = [&](const int lo[3], const int hi[3]) {
    const int x0 = lo[0], y0 = lo[1], z0 = lo[2], x1 = hi[0] + 1, y1 = hi[1] + 1, z1 = hi[2] + 1;
    return P[pa(x1, y1, z1)] - P[pa(x0, y1, z1)] - P[pa(x1, y0, z1)] - P[pa(x1, y1, z0)] + P[pa(x0, y0, z1)] +
           P[pa(x0, y1, z0)] + P[pa(x1, y0, z0)] - P[pa(x0, y0, z0)];
  };
  for (int x = 0; x < n; ++x)
    for (int y = 0; y < n; ++y)
      for (int z = 0; z < n; ++z) {
        const size_t q = ((size_t)x * n + y) * n + z;
        if (occ[q]) continue;
        const int c[3] = {x, y, z}, r = std::max(dist[q] - 1, 0);
        int lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
          lo[a] = std::max(c[a] - r, 0);
          hi[a] = std::min(c[a] + r, n - 1);
        }
        for (int round = 0; round < 2; ++round)
          for (int f = 0; f < 6; ++f) {
            const int a = f >> 1;
            const bool up = (f & 1) == 0;
            const int room = up ? n - 1 - hi[a] : lo[a];
            int best = 0, top = round == 0 ? std::min(room, 2 * r + 1) : room;
            // largest extension g <= top whose slab keeps the box empty (monotone in g)
            int l = 1, h = top;
            while (l <= h) {
              const int g = (l + h) / 2;
              int slo[3] = {lo[0], lo[1], lo[2]}, shi[3] = {hi[0], hi[1], hi[2]};
              if (up) { slo[a] = hi[a] + 1; shi[a] = hi[a] + g; }
              else { slo[a] = lo[a] - g; shi[a] = lo[a] - 1; }
              if (count(slo, shi) == 0) { best = g; l = g + 1; }
              else h = g - 1;
            }
            if (up) hi[a] += best;
            else lo[a] -= best;
          }
        int e[6], emax = 0;
        for (int a = 0; a < 3; ++a) {
          e[2 * a] = c[a] - lo[a];
          e[2 * a + 1] = hi[a] - c[a];
          emax = std::max(emax, std::max(e[2 * a], e[2 * a + 1]));
        }
        uint32_t sh = 0;
        while ((emax >> sh) > 15) ++sh;
        uint32_t w = (kCoarseEmpty << 28) | (sh << 24);
        for (int i = 0; i < 6; ++i) w |= (uint32_t)(e[i] >> sh) << (4 * i);
        map[q] = w;
      }
}

// Empty boxes inside bricks.  For each empty finest cell of a brick the box
// starts as the empty octree node holding it (aligned, from the entry's
// level) and grows face by face (+x, -x, +y, -y, +z, -z, one binary search
// each) as far as it stays empty within the 3x3x3 brick-map neighbourhood of
// the brick (24^3 finest cells, occupancy from the neighbours' bricks and
// leaves, cells outside the root box counted as occupied).  Its extents below
// and above the cell (at most 15 per side) go into the entry as
// kBrickBoxBase | extents (4 bits each: x in bits 0-7, y 8-15, z 16-23, below
// in the low nibble); the level bits stay.  Bricks are split over host
// threads; `in` is only read and `out` only written.
void brick_empty_boxes(const std::vector<uint32_t> &in, std::vector<uint32_t> &out, const std::vector<uint32_t> &map,
                       int nc, int depth) {
  constexpr int W = 24, M = W + 1;
  const int64_t n_bricks = (int64_t)(in.size() / 512);
  // brick index -> its brick-map cell
  std::vector<int32_t> cell_of_brick(n_bricks, -1);
  for (size_t q = 0; q < map.size(); ++q)
    if ((map[q] >> 28) == 0 && (int64_t)(map[q] & 0x0FFFFFFFu) < n_bricks) cell_of_brick[map[q] & 0x0FFFFFFFu] = (int32_t)q;
  auto work = [&](int64_t b0, int64_t b1) {
    std::vector<uint8_t> occ(W * W * W);
    std::vector<int32_t> P(M * M * M);
    auto pa = [&](int x, int y, int z) { return (x * M + y) * M + z; };
    auto count = [&](const int lo[3], const int hi[3]) {
      const int x0 = lo[0], y0 = lo[1], z0 = lo[2], x1 = hi[0] + 1, y1 = hi[1] + 1, z1 = hi[2] + 1;
      return P[pa(x1, y1, z1)] - P[pa(x0, y1, z1)] - P[pa(x1, y0, z1)] - P[pa(x1, y1, z0)] + P[pa(x0, y0, z1)] +
             P[pa(x0, y1, z0)] + P[pa(x1, y0, z0)] - P[pa(x0, y0, z0)];
    };
    for (int64_t b = b0; b < b1; ++b) {
      const int32_t q = cell_of_brick[b];
      if (q < 0) continue;
      const int cx = q / (nc * nc), cy = (q / nc) % nc, cz = q % nc;
      // occupancy of the window: finest cells of the 27 brick-map cells around
      for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dz = -1; dz <= 1; ++dz) {
            const int ux = cx + dx, uy = cy + dy, uz = cz + dz;
            const bool inside = ux >= 0 && uy >= 0 && uz >= 0 && ux < nc && uy < nc && uz < nc;
            const uint32_t w = inside ? map[((size_t)ux * nc + uy) * nc + uz] : 0u;
            const uint32_t kind = w >> 28;
            const uint32_t *nb = inside && kind == 0 ? in.data() + (size_t)(w & 0x0FFFFFFFu) * 512 : nullptr;
            for (int x = 0; x < 8; ++x)
              for (int y = 0; y < 8; ++y)
                for (int z = 0; z < 8; ++z) {
                  uint8_t o;
                  if (!inside) o = 1;
                  else if (kind == kCoarseEmpty) o = 0;
                  else if (kind != 0) o = 1;
                  else o = (nb[(x << 6) | (y << 3) | z] & 0x0FFFFFFFu) < kBrickBoxBase;
                  occ[((dx + 1) * 8 + x) * W * W + ((dy + 1) * 8 + y) * W + (dz + 1) * 8 + z] = o;
                }
          }
      for (int x = 0; x < W; ++x)
        for (int y = 0; y < W; ++y)
          for (int z = 0; z < W; ++z)
            P[pa(x + 1, y + 1, z + 1)] = occ[(x * W + y) * W + z] + P[pa(x, y + 1, z + 1)] + P[pa(x + 1, y, z + 1)] +
                                         P[pa(x + 1, y + 1, z)] - P[pa(x, y, z + 1)] - P[pa(x, y + 1, z)] -
                                         P[pa(x + 1, y, z)] + P[pa(x, y, z)];
      for (int x = 0; x < 8; ++x)
        for (int y = 0; y < 8; ++y)
          for (int z = 0; z < 8; ++z) {
            const size_t k = (size_t)b * 512 + ((x << 6) | (y << 3) | z);
            const uint32_t v = in[k];
            if ((v & 0x0FFFFFFFu) != kBrickEmpty) continue;
            // the empty node holding the cell (aligned, from its level)
            const int size = 1 << std::max(0, depth - (int)(v >> 28));
            const int c[3] = {8 + x, 8 + y, 8 + z};
            int lo[3], hi[3];
            for (int a = 0; a < 3; ++a) {
              lo[a] = 8 + ((c[a] - 8) & -size);
              hi[a] = lo[a] + size - 1;
            }
            for (int f = 0; f < 6; ++f) {
              const int a = f >> 1;
              const bool up = (f & 1) == 0;
              int best = 0, l = 1, h = up ? W - 1 - hi[a] : lo[a];
              while (l <= h) {
                const int g = (l + h) / 2;
                int slo[3] = {lo[0], lo[1], lo[2]}, shi[3] = {hi[0], hi[1], hi[2]};
                if (up) { slo[a] = hi[a] + 1; shi[a] = hi[a] + g; }
                else { slo[a] = lo[a] - g; shi[a] = lo[a] - 1; }
                if (count(slo, shi) == 0) { best = g; l = g + 1; }
                else h = g - 1;
              }
              if (up) hi[a] += best;
              else lo[a] -= best;
            }
            uint32_t ext = 0;
            for (int a = 0; a < 3; ++a) {
              ext |= (uint32_t)std::min(c[a] - lo[a], 15) << (8 * a);
              ext |= (uint32_t)std::min(hi[a] - c[a], 15) << (8 * a + 4);
            }
            out[k] = (v & 0xF0000000u) | kBrickBoxBase | ext;
          }
    }
  };
  const int nt = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  std::vector<std::thread> th;
  for (int i = 0; i < nt; ++i) th.emplace_back(work, n_bricks * i / nt, n_bricks * (i + 1) / nt);
  for (auto &x : th) x.join();
}

// Chebyshev (L-infinity) distance from every cell of an n^3 grid to the
// nearest occupied cell (0 for occupied cells; `far` when there is none):
// the one-dimensional distance along z, then two passes of
// g'(y) = min over y' of max(|y - y'|, g(y')) along y and along x.
std::vector<int32_t> chebyshev_distance(const std::vector<uint8_t> &occ, int n, int32_t far) {
  const size_t n3 = (size_t)n * n * n;
  std::vector<int32_t> g(n3), h(n3);
  auto at = [n](int x, int y, int z) { return ((size_t)x * n + y) * n + z; };
  for (int x = 0; x < n; ++x)
    for (int y = 0; y < n; ++y) {
      int32_t d = far;
      for (int z = 0; z < n; ++z) {
        d = occ[at(x, y, z)] ? 0 : std::min(far, d + 1);
        g[at(x, y, z)] = d;
      }
      d = far;
      for (int z = n - 1; z >= 0; --z) {
        d = occ[at(x, y, z)] ? 0 : std::min(far, d + 1);
        g[at(x, y, z)] = std::min(g[at(x, y, z)], d);
      }
    }
  // min-max passes; the search around y stops once |y - y'| reaches the best
  for (int pass = 0; pass < 2; ++pass) {
    for (int u = 0; u < n; ++u)
      for (int v = 0; v < n; ++v)
        for (int y = 0; y < n; ++y) {
          auto idx = [&](int yy) { return pass == 0 ? at(u, yy, v) : at(yy, u, v); };
          int32_t best = g[idx(y)];
          for (int r = 1; r < best; ++r) {
            if (y - r >= 0) best = std::min(best, std::max(r, g[idx(y - r)]));
            if (y + r < n) best = std::min(best, std::max(r, g[idx(y + r)]));
            if (y - r < 0 && y + r >= n) break;
          }
          h[idx(y)] = best;
        }
    g.swap(h);
  }
  return g;
}

}  // namespace

extern "C" {

const char *neuvv_last_error(void) { return g_err.c_str(); }

neuvv_status neuvv_tree_create(const neuvv_tree_desc *desc, neuvv_tree **out) {
  if (!desc || !out) return fail(NEUVV_ERR_INVALID_ARG, "desc/out is NULL");
  *out = nullptr;
  const neuvv_tree_desc &d = *desc;
  if (d.depth < 1 || d.depth > 14) return fail(NEUVV_ERR_INVALID_ARG, "depth must be in [1, 14]");
  if (d.K < 1 || d.K > 32) return fail(NEUVV_ERR_INVALID_ARG, "K must be in [1, 32]");
  if (d.T < 2) return fail(NEUVV_ERR_INVALID_ARG, "T must be >= 2");
  if (d.hh_degree < 1 || d.hh_degree > 3) return fail(NEUVV_ERR_INVALID_ARG, "hh_degree must be in [1, 3]");
  if (d.dtype != NEUVV_F32 && d.dtype != NEUVV_BF16 && d.dtype != NEUVV_FP8_E4M3)
    return fail(NEUVV_ERR_INVALID_ARG, "unknown dtype");
  if (d.dtype == NEUVV_FP8_E4M3 && !((kpad_of(d.K) == 8 && d.hh_degree == 2) || (kpad_of(d.K) == 16 && d.hh_degree == 3)))
    return fail(NEUVV_ERR_UNSUPPORTED, "FP8 storage is built for K <= 8 with degree 2 and 9 <= K <= 16 with degree 3");
  if (d.n_nodes < 1 || d.n_leaves < 0 || d.n_leaves >= 0x7FFFFFFF || d.n_nodes >= 0x7FFFFFFF)
    return fail(NEUVV_ERR_INVALID_ARG, "bad node/leaf counts");
  if (!d.child || !d.basis_A || !d.basis_B) return fail(NEUVV_ERR_INVALID_ARG, "child/basis pointer is NULL");
  if (d.n_leaves > 0 && (!d.w_sigma || !d.w_gamma || !d.w_hh))
    return fail(NEUVV_ERR_INVALID_ARG, "coefficient pointer is NULL");
  for (int a = 0; a < 3; ++a)
    if (!(d.aabb_max[a] > d.aabb_min[a]) || !std::isfinite(d.aabb_min[a]) || !std::isfinite(d.aabb_max[a]))
      return fail(NEUVV_ERR_INVALID_ARG, "aabb must satisfy min < max (finite)");

  // -- validate the child table: entries in range, breadth-first, one parent
  //    per node, internal nodes only above the finest level
  std::vector<int8_t> level((size_t)d.n_nodes, -1);
  level[0] = 0;
  for (int64_t n = 0; n < d.n_nodes; ++n) {
    for (int c = 0; c < 8; ++c) {
      const uint32_t e = d.child[n * 8 + c];
      if (e == kEmpty) continue;
      if (e & kLeafBit) {
        if ((int64_t)(e & ~kLeafBit) >= d.n_leaves)
          return fail(NEUVV_ERR_INVALID_ARG, "node %lld slot %d: leaf id out of range", (long long)n, c);
        continue;
      }
      if ((int64_t)e >= d.n_nodes || (int64_t)e <= n)
        return fail(NEUVV_ERR_INVALID_ARG, "node %lld slot %d: child index %u not in (node, n_nodes)",
                    (long long)n, c, e);
      if (level[n] >= 0) {
        if (level[e] >= 0) return fail(NEUVV_ERR_INVALID_ARG, "node %u has two parents", e);
        if (level[n] + 1 >= d.depth)
          return fail(NEUVV_ERR_INVALID_ARG, "internal node %u below the finest level", e);
        level[e] = (int8_t)(level[n] + 1);
      }
    }
  }

  neuvv_tree *t = new neuvv_tree();
  auto cleanup = [&](neuvv_status s) {
    neuvv_tree_destroy(t);
    return s;
  };
  neuvv_tree_info &I = t->info;
  I.depth = d.depth;
  I.K = d.K;
  I.K_pad = kpad_of(d.K);
  I.T = d.T;
  I.hh_degree = d.hh_degree;
  I.N_h = n_hh(d.hh_degree);
  I.rec_len = 2 * I.K_pad + 3 * I.N_h;
  I.rec_stride_f32 = (I.rec_len + 3) / 4 * 4;
  I.rec_stride = d.dtype == NEUVV_F32    ? I.rec_stride_f32
                 : d.dtype == NEUVV_BF16 ? (I.rec_len + 7) / 8 * 8
                                         : 16 + (I.rec_len + 15) / 16 * 16;  // FP8: bytes, scale header first
  I.dtype = d.dtype;
  I.n_nodes = d.n_nodes;
  I.n_leaves = d.n_leaves;
  if (cudaGetDevice(&I.device) != cudaSuccess) return cleanup(fail(NEUVV_ERR_CUDA, "no CUDA device"));
  cudaDeviceGetAttribute(&t->num_sms, cudaDevAttrMultiProcessorCount, I.device);
  for (int a = 0; a < 3; ++a) {
    t->bmin[a] = d.aabb_min[a];
    t->bmax[a] = d.aabb_max[a];
    t->scale[a] = (float)((double)(1 << d.depth) / ((double)d.aabb_max[a] - (double)d.aabb_min[a]));
  }
  for (int k = 0; k < 16; ++k) t->hh_norm[k] = 0.f;
  for (int n = 0; n <= 3; ++n)
    for (int l = 0; l <= n; ++l) t->hh_norm[4 * n + l] = (float)hh_norm_value(n, l);

  // -- records: FP32 first, then the storage dtype
  const size_t L = (size_t)d.n_leaves;
  const int Kp = I.K_pad, Nh = I.N_h, sf = I.rec_stride_f32;
  std::vector<float> recf(L * sf, 0.f);
  for (size_t l = 0; l < L; ++l) {
    float *r = recf.data() + l * sf;
    for (int k = 0; k < d.K; ++k) {
      r[k] = d.w_sigma[(size_t)k * L + l];
      r[Kp + k] = d.w_gamma[(size_t)k * L + l];
    }
    for (int q = 0; q < 3 * Nh; ++q) r[2 * Kp + q] = d.w_hh[(size_t)q * L + l];
  }
  std::vector<float> Ap((size_t)d.T * Kp, 0.f), Bp((size_t)d.T * Kp, 0.f);
  for (int f = 0; f < d.T; ++f)
    for (int k = 0; k < d.K; ++k) {
      Ap[(size_t)f * Kp + k] = d.basis_A[(size_t)f * d.K + k];
      Bp[(size_t)f * Kp + k] = d.basis_B[(size_t)f * d.K + k];
    }

  cudaError_t e;
#define NEUVV_TRY(call, what) \
  if ((e = (call)) != cudaSuccess) return cleanup(cuda_fail(e, what));
  NEUVV_TRY(cudaMalloc(&t->child, (size_t)d.n_nodes * 8 * 4), "cudaMalloc(child)");
  NEUVV_TRY(cudaMemcpy(t->child, d.child, (size_t)d.n_nodes * 8 * 4, cudaMemcpyHostToDevice), "copy child");
  NEUVV_TRY(cudaMalloc(&t->A, Ap.size() * 4), "cudaMalloc(A)");
  NEUVV_TRY(cudaMalloc(&t->B, Bp.size() * 4), "cudaMalloc(B)");
  NEUVV_TRY(cudaMemcpy(t->A, Ap.data(), Ap.size() * 4, cudaMemcpyHostToDevice), "copy A");
  NEUVV_TRY(cudaMemcpy(t->B, Bp.data(), Bp.size() * 4, cudaMemcpyHostToDevice), "copy B");
  NEUVV_TRY(cudaMalloc(&t->status, 4), "cudaMalloc(status)");
  NEUVV_TRY(cudaMemset(t->status, 0, 4), "memset status");
  NEUVV_TRY(cudaMalloc(&t->work, kWorkSlots * sizeof(unsigned long long)), "cudaMalloc(work)");
  NEUVV_TRY(cudaMemset(t->work, 0, kWorkSlots * sizeof(unsigned long long)), "memset work");
  const size_t recf_bytes = L * sf * 4 + 16;
  if (d.dtype == NEUVV_F32) {
    NEUVV_TRY(cudaMalloc(&t->rec, recf_bytes), "cudaMalloc(records)");
    if (L) NEUVV_TRY(cudaMemcpy(t->rec, recf.data(), L * sf * 4, cudaMemcpyHostToDevice), "copy records");
    if (d.with_optimizer) {
      t->master = static_cast<float *>(t->rec);
      t->master_is_storage = true;
    }
  } else if (d.dtype == NEUVV_FP8_E4M3) {
    // per leaf and group (w_sigma, w_gamma, w_hh): power-of-two scale, then
    // one E4M3 code per entry, nearest with ties to even
    const int sb = I.rec_stride;
    std::vector<uint8_t> rec8(L * sb, 0);
    for (size_t l = 0; l < L; ++l) {
      const float *r = recf.data() + l * sf;
      uint8_t *o = rec8.data() + l * sb;
      const int lo[3] = {0, Kp, 2 * Kp}, hi[3] = {Kp, 2 * Kp, I.rec_len};
      for (int g = 0; g < 3; ++g) {
        float mx = 0.f;
        for (int q = lo[g]; q < hi[g]; ++q) mx = std::max(mx, std::fabs(r[q]));
        const int p = fp8_scale_exp(mx);
        const float sc = std::ldexp(1.f, p);
        std::memcpy(o + 4 * g, &sc, 4);
        for (int q = lo[g]; q < hi[g]; ++q)
          o[16 + q] = (uint8_t)__nv_cvt_float_to_fp8(std::ldexp(r[q], -p), __NV_SATFINITE, __NV_E4M3);
      }
    }
    NEUVV_TRY(cudaMalloc(&t->rec, L * sb + 16), "cudaMalloc(records)");
    if (L) NEUVV_TRY(cudaMemcpy(t->rec, rec8.data(), L * sb, cudaMemcpyHostToDevice), "copy records");
    if (d.with_optimizer) {
      NEUVV_TRY(cudaMalloc(&t->master, recf_bytes), "cudaMalloc(master)");
      if (L) NEUVV_TRY(cudaMemcpy(t->master, recf.data(), L * sf * 4, cudaMemcpyHostToDevice), "copy master");
    }
  } else {
    const int sb = I.rec_stride;
    std::vector<uint16_t> recb(L * sb, 0);
    for (size_t l = 0; l < L; ++l)
      for (int q = 0; q < I.rec_len; ++q) recb[l * sb + q] = bf16_bits(recf[l * sf + q]);
    NEUVV_TRY(cudaMalloc(&t->rec, L * sb * 2 + 16), "cudaMalloc(records)");
    if (L) NEUVV_TRY(cudaMemcpy(t->rec, recb.data(), L * sb * 2, cudaMemcpyHostToDevice), "copy records");
    if (d.with_optimizer) {
      NEUVV_TRY(cudaMalloc(&t->master, recf_bytes), "cudaMalloc(master)");
      if (L) NEUVV_TRY(cudaMemcpy(t->master, recf.data(), L * sf * 4, cudaMemcpyHostToDevice), "copy master");
    }
  }
  if (d.with_optimizer) {
    NEUVV_TRY(cudaMalloc(&t->m, recf_bytes), "cudaMalloc(m)");
    NEUVV_TRY(cudaMalloc(&t->v, recf_bytes), "cudaMalloc(v)");
    NEUVV_TRY(cudaMemset(t->m, 0, recf_bytes), "memset m");
    NEUVV_TRY(cudaMemset(t->v, 0, recf_bytes), "memset v");
  }
  // -- bricks at level depth-3 (8^3 finest cells per internal node there),
  //    when those nodes form one contiguous index range and leaf ids fit
  if (!(d.flags & NEUVV_TREE_NO_BRICKS) && d.depth >= 3 && d.n_leaves < (int64_t)kBrickBoxBase) {
    const int Lb = d.depth - 3, sh = 3;
    int64_t first = -1, last = -1;
    bool contiguous = true;
    for (int64_t n = 0; n < d.n_nodes; ++n)
      if (level[n] == Lb) {
        if (first < 0) first = n;
        else if (n != last + 1) contiguous = false;
        last = n;
      }
    const int64_t count = first < 0 ? 0 : last - first + 1;
    if (contiguous && count > 0 && count * 512 * 4 <= ((int64_t)1 << 30)) {
      std::vector<uint32_t> br((size_t)count * 512, 0);
      for (int64_t n = first; n <= last; ++n)
        fill_brick(d.child, (uint32_t)n, Lb, d.depth, sh, 0, 0, 0, br.data() + (size_t)(n - first) * 512);
      t->brick_level = Lb;
      t->brick_first = (int)first;
      t->brick_count = (int)count;
      // brick map over the level-Lb cells (kept to 128^3 cells, 8 MB), and
      // with it the empty boxes inside the bricks
      if (Lb >= 1 && Lb <= 7) {
        const int nc = 1 << Lb;
        const size_t n3 = (size_t)nc * nc * nc;
        std::vector<uint32_t> map(n3, kCoarseEmpty << 28);
        fill_coarse(d.child, 0, 0, Lb, 0, 0, 0, first, map.data());
        std::vector<uint8_t> occ(n3);
        for (size_t q = 0; q < n3; ++q) occ[q] = (map[q] >> 28) != kCoarseEmpty;
        const std::vector<int32_t> dist = chebyshev_distance(occ, nc, nc);
        std::vector<uint32_t> boxed(br);
        brick_empty_boxes(br, boxed, map, nc, d.depth);
        br.swap(boxed);
        coarse_empty_boxes(occ, dist, nc, map);
        NEUVV_TRY(cudaMalloc(&t->coarse, n3 * 4), "cudaMalloc(brick map)");
        NEUVV_TRY(cudaMemcpy(t->coarse, map.data(), n3 * 4, cudaMemcpyHostToDevice), "copy brick map");
      }
      NEUVV_TRY(cudaMalloc(&t->bricks, br.size() * 4), "cudaMalloc(bricks)");
      NEUVV_TRY(cudaMemcpy(t->bricks, br.data(), br.size() * 4, cudaMemcpyHostToDevice), "copy bricks");
    }
  }
#undef NEUVV_TRY
  t->plain.num_sms = t->packet.num_sms = t->compose.num_sms = t->num_sms > 0 ? t->num_sms : 1;
  *out = t;
  return NEUVV_OK;
}

neuvv_status neuvv_tree_destroy(neuvv_tree *t) {
  if (!t) return NEUVV_OK;
  DeviceGuard g(t->info.device);
  if (!t->master_is_storage) cudaFree(t->master);
  cudaFree(t->rec);
  cudaFree(t->child);
  cudaFree(t->bricks);
  cudaFree(t->coarse);
  cudaFree(t->m);
  cudaFree(t->v);
  cudaFree(t->A);
  cudaFree(t->B);
  cudaFree(t->status);
  cudaFree(t->work);
  free_gather(t);
  delete t;
  return NEUVV_OK;
}

neuvv_status neuvv_tree_reserve_adjoint(neuvv_tree *t, int64_t n_slots) {
  if (!t) return fail(NEUVV_ERR_INVALID_ARG, "tree is NULL");
  if (n_slots < 0 || n_slots > (int64_t)0xFFFFFFFFll - kLogRounds * 32)
    return fail(NEUVV_ERR_INVALID_ARG, "n_slots must be in [0, 2^32 - 256]");
  const long long nl = t->info.n_leaves;
  if (n_slots > 0 && nl > (long long)kScanTile * kScanParts)
    return fail(NEUVV_ERR_UNSUPPORTED, "the leaf-major adjoint handles up to %d leaves", kScanTile * kScanParts);
  DeviceGuard g(t->info.device);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "synchronize");
  free_gather(t);
  const long long chunks = n_slots / (kLogRounds * 32);
  if (chunks == 0) return NEUVV_OK;
  const size_t slots = (size_t)chunks * kLogRounds * 32;
  GatherWs w{};
  if (cudaMalloc(&w.fac, slots * 2 * sizeof(float4)) != cudaSuccess ||
      cudaMalloc(&w.off, (size_t)(nl + 1) * sizeof(uint32_t)) != cudaSuccess ||
      cudaMalloc(&w.cur, (size_t)(nl + 1) * sizeof(uint32_t)) != cudaSuccess ||
      cudaMalloc(&w.part, kScanParts * sizeof(uint32_t)) != cudaSuccess) {
    cudaGetLastError();
    t->gws = w;
    free_gather(t);
    return fail(NEUVV_ERR_OOM, "cudaMalloc of the adjoint workspace (%zu slots)", slots);
  }
  w.cap_chunks = (uint32_t)chunks;
  t->gws = w;
  return NEUVV_OK;
}

neuvv_status neuvv_tree_get_info(const neuvv_tree *t, neuvv_tree_info *info) {
  if (!t || !info) return fail(NEUVV_ERR_INVALID_ARG, "tree/info is NULL");
  *info = t->info;
  info->packet_block = t->packet.block;
  info->packet_queue = t->packet.queue;
  info->packet_ready = t->packet.ready;
  info->packet_order = t->packet.order;
  info->packet_tiles = t->packet_tiles;
  return NEUVV_OK;
}

neuvv_status neuvv_tree_coeff_ptrs(neuvv_tree *t, void **storage, float **master, float **m, float **v) {
  if (!t) return fail(NEUVV_ERR_INVALID_ARG, "tree is NULL");
  if (storage) *storage = t->rec;
  if (master) *master = t->master;
  if (m) *m = t->m;
  if (v) *v = t->v;
  return NEUVV_OK;
}

neuvv_status neuvv_tree_set_records(neuvv_tree *t, const float *records, neuvv_stream stream) {
  if (!t) return fail(NEUVV_ERR_INVALID_ARG, "tree is NULL");
  if (t->info.n_leaves == 0) return NEUVV_OK;
  if (!records || ((uintptr_t)records & 15)) return fail(NEUVV_ERR_INVALID_ARG, "records must be a 16-byte aligned pointer");
  DeviceGuard g(t->info.device);
  float *master = t->master_is_storage ? nullptr : t->master;
  cudaError_t e = launch_store_records(records, master, t->rec, (DType)t->info.dtype, t->info.rec_stride,
                                       t->info.n_leaves, t->info.rec_stride_f32, t->info.rec_len, t->info.K_pad,
                                       (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "store records launch");
  return NEUVV_OK;
}

neuvv_status neuvv_tree_status(neuvv_tree *t, uint32_t *flags) {
  if (!t || !flags) return fail(NEUVV_ERR_INVALID_ARG, "tree/flags is NULL");
  DeviceGuard g(t->info.device);
  cudaError_t e = cudaMemcpy(flags, t->status, 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "read status");
  e = cudaMemset(t->status, 0, 4);
  if (e != cudaSuccess) return cuda_fail(e, "clear status");
  return NEUVV_OK;
}

neuvv_status neuvv_render(const neuvv_tree *t, const neuvv_rays *rays, float time, const neuvv_render_opts *opts,
                          neuvv_out *out, neuvv_stream stream) {
  if (!t) return fail(NEUVV_ERR_INVALID_ARG, "tree is NULL");
  neuvv_status s;
  if ((s = check_rays(rays)) != NEUVV_OK || (s = check_opts(opts)) != NEUVV_OK || (s = check_time(rays, time)))
    return s;
  if (!out || (rays->n > 0 && (!out->rgb || !out->alpha)))
    return fail(NEUVV_ERR_INVALID_ARG, "out->rgb and out->alpha are required");
  if ((s = check_log(out)) != NEUVV_OK) return s;
  if (rays->n == 0) return NEUVV_OK;
  DeviceGuard g(t->info.device);
  cudaStream_t st = (cudaStream_t)stream;
  FwdArgs a{};
  a.tr = dev_tree(t);
  a.rays = dev_rays(rays, time);
  a.out = DevOut{out->rgb, out->alpha, out->depth, out->tau, out->nseg};
  a.t_stop = opts->t_stop;
  a.act = opts->color_act;
  const bool packet = opts->kernel != NEUVV_KERNEL_PLAIN;
  const LaunchCfg &cfg = packet ? t->packet : t->plain;
  a.work = packet && cfg.dynamic_queue ? t->work + 0 : nullptr;
  int64_t chunk_bytes = 0;
  a.log = packet ? log_view(out->log, out->log_bytes, rays->n, &chunk_bytes) : log_view(nullptr, 0, 0);
  a.slice = nullptr;
  a.slice_stride = 0;
  a.edits = nullptr;
  a.edit_beta = 0.f;
  a.order = nullptr;
  cudaError_t e;
  if (a.log.n_chunks) {
    e = cudaMemsetAsync(a.log.counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_fail(e, "reset log");
    if (cfg.order == 1 && a.work) {
      // persistent warps take the packets in the order of the regions they reach
      if ((e = launch_packet_order(a.tr, a.rays, a.log, cfg.num_sms, st)) != cudaSuccess)
        return cuda_fail(e, "packet order");
      a.order = a.log.order;
    } else if (cfg.order == 2 && (size_t)chunk_bytes >= ray_order_scratch_bytes(rays->n)) {
      // packets re-formed from the rays sorted by direction and region (the
      // chunk area is the sort's scratch until the forward writes it)
      if ((e = launch_ray_order(a.tr, a.rays, a.log.perm, a.log.next, cfg.num_sms, st)) != cudaSuccess)
        return cuda_fail(e, "ray order");
      a.perm = a.log.perm;
    }
  } else if ((e = clear_log(out, st)) != cudaSuccess) {
    return cuda_fail(e, "clear log");
  }
  e = launch_render_fwd(t->info.K_pad, t->info.hh_degree, (DType)t->info.dtype, packet, a, cfg, st);
  if (e != cudaSuccess) return cuda_fail(e, "render launch");
  return NEUVV_OK;
}

neuvv_status neuvv_render_alpha(const neuvv_tree *t, const neuvv_rays *rays, float time, const neuvv_render_opts *opts,
                                neuvv_out *out, neuvv_stream stream) {
  if (!t) return fail(NEUVV_ERR_INVALID_ARG, "tree is NULL");
  neuvv_status s;
  if ((s = check_rays(rays)) != NEUVV_OK || (s = check_opts(opts)) != NEUVV_OK || (s = check_time(rays, time)))
    return s;
  if (!out || (rays->n > 0 && !out->alpha)) return fail(NEUVV_ERR_INVALID_ARG, "out->alpha is required");
  if (rays->n == 0) return NEUVV_OK;
  DeviceGuard g(t->info.device);
  FwdArgs a{};
  a.tr = dev_tree(t);
  a.rays = dev_rays(rays, time);
  a.out = DevOut{nullptr, out->alpha, out->depth, out->tau, out->nseg};
  a.t_stop = opts->t_stop;
  a.act = opts->color_act;
  a.work = nullptr;
  a.log = log_view(nullptr, 0, 0);
  a.slice = nullptr;
  a.slice_stride = 0;
  a.edits = nullptr;
  a.edit_beta = 0.f;
  cudaError_t e = launch_render_alpha(t->info.K_pad, t->info.hh_degree, (DType)t->info.dtype, a, t->packet,
                                      (cudaStream_t)stream);
  if (e == cudaErrorNotSupported)
    return fail(NEUVV_ERR_UNSUPPORTED, "density-only render is built for K_pad 8 / degree 2 and K_pad 16 / degree 3");
  if (e != cudaSuccess) return cuda_fail(e, "alpha render launch");
  return NEUVV_OK;
}

neuvv_status neuvv_slice(const neuvv_tree *t, float time, float *slice, int32_t slice_stride, neuvv_stream stream) {
  if (!t) return fail(NEUVV_ERR_INVALID_ARG, "tree is NULL");
  if (!(time >= 0.f && time <= 1.f)) return fail(NEUVV_ERR_INVALID_ARG, "t must be in [0, 1]");
  const int deg = t->info.hh_degree;
  if (slice_stride < slice_min_stride(deg) || (slice_stride & 3))
    return fail(NEUVV_ERR_INVALID_ARG, "slice_stride must be a multiple of 4 and >= %d", slice_min_stride(deg));
  if (t->info.n_leaves == 0) return NEUVV_OK;
  if (!slice || ((uintptr_t)slice & 15)) return fail(NEUVV_ERR_INVALID_ARG, "slice must be a 16-byte aligned pointer");
  DeviceGuard g(t->info.device);
  const DevTree d = dev_tree(t);
  const int esize = t->info.dtype == NEUVV_F32 ? 4 : (t->info.dtype == NEUVV_BF16 ? 2 : 1);
  cudaError_t e = launch_slice(t->info.K_pad, deg, (DType)t->info.dtype, d, time * (float)(t->info.T - 1), slice,
                               slice_stride, t->info.rec_stride * esize, t->num_sms > 0 ? t->num_sms : 1,
                               (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "slice launch");
  return NEUVV_OK;
}

neuvv_status neuvv_render_slice(const neuvv_tree *t, const float *slice, int32_t slice_stride, const neuvv_rays *rays,
                                const neuvv_render_opts *opts, neuvv_out *out, neuvv_stream stream) {
  if (!t) return fail(NEUVV_ERR_INVALID_ARG, "tree is NULL");
  neuvv_status s;
  if ((s = check_rays(rays)) != NEUVV_OK || (s = check_opts(opts)) != NEUVV_OK) return s;
  const int deg = t->info.hh_degree;
  if (slice_stride < slice_min_stride(deg) || (slice_stride & 3))
    return fail(NEUVV_ERR_INVALID_ARG, "slice_stride must be a multiple of 4 and >= %d", slice_min_stride(deg));
  if (!out || (rays->n > 0 && (!out->rgb || !out->alpha)))
    return fail(NEUVV_ERR_INVALID_ARG, "out->rgb and out->alpha are required");
  if ((s = check_log(out)) != NEUVV_OK) return s;
  if (rays->n == 0) return NEUVV_OK;
  if (t->info.n_leaves > 0 && (!slice || ((uintptr_t)slice & 15)))
    return fail(NEUVV_ERR_INVALID_ARG, "slice must be a 16-byte aligned pointer");
  DeviceGuard g(t->info.device);
  cudaStream_t st = (cudaStream_t)stream;
  FwdArgs a{};
  a.tr = dev_tree(t);
  a.rays = dev_rays(rays, 0.f);
  a.out = DevOut{out->rgb, out->alpha, out->depth, out->tau, out->nseg};
  a.t_stop = opts->t_stop;
  a.act = opts->color_act;
  const LaunchCfg &cfg = t->packet;
  a.work = cfg.dynamic_queue ? t->work + 0 : nullptr;
  a.log = log_view(nullptr, 0, 0);
  a.slice = slice;
  a.slice_stride = slice_stride;
  a.edits = nullptr;
  a.edit_beta = 0.f;
  cudaError_t e = clear_log(out, st);
  if (e != cudaSuccess) return cuda_fail(e, "clear log");
  e = launch_render_slice(deg, a, cfg, st);
  if (e != cudaSuccess) return cuda_fail(e, "slice render launch");
  return NEUVV_OK;
}

namespace {

// Checks the arguments of an adjoint call and fills its launch arguments;
// shared by neuvv_render_backward and neuvv_render_backward_adam.
neuvv_status prepare_backward(const neuvv_tree *t, const neuvv_rays *rays, float time, const neuvv_render_opts *opts,
                              const neuvv_out *saved, const float *grad_rgb, const float *grad_alpha, float *grad,
                              uint32_t *touched, BwdArgs &a) {
  if (!t) return fail(NEUVV_ERR_INVALID_ARG, "tree is NULL");
  neuvv_status s;
  if ((s = check_rays(rays)) != NEUVV_OK || (s = check_opts(opts)) != NEUVV_OK || (s = check_time(rays, time)))
    return s;
  if (rays->n == 0) return NEUVV_OK;
  if (!saved || !saved->rgb || !saved->tau || !saved->nseg)
    return fail(NEUVV_ERR_INVALID_ARG, "saved rgb, tau and nseg are required");
  if ((s = check_log(saved)) != NEUVV_OK) return s;
  if (!grad_rgb || !grad) return fail(NEUVV_ERR_INVALID_ARG, "grad_rgb and grad are required");
  if (((uintptr_t)grad & 15) != 0) return fail(NEUVV_ERR_INVALID_ARG, "grad must be 16-byte aligned");
  a.tr = dev_tree(t);
  a.rays = dev_rays(rays, time);
  a.rgb = saved->rgb;
  a.tau = saved->tau;
  a.nseg = saved->nseg;
  a.grad_rgb = grad_rgb;
  a.grad_alpha = grad_alpha;
  a.grad = grad;
  a.grad_stride = t->info.rec_stride_f32;
  a.touched = touched;
  a.t_stop = opts->t_stop;
  a.act = opts->color_act;
  a.log = log_view(saved->log, saved->log_bytes, rays->n);
  const bool packet = opts->kernel != NEUVV_KERNEL_PLAIN;
  a.key_order = 1;
  a.gws = packet && a.log.n_chunks ? t->gws : GatherWs{};
  return NEUVV_OK;
}

neuvv_status check_adam(const neuvv_tree *t, float lr, float b1, float b2, float eps, int32_t step) {
  if (!t->m || !t->v || !t->master) return fail(NEUVV_ERR_INVALID_ARG, "tree was created without optimizer state");
  if (step < 1) return fail(NEUVV_ERR_INVALID_ARG, "step must be >= 1");
  if (!(b1 >= 0.f && b1 < 1.f && b2 >= 0.f && b2 < 1.f && eps > 0.f && std::isfinite(lr)))
    return fail(NEUVV_ERR_INVALID_ARG, "bad Adam hyper-parameters");
  return NEUVV_OK;
}

// Adam on the touched leaves, then the bitmap cleared (neuvv_adam_step).
cudaError_t run_adam(neuvv_tree *t, float *grad, uint32_t *touched, float lr, float b1, float b2, float eps,
                     int32_t step, cudaStream_t st) {
  const float c1 = (float)(1.0 - std::pow((double)b1, step));
  const float c2 = (float)(1.0 - std::pow((double)b2, step));
  cudaError_t e = launch_adam(t->master, t->m, t->v, t->master_is_storage ? nullptr : t->rec, (DType)t->info.dtype,
                              t->info.rec_stride, grad, touched, t->info.n_leaves, t->info.rec_stride_f32,
                              t->info.rec_len, t->info.K_pad, lr, b1, b2, eps, c1, c2, st);
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(touched, 0, (size_t)((t->info.n_leaves + 31) / 32) * 4, st);
}

}  // namespace

neuvv_status neuvv_render_backward(const neuvv_tree *t, const neuvv_rays *rays, float time,
                                   const neuvv_render_opts *opts, const neuvv_out *saved, const float *grad_rgb,
                                   const float *grad_alpha, float *grad, uint32_t *touched, neuvv_stream stream) {
  BwdArgs a;
  neuvv_status s = prepare_backward(t, rays, time, opts, saved, grad_rgb, grad_alpha, grad, touched, a);
  if (s != NEUVV_OK || rays->n == 0) return s;
  DeviceGuard g(t->info.device);
  const bool packet = opts->kernel != NEUVV_KERNEL_PLAIN;
  const LaunchCfg &cfg = packet ? t->packet : t->plain;
  cudaError_t e = launch_render_bwd(t->info.K_pad, t->info.hh_degree, (DType)t->info.dtype, packet, a, cfg,
                                    (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "backward launch");
  return NEUVV_OK;
}

neuvv_status neuvv_render_backward_adam(neuvv_tree *t, const neuvv_rays *rays, float time,
                                        const neuvv_render_opts *opts, const neuvv_out *saved, const float *grad_rgb,
                                        const float *grad_alpha, float *grad, uint32_t *touched, float lr, float b1,
                                        float b2, float eps, int32_t step, neuvv_stream stream) {
  BwdArgs a;
  neuvv_status s = prepare_backward(t, rays, time, opts, saved, grad_rgb, grad_alpha, grad, touched, a);
  if (s != NEUVV_OK) return s;
  if (!touched) return fail(NEUVV_ERR_INVALID_ARG, "touched is required");
  if ((s = check_adam(t, lr, b1, b2, eps, step)) != NEUVV_OK) return s;
  DeviceGuard g(t->info.device);
  cudaStream_t st = (cudaStream_t)stream;
  bool fused = false;
  if (rays->n > 0) {
    AdamArgs ad;
    ad.master = t->master;
    ad.m = t->m;
    ad.v = t->v;
    ad.storage = t->master_is_storage ? nullptr : t->rec;
    ad.dt = t->info.dtype;
    ad.storage_stride = t->info.rec_stride;
    ad.lr = lr;
    ad.b1 = b1;
    ad.b2 = b2;
    ad.eps = eps;
    ad.c1 = (float)(1.0 - std::pow((double)b1, step));
    ad.c2 = (float)(1.0 - std::pow((double)b2, step));
    ad.on = 1;
    const bool packet = opts->kernel != NEUVV_KERNEL_PLAIN;
    const LaunchCfg &cfg = packet ? t->packet : t->plain;
    cudaError_t e = launch_render_bwd(t->info.K_pad, t->info.hh_degree, (DType)t->info.dtype, packet, a, cfg, st, &ad,
                                      &fused);
    if (e != cudaSuccess) return cuda_fail(e, "backward launch");
  }
  if (!fused) {
    cudaError_t e = run_adam(t, grad, touched, lr, b1, b2, eps, step, st);
    if (e != cudaSuccess) return cuda_fail(e, "adam launch");
  }
  return NEUVV_OK;
}

namespace {

// Checks the arguments of a composition and fills the launch arguments (all
// but the work counter); shared by neuvv_compose and neuvv_compose_noalloc.
neuvv_status prepare_compose(const neuvv_tree *const *trees, const float *transforms, const float *time_offsets,
                             const float *tints, int32_t n_prims, const neuvv_rays *rays, float time,
                             const neuvv_render_opts *opts, neuvv_out *out, ComposeArgs &a, const neuvv_tree *&t0) {
  if (!trees || !transforms || !time_offsets || !tints)
    return fail(NEUVV_ERR_INVALID_ARG, "trees/transforms/time_offsets/tints is NULL");
  if (n_prims < 1 || n_prims > kMaxPrims) return fail(NEUVV_ERR_INVALID_ARG, "n_prims must be in [1, %d]", kMaxPrims);
  neuvv_status s;
  if ((s = check_rays(rays)) != NEUVV_OK || (s = check_opts(opts)) != NEUVV_OK || (s = check_time(rays, time)))
    return s;
  if (!out || (rays->n > 0 && (!out->rgb || !out->alpha)))
    return fail(NEUVV_ERR_INVALID_ARG, "out->rgb and out->alpha are required");
  t0 = trees[0];
  if (!t0) return fail(NEUVV_ERR_INVALID_ARG, "trees[0] is NULL");
  std::memset(&a, 0, sizeof a);
  int n_trees = 0;
  const neuvv_tree *uniq[kMaxPrims];
  for (int j = 0; j < n_prims; ++j) {
    const neuvv_tree *t = trees[j];
    if (!t) return fail(NEUVV_ERR_INVALID_ARG, "trees[%d] is NULL", j);
    if (t->info.K_pad != t0->info.K_pad || t->info.hh_degree != t0->info.hh_degree || t->info.dtype != t0->info.dtype ||
        t->info.device != t0->info.device)
      return fail(NEUVV_ERR_UNSUPPORTED, "all trees of one compose call must share K_pad, degree, dtype, device");
    int slot = -1;
    for (int k = 0; k < n_trees; ++k)
      if (uniq[k] == t) slot = k;
    if (slot < 0) {
      slot = n_trees;
      uniq[n_trees++] = t;
      a.trees[slot] = dev_tree(t);
    }
    const float *M = transforms + 12 * j;
    double m[3][3], tr[3];
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 3; ++c) m[r][c] = M[4 * r + c];
      tr[r] = M[4 * r + 3];
    }
    // uniform scale: M^T M = s^2 I
    double s2 = 0.0;
    for (int r = 0; r < 3; ++r) s2 += m[r][0] * m[r][0];
    if (!(s2 > 0.0) || !std::isfinite(s2)) return fail(NEUVV_ERR_INVALID_ARG, "transform %d is degenerate", j);
    for (int c1 = 0; c1 < 3; ++c1)
      for (int c2 = 0; c2 < 3; ++c2) {
        double dot = 0.0;
        for (int r = 0; r < 3; ++r) dot += m[r][c1] * m[r][c2];
        const double want = c1 == c2 ? s2 : 0.0;
        if (std::fabs(dot - want) > 1e-4 * s2)
          return fail(NEUVV_ERR_INVALID_ARG, "transform %d is not a rotation times a uniform scale", j);
      }
    for (int r = 0; r < 3; ++r)
      if (!std::isfinite(tr[r])) return fail(NEUVV_ERR_INVALID_ARG, "transform %d translation not finite", j);
    const double det = m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) -
                       m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
                       m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
    if (!(det > 0.0)) return fail(NEUVV_ERR_INVALID_ARG, "transform %d must have positive determinant", j);
    PrimParam &p = a.prim[j];
    // the inverse of the given 3x3 part in double (cofactors / determinant),
    // kept as FP32 value + FP32 remainder for the kernel's double-float ray
    double inv[3][3];
    inv[0][0] = (m[1][1] * m[2][2] - m[1][2] * m[2][1]) / det;
    inv[0][1] = (m[0][2] * m[2][1] - m[0][1] * m[2][2]) / det;
    inv[0][2] = (m[0][1] * m[1][2] - m[0][2] * m[1][1]) / det;
    inv[1][0] = (m[1][2] * m[2][0] - m[1][0] * m[2][2]) / det;
    inv[1][1] = (m[0][0] * m[2][2] - m[0][2] * m[2][0]) / det;
    inv[1][2] = (m[0][2] * m[1][0] - m[0][0] * m[1][2]) / det;
    inv[2][0] = (m[1][0] * m[2][1] - m[1][1] * m[2][0]) / det;
    inv[2][1] = (m[0][1] * m[2][0] - m[0][0] * m[2][1]) / det;
    inv[2][2] = (m[0][0] * m[1][1] - m[0][1] * m[1][0]) / det;
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        p.minv[3 * r + c] = (float)inv[r][c];
        p.minv_lo[3 * r + c] = (float)(inv[r][c] - (double)p.minv[3 * r + c]);
      }
    for (int r = 0; r < 3; ++r) p.trans[r] = (float)tr[r];
    p.scale = (float)std::sqrt(s2);
    if (!std::isfinite(time_offsets[j])) return fail(NEUVV_ERR_INVALID_ARG, "time offset %d not finite", j);
    p.toff = time_offsets[j];
    for (int c = 0; c < 3; ++c) {
      if (!std::isfinite(tints[3 * j + c])) return fail(NEUVV_ERR_INVALID_ARG, "tint %d not finite", j);
      p.tint[c] = tints[3 * j + c];
    }
    p.tree = slot;
  }
  a.n_prims = n_prims;
  a.rays = dev_rays(rays, time);
  a.out = DevOut{out->rgb, out->alpha, out->depth, nullptr, nullptr};
  a.t_stop = opts->t_stop;
  a.act = opts->color_act;
  a.mode = opts->compose_mode;
  return NEUVV_OK;
}

}  // namespace

neuvv_status neuvv_compose(const neuvv_tree *const *trees, const float *transforms, const float *time_offsets,
                           const float *tints, int32_t n_prims, const neuvv_rays *rays, float time,
                           const neuvv_render_opts *opts, neuvv_out *out, neuvv_stream stream) {
  ComposeArgs a;
  const neuvv_tree *t0 = nullptr;
  neuvv_status s = prepare_compose(trees, transforms, time_offsets, tints, n_prims, rays, time, opts, out, a, t0);
  if (s != NEUVV_OK) return s;
  if (rays->n == 0) return NEUVV_OK;
  DeviceGuard g(t0->info.device);
  cudaStream_t st = (cudaStream_t)stream;
  a.work = t0->work + 2;
  const LaunchCfg &cfg = t0->compose;
  if (cfg.dynamic_queue) {
    cudaError_t e = cudaMemsetAsync(a.work, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_fail(e, "reset work counter");
  }
  cudaError_t e = clear_log(out, st);
  if (e != cudaSuccess) return cuda_fail(e, "clear log");
  e = launch_compose(t0->info.K_pad, t0->info.hh_degree, (DType)t0->info.dtype, a, cfg, st);
  if (e != cudaSuccess) return cuda_fail(e, "compose launch");
  return NEUVV_OK;
}

neuvv_status neuvv_compose_noalloc(const neuvv_tree *const *trees, const float *transforms, const float *time_offsets,
                                   const float *tints, int32_t n_prims, const neuvv_rays *rays, float time,
                                   const neuvv_render_opts *opts, neuvv_out *out, neuvv_stream stream) {
  ComposeArgs a;
  const neuvv_tree *t0 = nullptr;
  neuvv_status s = prepare_compose(trees, transforms, time_offsets, tints, n_prims, rays, time, opts, out, a, t0);
  if (s != NEUVV_OK) return s;
  if (rays->n > NEUVV_NOALLOC_MAX_RAYS)
    return fail(NEUVV_ERR_INVALID_ARG, "neuvv_compose_noalloc: %lld rays exceed the maximum of %lld",
                (long long)rays->n, (long long)NEUVV_NOALLOC_MAX_RAYS);
  if (rays->n == 0) return NEUVV_OK;
  DeviceGuard g(t0->info.device);
  cudaStream_t st = (cudaStream_t)stream;
  // the packet counter is the library's static device array, not tree memory
  cudaError_t e = noalloc_queue(&a.work);
  if (e != cudaSuccess) return cuda_fail(e, "neuvv_compose_noalloc: device address of the static counter");
  e = cudaMemsetAsync(a.work, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return cuda_fail(e, "neuvv_compose_noalloc: reset counter");
  LaunchCfg cfg = t0->compose;
  cfg.dynamic_queue = 1;
  if ((e = clear_log(out, st)) != cudaSuccess) return cuda_fail(e, "clear log");
  e = launch_compose(t0->info.K_pad, t0->info.hh_degree, (DType)t0->info.dtype, a, cfg, st);
  if (e != cudaSuccess) return cuda_fail(e, "compose launch");
  return NEUVV_OK;
}

neuvv_status neuvv_adam_step(neuvv_tree *t, float *grad, uint32_t *touched, float lr, float b1, float b2, float eps,
                             int32_t step, neuvv_stream stream) {
  if (!t) return fail(NEUVV_ERR_INVALID_ARG, "tree is NULL");
  neuvv_status s;
  if ((s = check_adam(t, lr, b1, b2, eps, step)) != NEUVV_OK) return s;
  if (!grad || !touched) return fail(NEUVV_ERR_INVALID_ARG, "grad and touched are required");
  if (((uintptr_t)grad & 15) != 0) return fail(NEUVV_ERR_INVALID_ARG, "grad must be 16-byte aligned");
  DeviceGuard g(t->info.device);
  cudaError_t e = run_adam(t, grad, touched, lr, b1, b2, eps, step, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "adam launch");
  return NEUVV_OK;
}

neuvv_status neuvv_mse_grad(const float *rgb, const float *target, int64_t n, float scale, float *grad_rgb,
                            float *loss_accum, neuvv_stream stream) {
  if (n < 0) return fail(NEUVV_ERR_INVALID_ARG, "n < 0");
  if (n > 0 && (!rgb || !target || !grad_rgb)) return fail(NEUVV_ERR_INVALID_ARG, "rgb/target/grad_rgb is NULL");
  cudaError_t e = launch_mse(rgb, target, (long long)n, scale, grad_rgb, loss_accum, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "mse launch");
  return NEUVV_OK;
}

neuvv_status neuvv_grad_loss(const float *rgb, const float *target, int64_t n, const int32_t *ray_of_pixel,
                             int32_t width, int32_t height, int32_t n_views, float lambda, float *grad_rgb,
                             float *loss_accum, neuvv_stream stream) {
  if (n < 0 || width < 0 || height < 0 || n_views < 0) return fail(NEUVV_ERR_INVALID_ARG, "negative size");
  if (n >= 0x7FFFFFFF) return fail(NEUVV_ERR_INVALID_ARG, "n must be below 2^31 (int32 ray ids)");
  const long long n_pix = (long long)n_views * width * height;
  if (n_pix > 0 && (!rgb || !target || !grad_rgb || !ray_of_pixel))
    return fail(NEUVV_ERR_INVALID_ARG, "rgb/target/ray_of_pixel/grad_rgb is NULL");
  cudaError_t e = launch_grad_loss(rgb, target, ray_of_pixel, width, height, n_views, (long long)n, lambda, grad_rgb,
                                   loss_accum, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "grad loss launch");
  return NEUVV_OK;
}

neuvv_status neuvv_pick(const neuvv_tree *t, const neuvv_rays *rays, float time, float threshold, int32_t *leaf,
                        neuvv_stream stream) {
  if (!t) return fail(NEUVV_ERR_INVALID_ARG, "tree is NULL");
  neuvv_status s;
  if ((s = check_rays(rays)) != NEUVV_OK || (s = check_time(rays, time)) != NEUVV_OK) return s;
  if (!(threshold > 0.f && threshold < 1.f)) return fail(NEUVV_ERR_INVALID_ARG, "threshold must be in (0, 1)");
  if (rays->n == 0) return NEUVV_OK;
  if (!leaf) return fail(NEUVV_ERR_INVALID_ARG, "leaf is NULL");
  DeviceGuard g(t->info.device);
  FwdArgs a{};
  std::memset(&a, 0, sizeof a);
  a.tr = dev_tree(t);
  a.rays = dev_rays(rays, time);
  cudaError_t e = launch_pick(t->info.K_pad, t->info.hh_degree, (DType)t->info.dtype, a, threshold, leaf,
                              (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "pick launch");
  return NEUVV_OK;
}

neuvv_status neuvv_paint(const neuvv_tree *t, const int32_t *leaf, const float *color, int64_t n, float sigma_d,
                         float t_d, float *accum, float *edits, neuvv_stream stream) {
  if (!t) return fail(NEUVV_ERR_INVALID_ARG, "tree is NULL");
  if (n < 0) return fail(NEUVV_ERR_INVALID_ARG, "n < 0");
  if ((n > 0 && (!leaf || !color)) || (t->info.n_leaves > 0 && (!accum || !edits)))
    return fail(NEUVV_ERR_INVALID_ARG, "leaf/color/accum/edits is NULL");
  if (((uintptr_t)accum & 15) || ((uintptr_t)edits & 15))
    return fail(NEUVV_ERR_INVALID_ARG, "accum and edits must be 16-byte aligned");
  DeviceGuard g(t->info.device);
  cudaError_t e = launch_paint(leaf, color, n, t->info.n_leaves, accum, sigma_d, t_d, edits, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "paint launch");
  return NEUVV_OK;
}

neuvv_status neuvv_render_edit(const neuvv_tree *t, const neuvv_rays *rays, float time, const neuvv_render_opts *opts,
                               const float *edits, float beta, neuvv_out *out, neuvv_stream stream) {
  if (!t) return fail(NEUVV_ERR_INVALID_ARG, "tree is NULL");
  neuvv_status s;
  if ((s = check_rays(rays)) != NEUVV_OK || (s = check_opts(opts)) != NEUVV_OK || (s = check_time(rays, time)))
    return s;
  if (!(beta >= 0.f && beta <= 1.f)) return fail(NEUVV_ERR_INVALID_ARG, "beta must be in [0, 1]");
  if (!out || (rays->n > 0 && (!out->rgb || !out->alpha)))
    return fail(NEUVV_ERR_INVALID_ARG, "out->rgb and out->alpha are required");
  if ((s = check_log(out)) != NEUVV_OK) return s;
  if (rays->n == 0) return NEUVV_OK;
  if (t->info.n_leaves > 0 && (!edits || ((uintptr_t)edits & 15)))
    return fail(NEUVV_ERR_INVALID_ARG, "edits must be a 16-byte aligned pointer");
  DeviceGuard g(t->info.device);
  cudaStream_t st = (cudaStream_t)stream;
  FwdArgs a{};
  std::memset(&a, 0, sizeof a);
  a.tr = dev_tree(t);
  a.rays = dev_rays(rays, time);
  a.out = DevOut{out->rgb, out->alpha, out->depth, out->tau, out->nseg};
  a.t_stop = opts->t_stop;
  a.act = opts->color_act;
  const LaunchCfg &cfg = t->packet;
  a.work = cfg.dynamic_queue ? t->work + 0 : nullptr;
  a.log = log_view(nullptr, 0, 0);
  a.edits = edits;
  a.edit_beta = beta;
  cudaError_t e = clear_log(out, st);
  if (e != cudaSuccess) return cuda_fail(e, "clear log");
  e = launch_render_edit(t->info.K_pad, t->info.hh_degree, (DType)t->info.dtype, a, cfg, st);
  if (e == cudaErrorNotSupported)
    return fail(NEUVV_ERR_UNSUPPORTED, "edited renders are built for K <= 8 with degree 2 and 9 <= K <= 16 with degree 3, FP32 or BF16 storage");
  if (e != cudaSuccess) return cuda_fail(e, "edit render launch");
  return NEUVV_OK;
}

neuvv_status neuvv_gaussian_blur(const float *in, float *out, int32_t width, int32_t height, int32_t n_images,
                                 float sigma, neuvv_stream stream) {
  if (width < 0 || height < 0 || n_images < 0) return fail(NEUVV_ERR_INVALID_ARG, "negative size");
  if (!(sigma > 0.f && sigma <= 5.f)) return fail(NEUVV_ERR_INVALID_ARG, "sigma must be in (0, 5]");
  const long long n_pix = (long long)n_images * width * height;
  if (n_pix == 0) return NEUVV_OK;
  if (!in || !out || in == out) return fail(NEUVV_ERR_INVALID_ARG, "in/out NULL or the same buffer");
  BlurWeights bw;
  bw.radius = (int)(3.0 * sigma + 0.5);
  if (bw.radius > kMaxBlurRadius) bw.radius = kMaxBlurRadius;
  double sum = 0.0, w[2 * kMaxBlurRadius + 1];
  for (int k = -bw.radius; k <= bw.radius; ++k) sum += (w[k + bw.radius] = std::exp(-0.5 * k * k / ((double)sigma * sigma)));
  for (int k = 0; k <= 2 * bw.radius; ++k) bw.w[k] = (float)(w[k] / sum);
  cudaError_t e = launch_gaussian_blur(in, out, width, height, n_images, bw, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "blur launch");
  return NEUVV_OK;
}

neuvv_status neuvv_spotlight(const neuvv_rays *rays, const float *rgb, const float *alpha, const float *depth,
                             const neuvv_light *light, const float *light_alpha, float ground_z, const float albedo[3],
                             float r_ref, float *rgb_out, neuvv_stream stream) {
  neuvv_status s;
  if ((s = check_rays(rays)) != NEUVV_OK) return s;
  if (!light || !albedo) return fail(NEUVV_ERR_INVALID_ARG, "light/albedo is NULL");
  if (light->width < 1 || light->height < 1 || !(light->fov_y_deg > 0.f && light->fov_y_deg < 180.f))
    return fail(NEUVV_ERR_INVALID_ARG, "light camera needs a positive size and a field of view in (0, 180)");
  if (!(r_ref > 0.f)) return fail(NEUVV_ERR_INVALID_ARG, "r_ref must be positive");
  if (rays->n == 0) return NEUVV_OK;
  if (!rgb || !alpha || !depth || !light_alpha || !rgb_out || rgb_out == rgb)
    return fail(NEUVV_ERR_INVALID_ARG, "rgb/alpha/depth/light_alpha/rgb_out NULL or rgb_out == rgb");
  SpotArgs a;
  a.rays = dev_rays(rays, 0.f);
  a.rgb = rgb;
  a.alpha = alpha;
  a.depth = depth;
  for (int k = 0; k < 3; ++k) {
    a.light.eye[k] = light->eye[k];
    a.light.right[k] = light->right[k];
    a.light.up[k] = light->up[k];
    a.light.forward[k] = light->forward[k];
    a.albedo[k] = albedo[k];
  }
  a.light.fov_y_deg = light->fov_y_deg;
  a.light.width = light->width;
  a.light.height = light->height;
  a.light_alpha = light_alpha;
  a.ground_z = ground_z;
  a.r_ref = r_ref;
  a.out = rgb_out;
  cudaError_t e = launch_spotlight(a, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "spotlight launch");
  return NEUVV_OK;
}

neuvv_status neuvv_camera_rays(const neuvv_camera *cams, const float *times, int32_t n_cams, int32_t tiled,
                               float *origins, float *dirs, float *times_out, int32_t *pixel_of_ray, int64_t n,
                               neuvv_stream stream) {
  if (n_cams < 1 || n_cams > kMaxCams) return fail(NEUVV_ERR_INVALID_ARG, "n_cams must be in [1, 32]");
  if (!cams || !times) return fail(NEUVV_ERR_INVALID_ARG, "cams/times is NULL");
  CamBatch cb;
  std::memset(&cb, 0, sizeof cb);
  long long total = 0;
  for (int c = 0; c < n_cams; ++c) {
    const neuvv_camera &k = cams[c];
    if (k.width < 1 || k.height < 1 || !(k.fov_y_deg > 0.f && k.fov_y_deg < 180.f))
      return fail(NEUVV_ERR_INVALID_ARG, "camera needs a positive size and a field of view in (0, 180)");
    if ((long long)k.width * k.height >= 0x7FFFFFFFll)
      return fail(NEUVV_ERR_INVALID_ARG, "a camera's pixel count must be below 2^31 (int32 pixel ids)");
    if (!(times[c] >= 0.f && times[c] <= 1.f)) return fail(NEUVV_ERR_INVALID_ARG, "camera time outside [0, 1]");
    for (int a = 0; a < 3; ++a) {
      cb.cam[c].eye[a] = k.eye[a];
      cb.cam[c].right[a] = k.right[a];
      cb.cam[c].up[a] = k.up[a];
      cb.cam[c].forward[a] = k.forward[a];
    }
    cb.cam[c].fov_y_deg = k.fov_y_deg;
    cb.cam[c].width = k.width;
    cb.cam[c].height = k.height;
    cb.tan_half[c] = (float)std::tan((double)k.fov_y_deg * 3.14159265358979323846 / 360.0);
    cb.aspect[c] = (float)((double)k.width / (double)k.height);
    cb.t[c] = times[c];
    cb.off[c] = total;
    total += (long long)k.width * k.height;
  }
  for (int c = n_cams; c <= kMaxCams; ++c) cb.off[c] = total;
  cb.n_cams = n_cams;
  static const int kTiles[4][2] = {{0, 0}, {8, 4}, {4, 8}, {16, 2}};
  if (tiled < NEUVV_TILES_NONE || tiled > NEUVV_TILES_16X2)
    return fail(NEUVV_ERR_INVALID_ARG, "unknown tile shape %d", tiled);
  cb.tile_w = kTiles[tiled][0];
  cb.tile_h = kTiles[tiled][1];
  if (n != total) return fail(NEUVV_ERR_INVALID_ARG, "n differs from the cameras' total pixel count");
  if (!origins || !dirs || !times_out) return fail(NEUVV_ERR_INVALID_ARG, "origins/dirs/times_out is NULL");
  cudaError_t e = launch_camera_rays(cb, origins, dirs, times_out, pixel_of_ray, (long long)n, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "camera rays launch");
  return NEUVV_OK;
}

neuvv_status neuvv_trace(const neuvv_tree *t, const neuvv_rays *rays, int32_t max_out, int32_t *leaf, float *t0,
                         float *t1, int32_t *count, neuvv_stream stream) {
  if (!t) return fail(NEUVV_ERR_INVALID_ARG, "tree is NULL");
  neuvv_status s;
  if ((s = check_rays(rays)) != NEUVV_OK) return s;
  if (max_out < 0) return fail(NEUVV_ERR_INVALID_ARG, "max_out < 0");
  if (rays->n > 0 && (!count || (max_out > 0 && (!leaf || !t0 || !t1))))
    return fail(NEUVV_ERR_INVALID_ARG, "trace output pointer is NULL");
  if (rays->n == 0) return NEUVV_OK;
  DeviceGuard g(t->info.device);
  TraceArgs a;
  a.tr = dev_tree(t);
  a.rays = dev_rays(rays, 0.f);
  a.max_out = max_out;
  a.leaf = leaf;
  a.t0 = t0;
  a.t1 = t1;
  a.count = count;
  cudaError_t e = launch_trace(a, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "trace launch");
  return NEUVV_OK;
}

neuvv_status neuvv_tree_set_limits(neuvv_tree *t, int32_t step_cap, int32_t wait_polls) {
  if (!t) return fail(NEUVV_ERR_INVALID_ARG, "tree is NULL");
  if (step_cap < 0) return fail(NEUVV_ERR_INVALID_ARG, "step_cap must be >= 0");
  if (wait_polls < 0) return fail(NEUVV_ERR_INVALID_ARG, "wait_polls must be >= 0");
  t->step_cap = step_cap;
  t->wait_polls = wait_polls;
  return NEUVV_OK;
}

neuvv_status neuvv_log_read(const neuvv_out *saved, int64_t n, int32_t max_out, int32_t *leaf, float *chord,
                            int32_t *count, neuvv_stream stream) {
  if (!saved || !saved->nseg) return fail(NEUVV_ERR_INVALID_ARG, "saved and saved->nseg are required");
  neuvv_status s;
  if ((s = check_log(saved)) != NEUVV_OK) return s;
  if (n < 0 || n > ((int64_t)1 << 37)) return fail(NEUVV_ERR_INVALID_ARG, "n out of range");
  if (max_out < 0) return fail(NEUVV_ERR_INVALID_ARG, "max_out < 0");
  if (n > 0 && (!count || (max_out > 0 && (!leaf || !chord))))
    return fail(NEUVV_ERR_INVALID_ARG, "output pointer is NULL");
  if (n == 0) return NEUVV_OK;
  const SampleLog l = log_view(saved->log, saved->log_bytes, n);
  cudaError_t e = launch_log_read(l, (long long)n, saved->nseg, max_out, leaf, chord, count, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "log read launch");
  return NEUVV_OK;
}

neuvv_status neuvv_tree_set_packet_order(neuvv_tree *t, int32_t order) {
  if (!t) return fail(NEUVV_ERR_INVALID_ARG, "tree is NULL");
  if (order != NEUVV_ORDER_AS_GIVEN && order != NEUVV_ORDER_BY_REGION && order != NEUVV_ORDER_BY_RAY)
    return fail(NEUVV_ERR_INVALID_ARG, "unknown packet order %d", order);
  t->packet.order = order;
  return NEUVV_OK;
}

neuvv_status neuvv_tree_set_launch(neuvv_tree *t, int32_t block, int32_t queue, int32_t ready) {
  if (!t) return fail(NEUVV_ERR_INVALID_ARG, "tree is NULL");
  if (block < 32 || block > 256 || block % 32 != 0)
    return fail(NEUVV_ERR_INVALID_ARG, "block must be a multiple of 32 in [32, 256]");
  if (queue < 1 || queue > kMaxQueue || (queue & (queue - 1)) != 0)
    return fail(NEUVV_ERR_INVALID_ARG, "queue must be a power of two in [1, %d]", kMaxQueue);
  if (ready < 1 || ready > 32) return fail(NEUVV_ERR_INVALID_ARG, "ready must be in [1, 32]");
  t->packet.block = block;
  t->packet.queue = queue;
  t->packet.ready = ready;
  return NEUVV_OK;
}

namespace {

// Autotuner choices kept for the life of the process, one per tree shape,
// storage type, device and sample size (see neuvv_autotune).
struct TuneKey {
  int device, num_sms, depth, K_pad, degree, dtype, bricks, log2_rays;
  long long n_nodes, n_leaves;
  bool operator==(const TuneKey &o) const {
    return device == o.device && num_sms == o.num_sms && depth == o.depth && K_pad == o.K_pad &&
           degree == o.degree && dtype == o.dtype && bricks == o.bricks && log2_rays == o.log2_rays &&
           n_nodes == o.n_nodes && n_leaves == o.n_leaves;
  }
};
struct TuneRecord {
  TuneKey key;
  LaunchCfg best;
  float best_ms;
  std::vector<neuvv_tune_entry> table;
};
std::mutex g_tune_mu;
std::vector<TuneRecord> g_tune_cache;

TuneKey tune_key(const neuvv_tree *t, long long n_rays) {
  TuneKey k{};
  k.device = t->info.device;
  k.num_sms = t->num_sms;
  k.depth = t->info.depth;
  k.K_pad = t->info.K_pad;
  k.degree = t->info.hh_degree;
  k.dtype = t->info.dtype;
  k.bricks = t->coarse ? 2 : (t->bricks ? 1 : 0);
  int b = 0;
  while (b < 62 && ((long long)1 << (b + 1)) <= n_rays) ++b;
  k.log2_rays = b;
  k.n_nodes = t->info.n_nodes;
  k.n_leaves = t->info.n_leaves;
  return k;
}

}  // namespace

neuvv_status neuvv_autotune(neuvv_tree *t, const neuvv_rays *sample, float time, float *best_ms,
                            neuvv_stream stream) {
  if (!t) return fail(NEUVV_ERR_INVALID_ARG, "tree is NULL");
  neuvv_status s;
  if ((s = check_rays(sample)) != NEUVV_OK || (s = check_time(sample, time)) != NEUVV_OK) return s;
  if (sample->n == 0) return NEUVV_OK;
  DeviceGuard g(t->info.device);
  cudaStream_t st = (cudaStream_t)stream;
  neuvv_rays r = *sample;
  if (r.n > (1 << 20)) r.n = 1 << 20;
  const TuneKey key = tune_key(t, r.n);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const TuneRecord &rec : g_tune_cache)
      if (rec.key == key) {  // the same shape was timed before: keep its choice
        const int sms = t->packet.num_sms;
        t->packet = rec.best;
        t->packet.num_sms = sms;
        t->tune_table = rec.table;
        t->tune_cached = 1;
        if (best_ms) *best_ms = rec.best_ms;
        return NEUVV_OK;
      }
  }
  // outputs and a segment log of 64 bytes per ray, as a training step uses
  float *rgb = nullptr, *alpha = nullptr;
  void *logbuf = nullptr;
  const int64_t log_bytes = r.n * 64 + 65536;
  cudaError_t e;
  if ((e = cudaMalloc(&rgb, r.n * 12)) != cudaSuccess || (e = cudaMalloc(&alpha, r.n * 4)) != cudaSuccess ||
      (e = cudaMalloc(&logbuf, log_bytes)) != cudaSuccess) {
    cudaFree(rgb);
    cudaFree(alpha);
    return cuda_fail(e, "autotune alloc");
  }
  cudaEvent_t ev0, ev1;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  neuvv_render_opts opts{1e-4f, NEUVV_ACT_SIGMOID, NEUVV_KERNEL_PACKET, NEUVV_COMPOSE_SORTED};
  neuvv_out out{rgb, alpha, nullptr, nullptr, nullptr, logbuf, log_bytes};
  const LaunchCfg saved = t->packet;
  LaunchCfg best = saved;
  float best_t = 1e30f;
  std::vector<neuvv_tune_entry> table;
  struct Cand { int block, queue, ready; };
  const Cand cands[] = {{64, 8, 16}, {64, 1, 1}, {64, 4, 8}, {128, 8, 16}, {128, 1, 1}, {32, 8, 16}, {64, 16, 16}};
  for (int order = NEUVV_ORDER_AS_GIVEN; order <= NEUVV_ORDER_BY_RAY && s == NEUVV_OK; ++order)
    for (const Cand &c : cands) {
      t->packet = saved;
      t->packet.block = c.block;
      t->packet.queue = c.queue;
      t->packet.ready = c.ready;
      t->packet.order = order;
      t->packet.dynamic_queue = 1;
      float ms_best = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(ev0, st);
        s = neuvv_render(t, &r, time, &opts, &out, stream);
        cudaEventRecord(ev1, st);
        if (s != NEUVV_OK) break;
        cudaEventSynchronize(ev1);
        float ms;
        cudaEventElapsedTime(&ms, ev0, ev1);
        if (ms < ms_best) ms_best = ms;
      }
      if (s != NEUVV_OK) break;
      table.push_back(neuvv_tune_entry{c.block, c.queue, c.ready, order, ms_best});
      if (ms_best < best_t) {
        best_t = ms_best;
        best = t->packet;
      }
    }
  t->packet = s == NEUVV_OK ? best : saved;
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  cudaStreamSynchronize(st);
  cudaFree(rgb);
  cudaFree(alpha);
  cudaFree(logbuf);
  if (s != NEUVV_OK) return s;
  t->tune_table = table;
  t->tune_cached = 0;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache.push_back(TuneRecord{key, best, best_t, table});
  }
  if (best_ms) *best_ms = best_t;
  return NEUVV_OK;
}

neuvv_status neuvv_autotune_tiles(neuvv_tree *t, const neuvv_camera *cams, const float *times, int32_t n_cams,
                                  int32_t *best_tiles, float *best_ms, neuvv_stream stream) {
  if (!t || !best_tiles) return fail(NEUVV_ERR_INVALID_ARG, "tree/best_tiles is NULL");
  if (n_cams < 1 || n_cams > kMaxCams || !cams || !times)
    return fail(NEUVV_ERR_INVALID_ARG, "cams/times must hold 1..32 cameras");
  long long n = 0;
  for (int c = 0; c < n_cams; ++c) n += (long long)std::max(cams[c].width, 0) * std::max(cams[c].height, 0);
  if (n <= 0 || n > ((int64_t)1 << 31)) return fail(NEUVV_ERR_INVALID_ARG, "the cameras' pixel count must be in [1, 2^31]");
  DeviceGuard g(t->info.device);
  cudaStream_t st = (cudaStream_t)stream;
  float *buf = nullptr, *rgb = nullptr, *alpha = nullptr;
  void *logbuf = nullptr;
  const int64_t log_bytes = n * 64 + 65536;
  cudaError_t e;
  if ((e = cudaMalloc(&buf, (size_t)n * 7 * 4)) != cudaSuccess || (e = cudaMalloc(&rgb, (size_t)n * 12)) != cudaSuccess ||
      (e = cudaMalloc(&alpha, (size_t)n * 4)) != cudaSuccess || (e = cudaMalloc(&logbuf, log_bytes)) != cudaSuccess) {
    cudaFree(buf);
    cudaFree(rgb);
    cudaFree(alpha);
    return cuda_fail(e, "tile autotune alloc");
  }
  neuvv_rays r{buf, buf + n, buf + 2 * n, buf + 3 * n, buf + 4 * n, buf + 5 * n, buf + 6 * n, n};
  neuvv_render_opts opts{1e-4f, NEUVV_ACT_SIGMOID, NEUVV_KERNEL_PACKET, NEUVV_COMPOSE_SORTED};
  neuvv_out out{rgb, alpha, nullptr, nullptr, nullptr, logbuf, log_bytes};
  cudaEvent_t ev0, ev1;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  neuvv_status s = NEUVV_OK;
  int best = NEUVV_TILES_8X4;
  float best_t = 1e30f;
  for (int mode = NEUVV_TILES_8X4; mode <= NEUVV_TILES_16X2 && s == NEUVV_OK; ++mode) {
    s = neuvv_camera_rays(cams, times, n_cams, mode, buf, buf + 3 * n, buf + 6 * n, nullptr, n, stream);
    float ms_best = 1e30f;
    for (int rep = 0; rep < 3 && s == NEUVV_OK; ++rep) {
      cudaEventRecord(ev0, st);
      s = neuvv_render(t, &r, 0.f, &opts, &out, stream);
      cudaEventRecord(ev1, st);
      if (s != NEUVV_OK) break;
      cudaEventSynchronize(ev1);
      float ms;
      cudaEventElapsedTime(&ms, ev0, ev1);
      ms_best = std::min(ms_best, ms);
    }
    if (s == NEUVV_OK && ms_best < best_t) {
      best_t = ms_best;
      best = mode;
    }
  }
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  cudaStreamSynchronize(st);
  cudaFree(buf);
  cudaFree(rgb);
  cudaFree(alpha);
  cudaFree(logbuf);
  if (s != NEUVV_OK) return s;
  t->packet_tiles = best;
  *best_tiles = best;
  if (best_ms) *best_ms = best_t;
  return NEUVV_OK;
}

neuvv_status neuvv_autotune_report(const neuvv_tree *t, neuvv_tune_entry *entries, int32_t max_entries,
                                   int32_t *n_entries, int32_t *from_cache) {
  if (!t || !n_entries) return fail(NEUVV_ERR_INVALID_ARG, "tree/n_entries is NULL");
  if (max_entries < 0 || (max_entries > 0 && !entries)) return fail(NEUVV_ERR_INVALID_ARG, "bad entries buffer");
  const int n = (int)t->tune_table.size();
  for (int i = 0; i < n && i < max_entries; ++i) entries[i] = t->tune_table[i];
  *n_entries = n;
  if (from_cache) *from_cache = t->tune_cached;
  return NEUVV_OK;
}

neuvv_status neuvv_autotune_clear_cache(void) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache.clear();
  return NEUVV_OK;
}

}  // extern "C"
