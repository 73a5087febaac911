// Ray order of the packet kernels, and the scans both it and the leaf-major
// adjoint use.
//
// A batch of rays from many views and time stamps, in any order, is re-formed
// into coherent 32-ray packets (batching of uneven rays): every ray gets a
// 24-bit key -- a bucket of its direction (octahedral map, 8 x 8 buckets) in
// the high 6 bits, the region of the first leaf it reaches (the top 18 bits
// of the leaf id, which follows the Morton order of the leaves) in the low
// 18 -- and a stable LSD radix sort (three passes of 8-bit digits) lists the
// rays by key.  Rays of one view that enter one region of the tree become
// neighbours; rays with equal keys keep the caller's order.  The result is a
// permutation (position -> ray) that the packet forward and adjoint read
// their rays through; outputs stay in the caller's order.
#include <algorithm>

#include "neuvv_kernels.h"

namespace neuvv {

// Exclusive scan of uint32 counts, in place, tile by tile: each block scans
// kScanTile counts (4 per thread) and leaves the tile's total in part[tile].
__global__ void __launch_bounds__(1024) scan_tiles_kernel(uint32_t *v, long long n, uint32_t *part) {
  __shared__ uint32_t warp_sum[32];
  const long long base = (long long)blockIdx.x * kScanTile + 4 * threadIdx.x;
  uint32_t x[4], sum = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    x[k] = base + k < n ? v[base + k] : 0u;
    sum += x[k];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t incl = sum;  // inclusive scan of the threads' sums within the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_sum[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    uint32_t ws = warp_sum[lane], wi = ws;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
      if (lane >= o) wi += y;
    }
    warp_sum[lane] = wi - ws;  // exclusive over warps
    if (lane == 31) part[blockIdx.x] = wi;
  }
  __syncthreads();
  uint32_t run = warp_sum[wid] + incl - sum;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (base + k < n) v[base + k] = run;
    run += x[k];
  }
}

// Exclusive scan of the tile totals (one block; at most kScanParts tiles);
// v[n] receives the number of samples.
__global__ void __launch_bounds__(1024) scan_parts_kernel(uint32_t *part, int n_parts, uint32_t *v, long long n) {
  __shared__ uint32_t warp_sum[32];
  uint32_t x[4], sum = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int j = 4 * threadIdx.x + k;
    x[k] = j < n_parts ? part[j] : 0u;
    sum += x[k];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_sum[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    uint32_t ws = warp_sum[lane], wi = ws;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
      if (lane >= o) wi += y;
    }
    warp_sum[lane] = wi - ws;
    if (lane == 31) v[n] = wi;
  }
  __syncthreads();
  uint32_t run = warp_sum[wid] + incl - sum;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int j = 4 * threadIdx.x + k;
    if (j < n_parts) part[j] = run;
    run += x[k];
  }
}

__global__ void __launch_bounds__(256) scan_add_kernel(uint32_t *v, long long n, const uint32_t *part) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    v[i] += __ldg(part + i / kScanTile);
}

cudaError_t launch_exclusive_scan(uint32_t *v, long long n, uint32_t *part, int num_sms, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int tiles = (int)((n + kScanTile - 1) / kScanTile);
  if (tiles > kScanParts) return cudaErrorInvalidValue;
  scan_tiles_kernel<<<tiles, 1024, 0, s>>>(v, n, part);
  scan_parts_kernel<<<1, 1024, 0, s>>>(part, tiles, v, n);
  scan_add_kernel<<<(unsigned)std::min<long long>((n + 255) / 256, 8LL * num_sms), 256, 0, s>>>(v, n, part);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Keys
// ---------------------------------------------------------------------------
constexpr uint32_t kMissKey = 0xFFFFFFu;

// Octahedral bucket of a unit direction: the direction scaled to the L1 unit
// sphere, the lower half folded over the diagonals, then an 8 x 8 grid.
__device__ __forceinline__ uint32_t direction_bucket(const float d[3]) {
  const float s = fabsf(d[0]) + fabsf(d[1]) + fabsf(d[2]);
  float x = d[0] / s, y = d[1] / s;
  if (d[2] < 0.f) {
    const float fx = (1.f - fabsf(y)) * (x >= 0.f ? 1.f : -1.f);
    const float fy = (1.f - fabsf(x)) * (y >= 0.f ? 1.f : -1.f);
    x = fx;
    y = fy;
  }
  const int u = min(max((int)((x + 1.f) * 4.f), 0), 7), v = min(max((int)((y + 1.f) * 4.f), 0), 7);
  return (uint32_t)(u * 8 + v);
}

__global__ void __launch_bounds__(256) ray_key_kernel(const __grid_constant__ DevTree tr, const DevRays rays,
                                                      uint32_t *keys, uint32_t *perm, int shift) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rays.n) return;
  float o[3], d[3], t, dn[3];
  load_ray(rays, i, o, d, t);
  RayWalk w;
  uint32_t leaf, key = kMissKey;
  float t0, dt;
  if (walk_init(tr, o, d, w, dn) && walk_next<false>(tr, nullptr, w, leaf, t0, dt))
    key = (direction_bucket(dn) << 18) | ((leaf >> shift) & 0x3FFFFu);
  keys[i] = key;
  perm[i] = (uint32_t)i;
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of (key, ray) pairs, 8-bit digits.  A tile of
// kRadixTile pairs is one block of kRadixWarps warps; warp w owns the
// tile's pairs [w * kRadixPerWarp, (w + 1) * kRadixPerWarp), in steps of 32.
// ---------------------------------------------------------------------------
constexpr int kRadixWarps = 8, kRadixPerWarp = 512, kRadixTile = kRadixWarps * kRadixPerWarp;
constexpr int kRadixSteps = kRadixPerWarp / 32;

// table[d * n_tiles + tile] = pairs of the tile with digit d.
__global__ void __launch_bounds__(kRadixWarps * 32) radix_hist_kernel(const uint32_t *keys, long long n, int sh,
                                                                       uint32_t *table, int n_tiles) {
  __shared__ uint32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const long long first = (long long)blockIdx.x * kRadixTile;
  for (int k = threadIdx.x; k < kRadixTile; k += blockDim.x) {
    const long long e = first + k;
    if (e < n) atomicAdd(&cnt[(keys[e] >> sh) & 0xFFu], 1u);
  }
  __syncthreads();
  table[(size_t)threadIdx.x * n_tiles + blockIdx.x] = cnt[threadIdx.x];
}

// After the exclusive scan of the table (digit-major, then tile), each pair
// goes to its digit's start for its tile plus its rank among the tile's
// earlier pairs with that digit: warps in order, and within a warp steps in
// order and lanes in order (ranks from __match_any_sync), so equal digits
// keep their order.
__global__ void __launch_bounds__(kRadixWarps * 32) radix_scatter_kernel(const uint32_t *keys_in, const uint32_t *perm_in,
                                                                          uint32_t *keys_out, uint32_t *perm_out,
                                                                          long long n, int sh, const uint32_t *table,
                                                                          int n_tiles) {
  __shared__ uint32_t wcnt[kRadixWarps][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = threadIdx.x; k < kRadixWarps * 256; k += blockDim.x) (&wcnt[0][0])[k] = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * kRadixTile + (long long)warp * kRadixPerWarp;
  const unsigned lt = (1u << lane) - 1u;
  uint32_t rank[kRadixSteps];
#pragma unroll
  for (int st = 0; st < kRadixSteps; ++st) {
    const long long e = base + 32 * st + lane;
    const bool in = e < n;
    const uint32_t dgt = in ? (keys_in[e] >> sh) & 0xFFu : 256u;  // 256: past the end, a group of its own
    const unsigned grp = __match_any_sync(0xFFFFFFFFu, dgt);
    rank[st] = in ? wcnt[warp][dgt] + (uint32_t)__popc(grp & lt) : 0u;
    __syncwarp();
    if (in && lane == __ffs(grp) - 1) wcnt[warp][dgt] += (uint32_t)__popc(grp);
    __syncwarp();
  }
  __syncthreads();
  // per digit: the pairs of the earlier warps of this tile come first
  {
    const int dgt = threadIdx.x;  // 256 threads, one per digit
    uint32_t run = table[(size_t)dgt * n_tiles + blockIdx.x];
#pragma unroll
    for (int w = 0; w < kRadixWarps; ++w) {
      const uint32_t c = wcnt[w][dgt];
      wcnt[w][dgt] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int st = 0; st < kRadixSteps; ++st) {
    const long long e = base + 32 * st + lane;
    if (e >= n) continue;
    const uint32_t key = keys_in[e];
    const uint32_t pos = wcnt[warp][(key >> sh) & 0xFFu] + rank[st];
    keys_out[pos] = key;
    perm_out[pos] = perm_in[e];
  }
}

size_t ray_order_scratch_bytes(long long n) {
  const long long tiles = (n + kRadixTile - 1) / kRadixTile;
  return (size_t)n * 16 + (size_t)(256 * tiles + 1) * 4 + (size_t)kScanParts * 4 + 256;
}

cudaError_t launch_ray_order(const DevTree &tr, const DevRays &rays, uint32_t *perm, void *scratch, int num_sms,
                             cudaStream_t s) {
  const long long n = rays.n;
  if (n == 0) return cudaSuccess;
  const long long tiles = (n + kRadixTile - 1) / kRadixTile;
  if (tiles * 256 > (long long)kScanTile * kScanParts || n > 0xFFFFFFFFll) return cudaErrorInvalidValue;
  // scratch: keys A, ray A, keys B, ray B [n] each, the digit table, scan parts
  char *p = static_cast<char *>(scratch);
  p = reinterpret_cast<char *>(((uintptr_t)p + 15) & ~(uintptr_t)15);
  uint32_t *ka = reinterpret_cast<uint32_t *>(p), *pa = ka + n, *kb = pa + n, *pb = kb + n;
  uint32_t *table = pb + n, *part = table + 256 * tiles + 1;
  int bits = 0;
  while (bits < 32 && ((long long)1 << bits) <= tr.n_leaves) ++bits;
  const int shift = bits > 18 ? bits - 18 : 0;
  ray_key_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(tr, rays, ka, pa, shift);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const uint32_t *kin = ka, *pin = pa;
  uint32_t *kout = kb, *pout = pb;
  for (int pass = 0; pass < 3; ++pass) {
    if (pass == 2) pout = perm;  // the last pass writes the permutation in place
    radix_hist_kernel<<<(unsigned)tiles, kRadixWarps * 32, 0, s>>>(kin, n, 8 * pass, table, (int)tiles);
    if ((e = launch_exclusive_scan(table, 256 * tiles, part, num_sms, s)) != cudaSuccess) return e;
    radix_scatter_kernel<<<(unsigned)tiles, kRadixWarps * 32, 0, s>>>(kin, pin, kout, pout, n, 8 * pass, table,
                                                                      (int)tiles);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const uint32_t *tk = kout, *tp = pout;
    kout = const_cast<uint32_t *>(kin);
    pout = const_cast<uint32_t *>(pin);
    kin = tk;
    pin = tp;
  }
  return cudaSuccess;
}

}  // namespace neuvv
