// Spatial-temporal composition of several VOctree primitives in one persistent
// launch (Eq. st_composite_affine; Sec. 5.1 "Varied Manifestations":
// duplicates share one tree; Algorithm 1, depth-aware alpha blending).
//
// Per ray and primitive j: the world ray is taken to the primitive's local
// frame, o' = (sR)^-1 (o - t_j), d' = (sR)^-1 d (then normalised, so chords
// are in local units and the optical depth of the object does not depend on
// its size), culled against the local box, rendered at frame
// u' = (t (T-1) + offset_j) mod (T-1), and kept as a layer
// (tint_j * C_j, A_j, s * D_j).  The layers are then merged: sorted by depth
// (stable) with front-to-back "over" on premultiplied colour, or Algorithm 1
// taken literally (sequential pairwise merge) on premultiplied colour.
//
// The local ray is formed in double-float arithmetic (a value carried as an
// unevaluated sum hi + lo of two FP32 numbers; Dekker's error-free products
// and Knuth's two-sum), and so is its entry point into the local box: a ray
// from a camera far from the primitive then reaches the voxels with the
// precision of a ray given in the tree's own frame, and a grazing crossing
// of a voxel face does not magnify the rounding of the transform.
#include <cuda.h>

#include <mutex>

#include "neuvv_kernels.h"
#include "neuvv_ray.cuh"

namespace neuvv {

struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df_norm(float s, float e) {
  const float hi = s + e;
  return DF{hi, e - (hi - s)};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  return df_norm(s, e + (a.lo + b.lo));
}
__device__ __forceinline__ DF df_mul(DF a, float b) {
  float p, e;
  two_prod(a.hi, b, p, e);
  return df_norm(p, fmaf(a.lo, b, e));
}
// sum_j m[j] q[j] with m = mh + ml given as two FP32 rows
__device__ __forceinline__ DF df_dot3(const float *mh, const float *ml, const DF q[3]) {
  DF acc{0.f, 0.f};
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    DF p = df_mul(q[j], mh[j]);
    p.lo = fmaf(q[j].hi, ml[j], p.lo);
    acc = df_add(acc, p);
  }
  return acc;
}

// Starts the walk of world ray (o, d) through primitive pp's tree in the
// tree's frame.  Returns false when the ray misses the local box; otherwise
// dn (unit local direction), the world distance of the entry point from o
// and the world length of one local unit along the ray.
__device__ __forceinline__ bool walk_init_local(const DevTree &tr, const PrimParam &pp, const float o[3],
                                                const float d[3], RayWalk &w, float dn[3], float &t_base,
                                                float &dist_scale) {
  {
    // FP32 cull first: most (ray, primitive) pairs miss the primitive's box
    // (margin for the rounding of this rough ray)
    const float q0[3] = {o[0] - pp.trans[0], o[1] - pp.trans[1], o[2] - pp.trans[2]};
    float ro[3], rd[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      ro[r] = pp.minv[3 * r] * q0[0] + pp.minv[3 * r + 1] * q0[1] + pp.minv[3 * r + 2] * q0[2];
      rd[r] = pp.minv[3 * r] * d[0] + pp.minv[3 * r + 1] * d[1] + pp.minv[3 * r + 2] * d[2];
    }
    float sn = -INFINITY, sf = INFINITY;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float ext = 1e-3f * (tr.bmax[a] - tr.bmin[a]);
      const float lo = tr.bmin[a] - ext, hi = tr.bmax[a] + ext;
      if (rd[a] == 0.f) {
        if (ro[a] < lo || ro[a] > hi) return false;
      } else {
        const float s0 = (lo - ro[a]) / rd[a], s1 = (hi - ro[a]) / rd[a];
        sn = fmaxf(sn, fminf(s0, s1));
        sf = fminf(sf, fmaxf(s0, s1));
      }
    }
    if (!(fmaxf(sn, 0.f) <= sf)) return false;
  }
  DF q[3], dd[3], ol[3], dl[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float s, e;
    two_sum(o[k], -pp.trans[k], s, e);
    q[k] = DF{s, e};
    dd[k] = DF{d[k], 0.f};
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    ol[r] = df_dot3(pp.minv + 3 * r, pp.minv_lo + 3 * r, q);
    dl[r] = df_dot3(pp.minv + 3 * r, pp.minv_lo + 3 * r, dd);
  }
  const float olh[3] = {ol[0].hi, ol[1].hi, ol[2].hi}, dlh[3] = {dl[0].hi, dl[1].hi, dl[2].hi};
  const float dlen = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  const float llen = sqrtf(dlh[0] * dlh[0] + dlh[1] * dlh[1] + dlh[2] * dlh[2]);
  float s_in, s_out;
  int ax;
  if (!(dlen > 0.f && llen > 0.f) || !box_interval(tr, olh, dlh, s_in, s_out, ax)) return false;
  // entry point ol + s dl in double-float: s from the entry face's equation,
  // the entry coordinate set to the face exactly
  float p[3], pl[3];
  float s_hi = 0.f;
  if (ax < 0) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      p[k] = ol[k].hi;
      pl[k] = ol[k].lo;
    }
  } else {
    DF ola = ol[0], dla = dl[0];
    float f = tr.bmin[0];
#pragma unroll
    for (int k = 1; k < 3; ++k)
      if (k == ax) { ola = ol[k]; dla = dl[k]; f = tr.bmin[k]; }
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (k == ax && dla.hi < 0.f) f = tr.bmax[k];
    const DF num = df_add(DF{f, 0.f}, DF{-ola.hi, -ola.lo});
    s_hi = num.hi / dla.hi;
    const float s_lo = ((fmaf(-s_hi, dla.hi, num.hi) + num.lo) - s_hi * dla.lo) / dla.hi;
    const DF s = df_norm(s_hi, s_lo);
    s_hi = s.hi;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (k == ax) {
        p[k] = f;
        pl[k] = 0.f;
      } else {
        DF sd = df_mul(dl[k], s.hi);
        sd.lo = fmaf(dl[k].hi, s.lo, sd.lo);
        const DF pk = df_add(ol[k], sd);
        p[k] = pk.hi;
        pl[k] = pk.lo;
      }
    }
  }
  // unit direction rounded as the render path rounds it (times 1/|d|)
  const float il = 1.f / llen;
#pragma unroll
  for (int k = 0; k < 3; ++k) dn[k] = dlh[k] * il;
  walk_start(tr, p, pl, dn, w);
  // the local point ol + s dl is the world point o + s d
  t_base = s_hi * dlen;
  dist_scale = dlen / llen;
  return w.alive;
}

template <int KP, int DEG, typename E>
__global__ void __launch_bounds__(256) compose_kernel(const __grid_constant__ ComposeArgs a, int dynamic) {
  const long long n = a.rays.n;
  const long long n_packets = (n + 31) >> 5;
  const long long stride = ((long long)gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  long long p;
  if (dynamic) {
    unsigned long long q = 0;
    if (lane == 0) q = atomicAdd(a.work, 1ull);
    p = (long long)__shfl_sync(0xFFFFFFFFu, q, 0);
  } else {
    p = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  }
  while (p < n_packets) {
    const long long i = (p << 5) + lane;
    if (i < n) {
      float o[3], d[3], t;
      load_ray(a.rays, i, o, d, t);
      float Lc[kMaxPrims][3], La[kMaxPrims], Ld[kMaxPrims];
      for (int j = 0; j < a.n_prims; ++j) {
        const PrimParam &pp = a.prim[j];
        const DevTree &tr = a.trees[pp.tree];
        RayResult r;
        clear(r);
        RayWalk w;
        float dn[3], t_base, dist_scale;
        if (walk_init_local(tr, pp, o, d, w, dn, t_base, dist_scale)) {
          const float period = (float)(tr.T - 1);
          float u = fmodf(t * period + pp.toff, period);
          if (u < 0.f) u += period;
          // world distance = t_base + (local distance) * |d| / |dl|
          integrate_walk<KP, DEG, E, false>(tr, nullptr, w, dn, u, a.t_stop, a.act, t_base, dist_scale, r);
        }
        Lc[j][0] = pp.tint[0] * r.C[0];
        Lc[j][1] = pp.tint[1] * r.C[1];
        Lc[j][2] = pp.tint[2] * r.C[2];
        La[j] = r.A;
        Ld[j] = depth_of(r);
      }
      float I0, I1, I2, A, D;
      if (a.mode == 0) {
        // stable order by depth: repeatedly take the nearest unused layer
        unsigned int used = 0;
        I0 = I1 = I2 = 0.f;
        A = 0.f;
        D = INFINITY;
        for (int k = 0; k < a.n_prims; ++k) {
          int best = -1;
          float bd = 0.f;
          for (int j = 0; j < a.n_prims; ++j) {
            if (used & (1u << j)) continue;
            if (best < 0 || Ld[j] < bd) {
              best = j;
              bd = Ld[j];
            }
          }
          used |= 1u << best;
          const float tr_ = 1.f - A;
          I0 = fmaf(tr_, Lc[best][0], I0);
          I1 = fmaf(tr_, Lc[best][1], I1);
          I2 = fmaf(tr_, Lc[best][2], I2);
          A = fmaf(tr_, La[best], A);
          D = fminf(D, Ld[best]);
        }
      } else {
        I0 = Lc[0][0];
        I1 = Lc[0][1];
        I2 = Lc[0][2];
        A = La[0];
        D = Ld[0];
        for (int j = 1; j < a.n_prims; ++j) {
          if (Ld[j] <= D) {
            const float keep = 1.f - La[j];
            I0 = fmaf(keep, I0, Lc[j][0]);
            I1 = fmaf(keep, I1, Lc[j][1]);
            I2 = fmaf(keep, I2, Lc[j][2]);
            D = Ld[j];
          } else {
            const float behind = 1.f - A;
            I0 = fmaf(behind, Lc[j][0], I0);
            I1 = fmaf(behind, Lc[j][1], I1);
            I2 = fmaf(behind, Lc[j][2], I2);
          }
          A = fmaf(La[j], 1.f - A, A);
        }
      }
      a.out.rgb[3 * i + 0] = I0;
      a.out.rgb[3 * i + 1] = I1;
      a.out.rgb[3 * i + 2] = I2;
      a.out.alpha[i] = A;
      if (a.out.depth) a.out.depth[i] = D;
    }
    __syncwarp();
    if (dynamic) {
      unsigned long long q = 0;
      if (lane == 0) q = atomicAdd(a.work, 1ull);
      p = (long long)__shfl_sync(0xFFFFFFFFu, q, 0);
    } else {
      p += stride;
    }
  }
}

template <int KP, int DEG, typename E>
static cudaError_t compose_one(const ComposeArgs &a, const LaunchCfg &cfg, cudaStream_t s) {
  if (a.rays.n == 0) return cudaSuccess;
  int grid = cfg.grid;
  if (grid <= 0) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, compose_kernel<KP, DEG, E>, cfg.block, 0);
    if (e != cudaSuccess) return e;
    grid = (per_sm > 0 ? per_sm : 1) * cfg.num_sms;
  }
  compose_kernel<KP, DEG, E><<<grid, cfg.block, 0, s>>>(a, cfg.dynamic_queue);
  return cudaGetLastError();
}

template <typename E>
static cudaError_t compose_dispatch(int KP, int DEG, const ComposeArgs &a, const LaunchCfg &cfg, cudaStream_t s) {
  switch (KP * 10 + DEG) {
    case 81: return compose_one<8, 1, E>(a, cfg, s);
    case 82: return compose_one<8, 2, E>(a, cfg, s);
    case 83: return compose_one<8, 3, E>(a, cfg, s);
    case 161: return compose_one<16, 1, E>(a, cfg, s);
    case 162: return compose_one<16, 2, E>(a, cfg, s);
    case 163: return compose_one<16, 3, E>(a, cfg, s);
    case 321: return compose_one<32, 1, E>(a, cfg, s);
    case 322: return compose_one<32, 2, E>(a, cfg, s);
    case 323: return compose_one<32, 3, E>(a, cfg, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_compose(int KP, int DEG, DType dt, const ComposeArgs &a, const LaunchCfg &cfg, cudaStream_t s) {
  if (dt == kF32) return compose_dispatch<float>(KP, DEG, a, cfg, s);
  if (dt == kBF16) return compose_dispatch<__nv_bfloat16>(KP, DEG, a, cfg, s);
  if (KP == 8 && DEG == 2) return compose_one<8, 2, Fp8E4M3>(a, cfg, s);
  if (KP == 16 && DEG == 3) return compose_one<16, 3, Fp8E4M3>(a, cfg, s);
  return cudaErrorInvalidValue;
}

// Work counter for neuvv_compose_noalloc: file-scope device memory (one
// 64-bit packet counter, 256-byte aligned) that exists in every context where
// the library's module is loaded, so that entry point needs no allocation.
// Host code must not use the symbol as an address: noalloc_queue() asks the
// runtime for the device address once per CUDA context (with the context
// current) and caches it under the context's unique id, which is never
// reused within a process.  A device reset makes a new primary context (a new
// id), so a stale address is never handed out: the first call after a reset
// looks the address up again.
static __device__ __align__(256) unsigned long long g_noalloc_queue[1];

namespace {
using CtxGetCurrentFn = CUresult(CUDAAPI *)(CUcontext *);
using CtxGetIdFn = CUresult(CUDAAPI *)(CUcontext, unsigned long long *);
}  // namespace

cudaError_t noalloc_queue(unsigned long long **out) {
  constexpr int kMaxContexts = 64;
  static std::mutex mu;
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static unsigned long long ids[kMaxContexts] = {};
  static unsigned long long *ptrs[kMaxContexts] = {};
  static int used = 0;
  std::lock_guard<std::mutex> lock(mu);
  // cudaSetDevice makes the device's primary context current on this thread
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || (e = cudaSetDevice(dev)) != cudaSuccess) return e;
  if (!get_current || !get_id) {
    void *f1 = nullptr, *f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if ((e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1)) != cudaSuccess)
      return e;
    if ((e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2)) != cudaSuccess)
      return e;
    if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return cudaErrorSymbolNotFound;
    get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    get_id = reinterpret_cast<CtxGetIdFn>(f2);
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  for (int k = 0; k < used; ++k)
    if (ids[k] == id) {
      *out = ptrs[k];
      return cudaSuccess;
    }
  void *p = nullptr;
  if ((e = cudaGetSymbolAddress(&p, g_noalloc_queue)) != cudaSuccess) return e;
  const int slot = used < kMaxContexts ? used++ : (int)(id % kMaxContexts);  // evict when full
  ids[slot] = id;
  ptrs[slot] = static_cast<unsigned long long *>(p);
  *out = ptrs[slot];
  return cudaSuccess;
}

}  // namespace neuvv
