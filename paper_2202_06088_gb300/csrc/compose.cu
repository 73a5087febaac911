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
#include <mutex>

#include "neuvv_kernels.h"
#include "neuvv_ray.cuh"

namespace neuvv {

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
        // rough local ray: enough to find where the line enters the local box
        const float q[3] = {o[0] - pp.trans[0], o[1] - pp.trans[1], o[2] - pp.trans[2]};
        float ol[3], dl[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          ol[r] = pp.minv[3 * r] * q[0] + pp.minv[3 * r + 1] * q[1] + pp.minv[3 * r + 2] * q[2];
          dl[r] = pp.minv[3 * r] * d[0] + pp.minv[3 * r + 1] * d[1] + pp.minv[3 * r + 2] * d[2];
        }
        RayResult r;
        clear(r);
        float s_in, s_out;
        int ax;
        const float dlen = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        const float llen = sqrtf(dl[0] * dl[0] + dl[1] * dl[1] + dl[2] * dl[2]);
        if (dlen > 0.f && llen > 0.f && box_interval(tr, ol, dl, s_in, s_out, ax)) {
          // entry point formed in world space from the exact input line, then
          // taken to the local frame (small magnitudes: little rounding)
          float pw[3], pl[3], dn[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) pw[k] = fmaf(s_in, d[k], o[k]) - pp.trans[k];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            pl[k] = pp.minv[3 * k] * pw[0] + pp.minv[3 * k + 1] * pw[1] + pp.minv[3 * k + 2] * pw[2];
            dn[k] = dl[k] / llen;
          }
#pragma unroll
          for (int k = 0; k < 3; ++k)
            if (k == ax) pl[k] = dl[k] > 0.f ? tr.bmin[k] : tr.bmax[k];
          RayWalk w;
          const float zero[3] = {0.f, 0.f, 0.f};
          walk_start(tr, pl, zero, dn, w);
          if (w.alive) {
            const float period = (float)(tr.T - 1);
            float u = fmodf(t * period + pp.toff, period);
            if (u < 0.f) u += period;
            // world distance = s_in |d| + (local distance) * |d| / |dl|
            integrate_walk<KP, DEG, E, false>(tr, nullptr, w, dn, u, a.t_stop, a.act, s_in * dlen, dlen / llen, r);
          }
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
// 64-bit packet counter, 256-byte aligned) that exists on every device where
// the library is loaded, so that entry point needs no allocation.  Host code
// must not use the symbol as an address: noalloc_queue() asks the runtime for
// the device address once per device (with that device current) and caches it.
static __device__ __align__(256) unsigned long long g_noalloc_queue[1];

cudaError_t noalloc_queue(unsigned long long **out) {
  constexpr int kMaxDevices = 64;
  static std::mutex mu;
  static unsigned long long *ptrs[kMaxDevices] = {};
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!ptrs[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_queue);
    if (e != cudaSuccess) return e;
    ptrs[dev] = static_cast<unsigned long long *>(p);
  }
  *out = ptrs[dev];
  return cudaSuccess;
}

}  // namespace neuvv
