// One ray through one VOctree: the forward integrator shared by the render and
// compose kernels (Sec. 4.3 "Rendering"; Eq. volume-rendering).
#pragma once

#include "neuvv_device.cuh"

namespace neuvv {

struct RayResult {
  float C[3];    // premultiplied colour, sum w_i c_i
  float A;       // alpha, sum w_i
  float dnum;    // sum w_i t_mid,i (world distance from the ray origin)
  float tau;     // sum sigma_i delta_i
  int nseg;      // composited segments
};

// Composites front to back along a started walk, stopping after the segment
// that brings the transmittance below t_stop.  dn: unit direction in the
// tree's frame (the view direction of the harmonics); u: frame coordinate;
// t_base + dist_scale * t converts a walk distance t to the caller's frame.
template <int KP, int DEG, typename E, bool kSmem>
__device__ __forceinline__ void integrate_walk(const DevTree &tr, const uint32_t *s_child, RayWalk &w,
                                               const float dn[3], float u, float t_stop, int act, float t_base,
                                               float dist_scale, RayResult &res) {
  RayConst<KP, DEG> rc;
  ray_const_basis<KP, DEG>(tr, u, rc);
  sh_real<DEG>(dn, rc.Y);
  float T = 1.f;
  uint32_t leaf;
  float t0, dt;
  while (walk_next<kSmem>(tr, s_child, w, leaf, t0, dt)) {
    LeafRecord<KP, DEG, E> rec;
    rec.load(tr, leaf);
    Sample<DEG> s;
    eval_sample<KP, DEG, E>(tr, rc, rec, act, s);
    res.nseg += 1;
    if (s.sigma > 0.f) {
      const float sd = s.sigma * dt;
      const float e = __expf(-sd);
      const float wgt = T * alpha_of(sd);
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) res.C[ch] = fmaf(wgt, s.c[ch], res.C[ch]);
      res.A += wgt;
      res.dnum = fmaf(wgt, fmaf(dist_scale, fmaf(0.5f, dt, t0), t_base), res.dnum);
      res.tau += sd;
      T *= e;
      if (T < t_stop) break;
    }
  }
}

__device__ __forceinline__ void clear(RayResult &res) {
  res.C[0] = res.C[1] = res.C[2] = 0.f;
  res.A = 0.f;
  res.dnum = 0.f;
  res.tau = 0.f;
  res.nseg = 0;
}

// One ray given in the tree's own frame (render kernels).
template <int KP, int DEG, typename E, bool kSmem>
__device__ __forceinline__ void integrate_ray(const DevTree &tr, const uint32_t *s_child, const float o[3],
                                              const float d[3], float u, float t_stop, int act, RayResult &res) {
  clear(res);
  RayWalk w;
  float dn[3];
  if (!walk_init(tr, o, d, w, dn)) return;
  integrate_walk<KP, DEG, E, kSmem>(tr, s_child, w, dn, u, t_stop, act, w.t_base, 1.f, res);
}

__device__ __forceinline__ float depth_of(const RayResult &r) { return r.A >= 1e-4f ? r.dnum / r.A : INFINITY; }

}  // namespace neuvv
