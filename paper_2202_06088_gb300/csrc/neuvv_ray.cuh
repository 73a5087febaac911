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

// Walks the ray and composites front to back, stopping after the segment that
// brings the transmittance below t_stop.  u is the frame coordinate.
template <int KP, int DEG, typename E, bool kSmem>
__device__ __forceinline__ void integrate_ray(const DevTree &tr, const uint32_t *s_child, const float o[3],
                                              const float d[3], float u, float t_stop, int act, RayResult &res) {
  res.C[0] = res.C[1] = res.C[2] = 0.f;
  res.A = 0.f;
  res.dnum = 0.f;
  res.tau = 0.f;
  res.nseg = 0;
  RayWalk w;
  float dn[3];
  if (!walk_init(tr, o, d, w, dn)) return;
  RayConst<KP, DEG> rc;
  ray_const_basis<KP, DEG>(tr, u, rc);
  sh_real<DEG>(dn, rc.Y);
  float T = 1.f;
  uint32_t leaf;
  float t0, t1;
  while (walk_next<kSmem>(tr, s_child, w, leaf, t0, t1)) {
    LeafRecord<KP, DEG, E> rec;
    rec.load(tr, leaf);
    Sample<DEG> s;
    eval_sample<KP, DEG, E>(tr, rc, rec, act, s);
    res.nseg += 1;
    if (s.sigma > 0.f) {
      const float delta = t1 - t0;
      const float sd = s.sigma * delta;
      const float e = __expf(-sd);
      const float wgt = T * (1.f - e);
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) res.C[ch] = fmaf(wgt, s.c[ch], res.C[ch]);
      res.A += wgt;
      res.dnum = fmaf(wgt, w.t_base + 0.5f * (t0 + t1), res.dnum);
      res.tau += sd;
      T *= e;
      if (T < t_stop) break;
    }
  }
}

__device__ __forceinline__ float depth_of(const RayResult &r) { return r.A >= 1e-4f ? r.dnum / r.A : INFINITY; }

}  // namespace neuvv
