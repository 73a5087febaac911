// Fused adjoint of the VOctree renderer (Sec. 4.3 "Optimization": the
// derivatives of the volume-rendering loss with respect to the leaf
// coefficients, for SGD/Adam directly on the VOctree).
//
// No per-sample state is stored by the forward pass.  Each ray is replayed
// with the forward's traversal; per sample the kernel recomputes sigma,
// gamma, the harmonics and the colour, and forms
//   dL/dc_i     = w_i g
//   dL/dsigma_i = delta_i ( g . (T_{i+1} c_i - S_{>i}) + g_alpha T_final )
// where S_{>i} = C - sum_{j<=i} w_j c_j is the radiance still to come behind
// sample i (the back-to-front quantity, taken from the saved C without a
// reverse walk or a division) and T_final = exp(-tau) from the saved optical
// depth.  The chain continues through ReLU (zero slope at pre-activation <= 0),
// pi*sigmoid and d H / d gamma.  Gradients are scattered into an FP32
// record-layout buffer with 16-byte vector atomics.
#include "neuvv_kernels.h"
#include "neuvv_ray.cuh"

namespace neuvv {

__device__ __forceinline__ void red_add_v4(float *addr, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}

template <int KP, int DEG, typename E, bool kSmem>
__device__ __forceinline__ void adjoint_ray(const BwdArgs &a, const uint32_t *s_child, long long i) {
  constexpr int NH = n_hh(DEG);
  constexpr int LEN = 2 * KP + 3 * NH;
  constexpr int LEN4 = (LEN + 3) / 4 * 4;
  const int nseg = a.nseg[i];
  if (nseg <= 0) return;
  float o[3], d[3], t;
  load_ray(a.rays, i, o, d, t);
  const float g[3] = {a.grad_rgb[3 * i], a.grad_rgb[3 * i + 1], a.grad_rgb[3 * i + 2]};
  const float gA = a.grad_alpha ? a.grad_alpha[i] : 0.f;
  const float C[3] = {a.rgb[3 * i], a.rgb[3 * i + 1], a.rgb[3 * i + 2]};
  const float T_final = __expf(-a.tau[i]);
  const DevTree &tr = a.tr;
  RayWalk w;
  float dn[3];
  if (!walk_init(tr, o, d, w, dn)) return;
  RayConst<KP, DEG> rc;
  ray_const_basis<KP, DEG>(tr, t * (float)(tr.T - 1), rc);
  sh_real<DEG>(dn, rc.Y);
  float T = 1.f, acc[3] = {0.f, 0.f, 0.f};
  uint32_t leaf;
  float t0, t1;
  int count = 0;
  while (count < nseg && walk_next<kSmem>(tr, s_child, w, leaf, t0, t1)) {
    ++count;
    LeafRecord<KP, DEG, E> rec;
    rec.load(tr, leaf);
    Sample<DEG> s;
    eval_sample<KP, DEG, E>(tr, rc, rec, a.act, s);
    if (!(s.sigma > 0.f)) continue;  // alpha = 0: no path from this sample to L
    const float delta = t1 - t0;
    const float e = __expf(-s.sigma * delta);
    const float wgt = T * (1.f - e);
    const float Tn = T * e;
    float dsig = gA * T_final;
    float dz[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      acc[ch] = fmaf(wgt, s.c[ch], acc[ch]);
      const float S_after = C[ch] - acc[ch];
      dsig = fmaf(g[ch], Tn * s.c[ch] - S_after, dsig);
      const float dc = wgt * g[ch];
      dz[ch] = a.act == 0 ? dc * s.c[ch] * (1.f - s.c[ch]) : dc;
    }
    dsig *= delta;
    T = Tn;
    // d/dgamma of the colour pre-activations
    float R[(DEG + 1) * (DEG + 2) / 2], dR[(DEG + 1) * (DEG + 2) / 2];
    hh_radial<DEG, true>(s.cg, s.sg, tr.hh_norm, R, dR);
    float grad[LEN4];
    float dgam = 0.f;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
#pragma unroll
      for (int n = 0; n <= DEG; ++n)
#pragma unroll
        for (int l = 0; l <= n; ++l) {
          float wy = 0.f;
#pragma unroll
          for (int m = -l; m <= l; ++m) {
            const int idx = hh_index(n, l, m);
            const float Y = rc.Y[l * l + l + m];
            grad[2 * KP + ch * NH + idx] = dz[ch] * R[radial_index(n, l)] * Y;
            wy = fmaf(rec.hh(ch, idx), Y, wy);
          }
          dgam = fmaf(dz[ch] * wy, dR[radial_index(n, l)], dgam);
        }
    }
    const float dpre_g = dgam * kPi * s.s_gamma * (1.f - s.s_gamma);
    const float dpre_s = s.pre_sigma > 0.f ? dsig : 0.f;
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      grad[k] = dpre_s * rc.a[k];
      grad[KP + k] = dpre_g * rc.b[k];
    }
#pragma unroll
    for (int k = LEN; k < LEN4; ++k) grad[k] = 0.f;
    float *dst = a.grad + (size_t)leaf * a.grad_stride;
#pragma unroll
    for (int q = 0; q < LEN4 / 4; ++q)
      red_add_v4(dst + 4 * q, grad[4 * q], grad[4 * q + 1], grad[4 * q + 2], grad[4 * q + 3]);
    if (a.touched) {
      const unsigned int bit = 1u << (leaf & 31);
      unsigned int *word = a.touched + (leaf >> 5);
      if (!(__ldcg(word) & bit)) atomicOr(word, bit);
    }
  }
}

template <int KP, int DEG, typename E>
__global__ void __launch_bounds__(256) render_bwd_plain_kernel(BwdArgs a) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.rays.n) return;
  adjoint_ray<KP, DEG, E, false>(a, nullptr, i);
}

template <int KP, int DEG, typename E>
__global__ void __launch_bounds__(256) render_bwd_packet_kernel(BwdArgs a, int dynamic) {
  extern __shared__ __align__(16) uint32_t s_child[];
  {
    const int words = a.tr.smem_nodes * 8;
    const uint4 *src = reinterpret_cast<const uint4 *>(a.tr.child);
    uint4 *dst = reinterpret_cast<uint4 *>(s_child);
    for (int k = threadIdx.x; k < words / 4; k += blockDim.x) dst[k] = __ldg(src + k);
    __syncthreads();
  }
  const long long n = a.rays.n;
  const long long n_packets = (n + 31) >> 5;
  const long long stride = ((long long)gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  long long p;
  if (dynamic) {
    unsigned int q = 0;
    if (lane == 0) q = atomicAdd(a.work, 1u);
    p = (long long)__shfl_sync(0xFFFFFFFFu, q, 0);
  } else {
    p = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  }
  while (p < n_packets) {
    const long long i = (p << 5) + lane;
    if (i < n) adjoint_ray<KP, DEG, E, true>(a, s_child, i);
    __syncwarp();
    if (dynamic) {
      unsigned int q = 0;
      if (lane == 0) q = atomicAdd(a.work, 1u);
      p = (long long)__shfl_sync(0xFFFFFFFFu, q, 0);
    } else {
      p += stride;
    }
  }
}

template <int KP, int DEG, typename E>
static cudaError_t bwd_one(bool packet, const BwdArgs &a, const LaunchCfg &cfg, cudaStream_t s) {
  if (a.rays.n == 0) return cudaSuccess;
  if (!packet) {
    const long long blocks = (a.rays.n + cfg.block - 1) / cfg.block;
    render_bwd_plain_kernel<KP, DEG, E><<<(unsigned)blocks, cfg.block, 0, s>>>(a);
  } else {
    const size_t sm = smem_bytes(a.tr.smem_nodes);
    if (sm > 48 * 1024)
      cudaFuncSetAttribute(render_bwd_packet_kernel<KP, DEG, E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    render_bwd_packet_kernel<KP, DEG, E><<<cfg.grid, cfg.block, sm, s>>>(a, cfg.dynamic_queue);
  }
  return cudaGetLastError();
}

template <typename E>
static cudaError_t bwd_dispatch(int KP, int DEG, bool packet, const BwdArgs &a, const LaunchCfg &cfg, cudaStream_t s) {
  switch (KP * 10 + DEG) {
    case 81: return bwd_one<8, 1, E>(packet, a, cfg, s);
    case 82: return bwd_one<8, 2, E>(packet, a, cfg, s);
    case 83: return bwd_one<8, 3, E>(packet, a, cfg, s);
    case 161: return bwd_one<16, 1, E>(packet, a, cfg, s);
    case 162: return bwd_one<16, 2, E>(packet, a, cfg, s);
    case 163: return bwd_one<16, 3, E>(packet, a, cfg, s);
    case 321: return bwd_one<32, 1, E>(packet, a, cfg, s);
    case 322: return bwd_one<32, 2, E>(packet, a, cfg, s);
    case 323: return bwd_one<32, 3, E>(packet, a, cfg, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_render_bwd(int KP, int DEG, DType dt, bool packet, const BwdArgs &a, const LaunchCfg &cfg,
                              cudaStream_t s) {
  if (dt == kF32) return bwd_dispatch<float>(KP, DEG, packet, a, cfg, s);
  return bwd_dispatch<__nv_bfloat16>(KP, DEG, packet, a, cfg, s);
}

}  // namespace neuvv
