// Forward render and trace kernels (Sec. 4.3 "Rendering").
//
// render_plain_kernel  : one thread per ray, child table read from global
//                        memory -- the baseline single-view path.
// render_packet_kernel : persistent grid; each block stages the top of the
//                        child table in shared memory once, then its warps
//                        take 32-ray packets (coherent 8x4 pixel tiles when the
//                        caller orders rays that way) from a global counter or
//                        a static stride until the batch is done.
#include "neuvv_kernels.h"
#include "neuvv_ray.cuh"

namespace neuvv {

template <int KP, int DEG, typename E>
__global__ void __launch_bounds__(256) render_plain_kernel(FwdArgs a) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.rays.n) return;
  float o[3], d[3], t;
  load_ray(a.rays, i, o, d, t);
  RayResult r;
  integrate_ray<KP, DEG, E, false>(a.tr, nullptr, o, d, t * (float)(a.tr.T - 1), a.t_stop, a.act, r);
  a.out.rgb[3 * i + 0] = r.C[0];
  a.out.rgb[3 * i + 1] = r.C[1];
  a.out.rgb[3 * i + 2] = r.C[2];
  a.out.alpha[i] = r.A;
  if (a.out.depth) a.out.depth[i] = depth_of(r);
  if (a.out.tau) a.out.tau[i] = r.tau;
  if (a.out.nseg) a.out.nseg[i] = r.nseg;
}

// Copies the first `rows` rows of the child table to shared memory.
__device__ __forceinline__ void stage_child(const DevTree &tr, uint32_t *s_child) {
  const int words = tr.smem_nodes * 8;
  const uint4 *src = reinterpret_cast<const uint4 *>(tr.child);
  uint4 *dst = reinterpret_cast<uint4 *>(s_child);
  for (int i = threadIdx.x; i < words / 4; i += blockDim.x) dst[i] = __ldg(src + i);
  __syncthreads();
}

// Next packet of a warp: from the counter (dynamic) or by static stride.
__device__ __forceinline__ long long next_packet(unsigned int *work, bool dynamic, long long cur, long long stride) {
  if (dynamic) {
    unsigned int p = 0;
    if ((threadIdx.x & 31) == 0) p = atomicAdd(work, 1u);
    return (long long)__shfl_sync(0xFFFFFFFFu, p, 0);
  }
  return cur + stride;
}

__device__ __forceinline__ long long first_packet(unsigned int *work, bool dynamic) {
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  return dynamic ? next_packet(work, true, 0, 0) : warp;
}

template <int KP, int DEG, typename E>
__global__ void __launch_bounds__(256) render_packet_kernel(FwdArgs a, int dynamic) {
  extern __shared__ __align__(16) uint32_t s_child[];
  stage_child(a.tr, s_child);
  const long long n = a.rays.n;
  const long long n_packets = (n + 31) >> 5;
  const long long stride = ((long long)gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  for (long long p = first_packet(a.work, dynamic); p < n_packets; p = next_packet(a.work, dynamic, p, stride)) {
    const long long i = (p << 5) + lane;
    if (i < n) {
      float o[3], d[3], t;
      load_ray(a.rays, i, o, d, t);
      RayResult r;
      integrate_ray<KP, DEG, E, true>(a.tr, s_child, o, d, t * (float)(a.tr.T - 1), a.t_stop, a.act, r);
      a.out.rgb[3 * i + 0] = r.C[0];
      a.out.rgb[3 * i + 1] = r.C[1];
      a.out.rgb[3 * i + 2] = r.C[2];
      a.out.alpha[i] = r.A;
      if (a.out.depth) a.out.depth[i] = depth_of(r);
      if (a.out.tau) a.out.tau[i] = r.tau;
      if (a.out.nseg) a.out.nseg[i] = r.nseg;
    }
    __syncwarp();
  }
}

__global__ void __launch_bounds__(256) trace_kernel(TraceArgs a) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.rays.n) return;
  float o[3], d[3], t;
  load_ray(a.rays, i, o, d, t);
  RayWalk w;
  float dn[3];
  int c = 0;
  if (walk_init(a.tr, o, d, w, dn)) {
    uint32_t leaf;
    float t0, t1;
    while (walk_next<false>(a.tr, nullptr, w, leaf, t0, t1)) {
      if (c < a.max_out) {
        a.leaf[i * a.max_out + c] = (int)leaf;
        a.t0[i * a.max_out + c] = w.t_base + t0;
        a.t1[i * a.max_out + c] = w.t_base + t1;
      }
      ++c;
    }
  }
  for (int k = c; k < a.max_out; ++k) {
    a.leaf[i * a.max_out + k] = -1;
    a.t0[i * a.max_out + k] = 0.f;
    a.t1[i * a.max_out + k] = 0.f;
  }
  a.count[i] = c;
}

template <int KP, int DEG, typename E>
static cudaError_t fwd_one(bool packet, const FwdArgs &a, const LaunchCfg &cfg, cudaStream_t s) {
  if (a.rays.n == 0) return cudaSuccess;
  if (!packet) {
    const long long blocks = (a.rays.n + cfg.block - 1) / cfg.block;
    render_plain_kernel<KP, DEG, E><<<(unsigned)blocks, cfg.block, 0, s>>>(a);
  } else {
    const size_t sm = smem_bytes(a.tr.smem_nodes);
    if (sm > 48 * 1024)
      cudaFuncSetAttribute(render_packet_kernel<KP, DEG, E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    render_packet_kernel<KP, DEG, E><<<cfg.grid, cfg.block, sm, s>>>(a, cfg.dynamic_queue);
  }
  return cudaGetLastError();
}

#define NEUVV_DISPATCH_KD(FN, ...)                                              \
  switch (KP * 10 + DEG) {                                                       \
    case 81: return FN<8, 1, E>(__VA_ARGS__);                                   \
    case 82: return FN<8, 2, E>(__VA_ARGS__);                                   \
    case 83: return FN<8, 3, E>(__VA_ARGS__);                                   \
    case 161: return FN<16, 1, E>(__VA_ARGS__);                                 \
    case 162: return FN<16, 2, E>(__VA_ARGS__);                                 \
    case 163: return FN<16, 3, E>(__VA_ARGS__);                                 \
    case 321: return FN<32, 1, E>(__VA_ARGS__);                                 \
    case 322: return FN<32, 2, E>(__VA_ARGS__);                                 \
    case 323: return FN<32, 3, E>(__VA_ARGS__);                                 \
    default: return cudaErrorInvalidValue;                                      \
  }

template <typename E>
static cudaError_t fwd_dispatch(int KP, int DEG, bool packet, const FwdArgs &a, const LaunchCfg &cfg, cudaStream_t s) {
  NEUVV_DISPATCH_KD(fwd_one, packet, a, cfg, s)
}

cudaError_t launch_render_fwd(int KP, int DEG, DType dt, bool packet, const FwdArgs &a, const LaunchCfg &cfg,
                              cudaStream_t s) {
  if (dt == kF32) return fwd_dispatch<float>(KP, DEG, packet, a, cfg, s);
  return fwd_dispatch<__nv_bfloat16>(KP, DEG, packet, a, cfg, s);
}

cudaError_t launch_trace(const TraceArgs &a, cudaStream_t s) {
  if (a.rays.n == 0) return cudaSuccess;
  const long long blocks = (a.rays.n + 127) / 128;
  trace_kernel<<<(unsigned)blocks, 128, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace neuvv
