// Forward render and trace kernels (Sec. 4.3 "Rendering").
//
// render_plain_kernel  : one thread per ray, child table read from global
//                        memory -- the baseline single-view path.
// render_packet_kernel : one thread per ray with warps as 32-ray packets;
//                        walking and shading decoupled through a per-lane
//                        queue of found segments; descents restart at the
//                        lowest common ancestor of successive cells.
#include "neuvv_kernels.h"
#include "neuvv_ray.cuh"

namespace neuvv {

template <int KP, int DEG, typename E>
__global__ void __launch_bounds__(256) render_plain_kernel(const __grid_constant__ FwdArgs a) {
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

// Outputs and the segment log are written once and read by later launches:
// stores with the evict-first (streaming) policy.
__device__ __forceinline__ void write_miss(const DevOut &out, long long i) {
  if (out.rgb) {
    __stcs(out.rgb + 3 * i + 0, 0.f);
    __stcs(out.rgb + 3 * i + 1, 0.f);
    __stcs(out.rgb + 3 * i + 2, 0.f);
  }
  __stcs(out.alpha + i, 0.f);
  if (out.depth) __stcs(out.depth + i, INFINITY);
  if (out.tau) __stcs(out.tau + i, 0.f);
  if (out.nseg) __stcs(out.nseg + i, 0);
}

// Packet forward kernel: one thread per ray, so each warp is a packet of 32
// consecutive rays (an 8x4 pixel tile when the caller orders rays that way).
// Walking and shading are decoupled: in every iteration of one warp-uniform
// loop each lane takes at most one walk step and queues the occupied-leaf
// segment it finds; the warp runs a shading round (each lane evaluates and
// composites its oldest queued segment, in ray order) once `ready` lanes hold
// one, or when no lane can step any further.  Lanes therefore do not wait at
// every sample for the slowest searcher of the packet, and shading rounds run
// nearly full.  Descents restart at the lowest common ancestor of successive
// cells (path per thread in shared memory); basis rows and the queue live in
// shared memory too.
// kShade: kShadeTree (the tree's records), kShadeSlice (a time slice,
// a.slice), kShadeEdit (the tree's records with appearance edits, a.edits) or
// kShadeAlpha (density only: the w_sigma part of each record is read, colour
// is neither evaluated nor written; alpha, depth, tau and nseg are those of
// the full render).
constexpr int kShadeTree = 0, kShadeSlice = 1, kShadeEdit = 2, kShadeAlpha = 3;
template <int KP, int DEG, typename E, int kShade = kShadeTree>
__device__ __forceinline__ void packet_forward(const FwdArgs &a, long long pos, long long i, unsigned present,
                                               int queue, int ready) {
  extern __shared__ __align__(16) uint32_t smem[];
  const DevTree &tr = a.tr;
  const int B = blockDim.x, tid = threadIdx.x;
  float *my_rows = reinterpret_cast<float *>(smem) + tid;
  const PathRef pr{smem + 2 * KP * B + tid, B};
  uint32_t *q_leaf = smem + (2 * KP + path_words(tr)) * B + tid;
  float *q_t0 = reinterpret_cast<float *>(q_leaf + queue * B);
  float *q_dt = q_t0 + queue * B;
  const SmemRows<KP> rows{my_rows, B};
  float o[3], d[3], t, dn[3];
  load_ray(a.rays, i, o, d, t);
  RayWalk w;
  const bool hit = walk_init(tr, o, d, w, dn);
  if (!hit) write_miss(a.out, i);
  // i: the ray (its data and outputs); pos: its position (packet pos >> 5, lane)
  if (a.log.n_chunks && (threadIdx.x & 31) == __ffs(present) - 1) {
    a.log.key[pos >> 5] = kNoKey;
    a.log.heads[pos >> 5] = kNoLog;  // until the packet's first chunk
  }
  if (__ballot_sync(present, hit) == 0) return;  // the whole packet missed the tree
  if (hit && kShade != kShadeSlice) rows_to_smem<KP>(tr, t * (float)(tr.T - 1), my_rows, B);
  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, A = 0.f, dnum = 0.f, tau = 0.f;
  int nseg = 0;
  bool walking = hit && w.alive;
  int qh = 0, qn = 0;  // queue head and length
  const int qmask = queue - 1;
  // segment log of this packet (warp-uniform state): current chunk and round
  const int lane = threadIdx.x & 31;
  const long long pk = pos >> 5;
  bool logging = a.log.n_chunks != 0;
  uint32_t chunk = kNoLog;
  int round = kLogRounds;
  for (;;) {
    if (walking && qn < queue) {
      uint32_t leaf;
      float t0, dt;
      if (walk_step<false, true>(tr, nullptr, w, leaf, t0, dt, pr)) {
        const int slot = (qh + qn) & qmask;
        q_leaf[slot * B] = leaf;
        q_t0[slot * B] = t0;
        q_dt[slot * B] = dt;
        ++qn;
        // the record is read when the segment's round comes: ask L2 for it now
        if (kShade == kShadeSlice) slice_prefetch_l2(a.slice, a.slice_stride, DEG, leaf);
        else if (kShade == kShadeAlpha) LeafRecord<KP, DEG, E>::prefetch_sigma_l2(tr, leaf);
        else LeafRecord<KP, DEG, E>::prefetch_l2(tr, leaf);
      }
      walking = w.alive;
    }
    const unsigned have = __ballot_sync(present, qn > 0);
    const unsigned stepping = __ballot_sync(present, walking && qn < queue);
    if (!have && !stepping) break;
    const int active = __popc(__ballot_sync(present, walking || qn > 0));
    if (stepping && __popc(have) < min(ready, active)) continue;
    if (logging) {
      if (round == kLogRounds) {  // next chunk: one counter add per 8 rounds
        const int leader = __ffs(present) - 1;
        if (chunk == kNoLog) {  // the packet's sort key: the smallest leaf of its first round
          const uint32_t k = __reduce_min_sync(present, qn > 0 ? q_leaf[qh * B] : kNoKey);
          if (lane == leader) a.log.key[pk] = k;
        }
        uint32_t nc = kNoLog;
        if (lane == leader) {
          const unsigned long long c = atomicAdd(a.log.counter, 1ull);
          if (c < a.log.n_chunks) {
            nc = (uint32_t)c;
            if (chunk == kNoLog) a.log.heads[pk] = nc;
            else a.log.next[chunk] = nc;
          } else {
            a.log.heads[pk] = kNoLog;  // out of room: the adjoint walks this packet
          }
        }
        nc = __shfl_sync(present, nc, leader);
        logging = nc != kNoLog;
        chunk = nc;
        round = 0;
      }
      if (logging) {
        const size_t slot = ((size_t)chunk * kLogRounds + round) * 32 + lane;
        __stcs(a.log.leaf + slot, qn > 0 ? q_leaf[qh * B] : kEmpty);
        __stcs(a.log.dt + slot, qn > 0 ? q_dt[qh * B] : 0.f);
        ++round;
      }
    }
    if (qn > 0) {
      const uint32_t leaf = q_leaf[qh * B];
      const float t0 = q_t0[qh * B], dt = q_dt[qh * B];
      qh = (qh + 1) & qmask;
      --qn;
      float sigma, col[3];
      // the harmonics of the ray's direction, formed per round rather than
      // held through the walk (16 registers fewer across the loop)
      float Y[(DEG + 1) * (DEG + 1)];
      if (kShade != kShadeAlpha) sh_real<DEG>(dn, Y);
      if constexpr (kShade == kShadeSlice) {
        shade_slice<DEG>(a.slice, a.slice_stride, leaf, Y, a.act, sigma, col);
      } else if constexpr (kShade == kShadeAlpha) {
        LeafRecord<KP, DEG, E> rec;
        rec.load_sigma(tr, leaf);
        sigma = fmaxf(pre_sigma_of<KP>(rows, rec), 0.f);
        col[0] = col[1] = col[2] = 0.f;
      } else {
        LeafRecord<KP, DEG, E> rec;
        rec.load(tr, leaf);
        Sample<DEG> s;
        eval_sample<KP, DEG, E>(tr, rows, Y, rec, a.act, s);
        sigma = s.sigma;
        col[0] = s.c[0];
        col[1] = s.c[1];
        col[2] = s.c[2];
        if constexpr (kShade == kShadeEdit) {
          // appearance edit of the voxel, active from its time t_d on
          const float4 e0 = __ldg(reinterpret_cast<const float4 *>(a.edits) + 2 * (size_t)leaf);
          const float4 e1 = __ldg(reinterpret_cast<const float4 *>(a.edits) + 2 * (size_t)leaf + 1);
          if (t >= e1.x) {
            if (e0.w >= 0.f) sigma = e0.w;
            col[0] = fmaf(a.edit_beta, e0.x - col[0], col[0]);
            col[1] = fmaf(a.edit_beta, e0.y - col[1], col[1]);
            col[2] = fmaf(a.edit_beta, e0.z - col[2], col[2]);
          }
        }
      }
      ++nseg;
      if (sigma > 0.f) {
        const float sd = sigma * dt;
        const float e = __expf(-sd);
        const float wgt = T * alpha_of(sd);
        C0 = fmaf(wgt, col[0], C0);
        C1 = fmaf(wgt, col[1], C1);
        C2 = fmaf(wgt, col[2], C2);
        A += wgt;
        dnum = fmaf(wgt, w.t_base + fmaf(0.5f, dt, t0), dnum);
        tau += sd;
        T *= e;
        if (T < a.t_stop) {  // early termination: drop what is still queued
          walking = false;
          qn = 0;
        }
      }
    }
  }
  if (logging) {
    // slots that hold no segment read kEmpty, so that the log can be read
    // slot by slot: the rounds of the last chunk that the packet did not
    // reach, and in the packet past the last ray, the slots of its absent
    // lanes in every chunk
    for (int r = round; r < kLogRounds; ++r) a.log.leaf[((size_t)chunk * kLogRounds + r) * 32 + lane] = kEmpty;
    if (present != 0xFFFFFFFFu && lane == __ffs(present) - 1) {
      uint32_t c = a.log.heads[pk];
      for (uint32_t k = 0; k < a.log.n_chunks && c < a.log.n_chunks; ++k) {
        for (int j = 0; j < kLogRounds * 32; ++j)
          if (!((present >> (j & 31)) & 1u)) a.log.leaf[(size_t)c * kLogRounds * 32 + j] = kEmpty;
        if (c == chunk) break;
        c = a.log.next[c];
      }
    }
  }
  if (!hit) return;
  if (kShade != kShadeAlpha) {
    __stcs(a.out.rgb + 3 * i + 0, C0);
    __stcs(a.out.rgb + 3 * i + 1, C1);
    __stcs(a.out.rgb + 3 * i + 2, C2);
  }
  __stcs(a.out.alpha + i, A);
  if (a.out.depth) __stcs(a.out.depth + i, A >= 1e-4f ? dnum / A : INFINITY);
  if (a.out.tau) __stcs(a.out.tau + i, tau);
  if (a.out.nseg) __stcs(a.out.nseg + i, nseg);
}

// Packet forward kernel.  With a work counter the grid is persistent: each
// warp takes the next 32-ray packet from the counter when it finishes one, so
// a long ray holds up only its own warp, not the other warps of its block.
template <int KP, int DEG, typename E, int kShade = kShadeTree>
__global__ void __launch_bounds__(256, packet_min_blocks<E>()) render_packet_kernel(const __grid_constant__ FwdArgs a, int queue, int ready) {
  // one packet per warp of the grid, or (with a work counter) packets pulled
  // one after another until the counter passes the last
  const int lane = threadIdx.x & 31;
  const long long n_packets = (a.rays.n + 31) >> 5;
  if (a.log.n_chunks && blockIdx.x == 0 && threadIdx.x == 0) {
    a.log.header[0] = a.log.n_chunks;
    a.log.header[1] = kLogRounds;
    a.log.header[2] = (uint32_t)(a.rays.n & 0xFFFFFFFFll);
    a.log.header[3] = (uint32_t)(a.rays.n >> 32);
    a.log.header[4] = 1u;
    a.log.header[5] = a.perm ? 1u : 0u;
  }
  long long pk = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (a.work) {
    unsigned long long q = 0;
    if (lane == 0) q = atomicAdd(a.work, 1ull);
    pk = (long long)__shfl_sync(0xFFFFFFFFu, q, 0);
  }
  while (pk < n_packets) {
    if (a.order) pk = (long long)min(__ldg(a.order + pk), (uint32_t)(n_packets - 1));
    const long long pos = (pk << 5) + lane;
    // lanes past the end sit the packet out; the others stay to its end
    const unsigned present = __ballot_sync(0xFFFFFFFFu, pos < a.rays.n);
    if (pos < a.rays.n) {
      const long long i = a.perm ? (long long)min(__ldg(a.perm + pos), (uint32_t)(a.rays.n - 1)) : pos;
      packet_forward<KP, DEG, E, kShade>(a, pos, i, present, queue, ready);
    }
    __syncwarp();
    if (!a.work) break;
    unsigned long long q = 0;
    if (lane == 0) q = atomicAdd(a.work, 1ull);
    pk = (long long)__shfl_sync(0xFFFFFFFFu, q, 0);
  }
}

__global__ void __launch_bounds__(256) trace_kernel(const __grid_constant__ TraceArgs a) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.rays.n) return;
  float o[3], d[3], t;
  load_ray(a.rays, i, o, d, t);
  RayWalk w;
  float dn[3];
  int c = 0;
  if (walk_init(a.tr, o, d, w, dn)) {
    uint32_t leaf;
    float t0, dt;
    while (walk_next<false>(a.tr, nullptr, w, leaf, t0, dt)) {
      if (c < a.max_out) {
        a.leaf[i * a.max_out + c] = (int)leaf;
        a.t0[i * a.max_out + c] = w.t_base + t0;
        a.t1[i * a.max_out + c] = w.t_base + (t0 + dt);
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
  const long long blocks = (a.rays.n + cfg.block - 1) / cfg.block;
  if (!packet) {
    render_plain_kernel<KP, DEG, E><<<(unsigned)blocks, cfg.block, 0, s>>>(a);
  } else {
    const size_t sm = smem_bytes(cfg.block, KP, cfg.queue, a.tr);
    if (sm > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(render_packet_kernel<KP, DEG, E>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
    }
    if (!a.work) {
      render_packet_kernel<KP, DEG, E><<<(unsigned)blocks, cfg.block, sm, s>>>(a, cfg.queue, cfg.ready);
    } else {
      int per_sm = 0;
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, render_packet_kernel<KP, DEG, E>,
                                                                    cfg.block, sm);
      if (e != cudaSuccess) return e;
      const long long want = (long long)(per_sm > 0 ? per_sm : 1) * cfg.num_sms;
      e = cudaMemsetAsync(a.work, 0, sizeof(unsigned long long), s);
      if (e != cudaSuccess) return e;
      render_packet_kernel<KP, DEG, E><<<(unsigned)(want < blocks ? want : blocks), cfg.block, sm, s>>>(
          a, cfg.queue, cfg.ready);
    }
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
  if (dt == kBF16) return fwd_dispatch<__nv_bfloat16>(KP, DEG, packet, a, cfg, s);
  // FP8 storage is built for the two record shapes of the workloads only
  if (KP == 8 && DEG == 2) return fwd_one<8, 2, Fp8E4M3>(packet, a, cfg, s);
  if (KP == 16 && DEG == 3) return fwd_one<16, 3, Fp8E4M3>(packet, a, cfg, s);
  return cudaErrorInvalidValue;
}

// Time slice of one leaf whose record is loaded: density and hyper angle from
// the basis rows at frame coordinate u (Eq. project-sigma, Eq. project-gamma),
// the radial factors R_nl(gamma) by the Gegenbauer recurrence, then
// s[ch][l,m] = sum_{n >= l} w[ch][n,l,m] R_nl (Eq. HH-color-2 with gamma
// fixed), written as one slice row of NV float4.
template <int KP, int DEG, typename E>
__device__ __forceinline__ void slice_row(const DevTree &tr, const RegRows<KP> &rows, const LeafRecord<KP, DEG, E> &rec,
                                          float4 *dst) {
  constexpr int NY = (DEG + 1) * (DEG + 1), NV = slice_min_stride(DEG) / 4;
  float out[NV * 4];
#pragma unroll
  for (int k = 0; k < NV * 4; ++k) out[k] = 0.f;
  out[0] = fmaxf(pre_sigma_of<KP>(rows, rec), 0.f);
  float q4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < KP; ++k) q4[k & 3] = fmaf(rows.B(k), rec.gam(k), q4[k & 3]);
  const float pg = ((q4[0] + q4[1]) + (q4[2] + q4[3])) * rec.scale_gamma();
  float sg, cg, R[(DEG + 1) * (DEG + 2) / 2];
  sincospif(sigmoidf_fast(pg), &sg, &cg);
  hh_radial<DEG, false>(cg, sg, tr.hh_norm, R, nullptr);
#pragma unroll
  for (int ch = 0; ch < 3; ++ch)
#pragma unroll
    for (int l = 0; l <= DEG; ++l)
#pragma unroll
      for (int m = -l; m <= l; ++m) {
        float acc = 0.f;
#pragma unroll
        for (int n = l; n <= DEG; ++n) acc = fmaf(rec.hh(ch, hh_index(n, l, m)), R[radial_index(n, l)], acc);
        out[4 + ch * NY + l * l + l + m] = acc * rec.scale_hh();
      }
#pragma unroll
  for (int i = 0; i < NV; ++i) dst[i] = make_float4(out[4 * i], out[4 * i + 1], out[4 * i + 2], out[4 * i + 3]);
}

// Time slice, one thread per leaf, records read from global memory (any
// record and row size).
template <int KP, int DEG, typename E>
__global__ void __launch_bounds__(256) slice_kernel(const __grid_constant__ DevTree tr, float u, float *slice,
                                                    int stride) {
  const long long leaf = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (leaf >= tr.n_leaves) return;
  RayConst<KP, DEG> rc;
  ray_const_basis<KP, DEG>(tr, u, rc);
  LeafRecord<KP, DEG, E> rec;
  rec.load(tr, (uint32_t)leaf);
  slice_row<KP, DEG, E>(tr, RegRows<KP>{rc.a, rc.b}, rec, reinterpret_cast<float4 *>(slice + (size_t)leaf * stride));
}

// Bulk copies between global and shared memory through the TMA unit.
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Waits until the mbarrier's phase `parity` completes, for at most `limit`
// polls; false on time-out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int limit) {
  for (int k = 0; k < limit; ++k) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

constexpr int kSliceTile = 64;    // leaves per tile (one per thread)
// Polls of the wait that lets a tile's copy in flight land after the tile's
// own wait gave up (the block must not exit while the copy writes into its
// shared memory).
constexpr int kSliceDrainPolls = 1 << 22;

// Time slice with TMA staging: a block takes tiles of kSliceTile consecutive
// leaves; one thread loads the tile's records (consecutive in memory) into
// shared memory with a single bulk copy completed on an mbarrier, every
// thread turns its record into its slice row in a shared output tile, and one
// bulk copy stores the tile's rows (consecutive in memory when the row
// stride is the minimal one).  A wait that does not complete within the
// tree's poll limit flags kStatusTimeout; the whole block then waits (again
// bounded) for its copy in flight to land and ends.
template <int KP, int DEG, typename E>
__global__ void __launch_bounds__(kSliceTile) slice_tma_kernel(const __grid_constant__ DevTree tr, float u,
                                                               float *slice, int rec_bytes) {
  constexpr int NV = slice_min_stride(DEG) / 4;
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ __align__(8) unsigned long long bar;
  uint4 *in = reinterpret_cast<uint4 *>(sm);
  float4 *out = reinterpret_cast<float4 *>(sm + (size_t)kSliceTile * rec_bytes);
  const uint32_t bar_a = smem_addr(&bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  RayConst<KP, DEG> rc;
  ray_const_basis<KP, DEG>(tr, u, rc);
  const RegRows<KP> rows{rc.a, rc.b};
  const long long n_tiles = (tr.n_leaves + kSliceTile - 1) / kSliceTile;
  uint32_t parity = 0;
  for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, parity ^= 1u) {
    const long long first = tile * kSliceTile;
    const int count = (int)min((long long)kSliceTile, tr.n_leaves - first);
    if (threadIdx.x == 0) {
      const uint32_t bytes = (uint32_t)count * (uint32_t)rec_bytes;
      const char *src = static_cast<const char *>(tr.rec) + (size_t)first * rec_bytes;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_a), "r"(bytes) : "memory");
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(in)),
          "l"(src), "r"(bytes), "r"(bar_a)
          : "memory");
    }
    // one decision for the block, so that no thread leaves while others sync
    if (!__syncthreads_and(mbar_wait(bar_a, parity, tr.wait_polls))) {
      if (threadIdx.x == 0) raise_status(tr, kStatusTimeout);
      mbar_wait(bar_a, parity, kSliceDrainPolls);
      if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
      return;
    }
    if ((int)threadIdx.x < count) {
      LeafRecord<KP, DEG, E> rec;
      rec.load_shared(in + (size_t)threadIdx.x * (rec_bytes / 16));
      slice_row<KP, DEG, E>(tr, rows, rec, out + (size_t)threadIdx.x * NV);
    }
    // the rows become visible to the bulk copy (async proxy), then one store
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(slice + (size_t)first * NV * 4),
                   "r"(smem_addr(out)), "r"((uint32_t)count * NV * 16)
                   : "memory");
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      // the output tile and the input buffer are reused by the next tile
      asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // stores complete
}

template <int KP, int DEG, typename E>
static cudaError_t slice_one(const DevTree &tr, float u, float *slice, int stride, int rec_bytes, int num_sms,
                             cudaStream_t s) {
  if (tr.n_leaves == 0) return cudaSuccess;
  if (stride == slice_min_stride(DEG) && rec_bytes % 16 == 0) {
    const size_t sm = (size_t)kSliceTile * (rec_bytes + slice_min_stride(DEG) * 4);
    cudaError_t e;
    if (sm > 48 * 1024 &&
        (e = cudaFuncSetAttribute(slice_tma_kernel<KP, DEG, E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sm)) != cudaSuccess)
      return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, slice_tma_kernel<KP, DEG, E>, kSliceTile, sm)) !=
        cudaSuccess)
      return e;
    const long long tiles = (tr.n_leaves + kSliceTile - 1) / kSliceTile;
    long long grid = (long long)(per_sm > 0 ? per_sm : 1) * num_sms;
    if (grid > tiles) grid = tiles;
    slice_tma_kernel<KP, DEG, E><<<(unsigned)grid, kSliceTile, sm, s>>>(tr, u, slice, rec_bytes);
    return cudaGetLastError();
  }
  slice_kernel<KP, DEG, E><<<(unsigned)((tr.n_leaves + 255) / 256), 256, 0, s>>>(tr, u, slice, stride);
  return cudaGetLastError();
}

cudaError_t launch_slice(int KP, int DEG, DType dt, const DevTree &tr, float u, float *slice, int stride,
                         int rec_bytes, int num_sms, cudaStream_t s) {
#define NEUVV_SLICE_KD(E)                                   \
  switch (KP * 10 + DEG) {                                  \
    case 81: return slice_one<8, 1, E>(tr, u, slice, stride, rec_bytes, num_sms, s);   \
    case 82: return slice_one<8, 2, E>(tr, u, slice, stride, rec_bytes, num_sms, s);   \
    case 83: return slice_one<8, 3, E>(tr, u, slice, stride, rec_bytes, num_sms, s);   \
    case 161: return slice_one<16, 1, E>(tr, u, slice, stride, rec_bytes, num_sms, s); \
    case 162: return slice_one<16, 2, E>(tr, u, slice, stride, rec_bytes, num_sms, s); \
    case 163: return slice_one<16, 3, E>(tr, u, slice, stride, rec_bytes, num_sms, s); \
    case 321: return slice_one<32, 1, E>(tr, u, slice, stride, rec_bytes, num_sms, s); \
    case 322: return slice_one<32, 2, E>(tr, u, slice, stride, rec_bytes, num_sms, s); \
    case 323: return slice_one<32, 3, E>(tr, u, slice, stride, rec_bytes, num_sms, s); \
    default: return cudaErrorInvalidValue;                  \
  }
  if (dt == kF32) NEUVV_SLICE_KD(float)
  if (dt == kBF16) NEUVV_SLICE_KD(__nv_bfloat16)
#undef NEUVV_SLICE_KD
  if (KP == 8 && DEG == 2) return slice_one<8, 2, Fp8E4M3>(tr, u, slice, stride, rec_bytes, num_sms, s);
  if (KP == 16 && DEG == 3) return slice_one<16, 3, Fp8E4M3>(tr, u, slice, stride, rec_bytes, num_sms, s);
  return cudaErrorInvalidValue;
}

// Packet render of a slice: the packet forward with the slice shader (the
// basis-row part of its shared memory is laid out for K_pad = 8 and unused;
// the storage type only sets the register budget, 128 per thread).
template <int DEG>
static cudaError_t render_slice_one(const FwdArgs &a, const LaunchCfg &cfg, cudaStream_t s) {
  if (a.rays.n == 0) return cudaSuccess;
  const long long blocks = (a.rays.n + cfg.block - 1) / cfg.block;
  const bool persistent = a.work != nullptr;
  cudaError_t e;
  if (persistent && (e = cudaMemsetAsync(a.work, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
  const size_t sm = smem_bytes(cfg.block, 8, cfg.queue, a.tr);
  if (sm > 48 * 1024 && (e = cudaFuncSetAttribute(render_packet_kernel<8, DEG, __nv_bfloat16, kShadeSlice>,
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess)
    return e;
  long long grid = blocks;
  if (persistent) {
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, render_packet_kernel<8, DEG, __nv_bfloat16, kShadeSlice>,
                                                           cfg.block, sm)) != cudaSuccess)
      return e;
    const long long want = (long long)(per_sm > 0 ? per_sm : 1) * cfg.num_sms;
    if (want < grid) grid = want;
  }
  render_packet_kernel<8, DEG, __nv_bfloat16, kShadeSlice><<<(unsigned)grid, cfg.block, sm, s>>>(a, cfg.queue, cfg.ready);
  return cudaGetLastError();
}

cudaError_t launch_render_slice(int DEG, const FwdArgs &a, const LaunchCfg &cfg, cudaStream_t s) {
  if (DEG == 1) return render_slice_one<1>(a, cfg, s);
  if (DEG == 2) return render_slice_one<2>(a, cfg, s);
  if (DEG == 3) return render_slice_one<3>(a, cfg, s);
  return cudaErrorInvalidValue;
}

// Terminating voxel of each ray (Sec. 5 "Appearance editing"): the leaf of the
// segment at which 1 - exp(-sum sigma delta) of the unedited render first
// reaches the threshold; -1 when it never does.  One thread per ray.
template <int KP, int DEG, typename E>
__global__ void __launch_bounds__(256) pick_kernel(const __grid_constant__ FwdArgs a, float threshold, int *leaf_out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.rays.n) return;
  float o[3], d[3], t, dn[3];
  load_ray(a.rays, i, o, d, t);
  int picked = -1;
  RayWalk w;
  if (walk_init(a.tr, o, d, w, dn)) {
    RayConst<KP, DEG> rc;
    ray_const_basis<KP, DEG>(a.tr, t * (float)(a.tr.T - 1), rc);
    const RegRows<KP> rows{rc.a, rc.b};
    float optical = 0.f;
    uint32_t leaf;
    float t0, dt;
    while (walk_next<false>(a.tr, nullptr, w, leaf, t0, dt)) {
      LeafRecord<KP, DEG, E> rec;
      rec.load(a.tr, leaf);
      optical = fmaf(fmaxf(pre_sigma_of<KP>(rows, rec), 0.f), dt, optical);
      if (-expm1f(-optical) >= threshold) {
        picked = (int)leaf;
        break;
      }
    }
  }
  leaf_out[i] = picked;
}

template <int KP, int DEG, typename E>
static cudaError_t pick_one(const FwdArgs &a, float threshold, int *leaf_out, cudaStream_t s) {
  if (a.rays.n == 0) return cudaSuccess;
  pick_kernel<KP, DEG, E><<<(unsigned)((a.rays.n + 127) / 128), 128, 0, s>>>(a, threshold, leaf_out);
  return cudaGetLastError();
}

cudaError_t launch_pick(int KP, int DEG, DType dt, const FwdArgs &a, float threshold, int *leaf_out, cudaStream_t s) {
#define NEUVV_PICK_KD(E)                                   \
  switch (KP * 10 + DEG) {                                 \
    case 81: return pick_one<8, 1, E>(a, threshold, leaf_out, s);   \
    case 82: return pick_one<8, 2, E>(a, threshold, leaf_out, s);   \
    case 83: return pick_one<8, 3, E>(a, threshold, leaf_out, s);   \
    case 161: return pick_one<16, 1, E>(a, threshold, leaf_out, s); \
    case 162: return pick_one<16, 2, E>(a, threshold, leaf_out, s); \
    case 163: return pick_one<16, 3, E>(a, threshold, leaf_out, s); \
    case 321: return pick_one<32, 1, E>(a, threshold, leaf_out, s); \
    case 322: return pick_one<32, 2, E>(a, threshold, leaf_out, s); \
    case 323: return pick_one<32, 3, E>(a, threshold, leaf_out, s); \
    default: return cudaErrorInvalidValue;                 \
  }
  if (dt == kF32) NEUVV_PICK_KD(float)
  if (dt == kBF16) NEUVV_PICK_KD(__nv_bfloat16)
#undef NEUVV_PICK_KD
  if (KP == 8 && DEG == 2) return pick_one<8, 2, Fp8E4M3>(a, threshold, leaf_out, s);
  if (KP == 16 && DEG == 3) return pick_one<16, 3, Fp8E4M3>(a, threshold, leaf_out, s);
  return cudaErrorInvalidValue;
}

// Painting: the colours of the rays that picked each leaf are summed (with
// their count) into accum [n_leaves][4], then every leaf with a count gets
// the mean colour, sigma_d and t_d in its edit record [n_leaves][8].
__global__ void __launch_bounds__(256) paint_accum_kernel(const int *leaf, const float *color, long long n,
                                                          long long n_leaves, float *accum) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int l = leaf[i];
  if (l < 0 || l >= n_leaves) return;
  atomicAdd(accum + 4 * (size_t)l + 0, color[3 * i + 0]);
  atomicAdd(accum + 4 * (size_t)l + 1, color[3 * i + 1]);
  atomicAdd(accum + 4 * (size_t)l + 2, color[3 * i + 2]);
  atomicAdd(accum + 4 * (size_t)l + 3, 1.f);
}

__global__ void __launch_bounds__(256) paint_finish_kernel(const float *accum, long long n_leaves, float sigma_d,
                                                           float t_d, float *edits) {
  const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n_leaves) return;
  const float4 s = reinterpret_cast<const float4 *>(accum)[l];
  if (s.w > 0.f) {
    float4 *e = reinterpret_cast<float4 *>(edits) + 2 * l;
    e[0] = make_float4(s.x / s.w, s.y / s.w, s.z / s.w, sigma_d);
    e[1] = make_float4(t_d, 0.f, 0.f, 0.f);
  }
}

cudaError_t launch_paint(const int *leaf, const float *color, long long n, long long n_leaves, float *accum,
                         float sigma_d, float t_d, float *edits, cudaStream_t s) {
  if (n > 0) paint_accum_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(leaf, color, n, n_leaves, accum);
  if (n_leaves > 0)
    paint_finish_kernel<<<(unsigned)((n_leaves + 255) / 256), 256, 0, s>>>(accum, n_leaves, sigma_d, t_d, edits);
  return cudaGetLastError();
}

// Packet render with appearance edits (built for the two record shapes of the
// workloads: K_pad 8 with degree 2, K_pad 16 with degree 3).
template <int KP, int DEG, typename E>
static cudaError_t edit_one(const FwdArgs &a, const LaunchCfg &cfg, cudaStream_t s) {
  if (a.rays.n == 0) return cudaSuccess;
  const long long blocks = (a.rays.n + cfg.block - 1) / cfg.block;
  const size_t sm = smem_bytes(cfg.block, KP, cfg.queue, a.tr);
  cudaError_t e;
  if (sm > 48 * 1024 && (e = cudaFuncSetAttribute(render_packet_kernel<KP, DEG, E, kShadeEdit>,
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess)
    return e;
  long long grid = blocks;
  if (a.work) {
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, render_packet_kernel<KP, DEG, E, kShadeEdit>,
                                                           cfg.block, sm)) != cudaSuccess)
      return e;
    const long long want = (long long)(per_sm > 0 ? per_sm : 1) * cfg.num_sms;
    if (want < grid) grid = want;
    if ((e = cudaMemsetAsync(a.work, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
  }
  render_packet_kernel<KP, DEG, E, kShadeEdit><<<(unsigned)grid, cfg.block, sm, s>>>(a, cfg.queue, cfg.ready);
  return cudaGetLastError();
}

// Density-only packet render (alpha, depth, tau and nseg of the full render,
// no colour): one packet per warp of a full grid, no work counter, so it may
// run beside other calls on the same tree.  Built for the two record shapes
// of the workloads (K_pad 8 with degree 2, K_pad 16 with degree 3).
template <int KP, int DEG, typename E>
static cudaError_t alpha_one(const FwdArgs &a, const LaunchCfg &cfg, cudaStream_t s) {
  if (a.rays.n == 0) return cudaSuccess;
  const long long blocks = (a.rays.n + cfg.block - 1) / cfg.block;
  const size_t sm = smem_bytes(cfg.block, KP, cfg.queue, a.tr);
  cudaError_t e;
  if (sm > 48 * 1024 && (e = cudaFuncSetAttribute(render_packet_kernel<KP, DEG, E, kShadeAlpha>,
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess)
    return e;
  render_packet_kernel<KP, DEG, E, kShadeAlpha><<<(unsigned)blocks, cfg.block, sm, s>>>(a, cfg.queue, cfg.ready);
  return cudaGetLastError();
}

cudaError_t launch_render_alpha(int KP, int DEG, DType dt, const FwdArgs &a, const LaunchCfg &cfg, cudaStream_t s) {
  if (a.work || a.log.n_chunks) return cudaErrorInvalidValue;
  if (KP == 8 && DEG == 2) {
    if (dt == kF32) return alpha_one<8, 2, float>(a, cfg, s);
    if (dt == kBF16) return alpha_one<8, 2, __nv_bfloat16>(a, cfg, s);
    return alpha_one<8, 2, Fp8E4M3>(a, cfg, s);
  }
  if (KP == 16 && DEG == 3) {
    if (dt == kF32) return alpha_one<16, 3, float>(a, cfg, s);
    if (dt == kBF16) return alpha_one<16, 3, __nv_bfloat16>(a, cfg, s);
    return alpha_one<16, 3, Fp8E4M3>(a, cfg, s);
  }
  return cudaErrorNotSupported;
}

cudaError_t launch_render_edit(int KP, int DEG, DType dt, const FwdArgs &a, const LaunchCfg &cfg, cudaStream_t s) {
  if (KP == 8 && DEG == 2) {
    if (dt == kF32) return edit_one<8, 2, float>(a, cfg, s);
    if (dt == kBF16) return edit_one<8, 2, __nv_bfloat16>(a, cfg, s);
  }
  if (KP == 16 && DEG == 3) {
    if (dt == kF32) return edit_one<16, 3, float>(a, cfg, s);
    if (dt == kBF16) return edit_one<16, 3, __nv_bfloat16>(a, cfg, s);
  }
  return cudaErrorNotSupported;
}

// Segment log decoder: ray i's composited segments are the entries of its
// lane in its packet's chunks that hold a leaf, in round order, nseg[i] of
// them.  count[i] = -1 when the ray's packet is not in the log (no log, a log
// of other rays, or a packet that did not fit); chunk links are checked
// against the log's size.
__global__ void __launch_bounds__(256) log_read_kernel(const SampleLog l, long long n, const int *nseg, int max_out,
                                                        int *leaf, float *chord, int *count) {
  const long long pos = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= n) return;
  int c = -1;
  const bool valid = l.n_chunks && __ldg(l.header + 4) == 1u && __ldg(l.header) == l.n_chunks &&
                     __ldg(l.header + 1) == (uint32_t)kLogRounds &&
                     __ldg(l.header + 2) == (uint32_t)(n & 0xFFFFFFFFll) && __ldg(l.header + 3) == (uint32_t)(n >> 32);
  // the ray at this position (its outputs are written at the ray's index)
  const long long i = valid && __ldg(l.header + 5) == 1u ? (long long)min(__ldg(l.perm + pos), (uint32_t)(n - 1)) : pos;
  if (valid) {
    uint32_t chunk = __ldg(l.heads + (pos >> 5));
    const int want = __ldg(nseg + i);
    if (want == 0) {
      c = 0;
    } else if (chunk != kNoLog) {
      c = 0;
      int round = 0;
      for (long long guard = 0; c < want && guard < (long long)l.n_chunks * kLogRounds; ++guard) {
        if (chunk >= l.n_chunks) {
          c = -1;
          break;
        }
        const size_t slot = ((size_t)chunk * kLogRounds + round) * 32 + (pos & 31);
        const uint32_t lf = __ldg(l.leaf + slot);
        if (lf != kEmpty) {
          if (c < max_out) {
            leaf[i * max_out + c] = (int)lf;
            chord[i * max_out + c] = __ldg(l.dt + slot);
          }
          ++c;
        }
        if (++round == kLogRounds) {
          round = 0;
          chunk = __ldg(l.next + chunk);
        }
      }
    }
  }
  for (int k = c < 0 ? 0 : c; k < max_out; ++k) {
    leaf[i * max_out + k] = -1;
    chord[i * max_out + k] = 0.f;
  }
  count[i] = c;
}

cudaError_t launch_log_read(const SampleLog &l, long long n_rays, const int *nseg, int max_out, int *leaf,
                            float *chord, int *count, cudaStream_t s) {
  if (n_rays == 0) return cudaSuccess;
  log_read_kernel<<<(unsigned)((n_rays + 255) / 256), 256, 0, s>>>(l, n_rays, nseg, max_out, leaf, chord, count);
  return cudaGetLastError();
}

cudaError_t launch_trace(const TraceArgs &a, cudaStream_t s) {
  if (a.rays.n == 0) return cudaSuccess;
  const long long blocks = (a.rays.n + 127) / 128;
  trace_kernel<<<(unsigned)blocks, 128, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace neuvv
