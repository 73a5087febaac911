// Internal launch interface between the C ABI (abi.cu) and the kernel files.
#pragma once

#include <cuda_runtime.h>

#include "neuvv_device.cuh"

namespace neuvv {

enum DType { kF32 = 0, kBF16 = 1, kFP8 = 2 };

struct LaunchCfg {
  int block;          // threads per block
  int queue;          // packet kernels: per-lane queue of found leaf segments (power of 2, <= kMaxQueue)
  int ready;          // packet kernels: lanes with a queued segment that trigger a shading round
  int grid;           // compose: persistent blocks (0 = as many as fit, from the occupancy API)
  int dynamic_queue;  // compose and the packet forward: 1 = persistent warps pull 32-ray
                      // packets from a counter, 0 = one packet per warp of the grid
  int num_sms;        // multiprocessors of the device
  int order;          // packet forward with a segment log: 0 = packets in ray order,
                      // 1 = packets in the order of the region they reach first,
                      // 2 = packets re-formed from the rays sorted by direction and region
};

// Segment log of the packet forward (device view of neuvv_out.log).  Chunks
// of kLogRounds shading rounds x 32 lanes hold (leaf, chord) per lane, kEmpty
// for a lane that shaded nothing in that round; a packet's chunks are linked
// from heads[packet] through next[].  heads[packet] = kNoLog: not logged
// (replay by walking).  Header: chunk counter (u64), then n_chunks, rounds,
// n_rays (i64), a valid word and a permuted word, all written by the forward
// that fills it.  Packets are formed from positions: position p holds ray
// perm[p] when the permuted word is 1 (a ray order of the library), else ray p.
constexpr int kLogRounds = 8;
constexpr uint32_t kNoLog = 0xFFFFFFFFu;
struct SampleLog {
  unsigned long long *counter;
  uint32_t *header;   // [0] n_chunks, [1] rounds, [2..3] n_rays, [4] valid, [5] permuted
  uint32_t *perm;     // [n_rays] ray of each position (when permuted)
  uint32_t *heads;    // [n_packets]
  uint32_t *key;      // [n_packets] first leaf the packet shaded (kNoKey: none)
  uint32_t *order;    // [n_packets] packets sorted by key (filled by the adjoint)
  uint32_t *bins;     // [kSortBins] counting-sort scratch
  uint32_t *next;     // [n_chunks]
  uint32_t *leaf;     // [n_chunks][kLogRounds][32]
  float *dt;          // [n_chunks][kLogRounds][32]
  uint32_t n_chunks;  // 0: no log
};
constexpr uint32_t kNoKey = 0xFFFFFFFFu;
// Bins of the counting sort that orders the adjoint's packets by key (leaf
// ids follow the Morton order of the leaves, so a bin is a compact region).
constexpr int kSortBins = 4096;

struct FwdArgs {
  DevTree tr;
  DevRays rays;
  DevOut out;
  float t_stop;
  int act;
  unsigned long long *work;  // packet counter of persistent warps (null: one packet per warp)
  SampleLog log;             // segments to record (n_chunks == 0: none)
  const float *slice;        // render of a time slice: [n_leaves][slice_stride] (null: the tree's records)
  int slice_stride;
  const float *edits;        // appearance edits [n_leaves][8]: c_d (3), sigma_d, t_d, 0, 0, 0
  float edit_beta;           // colour blend weight of an active edit
  const uint32_t *order;     // persistent warps take packets in this order (null: packet index order)
  const uint32_t *perm;      // ray at each position (null: position = ray)
};

// Workspace of the leaf-major adjoint (owned by the tree; fac has one
// 32-byte record per slot of the first cap_chunks chunks of a segment log).
// A count over the log gives each leaf's samples and, scanned, the first
// position of its run in leaf order; the replay takes each sample's position
// from cur (a warp-aggregated atomic per leaf and round) and writes the
// sample's gradient factors there; one thread per leaf then reads its run
// [off[leaf], cur[leaf]) front to back.
struct GatherWs {
  float4 *fac;           // [slots][2]: dpre_s, dpre_g, dz0, dz1 | dz2, u, e0, e1 ((e0, e1): octahedral
                         // code of the unit direction; e0 = kNoFactor: a sample of zero density)
  uint32_t *off;         // [n_leaves + 1] samples per leaf, then the first position of each leaf's run
  uint32_t *cur;         // [n_leaves + 1] next free position of each leaf's run
  uint32_t *part;        // [kScanParts] block sums of the offsets' scan
  uint32_t cap_chunks;   // 0: no workspace (the atomic scatter only)
};
// Marks a factor record without a contribution (octahedral codes lie in [-1, 1]).
constexpr float kNoFactor = 4.f;
// Offsets are scanned in tiles of kScanTile leaves, at most kScanParts tiles.
constexpr int kScanTile = 4096, kScanParts = 4096;

struct BwdArgs {
  GatherWs gws;
  DevTree tr;
  DevRays rays;
  const float *rgb;       // saved C [n][3]
  const float *tau;       // saved optical depth [n]
  const int *nseg;        // saved segment count [n]
  const float *grad_rgb;  // [n][3]
  const float *grad_alpha;  // [n] or null
  float *grad;            // [n_leaves][rec_stride_f32]
  int grad_stride;
  unsigned int *touched;  // bitmap or null
  float t_stop;
  int act;
  SampleLog log;          // the forward's segment log (n_chunks == 0: walk every packet)
  int key_order;          // the replay takes the logged packets in key order (1) or in ray order (0)
};

// Adam step applied by the per-leaf reduction of the adjoint (the fused
// adjoint + optimizer call): the hyper-parameters of neuvv_adam_step, the
// tree's optimizer state and its storage records.
struct AdamArgs {
  float *master, *m, *v;   // FP32 record layout, BwdArgs::grad_stride floats per leaf
  void *storage;           // storage records, null when they are the master
  int dt, storage_stride;  // storage type; entries (FP8: bytes) per leaf
  float lr, b1, b2, eps, c1, c2;
  int on;                  // 0: accumulate into the gradient buffer instead
};

constexpr int kMaxPrims = 16;

struct PrimParam {
  float minv[9];     // (s R)^-1, row-major, rounded to FP32 ...
  float minv_lo[9];  // ... and the remainders: minv + minv_lo is the inverse to ~2^-48
  float trans[3];    // translation of world-from-local
  float scale;     // s
  float toff;      // time offset, frames
  float tint[3];
  int tree;        // index into ComposeArgs::trees
};

struct ComposeArgs {
  DevTree trees[kMaxPrims];
  PrimParam prim[kMaxPrims];
  int n_prims;
  DevRays rays;
  DevOut out;
  float t_stop;
  int act;
  int mode;  // 0 sorted, 1 Algorithm 1 literally
  unsigned long long *work;
};

struct TraceArgs {
  DevTree tr;
  DevRays rays;
  int max_out;
  int *leaf;
  float *t0, *t1;
  int *count;
};

// Normalised 1D Gaussian weights w[0 .. 2 radius] of the shadow-map filter.
constexpr int kMaxBlurRadius = 16;
struct BlurWeights {
  float w[2 * kMaxBlurRadius + 1];
  int radius;
};

struct LightCam {
  float eye[3], right[3], up[3], forward[3];
  float fov_y_deg;
  int width, height;
};

// Pinhole cameras of one ray-setup launch (camera_rays_kernel).  Camera c
// owns rays [off[c], off[c + 1]); tan_half = tan(fov_y / 2) and
// aspect = width / height, both rounded from double on the host.
constexpr int kMaxCams = 32;
struct CamBatch {
  LightCam cam[kMaxCams];
  float tan_half[kMaxCams], aspect[kMaxCams], t[kMaxCams];
  long long off[kMaxCams + 1];
  int n_cams;
  int tile_w, tile_h;  // pixel tile of a 32-ray packet (0 x 0: row-major order)
};

struct SpotArgs {
  DevRays rays;
  const float *rgb, *alpha, *depth;  // the viewer's render [n][3], [n], [n]
  LightCam light;
  const float *light_alpha;          // filtered alpha map [height][width] of the light camera
  float ground_z, r_ref;
  float albedo[3];
  float *out;                        // [n][3]
};

// Each returns cudaGetLastError() of its launch (or cudaErrorInvalidValue for
// an unsupported template combination).
cudaError_t launch_camera_rays(const CamBatch &cb, float *o, float *d, float *t, int *pixel, long long n,
                               cudaStream_t s);
cudaError_t launch_render_fwd(int KP, int DEG, DType dt, bool packet, const FwdArgs &a, const LaunchCfg &cfg,
                              cudaStream_t s);
// Exclusive scan of n uint32 counts in place; v[n] receives the total (v has
// n + 1 entries; part: kScanParts scratch words; n <= kScanTile * kScanParts).
cudaError_t launch_exclusive_scan(uint32_t *v, long long n, uint32_t *part, int num_sms, cudaStream_t s);
// Rays re-formed into packets (cfg.order == 2): perm[position] = ray, sorted
// by (direction bucket, region of the first leaf), stable; scratch of
// ray_order_scratch_bytes(n) bytes.
size_t ray_order_scratch_bytes(long long n);
cudaError_t launch_ray_order(const DevTree &tr, const DevRays &rays, uint32_t *perm, void *scratch, int num_sms,
                             cudaStream_t s);
// Packets in region order for the forward (cfg.order == 1): each packet's key
// is the first leaf that its first hitting ray (of lanes 0, 8, 16, 24)
// reaches (leaf ids follow the Morton order of the leaves), counting-sorted
// into l.order.
cudaError_t launch_packet_order(const DevTree &tr, const DevRays &rays, const SampleLog &l, int num_sms,
                                cudaStream_t s);
// With adam (nullable, adam->on = 1) the per-leaf reduction also applies the
// Adam step and clears the touched bitmap; *fused tells whether it did (the
// caller runs the separate Adam step otherwise).
cudaError_t launch_render_bwd(int KP, int DEG, DType dt, bool packet, const BwdArgs &a, const LaunchCfg &cfg,
                              cudaStream_t s, const AdamArgs *adam = nullptr, bool *fused = nullptr);
cudaError_t launch_compose(int KP, int DEG, DType dt, const ComposeArgs &a, const LaunchCfg &cfg, cudaStream_t s);
cudaError_t launch_trace(const TraceArgs &a, cudaStream_t s);
cudaError_t launch_pick(int KP, int DEG, DType dt, const FwdArgs &a, float threshold, int *leaf_out, cudaStream_t s);
cudaError_t launch_paint(const int *leaf, const float *color, long long n, long long n_leaves, float *accum,
                         float sigma_d, float t_d, float *edits, cudaStream_t s);
cudaError_t launch_render_edit(int KP, int DEG, DType dt, const FwdArgs &a, const LaunchCfg &cfg, cudaStream_t s);
cudaError_t launch_render_alpha(int KP, int DEG, DType dt, const FwdArgs &a, const LaunchCfg &cfg, cudaStream_t s);
cudaError_t launch_gaussian_blur(const float *in, float *out, int width, int height, long long n_images,
                                 const BlurWeights &bw, cudaStream_t s);
cudaError_t launch_spotlight(const SpotArgs &a, cudaStream_t s);
// Time slice of a tree at frame coordinate u into slice [n_leaves][stride].
cudaError_t launch_slice(int KP, int DEG, DType dt, const DevTree &tr, float u, float *slice, int stride,
                         int rec_bytes, int num_sms, cudaStream_t s);
// Packet render of a time slice (a.slice set), with the tree's launch configuration.
cudaError_t launch_render_slice(int DEG, const FwdArgs &a, const LaunchCfg &cfg, cudaStream_t s);
// Device address of the static work counter used by neuvv_compose_noalloc in
// the current CUDA context (looked up on first use per context).
cudaError_t noalloc_queue(unsigned long long **out);
// Decodes a packet forward's segment log into per-ray (leaf, chord) lists.
cudaError_t launch_log_read(const SampleLog &l, long long n_rays, const int *nseg, int max_out, int *leaf,
                            float *chord, int *count, cudaStream_t s);
cudaError_t launch_adam(float *master, float *m, float *v, void *storage, DType dt, int storage_stride, float *grad,
                        const unsigned int *touched, long long n_leaves, int stride_f32, int rec_len, int kp,
                        float lr, float b1, float b2, float eps, float c1, float c2, cudaStream_t s);
cudaError_t launch_store_records(const float *src, float *master, void *storage, DType dt, int storage_stride,
                                 long long n_leaves, int stride_f32, int rec_len, int kp, cudaStream_t s);
cudaError_t launch_mse(const float *rgb, const float *target, long long n, float scale, float *grad, float *loss,
                       cudaStream_t s);
cudaError_t launch_grad_loss(const float *rgb, const float *target, const int *map, int width, int height,
                             long long n_views, long long n_rays, float lam, float *grad, float *loss, cudaStream_t s);

// Dynamic shared memory of the packet kernels: per thread the basis rows
// (2 K_pad floats), the descent path (kPathWords levels; none for a tree with
// a brick map, whose walk never descends the child table) and the segment
// queue (queue x {leaf, t0, t1}).
constexpr int kPathWords = 16;
__host__ __device__ inline int path_words(const DevTree &tr) { return tr.path_words; }
inline size_t smem_bytes(int block, int KP, int queue, const DevTree &tr) {
  return (size_t)block * (2 * KP + path_words(tr) + 3 * queue) * sizeof(float);
}
constexpr int kMaxQueue = 32;
// Packet kernels are latency bound: two 256-thread blocks per SM (128
// registers a thread) keep enough warps resident; FP32 records need the
// registers of one block per SM instead.
template <typename E>
constexpr int packet_min_blocks() { return sizeof(E) == 4 ? 1 : 2; }
constexpr int kMaxDepth = 14;

}  // namespace neuvv
