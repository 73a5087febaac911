/*
 * neuvv.h -- C ABI of the GB300 VOctree renderer (NeuVV, arxiv 2202.06088).
 *
 * A VOctree (Sec. 4.3) is a sparse octree over a primitive's bounding box whose
 * occupied leaves each store three coefficient vectors: w_sigma (K weights of a
 * shared temporal density basis A, Eq. project-sigma), w_gamma (K weights of a
 * shared hyper-angle basis B, Eq. project-gamma) and w_HH (3 x N_h coefficients
 * of real 4D hyperspherical harmonics, Eq. HH-color-2).  Rendering a ray
 * (Sec. 4.3 "Rendering") walks the voxels it crosses, turns each leaf's
 * coefficients into density and colour at time t and composites them front to
 * back (Eq. volume-rendering).
 *
 * Conventions for every call:
 *  - Every entry point returns a neuvv_status; on failure neuvv_last_error()
 *    returns a message for the calling thread.  Argument errors are detected on
 *    the host before anything is launched.
 *  - "device" pointers are CUDA global-memory pointers on the tree's device and
 *    are owned by the caller unless stated otherwise.  "host" pointers are read
 *    during the call only.
 *  - Calls that take a stream are asynchronous on it: no host synchronisation,
 *    no allocation.  neuvv_tree_create/destroy/status/autotune synchronise.
 *  - The packet kernels of neuvv_render, neuvv_render_slice, neuvv_render_edit
 *    and neuvv_compose pull work from a counter owned by the tree (by the
 *    first tree for compose; neuvv_compose_noalloc's is a library global):
 *    two such calls on one tree must be ordered (one stream, or events
 *    between streams).  So must two neuvv_render_backward calls on a tree with
 *    an adjoint reservation (they share its workspace).  The plain kernel
 *    (NEUVV_KERNEL_PLAIN) and the other calls use no such counter and may run
 *    concurrently on different streams, as long as their outputs do not
 *    overlap.
 *  - Errors found on the device (a ray that exceeds its walk-step cap, an
 *    index outside the tree, a bounded wait that gives up) are recorded in a
 *    per-tree status word read by neuvv_tree_status(); the affected ray or
 *    tile ends early, nothing traps and no wait is unbounded.
 *  - Ray directions need not be normalised.  Per-ray times are clamped to [0,1].
 *
 * Numerical readings of the paper that the library implements (the FP64
 * oracle in the test suite implements the same ones independently):
 *  - harmonic H_nlm = Abar_{n,l} sin^l(gamma) C^{l+1}_{n-l}(cos gamma) Y_lm(d),
 *    Abar_{n,l} = 2^l l! sqrt(2(n+1)(n-l)! / (pi (n+l+1)!)) (orthonormal on S^3);
 *    Y_lm real, on the unit view direction, polar axis +z, no Condon-Shortley
 *    phase, cos(m phi) for m > 0, sin(|m| phi) for m < 0;
 *    index idx(n,l,m) = n(n+1)(2n+1)/6 + l^2 + l + m;
 *  - frame coordinate u = t (T-1); basis rows linearly interpolated in u;
 *  - colour = sigmoid(sum_idx w[ch][idx] H_idx) (or identity);
 *  - a leaf segment's chord delta is the exact length of the ray inside the
 *    voxel; alpha_i = 1 - exp(-sigma_i delta_i); compositing stops after the
 *    segment that brings transmittance below t_stop;
 *  - outputs: premultiplied colour C = sum w_i c_i, alpha = sum w_i,
 *    depth = sum w_i t_mid,i / alpha if alpha >= 1e-4 else +inf, tau = sum sigma_i delta_i.
 */
#ifndef NEUVV_H
#define NEUVV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct neuvv_tree neuvv_tree; /* opaque; owned by the library */

typedef enum {
  NEUVV_OK = 0,
  NEUVV_ERR_INVALID_ARG = 1, /* bad pointer, size, shape or value */
  NEUVV_ERR_CUDA = 2,        /* a CUDA runtime call failed */
  NEUVV_ERR_OOM = 3,         /* device allocation failed */
  NEUVV_ERR_TIMEOUT = 4,     /* reserved (device-detected limits are reported as status bits) */
  NEUVV_ERR_UNSUPPORTED = 5, /* a valid request this build does not implement */
  NEUVV_ERR_DEVICE = 6       /* other device-detected error (status word) */
} neuvv_status;

/* Storage of the leaf coefficients on the device.  Arithmetic is FP32 for all.
 * NEUVV_FP8_E4M3 is a storage ablation (no counterpart in the paper, which
 * stores FP32): E4M3 codes with one power-of-two scale per leaf and group,
 * built for K <= 8 with hh_degree 2 and 9 <= K <= 16 with hh_degree 3. */
typedef enum { NEUVV_F32 = 0, NEUVV_BF16 = 1, NEUVV_FP8_E4M3 = 2 } neuvv_dtype;

/* Device status bits (neuvv_tree_status). */
#define NEUVV_STATUS_SEGMENT_CAP 0x1u /* a ray reached its walk-step cap (neuvv_tree_set_limits;
                                         by default 3*2^depth+8, more than any ray needs) and ended */
#define NEUVV_STATUS_BAD_INDEX 0x2u   /* a child, brick, leaf or log entry pointed outside its table */
#define NEUVV_STATUS_TIMEOUT 0x4u     /* a bounded device wait (the time slice's copy into shared
                                         memory) gave up; the block ended after its copy landed */

/* Tree description, all host memory, read during neuvv_tree_create only.
 * child: [n_nodes][8] uint32, slot c = 4*xbit + 2*ybit + zbit; entry 0xFFFFFFFF
 *   = empty, 0x80000000|leaf = occupied leaf, else index of an internal node.
 *   Node 0 is the root covering [aabb_min, aabb_max]; children of a node at
 *   level L are cells at level L+1; the finest level is `depth` (1..14).
 *   Internal node indices must be breadth first (a child's index is larger
 *   than its parent's).
 * w_sigma: [K][n_leaves], w_gamma: [K][n_leaves], w_hh: [3][N_h][n_leaves] float32
 *   planes (N_h = sum_{n<=hh_degree} (n+1)^2), the paper's per-voxel vectors.
 * basis_A, basis_B: [T][K] float32 (T >= 2 frames).
 * K in 1..32, hh_degree in 1..3. */
typedef struct {
  int32_t depth, K, T, hh_degree;
  neuvv_dtype dtype;        /* storage of the leaf coefficients on the device */
  int32_t with_optimizer;   /* 1: also allocate FP32 master (if dtype != F32) and Adam m, v */
  int64_t n_nodes, n_leaves;
  const uint32_t *child;
  const float *w_sigma, *w_gamma, *w_hh;
  const float *basis_A, *basis_B;
  float aabb_min[3], aabb_max[3];
  uint32_t flags;           /* NEUVV_TREE_* bits */
} neuvv_tree_desc;

/* neuvv_tree_desc.flags: skip the bricks (dense per-node tables of the last
 * three levels that shorten descents; built by default when depth >= 3). */
#define NEUVV_TREE_NO_BRICKS 0x1u

/* Layout of a tree's per-leaf records, for views over its device buffers and
 * for gradient buffers.  A record holds, in order, w_sigma (K_pad entries, the
 * last K_pad-K zero), w_gamma (K_pad), w_hh (3*N_h, channel-major), then zero
 * padding to rec_stride entries.  The FP32 gradient/master layout uses
 * rec_stride_f32 floats per leaf (a multiple of 4, 16-byte rows).
 * FP8_E4M3 records (rec_stride counts bytes): a 16-byte header of three FP32
 * scales (w_sigma, w_gamma, w_hh groups) and a zero word, then one E4M3 code
 * per entry in the order above, zero padded to a 16-byte multiple.  An entry
 * is its code's value times its group's scale; each scale is the smallest
 * power of two 2^p with max |w| <= 448 * 2^p over the group (1 if all zero),
 * and codes are the nearest E4M3 values (ties to even) of w / 2^p.  Adam
 * re-derives scales and codes from the FP32 master for each touched leaf. */
typedef struct {
  int32_t depth, K, K_pad, T, hh_degree, N_h;
  int32_t rec_len;          /* 2*K_pad + 3*N_h meaningful entries */
  int32_t rec_stride;       /* storage entries per leaf (16-byte multiple); FP8: bytes */
  int32_t rec_stride_f32;   /* FP32 floats per leaf in grad / master / m / v */
  neuvv_dtype dtype;
  int64_t n_nodes, n_leaves;
  int32_t device;
  int32_t packet_block;     /* packet kernels: threads per block */
  int32_t packet_queue;     /* packet kernels: leaf segments a ray may queue ahead of shading */
  int32_t packet_ready;     /* packet kernels: lanes holding a queued segment that start a
                               shading round (all three set by neuvv_autotune) */
  int32_t packet_order;     /* packet forward with a segment log: NEUVV_ORDER_* (neuvv_autotune) */
  int32_t packet_tiles;     /* pixel tile of a 32-ray packet of camera rays, NEUVV_TILES_*
                               (neuvv_autotune_tiles; default 8x4) */
} neuvv_tree_info;

/* The order in which the packet forward runs its 32-ray packets when the
 * call has a segment log (the rays themselves, their outputs and the packets'
 * contents do not change).  AS_GIVEN: in ray order.  BY_REGION: a pre-pass
 * finds the first leaf each packet reaches and the packets run sorted by
 * that leaf's region (leaf ids follow the Morton order of the leaves), so
 * packets of different views that see the same part of the tree run
 * together and share its records in L2.  BY_RAY: the packets themselves are
 * re-formed: the rays are sorted (stable) by a bucket of their direction and
 * the region of the first leaf they reach, so a batch of rays from many
 * views and times in any order gets packets of rays that cross the same
 * cells; outputs stay in the caller's order, and the order is kept in the
 * log for the adjoint (it needs about 17 bytes per ray of the log as scratch,
 * else the rays stay as given). */
#define NEUVV_ORDER_AS_GIVEN 0
#define NEUVV_ORDER_BY_REGION 1
#define NEUVV_ORDER_BY_RAY 2

/* Rays, device SoA float32 arrays of length n.  t may be NULL: then the
 * scalar time argument of the call is used for every ray. */
typedef struct {
  const float *ox, *oy, *oz, *dx, *dy, *dz;
  const float *t;
  int64_t n;
} neuvv_rays;

/* Per-ray outputs, device, caller-owned.  rgb: [n][3]; alpha, depth, tau: [n];
 * nseg: [n] segments composited (needed by the backward pass).  Any member may
 * be NULL except where a call says otherwise.
 * log, log_bytes: optional device buffer (16-byte aligned) in which the packet
 * forward records, per 32-ray packet, the leaf and chord of every segment it
 * composites, in shading order; neuvv_render_backward given the same saved
 * outputs replays a packet from the log instead of walking the tree again.
 * The layout is private to the library.  A packet whose segments do not fit
 * is marked and replayed by walking, so any size (including 0) is correct;
 * about 64 bytes per ray holds the segments of a typical batch.  Other calls
 * (plain forward, compose) mark the log empty. */
typedef struct {
  float *rgb, *alpha, *depth, *tau;
  int32_t *nseg;
  void *log;
  int64_t log_bytes;
} neuvv_out;

typedef enum { NEUVV_ACT_SIGMOID = 0, NEUVV_ACT_IDENTITY = 1 } neuvv_color_act;
typedef enum { NEUVV_KERNEL_AUTO = 0, NEUVV_KERNEL_PLAIN = 1, NEUVV_KERNEL_PACKET = 2 } neuvv_kernel;
typedef enum { NEUVV_COMPOSE_SORTED = 0, NEUVV_COMPOSE_ALG1 = 1 } neuvv_compose_mode;

typedef struct {
  float t_stop;        /* early termination: stop after T < t_stop (1e-4) */
  int32_t color_act;   /* neuvv_color_act */
  int32_t kernel;      /* neuvv_kernel: plain = one thread per ray, descents from
                          the root, walk and shading in lockstep; packet = warps
                          of 32 consecutive rays, descents restarted at the
                          lowest common ancestor, walk and shading decoupled by
                          a per-ray queue, tuned launch */
  int32_t compose_mode;/* neuvv_compose_mode */
} neuvv_render_opts;

typedef void *neuvv_stream; /* a cudaStream_t; NULL = legacy default stream */

/* Last error message of the calling thread ("" if none). */
const char *neuvv_last_error(void);

/* Copies the tree to the current CUDA device (Sec. 4.3: the VOctree holds
 * w_sigma, w_gamma, w_HH per voxel).  Validates the child table on the host;
 * errors: INVALID_ARG (malformed table, sizes), OOM, CUDA.  Synchronous. */
neuvv_status neuvv_tree_create(const neuvv_tree_desc *desc, neuvv_tree **out);
neuvv_status neuvv_tree_destroy(neuvv_tree *tree);
neuvv_status neuvv_tree_get_info(const neuvv_tree *tree, neuvv_tree_info *info);

/* Device pointers owned by the tree (valid until destroy): storage records
 * ([n_leaves][rec_stride] in dtype), FP32 master records (== storage when
 * dtype is F32; NULL without optimizer state), Adam moments m and v (NULL
 * without optimizer state).  For views from PyTorch and for tests. */
neuvv_status neuvv_tree_coeff_ptrs(neuvv_tree *tree, void **storage, float **master, float **adam_m, float **adam_v);

/* Replaces the tree's coefficients (Sec. 4.3: the VOctree's per-voxel
 * vectors w_sigma, w_gamma, w_HH, optimised by gradient descent) with
 * records: device FP32 [n_leaves][rec_stride_f32] in the record layout of
 * neuvv_tree_info (the layout of gradients and of the master copy; entries
 * past rec_len are ignored), 16-byte aligned, caller-owned, read on the
 * stream.  Writes the FP32 master copy (when the tree has optimizer state
 * and its storage is not FP32) and the storage records, rounded to nearest
 * even for BF16 and re-encoded with fresh per-leaf group scales for
 * FP8_E4M3, exactly as at tree creation.  Adam's moments are kept.  The
 * records may be the tree's own master copy (then only the storage is
 * refreshed from it).  Asynchronous. */
neuvv_status neuvv_tree_set_records(neuvv_tree *tree, const float *records, neuvv_stream stream);

/* Reads and clears the device status word (NEUVV_STATUS_* bits).  Synchronous. */
neuvv_status neuvv_tree_status(neuvv_tree *tree, uint32_t *flags);

/* Forward render (Sec. 4.3 "Rendering"; Eq. project-sigma, project-gamma,
 * HH-color-2, volume-rendering).  out->rgb, alpha must be non-NULL; depth, tau,
 * nseg optional (tau and nseg are the saved state of the backward pass).
 * t: scalar time in [0,1] used when rays->t is NULL (else ignored). */
neuvv_status neuvv_render(const neuvv_tree *tree, const neuvv_rays *rays, float t, const neuvv_render_opts *opts,
                          neuvv_out *out, neuvv_stream stream);

/* Time slice (Sec. 7, which proposes slicing a VOctree at one time into a
 * PlenOctree-like representation, and the caption of the HH-colour figure: at
 * a fixed time the hyper angle gamma(t) is a constant and the 4D harmonics
 * reduce to 3D spherical harmonics).  Writes, for every leaf, its density
 * sigma(t) = ReLU(a(u) . w_sigma) and its spherical-harmonic colour
 * coefficients s[ch][l^2+l+m] = sum_{n>=l} w_HH[ch][n,l,m] R_nl(gamma(t)),
 * gamma(t) = pi sigmoid(b(u) . w_gamma), u = t (T-1) (Eq. project-sigma,
 * Eq. project-gamma, Eq. HH-color-2 with gamma fixed).
 * slice: device FP32 [n_leaves][slice_stride], caller-owned, 16-byte aligned;
 * per leaf [sigma, 0, 0, 0, s[0][0..NY), s[1][..], s[2][..]], NY =
 * (hh_degree+1)^2, the rest of the row untouched.  slice_stride: floats per
 * leaf, a multiple of 4 and at least 4 + 3 NY rounded up to 4 (16, 32, 52 for
 * degree 1, 2, 3).  t must be in [0, 1]. */
neuvv_status neuvv_slice(const neuvv_tree *tree, float t, float *slice, int32_t slice_stride, neuvv_stream stream);

/* Volume rendering of a time slice made by neuvv_slice (Eq. volume-rendering
 * over the tree's voxels and chords, density slice[leaf][0], colour
 * act(sum_lm s_lm Y_lm(d))): the same outputs as neuvv_render at the slice's
 * time, without evaluating the temporal bases and the hyper-angle radial
 * factors per sample.  Always the packet kernel with the tree's launch
 * configuration; ray times are ignored; a log in out is marked empty. */
neuvv_status neuvv_render_slice(const neuvv_tree *tree, const float *slice, int32_t slice_stride,
                                const neuvv_rays *rays, const neuvv_render_opts *opts, neuvv_out *out,
                                neuvv_stream stream);

/* Reserves device memory for the leaf-major adjoint (synchronous; frees an
 * earlier reservation; n_slots = 0 only frees).  A slot is one lane of one
 * shading round of a segment log (a log of B bytes holds fewer than B / 8);
 * the reservation takes 32 B per slot plus 8 B per leaf.  With it,
 * neuvv_render_backward (packet kernel, with a log from the forward over the
 * same rays) counts each leaf's logged samples, writes each replayed
 * sample's gradient factors at the next position of its leaf's run (leaf
 * order), and sums each run one leaf per thread into the leaf's gradient
 * record: no gradient atomics for those samples.
 * Samples in chunks beyond the reservation, and packets the log could not
 * hold, use the atomic scatter.  The result equals the atomic path's up to
 * FP32 summation order.  It pays when a call has many samples per leaf (8
 * views at 1080p over 2 M leaves, 17 samples per leaf: adjoint with Adam 6.5
 * against 7.4 ms); with fewer samples than leaves its per-leaf pass costs
 * more than the atomics it saves (1 M rays over 8 M leaves: training step
 * 5.8 against 4.8 ms).  Trees of more than 2^24 leaves: NEUVV_ERR_UNSUPPORTED;
 * n_slots outside [0, 2^32 - 256]: NEUVV_ERR_INVALID_ARG; allocation failure:
 * NEUVV_ERR_OOM (the tree keeps no reservation). */
neuvv_status neuvv_tree_reserve_adjoint(neuvv_tree *tree, int64_t n_slots);

/* Fused adjoint (Sec. 4.3 "Optimization": the renderer is differentiated by
 * hand for gradient descent on the leaf coefficients).  Replays every ray with
 * the forward traversal, recomputes each sample, and accumulates dL/dw for
 * L(C, alpha) given grad_rgb = dL/dC [n][3] and grad_alpha = dL/dalpha [n]
 * (nullable).  saved: the forward's rgb, tau and nseg (all required).
 * grad: device FP32 [n_leaves][rec_stride_f32], accumulated into (+=).
 * touched: device bitmap of ceil(n_leaves/32) uint32 words, bits OR-ed for
 * every leaf that received a gradient (nullable). */
neuvv_status neuvv_render_backward(const neuvv_tree *tree, const neuvv_rays *rays, float t,
                                   const neuvv_render_opts *opts, const neuvv_out *saved, const float *grad_rgb,
                                   const float *grad_alpha, float *grad, uint32_t *touched, neuvv_stream stream);

/* One optimisation step on the leaf coefficients (Sec. 4.3 "Optimization":
 * the renderer's gradient followed by Adam): the same result as
 * neuvv_render_backward(tree, ..., grad, touched) followed by
 * neuvv_adam_step(tree, grad, touched, lr, beta1, beta2, eps, step), in one
 * call.  When the adjoint takes the leaf-major path (packet kernel, a log
 * from the forward over these rays, a reservation from
 * neuvv_tree_reserve_adjoint, K_pad <= 16), the Adam update runs inside the
 * per-leaf reduction: each leaf's gradient is summed in registers and
 * applied to its FP32 master, m, v and storage record at once, without
 * passing through grad; otherwise the two steps run one after the other.
 * grad (device FP32 [n_leaves][rec_stride_f32], 16-byte aligned) holds what
 * the atomic scatter adds for samples beyond the reservation; as after
 * neuvv_adam_step, its rows of touched leaves are zero afterwards, and rows
 * of leaves whose touched bit is clear must be zero on entry.  touched
 * (required) is clear afterwards.  Needs optimizer state; errors as the two
 * calls. */
neuvv_status neuvv_render_backward_adam(neuvv_tree *tree, const neuvv_rays *rays, float t,
                                        const neuvv_render_opts *opts, const neuvv_out *saved, const float *grad_rgb,
                                        const float *grad_alpha, float *grad, uint32_t *touched, float lr,
                                        float beta1, float beta2, float eps, int32_t step, neuvv_stream stream);

/* Spatial-temporal composition (Eq. st_composite_affine) with depth-aware
 * blending (Algorithm 1).  n_prims in 1..16 primitives; trees[j] may repeat
 * (duplicates share one tree, Sec. 5.1 "Varied Manifestations"); all trees
 * must share K_pad, hh_degree and dtype.  transforms: host [n_prims][12],
 * row-major 3x4 world-from-local [s R | translation] with uniform scale s > 0.
 * time_offsets: host [n_prims] frames; frame u' = (t (T-1) + offset) mod (T-1).
 * tints: host [n_prims][3] multiplying the colour.  Rays are in world space;
 * out->rgb, alpha required, depth optional (world units). */
neuvv_status neuvv_compose(const neuvv_tree *const *trees, const float *transforms, const float *time_offsets,
                           const float *tints, int32_t n_prims, const neuvv_rays *rays, float t,
                           const neuvv_render_opts *opts, neuvv_out *out, neuvv_stream stream);

/* neuvv_compose without any allocation: the same composition as
 * neuvv_compose (same arguments, same results), but its packet work counter
 * is one 64-bit word of file-scope device memory inside the library instead
 * of memory owned by the trees.  The paper has no counterpart; it is for
 * callers that cannot allocate device memory, or touch memory they did not
 * set up, at the moment they render: e.g. a frame callback of an interactive
 * viewer that must not call into the allocator, or a process whose device
 * memory is all reserved up front by another framework.  (The trees must
 * still have been created earlier.)
 *  - Allocates nothing: no cudaMalloc/cudaFree or allocating library routine.
 *  - The first call on a device looks the counter's device address up with
 *    cudaGetSymbolAddress (with that device current) and caches it; make that
 *    first call before any stream capture.
 *  - Every call on a device shares the one counter, which is reset on the
 *    call's stream before the launch: calls that overlap on the GPU (other
 *    streams, or several threads) race and must be serialised by the caller.
 *  - At most NEUVV_NOALLOC_MAX_RAYS rays per call; more is INVALID_ARG. */
#define NEUVV_NOALLOC_MAX_RAYS ((int64_t)1 << 37)
neuvv_status neuvv_compose_noalloc(const neuvv_tree *const *trees, const float *transforms, const float *time_offsets,
                                   const float *tints, int32_t n_prims, const neuvv_rays *rays, float t,
                                   const neuvv_render_opts *opts, neuvv_out *out, neuvv_stream stream);

/* Sparse Adam on the leaves whose touched bit is set (Sec. 4.3 "Optimization":
 * SGD or Adam).  Updates the FP32 master, m and v, writes the storage copy
 * (rounded to nearest even for BF16), zeroes those leaves' rows of grad and
 * clears touched.  Untouched leaves keep weights and moments.  step >= 1 is
 * the bias-correction step.  Needs a tree created with with_optimizer = 1. */
neuvv_status neuvv_adam_step(neuvv_tree *tree, float *grad, uint32_t *touched, float lr, float beta1, float beta2,
                             float eps, int32_t step, neuvv_stream stream);

/* Loss of Eq. rgb-loss scaled by `scale` and its gradient:
 * loss_accum[0] += scale * sum ||C - target||^2 (device float, nullable);
 * grad_rgb = 2 * scale * (C - target).  All device [n][3]. */
neuvv_status neuvv_mse_grad(const float *rgb, const float *target, int64_t n, float scale, float *grad_rgb,
                            float *loss_accum, neuvv_stream stream);

/* Image-gradient regulariser of Sec. 4.3 "Optimization" (the equation after
 * Eq. rgb-loss; the paper weights it by lambda_grad = 0.1 in the total loss):
 * loss_accum[0] += lambda * sum over views and pixels of ||grad |I - I_hat|||^2,
 * with E = |target - rgb| per channel and the image gradient taken as forward
 * differences E(x+1, y) - E(x, y) and E(x, y+1) - E(x, y) between pixels that
 * both have a ray, summed over the three channels.  grad_rgb += its gradient
 * (d|I - I_hat|/d I_hat = sign(I_hat - I), 0 where equal), so it can follow
 * neuvv_mse_grad on the same buffer.
 * rgb, target, grad_rgb: device [n][3]; ray_of_pixel: device int32
 * [n_views][height][width], the ray index of each pixel or -1 (pixels of a
 * view are its rays' image in any ray order); n < 2^31.  loss_accum nullable. */
neuvv_status neuvv_grad_loss(const float *rgb, const float *target, int64_t n, const int32_t *ray_of_pixel,
                             int32_t width, int32_t height, int32_t n_views, float lambda, float *grad_rgb,
                             float *loss_accum, neuvv_stream stream);

/* Terminating voxel of each ray (Sec. 5 "Appearance editing": the voxel
 * where the accumulated alpha of the NeuVV render first reaches a threshold,
 * 0.99 in the paper): leaf[i] = the leaf of the segment at which
 * 1 - exp(-sum sigma delta) first reaches `threshold` (in (0, 1)), or -1.
 * leaf: device int32 [n], caller-owned.  t: scalar time when rays->t is NULL. */
neuvv_status neuvv_pick(const neuvv_tree *tree, const neuvv_rays *rays, float t, float threshold, int32_t *leaf,
                        neuvv_stream stream);

/* Assigns target colours to picked voxels (Sec. 5 "Appearance editing": a
 * pattern painted over the performer from a view).  Each leaf that at least
 * one of the n rays picked (leaf[i] >= 0, from neuvv_pick) gets the mean of
 * those rays' colours (color [n][3]), target density sigma_d (< 0: keep the
 * density) and time t_d (the edit is active at times >= t_d) in its edit
 * record; other leaves keep theirs.  edits: device FP32 [n_leaves][8] =
 * c_d (3), sigma_d, t_d, 3 unused; a record with t_d > 1 is inactive.
 * accum: device FP32 [n_leaves][4] scratch, zeroed by the caller before the
 * call.  Both 16-byte aligned, caller-owned. */
neuvv_status neuvv_paint(const neuvv_tree *tree, const int32_t *leaf, const float *color, int64_t n, float sigma_d,
                         float t_d, float *accum, float *edits, neuvv_stream stream);

/* neuvv_render with appearance edits: a voxel whose edit is active at the
 * ray's time (t >= t_d) has density sigma_d when sigma_d >= 0 and colour
 * (1 - beta) c + beta c_d (beta in [0, 1]: 1 replaces, smaller values blend the
 * target with the NeuVV colour).  Packet kernel; built for K <= 8 with
 * degree 2 and 9 <= K <= 16 with degree 3, FP32 or BF16 storage
 * (NEUVV_ERR_UNSUPPORTED otherwise).  A log in out is marked empty. */
neuvv_status neuvv_render_edit(const neuvv_tree *tree, const neuvv_rays *rays, float t, const neuvv_render_opts *opts,
                               const float *edits, float beta, neuvv_out *out, neuvv_stream stream);

/* Gaussian low-pass filter of single-channel images (Sec. 5 "Spotlight
 * Lighting": the shadow map is rendered at low resolution and filtered
 * against Moire patterns).  in, out: distinct device FP32 buffers
 * [n_images][height][width].  Weights exp(-k^2 / (2 sigma^2)) for
 * |k| <= floor(3 sigma + 0.5) (sigma in (0, 5]), normalised, along x and along
 * y; pixels beyond the border repeat the edge pixel. */
neuvv_status neuvv_gaussian_blur(const float *in, float *out, int32_t width, int32_t height, int32_t n_images,
                                 float sigma, neuvv_stream stream);

/* Density-only render (Sec. 5 "Spotlight Lighting": the shadow map is the
 * alpha of the VOctree seen from the light).  Walks and composites exactly as
 * neuvv_render's packet kernel but reads only the w_sigma part of each leaf
 * record and evaluates no colour: out->alpha (required), depth, tau and nseg
 * (each optional) equal neuvv_render's for the same rays; out->rgb and
 * out->log are not used.  Launches one packet per warp without the tree's
 * work counter, so it may run on another stream beside any call on the same
 * tree.  Built for K_pad 8 with degree 2 and K_pad 16 with degree 3 (else
 * NEUVV_ERR_UNSUPPORTED); other errors as neuvv_render. */
neuvv_status neuvv_render_alpha(const neuvv_tree *tree, const neuvv_rays *rays, float t, const neuvv_render_opts *opts,
                                neuvv_out *out, neuvv_stream stream);

/* Pixel order of neuvv_camera_rays: row-major, or tiles of 32 pixels. */
#define NEUVV_TILES_NONE 0
#define NEUVV_TILES_8X4 1
#define NEUVV_TILES_4X8 2
#define NEUVV_TILES_16X2 3

/* A pinhole camera (the viewers' and the light's): ray through pixel (px, py)
 * (pixel centres at +0.5) from eye along forward + sx right + sy up,
 * sx = (2 (px+0.5)/width - 1) tan(fov_y/2) width/height,
 * sy = (1 - 2 (py+0.5)/height) tan(fov_y/2); right, up, forward orthonormal. */
typedef struct {
  float eye[3], right[3], up[3], forward[3];
  float fov_y_deg;
  int32_t width, height;
} neuvv_camera;
typedef neuvv_camera neuvv_light;

/* Ray setup (Sec. 4.3 "Rendering": a ray through the centre of each pixel of
 * each view).  cams: host [n_cams] (1..32 per call; chunk longer lists);
 * times: host [n_cams], each in [0, 1].  Camera c owns rays
 * [off_c, off_c + width_c * height_c), off_c the sum of the earlier cameras'
 * pixel counts; n must equal the total.  Ray j of a camera goes through pixel
 * j in row-major order when tiled == NEUVV_TILES_NONE; otherwise the pixels
 * are listed by tiles of 32 pixels, 8x4, 4x8 or 16x2 (NEUVV_TILES_*: tiles in
 * row-major order, pixels of a tile row-major, the tiles at the right and
 * bottom edges narrower or shorter), so a 32-ray packet covers one tile; any
 * other value is INVALID_ARG.  Writes, all device and caller-owned: origins [3][n] (the
 * eye), dirs [3][n] (unit: the direction above divided by its FP32 norm),
 * times_out [n] (times[c]) and, when pixel_of_ray is not NULL, pixel_of_ray
 * [n] (py * width + px of the ray's own camera).  Errors: NULL pointers, a
 * camera with a non-positive size or a field of view outside (0, 180), a time
 * outside [0, 1] or a mismatched n give NEUVV_ERR_INVALID_ARG before any
 * launch. */
neuvv_status neuvv_camera_rays(const neuvv_camera *cams, const float *times, int32_t n_cams, int32_t tiled,
                               float *origins, float *dirs, float *times_out, int32_t *pixel_of_ray, int64_t n,
                               neuvv_stream stream);

/* Spotlight shadow and distance falloff (Sec. 5 "Spotlight Lighting").  For
 * each viewer ray with its render (rgb premultiplied [n][3], alpha [n], depth
 * [n] along the unit direction, +inf where nothing was hit), with
 * f(r) = (r_ref / r)^2 the falloff with the distance r to the light:
 *   C_lit = rgb * f(|X - L|), X = o + depth * d (rgb where depth is +inf);
 *   where the ray meets the ground plane z = ground_z ahead of its origin at
 *   P, P is projected into the light camera and its alpha map light_alpha
 *   [height][width] (rendered from the light and filtered; 0 outside the map)
 *   is sampled bilinearly (texel centres at +0.5): a_L;
 *   rgb_out = C_lit + (1 - alpha) * albedo * (1 - a_L) * f(|P - L|).
 * All arrays device FP32, caller-owned; rgb_out may not alias rgb. */
neuvv_status neuvv_spotlight(const neuvv_rays *rays, const float *rgb, const float *alpha, const float *depth,
                             const neuvv_light *light, const float *light_alpha, float ground_z, const float albedo[3],
                             float r_ref, float *rgb_out, neuvv_stream stream);

/* Occupied leaves each ray crosses, in order (Sec. 4.3 "Rendering": the voxels
 * on the ray and their segment lengths), without early termination.  Writes up
 * to max_out entries per ray: leaf [n][max_out] int32 (-1 past the end),
 * t0/t1 [n][max_out] entry and exit distances along the normalised direction,
 * count [n] (total, may exceed max_out).  Uses the renderer's traversal. */
neuvv_status neuvv_trace(const neuvv_tree *tree, const neuvv_rays *rays, int32_t max_out, int32_t *leaf, float *t0,
                         float *t1, int32_t *count, neuvv_stream stream);

/* Device limits of a tree's calls (host only; no counterpart in the paper:
 * failure detection).  step_cap: walk steps a ray may take before it ends and
 * raises NEUVV_STATUS_SEGMENT_CAP (0 = the default 3*2^depth+8, which no ray
 * reaches); wait_polls: polls of a bounded wait on the device before it gives
 * up and raises NEUVV_STATUS_TIMEOUT (default 2^22; 0 gives up at once).
 * Both >= 0, else NEUVV_ERR_INVALID_ARG.  Small values exist to exercise the
 * error paths: the affected rays or tiles end early, no kernel waits forever
 * and nothing traps. */
neuvv_status neuvv_tree_set_limits(neuvv_tree *tree, int32_t step_cap, int32_t wait_polls);

/* Reads back the segment log written by a packet neuvv_render into saved->log
 * (Sec. 4.3 "Rendering": the voxels each ray composited and their chord
 * lengths, as the timed kernel found them).  n: the rays of that render;
 * saved->nseg: its segment counts (required).  Writes leaf [n][max_out]
 * (-1 past the end) and chord [n][max_out] (length along the unit direction)
 * of each ray's first max_out composited segments in order, and count [n]:
 * the ray's number of segments, or -1 when its packet is not in the log (no
 * log, a log written for other rays, or a packet that did not fit).  All
 * device, caller-owned; asynchronous. */
neuvv_status neuvv_log_read(const neuvv_out *saved, int64_t n, int32_t max_out, int32_t *leaf, float *chord,
                            int32_t *count, neuvv_stream stream);

/* Sets the packet forward's order (NEUVV_ORDER_*; else INVALID_ARG) instead
 * of neuvv_autotune.  Host only. */
neuvv_status neuvv_tree_set_packet_order(neuvv_tree *tree, int32_t order);

/* Sets the packet kernels' launch explicitly instead of neuvv_autotune:
 * block (a multiple of 32 in [32, 256]), queue (a power of two in [1, 32]:
 * leaf segments a ray's walk may run ahead of its shading) and ready (1..32:
 * lanes with a queued segment that start a shading round).  Host only. */
neuvv_status neuvv_tree_set_launch(neuvv_tree *tree, int32_t block, int32_t queue, int32_t ready);

/* Picks the packet kernels' launch -- block size, queue, ready count and the
 * forward's packet order (NEUVV_ORDER_*) -- by timing candidates with the
 * packet forward (with a segment log of 64 bytes per ray) on a sample of
 * rays (the first min(n, 2^20)); the fastest is stored in the tree.  The
 * choice is kept for the life of the process under the tree's shape (depth,
 * node and leaf counts, K_pad, degree, storage type, bricks), the device and
 * its multiprocessor count and the sample size (power of two): a later call
 * for a tree of the same key reuses it without timing anything.
 * Synchronous (allocates and frees its sample outputs when it times).
 * best_ms (nullable) receives the best forward time. */
neuvv_status neuvv_autotune(neuvv_tree *tree, const neuvv_rays *sample, float t, float *best_ms, neuvv_stream stream);

/* Picks the pixel tile of the camera rays' packets (NEUVV_TILES_8X4, _4X8 or
 * _16X2) for this tree: generates the rays of the given cameras (host
 * [n_cams], 1..32, at most 2^31 pixels in all; times host [n_cams] in
 * [0, 1]) in each tiling with neuvv_camera_rays and times the packet
 * forward (tree's launch, segment log of 64 bytes per ray) on them; the
 * fastest is stored in the tree (neuvv_tree_info.packet_tiles) and written
 * to *best_tiles.  The caller generates its rays with that tiling.
 * Synchronous; allocates and frees its buffers.  best_ms nullable. */
neuvv_status neuvv_autotune_tiles(neuvv_tree *tree, const neuvv_camera *cams, const float *times, int32_t n_cams,
                                  int32_t *best_tiles, float *best_ms, neuvv_stream stream);

/* One candidate of neuvv_autotune and its best time of three. */
typedef struct {
  int32_t block, queue, ready, order;
  float ms;
} neuvv_tune_entry;

/* The candidates the tree's last neuvv_autotune timed (or the kept table it
 * reused), in timing order: up to max_entries copied to entries (host),
 * their number to *n_entries; *from_cache (nullable) is 1 when that call
 * reused a kept choice.  Host only. */
neuvv_status neuvv_autotune_report(const neuvv_tree *tree, neuvv_tune_entry *entries, int32_t max_entries,
                                   int32_t *n_entries, int32_t *from_cache);

/* Forgets every choice neuvv_autotune kept (the next call times again). */
neuvv_status neuvv_autotune_clear_cache(void);

#ifdef __cplusplus
}
#endif

#endif /* NEUVV_H */
