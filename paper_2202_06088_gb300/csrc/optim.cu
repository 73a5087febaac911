// Training-step kernels around the renderer (Sec. 4.3 "Optimization"):
//   * mse_kernel  -- Eq. rgb-loss, sum ||C - C_gt||^2 (scaled) and dL/dC;
//   * adam_kernel -- Adam restricted to leaves whose touched bit is set
//     (sparse: other leaves keep weights and moments), FP32 master + moments,
//     storage copy rewritten (BF16 rounded to nearest even, or FP8 E4M3 with
//     fresh per-leaf scales), gradient rows of
//     updated leaves reset to zero for the next step.
#include "neuvv_kernels.h"

namespace neuvv {

__global__ void __launch_bounds__(256) mse_kernel(const float *__restrict__ rgb, const float *__restrict__ target,
                                                  long long n, float scale, float *__restrict__ grad,
                                                  float *__restrict__ loss) {
  float part = 0.f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < 3 * n;
       i += (long long)gridDim.x * blockDim.x) {
    const float r = rgb[i] - target[i];
    grad[i] = 2.f * scale * r;
    part = fmaf(r, r, part);
  }
  if (loss) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, o);
    __shared__ float red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      float s = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
      atomicAdd(loss, scale * s);
    }
  }
}

// Image-gradient regulariser L_grad (Sec. 4.3 "Optimization"): with
// E = |I - I_hat| per channel, lam * sum over views of the squared forward
// differences of E between horizontally and vertically adjacent pixels.
// map: ray of each pixel [n_views][height][width], -1 for none.
//
// A block takes tiles of kGradTileW x kGradTileH pixels of one view.  It
// stages I - I_hat of the tile and a one-pixel halo in shared memory (the
// map, rendered colours and targets are read about 1.3 times each instead of
// five), then each thread adds to its own ray's dL/dI_hat the derivative of
// the (up to four) differences its pixel takes part in, and to the loss the
// two it owns (towards its right and lower neighbours).
constexpr int kGradTileW = 32, kGradTileH = 8;
constexpr int kGradHaloW = kGradTileW + 2, kGradHaloH = kGradTileH + 2;

__global__ void __launch_bounds__(kGradTileW *kGradTileH)
    grad_loss_kernel(const float *__restrict__ rgb, const float *__restrict__ target, const int *__restrict__ map,
                     int width, int height, long long n_views, long long n_rays, float lam, float *__restrict__ grad,
                     float *__restrict__ loss) {
  __shared__ float dv[3][kGradHaloH][kGradHaloW];  // I - I_hat, per channel
  __shared__ int ray[kGradHaloH][kGradHaloW];      // -1: no ray (missing pixel or outside the image)
  const int tiles_x = (width + kGradTileW - 1) / kGradTileW, tiles_y = (height + kGradTileH - 1) / kGradTileH;
  const long long per_view = (long long)tiles_x * tiles_y, n_tiles = per_view * n_views;
  const int lx = threadIdx.x % kGradTileW, ly = threadIdx.x / kGradTileW;
  float part = 0.f;
  for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const long long view = tile / per_view;
    const long long rest = tile - view * per_view;
    const int y0 = (int)(rest / tiles_x) * kGradTileH - 1, x0 = (int)(rest % tiles_x) * kGradTileW - 1;
    const int *vmap = map + view * (long long)width * height;
    for (int h = threadIdx.x; h < kGradHaloH * kGradHaloW; h += blockDim.x) {
      const int hy = h / kGradHaloW, hx = h - hy * kGradHaloW;
      const int y = y0 + hy, x = x0 + hx;
      int q = -1;
      if (x >= 0 && x < width && y >= 0 && y < height) q = __ldg(vmap + (long long)y * width + x);
      if (q >= n_rays) q = -1;
      ray[hy][hx] = q < 0 ? -1 : q;
      if (q >= 0) {
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) dv[ch][hy][hx] = __ldg(rgb + 3LL * q + ch) - __ldg(target + 3LL * q + ch);
      }
    }
    __syncthreads();
    const int hy = ly + 1, hx = lx + 1;
    const int r = ray[hy][hx];
    if (r >= 0) {
      float g[3] = {0.f, 0.f, 0.f};
      // neighbours: left, right, up, down; sgn = +1 when this pixel is the
      // second of the pair (the difference is E_this - E_other), -1 otherwise
      const int ny[4] = {hy, hy, hy - 1, hy + 1};
      const int nx[4] = {hx - 1, hx + 1, hx, hx};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (ray[ny[k]][nx[k]] < 0) continue;
        const bool second = (k == 0 || k == 2);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
          const float E = fabsf(dv[ch][hy][hx]), Eq = fabsf(dv[ch][ny[k]][nx[k]]);
          const float D = second ? E - Eq : Eq - E;
          g[ch] = second ? fmaf(2.f, D, g[ch]) : fmaf(-2.f, D, g[ch]);
          if (!second) part = fmaf(D, D, part);
        }
      }
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        const float d = dv[ch][hy][hx];
        const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
        grad[3LL * r + ch] += lam * sgn * g[ch];
      }
    }
    __syncthreads();  // the staging arrays are refilled by the next tile
  }
  if (loss) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, o);
    __shared__ float red[kGradTileW * kGradTileH / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      float s = 0.f;
      for (int w = 0; w < kGradTileW * kGradTileH / 32; ++w) s += red[w];
      atomicAdd(loss, lam * s);
    }
  }
}


// One warp per word of the touched bitmap (32 leaves): an empty word is
// skipped at once, and each set bit's leaf is updated by the warp, one
// 4-float quad of its record per lane, so a row is one coalesced access.
__global__ void __launch_bounds__(256) adam_kernel(float *__restrict__ master, float *__restrict__ m,
                                                   float *__restrict__ v, void *__restrict__ storage, int dt,
                                                   int storage_stride, float *__restrict__ grad,
                                                   const unsigned int *__restrict__ touched, long long n_leaves,
                                                   int stride_f32, int rec_len, float lr, float b1, float b2,
                                                   float eps, float c1, float c2) {
  const int quads = (rec_len + 3) / 4;  // quads past the record's entries are padding and stay zero
  const int lane = threadIdx.x & 31;
  const float lr_c1 = lr / c1, inv_c2 = 1.f / c2;
  const long long n_words = (n_leaves + 31) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long wd = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; wd < n_words; wd += nwarps) {
    unsigned int bits = __ldg(touched + wd);  // the same for the whole warp
    while (bits) {
      const long long leaf = (wd << 5) + (__ffs(bits) - 1);
      bits &= bits - 1u;
      for (int q = lane; q < quads; q += 32) {
        const size_t off = (size_t)leaf * stride_f32 + 4 * q;
        float4 g = *reinterpret_cast<const float4 *>(grad + off);
        float4 w = *reinterpret_cast<const float4 *>(master + off);
        float4 mm = *reinterpret_cast<const float4 *>(m + off);
        float4 vv = *reinterpret_cast<const float4 *>(v + off);
        float gs[4] = {g.x, g.y, g.z, g.w}, ws[4] = {w.x, w.y, w.z, w.w};
        float ms[4] = {mm.x, mm.y, mm.z, mm.w}, vs[4] = {vv.x, vv.y, vv.z, vv.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (4 * q + k >= rec_len) continue;  // padding stays zero
          adam_entry(gs[k], b1, b2, lr_c1, inv_c2, eps, ws[k], ms[k], vs[k]);
        }
        *reinterpret_cast<float4 *>(master + off) = make_float4(ws[0], ws[1], ws[2], ws[3]);
        *reinterpret_cast<float4 *>(m + off) = make_float4(ms[0], ms[1], ms[2], ms[3]);
        *reinterpret_cast<float4 *>(v + off) = make_float4(vs[0], vs[1], vs[2], vs[3]);
        *reinterpret_cast<float4 *>(grad + off) = make_float4(0.f, 0.f, 0.f, 0.f);
        if (dt == kBF16) {
          unsigned short *st = static_cast<unsigned short *>(storage) + (size_t)leaf * storage_stride + 4 * q;
          const unsigned int lo = f32_to_bf16_rne(ws[0]) | ((unsigned int)f32_to_bf16_rne(ws[1]) << 16);
          const unsigned int hi = f32_to_bf16_rne(ws[2]) | ((unsigned int)f32_to_bf16_rne(ws[3]) << 16);
          *reinterpret_cast<uint2 *>(st) = make_uint2(lo, hi);
        }
      }
    }
  }
}

// FP8 storage: one warp per leaf.  The warp applies the same Adam update,
// then takes the largest magnitude of each group (w_sigma, w_gamma, w_hh),
// picks its power-of-two scale and re-encodes the whole record: header of
// scales, then one E4M3 code (nearest, ties to even) per entry.
__global__ void __launch_bounds__(256) adam_fp8_kernel(float *__restrict__ master, float *__restrict__ m,
                                                       float *__restrict__ v, unsigned char *__restrict__ storage,
                                                       int storage_stride, float *__restrict__ grad,
                                                       const unsigned int *__restrict__ touched, long long n_leaves,
                                                       int stride_f32, int rec_len, int kp, float lr, float b1,
                                                       float b2, float eps, float c1, float c2) {
  constexpr int kMaxRounds = 2;  // stride_f32 <= 256 floats (64 quads) per leaf
  const int lane = threadIdx.x & 31;
  const float lr_c1 = lr / c1, inv_c2 = 1.f / c2;
  const int quads = stride_f32 / 4;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long n_words = (n_leaves + 31) >> 5;
  // one warp per word of the touched bitmap: empty words are skipped at once
  for (long long wd = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; wd < n_words; wd += nwarps)
  for (unsigned int bits = __ldg(touched + wd); bits; bits &= bits - 1u) {
    const long long leaf = (wd << 5) + (__ffs(bits) - 1);
    float ws[kMaxRounds][4];
    float mx[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int r = 0; r < kMaxRounds; ++r) {
      const int q = lane + 32 * r;
      if (q >= quads) continue;
      const size_t off = (size_t)leaf * stride_f32 + 4 * q;
      const float4 g = *reinterpret_cast<const float4 *>(grad + off);
      const float4 w = *reinterpret_cast<const float4 *>(master + off);
      const float4 mm = *reinterpret_cast<const float4 *>(m + off);
      const float4 vv = *reinterpret_cast<const float4 *>(v + off);
      float gs[4] = {g.x, g.y, g.z, g.w}, ms[4] = {mm.x, mm.y, mm.z, mm.w}, vs[4] = {vv.x, vv.y, vv.z, vv.w};
      ws[r][0] = w.x;
      ws[r][1] = w.y;
      ws[r][2] = w.z;
      ws[r][3] = w.w;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int j = 4 * q + k;
        if (j >= rec_len) continue;  // padding stays zero
        adam_entry(gs[k], b1, b2, lr_c1, inv_c2, eps, ws[r][k], ms[k], vs[k]);
        const int grp = j < kp ? 0 : (j < 2 * kp ? 1 : 2);
        mx[grp] = fmaxf(mx[grp], fabsf(ws[r][k]));
      }
      *reinterpret_cast<float4 *>(master + off) = make_float4(ws[r][0], ws[r][1], ws[r][2], ws[r][3]);
      *reinterpret_cast<float4 *>(m + off) = make_float4(ms[0], ms[1], ms[2], ms[3]);
      *reinterpret_cast<float4 *>(v + off) = make_float4(vs[0], vs[1], vs[2], vs[3]);
      *reinterpret_cast<float4 *>(grad + off) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    int p[3];
#pragma unroll
    for (int g = 0; g < 3; ++g) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx[g] = fmaxf(mx[g], __shfl_xor_sync(0xFFFFFFFFu, mx[g], o));
      p[g] = fp8_scale_exp(mx[g]);
    }
    unsigned char *rec = storage + (size_t)leaf * storage_stride;
    if (lane == 0)
      *reinterpret_cast<uint4 *>(rec) = make_uint4(__float_as_uint(ldexpf(1.f, p[0])), __float_as_uint(ldexpf(1.f, p[1])),
                                                   __float_as_uint(ldexpf(1.f, p[2])), 0u);
#pragma unroll
    for (int r = 0; r < kMaxRounds; ++r) {
      const int q = lane + 32 * r;
      if (q >= quads) continue;
      unsigned int word = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int j = 4 * q + k;
        if (j >= rec_len) continue;
        const int grp = j < kp ? 0 : (j < 2 * kp ? 1 : 2);
        const unsigned int code = __nv_cvt_float_to_fp8(ldexpf(ws[r][k], -p[grp]), __NV_SATFINITE, __NV_E4M3);
        word |= code << (8 * k);
      }
      *reinterpret_cast<unsigned int *>(rec + 16 + 4 * q) = word;
    }
  }
}

// Writes FP32 records (the gradient / master layout) into a tree: the master
// copy when there is one, and the storage records in the storage type (BF16
// rounded to nearest even; FP8 with the per-leaf group scales of tree
// creation).  One warp per leaf; entries past rec_len stay zero.
__global__ void __launch_bounds__(256) store_records_kernel(const float *__restrict__ src, float *__restrict__ master,
                                                            void *__restrict__ storage, int dt, int storage_stride,
                                                            long long n_leaves, int stride_f32, int rec_len, int kp) {
  const int lane = threadIdx.x & 31;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long leaf = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; leaf < n_leaves; leaf += nwarps) {
    const float *r = src + (size_t)leaf * stride_f32;
    float mx[3] = {0.f, 0.f, 0.f};
    for (int j = lane; j < stride_f32; j += 32) {
      const float w = j < rec_len ? r[j] : 0.f;
      if (master) master[(size_t)leaf * stride_f32 + j] = w;
      if (dt == kF32) static_cast<float *>(storage)[(size_t)leaf * storage_stride + j] = w;
      else if (dt == kBF16 && j < storage_stride)
        static_cast<unsigned short *>(storage)[(size_t)leaf * storage_stride + j] = f32_to_bf16_rne(w);
      const int grp = j < kp ? 0 : (j < 2 * kp ? 1 : 2);
      mx[grp] = fmaxf(mx[grp], fabsf(w));
    }
    if (dt != kFP8) continue;
    int p[3];
#pragma unroll
    for (int g = 0; g < 3; ++g) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx[g] = fmaxf(mx[g], __shfl_xor_sync(0xFFFFFFFFu, mx[g], o));
      p[g] = fp8_scale_exp(mx[g]);
    }
    unsigned char *rec = static_cast<unsigned char *>(storage) + (size_t)leaf * storage_stride;
    if (lane == 0)
      *reinterpret_cast<uint4 *>(rec) = make_uint4(__float_as_uint(ldexpf(1.f, p[0])), __float_as_uint(ldexpf(1.f, p[1])),
                                                   __float_as_uint(ldexpf(1.f, p[2])), 0u);
    for (int j = lane; 16 + j < storage_stride; j += 32) {
      unsigned char code = 0;
      if (j < rec_len) {
        const int grp = j < kp ? 0 : (j < 2 * kp ? 1 : 2);
        code = (unsigned char)__nv_cvt_float_to_fp8(ldexpf(r[j], -p[grp]), __NV_SATFINITE, __NV_E4M3);
      }
      rec[16 + j] = code;
    }
  }
}

cudaError_t launch_store_records(const float *src, float *master, void *storage, DType dt, int storage_stride,
                                 long long n_leaves, int stride_f32, int rec_len, int kp, cudaStream_t s) {
  if (n_leaves == 0) return cudaSuccess;
  const long long want = (n_leaves * 32 + 255) / 256;
  const int blocks = (int)(want < 152 * 16 ? want : 152 * 16);
  store_records_kernel<<<blocks, 256, 0, s>>>(src, master, storage, (int)dt, storage_stride, n_leaves, stride_f32,
                                              rec_len, kp);
  return cudaGetLastError();
}

cudaError_t launch_mse(const float *rgb, const float *target, long long n, float scale, float *grad, float *loss,
                       cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const long long want = (3 * n + 255) / 256;
  const int blocks = (int)(want < 152 * 8 ? want : 152 * 8);
  mse_kernel<<<blocks, 256, 0, s>>>(rgb, target, n, scale, grad, loss);
  return cudaGetLastError();
}

cudaError_t launch_grad_loss(const float *rgb, const float *target, const int *map, int width, int height,
                             long long n_views, long long n_rays, float lam, float *grad, float *loss, cudaStream_t s) {
  if (n_views * width * height == 0) return cudaSuccess;
  const long long tiles = n_views * ((width + kGradTileW - 1) / kGradTileW) * ((height + kGradTileH - 1) / kGradTileH);
  const int blocks = (int)(tiles < 152 * 8 ? tiles : 152 * 8);
  grad_loss_kernel<<<blocks, kGradTileW * kGradTileH, 0, s>>>(rgb, target, map, width, height, n_views, n_rays, lam,
                                                              grad, loss);
  return cudaGetLastError();
}

cudaError_t launch_adam(float *master, float *m, float *v, void *storage, DType dt, int storage_stride, float *grad,
                        const unsigned int *touched, long long n_leaves, int stride_f32, int rec_len, int kp,
                        float lr, float b1, float b2, float eps, float c1, float c2, cudaStream_t s) {
  if (n_leaves == 0) return cudaSuccess;
  if (dt == kFP8) {
    if (stride_f32 > 256 || !storage) return cudaErrorInvalidValue;
    const long long want = ((n_leaves + 31) / 32 * 32 + 255) / 256;
    const int blocks = (int)(want < 152 * 16 ? want : 152 * 16);
    adam_fp8_kernel<<<blocks, 256, 0, s>>>(master, m, v, static_cast<unsigned char *>(storage), storage_stride, grad,
                                           touched, n_leaves, stride_f32, rec_len, kp, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
  }
  const long long want = ((n_leaves + 31) / 32 * 32 + 255) / 256;  // one warp per bitmap word
  const int blocks = (int)(want < 152 * 16 ? want : 152 * 16);
  adam_kernel<<<blocks, 256, 0, s>>>(master, m, v, storage, (int)dt, storage_stride, grad, touched, n_leaves,
                                     stride_f32, rec_len, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

}  // namespace neuvv
