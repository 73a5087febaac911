// Spotlight lighting of a rendered VOctree (Sec. 5 "Spotlight Lighting"):
//   * gaussian_blur_kernel -- the low-pass filter of the low-resolution alpha
//     map rendered from a camera at the light (against Moire patterns);
//   * spotlight_kernel     -- per viewer ray, the distance falloff of the
//     performer's colour at its depth point, and the ground lit through the
//     reversed, filtered alpha map projected from the light.
#include "neuvv_kernels.h"

namespace neuvv {

// One thread per output pixel: the 2D product of the 1D weights, taps
// clamped to the image (edge pixels repeat beyond the border).
__global__ void __launch_bounds__(256) gaussian_blur_kernel(const float *__restrict__ in, float *__restrict__ out,
                                                            int width, int height, long long n_pix,
                                                            const __grid_constant__ BlurWeights bw) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n_pix;
       p += (long long)gridDim.x * blockDim.x) {
    const long long img = p / ((long long)width * height);
    const long long q = p - img * width * height;
    const int y = (int)(q / width), x = (int)(q - (long long)y * width);
    const float *base = in + img * width * height;
    float acc = 0.f;
    for (int j = -bw.radius; j <= bw.radius; ++j) {
      const int yy = min(max(y + j, 0), height - 1);
      float row = 0.f;
      for (int i = -bw.radius; i <= bw.radius; ++i) {
        const int xx = min(max(x + i, 0), width - 1);
        row = fmaf(bw.w[i + bw.radius], __ldg(base + (long long)yy * width + xx), row);
      }
      acc = fmaf(bw.w[j + bw.radius], row, acc);
    }
    out[p] = acc;
  }
}

__device__ __forceinline__ float falloff(const float p[3], const float L[3], float r2_ref) {
  const float dx = p[0] - L[0], dy = p[1] - L[1], dz = p[2] - L[2];
  return r2_ref / fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

// Texel (x, y) of the light's alpha map; 0 outside it (no occluder).
__device__ __forceinline__ float texel(const float *map, int w, int h, int x, int y) {
  return (x >= 0 && x < w && y >= 0 && y < h) ? __ldg(map + (long long)y * w + x) : 0.f;
}

__global__ void __launch_bounds__(256) spotlight_kernel(const __grid_constant__ SpotArgs a) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.rays.n) return;
  float o[3], d[3], t;
  load_ray(a.rays, i, o, d, t);
  const float len = sqrtf(fmaf(d[2], d[2], fmaf(d[1], d[1], d[0] * d[0])));
  const float il = 1.f / len;
  const float dn[3] = {d[0] * il, d[1] * il, d[2] * il};
  const float r2 = a.r_ref * a.r_ref;
  float c[3] = {a.rgb[3 * i], a.rgb[3 * i + 1], a.rgb[3 * i + 2]};
  const float depth = a.depth[i];
  if (len > 0.f && isfinite(depth)) {
    const float X[3] = {fmaf(depth, dn[0], o[0]), fmaf(depth, dn[1], o[1]), fmaf(depth, dn[2], o[2])};
    const float f = falloff(X, a.light.eye, r2);
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) c[ch] *= f;
  }
  const float s = len > 0.f && dn[2] != 0.f ? (a.ground_z - o[2]) / dn[2] : -1.f;
  if (s > 0.f && isfinite(s)) {
    const float P[3] = {fmaf(s, dn[0], o[0]), fmaf(s, dn[1], o[1]), fmaf(s, dn[2], o[2])};
    const float v[3] = {P[0] - a.light.eye[0], P[1] - a.light.eye[1], P[2] - a.light.eye[2]};
    const float zc = a.light.forward[0] * v[0] + a.light.forward[1] * v[1] + a.light.forward[2] * v[2];
    float al = 0.f;
    if (zc > 0.f) {
      const float sx = (a.light.right[0] * v[0] + a.light.right[1] * v[1] + a.light.right[2] * v[2]) / zc;
      const float sy = (a.light.up[0] * v[0] + a.light.up[1] * v[1] + a.light.up[2] * v[2]) / zc;
      const int W = a.light.width, H = a.light.height;
      const float th = tanf(a.light.fov_y_deg * (kPi / 360.f));
      const float px = (sx / (th * (float)W / (float)H) + 1.f) * 0.5f * (float)W - 0.5f;
      const float py = (1.f - sy / th) * 0.5f * (float)H - 0.5f;
      if (px > -2.f && px < (float)W + 1.f && py > -2.f && py < (float)H + 1.f) {
        const float fx0 = floorf(px), fy0 = floorf(py);
        const int x0 = (int)fx0, y0 = (int)fy0;
        const float fx = px - fx0, fy = py - fy0;
        al = (1.f - fx) * (1.f - fy) * texel(a.light_alpha, W, H, x0, y0) +
             fx * (1.f - fy) * texel(a.light_alpha, W, H, x0 + 1, y0) +
             (1.f - fx) * fy * texel(a.light_alpha, W, H, x0, y0 + 1) + fx * fy * texel(a.light_alpha, W, H, x0 + 1, y0 + 1);
      }
    }
    const float g = (1.f - a.alpha[i]) * (1.f - al) * falloff(P, a.light.eye, r2);
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) c[ch] = fmaf(g, a.albedo[ch], c[ch]);
  }
  a.out[3 * i] = c[0];
  a.out[3 * i + 1] = c[1];
  a.out[3 * i + 2] = c[2];
}

cudaError_t launch_gaussian_blur(const float *in, float *out, int width, int height, long long n_images,
                                 const BlurWeights &bw, cudaStream_t s) {
  const long long n_pix = n_images * width * height;
  if (n_pix == 0) return cudaSuccess;
  const long long want = (n_pix + 255) / 256;
  gaussian_blur_kernel<<<(unsigned)(want < 152 * 16 ? want : 152 * 16), 256, 0, s>>>(in, out, width, height, n_pix,
                                                                                    bw);
  return cudaGetLastError();
}

cudaError_t launch_spotlight(const SpotArgs &a, cudaStream_t s) {
  if (a.rays.n == 0) return cudaSuccess;
  spotlight_kernel<<<(unsigned)((a.rays.n + 255) / 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace neuvv
