// Ray setup (Sec. 4.3 "Rendering"): one pinhole-camera ray through the centre
// of every pixel of each view, written straight into the renderer's ray SoA so
// that a training step uploads only its target images and camera poses.
//
// Order of the rays of one camera: row-major, or by TW x TH pixel tiles of 32
// pixels (8x4, 4x8 or 16x2; tiles in row-major order, the pixels of a tile
// row-major, narrower tiles at the right edge and shorter ones at the
// bottom), so that the 32 rays of a packet cover one compact tile.
#include "neuvv_kernels.h"

namespace neuvv {

// Pixel (px, py) of the j-th ray of a width x height camera.
__device__ __forceinline__ void pixel_of_ray(long long j, int width, int height, int TW, int TH, int &px, int &py) {
  if (TW == 0) {
    py = (int)(j / width);
    px = (int)(j - (long long)py * width);
    return;
  }
  const long long band_pixels = (long long)TH * width;  // a full band of TH rows
  const int band = (int)(j / band_pixels);
  const int y0 = band * TH, h = min(TH, height - y0);
  const long long o = j - (long long)band * band_pixels;  // offset within the band (h rows)
  const int full = width / TW;
  const long long tile_pixels = (long long)TW * h;
  const long long c = o / tile_pixels;
  int x0, w;
  long long within;
  if (c < full) {
    x0 = (int)c * TW;
    w = TW;
    within = o - c * tile_pixels;
  } else {  // the narrower tile at the right edge
    x0 = full * TW;
    w = width - x0;
    within = o - (long long)full * tile_pixels;
  }
  py = y0 + (int)(within / w);
  px = x0 + (int)(within - (within / w) * w);
}

__global__ void __launch_bounds__(256) camera_rays_kernel(const __grid_constant__ CamBatch cb, float *__restrict__ o,
                                                          float *__restrict__ d, float *__restrict__ t,
                                                          int *__restrict__ pixel, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    int c = 0;  // the camera owning ray i: the last offset <= i
    for (int step = kMaxCams / 2; step > 0; step >>= 1)
      if (c + step < cb.n_cams && cb.off[c + step] <= i) c += step;
    const LightCam &cam = cb.cam[c];
    int px, py;
    pixel_of_ray(i - cb.off[c], cam.width, cam.height, cb.tile_w, cb.tile_h, px, py);
    const float sx = (2.f * ((float)px + 0.5f) / (float)cam.width - 1.f) * cb.tan_half[c] * cb.aspect[c];
    const float sy = (1.f - 2.f * ((float)py + 0.5f) / (float)cam.height) * cb.tan_half[c];
    float v[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) v[k] = fmaf(cam.up[k], sy, fmaf(cam.right[k], sx, cam.forward[k]));
    const float inv = 1.f / sqrtf(fmaf(v[0], v[0], fmaf(v[1], v[1], v[2] * v[2])));
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      o[k * n + i] = cam.eye[k];
      d[k * n + i] = v[k] * inv;
    }
    t[i] = cb.t[c];
    if (pixel) pixel[i] = py * cam.width + px;
  }
}

cudaError_t launch_camera_rays(const CamBatch &cb, float *o, float *d, float *t, int *pixel, long long n,
                               cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const long long want = (n + 255) / 256;
  const int blocks = (int)(want < 152 * 8 ? want : 152 * 8);
  camera_rays_kernel<<<blocks, 256, 0, s>>>(cb, o, d, t, pixel, n);
  return cudaGetLastError();
}

}  // namespace neuvv
