// Allocation-free forward warp: the depth-tested warp of the dominant eye into
// the affiliated eye, with its per-pixel scratch in a static device array.
//
// Who needs it: code that must not allocate device memory while it renders,
// for instance a compositor or plugin running inside a host framework that
// owns the GPU memory pool and forbids outside allocations, or a frame loop
// with a hard per-frame deadline where a cudaMalloc may stall or fail. Such a
// caller still passes its own input and output buffers; the only scratch, one
// 64-bit key per affiliated pixel, lives in g_warp_keys below, which every
// device that loads this library keeps for the life of the process.
#include <mutex>

#include "gs_internal.cuh"

namespace gs {
namespace {

// GS_WARP_NOALLOC_MAX_PIXELS = 2^22 pixels (2048 x 2048, or any frame with no
// more pixels): 32 MiB of packed keys.
constexpr int64_t kNoAllocMaxPixels = GS_WARP_NOALLOC_MAX_PIXELS;
constexpr unsigned long long kEmptyKey = ~0ull;
constexpr uint32_t kBackgroundBits = 0x7f800000u;

__device__ __align__(256) unsigned long long g_warp_keys[kNoAllocMaxPixels];

struct WarpCams {
  float Rrel[9], trel[3];
  float fx, fy, cx, cy;  // shared by both eyes
};

// FP64 composition of the relative pose on one thread (dominant camera ->
// affiliated camera, Eq. 4 then Eq. 5), rounded to float like the renderer's.
struct PosePair {
  double Rd[9], td[3], Ra[9], ta[3];
  double fx, fy, cx, cy;
};

__global__ void noalloc_pose_kernel(PosePair pp, WarpCams *out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  WarpCams wc;
  for (int i = 0; i < 3; ++i) {
    double tr = 0.0;
    for (int j = 0; j < 3; ++j) {
      double r = 0.0;
      for (int k = 0; k < 3; ++k) r += pp.Ra[k * 3 + i] * pp.Rd[k * 3 + j];
      wc.Rrel[i * 3 + j] = (float)r;
      tr += pp.Ra[j * 3 + i] * (pp.td[j] - pp.ta[j]);
    }
    wc.trel[i] = (float)tr;
  }
  wc.fx = (float)pp.fx; wc.fy = (float)pp.fy; wc.cx = (float)pp.cx; wc.cy = (float)pp.cy;
  *out = wc;
}

__device__ WarpCams g_warp_cams;

__global__ void noalloc_clear_kernel(unsigned long long *keys, int64_t n) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    keys[p] = kEmptyKey;
}

// Source pixel -> destination pixel, as the renderer's warp: a surface sample
// (coverage 1 - T >= 0.5) at depth D / (1 - T), else a background sample at
// infinite depth; the packed (float depth bits << 32 | source index) key makes
// one 64-bit atomicMin the depth test.
__global__ void noalloc_scatter_kernel(const WarpCams *__restrict__ wcp, const float *__restrict__ depth,
                                       const float *__restrict__ trans, unsigned long long *__restrict__ keys, int W,
                                       int H) {
  const WarpCams &c = *wcp;
  const int64_t npix = (int64_t)W * H;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x) {
    const float cov = 1.f - trans[p];
    const bool surface = cov >= 0.5f;
    const float d = surface ? depth[p] / cov : 0.f;
    const float rx = ((float)(p % W) - c.cx) / c.fx, ry = ((float)(p / W) - c.cy) / c.fy;
    const float *R = c.Rrel;
    float X, Y, Z;
    if (surface) {
      X = fmaf(R[0], rx * d, fmaf(R[1], ry * d, fmaf(R[2], d, c.trel[0])));
      Y = fmaf(R[3], rx * d, fmaf(R[4], ry * d, fmaf(R[5], d, c.trel[1])));
      Z = fmaf(R[6], rx * d, fmaf(R[7], ry * d, fmaf(R[8], d, c.trel[2])));
      if (!(Z > kZNear)) continue;
    } else {
      X = fmaf(R[0], rx, fmaf(R[1], ry, R[2]));
      Y = fmaf(R[3], rx, fmaf(R[4], ry, R[5]));
      Z = fmaf(R[6], rx, fmaf(R[7], ry, R[8]));
      if (!(Z > 0.f)) continue;
    }
    const float u = fmaf(c.fx, X / Z, c.cx), v = fmaf(c.fy, Y / Z, c.cy);
    const float fx = floorf(u + 0.5f), fy = floorf(v + 0.5f);
    if (!(fx >= 0.f && fx <= (float)(W - 1) && fy >= 0.f && fy <= (float)(H - 1))) continue;
    const uint32_t zb = surface ? __float_as_uint(Z) : kBackgroundBits;
    const int64_t q = (int64_t)fy * W + (int64_t)fx;
    atomicMin(keys + q, ((unsigned long long)zb << 32) | (unsigned long long)(uint32_t)p);
  }
}

// Destination pixel: the winner's colour and depth (+inf for a background
// sample), or a hole (colour 0, depth 0, hole = 1).
__global__ void noalloc_resolve_kernel(const unsigned long long *__restrict__ keys, const float *__restrict__ rgb_dom,
                                       int W, int H, float *__restrict__ rgb_out, float *__restrict__ depth_out,
                                       uint8_t *__restrict__ hole_out) {
  const int64_t npix = (int64_t)W * H;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = keys[p];
    const bool hole = k == kEmptyKey;
    const uint32_t s = (uint32_t)(k & 0xffffffffull);
    for (int ch = 0; ch < 3; ++ch) rgb_out[ch * npix + p] = hole ? 0.f : rgb_dom[ch * npix + s];
    if (depth_out) depth_out[p] = hole ? 0.f : __uint_as_float((uint32_t)(k >> 32));
    if (hole_out) hole_out[p] = hole ? 1 : 0;
  }
}

std::mutex g_mu;
unsigned long long *g_keys_ptr[64];
WarpCams *g_cams_ptr[64];

// Device addresses of the static scratch on the current device, looked up once
// per device (with that device current).
cudaError_t scratch_on_current_device(unsigned long long **keys, WarpCams **cams) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_keys_ptr[dev]) {
    void *k = nullptr, *c = nullptr;
    if ((e = cudaGetSymbolAddress(&k, g_warp_keys)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress(&c, g_warp_cams)) != cudaSuccess) return e;
    g_keys_ptr[dev] = (unsigned long long *)k;
    g_cams_ptr[dev] = (WarpCams *)c;
  }
  *keys = g_keys_ptr[dev];
  *cams = g_cams_ptr[dev];
  return cudaSuccess;
}

int grid_for_pixels(int64_t n) {
  const int64_t b = (n + 255) / 256;
  const int64_t cap = sm_grid_cap(16);
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" gs_status gs_warp_noalloc(const float *rgb_dom, const float *depth_dom, const float *trans_dom,
                                     const gs_pose *pose_dom, const gs_pose *pose_aff, const gs_intrinsics *intr,
                                     float *rgb_warp, float *depth_warp, uint8_t *hole, void *stream) {
  if (!rgb_dom || !depth_dom || !trans_dom || !pose_dom || !pose_aff || !intr || !rgb_warp) return GS_ERR_BAD_ARG;
  if (intr->width <= 0 || intr->height <= 0 || !(intr->fx > 0) || !(intr->fy > 0)) return GS_ERR_BAD_ARG;
  const int64_t npix = (int64_t)intr->width * intr->height;
  if (npix > kNoAllocMaxPixels) return GS_ERR_CAPACITY;  // larger than the static scratch
  unsigned long long *keys = nullptr;
  WarpCams *cams = nullptr;
  cudaError_t e = scratch_on_current_device(&keys, &cams);
  if (e != cudaSuccess) return record_cuda_failure("gs_noalloc.cu", __LINE__, e);
  cudaStream_t s = (cudaStream_t)stream;
  PosePair pp;
  memcpy(pp.Rd, pose_dom->R, sizeof(pp.Rd));
  memcpy(pp.td, pose_dom->t, sizeof(pp.td));
  memcpy(pp.Ra, pose_aff->R, sizeof(pp.Ra));
  memcpy(pp.ta, pose_aff->t, sizeof(pp.ta));
  pp.fx = intr->fx; pp.fy = intr->fy; pp.cx = intr->cx; pp.cy = intr->cy;
  noalloc_pose_kernel<<<1, 32, 0, s>>>(pp, cams);
  noalloc_clear_kernel<<<grid_for_pixels(npix), 256, 0, s>>>(keys, npix);
  noalloc_scatter_kernel<<<grid_for_pixels(npix), 256, 0, s>>>(cams, depth_dom, trans_dom, keys, intr->width,
                                                               intr->height);
  noalloc_resolve_kernel<<<grid_for_pixels(npix), 256, 0, s>>>(keys, rgb_dom, intr->width, intr->height, rgb_warp,
                                                               depth_warp, hole);
  GS_LAUNCHED(4);
  e = cudaGetLastError();
  return e == cudaSuccess ? GS_OK : record_cuda_failure("gs_noalloc.cu", __LINE__, e);
}
