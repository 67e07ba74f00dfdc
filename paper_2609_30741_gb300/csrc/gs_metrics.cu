// SSIM of an image against a reference on the GPU (the quality metric Table 2
// reports beside PSNR), in the convention of the 2DGS/3DGS evaluation code:
// 11 x 11 Gaussian window (sigma 1.5), same-size filtering with zero padding,
// C1 = 0.01^2, C2 = 0.03^2, the mean of the SSIM map over every pixel of every
// channel.
//
// One CTA per 32 x 32 output tile and channel: the 42 x 42 window of both
// images (zero outside) goes to shared memory, a horizontal pass filters the
// five quantities x, y, x^2, y^2, xy into 42 x 32 rows, a vertical pass gives
// the local means and second moments of every output pixel, and the CTA's sum
// of the SSIM map is written in double. A one-block kernel adds the partial
// sums in a fixed order (the result does not depend on scheduling) and divides.
#include "gs_internal.cuh"
#include "gs_launch.cuh"

namespace gs {

namespace {

constexpr int kSsT = 32;                 // output tile edge
constexpr int kSsR = 5;                  // window radius
constexpr int kSsW = kSsT + 2 * kSsR;    // 42: input window edge
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

struct GaussW {
  float w[2 * kSsR + 1];  // normalised 1-D weights; the 2-D window is their outer product
};

__global__ void __launch_bounds__(256) ssim_tile_kernel(const float *__restrict__ a, const float *__restrict__ b,
                                                        int W, int H, GaussW gw, double *__restrict__ part) {
  griddep_wait();
  __shared__ float sa[kSsW][kSsW + 1], sb[kSsW][kSsW + 1];
  __shared__ float hq[5][kSsW][kSsT + 1];
  const int tx0 = blockIdx.x * kSsT, ty0 = blockIdx.y * kSsT, ch = blockIdx.z;
  const size_t plane = (size_t)W * H * ch;
  for (int i = threadIdx.x; i < kSsW * kSsW; i += blockDim.x) {
    const int r = i / kSsW, c = i % kSsW;
    const int y = ty0 - kSsR + r, x = tx0 - kSsR + c;
    const bool in = y >= 0 && y < H && x >= 0 && x < W;
    const size_t p = plane + (size_t)y * W + x;
    sa[r][c] = in ? a[p] : 0.f;
    sb[r][c] = in ? b[p] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kSsW * kSsT; i += blockDim.x) {
    const int r = i / kSsT, c = i % kSsT;
    float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f, m4 = 0.f;
#pragma unroll
    for (int k = 0; k < 2 * kSsR + 1; ++k) {
      const float x = sa[r][c + k], y = sb[r][c + k], g = gw.w[k];
      m0 = fmaf(g, x, m0);
      m1 = fmaf(g, y, m1);
      m2 = fmaf(g, x * x, m2);
      m3 = fmaf(g, y * y, m3);
      m4 = fmaf(g, x * y, m4);
    }
    hq[0][r][c] = m0;
    hq[1][r][c] = m1;
    hq[2][r][c] = m2;
    hq[3][r][c] = m3;
    hq[4][r][c] = m4;
  }
  __syncthreads();
  double acc = 0.0;
  for (int i = threadIdx.x; i < kSsT * kSsT; i += blockDim.x) {
    const int r = i / kSsT, c = i % kSsT;
    if (ty0 + r >= H || tx0 + c >= W) continue;
    float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 2 * kSsR + 1; ++k) {
      const float g = gw.w[k];
#pragma unroll
      for (int q = 0; q < 5; ++q) m[q] = fmaf(g, hq[q][r + k][c], m[q]);
    }
    const float mx = m[0], my = m[1];
    const float sxx = m[2] - mx * mx, syy = m[3] - my * my, sxy = m[4] - mx * my;
    const float v = ((2.f * mx * my + kC1) * (2.f * sxy + kC2)) / ((mx * mx + my * my + kC1) * (sxx + syy + kC2));
    acc += (double)v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double s_red[8];
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
    part[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(256) ssim_finish_kernel(const double *__restrict__ part, int n, double count,
                                                          float *__restrict__ out) {
  griddep_wait();
  __shared__ double s[256];
  double t = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) t += part[i];
  s[threadIdx.x] = t;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = (float)(s[0] / count);
}

}  // namespace

size_t ssim_partials(int max_w, int max_h) {
  return (size_t)((max_w + kSsT - 1) / kSsT) * (size_t)((max_h + kSsT - 1) / kSsT) * 3;
}

cudaError_t launch_ssim(const float *a, const float *b, int W, int H, int C, double *part, float *out,
                        cudaStream_t s) {
  GaussW gw;
  double g[2 * kSsR + 1], sum = 0.0;
  for (int k = 0; k <= 2 * kSsR; ++k) {
    const double x = (double)(k - kSsR);
    g[k] = exp(-x * x / (2.0 * 1.5 * 1.5));
    sum += g[k];
  }
  for (int k = 0; k <= 2 * kSsR; ++k) gw.w[k] = (float)(g[k] / sum);
  const dim3 grid((W + kSsT - 1) / kSsT, (H + kSsT - 1) / kSsT, C);
  cudaError_t e = launch_k(ssim_tile_kernel, grid, 256, 0, s, a, b, W, H, gw, part);
  if (e == cudaSuccess)
    e = launch_k(ssim_finish_kernel, 1, 256, 0, s, (const double *)part, (int)(grid.x * grid.y * grid.z),
                 (double)W * H * C, out);
  GS_LAUNCHED(2);
  return e;
}

}  // namespace gs
