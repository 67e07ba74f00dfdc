// Learned repair of the affiliated eye's holes (a data-parallel extension: the
// paper repairs holes by interpolation and ROI re-rendering only, Sec. 3.1
// Stage 3 and Sec. 3.5; this network, its inputs and its per-tile gate are this
// library's own).
//
//   features: warped RGB, inverse depth of the winner, hole mask and the
//     distance to the nearest hole (min(d, 8) / 8), 8 x bf16 per pixel;
//   network: six 3x3 convolutions 6 -> 32 -> 32 -> 32 -> 32 -> 32 -> 4 with
//     zero padding at the image border and ReLU after the first five; output
//     0-2 is an RGB fill, output 3 a gate logit averaged over each 16x16 tile;
//   gate: a tile whose sigmoid(gate) >= tau takes the fill at its hole pixels
//     and leaves the ROI re-render; the others keep the plain path.
//
// The forward pass is one persistent kernel: a CTA loads all six layers' BF16
// weights into shared memory once and then, per 16x16 output tile, runs the six
// convolutions on a 28x28 window (6-pixel halo) as implicit GEMMs on the tensor
// cores. Activations stay in shared memory in the canonical no-swizzle K-major
// layout [channel group][position][8 channels]; a 3x3 tap is just a shift of the
// A operand's start address along the 28-wide grid, so no im2col copy exists.
// One thread issues tcgen05.mma (M = 128 positions, N = 32 channels, K = 16)
// into tensor memory; four warps read the accumulators back, add the bias,
// apply ReLU and the image-border zeroing, and store BF16 for the next layer.
//
// Training runs the same forward kernel (keeping every layer's input), then a
// loss kernel, data-parallel FP32 weight- and input-gradient kernels and AdamW
// on FP32 master weights.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "gs_internal.cuh"
#include "gs_launch.cuh"
#include "gs_scan.cuh"
#include "gs_umma.cuh"

namespace gs {
namespace {

constexpr int kRT = 16;                 // output tile edge
constexpr int kHalo = 6;                // receptive-field radius of six 3x3 layers
constexpr int kGW = kRT + 2 * kHalo;    // 28: width of the position grid
constexpr int kNPos = 832;              // positions per activation buffer (6 M tiles + tap reach)
constexpr int kQ = 26 * kGW;            // gradient grid: rows < 26 of any layer >= 1 output
constexpr int kNetThreads = 256;  // two warpgroups take alternate M tiles of the epilogue
constexpr int kTmemCols = 256;

__host__ __device__ constexpr int cin(int l) { return l == 0 ? 6 : 32; }
__host__ __device__ constexpr int cout(int l) { return l == 5 ? 4 : 32; }
__host__ __device__ constexpr int kgroups(int l) { return l == 0 ? 2 : 4; }   // padded C_in / 8
__host__ __device__ constexpr int ngroups(int l) { return l == 5 ? 2 : 4; }   // padded C_out / 8
__host__ __device__ constexpr int wbytes(int l) { return 9 * kgroups(l) * ngroups(l) * 128; }
__host__ __device__ constexpr int woff(int l) {
  int o = 0;
  for (int i = 0; i < l; ++i) o += wbytes(i);
  return o;
}
__host__ __device__ constexpr int poff(int l) {  // canonical flat parameter offsets
  int o = 0;
  for (int i = 0; i < l; ++i) o += cout(i) * 9 * cin(i) + cout(i);
  return o;
}
__host__ __device__ constexpr int mtiles(int l) { return ((kGW - 2 * (l + 1)) * kGW + 127) / 128; }

constexpr int kMaxMT = 6;  // M tiles of the widest layer
constexpr int kWPackBytes = woff(6);
static_assert(kWPackBytes == 92160, "packed weight image size");
// FP8 images: [tap][2 c_in groups of 16][c_out groups][8][16 B]
__host__ __device__ constexpr int wbytes8(int l) { return 9 * 2 * ngroups(l) * 128; }
__host__ __device__ constexpr int woff8(int l) {
  int o = 0;
  for (int i = 0; i < l; ++i) o += wbytes8(i);
  return o;
}
constexpr int kWPack8Bytes = woff8(6);
static_assert(kWPack8Bytes == 50688, "packed FP8 weight image size");
static_assert(poff(6) == kRepairParams, "parameter count");
static_assert(mtiles(0) <= kMaxMT, "M tiles per layer");
static_assert(kMaxMT <= kNetThreads / 32, "one issuing warp per M tile");
static_assert(kMaxMT * 128 + 2 * kGW + 2 <= kNPos, "activation buffer reach");
// shared memory of the network kernel: two activation buffers, the weight image,
// bias, FP8 scales, barriers, reductions and calibration maxima
__host__ __device__ constexpr size_t net_smem(bool fp8) {
  return 128 + 2 * (size_t)((fp8 ? 2 : 4) * kNPos * 16) + (fp8 ? kWPack8Bytes : kWPackBytes) + 3 * 6 * 32 * 4 +
         8 * kMaxMT + 4 + 16 * 4 + 6 * 32 * 4 + 64;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t *>(&h);
}
__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

// ---------------------------------------------------------------- weights
// FP32 master (canonical order: per layer W[c_out][3][3][c_in], then b[c_out])
// -> BF16 B-operand images [tap][c_in group][c_out group][8 c_out][8 c_in] with
// zero padding, and biases [6][32].
__global__ void repair_pack_kernel(const float *__restrict__ master, uint16_t *__restrict__ wpack,
                                   float *__restrict__ bias) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < 6 * 32) {
    const int l = e / 32, co = e % 32;
    bias[e] = co < cout(l) ? master[poff(l) + cout(l) * 9 * cin(l) + co] : 0.f;
  }
  if (e >= kWPackBytes / 2) return;
  int l = 0;
  while (l < 5 && e >= woff(l + 1) / 2) ++l;
  const int r = e - woff(l) / 2;
  const int kg = kgroups(l), ng = ngroups(l);
  const int ci8 = r % 8, co8 = (r / 8) % 8, ngi = (r / 64) % ng, kgi = (r / (64 * ng)) % kg, tap = r / (64 * ng * kg);
  const int co = ngi * 8 + co8, ci = kgi * 8 + ci8;
  float v = 0.f;
  if (co < cout(l) && ci < cin(l)) v = master[poff(l) + (co * 9 + tap) * cin(l) + ci];
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  wpack[e] = *reinterpret_cast<const uint16_t *>(&h);
}

// ---------------------------------------------------------------- features
// One block per 16x16 tile; the hole bits of the tile plus an 8-pixel border are
// staged in shared memory and every pixel takes the nearest hole by brute force.
// RGB is the affiliated image after hole classification: the warped colour, or
// at a hole outside the edge strips the method's own fill (gap interpolation,
// else the row/column fill), 0 inside the strips.
__global__ void __launch_bounds__(256) repair_features_kernel(const unsigned long long *__restrict__ warp,
                                                              const uint8_t *__restrict__ cls,
                                                              const float *__restrict__ rgb_aff, int W, int H,
                                                              uint4 *__restrict__ feat) {
  griddep_wait();
  // The distance to the nearest hole, capped at 8, is exact and separable:
  // d^2 = min over rows dy in [-8, 8] of dy^2 + g(dy)^2, with g the distance
  // along that row to its nearest hole within 8 columns. The 32x32 window
  // (tile + 8-pixel halo) is kept as one 32-bit hole mask per row; g comes
  // from the nearest set bit on either side of the column.
  __shared__ uint32_t s_row[32];
  __shared__ uint8_t s_g[32][kRT];  // 9: no hole within 8 columns
  const int tx0 = blockIdx.x * kRT, ty0 = blockIdx.y * kRT;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int r = wid; r < 32; r += 8) {
    const int yy = ty0 - 8 + r, xx = tx0 - 8 + lane;
    const bool h = yy >= 0 && yy < H && xx >= 0 && xx < W && (cls[(size_t)yy * W + xx] & kClsHole);
    const uint32_t m = __ballot_sync(0xffffffffu, h);
    if (lane == 0) s_row[r] = m;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 32 * kRT; i += 256) {
    const int r = i / kRT, c = i % kRT, bit = c + 8;
    const uint32_t m = s_row[r];
    const uint32_t left = m & (0xffffffffu >> (31 - bit));  // columns up to this one
    const uint32_t right = m >> bit;                       // this column and those to the right
    int g = 9;
    if (left) g = min(g, bit - (31 - __clz(left)));
    if (right) g = min(g, __ffs(right) - 1);
    s_g[r][c] = (uint8_t)g;
  }
  __syncthreads();
  const int lx = threadIdx.x & 15, ly = threadIdx.x >> 4;
  const int x = tx0 + lx, y = ty0 + ly;
  if (x >= W || y >= H) return;
  const size_t p = (size_t)y * W + x;
  const unsigned long long k = warp[p];
  const bool hole = k == ~0ull;
  int best = 65;
#pragma unroll
  for (int dy = -8; dy <= 8; ++dy) {
    const int g = s_g[ly + 8 + dy][lx];
    if (g <= 8) best = min(best, dy * dy + g * g);
  }
  const float dist = fminf(sqrtf((float)best), 8.f) * 0.125f;
  const size_t hw = (size_t)W * H;
  const float r = rgb_aff[p], g = rgb_aff[hw + p], b = rgb_aff[2 * hw + p];
  float inv = 0.f;
  if (!hole) {
    const float z = __uint_as_float((uint32_t)(k >> 32));
    inv = isfinite(z) && z > 0.f ? 1.f / z : 0.f;
  }
  feat[p] = make_uint4(pack_bf16(r, g), pack_bf16(b, inv), pack_bf16(hole ? 1.f : 0.f, dist), 0u);
}

// ---------------------------------------------------------------- the network
struct NetArgs {
  const uint4 *feat;         // [frames][H][W] 8 x bf16
  int W, H;
  const uint32_t *tiles;     // frame << 24 | ty << 12 | tx
  const uint32_t *n_tiles;   // device count, or null for n_max
  uint32_t n_max;
  const uint8_t *wpack;      // BF16 or FP8 B-operand images
  const float *bias;         // [6][32]
  const float *sx;           // FP8: [6][32] input scales of every layer
  const float *sw;           // FP8: [6][32] output-channel weight scales
  float *fill;               // [frames][3][H][W], or null
  float *gate;               // [n] mean gate logit per listed tile
  float *out4;               // training: [n][4][16][16] raw outputs, or null
  uint4 *acts;               // training: [n][6 layer inputs][4 groups][kNPos] (16 B each), or null
  uint32_t *amax;            // calibration: [6][32] largest |layer input| (float bits), or null
  uint32_t *status;
};

__device__ __forceinline__ uint32_t e4m3x4(float a, float b, float c, float d) {
  const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
  const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
  return (lo & 0xffffu) | (hi << 16);
}

template <bool FP8>
__global__ void __launch_bounds__(kNetThreads, FP8 ? 2 : 1) repair_net_kernel(NetArgs a) {
  griddep_wait();
  // BF16: 8 channels per 16-byte group, 4 groups, K = 16 per MMA (two per tap);
  // FP8: 16 channels per group, 2 groups, K = 32 per MMA (one per tap)
  constexpr int kChPerGroup = FP8 ? 16 : 8;
  constexpr int kGroups = 32 / kChPerGroup;
  constexpr int kBuf = kGroups * kNPos * 16;
  constexpr int kWBytes = FP8 ? kWPack8Bytes : kWPackBytes;
  extern __shared__ uint8_t s_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)s_raw + 127) & ~(uintptr_t)127);
  uint8_t *bufA = smem;
  uint8_t *bufB = smem + kBuf;
  uint8_t *wsm = smem + 2 * kBuf;
  float *s_bias = (float *)(wsm + kWBytes);
  float *s_sw = s_bias + 6 * 32;        // FP8: weight scales
  float *s_isx = s_sw + 6 * 32;         // FP8: reciprocal input scales
  uint64_t *mbar = (uint64_t *)(s_isx + 6 * 32);  // one per M tile of a layer
  uint32_t *s_taddr = (uint32_t *)(mbar + kMaxMT);
  float *s_red = (float *)(s_taddr + 1);          // [8 warps][2]
  uint32_t *s_amax = (uint32_t *)(s_red + 16);    // [6][32] calibration maxima
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int wq = wid & 3, wg = wid >> 2;  // TMEM lane quarter of the warp; its warpgroup
  const uint32_t n = load_n(a.n_tiles, a.n_max);
  if (blockIdx.x >= n) return;

  // one-time set-up: weights, scales, cleared activation buffers, barriers, TMEM
  {
    const uint4 *src = (const uint4 *)a.wpack;
    uint4 *dst = (uint4 *)wsm;
    for (int i = tid; i < kWBytes / 16; i += kNetThreads) dst[i] = src[i];
    for (int i = tid; i < 6 * 32; i += kNetThreads) {
      s_bias[i] = a.bias[i];
      if (FP8) {
        s_sw[i] = a.sw[i];
        s_isx[i] = 1.f / a.sx[i];
      }
      s_amax[i] = 0u;
    }
    uint4 *z = (uint4 *)smem;
    for (int i = tid; i < 2 * kBuf / 16; i += kNetThreads) z[i] = make_uint4(0, 0, 0, 0);
    if (tid < kMaxMT) umma::mbar_init(mbar + tid, 1);
    if (wid == 0) {
      umma::tmem_alloc(s_taddr, kTmemCols);
      umma::tmem_relinquish();
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
  }
  const uint32_t taddr = *s_taddr;
  const uint32_t sA = umma::smem_u32(bufA), sB = umma::smem_u32(bufB), sW = umma::smem_u32(wsm);
  uint32_t phases = 0;  // bit mt: parity the next completion of mbar[mt] flips to
  bool failed = false;

  for (uint32_t t = blockIdx.x; t < n && !failed; t += gridDim.x) {
    const uint32_t te = a.tiles[t];
    const int frame = (int)(te >> 24), ty0 = (int)((te >> 12) & 0xfffu) * kRT, tx0 = (int)(te & 0xfffu) * kRT;
    const uint4 *fin = a.feat + (size_t)frame * a.W * a.H;
    // layer-1 input: the 28x28 feature window (zeros outside the image); the
    // 6 features + zeros fill channel group 0, the other groups are zero (K padding)
    for (int q = tid; q < kNPos; q += kNetThreads) {
      uint4 v = make_uint4(0, 0, 0, 0);
      if (q < kGW * kGW) {
        const int y = ty0 - kHalo + q / kGW, x = tx0 - kHalo + q % kGW;
        if (y >= 0 && y < a.H && x >= 0 && x < a.W) v = fin[(size_t)y * a.W + x];
      }
      if (a.amax) {
        const float f[6] = {bf16_lo(v.x), bf16_hi(v.x), bf16_lo(v.y), bf16_hi(v.y), bf16_lo(v.z), bf16_hi(v.z)};
        for (int c = 0; c < 6; ++c) atomicMax(&s_amax[c], __float_as_uint(fabsf(f[c])));
      }
      if (FP8) {
        const float *is = s_isx;  // layer-0 input scales
        v = make_uint4(e4m3x4(bf16_lo(v.x) * is[0], bf16_hi(v.x) * is[1], bf16_lo(v.y) * is[2], bf16_hi(v.y) * is[3]),
                       e4m3x4(bf16_lo(v.z) * is[4], bf16_hi(v.z) * is[5], 0.f, 0.f), 0u, 0u);
      }
      ((uint4 *)bufA)[q] = v;
      for (int g = 1; g < kGroups; ++g) ((uint4 *)bufA)[g * kNPos + q] = make_uint4(0, 0, 0, 0);
    }
    float gsum = 0.f, gcnt = 0.f;
#pragma unroll 1
    for (int l = 0; l < 6; ++l) {
      uint8_t *in = (l & 1) ? bufB : bufA;
      uint8_t *out = (l & 1) ? bufA : bufB;
      const uint32_t sin = (l & 1) ? sB : sA;
      const int ng = ngroups(l), N = ng * 8, MT = mtiles(l);
      const int kg = FP8 ? 2 : kgroups(l);  // 16-byte K groups of this layer's input
      // this layer's input (written by all threads) is complete and visible to
      // the tensor core
      umma::fence_proxy_async();
      umma::fence_before_sync();
      __syncthreads();
      umma::fence_after_sync();
      if (!FP8 && a.acts) {  // training: keep this layer's input (read beside the MMAs)
        uint4 *dst = a.acts + ((size_t)t * 6 + l) * 4 * kNPos;
        const uint4 *srcb = (const uint4 *)in;
        for (int i = tid; i < kg * kNPos; i += kNetThreads) dst[i] = srcb[i];
      }
      // lane 0 of warp mt issues the MMAs of M tile mt (the M tiles are issued
      // in parallel) and commits them to barrier mt, so every M tile's epilogue
      // starts as soon as its own accumulator is complete
      if (lane == 0 && wid < MT) {
        const int mt = wid;
        const uint32_t idesc = FP8 ? umma::idesc_e4m3(128, N) : umma::idesc_bf16(128, N);
        const uint32_t wl = sW + (uint32_t)(FP8 ? woff8(l) : woff(l));
        const uint64_t a0 = umma::desc(sin + (uint32_t)(mt * 128 * 16), kNPos * 16, 128);
        const uint64_t b0 = umma::desc(wl, ng * 128, 128);
        const uint32_t d = taddr + (uint32_t)(mt * N);
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
          const int shift = (tap / 3) * kGW + (tap % 3);
          for (int kp = 0; kp < kg / 2; ++kp) {  // two 16-byte groups per MMA
            const uint64_t ad = umma::desc_add(a0, (uint32_t)(((2 * kp) * kNPos + shift) * 16));
            const uint64_t bd = umma::desc_add(b0, (uint32_t)((tap * kg + 2 * kp) * ng * 128));
            if (FP8) umma::mma_e4m3(d, ad, bd, idesc, (tap | kp) != 0 ? 1u : 0u);
            else umma::mma_bf16(d, ad, bd, idesc, (tap | kp) != 0 ? 1u : 0u);
          }
        }
        umma::mma_commit(mbar + mt);
      }
      __syncwarp();
      // epilogue: accumulator rows -> scale, bias, ReLU, border zeroing -> next buffer
      const int shiftL = l + 1;  // this layer's output grid starts (l + 1) pixels in
      bool layer_ok = true;
      for (int mt = 0; mt < MT; ++mt) {
        // warpgroup mt % 2 reads M tile mt; every thread tracks every barrier's phase
        const uint32_t par = (phases >> mt) & 1u;
        phases ^= 1u << mt;
        if ((mt & 1) != wg) continue;
        // the same decision on every lane of the warp (tcgen05.ld is warp-wide)
        const bool ok = __all_sync(0xffffffffu, umma::mbar_wait(mbar + mt, par));
        if (!ok) {
          layer_ok = false;
          break;
        }
        umma::fence_after_sync();
        const int q = mt * 128 + wq * 32 + lane;
        const int r = q / kGW, c = q % kGW;
        const int y = ty0 - kHalo + shiftL + r, x = tx0 - kHalo + shiftL + c;
        const bool inside = y >= 0 && y < a.H && x >= 0 && x < a.W;
        const uint32_t tl = taddr + ((uint32_t)(wq * 32) << 16) + (uint32_t)(mt * N);
        const float *bl = s_bias + l * 32;
        const float *swl = s_sw + l * 32;
        if (l < 5) {
          float v[32];
          float h[16];
          umma::tmem_ld16(tl, h);
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = h[i];
          umma::tmem_ld16(tl + 16, h);
#pragma unroll
          for (int i = 0; i < 16; ++i) v[16 + i] = h[i];
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const float yv = FP8 ? fmaf(v[i], swl[i], bl[i]) : v[i] + bl[i];
            v[i] = inside ? fmaxf(yv, 0.f) : 0.f;
          }
          if (FP8) {
            const float *is = s_isx + (l + 1) * 32;  // next layer's input scales
#pragma unroll
            for (int g = 0; g < 2; ++g) {
              const int o = g * 16;
              ((uint4 *)out)[g * kNPos + q] =
                  make_uint4(e4m3x4(v[o] * is[o], v[o + 1] * is[o + 1], v[o + 2] * is[o + 2], v[o + 3] * is[o + 3]),
                             e4m3x4(v[o + 4] * is[o + 4], v[o + 5] * is[o + 5], v[o + 6] * is[o + 6],
                                    v[o + 7] * is[o + 7]),
                             e4m3x4(v[o + 8] * is[o + 8], v[o + 9] * is[o + 9], v[o + 10] * is[o + 10],
                                    v[o + 11] * is[o + 11]),
                             e4m3x4(v[o + 12] * is[o + 12], v[o + 13] * is[o + 13], v[o + 14] * is[o + 14],
                                    v[o + 15] * is[o + 15]));
            }
          } else {
#pragma unroll
            for (int g = 0; g < 4; ++g) {
              uint32_t w4[4];
#pragma unroll
              for (int j = 0; j < 4; ++j) w4[j] = pack_bf16(v[g * 8 + 2 * j], v[g * 8 + 2 * j + 1]);
              ((uint4 *)out)[g * kNPos + q] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
              if (a.amax && inside && r < kGW - 2 * (l + 1) && c < kGW - 2 * (l + 1)) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                  atomicMax(&s_amax[(l + 1) * 32 + g * 8 + 2 * j], w4[j] << 16);
                  atomicMax(&s_amax[(l + 1) * 32 + g * 8 + 2 * j + 1], w4[j] & 0xffff0000u);
                }
              }
            }
          }
        } else {
          float v[16];
          umma::tmem_ld16(tl, v);
          if (r < kRT && c < kRT) {
            const float o0 = FP8 ? fmaf(v[0], swl[0], bl[0]) : v[0] + bl[0];
            const float o1 = FP8 ? fmaf(v[1], swl[1], bl[1]) : v[1] + bl[1];
            const float o2 = FP8 ? fmaf(v[2], swl[2], bl[2]) : v[2] + bl[2];
            const float o3 = FP8 ? fmaf(v[3], swl[3], bl[3]) : v[3] + bl[3];
            if (a.out4) {
              float *o = a.out4 + (size_t)t * 4 * kRT * kRT + r * kRT + c;
              o[0] = o0;
              o[kRT * kRT] = o1;
              o[2 * kRT * kRT] = o2;
              o[3 * kRT * kRT] = o3;
            }
            if (inside) {
              if (a.fill) {  // the network corrects the method's fill (feature RGB)
                const size_t hw = (size_t)a.W * a.H;
                const uint4 fv = fin[(size_t)y * a.W + x];
                float *f = a.fill + (size_t)frame * 3 * hw + (size_t)y * a.W + x;
                f[0] = bf16_lo(fv.x) + o0;
                f[hw] = bf16_hi(fv.x) + o1;
                f[2 * hw] = bf16_lo(fv.y) + o2;
              }
              gsum += o3;
              gcnt += 1.f;
            }
          }
        }
      }
      umma::fence_before_sync();
      failed = __syncthreads_or(!layer_ok) != 0;  // the same decision on every thread
      if (failed) {
        if (tid == 0) atomicOr(a.status, kStTimeout);
        break;
      }
    }
    if (failed) break;
    // gate logit: mean over the tile's pixels inside the image
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      gsum += __shfl_xor_sync(0xffffffffu, gsum, o);
      gcnt += __shfl_xor_sync(0xffffffffu, gcnt, o);
    }
    if (lane == 0) {
      s_red[wid * 2] = gsum;
      s_red[wid * 2 + 1] = gcnt;
    }
    __syncthreads();
    if (tid == 0) {
      float sm = 0.f, cn = 0.f;
      for (int w = 0; w < kNetThreads / 32; ++w) {
        sm += s_red[2 * w];
        cn += s_red[2 * w + 1];
      }
      a.gate[t] = cn > 0.f ? sm / cn : 0.f;
    }
    __syncthreads();
  }
  umma::fence_before_sync();
  __syncthreads();
  if (a.amax)
    for (int i = tid; i < 6 * 32; i += kNetThreads) atomicMax(&a.amax[i], s_amax[i]);
  if (failed) {
    // MMA batches may still be in flight: give each barrier a bounded chance to
    // complete before the accumulator columns are released
    for (int mt = 0; mt < kMaxMT; ++mt) umma::mbar_wait(mbar + mt, (phases >> mt) & 1u, 1u << 18);
  }
  if (wid == 0) umma::tmem_dealloc(taddr, kTmemCols);
}

// FP8 weights: W' = W * sx (input scales folded in), per output channel
// sw = max |W'| / 448 and codes e4m3(W' / sw) in the B-operand image
// [tap][c_in group of 16][c_out group][8 c_out][16 c_in]. One block per (layer,
// output channel); scales of the layer inputs come from the calibration maxima.
__global__ void __launch_bounds__(256) repair_pack8_kernel(const float *__restrict__ master,
                                                           const uint32_t *__restrict__ amax,
                                                           uint8_t *__restrict__ wpack8, float *__restrict__ sx,
                                                           float *__restrict__ sw) {
  __shared__ float s_max[8];
  const int l = blockIdx.x / 32, co = blockIdx.x % 32;
  const int ci_n = cin(l), ng = ngroups(l);
  if (threadIdx.x < 32 && co == 0) sx[l * 32 + threadIdx.x] = fmaxf(__uint_as_float(amax[l * 32 + threadIdx.x]), 1e-30f) / 448.f;
  float m = 0.f;
  if (co < cout(l))
    for (int i = threadIdx.x; i < 9 * ci_n; i += blockDim.x) {
      const int ci = i % ci_n;
      const float s = fmaxf(__uint_as_float(amax[l * 32 + ci]), 1e-30f) / 448.f;
      m = fmaxf(m, fabsf(master[poff(l) + co * 9 * ci_n + i] * s));
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = m;
  __syncthreads();
  float wmax = 0.f;
  for (int i = 0; i < 8; ++i) wmax = fmaxf(wmax, s_max[i]);
  const float s_w = fmaxf(wmax, 1e-30f) / 448.f;
  if (threadIdx.x == 0) sw[l * 32 + co] = co < cout(l) ? s_w : 1.f;
  if (co >= ng * 8) return;  // beyond the padded output channels
  // this output channel's 9 x 32 codes (zero for padded input channels)
  for (int i = threadIdx.x; i < 9 * 32; i += blockDim.x) {
    const int tap = i / 32, ci = i % 32;
    float v = 0.f;
    if (co < cout(l) && ci < ci_n) {
      const float s = fmaxf(__uint_as_float(amax[l * 32 + ci]), 1e-30f) / 448.f;
      v = master[poff(l) + (co * 9 + tap) * ci_n + ci] * s / s_w;
    }
    const int kgi = ci / 16, ngi = co / 8;
    const size_t byte = (size_t)woff8(l) + ((size_t)((tap * 2 + kgi) * ng + ngi) * 8 + (co % 8)) * 16 + (ci % 16);
    wpack8[byte] = (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
  }
}

// ---------------------------------------------------------------- inference wiring
// Candidate tiles (frame 0): tiles the ROI re-render would redraw that hold a hole
// outside the edge strips. Only there can the gate save work; gap-only tiles
// keep the cheap interpolation, and strip holes show content the dominant eye
// never saw.
__global__ void repair_tile_flags_kernel(const uint8_t *__restrict__ cls, const uint8_t *__restrict__ tile_mask,
                                         int W, int H, uint8_t *__restrict__ flags) {
  griddep_wait();
  const int t = blockIdx.y * gridDim.x + blockIdx.x;
  if (!tile_mask[t]) {
    if (threadIdx.x == 0) flags[t] = 0;
    return;
  }
  const int x = blockIdx.x * kRT + (threadIdx.x & 15), y = blockIdx.y * kRT + (threadIdx.x >> 4);
  bool h = false;
  if (x < W && y < H) {
    const uint8_t c = cls[(size_t)y * W + x];
    h = (c & kClsHole) && !(c & kClsStrip);
  }
  const int any = __syncthreads_or(h);
  if (threadIdx.x == 0) flags[t] = any ? 1 : 0;
}

struct TileFlagLoad {
  const uint8_t *flags;
  __device__ uint32_t operator()(uint32_t i) const { return flags[i]; }
};
struct TileListApply {
  uint32_t *list;
  uint32_t *n_out;
  int tiles_x;
  __device__ void operator()(uint32_t i, uint32_t prefix, uint32_t v) const {
    if (v) list[prefix] = ((i / (uint32_t)tiles_x) << 12) | (i % (uint32_t)tiles_x);
  }
  __device__ void end(uint32_t, uint32_t total) const { *n_out = total; }
};

// Gate >= tau: the tile's hole pixels take the (non-negative) fill, the tile
// leaves the ROI re-render and its pixels are marked as repaired.
__global__ void repair_merge_kernel(const uint32_t *__restrict__ list, const uint32_t *__restrict__ n_list,
                                    const float *__restrict__ gate, float logit_tau,
                                    const unsigned long long *__restrict__ warp, const float *__restrict__ fill,
                                    int W, int H, int tiles_x, float *__restrict__ rgb_aff,
                                    uint8_t *__restrict__ cls, uint8_t *__restrict__ tile_mask) {
  griddep_wait();
  const uint32_t t = blockIdx.x;
  if (t >= *n_list || !(gate[t] >= logit_tau)) return;
  const uint32_t te = list[t];
  const int ty = (int)((te >> 12) & 0xfffu), tx = (int)(te & 0xfffu);
  const int x = tx * kRT + (threadIdx.x & 15), y = ty * kRT + (threadIdx.x >> 4);
  if (threadIdx.x == 0) tile_mask[ty * tiles_x + tx] = 0;
  if (x >= W || y >= H) return;
  const size_t p = (size_t)y * W + x, hw = (size_t)W * H;
  if (warp[p] != ~0ull) return;
  rgb_aff[p] = fmaxf(fill[p], 0.f);
  rgb_aff[hw + p] = fmaxf(fill[hw + p], 0.f);
  rgb_aff[2 * hw + p] = fmaxf(fill[2 * hw + p], 0.f);
  cls[p] |= (uint8_t)kClsNet;
}

// ---------------------------------------------------------------- training
struct TrainArgs {
  const uint4 *feat;       // [frames][H][W]
  const float *target;     // [frames][3][H][W]
  const float *plain;      // [frames][3][H][W]
  int W, H;
  const uint32_t *tiles;
  int n;
  const float *out4;       // [n][4][16][16]
  const float *gate;       // [n]
  float *dy;               // [n][32][kQ] gradient of the current layer's output
  float *dx;               // [n][32][kQ]
  float *tile_stats;       // [n][4]: net MSE, plain MSE, holes, pixels
  float *sums;             // [8]: holes, L1 sum, BCE sum, labels, ...
  float lam;
};

// per tile: squared errors at the tile's hole pixels of the network fill and of
// the plain image, hole and pixel counts (the loss normalisers and the gate
// labels; the warped pixels carry view-dependent colour the features cannot
// see, so the label rates the fill alone)
__global__ void __launch_bounds__(256) repair_stats_kernel(TrainArgs a) {
  const int t = blockIdx.x;
  const uint32_t te = a.tiles[t];
  const int frame = (int)(te >> 24), ty0 = (int)((te >> 12) & 0xfffu) * kRT, tx0 = (int)(te & 0xfffu) * kRT;
  const int r = threadIdx.x >> 4, c = threadIdx.x & 15, y = ty0 + r, x = tx0 + c;
  float en = 0.f, ep = 0.f, nh = 0.f, np_ = 0.f, l1 = 0.f;
  if (y < a.H && x < a.W) {
    const size_t hw = (size_t)a.W * a.H, p = (size_t)y * a.W + x;
    const uint4 f = a.feat[(size_t)frame * hw + p];
    const bool hole = bf16_lo(f.z) > 0.5f;
    const float base[3] = {bf16_lo(f.x), bf16_hi(f.x), bf16_lo(f.y)};
    for (int ch = 0; ch < 3; ++ch) {
      const float tg = a.target[(size_t)frame * 3 * hw + ch * hw + p];
      const float pl = a.plain[(size_t)frame * 3 * hw + ch * hw + p];
      const float fl = base[ch] + a.out4[(size_t)t * 4 * kRT * kRT + ch * kRT * kRT + r * kRT + c];
      if (hole) {
        const float comp = fmaxf(fl, 0.f);
        en += (comp - tg) * (comp - tg);
        ep += (pl - tg) * (pl - tg);
        l1 += fabsf(fl - tg);
      }
    }
    nh = hole ? 1.f : 0.f;
    np_ = 1.f;
  }
  float v[5] = {en, ep, nh, np_, l1};
#pragma unroll
  for (int k = 0; k < 5; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  const int w = threadIdx.x >> 5;
  __shared__ float wred[8][5];
  if ((threadIdx.x & 31) == 0)
    for (int k = 0; k < 5; ++k) wred[w][k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    float s[5] = {0, 0, 0, 0, 0};
    for (int ww = 0; ww < 8; ++ww)
      for (int k = 0; k < 5; ++k) s[k] += wred[ww][k];
    a.tile_stats[t * 4 + 0] = s[2] > 0.f ? s[0] / (3.f * s[2]) : 1.f;  // a tile without holes never passes
    a.tile_stats[t * 4 + 1] = s[2] > 0.f ? s[1] / (3.f * s[2]) : 0.f;
    a.tile_stats[t * 4 + 2] = s[2];
    a.tile_stats[t * 4 + 3] = s[3];
    atomicAdd(&a.sums[0], s[2]);
    atomicAdd(&a.sums[1], s[4]);
  }
}

__device__ __forceinline__ float psnr_of(float mse) { return mse > 0.f ? -10.f * log10f(mse) : 1e9f; }

// dL/d(output) of the last layer on its 28-wide grid (rows < 16, cols < 16)
__global__ void __launch_bounds__(256) repair_dout_kernel(TrainArgs a) {
  const int t = blockIdx.x;
  const uint32_t te = a.tiles[t];
  const int frame = (int)(te >> 24), ty0 = (int)((te >> 12) & 0xfffu) * kRT, tx0 = (int)(te & 0xfffu) * kRT;
  float *dy = a.dy + (size_t)t * 32 * kQ;
  for (int i = threadIdx.x; i < 32 * kQ; i += 256) dy[i] = 0.f;
  __syncthreads();
  const float net_psnr = psnr_of(a.tile_stats[t * 4 + 0]), plain_psnr = psnr_of(a.tile_stats[t * 4 + 1]);
  // positive: the fill reaches 30 dB at the tile's holes and loses at most 0.5 dB
  // against the plain image there (exactly the re-render inside the edge strips,
  // so strip tiles stay negative)
  const float label = (net_psnr >= plain_psnr - 0.5f && net_psnr >= 30.f) ? 1.f : 0.f;
  const float p = 1.f / (1.f + expf(-a.gate[t]));
  const float npx = a.tile_stats[t * 4 + 3];
  const float nh_total = fmaxf(a.sums[0], 1.f);
  const int r = threadIdx.x >> 4, c = threadIdx.x & 15, y = ty0 + r, x = tx0 + c;
  if (threadIdx.x == 0) {
    atomicAdd(&a.sums[2], -(label * logf(p + 1e-12f) + (1.f - label) * logf(1.f - p + 1e-12f)));
    atomicAdd(&a.sums[3], label);
  }
  if (y >= a.H || x >= a.W) return;
  const size_t hw = (size_t)a.W * a.H, pix = (size_t)y * a.W + x;
  const uint4 f = a.feat[(size_t)frame * hw + pix];
  const bool hole = bf16_lo(f.z) > 0.5f;
  const int q = r * kGW + c;
  const float base[3] = {bf16_lo(f.x), bf16_hi(f.x), bf16_lo(f.y)};
  for (int ch = 0; ch < 3; ++ch) {
    const float o = base[ch] + a.out4[(size_t)t * 4 * kRT * kRT + ch * kRT * kRT + r * kRT + c];
    const float tg = a.target[(size_t)frame * 3 * hw + ch * hw + pix];
    const float d = o - tg;
    dy[ch * kQ + q] = hole ? (d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f)) / (3.f * nh_total) : 0.f;
  }
  dy[3 * kQ + q] = a.lam * (p - label) / ((float)a.n * npx);
}

// X_l[ci][p] of tile t from the stored BF16 layer input
__device__ __forceinline__ float act_at(const uint4 *acts, size_t t, int l, int ci, int p) {
  const uint16_t *v = (const uint16_t *)(acts + ((t * 6 + l) * 4 + ci / 8) * kNPos + p);
  return __uint_as_float((uint32_t)v[ci % 8] << 16);
}

// dW[l][co][tap][ci] and db: one block per (tile, co); threads over (tap, ci)
__global__ void __launch_bounds__(288) repair_wgrad_kernel(const uint4 *__restrict__ acts,
                                                           const float *__restrict__ dy, int l, int rows,
                                                           float *__restrict__ grad) {
  const size_t t = blockIdx.x / 32;
  const int co = blockIdx.x % 32;
  if (co >= cout(l)) return;
  const int tap = threadIdx.x / 32, ci = threadIdx.x % 32;
  const float *g = dy + (t * 32 + co) * kQ;
  const int shift = (tap / 3) * kGW + (tap % 3);
  float acc = 0.f, bacc = 0.f;
  if (ci < cin(l)) {
    for (int q = 0; q < rows * kGW; ++q) {
      const float d = g[q];
      if (d != 0.f) acc = fmaf(d, act_at(acts, t, l, ci, q + shift), acc);
    }
    atomicAdd(&grad[poff(l) + (co * 9 + tap) * cin(l) + ci], acc);
  }
  if (threadIdx.x == 0) {
    for (int q = 0; q < rows * kGW; ++q) bacc += g[q];
    atomicAdd(&grad[poff(l) + cout(l) * 9 * cin(l) + co], bacc);
  }
}

// dX of layer l's input (= layer l-1's output) on its valid window, times the
// ReLU derivative (the stored activation is 0 where ReLU or the border cut it)
__global__ void __launch_bounds__(256) repair_dgrad_kernel(const uint4 *__restrict__ acts,
                                                           const float *__restrict__ dy,
                                                           const float *__restrict__ master, int l, int rows_out,
                                                           int n, float *__restrict__ dx) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t total = (size_t)n * 32 * kQ;
  if (i >= total) return;
  const size_t t = i / (32 * kQ);
  const int ci = (int)((i / kQ) % 32), p = (int)(i % kQ);
  const int valid = kGW - 2 * l;  // layer l's input window edge
  const int r = p / kGW, c = p % kGW;
  float s = 0.f;
  if (ci < cin(l) && r < valid && c < valid && act_at(acts, t, l, ci, p) > 0.f) {
    const float *w = master + poff(l);
    for (int tap = 0; tap < 9; ++tap) {
      const int qr = r - tap / 3, qc = c - tap % 3;
      if (qr < 0 || qc < 0 || qr >= rows_out || qc >= kGW - 2 * (l + 1)) continue;
      const int q = qr * kGW + qc;
      for (int co = 0; co < cout(l); ++co) s = fmaf(w[(co * 9 + tap) * cin(l) + ci], dy[(t * 32 + co) * kQ + q], s);
    }
  }
  dx[i] = s;
}

__global__ void repair_adamw_kernel(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                                    float *__restrict__ v, int n, float lr, float b1, float b2, float eps, float wd,
                                    float bc1, float bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
  const float vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * ((mi / bc1) / (sqrtf(vi / bc2) + eps) + wd * w[i]);
}

}  // namespace

size_t repair_act_bytes_per_tile() { return (size_t)6 * 4 * kNPos * 16; }
size_t repair_train_scratch_bytes(int n_tiles) {
  const size_t n = (size_t)(n_tiles > 0 ? n_tiles : 1);
  return n * (repair_act_bytes_per_tile() + 4 * kRT * kRT * 4 + 4 + 2 * 32 * kQ * 4 + 16) + 64 + 1024;
}

cudaError_t prepare_repair() {
  cudaError_t e = cudaFuncSetAttribute(repair_net_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)net_smem(false));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(repair_net_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)net_smem(true));
  return e;
}

cudaError_t repair_pack(const Workspace &ws, cudaStream_t s) {
  repair_pack_kernel<<<(kWPackBytes / 2 + 255) / 256, 256, 0, s>>>(ws.rp_master, (uint16_t *)ws.rp_wpack,
                                                                   ws.rp_bias);
  GS_LAUNCHED(1);
  return cudaGetLastError();
}

cudaError_t repair_features(const Workspace &ws, int W, int H, const float *rgb_aff, uint4 *feat, cudaStream_t s) {
  const dim3 grid((W + kRT - 1) / kRT, (H + kRT - 1) / kRT);
  launch_k(repair_features_kernel, grid, 256, 0, s, ws.warpbuf, ws.cls, rgb_aff, W, H, feat);
  GS_LAUNCHED(1);
  return cudaGetLastError();
}

static int net_grid(uint32_t n_max) {
  const uint32_t sms = (uint32_t)sm_grid_cap(1);
  return (int)(n_max < sms ? (n_max < 1u ? 1u : n_max) : sms);
}

cudaError_t repair_forward(const Workspace &ws, const uint4 *feat, int W, int H, const uint32_t *tiles,
                           const uint32_t *n_ptr, uint32_t n_max, float *fill, float *gate, float *out4,
                           uint4 *acts, cudaStream_t s, bool fp8, uint32_t *amax) {
  if (n_max == 0) return cudaSuccess;
  NetArgs a;
  a.feat = feat;
  a.W = W;
  a.H = H;
  a.tiles = tiles;
  a.n_tiles = n_ptr;
  a.n_max = n_max;
  a.wpack = fp8 ? ws.rp_wpack8 : ws.rp_wpack;
  a.bias = ws.rp_bias;
  a.sx = ws.rp_sx;
  a.sw = ws.rp_sw;
  a.fill = fill;
  a.gate = gate;
  a.out4 = out4;
  a.acts = acts;
  a.amax = amax;
  a.status = &ws.ctr->status;
  if (fp8) {  // two CTAs per SM fit the FP8 kernel's shared memory
    const uint32_t g = n_max < 304u ? (n_max < 1u ? 1u : n_max) : 304u;
    launch_k(repair_net_kernel<true>, g, kNetThreads, net_smem(true), s, a);
  } else {
    launch_k(repair_net_kernel<false>, net_grid(n_max), kNetThreads, net_smem(false), s, a);
  }
  GS_LAUNCHED(1);
  return cudaGetLastError();
}

cudaError_t repair_calibrate_fp8(const Workspace &ws, const uint4 *feat, int W, int H, const uint32_t *tiles,
                                 uint32_t n_tiles, float *gate_scratch, cudaStream_t s) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(ws.rp_amax, 0, 6 * 32 * sizeof(uint32_t), s)) != cudaSuccess) return e;
  if ((e = repair_forward(ws, feat, W, H, tiles, nullptr, n_tiles, nullptr, gate_scratch, nullptr, nullptr, s, false,
                          ws.rp_amax)) != cudaSuccess)
    return e;
  if ((e = cudaMemsetAsync(ws.rp_wpack8, 0, kWPack8Bytes, s)) != cudaSuccess) return e;
  repair_pack8_kernel<<<6 * 32, 256, 0, s>>>(ws.rp_master, ws.rp_amax, ws.rp_wpack8, ws.rp_sx, ws.rp_sw);
  GS_LAUNCHED(1);
  return cudaGetLastError();
}

cudaError_t repair_stereo(const Workspace &ws, int W, int H, float gate_tau, float *rgb_aff, cudaStream_t s,
                          bool fp8) {
  cudaError_t e;
  const int tx = (W + kRT - 1) / kRT, ty = (H + kRT - 1) / kRT, nt = tx * ty;
  launch_k(repair_tile_flags_kernel, dim3(tx, ty), 256, 0, s, ws.cls, ws.tile_mask, W, H, ws.rp_flags);
  GS_LAUNCHED(1);
  if ((e = scan_launch(TileFlagLoad{ws.rp_flags}, TileListApply{ws.rp_list, ws.rp_nlist, tx},
                       (const uint32_t *)nullptr, (uint32_t)nt, ws.bin[0].scan_tiles, ws.bin[0].scan_ticket, &ws.ctr->status, s)) !=
      cudaSuccess)
    return e;
  if ((e = repair_forward(ws, ws.rp_feat, W, H, ws.rp_list, ws.rp_nlist, (uint32_t)nt, ws.rp_fill, ws.rp_gate,
                          nullptr, nullptr, s, fp8, nullptr)) != cudaSuccess)
    return e;
  // sigmoid(g) >= tau  <=>  g >= log(tau / (1 - tau))
  const float tau = fminf(fmaxf(gate_tau, 1e-6f), 1.f - 1e-6f);
  const float logit_tau = logf(tau / (1.f - tau));
  launch_k(repair_merge_kernel, nt, 256, 0, s, ws.rp_list, ws.rp_nlist, ws.rp_gate, logit_tau, ws.warpbuf, ws.rp_fill, W, H,
                                         tx, rgb_aff, ws.cls, ws.tile_mask);
  GS_LAUNCHED(1);
  return cudaGetLastError();
}

cudaError_t repair_train_step(const Workspace &ws, const RepairBatch &b, const RepairOpt &o, float *host_loss,
                              cudaStream_t s) {
  cudaError_t e;
  const int n = b.n_tiles;
  uint8_t *p = (uint8_t *)(((uintptr_t)b.scratch + 255) & ~(uintptr_t)255);
  uint4 *acts = (uint4 *)p;
  p += (size_t)n * repair_act_bytes_per_tile();
  float *out4 = (float *)p;
  p += (size_t)n * 4 * kRT * kRT * 4;
  float *gate = (float *)p;
  p += ((size_t)n * 4 + 255) / 256 * 256;
  float *dy = (float *)p;
  p += (size_t)n * 32 * kQ * 4;
  float *dx = (float *)p;
  p += (size_t)n * 32 * kQ * 4;
  float *stats = (float *)p;
  p += ((size_t)n * 16 + 255) / 256 * 256;
  float *sums = (float *)p;
  if ((e = cudaMemsetAsync(sums, 0, 8 * sizeof(float), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(ws.rp_grad, 0, kRepairParams * sizeof(float), s)) != cudaSuccess) return e;
  if ((e = repair_forward(ws, b.feat, b.W, b.H, b.tiles, nullptr, (uint32_t)n, nullptr, gate, out4, acts, s, false,
                          nullptr)) != cudaSuccess)
    return e;
  TrainArgs a;
  a.feat = b.feat;
  a.target = b.target;
  a.plain = b.plain;
  a.W = b.W;
  a.H = b.H;
  a.tiles = b.tiles;
  a.n = n;
  a.out4 = out4;
  a.gate = gate;
  a.dy = dy;
  a.dx = dx;
  a.tile_stats = stats;
  a.sums = sums;
  a.lam = o.gate_weight;
  repair_stats_kernel<<<n, 256, 0, s>>>(a);
  repair_dout_kernel<<<n, 256, 0, s>>>(a);
  GS_LAUNCHED(2);
  float *cur = dy, *nxt = dx;
  for (int l = 5; l >= 0; --l) {
    const int rows_out = kGW - 2 * (l + 1);  // this layer's valid output rows
    repair_wgrad_kernel<<<n * 32, 288, 0, s>>>(acts, cur, l, rows_out, ws.rp_grad);
    GS_LAUNCHED(1);
    if (l > 0) {
      const size_t total = (size_t)n * 32 * kQ;
      repair_dgrad_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(acts, cur, ws.rp_master, l, rows_out, n,
                                                                          nxt);
      GS_LAUNCHED(1);
      float *tmp = cur;
      cur = nxt;
      nxt = tmp;
    }
  }
  if (o.lr > 0.f) {
    repair_adamw_kernel<<<(kRepairParams + 255) / 256, 256, 0, s>>>(
        ws.rp_master, ws.rp_grad, ws.rp_m, ws.rp_v, kRepairParams, o.lr, o.beta1, o.beta2, o.eps, o.weight_decay,
        1.f - powf(o.beta1, (float)o.step), 1.f - powf(o.beta2, (float)o.step));
    GS_LAUNCHED(1);
    if ((e = repair_pack(ws, s)) != cudaSuccess) return e;
  }
  if (host_loss) {
    float h[8];
    if ((e = cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    const float nh = fmaxf(h[0], 1.f);
    host_loss[0] = h[1] / (3.f * nh) + o.gate_weight * h[2] / (float)n;  // total loss
    host_loss[1] = h[1] / (3.f * nh);                                     // L1 on holes
    host_loss[2] = h[2] / (float)n;                                       // gate BCE
    host_loss[3] = h[3] / (float)n;                                       // share of positive labels
  }
  return cudaGetLastError();
}

}  // namespace gs
