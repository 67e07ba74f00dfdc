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
// loss kernel, and per layer (last to first) one backward kernel on the tensor
// cores: the input gradient is the full convolution of the output gradient with
// the flipped, transposed weights (the forward's implicit GEMM with another
// weight image and the ReLU derivative in the epilogue), and the weight
// gradient is a GEMM over positions per 3x3 tap (M = c_out, N = c_in, K = the
// tile's positions, the tap again a shift of an operand's start address),
// accumulated in tensor memory over all tiles a CTA takes; the CTAs' partial
// sums are reduced in a fixed order (no atomics, so a step is deterministic).
// AdamW updates the FP32 master weights.
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
// backward: the input gradient of layer l (l >= 1) convolves dY_l, stored kDPad
// positions later in shared memory, with the flipped transposed weights
// W'[tap'][c_out group][c_in group][8 c_in][8 c_out] (W' at tap' = W at 8 - tap')
constexpr int kDPad = 2 * kGW + 2;
__host__ __device__ constexpr int kgd(int l) { return l == 5 ? 2 : 4; }  // c_out groups, padded to K = 16
__host__ __device__ constexpr int wbytesT(int l) { return l == 0 ? 0 : 9 * kgd(l) * 4 * 128; }
__host__ __device__ constexpr int woffT(int l) {
  int o = 0;
  for (int i = 1; i < l; ++i) o += wbytesT(i);
  return o;
}
constexpr int kWPackTBytes = woffT(6);
static_assert(kWPackTBytes == 82944, "packed transposed weight image size");
__host__ __device__ constexpr int vrows(int l) { return kGW - 2 * (l + 1); }            // layer l's output edge
__host__ __device__ constexpr int kchunks(int l) { return (vrows(l) * kGW + 15) / 16; }  // weight-gradient K = 16 steps
constexpr int kBwdThreads = 256;
constexpr int kBwdTmemCols = 512;   // 9 taps x 32 (weight gradient) + 6 M tiles x 32 (input gradient)
constexpr int kBufT = (kchunks(0) + 2) * 1024;  // dY^T, plus the reach of the padded A rows
constexpr int kBwdParts = 32 * 9 * 32 + 32;     // largest layer: weight and bias gradients
static_assert(9 * 32 + kMaxMT * 32 <= kBwdTmemCols, "tensor memory of the backward");
static_assert(kchunks(0) * 16 + 2 * kGW + 2 <= kNPos && kMaxMT * 128 + 2 * kGW + 2 <= kNPos,
              "backward operand reach");
__host__ __device__ constexpr size_t bwd_smem() {
  return 128 + 2 * (size_t)(4 * kNPos * 16) + kBufT + wbytesT(1) + (8 * 32 + 32) * 4 + 2 * 8 + 16;
}
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

// FP32 master -> the backward's BF16 images of layers 1-5 (see kDPad): element
// [tap'][c_out group][c_in group][8 c_in][8 c_out] = W[c_out][8 - tap'][c_in].
__global__ void repair_packT_kernel(const float *__restrict__ master, uint16_t *__restrict__ wpackT) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kWPackTBytes / 2) return;
  int l = 1;
  while (l < 5 && e >= woffT(l + 1) / 2) ++l;
  const int r = e - woffT(l) / 2;
  const int kg = kgd(l);
  const int co8 = r % 8, ci8 = (r / 8) % 8, ngi = (r / 64) % 4, kgi = (r / 256) % kg, tp = r / (256 * kg);
  const int co = kgi * 8 + co8, ci = ngi * 8 + ci8, tap = 8 - tp;
  float v = 0.f;
  if (co < cout(l) && ci < cin(l)) v = master[poff(l) + (co * 9 + tap) * cin(l) + ci];
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  wpackT[e] = *reinterpret_cast<const uint16_t *>(&h);
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
// never saw. One CTA per 16x16 tile appends its tile to the list (in no fixed
// order: a tile's network output and gate depend on that tile's pixels only)
// and clears the tile's skip flag.
__global__ void repair_tile_list_kernel(const uint8_t *__restrict__ cls, const uint8_t *__restrict__ tile_mask,
                                        int W, int H, uint32_t *__restrict__ list, uint32_t *__restrict__ n_list,
                                        uint8_t *__restrict__ skip) {
  griddep_wait();
  const int t = blockIdx.y * gridDim.x + blockIdx.x;
  if (skip && threadIdx.x == 0) skip[t] = 0;
  if (!tile_mask[t]) return;  // CTA-uniform
  const int x = blockIdx.x * kRT + (threadIdx.x & 15), y = blockIdx.y * kRT + (threadIdx.x >> 4);
  bool h = false;
  if (x < W && y < H) {
    const uint8_t c = cls[(size_t)y * W + x];
    h = (c & kClsHole) && !(c & kClsStrip);
  }
  if (__syncthreads_or(h) && threadIdx.x == 0)
    list[atomicAdd(n_list, 1u)] = ((uint32_t)blockIdx.y << 12) | (uint32_t)blockIdx.x;
}

// Gate >= tau: the tile's hole pixels take the (non-negative) fill, the tile
// leaves the ROI re-render and its pixels are marked as repaired.
__global__ void repair_merge_kernel(const uint32_t *__restrict__ list, const uint32_t *__restrict__ n_list,
                                    const float *__restrict__ gate, float logit_tau,
                                    const unsigned long long *__restrict__ warp, const float *__restrict__ fill,
                                    int W, int H, int tiles_x, float *__restrict__ rgb_aff,
                                    uint8_t *__restrict__ cls, uint8_t *__restrict__ tile_mask,
                                    uint8_t *__restrict__ skip) {
  griddep_wait();
  const uint32_t t = blockIdx.x;
  if (t >= *n_list || !(gate[t] >= logit_tau)) return;
  const uint32_t te = list[t];
  const int ty = (int)((te >> 12) & 0xfffu), tx = (int)(te & 0xfffu);
  const int x = tx * kRT + (threadIdx.x & 15), y = ty * kRT + (threadIdx.x >> 4);
  if (threadIdx.x == 0) {
    if (skip) skip[ty * tiles_x + tx] = 1;
    else tile_mask[ty * tiles_x + tx] = 0;
  }
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
  uint4 *dy;               // [n][4 groups][kNPos] BF16 gradient of the last layer's output
  float *tile_stats;       // [n][8]: net MSE, plain MSE, holes, pixels, L1 sum, BCE, label
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
    a.tile_stats[t * 8 + 0] = s[2] > 0.f ? s[0] / (3.f * s[2]) : 1.f;  // a tile without holes never passes
    a.tile_stats[t * 8 + 1] = s[2] > 0.f ? s[1] / (3.f * s[2]) : 0.f;
    a.tile_stats[t * 8 + 2] = s[2];
    a.tile_stats[t * 8 + 3] = s[3];
    a.tile_stats[t * 8 + 4] = s[4];
  }
}

// sums[s0] and sums[s0 + 1] = the sums over tiles of tile_stats[t][fa] and
// [t][fb], in a fixed order (one block: thread i takes tiles i, i + 1024, ...,
// then a tree), so a training step's loss terms do not depend on scheduling.
__global__ void __launch_bounds__(1024) repair_sums_kernel(const float *__restrict__ tile_stats, int n, int fa, int fb,
                                                           float *__restrict__ sums, int s0) {
  __shared__ float red[1024];
  for (int k = 0; k < 2; ++k) {
    const int f = k ? fb : fa;
    float v = 0.f;
    for (int t = threadIdx.x; t < n; t += 1024) v += tile_stats[t * 8 + f];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
      if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) sums[s0 + k] = red[0];
    __syncthreads();
  }
}

__device__ __forceinline__ float psnr_of(float mse) { return mse > 0.f ? -10.f * log10f(mse) : 1e9f; }

// dL/d(output) of the last layer on its 28-wide grid (rows < 16, cols < 16), as
// the BF16 operand of the backward: channel group 0 holds the 4 outputs, the
// other groups and every other position are zero
__global__ void __launch_bounds__(256) repair_dout_kernel(TrainArgs a) {
  const int t = blockIdx.x;
  const uint32_t te = a.tiles[t];
  const int frame = (int)(te >> 24), ty0 = (int)((te >> 12) & 0xfffu) * kRT, tx0 = (int)(te & 0xfffu) * kRT;
  uint4 *dy = a.dy + (size_t)t * 4 * kNPos;
  const float net_psnr = psnr_of(a.tile_stats[t * 8 + 0]), plain_psnr = psnr_of(a.tile_stats[t * 8 + 1]);
  // positive: the fill reaches 30 dB at the tile's holes and loses at most 0.5 dB
  // against the plain image there (exactly the re-render inside the edge strips,
  // so strip tiles stay negative)
  const float label = (net_psnr >= plain_psnr - 0.5f && net_psnr >= 30.f) ? 1.f : 0.f;
  const float p = 1.f / (1.f + expf(-a.gate[t]));
  const float npx = a.tile_stats[t * 8 + 3];
  const float nh_total = fmaxf(a.sums[0], 1.f);
  if (threadIdx.x == 0) {
    a.tile_stats[t * 8 + 5] = -(label * logf(p + 1e-12f) + (1.f - label) * logf(1.f - p + 1e-12f));
    a.tile_stats[t * 8 + 6] = label;
  }
  const size_t hw = (size_t)a.W * a.H;
  for (int q = threadIdx.x; q < kNPos; q += blockDim.x) {
    float g[4] = {0.f, 0.f, 0.f, 0.f};
    const int r = q / kGW, c = q % kGW, y = ty0 + r, x = tx0 + c;
    if (r < kRT && c < kRT && y < a.H && x < a.W) {
      const size_t pix = (size_t)y * a.W + x;
      const uint4 f = a.feat[(size_t)frame * hw + pix];
      const bool hole = bf16_lo(f.z) > 0.5f;
      const float base[3] = {bf16_lo(f.x), bf16_hi(f.x), bf16_lo(f.y)};
      for (int ch = 0; ch < 3; ++ch) {
        const float o = base[ch] + a.out4[(size_t)t * 4 * kRT * kRT + ch * kRT * kRT + r * kRT + c];
        const float d = o - a.target[(size_t)frame * 3 * hw + ch * hw + pix];
        g[ch] = hole ? (d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f)) / (3.f * nh_total) : 0.f;
      }
      g[3] = a.lam * (p - label) / ((float)a.n * npx);
    }
    dy[q] = make_uint4(pack_bf16(g[0], g[1]), pack_bf16(g[2], g[3]), 0u, 0u);
    for (int grp = 1; grp < 4; ++grp) dy[grp * kNPos + q] = make_uint4(0u, 0u, 0u, 0u);
  }
}

// ---------------------------------------------------------------- backward
struct BwdArgs {
  const uint4 *acts;       // [n][6][4 groups][kNPos]: every layer's BF16 input (forward)
  const uint4 *dy;         // [n][4][kNPos]: BF16 dL/d(output of layer l), zero outside its window
  uint4 *dyo;              // [n][4][kNPos]: BF16 dL/d(output of layer l - 1) (l >= 1)
  const uint8_t *wpackT;   // the transposed image of layer l
  float *part;             // [gridDim][cout(l) * 9 * cin(l) + cout(l)] weight and bias gradients per CTA
  int l, n;
  uint32_t *status;
};

// One layer of the backward pass on the tensor cores; a CTA takes tiles
// blockIdx.x, + gridDim.x, ... Per tile:
//   weight gradient: for each tap, D_tap[c_out][c_in] += sum over positions q of
//     dY[c_out][q] x[c_in][q + shift(tap)]: A = dY^T (K-major, K = positions,
//     M = 128 rows of which the first c_out are real; the other rows read the next
//     positions' data and are never used), B = x shifted (MN-major: the 8 c_in of a
//     position are contiguous), 16 positions per MMA. D_tap stays in tensor
//     memory across the CTA's tiles and goes to the CTA's partial sums at the end.
//   input gradient (l >= 1): dX[p][c_in] = sum over tap', c_out of dY[c_out]
//     [p + shift(tap') - kDPad] W[c_out][8 - tap'][c_in] (the forward's implicit
//     GEMM on dY stored kDPad positions later), times the ReLU derivative (the
//     stored input x > 0) inside layer l's input window, stored as BF16 dY of
//     layer l - 1.
// Warp 0 issues the weight-gradient MMAs, warp 1 the input-gradient MMAs, each
// committing to its own barrier; every wait is bounded.
__global__ void __launch_bounds__(kBwdThreads, 1) repair_bwd_kernel(BwdArgs a) {
  extern __shared__ uint8_t s_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)s_raw + 127) & ~(uintptr_t)127);
  constexpr int kBuf = 4 * kNPos * 16;
  uint8_t *bufD = smem;              // dY at positions + kDPad: input-gradient A
  uint8_t *bufX = smem + kBuf;       // x_l: weight-gradient B, ReLU derivative
  uint8_t *bufT = smem + 2 * kBuf;   // dY^T [8-position group][c_out group][8 c_out][8 positions]
  uint8_t *wsm = bufT + kBufT;
  float *s_part = (float *)(wsm + wbytesT(1));  // [8 warps][32]
  float *s_db = s_part + 8 * 32;                // [32] bias gradient over the CTA's tiles
  uint64_t *mbar = (uint64_t *)(s_db + 32);     // weight gradient, input gradient
  uint32_t *s_taddr = (uint32_t *)(mbar + 2);
  const int l = a.l;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int wq = wid & 3, wg = wid >> 2;
  const int ci_n = cin(l), co_n = cout(l);
  const int NW = l == 0 ? 16 : 32;            // weight-gradient N: c_in padded to 16
  const int nK = kchunks(l);
  const int MT = l > 0 ? mtiles(l - 1) : 0;   // input-gradient M tiles: layer l's input window
  const int vin = kGW - 2 * l, vout = vrows(l);
  const int kg = kgd(l);
  constexpr uint32_t kColG = 9 * 32;          // first input-gradient column
  {
    if (l > 0) {
      const uint4 *src = (const uint4 *)(a.wpackT + woffT(l));
      for (int i = tid; i < wbytesT(l) / 16; i += kBwdThreads) ((uint4 *)wsm)[i] = src[i];
    }
    for (int i = tid; i < kBuf / 16; i += kBwdThreads) ((uint4 *)bufD)[i] = make_uint4(0, 0, 0, 0);
    for (int i = tid; i < kBufT / 16; i += kBwdThreads) ((uint4 *)bufT)[i] = make_uint4(0, 0, 0, 0);
    if (tid < 32) s_db[tid] = 0.f;
    if (tid < 2) umma::mbar_init(mbar + tid, 1);
    if (wid == 0) {
      umma::tmem_alloc(s_taddr, kBwdTmemCols);
      umma::tmem_relinquish();
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
  }
  const uint32_t taddr = *s_taddr;
  const uint32_t sD = umma::smem_u32(bufD), sX = umma::smem_u32(bufX), sT = umma::smem_u32(bufT),
                 sW = umma::smem_u32(wsm);
  uint32_t ph_w = 0, ph_g = 0;
  bool failed = false, any = false;
  for (int t = blockIdx.x; t < a.n && !failed; t += gridDim.x) {
    // operands of this tile (the previous tile's MMAs have completed)
    const uint4 *xs = a.acts + ((size_t)t * 6 + l) * 4 * kNPos;
    for (int i = tid; i < 4 * kNPos; i += kBwdThreads) ((uint4 *)bufX)[i] = xs[i];
    const uint4 *ds = a.dy + (size_t)t * 4 * kNPos;
    for (int i = tid; i < 4 * nK * 16; i += kBwdThreads) {
      const int g = i / (nK * 16), q = i % (nK * 16);
      ((uint4 *)bufD)[g * kNPos + kDPad + q] = ds[g * kNPos + q];
    }
    // dY^T: every 8-position x 8-channel block transposed through registers
    for (int i = tid; i < 2 * nK * 4; i += kBwdThreads) {
      const int pg = i >> 2, g = i & 3;
      uint32_t m[8][4];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const uint4 v = ds[g * kNPos + pg * 8 + j];
        m[j][0] = v.x; m[j][1] = v.y; m[j][2] = v.z; m[j][3] = v.w;
      }
      uint4 *dst = (uint4 *)(bufT + pg * 512 + g * 128);
#pragma unroll
      for (int c = 0; c < 8; ++c) {  // row c: channel c at the 8 positions
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint32_t lo = (m[2 * j][c >> 1] >> ((c & 1) * 16)) & 0xffffu;
          const uint32_t hi = (m[2 * j + 1][c >> 1] >> ((c & 1) * 16)) & 0xffffu;
          w[j] = lo | (hi << 16);
        }
        dst[c] = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
    umma::fence_proxy_async();
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    if (lane == 0 && wid == 0) {  // weight gradient: 9 taps x nK MMAs
      const uint32_t idesc = umma::idesc_bf16(128, NW) | (1u << 16);  // B MN-major
#pragma unroll 1
      for (int tap = 0; tap < 9; ++tap) {
        const int shift = (tap / 3) * kGW + (tap % 3);
        for (int kc = 0; kc < nK; ++kc) {
          const uint64_t ad = umma::desc(sT + (uint32_t)(kc * 1024), 512, 128);
          const uint64_t bd = umma::desc(sX + (uint32_t)((kc * 16 + shift) * 16), 128, kNPos * 16);
          umma::mma_bf16(taddr + (uint32_t)(tap * NW), ad, bd, idesc, (any || kc > 0) ? 1u : 0u);
        }
      }
      umma::mma_commit(mbar + 0);
    }
    if (lane == 0 && wid == 1 && l > 0) {  // input gradient: MT tiles x 9 taps x kg / 2 MMAs
      const uint32_t idesc = umma::idesc_bf16(128, 32);
      const uint64_t b0 = umma::desc(sW, 4 * 128, 128);
      for (int mt = 0; mt < MT; ++mt) {
        const uint64_t a0 = umma::desc(sD + (uint32_t)(mt * 128 * 16), kNPos * 16, 128);
        const uint32_t d = taddr + kColG + (uint32_t)(mt * 32);
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
          const int shift = (tap / 3) * kGW + (tap % 3);
          for (int kp = 0; kp < kg / 2; ++kp) {
            const uint64_t ad = umma::desc_add(a0, (uint32_t)(((2 * kp) * kNPos + shift) * 16));
            const uint64_t bd = umma::desc_add(b0, (uint32_t)((tap * kg + 2 * kp) * 4 * 128));
            umma::mma_bf16(d, ad, bd, idesc, (tap | kp) != 0 ? 1u : 0u);
          }
        }
      }
      umma::mma_commit(mbar + 1);
    }
    __syncwarp();
    any = true;
    // bias gradient: sum of dY over the output window (fixed order per tile)
    {
      const int co = lane;
      float sum = 0.f;
      if (co < co_n) {
        const uint16_t *col = (const uint16_t *)(bufD + (co >> 3) * kNPos * 16) + (co & 7);
        for (int q = wid; q < vout * kGW; q += 8) sum += __uint_as_float((uint32_t)col[(kDPad + q) * 8] << 16);
      }
      s_part[wid * 32 + co] = sum;
    }
    __syncthreads();
    if (tid < 32) {
      float sum = 0.f;
#pragma unroll
      for (int w = 0; w < 8; ++w) sum += s_part[w * 32 + tid];
      s_db[tid] += sum;
    }
    bool ok = true;
    if (l > 0) {
      ok = __all_sync(0xffffffffu, umma::mbar_wait(mbar + 1, ph_g));
      ph_g ^= 1u;
      umma::fence_after_sync();
      uint4 *dout = a.dyo + (size_t)t * 4 * kNPos;
      for (int mt = wg; mt < MT && ok; mt += 2) {
        const int q = mt * 128 + wq * 32 + lane;
        const int r = q / kGW, c = q % kGW;
        const bool win = r < vin && c < vin;
        const uint32_t tl = taddr + ((uint32_t)(wq * 32) << 16) + kColG + (uint32_t)(mt * 32);
        float v[32], h[16];
        umma::tmem_ld16(tl, h);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = h[i];
        umma::tmem_ld16(tl + 16, h);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[16 + i] = h[i];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          const uint4 xv = ((const uint4 *)bufX)[g * kNPos + q];
          const uint32_t xw[4] = {xv.x, xv.y, xv.z, xv.w};
          uint32_t w4[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float m0 = (win && bf16_lo(xw[j]) > 0.f) ? 1.f : 0.f;
            const float m1 = (win && bf16_hi(xw[j]) > 0.f) ? 1.f : 0.f;
            w4[j] = pack_bf16(v[g * 8 + 2 * j] * m0, v[g * 8 + 2 * j + 1] * m1);
          }
          dout[g * kNPos + q] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
        }
      }
      for (int i = tid; i < 4 * (kNPos - MT * 128); i += kBwdThreads) {
        const int g = i / (kNPos - MT * 128), q = MT * 128 + i % (kNPos - MT * 128);
        dout[g * kNPos + q] = make_uint4(0, 0, 0, 0);
      }
    }
    // the weight-gradient MMAs read bufT and bufX: wait before the next tile
    ok = __all_sync(0xffffffffu, umma::mbar_wait(mbar + 0, ph_w)) && ok;
    ph_w ^= 1u;
    umma::fence_before_sync();
    failed = __syncthreads_or(!ok) != 0;
    umma::fence_after_sync();
  }
  if (failed) {
    if (tid == 0) atomicOr(a.status, kStTimeout);
    for (int k = 0; k < 2; ++k) umma::mbar_wait(mbar + k, k ? ph_g : ph_w, 1u << 18);
  } else if (wid == 0) {
    // weight gradient of the CTA's tiles: TMEM lane = c_out, column = tap * NW + c_in
    const int npar = co_n * 9 * ci_n;
    float *part = a.part + (size_t)blockIdx.x * (npar + co_n);
    const int co = lane;
#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap) {
      for (int c16 = 0; c16 < NW / 16; ++c16) {
        float h[16];
        if (any) {
          umma::tmem_ld16(taddr + (uint32_t)(tap * NW + c16 * 16), h);
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) h[i] = 0.f;
        }
        if (co < co_n)
          for (int i = 0; i < 16; ++i) {
            const int ci = c16 * 16 + i;
            if (ci < ci_n) part[(co * 9 + tap) * ci_n + ci] = h[i];
          }
      }
    }
    if (co < co_n) part[npar + co] = s_db[co];
  }
  umma::fence_before_sync();
  __syncthreads();
  if (wid == 0) umma::tmem_dealloc(taddr, kBwdTmemCols);
}

// grad[i] = sum over CTAs (in order) of the partials: deterministic
__global__ void repair_reduce_kernel(const float *__restrict__ part, int n_parts, int count, float *__restrict__ grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  float sum = 0.f;
  for (int k = 0; k < n_parts; ++k) sum += part[(size_t)k * count + i];
  grad[i] = sum;
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
static int bwd_grid(int n) {
  const int sms = sm_grid_cap(1);
  return n < sms ? (n < 1 ? 1 : n) : sms;
}
size_t repair_train_scratch_bytes(int n_tiles) {
  const size_t n = (size_t)(n_tiles > 0 ? n_tiles : 1);
  // activations, raw outputs, gate, two BF16 gradient buffers, tile stats, the
  // loss sums and the CTAs' partial gradients of one layer
  return n * (repair_act_bytes_per_tile() + 4 * kRT * kRT * 4 + 4 + 2 * 4 * kNPos * 16 + 32) +
         (size_t)bwd_grid((int)n) * kBwdParts * 4 + 10 * 256;  // + alignment of the 8 buffers
}

cudaError_t prepare_repair() {
  cudaError_t e = cudaFuncSetAttribute(repair_net_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)net_smem(false));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(repair_net_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)net_smem(true));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(repair_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwd_smem());
  return e;
}

cudaError_t repair_pack(const Workspace &ws, cudaStream_t s) {
  repair_pack_kernel<<<(kWPackBytes / 2 + 255) / 256, 256, 0, s>>>(ws.rp_master, (uint16_t *)ws.rp_wpack,
                                                                   ws.rp_bias);
  repair_packT_kernel<<<(kWPackTBytes / 2 + 255) / 256, 256, 0, s>>>(ws.rp_master, (uint16_t *)ws.rp_wpackT);
  GS_LAUNCHED(2);
  return cudaGetLastError();
}

cudaError_t repair_features(const Workspace &ws, int W, int H, const float *rgb_aff, uint4 *feat, cudaStream_t s) {
  const dim3 grid((W + kRT - 1) / kRT, (H + kRT - 1) / kRT);
  launch_k(repair_features_kernel, grid, 256, 0, s, ws.warpbuf, ws.cls, rgb_aff, W, H, feat);
  GS_LAUNCHED(1);
  return cudaGetLastError();
}

static int net_grid(uint32_t n_max, int per_sm = 1, int sm_share = 100) {
  uint32_t cap = (uint32_t)sm_grid_cap(per_sm) * (uint32_t)sm_share / 100u;
  if (cap < 1u) cap = 1u;
  return (int)(n_max < cap ? (n_max < 1u ? 1u : n_max) : cap);
}

cudaError_t repair_forward(const Workspace &ws, const uint4 *feat, int W, int H, const uint32_t *tiles,
                           const uint32_t *n_ptr, uint32_t n_max, float *fill, float *gate, float *out4,
                           uint4 *acts, cudaStream_t s, bool fp8, uint32_t *amax, int sm_share) {
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
    launch_k(repair_net_kernel<true>, net_grid(n_max, 2, sm_share), kNetThreads, net_smem(true), s, a);
  } else {
    launch_k(repair_net_kernel<false>, net_grid(n_max, 1, sm_share), kNetThreads, net_smem(false), s, a);
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
                          bool fp8, uint8_t *skip) {
  cudaError_t e;
  const int tx = (W + kRT - 1) / kRT, ty = (H + kRT - 1) / kRT, nt = tx * ty;
  if ((e = cudaMemsetAsync(ws.rp_nlist, 0, sizeof(uint32_t), s)) != cudaSuccess) return e;
  launch_k(repair_tile_list_kernel, dim3(tx, ty), 256, 0, s, ws.cls, ws.tile_mask, W, H, ws.rp_list, ws.rp_nlist,
           skip);
  GS_LAUNCHED(1);
  // beside the ROI binning (skip given) the network still takes every
  // multiprocessor: with a half or three quarters it became the longer branch on
  // the object workload
  if ((e = repair_forward(ws, ws.rp_feat, W, H, ws.rp_list, ws.rp_nlist, (uint32_t)nt, ws.rp_fill, ws.rp_gate,
                          nullptr, nullptr, s, fp8, nullptr, 100)) != cudaSuccess)
    return e;
  // sigmoid(g) >= tau  <=>  g >= log(tau / (1 - tau))
  const float tau = fminf(fmaxf(gate_tau, 1e-6f), 1.f - 1e-6f);
  const float logit_tau = logf(tau / (1.f - tau));
  launch_k(repair_merge_kernel, nt, 256, 0, s, ws.rp_list, ws.rp_nlist, ws.rp_gate, logit_tau, ws.warpbuf, ws.rp_fill, W, H,
           tx, rgb_aff, ws.cls, ws.tile_mask, skip);
  GS_LAUNCHED(1);
  return cudaGetLastError();
}

cudaError_t repair_train_step(const Workspace &ws, const RepairBatch &b, const RepairOpt &o, float *host_loss,
                              cudaStream_t s) {
  cudaError_t e;
  const int n = b.n_tiles;
  uint8_t *p = (uint8_t *)(((uintptr_t)b.scratch + 255) & ~(uintptr_t)255);
  auto take = [&p](size_t bytes) {
    uint8_t *q = p;
    p += (bytes + 255) / 256 * 256;
    return q;
  };
  uint4 *acts = (uint4 *)take((size_t)n * repair_act_bytes_per_tile());
  float *out4 = (float *)take((size_t)n * 4 * kRT * kRT * 4);
  float *gate = (float *)take((size_t)n * 4);
  uint4 *dy = (uint4 *)take((size_t)n * 4 * kNPos * 16);
  uint4 *dx = (uint4 *)take((size_t)n * 4 * kNPos * 16);
  float *stats = (float *)take((size_t)n * 32);
  float *sums = (float *)take(8 * sizeof(float));
  const int G = bwd_grid(n);
  float *part = (float *)take((size_t)G * kBwdParts * 4);
  if ((e = cudaMemsetAsync(sums, 0, 8 * sizeof(float), s)) != cudaSuccess) return e;
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
  a.tile_stats = stats;
  a.sums = sums;
  a.lam = o.gate_weight;
  repair_stats_kernel<<<n, 256, 0, s>>>(a);
  repair_sums_kernel<<<1, 1024, 0, s>>>(stats, n, 2, 4, sums, 0);  // holes, L1 sum
  repair_dout_kernel<<<n, 256, 0, s>>>(a);
  repair_sums_kernel<<<1, 1024, 0, s>>>(stats, n, 5, 6, sums, 2);  // BCE, positive labels
  GS_LAUNCHED(4);
  // backward, last layer first: per layer one tensor-core kernel (weight
  // gradient into per-CTA partials, input gradient into the other buffer) and
  // the fixed-order reduction of the partials into this layer's gradient
  uint4 *cur = dy, *nxt = dx;
  for (int l = 5; l >= 0; --l) {
    BwdArgs ba;
    ba.acts = acts;
    ba.dy = cur;
    ba.dyo = nxt;
    ba.wpackT = ws.rp_wpackT;
    ba.part = part;
    ba.l = l;
    ba.n = n;
    ba.status = &ws.ctr->status;
    repair_bwd_kernel<<<G, kBwdThreads, bwd_smem(), s>>>(ba);
    const int count = cout(l) * 9 * cin(l) + cout(l);
    repair_reduce_kernel<<<(count + 255) / 256, 256, 0, s>>>(part, G, count, ws.rp_grad + poff(l));
    GS_LAUNCHED(2);
    uint4 *tmp = cur;
    cur = nxt;
    nxt = tmp;
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
