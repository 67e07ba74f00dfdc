// Reprojection to the affiliated eye, hole categorisation and the adaptive ROI
// generator.
//
// Paper: Sec. 3.1 Stages 2-4; Sec. 3.4 Eq. 3-5 (unproject with the depth proxy,
// transfer, project); Sec. 3.5 Step 1 (edge ROIs, Eq. 6-8, margin m, 16x16
// tiles) and Step 2 (connected centre holes -> box -> margin -> tiles).
//
// Readings of passages the paper leaves open (the oracle states the same):
//  - a source pixel is a surface sample when its coverage 1 - T >= 0.5 and warps
//    with D / (1 - T); otherwise it is a background sample at infinite depth
//    (direction-only transfer) that loses every depth test;
//  - a sample lands on pixel (floor(x + 0.5), floor(y + 0.5)); the packed key
//    (float depth bits << 32 | source index) resolves the depth test with one
//    64-bit atomicMin, smallest depth first and then smallest source index;
//  - edge ROI samples are taken at the pixel they round to;
//  - gaps: holes outside the edge strips whose horizontal or vertical hole run is
//    at most gap_thresh long with valid pixels at both ends, filled by linear
//    interpolation along the shorter such run (horizontal on ties); the other
//    holes are centre holes (4-connected components -> ROIs).
#include "gs_internal.cuh"
#include "gs_launch.cuh"
#include "gs_scan.cuh"

namespace gs {

// The pixels of a grid-stride loop: the linear index and its column and row,
// advanced by the grid's stride with an add and a carry instead of a division
// per pixel.
struct PixelWalk {
  int64_t p, step;
  int x, y, sx, sy, W;
  __device__ explicit PixelWalk(int W_) : W(W_) {
    p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    step = (int64_t)gridDim.x * blockDim.x;
    x = (int)(p % W);
    y = (int)(p / W);
    sx = (int)(step % W);
    sy = (int)(step / W);
  }
  __device__ void next() {
    p += step;
    x += sx;
    y += sy;
    if (x >= W) {
      x -= W;
      ++y;
    }
  }
};

constexpr uint32_t kInfBits = 0x7f800000u;

__device__ __forceinline__ bool transfer(const CamBlock &cb, float x, float y, float d, bool surface, float &u,
                                         float &v, float &z) {
  const EyeCam &c = cb.eye[0];
  const float rx = (x - c.cx) / c.fx, ry = (y - c.cy) / c.fy;
  const float *R = cb.Rrel;
  float X, Y, Z;
  if (surface) {  // Eq. 4 then Eq. 5 with the composed relative pose
    X = fmaf(R[0], rx * d, fmaf(R[1], ry * d, fmaf(R[2], d, cb.trel[0])));
    Y = fmaf(R[3], rx * d, fmaf(R[4], ry * d, fmaf(R[5], d, cb.trel[1])));
    Z = fmaf(R[6], rx * d, fmaf(R[7], ry * d, fmaf(R[8], d, cb.trel[2])));
    if (!(Z > kZNear)) return false;
  } else {  // direction only
    X = fmaf(R[0], rx, fmaf(R[1], ry, R[2]));
    Y = fmaf(R[3], rx, fmaf(R[4], ry, R[5]));
    Z = fmaf(R[6], rx, fmaf(R[7], ry, R[8]));
    if (!(Z > 0.f)) return false;
  }
  const EyeCam &a = cb.eye[1];
  u = fmaf(a.fx, X / Z, a.cx);  // Eq. 3
  v = fmaf(a.fy, Y / Z, a.cy);
  z = Z;
  return true;
}

// ---------------------------------------------------------------- forward warp
struct EdgeArgs {
  Counters *ctr;
  int N, m, depth_mode;
  float fixed_min, fixed_max;
  int32_t *strips, *widths;
  float *drange;
  uint8_t *tile_mask;
  int assign;  // 1: the strips are the mask's only tiles; 0: added to a cleared mask
};
__device__ void edge_roi_block(const CamBlock *__restrict__ cams, const EdgeArgs &ea);

// The first block also computes the edge ROIs (Step 1) when `edge` is set: they
// need only the depth range of Stage 1, and the classification that reads them
// follows this kernel.
__global__ void __launch_bounds__(256) warp_scatter_kernel(const CamBlock *__restrict__ cams,
                                                           const float *__restrict__ depth,
                                                           const float *__restrict__ trans,
                                                           unsigned long long *__restrict__ buf, int W, int H,
                                                           int edge, EdgeArgs ea) {
  griddep_wait();
  if (edge && blockIdx.x == 0) edge_roi_block(cams, ea);
  const CamBlock &cb = *cams;
  const int64_t npix = (int64_t)W * H;
  for (PixelWalk pw(W); pw.p < npix; pw.next()) {
    const int64_t p = pw.p;
    const float cov = 1.f - trans[p];
    const bool surface = cov >= 0.5f;
    const float d = surface ? depth[p] / cov : 0.f;
    float u, v, z;
    if (!transfer(cb, (float)pw.x, (float)pw.y, d, surface, u, v, z)) continue;
    const float fx = floorf(u + 0.5f), fy = floorf(v + 0.5f);
    if (!(fx >= 0.f && fx <= (float)(W - 1) && fy >= 0.f && fy <= (float)(H - 1))) continue;
    const uint32_t zb = surface ? __float_as_uint(z) : kInfBits;
    const int64_t q = (int64_t)fy * W + (int64_t)fx;
    atomicMin(buf + q, ((unsigned long long)zb << 32) | (unsigned long long)(uint32_t)p);
  }
}

// ---------------------------------------------------------------- edge ROI (Step 1)
// One block (any size) computes the edge ROIs: samples at the two depth
// hypotheses, the extrema of Eq. 6, the widths of Eq. 7-8, the tile-aligned
// strips and their tiles in the mask.
__device__ void edge_roi_block(const CamBlock *__restrict__ cams, const EdgeArgs &ea) {
  Counters *ctr = ea.ctr;
  const int N = ea.N, m = ea.m, depth_mode = ea.depth_mode, assign = ea.assign;
  int32_t *strips = ea.strips, *widths = ea.widths;
  float *drange = ea.drange;
  uint8_t *tile_mask = ea.tile_mask;
  const CamBlock &cb = *cams;
  const int W = cb.eye[1].W, H = cb.eye[1].H;
  const int tiles_x = (W + kTile - 1) / kTile, tiles_y = (H + kTile - 1) / kTile;  // the ROI grid
  __shared__ int sxmin, sxmax, symin, symax, sany;
  __shared__ int sstrip[16];
  float dmin = ea.fixed_min, dmax = ea.fixed_max;
  if (depth_mode == 0 || depth_mode == 2) {  // this frame's range, or the previous frame's
    const uint32_t lo = depth_mode == 0 ? ctr->dmin_bits : ctr->prev_range[0];
    const uint32_t hi = depth_mode == 0 ? ctr->dmax_bits : ctr->prev_range[1];
    dmin = __uint_as_float(lo);
    dmax = __uint_as_float(hi);
    if (hi == 0u) dmin = dmax = 0.f;  // no valid pixel
  }
  if (threadIdx.x == 0) {
    sxmin = symin = 0x7fffffff;
    sxmax = symax = -0x7fffffff;
    sany = 0;
    drange[0] = dmin;
    drange[1] = dmax;
  }
  __syncthreads();
  const int nsamp = 4 * N * 2;
  for (int k = threadIdx.x; k < nsamp; k += blockDim.x) {
    const int e = k / (2 * N), r = (k / 2) % N, h = k & 1;
    const int along = e < 2 ? W : H;
    const int pos = (int)(((long long)2 * r * (along - 1) + (N - 1)) / (2LL * (N - 1)));
    const int x = e == 0 ? pos : e == 1 ? pos : e == 2 ? 0 : W - 1;
    const int y = e == 0 ? 0 : e == 1 ? H - 1 : pos;
    const float d = h ? dmax : dmin;
    float u, v, z;
    if (!(d > 0.f) || !transfer(cb, (float)x, (float)y, d, true, u, v, z)) continue;
    u = fminf(fmaxf(u, -1e9f), 1e9f);
    v = fminf(fmaxf(v, -1e9f), 1e9f);
    const int ix = (int)floorf(u + 0.5f), iy = (int)floorf(v + 0.5f);
    atomicMin(&sxmin, ix); atomicMax(&sxmax, ix);
    atomicMin(&symin, iy); atomicMax(&symax, iy);
    sany = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int lw, rw, th, bh;
    if (!sany) {
      lw = rw = W / 2;
      th = bh = H / 2;
    } else {  // Eq. 7, Eq. 8 and the vertical analogues
      lw = sxmin > 0 ? min(max(min(sxmin, W) + m, 0), W / 2) : 0;
      rw = sxmax < W - 1 ? min(max((W - 1) - max(sxmax, -1) + m, 0), W / 2) : 0;
      th = symin > 0 ? min(max(min(symin, H) + m, 0), H / 2) : 0;
      bh = symax < H - 1 ? min(max((H - 1) - max(symax, -1) + m, 0), H / 2) : 0;
    }
    widths[0] = lw; widths[1] = rw; widths[2] = th; widths[3] = bh;
    // tile-aligned strips (half-open pixels): left, right, top, bottom
    const int lx1 = lw > 0 ? min((lw + kTile - 1) / kTile * kTile, W) : 0;
    const int rx0 = rw > 0 ? (W - rw) / kTile * kTile : W;
    const int ty1 = th > 0 ? min((th + kTile - 1) / kTile * kTile, H) : 0;
    const int by0 = bh > 0 ? (H - bh) / kTile * kTile : H;
    const int s[16] = {0, 0, lx1, lw > 0 ? H : 0, rx0, 0, W, rw > 0 ? H : 0,
                       0, 0, th > 0 ? W : 0, ty1, 0, by0, bh > 0 ? W : 0, H};
    for (int k = 0; k < 16; ++k) {
      strips[k] = s[k];
      sstrip[k] = s[k];
    }
  }
  __syncthreads();
  const int ntiles = tiles_x * tiles_y;
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
    const int x0 = (t % tiles_x) * kTile, y0 = (t / tiles_x) * kTile;
    bool in = false;
    for (int k = 0; k < 4; ++k) {
      const int *r = sstrip + 4 * k;
      in |= x0 < r[2] && x0 + kTile > r[0] && y0 < r[3] && y0 + kTile > r[1];
    }
    if (assign) tile_mask[t] = in ? 1 : 0;  // a mask of its own
    else if (in) tile_mask[t] = 1;         // into the cleared ROI mask
  }
}

__global__ void __launch_bounds__(256) edge_roi_kernel(const CamBlock *__restrict__ cams, EdgeArgs ea) {
  griddep_wait();
  edge_roi_block(cams, ea);
}

// ------------------------------------------------ resolve + classification + fill
//
// Per affiliated pixel: resolve the warp buffer, then (outside the edge strips)
// classify holes into gaps and centre holes and fill gaps by interpolation. All
// neighbour reads go to the warp buffer (read-only here), so pixels never read
// another pixel's output.
struct WarpView {
  const unsigned long long *buf;
  const float *rgb_dom;
  int W, H;
  size_t hw;
  __device__ bool hole(int x, int y) const { return buf[(size_t)y * W + x] == kNoSample; }
  __device__ void colour(int x, int y, float c[3]) const {
    const uint32_t s = (uint32_t)(buf[(size_t)y * W + x] & 0xffffffffull);
    c[0] = rgb_dom[s];
    c[1] = rgb_dom[hw + s];
    c[2] = rgb_dom[2 * hw + s];
  }
};

__global__ void __launch_bounds__(256) classify_kernel(WarpView wv, const int32_t *__restrict__ strips, int gap,
                                                       int center_enabled, float *__restrict__ rgb_aff,
                                                       float *__restrict__ warp_depth, uint8_t *__restrict__ cls,
                                                       Counters *__restrict__ ctr, uint32_t *__restrict__ cc_list,
                                                       int32_t *__restrict__ labels) {
  griddep_wait();
  // this frame's measured depth range, kept for the next frame's edge ROI
  // (depth_mode 2); the edge ROI of this frame has read the previous one
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctr->prev_range[0] = ctr->dmin_bits;
    ctr->prev_range[1] = ctr->dmax_bits;
  }
  const int W = wv.W, H = wv.H;
  const int64_t npix = (int64_t)W * H;
  __shared__ int s[16];
  if (threadIdx.x < 16) s[threadIdx.x] = strips[threadIdx.x];
  __syncthreads();
  for (PixelWalk pw(W); pw.p < npix; pw.next()) {
    const int64_t p = pw.p;
    const int x = pw.x, y = pw.y;
    const unsigned long long key = wv.buf[p];
    const bool hole = key == kNoSample;
    bool strip = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) strip |= x >= s[4 * k] && x < s[4 * k + 2] && y >= s[4 * k + 1] && y < s[4 * k + 3];
    uint8_t c = (hole ? kClsHole : 0u) | (strip ? kClsStrip : 0u);
    float out[3] = {0.f, 0.f, 0.f};
    if (!hole) {
      const uint32_t src = (uint32_t)(key & 0xffffffffull);  // the source pixel
      out[0] = wv.rgb_dom[src];
      out[1] = wv.rgb_dom[wv.hw + src];
      out[2] = wv.rgb_dom[2 * wv.hw + src];
      const uint32_t zb = (uint32_t)(key >> 32);
      warp_depth[p] = __uint_as_float(zb);
    } else {
      warp_depth[p] = 0.f;
    }
    if (hole && !strip) {
      // bounded runs up to gap + 1 long decide gaps; longer runs are scanned in
      // full only for the centre-off fallback
      int a = x, b = x, at = y, bt = y;
      const int lim = gap + 1;
      while (a - 1 >= 0 && x - (a - 1) <= lim && wv.hole(a - 1, y)) --a;
      while (b + 1 <= W - 1 && (b + 1) - x <= lim && wv.hole(b + 1, y)) ++b;
      while (at - 1 >= 0 && y - (at - 1) <= lim && wv.hole(x, at - 1)) --at;
      while (bt + 1 <= H - 1 && (bt + 1) - y <= lim && wv.hole(x, bt + 1)) ++bt;
      const bool endL = a - 1 >= 0 && !wv.hole(a - 1, y), endR = b + 1 <= W - 1 && !wv.hole(b + 1, y);
      const bool endU = at - 1 >= 0 && !wv.hole(x, at - 1), endD = bt + 1 <= H - 1 && !wv.hole(x, bt + 1);
      const int Lh = b - a + 1, Lv = bt - at + 1;
      const bool gh = endL && endR && Lh <= gap, gv = endU && endD && Lv <= gap;
      int axis = -1;
      if (gh && gv) axis = Lv < Lh ? 1 : 0;
      else if (gh) axis = 0;
      else if (gv) axis = 1;
      if (axis >= 0) {
        c |= kClsGap;
        float e0[3], e1[3];
        float t;
        if (axis == 0) {
          wv.colour(a - 1, y, e0);
          wv.colour(b + 1, y, e1);
          t = (float)(x - (a - 1)) / (float)(b + 1 - (a - 1));
        } else {
          wv.colour(x, at - 1, e0);
          wv.colour(x, bt + 1, e1);
          t = (float)(y - (at - 1)) / (float)(bt + 1 - (at - 1));
        }
        for (int k = 0; k < 3; ++k) out[k] = fmaf(t, e1[k], fmaf(-t, e0[k], e0[k]));
      } else {
        c |= kClsCentre;
        if (!center_enabled) {
          // fallback fill along the row (full run), else the column
          while (a - 1 >= 0 && wv.hole(a - 1, y)) --a;
          while (b + 1 <= W - 1 && wv.hole(b + 1, y)) ++b;
          const bool hl = a - 1 >= 0, hr = b + 1 <= W - 1;
          int ex0 = -1, ey0 = -1, ex1 = -1, ey1 = -1;
          float t = 0.f;
          if (hl || hr) {
            if (hl) { ex0 = a - 1; ey0 = y; }
            if (hr) { ex1 = b + 1; ey1 = y; }
            t = (float)(x - (a - 1)) / (float)(b + 1 - (a - 1));
          } else {
            while (at - 1 >= 0 && wv.hole(x, at - 1)) --at;
            while (bt + 1 <= H - 1 && wv.hole(x, bt + 1)) ++bt;
            if (at - 1 >= 0) { ex0 = x; ey0 = at - 1; }
            if (bt + 1 <= H - 1) { ex1 = x; ey1 = bt + 1; }
            t = (float)(y - (at - 1)) / (float)(bt + 1 - (at - 1));
          }
          float e0[3], e1[3];
          if (ex0 >= 0 && ex1 >= 0) {
            wv.colour(ex0, ey0, e0);
            wv.colour(ex1, ey1, e1);
            for (int k = 0; k < 3; ++k) out[k] = fmaf(t, e1[k], fmaf(-t, e0[k], e0[k]));
          } else if (ex0 >= 0) {
            wv.colour(ex0, ey0, out);
          } else if (ex1 >= 0) {
            wv.colour(ex1, ey1, out);
          }
        }
      }
    }
    rgb_aff[p] = out[0];
    rgb_aff[wv.hw + p] = out[1];
    rgb_aff[2 * wv.hw + p] = out[2];
    cls[p] = c;
    // centre holes join the component labelling's list (one atomic per warp;
    // the list order does not reach any output)
    const bool cc = (c & kClsCentre) != 0;
    const unsigned am = __activemask();
    const unsigned bal = __ballot_sync(am, cc);
    if (bal) {
      const int lane = threadIdx.x & 31, leader = __ffs(bal) - 1;
      uint32_t base = 0;
      if (lane == leader) base = atomicAdd(&ctr->n_centre, (uint32_t)__popc(bal));
      base = __shfl_sync(am, base, leader);
      if (cc) {
        const uint32_t k = base + (uint32_t)__popc(bal & ((1u << lane) - 1u));
        cc_list[k] = (uint32_t)p;
        labels[p] = (int32_t)k;  // the pixel's place in the list
      }
    }
  }
}

// ---------------------------------------------------------------- centre ROIs (Step 2)
//
// Union-find labelling of the 4-connected centre-hole components; every root is
// the component's smallest linear index (links always go from the larger root to
// the smaller one), which also gives the canonical rectangle order.
constexpr int kMaxUnionSteps = 1 << 22;

// One CTA labels the components over the classification's list of centre-hole
// pixels (about 0.1 % of the frame on the workloads here, so a full-image pass
// per phase would cost more than the labelling). A pixel's neighbours are found
// through labels[] (its list position, written by the classification) once the
// class map says they are centre holes. Phases, separated by block barriers:
//   1. runs of consecutive entries point at their first entry, then links with
//      the left and upper neighbours (cc_union_all): the root with the larger
//      pixel is linked below the other by a CAS (bounded retries), so every
//      component's root is its smallest pixel, the canonical rectangle order;
//      finds halve their paths;
//   2. every entry's parent to its root;
//   3. the roots' ranks by pixel are the rectangle slots: up to one root per
//      thread counts the roots with a smaller pixel, up to kCcBoxes roots are
//      sorted (bitonic) and found by binary search, more are ranked through a
//      bitmap of the root pixels and its per-word prefix counts;
//   4. bounding boxes (shared-memory atomics up to kCcBoxes components, else
//      global atomics on the rectangles);
//   5. expand by m, align outward to tiles, clip, mark the tiles.
// Up to kCcFast entries the list and the parents live in shared memory, longer
// lists keep them in global memory.
constexpr int kCcThreads = 1024;
constexpr int kCcFast = 16384;   // entries whose list and parents stay in shared memory
constexpr int kCcBoxes = 4096;   // components sorted and boxed in shared memory
constexpr uint32_t kCcRank = 0x80000000u;
constexpr size_t kCcSmemBytes = sizeof(uint32_t) * (2 * kCcFast + kCcBoxes) + sizeof(int4) * kCcBoxes;

// Root of x with path halving. A concurrent link only turns a root into a child,
// and a halving store writes a grandparent (an ancestor), so every parent word
// keeps pointing into its own tree.
__device__ __forceinline__ uint32_t cc_find(volatile uint32_t *par, uint32_t x) {
  for (int steps = 0; steps < kMaxUnionSteps; ++steps) {
    const uint32_t p = par[x];
    if (p == x) return x;
    const uint32_t g = par[p];
    par[x] = g;
    x = g;
  }
  return x;
}

// The root of entry x without writing: while every entry is being set to its
// root, a halving walk could write a stale grandparent over an entry another
// thread has just set to its root. Read only, every pointer read is the entry's
// old parent or its root, both ancestors, so the walk ends at the root.
__device__ __forceinline__ uint32_t cc_root(const volatile uint32_t *par, uint32_t x) {
  for (int steps = 0; steps < kMaxUnionSteps; ++steps) {
    const uint32_t p = par[x];
    if (p == x) return x;
    x = p;
  }
  return x;
}

// Links the roots of entries a and b (pix: their pixels) with a CAS on the root
// with the larger pixel; bounded retries.
__device__ void cc_unite(uint32_t *par, const uint32_t *pix, uint32_t a, uint32_t b, uint32_t *status) {
  volatile uint32_t *vp = par;
  for (int it = 0; it < kMaxUnionSteps; ++it) {
    a = cc_find(vp, a);
    b = cc_find(vp, b);
    if (a == b) return;
    if (pix[a] < pix[b]) {
      const uint32_t t = a;
      a = b;
      b = t;
    }
    if (atomicCAS(par + a, a, b) == a) return;
  }
  atomicOr(status, kStTimeout);
}

// Phase 1. The classification appends the centre holes of 32 consecutive pixels
// together, so a horizontal run of them is mostly a run of consecutive list
// entries. First, without links, every entry that continues its left neighbour
// at the previous list position points straight at its run's first entry in
// the warp's 32 entries (a smaller pixel, so roots stay the smallest pixels).
// Then the links, all loads issued first: a run's first entry with its left
// neighbour elsewhere in the list, a run continuing from the previous 32
// entries, and an entry with its upper neighbour - skipped when its left
// neighbour is in its run and that neighbour's upper pixel is a centre hole too
// (the two upper pixels are then connected, and the left one's link covers
// both), so a run links about once per run above it.
__device__ __forceinline__ void cc_union_all(const uint8_t *__restrict__ cls, const int32_t *labels,
                                             const uint32_t *pix, uint32_t *par, uint32_t n, int W,
                                             uint32_t *status) {
  const uint32_t lane = threadIdx.x & 31u, uW = (uint32_t)W;
  for (uint32_t base = threadIdx.x & ~31u; base < n; base += kCcThreads) {  // warp-uniform
    const uint32_t k = base + lane;
    const bool valid = k < n;
    const uint32_t p = valid ? pix[k] : 0u;
    const bool cont = valid && k > 0u && p % uW != 0u && pix[k - 1] == p - 1u;
    const uint32_t heads = __ballot_sync(0xffffffffu, valid && !cont);
    if (cont) {
      const uint32_t le = heads & (0xffffffffu >> (31u - lane));  // heads at or before this lane
      if (le) par[k] = base + 31u - (uint32_t)__clz(le);
      else if (lane > 0u) par[k] = base;  // the run came in from the previous 32 entries
    }
  }
  __syncthreads();
  for (uint32_t base = threadIdx.x & ~31u; base < n; base += kCcThreads) {  // warp-uniform
    const uint32_t k = base + lane;
    if (k >= n) continue;
    const uint32_t p = pix[k];
    const bool cont = k > 0u && p % uW != 0u && pix[k - 1] == p - 1u;
    const bool need_l = !cont && p % uW != 0u, hu = p >= uW;
    const uint8_t cl = need_l ? cls[p - 1] : 0, cu = hu ? cls[p - uW] : 0, cul = hu && cont ? cls[p - 1 - uW] : 0;
    const bool link_l = need_l && (cl & kClsCentre), link_u = (cu & kClsCentre) && !(cont && (cul & kClsCentre));
    // list positions only of centre holes: the class map was just written and
    // sits in L2, but labels[] is written at centre holes only, so reading it at
    // any other pixel would wait on DRAM for a value that is never used
    const uint32_t kl = link_l ? (uint32_t)labels[p - 1] : 0u, ku = link_u ? (uint32_t)labels[p - uW] : 0u;
    if (link_l) cc_unite(par, pix, k, kl, status);
    if (cont && lane == 0u) cc_unite(par, pix, k, k - 1, status);
    if (link_u) cc_unite(par, pix, k, ku, status);
  }
}

// Phase 3 for many roots: bitmap of the root pixels in bits[] (W * H bits) and
// per-word prefix counts in pre[]; returns the root count.
__device__ uint32_t cc_rank_bitmap(const uint32_t *par, const uint32_t *pix, uint32_t n, uint32_t npx,
                                   uint32_t *bits, uint32_t *pre, uint32_t *s_scan) {
  const uint32_t nw = (npx + 31u) / 32u;
  for (uint32_t w = threadIdx.x; w < nw; w += kCcThreads) bits[w] = 0u;
  __syncthreads();
  for (uint32_t k = threadIdx.x; k < n; k += kCcThreads)
    if (par[k] == k) atomicOr(bits + pix[k] / 32u, 1u << (pix[k] % 32u));
  __syncthreads();
  const uint32_t per = (nw + kCcThreads - 1) / kCcThreads;
  const uint32_t w0 = min((uint32_t)threadIdx.x * per, nw), w1 = min(w0 + per, nw);
  uint32_t cnt = 0;
  for (uint32_t w = w0; w < w1; ++w) cnt += (uint32_t)__popc(bits[w]);
  uint32_t base;
  const uint32_t nr = block_exclusive_scan<kCcThreads>(cnt, &base, s_scan);
  for (uint32_t w = w0; w < w1; ++w) {
    pre[w] = base;
    base += (uint32_t)__popc(bits[w]);
  }
  __syncthreads();
  return nr;
}

__device__ __forceinline__ uint32_t cc_bitmap_slot(const uint32_t *bits, const uint32_t *pre, uint32_t rp) {
  return pre[rp / 32u] + (uint32_t)__popc(bits[rp / 32u] & ((1u << (rp % 32u)) - 1u));
}

// Phase 5: the component boxes to tile-aligned rectangles and the tile mask.
__device__ __forceinline__ void cc_finish(int4 *rects, const int4 *box, uint32_t nbox, int W, int H, int m,
                                          int tiles_x, int tiles_y, uint8_t *tile_mask) {
  for (uint32_t sl = threadIdx.x; sl < nbox; sl += kCcThreads) {
    const int4 bx = box[sl];
    const int tx0 = bx.x - m <= 0 ? 0 : (bx.x - m) / kTile, ty0 = bx.y - m <= 0 ? 0 : (bx.y - m) / kTile;
    const int tx1 = min((bx.z + m) / kTile, tiles_x - 1), ty1 = min((bx.w + m) / kTile, tiles_y - 1);
    rects[sl] = make_int4(tx0 * kTile, ty0 * kTile, min((tx1 + 1) * kTile, W), min((ty1 + 1) * kTile, H));
    for (int ty = ty0; ty <= ty1; ++ty)
      for (int tx = tx0; tx <= tx1; ++tx) tile_mask[ty * tiles_x + tx] = 1;
  }
}

__global__ void __launch_bounds__(kCcThreads) cc_label_kernel(const uint8_t *__restrict__ cls,
                                                              const uint32_t *__restrict__ list,
                                                              int32_t *__restrict__ labels,
                                                              uint32_t *__restrict__ gpar, int4 *rects,
                                                              Counters *ctr, uint32_t cap, int W, int H, int m,
                                                              int tiles_x, int tiles_y, uint8_t *__restrict__ tile_mask) {
  griddep_wait();
  extern __shared__ __align__(16) uint32_t s_cc[];
  __shared__ uint32_t s_scan[32];
  __shared__ uint32_t s_nr;
  const int tid = threadIdx.x;
  const uint32_t npx = (uint32_t)W * (uint32_t)H;
  const uint32_t n = min(ctr->n_centre, npx);
  const bool fast = n <= (uint32_t)kCcFast;
  uint32_t *pix = fast ? s_cc : const_cast<uint32_t *>(list);
  uint32_t *par = fast ? s_cc + kCcFast : gpar;
  uint32_t *s_roots = s_cc + 2 * kCcFast;                              // [kCcBoxes]
  int4 *s_box = reinterpret_cast<int4 *>(s_cc + 2 * kCcFast + kCcBoxes);  // [kCcBoxes]
  if (tid == 0) s_nr = 0u;
  for (uint32_t k = tid; k < n; k += kCcThreads) {
    if (fast) pix[k] = list[k];
    par[k] = k;
  }
  __syncthreads();
  // 1. union; 2. parents to roots
  cc_union_all(cls, labels, pix, par, n, W, &ctr->status);
  __syncthreads();
  for (uint32_t k = tid; k < n; k += kCcThreads) par[k] = cc_root(par, k);
  __syncthreads();
  // 3. the roots' slots: par[root] = kCcRank | slot
  uint32_t *s_rootk = reinterpret_cast<uint32_t *>(s_box);  // the roots' list positions, until the boxes
  for (uint32_t k = tid; k < n; k += kCcThreads) {
    if (par[k] == k) {
      const uint32_t j = atomicAdd(&s_nr, 1u);
      if (j < (uint32_t)kCcBoxes) {
        s_roots[j] = pix[k];
        s_rootk[j] = k;
      }
    }
  }
  __syncthreads();
  uint32_t nr = s_nr;
  const bool sorted = nr <= (uint32_t)kCcBoxes;
  uint32_t *bits = reinterpret_cast<uint32_t *>(labels), *pre = bits + (npx + 31u) / 32u;  // labels[] is free now
  if (nr <= (uint32_t)kCcThreads) {
    // up to one root per thread: its slot is the number of roots with a smaller
    // pixel. Every thread of a warp reads the same four roots at a time; the
    // roots are padded to a multiple of four with a value above every pixel.
    const uint32_t nr4 = (nr + 3u) & ~3u;
    if ((uint32_t)tid >= nr && (uint32_t)tid < nr4) s_roots[tid] = 0xffffffffu;
    __syncthreads();
    uint32_t sl = 0;
    if ((uint32_t)tid < nr) {
      const uint32_t mine = s_roots[tid];
      const uint4 *r4 = reinterpret_cast<const uint4 *>(s_roots);
      for (uint32_t j = 0; j < nr4 / 4u; ++j) {
        const uint4 v = r4[j];
        sl += (uint32_t)(v.x < mine) + (uint32_t)(v.y < mine) + (uint32_t)(v.z < mine) + (uint32_t)(v.w < mine);
      }
    }
    __syncthreads();
    if ((uint32_t)tid < nr) par[s_rootk[tid]] = kCcRank | sl;
    __syncthreads();  // s_rootk shares its memory with the boxes initialised below
  } else if (sorted) {
    uint32_t np2 = 1;
    while (np2 < nr) np2 <<= 1;
    for (uint32_t j = nr + tid; j < np2; j += kCcThreads) s_roots[j] = 0xffffffffu;
    __syncthreads();
    for (uint32_t size = 2; size <= np2; size <<= 1) {
      for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
        for (uint32_t i = tid; i < np2 / 2; i += kCcThreads) {
          const uint32_t lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
          const bool up = (lo & size) == 0;
          const uint32_t a = s_roots[lo], b = s_roots[hi];
          if ((a > b) == up) {
            s_roots[lo] = b;
            s_roots[hi] = a;
          }
        }
        __syncthreads();
      }
    }
  } else {
    nr = cc_rank_bitmap(par, pix, n, npx, bits, pre, s_scan);
  }
  for (uint32_t k = tid; nr > (uint32_t)kCcThreads && k < n; k += kCcThreads) {
    if (par[k] != k) continue;
    const uint32_t rp = pix[k];
    uint32_t sl;
    if (sorted) {
      uint32_t lo = 0, hi = nr;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (s_roots[mid] < rp) lo = mid + 1; else hi = mid;
      }
      sl = lo;
    } else {
      sl = cc_bitmap_slot(bits, pre, rp);
    }
    par[k] = kCcRank | sl;
  }
  const uint32_t nbox = min(nr, cap);
  int4 *box = sorted ? s_box : rects;
  for (uint32_t j = tid; j < nbox; j += kCcThreads) box[j] = make_int4(W, H, -1, -1);
  if (tid == 0) {
    ctr->n_rects = nr;
    if (nr > cap) atomicOr(&ctr->status, kStCapacity);
  }
  __syncthreads();
  // 4. bounding boxes. Consecutive list entries at consecutive pixels of one
  // row are one run of one component: only its first entry can lower the box's
  // x and set its rows, only its last can raise its x.
  for (uint32_t k = tid; k < n; k += kCcThreads) {
    const uint32_t p = pix[k];
    const uint32_t ux = p % (uint32_t)W;
    const bool first = k == 0u || ux == 0u || pix[k - 1] != p - 1u;
    const bool last = k + 1u >= n || ux + 1u == (uint32_t)W || pix[k + 1] != p + 1u;
    if (!first && !last) continue;
    const uint32_t r = par[k];
    const uint32_t sl = (r & kCcRank) ? (r & ~kCcRank) : (par[r] & ~kCcRank);
    if (sl >= nbox) continue;
    const int x = (int)ux, y = (int)(p / (uint32_t)W);
    int *q = reinterpret_cast<int *>(box + sl);
    if (first) {
      atomicMin(q + 0, x);
      atomicMin(q + 1, y);
      atomicMax(q + 3, y);
    }
    if (last) atomicMax(q + 2, x);
  }
  __syncthreads();
  // 5. rectangles and tiles
  cc_finish(rects, box, nbox, W, H, m, tiles_x, tiles_y, tile_mask);
}

// Clears the warp buffer (no sample) and the ROI tile mask.
__global__ void warp_init_kernel(unsigned long long *__restrict__ warpbuf, int64_t npix, uint8_t *__restrict__ mask,
                                 int ntiles) {
  griddep_wait();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += stride) warpbuf[i] = kNoSample;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ntiles; i += stride) mask[i] = 0;
}

static int grid_for(int64_t n, int per_block = 256) {
  const int64_t b = (n + per_block - 1) / per_block;
  const int64_t cap = sm_grid_cap(16);
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

// A grid-stride kernel's grid: at most one wave of resident 256-thread CTAs, so
// every CTA loops over the same number of pixels give or take one and no second,
// partly filled wave follows the first.
template <typename K>
static int grid_resident(K kernel, int64_t n, int &occupancy) {
  if (occupancy <= 0) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, 256, 0) != cudaSuccess || occ < 1) occ = 1;
    occupancy = occ;
  }
  const int64_t b = (n + 255) / 256;
  const int64_t cap = sm_grid_cap(occupancy);
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}
static int g_occ_scatter = 0, g_occ_classify = 0;

static EdgeArgs edge_args(const Workspace &ws, const gs_roi_params &roi, uint8_t *mask, bool assign) {
  return EdgeArgs{ws.ctr, roi.samples_per_edge, roi.margin, roi.depth_mode, roi.d_min, roi.d_max, ws.strips,
                  ws.widths, ws.drange, mask, assign ? 1 : 0};
}

static cudaError_t warp_launches(const Workspace &ws, int W, int H, const float *depth_dom, const float *trans_dom,
                                 const gs_roi_params *roi, cudaStream_t s, bool cleared = false) {
  const int64_t npix = (int64_t)W * H;
  const int tiles_x = (W + kTile - 1) / kTile, tiles_y = (H + kTile - 1) / kTile;
  cudaError_t err = cudaSuccess;
  if (!cleared) {
    err = launch_k(warp_init_kernel, grid_for(npix), 256, 0, s, ws.warpbuf, npix, ws.tile_mask, tiles_x * tiles_y);
    GS_LAUNCHED(1);
  }
  // with the buffer cleared by the rasterizer the mask is not cleared: the edge
  // ROI then writes every tile of it
  const EdgeArgs ea = roi ? edge_args(ws, *roi, ws.tile_mask, cleared) : EdgeArgs{};
  if (err == cudaSuccess)
    err = launch_k(warp_scatter_kernel, grid_resident(warp_scatter_kernel, npix, g_occ_scatter), 256, 0, s, ws.cams,
                   depth_dom, trans_dom, ws.warpbuf, W, H, roi ? 1 : 0, ea);
  GS_LAUNCHED(1);
  return err;
}

cudaError_t launch_warp(const Workspace &ws, int W, int H, const float *depth_dom, const float *trans_dom,
                        cudaStream_t s) {
  return warp_launches(ws, W, H, depth_dom, trans_dom, nullptr, s);
}

cudaError_t launch_edge_roi(const Workspace &ws, const gs_roi_params &roi, uint8_t *mask, bool assign,
                            cudaStream_t s) {
  const cudaError_t err = launch_k(edge_roi_kernel, 1, 256, 0, s, ws.cams, edge_args(ws, roi, mask, assign));
  GS_LAUNCHED(1);
  return err;
}

cudaError_t launch_classify(const Workspace &ws, int W, int H, int gap_thresh, const gs_roi_params &roi,
                            const float *rgb_dom, float *rgb_aff, cudaStream_t s) {
  const int64_t npix = (int64_t)W * H;
  WarpView wv{ws.warpbuf, rgb_dom, W, H, (size_t)npix};
  // the row/column fill of the remaining holes is the output when the centre step
  // is off, and the repair network's starting point in the repair modes (there
  // the ROI re-render or the network overwrites those pixels)
  const int fill_all = !roi.enable_center || roi.repair_mode != 0;
  const int grid = grid_resident(classify_kernel, npix, g_occ_classify);
  const cudaError_t err = launch_k(classify_kernel, grid, 256, 0, s, wv, ws.strips, gap_thresh, fill_all ? 0 : 1,
                                   rgb_aff, ws.warp_depth, ws.cls, ws.ctr, ws.cc_list, ws.labels);
  GS_LAUNCHED(1);
  return err;
}

cudaError_t launch_warp_classify(const Workspace &ws, int W, int H, int gap_thresh, const gs_roi_params &roi,
                                 const float *rgb_dom, const float *depth_dom, const float *trans_dom,
                                 float *rgb_aff, cudaStream_t s, bool cleared) {
  // warp and edge ROIs in one kernel, then the classification
  cudaError_t err = warp_launches(ws, W, H, depth_dom, trans_dom, &roi, s, cleared);
  if (err == cudaSuccess) err = launch_classify(ws, W, H, gap_thresh, roi, rgb_dom, rgb_aff, s);
  return err;
}

// Copies the strip tiles' pixels of an image rendered ahead (the edge strips of a
// reused depth range) into the affiliated image and marks them re-rendered.
__global__ void strip_composite_kernel(const uint8_t *__restrict__ strip_mask, int W, int H,
                                       const float *__restrict__ src, float *__restrict__ dst,
                                       uint8_t *__restrict__ cls) {
  griddep_wait();
  const int64_t npix = (int64_t)W * H;
  const int tiles_x = (W + kTile - 1) / kTile;
  for (PixelWalk pw(W); pw.p < npix; pw.next()) {
    const int64_t p = pw.p;
    const int x = pw.x, y = pw.y;
    if (!strip_mask[(y / kTile) * tiles_x + x / kTile]) continue;
    dst[p] = src[p];
    dst[npix + p] = src[npix + p];
    dst[2 * npix + p] = src[2 * npix + p];
    cls[p] |= (uint8_t)kClsRender;
  }
}

// mask &= ~minus (tiles already rendered elsewhere leave the mask)
__global__ void mask_minus_kernel(uint8_t *__restrict__ mask, const uint8_t *__restrict__ minus, int n) {
  griddep_wait();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (minus[i]) mask[i] = 0;
}

cudaError_t launch_strip_composite(const Workspace &ws, int W, int H, const float *src, float *rgb_aff,
                                   cudaStream_t s) {
  const int64_t npix = (int64_t)W * H;
  const cudaError_t err = launch_k(strip_composite_kernel, grid_for(npix), 256, 0, s, (const uint8_t *)ws.strip_mask,
                                   W, H, src, rgb_aff, ws.cls);
  GS_LAUNCHED(1);
  return err;
}

cudaError_t launch_mask_minus(uint8_t *mask, const uint8_t *minus, int n, cudaStream_t s) {
  const cudaError_t err = launch_k(mask_minus_kernel, grid_for(n), 256, 0, s, mask, minus, n);
  GS_LAUNCHED(1);
  return err;
}

cudaError_t launch_centre_rois(const Workspace &ws, int W, int H, int margin, cudaStream_t s) {
  const int tiles_x = (W + kTile - 1) / kTile, tiles_y = (H + kTile - 1) / kTile;
  launch_k(cc_label_kernel, 1, kCcThreads, kCcSmemBytes, s, (const uint8_t *)ws.cls, (const uint32_t *)ws.cc_list,
           ws.labels, ws.slots, ws.rects, ws.ctr, (uint32_t)ws.max_rects, W, H, margin, tiles_x,
           tiles_y, ws.tile_mask);
  GS_LAUNCHED(1);
  return cudaGetLastError();
}

// The centre-hole list of a class map: every pixel whose class has the centre bit,
// appended with one atomic per warp (the list order reaches no output), and its
// list position in labels[].
__global__ void centre_list_kernel(const uint8_t *__restrict__ cls, uint32_t npix, Counters *ctr,
                                   uint32_t *__restrict__ list, int32_t *__restrict__ labels) {
  griddep_wait();
  const int lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t b0 = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32u; b0 < npix; b0 += warps * 32u) {
    const uint32_t p = b0 + (uint32_t)lane;
    const bool cc = p < npix && (cls[p] & kClsCentre) != 0;
    const unsigned bal = __ballot_sync(0xffffffffu, cc);
    if (!bal) continue;  // warp-uniform
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&ctr->n_centre, (uint32_t)__popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (cc) {
      const uint32_t k = base + (uint32_t)__popc(bal & ((1u << lane) - 1u));
      list[k] = p;
      labels[p] = (int32_t)k;
    }
  }
}

cudaError_t launch_centre_rois_of(const Workspace &ws, const uint8_t *cls, int W, int H, int margin,
                                  uint8_t *tile_mask, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(&ws.ctr->n_centre, 0, sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  const uint32_t npix = (uint32_t)W * (uint32_t)H;
  launch_k(centre_list_kernel, grid_for((npix + 7) / 8), 256, 0, s, cls, npix, ws.ctr, ws.cc_list, ws.labels);
  GS_LAUNCHED(1);
  const int tiles_x = (W + kTile - 1) / kTile, tiles_y = (H + kTile - 1) / kTile;
  launch_k(cc_label_kernel, 1, kCcThreads, kCcSmemBytes, s, cls, (const uint32_t *)ws.cc_list, ws.labels, ws.slots,
           ws.rects, ws.ctr, (uint32_t)ws.max_rects, W, H, margin, tiles_x, tiles_y, tile_mask);
  GS_LAUNCHED(1);
  return cudaGetLastError();
}

// The component labelling's shared memory exceeds the default 48 KB: one opt-in
// per device (the attribute belongs to the kernel).
cudaError_t prepare_reproject() {
  return cudaFuncSetAttribute(cc_label_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCcSmemBytes);
}

}  // namespace gs
