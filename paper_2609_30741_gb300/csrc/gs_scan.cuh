// Device-wide exclusive scan with a device-resident element count, so a pipeline
// can size its work on the GPU without reading counts back to the host.
#pragma once

#include "gs_internal.cuh"
#include "gs_launch.cuh"

namespace gs {

__device__ __forceinline__ uint32_t load_n(const uint32_t *n_ptr, uint32_t n_max) {
  if (!n_ptr) return n_max;
  uint32_t n = *n_ptr;
  return n < n_max ? n : n_max;
}

// Block-wide exclusive scan of one value per thread; returns the block total.
template <int THREADS>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *excl, uint32_t *smem) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem[wid] = x;
  __syncthreads();
  if (wid == 0) {
    constexpr int NW = THREADS / 32;
    uint32_t w = lane < NW ? smem[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < NW) smem[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  const uint32_t warp_off = wid ? smem[wid - 1] : 0u;
  const uint32_t total = smem[THREADS / 32 - 1];
  *excl = warp_off + x - v;
  __syncthreads();
  return total;
}

// Single-pass exclusive scan with decoupled look-back. A CTA takes its tile of
// kScanTile elements from a device counter (so every tile it waits on belongs
// to a CTA that is already running), scans the tile in shared memory and
// publishes the tile total in a 64-bit status word: (epoch << 34) | (flag << 32)
// | value, flag 1 = the tile's own total, 2 = inclusive prefix through the tile.
// Warp 0 then walks back over the predecessors 32 at a time, adding totals up to
// the nearest inclusive prefix, and publishes its own. A word only counts when
// its epoch is this launch's; the last CTA out advances the epoch and clears the
// counters, so no status word needs clearing between launches (graph replays
// included). Every wait is bounded: after kLbSpinLimit reads a tile that has
// not published is taken as 0 and kStTimeout is raised in the status word.
//
// Scratch (per workspace, used by one scan at a time): `tiles`, one 64-bit
// word per tile, zero at context creation; `ctl` = {tile counter, exit
// counter, epoch}, zero at context creation.
constexpr uint32_t kLbAgg = 1u, kLbIncl = 2u;
constexpr uint32_t kLbSpinLimit = 1u << 20;

__device__ __forceinline__ unsigned long long lb_load(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void lb_store(unsigned long long *p, uint32_t epoch, uint32_t flag, uint32_t v) {
  const unsigned long long w = ((unsigned long long)((epoch << 2) | flag) << 32) | v;
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}

// Warp-collective: the sum of the totals of tiles [0, t) (t > 0).
__device__ __forceinline__ uint32_t lb_prefix(const unsigned long long *tiles, uint32_t t, uint32_t epoch,
                                              uint32_t *status) {
  const int lane = threadIdx.x & 31;
  uint32_t prefix = 0;
  for (int j = (int)t - 1; j >= 0; j -= 32) {  // warp-uniform
    const int idx = j - lane;  // lane 0: the nearest predecessor
    uint32_t flag = kLbIncl, v = 0;  // before tile 0: an inclusive zero
    if (idx >= 0) {
      for (uint32_t spin = 0;; ++spin) {
        const unsigned long long w = lb_load(tiles + idx);
        const uint32_t hi = (uint32_t)(w >> 32);
        if ((hi >> 2) == epoch && (hi & 3u) != 0u) {
          flag = hi & 3u;
          v = (uint32_t)w;
          break;
        }
        if (spin >= kLbSpinLimit) {  // never expected: give up on this tile, flag it
          atomicOr(status, kStTimeout);
          break;
        }
      }
    }
    const uint32_t incl = __ballot_sync(0xffffffffu, flag == kLbIncl);
    const int stop = incl ? __ffs(incl) - 1 : 31;
    uint32_t x = lane <= stop ? v : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    prefix += x;
    if (incl) break;
  }
  return prefix;
}

// ap(i, prefix, value, ap.fetch(i, value)) for every i < n, and ap.end(n, total)
// once. fetch only loads (its payload is gathered before the tile's prefix is
// known); the call with the prefix stores.
template <class Load, class Apply>
__global__ void __launch_bounds__(kScanThreads) scan_kernel(Load ld, Apply ap, const uint32_t *n_ptr, uint32_t n_max,
                                                            unsigned long long *tiles, uint32_t *ctl,
                                                            uint32_t *status) {
  griddep_wait();
  __shared__ uint32_t smem[32];
  __shared__ uint32_t vals[kScanTile];
  __shared__ uint32_t s_tile, s_prefix;
  const uint32_t n = load_n(n_ptr, n_max);
  if (threadIdx.x == 0) s_tile = atomicAdd(&ctl[0], 1u);
  __syncthreads();
  const uint32_t t = s_tile;
  const uint32_t epoch = (*(volatile uint32_t *)(ctl + 2)) & 0x3fffffffu;
  const uint32_t base = t * (uint32_t)kScanTile;
  if (base < n) {
    // coalesced loads, all issued before the first shared-memory store (a store
    // in between could alias the loaders' generic pointers and would serialise
    // their dependent chains)
    uint32_t ldv[kScanItems];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      const uint32_t i = base + k * kScanThreads + threadIdx.x;
      ldv[k] = i < n ? ld(i) : 0u;
    }
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) vals[k * kScanThreads + threadIdx.x] = ldv[k];
    __syncthreads();
    // each thread owns kScanItems consecutive elements
    uint32_t loc[kScanItems], acc = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      loc[k] = vals[threadIdx.x * kScanItems + k];
      acc += loc[k];
    }
    // the apply step's gathers, issued now: they land while the block scan and
    // the look-back run
    typename Apply::Payload pl[kScanItems];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      const uint32_t i = base + threadIdx.x * kScanItems + k;
      pl[k] = i < n ? ap.fetch(i, loc[k]) : typename Apply::Payload{};
    }
    uint32_t ex;
    const uint32_t tot = block_exclusive_scan<kScanThreads>(acc, &ex, smem);
    if (threadIdx.x < 32) {
      uint32_t prefix = 0;
      if (t == 0) {
        if (threadIdx.x == 0) lb_store(tiles, epoch, kLbIncl, tot);
      } else {
        if (threadIdx.x == 0) lb_store(tiles + t, epoch, kLbAgg, tot);
        prefix = lb_prefix(tiles, t, epoch, status);
        if (threadIdx.x == 0) lb_store(tiles + t, epoch, kLbIncl, prefix + tot);
      }
      if (threadIdx.x == 0) s_prefix = prefix;
    }
    __syncthreads();
    ex += s_prefix;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      const uint32_t i = base + threadIdx.x * kScanItems + k;
      if (i < n) ap(i, ex, loc[k], pl[k]);
      ex += loc[k];
    }
    if (base + kScanTile >= n && threadIdx.x == 0) ap.end(n, s_prefix + tot);
  } else if (t == 0 && threadIdx.x == 0) {
    ap.end(n, 0u);
  }
  // the last CTA out clears the counters and advances the epoch
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&ctl[1], 1u) == gridDim.x - 1) {
      ctl[0] = 0u;
      ctl[1] = 0u;
      ctl[2] = (epoch + 1u) & 0x3fffffffu;
      __threadfence();
    }
  }
}

// Scratch words: scan_tiles(n_max) 64-bit tile words, and 3 control words.
inline size_t scan_tiles(size_t n_max) { return (n_max + kScanTile - 1) / kScanTile + 1; }

template <class Load, class Apply>
cudaError_t scan_launch(Load ld, Apply ap, const uint32_t *n_ptr, uint32_t n_max, unsigned long long *tiles,
                        uint32_t *ctl, uint32_t *status, cudaStream_t s) {
  const int nblocks = (int)((n_max + kScanTile - 1) / kScanTile);
  launch_k(scan_kernel<Load, Apply>, nblocks < 1 ? 1 : nblocks, kScanThreads, 0, s, ld, ap, n_ptr, n_max, tiles, ctl,
           status);
  GS_LAUNCHED(1);
  return cudaGetLastError();
}

}  // namespace gs
