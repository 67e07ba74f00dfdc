// Stable LSD radix sort of (uint32 key, uint32 value) pairs, 8 bits per pass,
// with a device-resident element count ("one sweep" per pass).
//
//   1. One histogram kernel counts every pass's digits over all keys at once
//      (the digit counts of a pass do not depend on the order the earlier
//      passes leave); the last CTA out turns them into each pass's digit bases.
//   2. Per pass, one kernel: a CTA takes the next tile of 2048 pairs from a
//      device counter, ranks its pairs stably (per warp with bit ballots, then
//      across warps), publishes its per-digit counts, and finds every digit's
//      offset among the earlier tiles by decoupled look-back: it adds the
//      published counts of its predecessors, 8 tiles per step, down to the
//      nearest tile that has published an inclusive prefix, then publishes its
//      own. The tile is sorted in shared memory and each digit run is written
//      to its place with coalesced stores.
// Tiles are taken in counter order, so a CTA only ever waits for tiles that
// CTAs already running hold; every wait is bounded (kLbSpinLimit reads of a
// word, then kStTimeout is raised in the status word and the tile's count is
// taken as zero).
#pragma once

#include "gs_internal.cuh"
#include "gs_launch.cuh"
#include "gs_scan.cuh"

namespace gs {

constexpr int kRsThreads = 256;
constexpr int kRsItems = 8;
constexpr int kRsTile = kRsThreads * kRsItems;  // 2048 pairs per tile
constexpr int kRsPasses = 4;                    // 32-bit keys
constexpr int kRsWindow = 8;                    // predecessor tiles read per look-back step

struct RadixScratch {
  uint32_t *hist;              // [kRsPasses][256] digit counts (0 between sorts)
  uint32_t *base;              // [kRsPasses][256] exclusive digit bases
  unsigned long long *status;  // [tiles][256] look-back words (zero at context creation)
  uint32_t *ctl;               // {tile counter, exit counter, epoch, histogram exit counter}, zero at creation
  uint32_t *status_word;       // device status word
};

inline size_t radix_status_words(size_t n_max) { return 256 * ((n_max + kRsTile - 1) / kRsTile + 1); }

inline int radix_hist_grid(uint32_t n_max) {
  const uint32_t tiles = (n_max + kRsTile - 1) / kRsTile;
  const uint32_t cap = (uint32_t)sm_grid_cap(4);
  return (int)(tiles < 1 ? 1 : (tiles > cap ? cap : tiles));
}

// Digit counts of all passes; the last CTA out writes the bases and clears the
// counts and its ticket.
static __global__ void __launch_bounds__(kRsThreads) rs_hist_kernel(const uint32_t *__restrict__ keys,
                                                                     const uint32_t *n_ptr, uint32_t n_max,
                                                                     int npass, RadixScratch sc) {
  griddep_wait();
  __shared__ uint32_t h[kRsPasses][256];
  __shared__ uint32_t s_last, s_scan[32];
  for (int i = threadIdx.x; i < kRsPasses * 256; i += kRsThreads) (&h[0][0])[i] = 0u;
  __syncthreads();
  const uint32_t n = load_n(n_ptr, n_max);
  for (uint32_t i = blockIdx.x * kRsThreads + threadIdx.x; i < n; i += gridDim.x * kRsThreads) {
    const uint32_t k = keys[i];
    for (int p = 0; p < npass; ++p) atomicAdd(&h[p][(k >> (8 * p)) & 255u], 1u);
  }
  __syncthreads();
  for (int p = 0; p < npass; ++p) {
    const uint32_t v = h[p][threadIdx.x];
    if (v) atomicAdd(&sc.hist[p * 256 + threadIdx.x], v);
  }
  // every thread's counts are in before the CTA takes its exit ticket: without
  // the fence and the barrier a lagging warp could still be adding its counts
  // when the last CTA reads them
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&sc.ctl[3], 1u) == gridDim.x - 1 ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int p = 0; p < npass; ++p) {
    const uint32_t v = __ldcg(&sc.hist[p * 256 + threadIdx.x]);
    uint32_t ex;
    block_exclusive_scan<kRsThreads>(v, &ex, s_scan);
    sc.base[p * 256 + threadIdx.x] = ex;
    sc.hist[p * 256 + threadIdx.x] = 0u;
  }
  if (threadIdx.x == 0) sc.ctl[3] = 0u;
}

// Sum of digit d's counts over tiles [0, t) (t > 0) by decoupled look-back.
__device__ __forceinline__ uint32_t rs_lookback(const unsigned long long *status, uint32_t t, int d, uint32_t epoch,
                                                uint32_t *status_word) {
  uint32_t prefix = 0;
  for (int j = (int)t - 1; j >= 0; j -= kRsWindow) {
    unsigned long long w[kRsWindow];
#pragma unroll
    for (int k = 0; k < kRsWindow; ++k)  // independent loads: one round trip per window
      w[k] = j - k >= 0 ? lb_load(status + (size_t)(j - k) * 256 + d) : 0ull;
#pragma unroll
    for (int k = 0; k < kRsWindow; ++k) {
      if (j - k < 0) return prefix;
      unsigned long long x = w[k];
      uint32_t spin = 0;
      for (;;) {
        const uint32_t hi = (uint32_t)(x >> 32);
        if ((hi >> 2) == epoch && (hi & 3u) != 0u) break;
        if (++spin > kLbSpinLimit) {  // never expected: flag it and take the tile as empty, inclusive
          atomicOr(status_word, kStTimeout);
          x = ((unsigned long long)((epoch << 2) | kLbIncl) << 32);
          break;
        }
        x = lb_load(status + (size_t)(j - k) * 256 + d);
      }
      prefix += (uint32_t)x;
      if (((uint32_t)(x >> 32) & 3u) == kLbIncl) return prefix;
    }
  }
  return prefix;
}

static __global__ void __launch_bounds__(kRsThreads) rs_sweep_kernel(const uint32_t *__restrict__ kin,
                                                                      const uint32_t *__restrict__ vin,
                                                                      uint32_t *__restrict__ kout,
                                                                      uint32_t *__restrict__ vout,
                                                                      const uint32_t *n_ptr, uint32_t n_max, int pass,
                                                                      RadixScratch sc) {
  griddep_wait();
  constexpr int NW = kRsThreads / 32;
  __shared__ uint32_t s_warp[NW][256];
  __shared__ uint32_t s_local_base[256], s_global[256];
  __shared__ uint32_t s_keys[kRsTile], s_vals[kRsTile];
  __shared__ uint32_t s_scan[32];
  __shared__ uint32_t s_tile;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  const int shift = 8 * pass;
  if (tid == 0) s_tile = atomicAdd(&sc.ctl[0], 1u);
  __syncthreads();
  const uint32_t t = s_tile;
  const uint32_t epoch = (*(volatile uint32_t *)(sc.ctl + 2)) & 0x3fffffffu;
  const uint32_t n = load_n(n_ptr, n_max);
  const uint32_t base = t * (uint32_t)kRsTile;
  if (base < n) {
    for (int i = tid; i < NW * 256; i += kRsThreads) (&s_warp[0][0])[i] = 0;
    __syncthreads();
    // warp w owns pairs [w * 32 * kRsItems, (w + 1) * 32 * kRsItems) of the tile
    uint32_t k[kRsItems], r[kRsItems], v[kRsItems];
#pragma unroll
    for (int j = 0; j < kRsItems; ++j) {  // values loaded with the keys: no second wait
      const uint32_t i = base + (uint32_t)(wid * 32 * kRsItems + j * 32 + lane);
      k[j] = i < n ? kin[i] : 0u;
      v[j] = i < n ? vin[i] : 0u;
    }
#pragma unroll
    for (int j = 0; j < kRsItems; ++j) {
      const uint32_t i = base + (uint32_t)(wid * 32 * kRsItems + j * 32 + lane);
      const bool ok = i < n;
      const uint32_t d = (k[j] >> shift) & 255u;
      // lanes holding the same digit: intersect one ballot per digit bit
      uint32_t peers = __ballot_sync(0xffffffffu, ok);
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const uint32_t bit = (d >> b) & 1u;
        const uint32_t bb = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? bb : ~bb;
      }
      // the lowest such lane reserves the slots for the group in one shared atomic
      const int leader = __ffs(peers) - 1;
      uint32_t before = 0;
      if (ok && lane == leader) before = atomicAdd(&s_warp[wid][d], (uint32_t)__popc(peers));
      before = __shfl_sync(0xffffffffu, before, leader < 0 ? 0 : leader);
      r[j] = before + __popc(peers & lt);
    }
    __syncthreads();
    // digit d = tid: the tile's count, each warp's offset inside the digit run,
    // the run's place among the earlier tiles (look-back) and in the output
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      const uint32_t c = s_warp[w][tid];
      s_warp[w][tid] = cnt;
      cnt += c;
    }
    unsigned long long *my = sc.status + (size_t)t * 256 + tid;
    uint32_t prefix = 0;
    if (t == 0) {
      lb_store(my, epoch, kLbIncl, cnt);
    } else {
      lb_store(my, epoch, kLbAgg, cnt);
      prefix = rs_lookback(sc.status, t, tid, epoch, sc.status_word);
      lb_store(my, epoch, kLbIncl, prefix + cnt);
    }
    s_global[tid] = __ldg(&sc.base[pass * 256 + tid]) + prefix;
    {
      uint32_t ex;
      block_exclusive_scan<kRsThreads>(cnt, &ex, s_scan);
      s_local_base[tid] = ex;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kRsItems; ++j) {
      const uint32_t i = base + (uint32_t)(wid * 32 * kRsItems + j * 32 + lane);
      if (i < n) {
        const uint32_t d = (k[j] >> shift) & 255u;
        const uint32_t pos = s_local_base[d] + s_warp[wid][d] + r[j];
        s_keys[pos] = k[j];
        s_vals[pos] = v[j];
      }
    }
    __syncthreads();
    const uint32_t tn = min((uint32_t)kRsTile, n - base);
    for (uint32_t i = tid; i < tn; i += kRsThreads) {
      const uint32_t key = s_keys[i];
      const uint32_t d = (key >> shift) & 255u;
      const uint32_t gp = s_global[d] + (i - s_local_base[d]);
      kout[gp] = key;
      vout[gp] = s_vals[i];
    }
  }
  // the last CTA out clears the tile counter and advances the epoch
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(&sc.ctl[1], 1u) == gridDim.x - 1) {
      sc.ctl[0] = 0u;
      sc.ctl[1] = 0u;
      sc.ctl[2] = (epoch + 1u) & 0x3fffffffu;
      __threadfence();
    }
  }
}

// Sorts on bits [0, bits) (bits <= 32); the result lands in buffer index *which.
inline cudaError_t radix_sort(uint32_t *const keys[2], uint32_t *const vals[2], const uint32_t *n_ptr, uint32_t n_max,
                              int bits, const RadixScratch &sc, int *which, cudaStream_t s) {
  const int npass = (bits + 7) / 8;
  const int tiles = (int)((n_max + kRsTile - 1) / kRsTile);
  launch_k(rs_hist_kernel, radix_hist_grid(n_max), kRsThreads, 0, s, (const uint32_t *)keys[0], n_ptr, n_max, npass,
           sc);
  GS_LAUNCHED(1);
  int cur = 0;
  for (int p = 0; p < npass; ++p) {
    launch_k(rs_sweep_kernel, tiles < 1 ? 1 : tiles, kRsThreads, 0, s, (const uint32_t *)keys[cur],
             (const uint32_t *)vals[cur], keys[cur ^ 1], vals[cur ^ 1], n_ptr, n_max, p, sc);
    GS_LAUNCHED(1);
    cur ^= 1;
  }
  *which = cur;
  return cudaGetLastError();
}

}  // namespace gs
