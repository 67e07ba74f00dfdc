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

// Pass 1: per-tile sums. The last block to finish (counted on *ticket, which
// it resets to 0) then scans the tile sums in place, so no block ever waits on
// another.
template <class Load>
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(Load ld, const uint32_t *n_ptr,
                                                                   uint32_t n_max, uint32_t *sums,
                                                                   uint32_t *ticket, uint32_t *total_out) {
  griddep_wait();
  __shared__ uint32_t smem[32];
  __shared__ uint32_t s_last;
  const uint32_t n = load_n(n_ptr, n_max);
  const uint32_t base = blockIdx.x * (uint32_t)kScanTile;
  uint32_t acc = 0;
  if (base < n) {
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      const uint32_t i = base + k * kScanThreads + threadIdx.x;  // coalesced
      if (i < n) acc += ld(i);
    }
  }
  uint32_t ex;
  const uint32_t tot = block_exclusive_scan<kScanThreads>(acc, &ex, smem);
  if (threadIdx.x == 0) {
    sums[blockIdx.x] = tot;
    __threadfence();
    s_last = atomicAdd(ticket, 1u) == gridDim.x - 1 ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int nb = (int)gridDim.x;
  const int per = (nb + kScanThreads - 1) / kScanThreads;
  const int b0 = threadIdx.x * per;
  uint32_t a2 = 0;
  for (int k = 0; k < per; ++k)
    if (b0 + k < nb) a2 += __ldcg(sums + b0 + k);
  uint32_t ex2;
  const uint32_t all = block_exclusive_scan<kScanThreads>(a2, &ex2, smem);
  for (int k = 0; k < per; ++k) {
    if (b0 + k < nb) {
      const uint32_t v = __ldcg(sums + b0 + k);
      sums[b0 + k] = ex2;
      ex2 += v;
    }
  }
  if (threadIdx.x == 0) {
    if (total_out) *total_out = all;
    *ticket = 0u;
  }
}

// Pass 2: per-element exclusive prefix; ap(i, prefix, value) for every i < n and
// ap.end(n, total) once.
template <class Load, class Apply>
__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(Load ld, Apply ap, const uint32_t *n_ptr,
                                                                  uint32_t n_max, const uint32_t *sums) {
  griddep_wait();
  __shared__ uint32_t smem[32];
  __shared__ uint32_t vals[kScanTile];
  const uint32_t n = load_n(n_ptr, n_max);
  const uint32_t base = blockIdx.x * (uint32_t)kScanTile;
  if (base >= n) {
    if (blockIdx.x == 0) ap.end(n, 0u);
    return;
  }
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const uint32_t i = base + k * kScanThreads + threadIdx.x;
    vals[k * kScanThreads + threadIdx.x] = i < n ? ld(i) : 0u;
  }
  __syncthreads();
  // each thread owns kScanItems consecutive elements
  uint32_t loc[kScanItems], acc = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    loc[k] = vals[threadIdx.x * kScanItems + k];
    acc += loc[k];
  }
  uint32_t ex;
  const uint32_t tot = block_exclusive_scan<kScanThreads>(acc, &ex, smem);
  if (sums) ex += sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const uint32_t i = base + threadIdx.x * kScanItems + k;
    if (i < n) ap(i, ex, loc[k]);
    ex += loc[k];
  }
  if (base + kScanTile >= n && threadIdx.x == 0) ap.end(n, (sums ? sums[blockIdx.x] : 0u) + tot);
}

// block_sums: one word per tile of kScanTile elements (+1); ticket: one word that
// is 0 between scans (the scans of one workspace run one after another).
template <class Load, class Apply>
cudaError_t scan_launch(Load ld, Apply ap, const uint32_t *n_ptr, uint32_t n_max, uint32_t *block_sums,
                        uint32_t *ticket, uint32_t *total_out, cudaStream_t s) {
  const int nblocks = (int)((n_max + kScanTile - 1) / kScanTile);
  if (nblocks <= 1) {
    // one tile (or an empty result): its prefix starts at 0
    launch_k(scan_apply_kernel<Load, Apply>, 1, kScanThreads, 0, s, ld, ap, n_ptr, n_max, (const uint32_t *)nullptr);
    GS_LAUNCHED(1);
    return cudaGetLastError();
  }
  launch_k(scan_reduce_kernel<Load>, nblocks, kScanThreads, 0, s, ld, n_ptr, n_max, block_sums, ticket, total_out);
  launch_k(scan_apply_kernel<Load, Apply>, nblocks, kScanThreads, 0, s, ld, ap, n_ptr, n_max, block_sums);
  GS_LAUNCHED(2);
  return cudaGetLastError();
}

}  // namespace gs
