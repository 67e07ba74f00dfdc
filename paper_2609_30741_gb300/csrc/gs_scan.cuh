// Device-wide exclusive scan with a device-resident element count, so a pipeline
// can size its work on the GPU without reading counts back to the host.
#pragma once

#include "gs_internal.cuh"

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

// Pass 1: per-tile sums.
template <class Load>
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(Load ld, const uint32_t *n_ptr,
                                                                   uint32_t n_max, uint32_t *sums) {
  __shared__ uint32_t smem[32];
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
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Pass 2: exclusive scan of the tile sums in place (one block); total -> *total.
static __global__ void __launch_bounds__(1024) scan_sums_kernel(uint32_t *sums, int nblocks, uint32_t *total) {
  __shared__ uint32_t smem[32];
  const int per = (nblocks + 1023) / 1024;
  const int b0 = threadIdx.x * per;
  uint32_t acc = 0;
  for (int k = 0; k < per; ++k)
    if (b0 + k < nblocks) acc += sums[b0 + k];
  uint32_t ex;
  const uint32_t tot = block_exclusive_scan<1024>(acc, &ex, smem);
  for (int k = 0; k < per; ++k) {
    if (b0 + k < nblocks) {
      const uint32_t v = sums[b0 + k];
      sums[b0 + k] = ex;
      ex += v;
    }
  }
  if (threadIdx.x == 0 && total) *total = tot;
}

// Pass 3: per-element exclusive prefix; ap(i, prefix, value) for every i < n and
// ap.end(n, total) once.
template <class Load, class Apply>
__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(Load ld, Apply ap, const uint32_t *n_ptr,
                                                                  uint32_t n_max, const uint32_t *sums) {
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
  ex += sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const uint32_t i = base + threadIdx.x * kScanItems + k;
    if (i < n) ap(i, ex, loc[k]);
    ex += loc[k];
  }
  if (base + kScanTile >= n && threadIdx.x == 0) ap.end(n, sums[blockIdx.x] + tot);
}

template <class Load, class Apply>
cudaError_t scan_launch(Load ld, Apply ap, const uint32_t *n_ptr, uint32_t n_max, uint32_t *block_sums,
                        uint32_t *total_out, cudaStream_t s) {
  const int nblocks = (int)((n_max + kScanTile - 1) / kScanTile);
  if (nblocks == 0) {
    // still report an empty result
    scan_apply_kernel<<<1, kScanThreads, 0, s>>>(ld, ap, n_ptr, 0u, block_sums);
    GS_LAUNCHED(1);
    return cudaGetLastError();
  }
  scan_reduce_kernel<<<nblocks, kScanThreads, 0, s>>>(ld, n_ptr, n_max, block_sums);
  scan_sums_kernel<<<1, 1024, 0, s>>>(block_sums, nblocks, total_out);
  scan_apply_kernel<<<nblocks, kScanThreads, 0, s>>>(ld, ap, n_ptr, n_max, block_sums);
  GS_LAUNCHED(3);
  return cudaGetLastError();
}

}  // namespace gs
