// tilesort.cu -- depth order inside every screen tile (the "depth ordered list" of Eq. 2).
//
// After binning, each tile owns a contiguous slot range of 64-bit keys (float32 depth bits << 32 |
// Gaussian index); the keys are unique, so sorting them ascending gives depth order with ties in
// index order. Lists up to kSortCap keys are bitonic-sorted in shared memory by one CTA per tile;
// longer lists are queued and sorted by k_sort_long: shared-memory runs of kSortCap keys, then
// merge-path merges between the slot range and a scratch range of the same place.
#include <cuda_runtime.h>

#include "icgs_internal.h"
#include "walk.cuh"

namespace icgs {

namespace {

using walk::bitonic_sort_smem;

constexpr int kSortThreads = 256;
constexpr int kLongThreads = 1024;
constexpr unsigned long long kPad = ~0ull;

__device__ __forceinline__ void tile_range(const uint32_t* tile_off, int t, uint32_t capacity,
                                           uint32_t& b, uint32_t& e) {
  b = min(tile_off[t], capacity);
  e = min(tile_off[t + 1], capacity);
  if (e < b) e = b;
}

__global__ void __launch_bounds__(kSortThreads) k_sort_tiles(const uint32_t* __restrict__ tile_off,
                                                             unsigned long long* __restrict__ entries,
                                                             uint32_t capacity, uint32_t* __restrict__ big_list,
                                                             DevStatus* status) {
  __shared__ unsigned long long s[kSortCap];
  uint32_t b, e;
  tile_range(tile_off, blockIdx.x, capacity, b, e);
  const int n = (int)(e - b);
  if (n <= 1) return;
  if (n > kSortCap) {
    if (threadIdx.x == 0) big_list[atomicAdd(&status->big_tiles, 1u)] = blockIdx.x;
    return;
  }
  walk::sort_keys_block<kSortCap / kSortThreads>(entries + b, (uint32_t)n, s);
  for (int k = threadIdx.x; k < n; k += kSortThreads) entries[b + k] = s[k];
}

// Number of elements of A among the first d outputs of merging A and B (keys are unique).
__device__ __forceinline__ int merge_path(const unsigned long long* A, int na, const unsigned long long* B,
                                          int nb, int d) {
  int lo = max(0, d - nb), hi = min(d, na);
  while (lo < hi) {
    const int i = (lo + hi) >> 1;
    if (A[i] < B[d - 1 - i]) lo = i + 1;
    else hi = i;
  }
  return lo;
}

__global__ void __launch_bounds__(kLongThreads) k_sort_long(const uint32_t* __restrict__ tile_off,
                                                            unsigned long long* __restrict__ entries,
                                                            unsigned long long* __restrict__ scratch,
                                                            uint32_t capacity,
                                                            const uint32_t* __restrict__ big_list,
                                                            const DevStatus* status) {
  __shared__ unsigned long long s[kSortCap];
  const uint32_t count = status->big_tiles;
  for (uint32_t q = blockIdx.x; q < count; q += gridDim.x) {
    uint32_t b, e;
    tile_range(tile_off, big_list[q], capacity, b, e);
    const int n = (int)(e - b);
    // 1. sorted runs of kSortCap in shared memory
    for (int r0 = 0; r0 < n; r0 += kSortCap) {
      const int m = min(kSortCap, n - r0);
      for (int k = threadIdx.x; k < kSortCap; k += kLongThreads) s[k] = k < m ? entries[b + r0 + k] : kPad;
      __syncthreads();
      bitonic_sort_smem<kLongThreads>(s, kSortCap);
      for (int k = threadIdx.x; k < m; k += kLongThreads) entries[b + r0 + k] = s[k];
      __syncthreads();
    }
    // 2. pairwise merges, ping-ponging between the slot range and the scratch range
    unsigned long long* src = entries + b;
    unsigned long long* dst = scratch + b;
    for (int width = kSortCap; width < n; width <<= 1) {
      for (int lo = 0; lo < n; lo += 2 * width) {
        const int na = min(width, n - lo);
        const int nb = max(0, min(width, n - lo - width));
        const unsigned long long* A = src + lo;
        const unsigned long long* Bp = src + lo + na;
        const int tot = na + nb;
        const int per = (tot + kLongThreads - 1) / kLongThreads;
        const int d0 = min(tot, (int)threadIdx.x * per), d1 = min(tot, d0 + per);
        if (d0 < d1) {
          int ia = merge_path(A, na, Bp, nb, d0);
          int ib = d0 - ia;
          for (int d = d0; d < d1; ++d) {
            const bool takeA = ib >= nb || (ia < na && A[ia] < Bp[ib]);
            dst[lo + d] = takeA ? A[ia++] : Bp[ib++];
          }
        }
      }
      __syncthreads();
      unsigned long long* tmp = src;
      src = dst;
      dst = tmp;
    }
    if (src != entries + b)
      for (int k = threadIdx.x; k < n; k += kLongThreads) entries[b + k] = src[k];
    __syncthreads();
  }
}

// Queues the tiles whose list is longer than the walks sort in shared memory (kWalkSortCap).
__global__ void __launch_bounds__(kSortThreads) k_queue_long_tiles(const uint32_t* __restrict__ tile_off, int ntiles,
                                                                   uint32_t capacity, uint32_t* __restrict__ big_list,
                                                                   DevStatus* status) {
  const int t = blockIdx.x * kSortThreads + threadIdx.x;
  if (t >= ntiles) return;
  uint32_t b, e;
  tile_range(tile_off, t, capacity, b, e);
  if (e - b > (uint32_t)walk::kWalkSortCap) big_list[atomicAdd(&status->big_tiles, 1u)] = (uint32_t)t;
}

}  // namespace

// sort_all: order every tile list here (walks that read the lists from global memory); otherwise
// only the lists longer than the walks' shared-memory sort (kWalkSortCap).
void launch_tile_sort(const Problem& p, int cb, bool sort_all, const Workspace& ws, cudaStream_t s) {
  static_assert(walk::kWalkSortCap <= kSortCap, "the long-list sort takes everything the walks do not");
  const int ntiles = cb * p.tiles;
  cudaMemsetAsync(&ws.status->big_tiles, 0, sizeof(uint32_t), s);
  if (sort_all)
    k_sort_tiles<<<ntiles, kSortThreads, 0, s>>>(ws.tile_off, reinterpret_cast<unsigned long long*>(ws.entries),
                                                 p.capacity, ws.big_list, ws.status);
  else
    k_queue_long_tiles<<<(ntiles + kSortThreads - 1) / kSortThreads, kSortThreads, 0, s>>>(
        ws.tile_off, ntiles, p.capacity, ws.big_list, ws.status);
  k_sort_long<<<152, kLongThreads, 0, s>>>(ws.tile_off, reinterpret_cast<unsigned long long*>(ws.entries),
                                           reinterpret_cast<unsigned long long*>(ws.entries_tmp), p.capacity,
                                           ws.big_list, ws.status);
  note_launches(2);
}

}  // namespace icgs
