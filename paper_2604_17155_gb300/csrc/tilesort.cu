// tilesort.cu -- depth order inside every screen tile (the "depth ordered list" of Eq. 2).
//
// After binning, each tile owns a contiguous slot range of 64-bit keys (float32 depth bits << 32 |
// Gaussian index); the keys are unique, so sorting them ascending gives depth order with ties in
// index order. Every sort here is the stable LSD radix sort of radix.cuh, in shared memory, and
// every list of a pass is sorted before the walks read it: lists of up to kWarpSortCap keys by a
// persistent kernel in which each warp sorts one tile at a time (k_sort_tiles, no CTA barrier);
// longer lists are queued. Lists of up to kMidCap keys go to two warps each (k_sort_pairs: a warp
// sort per half, then one merge-path merge); longer ones to one CTA each (k_sort_queued: up to
// kSortCap keys by the block radix sort at once, longer lists as sorted runs of kSortCap keys
// followed by merge-path merges between the slot range and a scratch range of the same place).
#include <cuda_runtime.h>

#include "icgs_internal.h"
#include "radix.cuh"

namespace icgs {

namespace {

constexpr int kSortThreads = radix::kThreads;  // CTA of the queued sort
constexpr int kWarpSortCap = 1024;             // longest list a warp sorts alone
constexpr int kWarpSortWarps = 4;              // warps per CTA of k_sort_tiles
constexpr int kWarpSortChunk = 4;              // tiles a warp claims per work-counter increment
constexpr int kMidCap = 2 * kWarpSortCap;       // queued lists up to this length: two warps each (k_sort_pairs)

struct WarpSortSmem {
  unsigned long long a[kWarpSortCap], b[kWarpSortCap];
  radix::WarpScratch sc;
};

__device__ __forceinline__ void tile_range(const uint32_t* tile_off, int t, uint32_t capacity,
                                           uint32_t& b, uint32_t& e) {
  b = min(tile_off[t], capacity);
  e = min(tile_off[t + 1], capacity);
  if (e < b) e = b;
}

// Number of elements of A among the first d outputs of merging A and B (keys are unique).
__device__ __forceinline__ int merge_path(const unsigned long long* A, int na, const unsigned long long* B,
                                          int nb, int d);

// Every tile list of the pass, by warps that claim kWarpSortChunk tiles at a time from the work
// counter: lists of up to kWarpSortCap keys are sorted in place by the claiming warp, longer ones
// queued for k_sort_queued.
__global__ void __launch_bounds__(32 * kWarpSortWarps) k_sort_tiles(const uint32_t* __restrict__ tile_off,
                                                                    unsigned long long* __restrict__ entries,
                                                                    uint32_t capacity, int ntiles,
                                                                    uint32_t* __restrict__ queue, DevStatus* status) {
  extern __shared__ __align__(16) unsigned long long s_dyn[];  // kWarpSortWarps x WarpSortSmem
  WarpSortSmem& m = reinterpret_cast<WarpSortSmem*>(s_dyn)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < radix::kBins; i += 32) m.sc.match[i] = 0u;
  __syncwarp();
  while (true) {
    uint32_t t0 = 0;
    if (lane == 0) t0 = atomicAdd(&status->sort_next, (uint32_t)kWarpSortChunk);
    t0 = __shfl_sync(0xFFFFFFFFu, t0, 0);
    if (t0 >= (uint32_t)ntiles) break;
    const int t1 = min(ntiles, (int)t0 + kWarpSortChunk);
    {  // start the chunk's keys towards L2 while the first list is sorted
      uint32_t cb, ce, cx;
      tile_range(tile_off, (int)t0, capacity, cb, cx);
      tile_range(tile_off, t1 - 1, capacity, cx, ce);
      const char* p0 = reinterpret_cast<const char*>(entries + cb);
      const size_t bytes = (size_t)(ce - cb) * sizeof(unsigned long long);
      for (size_t o = (size_t)lane * 128; o < bytes; o += 32 * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(p0 + o));
    }
    for (int t = (int)t0; t < t1; ++t) {
      uint32_t b, e;
      tile_range(tile_off, t, capacity, b, e);
      const int n = (int)(e - b);
      if (n <= 1) continue;
      if (n > kWarpSortCap) {  // queued: up to kMidCap keys from the front, longer lists from the back
        if (lane == 0) {
          if (n <= kMidCap) queue[atomicAdd(&status->big_tiles, 1u)] = (uint32_t)t;
          else queue[ntiles - 1 - (int)atomicAdd(&status->long_tiles, 1u)] = (uint32_t)t;
        }
        continue;
      }
      radix::warp_sort(entries + b, n, m.a, m.b, m.sc);
    }
  }
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

// Merges the sorted runs A[0, na) and B[0, nb) into out[0, na + nb) with the CTA's NT threads,
// each producing an equal share of the outputs (merge path).
template <int NT>
__device__ __forceinline__ void merge_runs(const unsigned long long* A, int na, const unsigned long long* B, int nb,
                                           unsigned long long* out, int t) {
  const int n = na + nb;
  const int per = (n + NT - 1) / NT;
  const int d0 = min(n, t * per), d1 = min(n, d0 + per);
  if (d0 >= d1) return;
  int ia = merge_path(A, na, B, nb, d0);
  int ib = d0 - ia;
  for (int d = d0; d < d1; ++d) {
    const bool takeA = ib >= nb || (ia < na && A[ia] < B[ib]);
    out[d] = takeA ? A[ia++] : B[ib++];
  }
}

// Sorts the queued lists of 1025..kMidCap keys (queue[0, big_tiles)), a grid-stride loop with two
// warps per list: warp w sorts one half (at most kWarpSortCap keys) with the warp radix sort in its
// part of two shared pools, the halves are gathered into the first pool, and a merge-path merge
// (every thread an equal share of the outputs) writes the list back to its slot range.
__global__ void __launch_bounds__(64) k_sort_pairs(const uint32_t* __restrict__ tile_off,
                                                   unsigned long long* __restrict__ entries, uint32_t capacity,
                                                   const uint32_t* __restrict__ queue, const DevStatus* status) {
  extern __shared__ __align__(16) unsigned long long s_dyn[];  // pools P0, P1 of 2 x kWarpSortCap keys, scratch
  unsigned long long* P0 = s_dyn;
  unsigned long long* P1 = s_dyn + 2 * kWarpSortCap;
  radix::WarpScratch& sc = reinterpret_cast<radix::WarpScratch*>(P1 + 2 * kWarpSortCap)[threadIdx.x >> 5];
  __shared__ int s_len[2];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = lane; i < radix::kBins; i += 32) sc.match[i] = 0u;
  __syncwarp();
  const uint32_t count = status->big_tiles;
  for (uint32_t q = blockIdx.x; q < count; q += gridDim.x) {
    uint32_t b, e;
    tile_range(tile_off, queue[q], capacity, b, e);
    const int n = (int)(e - b);
    const int h = (n + 1) / 2;
    const int lo = min(n, w * h), len = min(h, n - lo);
    unsigned long long* a = P0 + w * kWarpSortCap;
    unsigned long long* bb = P1 + w * kWarpSortCap;
    if (len > 1) {
      const unsigned long long* run = radix::warp_sort_keys<false>(entries + b + lo, len, a, bb, sc);
      if (run != a) {  // gather the half into the first pool
        for (int pos = lane; pos < len; pos += 32) a[pos] = run[pos];
        __syncwarp();
      }
    } else if (len == 1 && lane == 0) {
      a[0] = entries[b + lo];
    }
    if (lane == 0) s_len[w] = max(0, len);
    __syncthreads();
    merge_runs<64>(P0, s_len[0], P0 + kWarpSortCap, s_len[1], entries + b, threadIdx.x);
    __syncthreads();
  }
}

// Sorts the m (1 < m <= kSortCap) keys at g in place with the block radix sort sized to m.
__device__ __forceinline__ void block_sort_list(unsigned long long* g, int m, unsigned long long* a,
                                                unsigned long long* b, radix::BlockScratch& sc) {
  if (m <= 1024) radix::block_sort<4>(g, m, a, b, sc);
  else if (m <= 2048) radix::block_sort<8>(g, m, a, b, sc);
  else if (m <= 3072) radix::block_sort<12>(g, m, a, b, sc);
  else radix::block_sort<16>(g, m, a, b, sc);
}

// Sorts the queued lists of more than kMidCap keys (the last long_tiles entries of the queue) in
// place, a grid-stride loop. A list of up to kSortCap keys is sorted at once by the block radix
// sort; a longer one as runs of kSortCap keys, then pairwise merge-path merges ping-ponging between
// its slot range and the same range of the scratch array.
__global__ void __launch_bounds__(kSortThreads, 2) k_sort_queued(const uint32_t* __restrict__ tile_off,
                                                                 unsigned long long* __restrict__ entries,
                                                                 unsigned long long* __restrict__ scratch,
                                                                 uint32_t capacity, const uint32_t* __restrict__ queue,
                                                                 int ntiles, const DevStatus* status) {
  constexpr int CAP = kSortCap;
  extern __shared__ __align__(16) unsigned long long s_dyn[];  // 2 x CAP keys
  __shared__ radix::BlockScratch sc;
  for (int i = threadIdx.x; i < radix::kWarps * radix::kBins; i += kSortThreads) sc.match[i] = 0u;
  __syncthreads();
  const uint32_t count = status->long_tiles;
  for (uint32_t q = blockIdx.x; q < count; q += gridDim.x) {
    uint32_t b, e;
    tile_range(tile_off, queue[ntiles - 1 - (int)q], capacity, b, e);
    const int n = (int)(e - b);
    for (int r0 = 0; r0 < n; r0 += CAP) {  // sorted runs (the whole list when it fits)
      const int m = min(CAP, n - r0);
      if (m > 1) block_sort_list(entries + b + r0, m, s_dyn, s_dyn + CAP, sc);
    }
    if (n <= CAP) continue;  // uniform
    unsigned long long* src = entries + b;
    unsigned long long* dst = scratch + b;
    for (int width = CAP; width < n; width <<= 1) {
      for (int lo = 0; lo < n; lo += 2 * width) {
        const int na = min(width, n - lo);
        const int nb = max(0, min(width, n - lo - width));
        const unsigned long long* A = src + lo;
        const unsigned long long* Bp = src + lo + na;
        const int tot = na + nb;
        const int per = (tot + kSortThreads - 1) / kSortThreads;
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
      for (int k = threadIdx.x; k < n; k += kSortThreads) entries[b + k] = src[k];
    __syncthreads();
  }
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

}  // namespace

// Orders every tile list of the pass: the warp-per-list kernel, then the queued long lists.
void launch_tile_sort(const Problem& p, int cb, const Workspace& ws, cudaStream_t s) {
  const int ntiles = cb * p.tiles;
  const int sms = sm_count();
  cudaMemsetAsync(&ws.status->big_tiles, 0, 3 * sizeof(uint32_t), s);  // big_tiles, sort_next, long_tiles
  const int smem = kWarpSortWarps * (int)sizeof(WarpSortSmem);
  cudaFuncSetAttribute(k_sort_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sort_tiles, 32 * kWarpSortWarps, smem);
  const int grid = sms * (per_sm > 0 ? per_sm : 1);
  k_sort_tiles<<<grid, 32 * kWarpSortWarps, smem, s>>>(ws.tile_off, reinterpret_cast<unsigned long long*>(ws.entries),
                                                       p.capacity, ntiles, ws.big_list, ws.status);
  unsigned long long* entries = reinterpret_cast<unsigned long long*>(ws.entries);
  unsigned long long* scratch = reinterpret_cast<unsigned long long*>(ws.entries_tmp);
  const int psmem = 2 * (2 * kWarpSortCap * (int)sizeof(unsigned long long) + (int)sizeof(radix::WarpScratch));
  cudaFuncSetAttribute(k_sort_pairs, cudaFuncAttributeMaxDynamicSharedMemorySize, psmem);
  int per_sm2 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, k_sort_pairs, 64, psmem);
  k_sort_pairs<<<sms * (per_sm2 > 0 ? per_sm2 : 1), 64, psmem, s>>>(ws.tile_off, entries, p.capacity, ws.big_list,
                                                                    ws.status);
  const int qsmem = 2 * kSortCap * (int)sizeof(unsigned long long);
  cudaFuncSetAttribute(k_sort_queued, cudaFuncAttributeMaxDynamicSharedMemorySize, qsmem);
  k_sort_queued<<<sms * 2, kSortThreads, qsmem, s>>>(ws.tile_off, entries, scratch, p.capacity, ws.big_list, ntiles,
                                                     ws.status);
  note_launches(3);
}

}  // namespace icgs
