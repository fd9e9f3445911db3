// tilesort.cu -- depth order inside every screen tile (the "depth ordered list" of Eq. 2).
//
// After binning, each tile owns a contiguous slot range of 64-bit keys (float32 depth bits << 32 |
// Gaussian index); the keys are unique, so sorting them ascending gives depth order with ties in
// index order. For the tensor-core walk every list is sorted here, one CTA per tile (k_sort_tiles):
// up to 1024 keys with the walks' register/shuffle bitonic network, 1025..kSortCap keys as sorted
// runs of 1024 merged in shared memory (no padding to a power of two). The CUDA-core walks sort
// lists of up to kWalkSortCap keys themselves; the longer ones are queued (k_queue_tiles) and sorted
// by a persistent kernel (k_sort_queued): up to kSortCap keys with a bitonic network over keys held
// in registers (blocked, 8 or 16 a thread, from 1025 keys), longer lists as runs of kSortCap keys
// followed by merge-path merges between the slot range and a scratch range of the same place.
#include <cuda_runtime.h>

#include "icgs_internal.h"
#include "walk.cuh"

namespace icgs {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortGrid = 152 * 6;  // CTAs of the queued sort (a grid-stride loop; three per SM are resident)

__device__ __forceinline__ void tile_range(const uint32_t* tile_off, int t, uint32_t capacity,
                                           uint32_t& b, uint32_t& e) {
  b = min(tile_off[t], capacity);
  e = min(tile_off[t + 1], capacity);
  if (e < b) e = b;
}

// Ascending bitonic sort of the len (<= P = 256 E) keys at g, written to dst[0, len). The keys are
// held blocked: thread t holds keys t E .. t E + E - 1 in v (padding ~0 beyond len). Strides below
// E are exchanges inside a thread, strides E .. 16 E warp shuffles (the partner is thread
// t ^ (stride / E)), and only the 6 stages with strides of 32 E or more go through shared memory
// (s, P + P / E keys: one pad slot every E keys keeps those accesses free of bank conflicts).
template <int E>
__device__ __forceinline__ void sort_blocked(const unsigned long long* __restrict__ g, int len,
                                             unsigned long long* s, unsigned long long* __restrict__ dst) {
  constexpr int P = kSortThreads * E;
  const int t = threadIdx.x;
  const int i0 = t * E;
  unsigned long long v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) v[e] = i0 + e < len ? g[i0 + e] : ~0ull;
  auto pad = [](int i) { return i + i / E; };
  for (int k = 2; k <= P; k <<= 1) {
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      if (jj < E) {
#pragma unroll
        for (int m = 1; m < E; m <<= 1) {  // m = jj, unrolled so that v is indexed statically
          if (m != jj) continue;
#pragma unroll
          for (int e = 0; e < E; ++e) {
            if (e & m) continue;
            const unsigned long long a = v[e], b = v[e | m];
            const bool up = ((i0 + e) & k) == 0;
            const bool swap = (a > b) == up;
            v[e] = swap ? b : a;
            v[e | m] = swap ? a : b;
          }
        }
      } else if (jj < 32 * E) {
        const int lm = jj / E;
#pragma unroll
        for (int e = 0; e < E; ++e)
          v[e] = walk::cmpx_keep(v[e], __shfl_xor_sync(0xFFFFFFFFu, v[e], lm), i0 + e, jj, k);
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) s[pad(i0 + e)] = v[e];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = walk::cmpx_keep(v[e], s[pad((i0 + e) ^ jj)], i0 + e, jj, k);
        __syncthreads();
      }
    }
  }
#pragma unroll
  for (int e = 0; e < E; ++e)
    if (i0 + e < len) dst[i0 + e] = v[e];
}

// Sorts len (<= kSortCap) keys from g into dst: up to 1024 keys through the walks' shared-memory
// sort, longer lists blocked (sort_blocked with 8 or 16 keys a thread). g may equal dst.
__device__ __forceinline__ void sort_list(const unsigned long long* g, int len, unsigned long long* s,
                                          unsigned long long* dst) {
  if (len > 2048) {
    sort_blocked<16>(g, len, s, dst);
  } else if (len > 1024) {
    sort_blocked<8>(g, len, s, dst);
  } else {
    walk::sort_keys_block<4>(g, (uint32_t)len, s);
    for (int k = threadIdx.x; k < len; k += kSortThreads) dst[k] = s[k];
  }
  __syncthreads();
}

// Queues every tile whose list has more than min_len keys (one thread per tile; one counter
// atomic per warp).
__global__ void __launch_bounds__(kSortThreads) k_queue_tiles(const uint32_t* __restrict__ tile_off, int ntiles,
                                                              uint32_t capacity, int min_len,
                                                              uint32_t* __restrict__ queue, DevStatus* status) {
  const int t = blockIdx.x * kSortThreads + threadIdx.x;
  bool want = false;
  if (t < ntiles) {
    uint32_t b, e;
    tile_range(tile_off, t, capacity, b, e);
    const uint32_t n = e - b;
    want = n > 1u && n > (uint32_t)min_len;
  }
  const uint32_t ballot = __ballot_sync(0xFFFFFFFFu, want);
  if (!ballot) return;  // uniform per warp
  const int lane = threadIdx.x & 31;
  uint32_t base = 0;
  if (lane == 0) base = atomicAdd(&status->big_tiles, (uint32_t)__popc(ballot));
  base = __shfl_sync(0xFFFFFFFFu, base, 0);
  if (want) queue[base + __popc(ballot & ((1u << lane) - 1u))] = (uint32_t)t;
}

// Number of elements of A among the first d outputs of merging A and B (keys are unique).
__device__ __forceinline__ int merge_path(const unsigned long long* A, int na, const unsigned long long* B,
                                          int nb, int d);

// Sorts len (1024 < len <= kSortCap) keys from g into dst without padding the list to a power of
// two: runs of 1024 keys are sorted in shared memory by the register/shuffle network of the walks,
// then merged pairwise (merge path: every thread produces an equal share of each merge's outputs)
// between the two shared buffers s0 and s1 (kSortCap keys each).
__device__ __forceinline__ void sort_runs_merge(const unsigned long long* g, int len, unsigned long long* s0,
                                                unsigned long long* s1, unsigned long long* __restrict__ dst) {
  constexpr int kRun = 1024;
  for (int r0 = 0; r0 < len; r0 += kRun) walk::sort_keys_block<4>(g + r0, (uint32_t)min(kRun, len - r0), s0 + r0);
  unsigned long long* src = s0;
  unsigned long long* out = s1;
  for (int width = kRun; width < len; width <<= 1) {
    for (int lo = 0; lo < len; lo += 2 * width) {
      const int na = min(width, len - lo);
      const int nb = max(0, min(width, len - lo - width));
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
          out[lo + d] = takeA ? A[ia++] : Bp[ib++];
        }
      }
    }
    __syncthreads();
    unsigned long long* t = src;
    src = out;
    out = t;
  }
  for (int k = threadIdx.x; k < len; k += kSortThreads) dst[k] = src[k];
  __syncthreads();
}

// Every tile list: sorted in place when it has at most kSortCap keys (one CTA per tile), queued
// for k_sort_queued when longer. Up to 1024 keys: the walks' shared-memory network; longer:
// sorted runs merged in shared memory.
__global__ void __launch_bounds__(kSortThreads, 3) k_sort_tiles(const uint32_t* __restrict__ tile_off,
                                                             unsigned long long* __restrict__ entries,
                                                             uint32_t capacity, uint32_t* __restrict__ queue,
                                                             DevStatus* status) {
  extern __shared__ unsigned long long s_dyn[];  // 2 x kSortCap keys
  uint32_t b, e;
  tile_range(tile_off, blockIdx.x, capacity, b, e);
  const int n = (int)(e - b);
  if (n <= 1) return;
  if (n > kSortCap) {
    if (threadIdx.x == 0) queue[atomicAdd(&status->big_tiles, 1u)] = blockIdx.x;
    return;
  }
  if (n > 1024) {
    sort_runs_merge(entries + b, n, s_dyn, s_dyn + kSortCap, entries + b);
  } else {
    walk::sort_keys_block<4>(entries + b, (uint32_t)n, s_dyn);
    for (int k = threadIdx.x; k < n; k += kSortThreads) entries[b + k] = s_dyn[k];
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

// Sorts the queued tile lists in place, a grid-stride loop over the queue. A list of up to
// kSortCap keys is sorted in shared memory with the register/shuffle bitonic network sized to it;
// a longer one as runs of kSortCap keys, then pairwise merge-path merges ping-ponging between its
// slot range and the same range of the scratch array.
__global__ void __launch_bounds__(kSortThreads, 3) k_sort_queued(const uint32_t* __restrict__ tile_off,
                                                              unsigned long long* __restrict__ entries,
                                                              unsigned long long* __restrict__ scratch,
                                                              uint32_t capacity, const uint32_t* __restrict__ queue,
                                                              const DevStatus* status) {
  __shared__ unsigned long long s[kSortCap + kSortCap / 16];
  const uint32_t count = status->big_tiles;
  for (uint32_t q = blockIdx.x; q < count; q += gridDim.x) {
    uint32_t b, e;
    tile_range(tile_off, queue[q], capacity, b, e);
    const int n = (int)(e - b);
    for (int r0 = 0; r0 < n; r0 += kSortCap) {  // sorted runs (the whole list when it fits)
      const int m = min(kSortCap, n - r0);
      sort_list(entries + b + r0, m, s, entries + b + r0);
    }
    if (n <= kSortCap) continue;  // uniform
    unsigned long long* src = entries + b;
    unsigned long long* dst = scratch + b;
    for (int width = kSortCap; width < n; width <<= 1) {
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

}  // namespace

// sort_all: order every tile list here (walks that read the lists from global memory): one CTA per
// tile, lists longer than kSortCap queued. Otherwise only the lists longer than the walks'
// shared-memory sort (kWalkSortCap), queued and sorted by the persistent kernel.
void launch_tile_sort(const Problem& p, int cb, bool sort_all, const Workspace& ws, cudaStream_t s) {
  const int ntiles = cb * p.tiles;
  cudaMemsetAsync(&ws.status->big_tiles, 0, sizeof(uint32_t), s);
  if (sort_all) {
    const int smem = 2 * kSortCap * (int)sizeof(unsigned long long);
    cudaFuncSetAttribute(k_sort_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k_sort_tiles<<<ntiles, kSortThreads, smem, s>>>(ws.tile_off, reinterpret_cast<unsigned long long*>(ws.entries),
                                                    p.capacity, ws.big_list, ws.status);
  }
  else
    k_queue_tiles<<<(ntiles + kSortThreads - 1) / kSortThreads, kSortThreads, 0, s>>>(
        ws.tile_off, ntiles, p.capacity, walk::kWalkSortCap, ws.big_list, ws.status);
  k_sort_queued<<<kSortGrid, kSortThreads, 0, s>>>(ws.tile_off, reinterpret_cast<unsigned long long*>(ws.entries),
                                                   reinterpret_cast<unsigned long long*>(ws.entries_tmp), p.capacity,
                                                   ws.big_list, ws.status);
  note_launches(2);
}

}  // namespace icgs
