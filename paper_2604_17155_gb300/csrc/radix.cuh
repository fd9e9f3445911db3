// radix.cuh -- depth order of one tile list in shared memory by a stable LSD radix sort (the "depth
// ordered list" of Eq. 2): by one warp (lists that fit its two buffers, no CTA barrier) or by
// one CTA of 256 threads (longer lists).
//
// A key is (float32 depth bits << 32) | Gaussian index. Depths are positive and finite, so their
// bit patterns order like the depths, and keys are unique. The sort takes 8-bit digits of
// (depth word - the tile's smallest depth word), from bit 0 up to the highest bit of the tile's
// depth-word range; each pass is stable, so the result is depth order with equal depths in input
// order. Input order is the binning's (atomic, so arbitrary), hence a tile in which two depths are
// equal is sorted again: first on the index word (over the tile's index range), then on the depth
// word. That gives the unique (depth, index) order for every tile, and the second sort runs only
// for tiles that have a tie.
//
// One pass: a histogram of the digits, an exclusive scan of it (the output offset of every digit),
// then the keys in position order, 32 at a time, each placed at its digit's offset plus its rank
// among the earlier keys with that digit. The lanes of a round that share a digit find each other
// through a per-warp table of lane masks in shared memory (every lane ORs its bit into the entry of
// its digit); the lowest of them then advances the digit's offset for the round.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace icgs {
namespace radix {

constexpr int kBins = 256;
constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint32_t key_word(unsigned long long k, bool hi) {
  return hi ? (uint32_t)(k >> 32) : (uint32_t)k;
}

__device__ __forceinline__ int bits_of(uint32_t x) { return x ? 32 - __clz(x) : 0; }

// The digit of key k in a pass over bits [shift, shift + 8) of (word - base).
__device__ __forceinline__ uint32_t digit(unsigned long long k, bool hi, uint32_t base, int shift) {
  return ((key_word(k, hi) - base) >> shift) & 0xFFu;
}

// Ranks the valid lanes' digits d among the lanes of the warp (peers: the valid lanes with the same
// digit, this lane included), through the warp's mask table m (zero before and after).
__device__ __forceinline__ uint32_t peers(uint32_t d, bool valid, uint32_t* m) {
  const int lane = threadIdx.x & 31;
  if (valid) atomicOr(&m[d], 1u << lane);
  __syncwarp();
  return m[d];
}

// ---------------------------------------------------------------------------------------------
// Warp sort: one warp, n <= the buffers' length (at most 65535). Each pass's scatter also counts
// the digits of the next pass, and the first pass's counts are taken while the keys are loaded:
// the digit of bits [0, 8) of (word - base) is (low byte of word - low byte of base) mod 256, so
// the histogram of the low bytes is the first pass's histogram rotated by the low byte of base.
struct WarpScratch {
  unsigned short count[2][kBins];  // histograms, then offsets, of the current and the next pass
  uint32_t match[kBins];           // lane masks; zero between rounds
};

struct Digit {
  bool hi;
  uint32_t base;
  int shift;
};

__device__ __forceinline__ void hist_add(unsigned short* c, uint32_t d) {
  atomicAdd(reinterpret_cast<unsigned int*>(c) + (d >> 1), 1u << ((d & 1u) * 16));
}

// Replaces the histogram in c (bin d stored at (d + rot) mod 256) by the exclusive offsets of the
// digits, bin d at d.
__device__ __forceinline__ void warp_scan(unsigned short* c, uint32_t rot) {
  const int lane = threadIdx.x & 31;
  uint32_t v[8], s = 0u;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    v[q] = c[(lane * 8 + q + rot) & (kBins - 1)];
    s += v[q];
  }
  uint32_t incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  __syncwarp();
  uint32_t run = incl - s;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    c[lane * 8 + q] = (unsigned short)run;
    run += v[q];
  }
  __syncwarp();
}

__device__ __forceinline__ void warp_zero(unsigned short* c) {
  const int lane = threadIdx.x & 31;
  reinterpret_cast<uint4*>(c)[lane] = make_uint4(0u, 0u, 0u, 0u);  // 32 x 16 bytes = 256 counts
  __syncwarp();
}

// The digit of the i-th pass of a sort that first takes n_lo passes on the index word (base lmin),
// then passes on the depth word (base hmin).
__device__ __forceinline__ Digit pass_digit(int i, int n_lo, uint32_t lmin, uint32_t hmin) {
  return i < n_lo ? Digit{false, lmin, 8 * i} : Digit{true, hmin, 8 * (i - n_lo)};
}

// Runs passes 0 .. total-1 (pass_digit), alternating between the buffers a and b from the one
// that holds the keys (np: passes so far, even: a). ws.count[cur] must hold pass 0's offsets.
__device__ __forceinline__ void warp_passes(unsigned long long* a, unsigned long long* b, int n, int& np, int& cur,
                                            int total, int n_lo, uint32_t lmin, uint32_t hmin, WarpScratch& ws) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = lanemask_lt();
  for (int i = 0; i < total; ++i, ++np) {
    const Digit dg = pass_digit(i, n_lo, lmin, hmin);
    const bool more = i + 1 < total;
    const Digit nx = pass_digit(i + 1, n_lo, lmin, hmin);
    const unsigned long long* src = np & 1 ? b : a;
    unsigned long long* dst = np & 1 ? a : b;
    unsigned short* cc = ws.count[cur];
    unsigned short* cn = ws.count[cur ^ 1];
    if (more) warp_zero(cn);
    for (int r0 = 0; r0 < n; r0 += 32) {
      const int pos = r0 + lane;
      const bool valid = pos < n;
      const unsigned long long k = valid ? src[pos] : 0ull;
      const uint32_t d = digit(k, dg.hi, dg.base, dg.shift);
      const uint32_t p = peers(d, valid, ws.match);
      const uint32_t c = cc[d];
      __syncwarp();
      if (valid) {
        if ((p & lt) == 0u) {  // the lowest peer advances the offset and clears the mask entry
          ws.match[d] = 0u;
          cc[d] = (unsigned short)(c + __popc(p));
        }
        dst[c + __popc(p & lt)] = k;
        if (more) hist_add(cn, digit(k, nx.hi, nx.base, nx.shift));
      }
      __syncwarp();
    }
    if (more) warp_scan(cn, 0u);
    cur ^= 1;
  }
}

// Rounds of odd-even transposition tried on a list in depth order before it is sorted again.
constexpr int kTieRounds = 8;

// r[0, n) is in depth order (ascending depth word) with equal depths in arbitrary order: sorts the
// runs of equal depths by the full key with odd-even transposition (a pair in two runs is in order
// already, so only pairs inside a run swap). Returns false when kTieRounds rounds did not settle
// every run; r then holds a permutation of the keys. One warp.
__device__ __forceinline__ bool warp_fix_ties(unsigned long long* r, int n) {
  const int lane = threadIdx.x & 31;
  for (int round = 0; round < kTieRounds; ++round) {
    bool sw = false;
#pragma unroll
    for (int phase = 0; phase < 2; ++phase) {
      for (int pos = 2 * lane + phase; pos + 1 < n; pos += 64) {
        const unsigned long long x = r[pos], y = r[pos + 1];
        if (x > y) {
          r[pos] = y;
          r[pos + 1] = x;
          sw = true;
        }
      }
      __syncwarp();
    }
    if (!__any_sync(kFull, sw)) return true;
  }
  return false;
}

// Sorts the n (1 < n <= 65535) keys at g with one warp; a and b are its two shared buffers of at
// least n keys, ws.match must be zero (it is again on return). Returns the buffer (a or b) that
// holds the sorted keys; WRITE also writes them back to g.
template <bool WRITE>
__device__ __forceinline__ const unsigned long long* warp_sort_keys(unsigned long long* g, int n, unsigned long long* a,
                                                                    unsigned long long* b, WarpScratch& ws) {
  const int lane = threadIdx.x & 31;
  // every key of the list in flight at once (asynchronous 8-byte copies into a), then one wait
  for (int pos = lane; pos < n; pos += 32) {
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(a + pos);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(g + pos) : "memory");
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  warp_zero(ws.count[0]);
  uint32_t hmin = 0xFFFFFFFFu, hmax = 0u, lmin = 0xFFFFFFFFu, lmax = 0u;
  for (int pos = lane; pos < n; pos += 32) {
    const unsigned long long k = a[pos];
    const uint32_t h = key_word(k, true), l = key_word(k, false);
    hist_add(ws.count[0], h & 0xFFu);
    hmin = min(hmin, h);
    hmax = max(hmax, h);
    lmin = min(lmin, l);
    lmax = max(lmax, l);
  }
  hmin = __reduce_min_sync(kFull, hmin);
  hmax = __reduce_max_sync(kFull, hmax);
  lmin = __reduce_min_sync(kFull, lmin);
  lmax = __reduce_max_sync(kFull, lmax);
  __syncwarp();
  const int n_hi = (bits_of(hmax - hmin) + 7) / 8, n_lo = (bits_of(lmax - lmin) + 7) / 8;
  int np = 0, cur = 0;  // passes so far (the keys are in b after an odd number, in a otherwise)
  bool tie = n_hi == 0;
  if (!tie) {
    warp_scan(ws.count[0], hmin & 0xFFu);
    warp_passes(a, b, n, np, cur, n_hi, 0, lmin, hmin, ws);
    const unsigned long long* r = np & 1 ? b : a;
    bool t = false;
    for (int pos = lane; pos < n; pos += 32) {  // write out; a tie means another sort and write
      const unsigned long long k = r[pos];
      if (WRITE) g[pos] = k;
      t |= pos > 0 && key_word(k, true) == key_word(r[pos - 1], true);
    }
    tie = __any_sync(kFull, t);
  }
  if (tie && n_hi > 0) {  // uniform over the warp: try the runs of equal depths by transposition
    unsigned long long* r = np & 1 ? b : a;
    if (warp_fix_ties(r, n)) {
      if (WRITE)
        for (int pos = lane; pos < n; pos += 32) g[pos] = r[pos];
      __syncwarp();
      return r;
    }
  }
  if (tie) {  // uniform over the warp: index order first, then depth order again
    const unsigned long long* r = np & 1 ? b : a;
    const Digit d0 = pass_digit(0, n_lo, lmin, hmin);
    warp_zero(ws.count[cur]);
    for (int pos = lane; pos < n; pos += 32) hist_add(ws.count[cur], digit(r[pos], d0.hi, d0.base, d0.shift));
    __syncwarp();
    warp_scan(ws.count[cur], 0u);
    warp_passes(a, b, n, np, cur, n_lo + n_hi, n_lo, lmin, hmin, ws);
    if (WRITE) {
      const unsigned long long* o = np & 1 ? b : a;
      for (int pos = lane; pos < n; pos += 32) g[pos] = o[pos];
    }
  }
  __syncwarp();
  return np & 1 ? b : a;
}

// Sorts the n (1 < n <= 65535) keys at g in place with one warp (warp_sort_keys, written back).
__device__ __forceinline__ void warp_sort(unsigned long long* g, int n, unsigned long long* a, unsigned long long* b,
                                          WarpScratch& ws) {
  warp_sort_keys<true>(g, n, a, b, ws);
}

// ---------------------------------------------------------------------------------------------
// Block sort: one CTA of kThreads threads, n <= 256 R. Warp w owns positions [32 R w, 32 R (w+1)),
// round r of it the 32 positions from 32 R w + 32 r; the block scan over (digit, warp) puts warp w
// before w + 1, so ranks follow position order.
constexpr int kThreads = 256;  // equal to kBins: thread t scans digit t
constexpr int kWarps = kThreads / 32;

struct BlockScratch {
  uint32_t count[kWarps * kBins];  // per-warp digit counts, then output offsets
  uint32_t match[kWarps * kBins];  // per-warp mask tables; zero between uses
  uint32_t warp_sum[kWarps];
  uint32_t range[4];               // min and max of the depth word, min and max of the index word
};

template <int R>
__device__ __forceinline__ void block_pass(const unsigned long long* src, unsigned long long* dst, int n, bool hi,
                                           uint32_t base, int shift, BlockScratch& sc) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t* cw = sc.count + w * kBins;
  uint32_t* mw = sc.match + w * kBins;
#pragma unroll
  for (int i = lane; i < kBins; i += 32) cw[i] = 0u;
  __syncwarp();
  const int first = w * 32 * R;
  const uint32_t lt = lanemask_lt();
  unsigned long long k[R];
  uint32_t rank[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int pos = first + 32 * r + lane;
    const bool valid = pos < n;
    k[r] = valid ? src[pos] : 0ull;
    const uint32_t d = digit(k[r], hi, base, shift);
    const uint32_t p = peers(d, valid, mw);
    const uint32_t c = cw[d];
    __syncwarp();
    if (valid && (p & lt) == 0u) {
      mw[d] = 0u;
      cw[d] = c + __popc(p);
    }
    rank[r] = c + __popc(p & lt);
    __syncwarp();
  }
  __syncthreads();
  {  // offsets: digit-major, warp-minor exclusive scan; thread t owns digit t
    const int t = threadIdx.x;
    uint32_t pre[kWarps];
    uint32_t tot = 0u;
#pragma unroll
    for (int v = 0; v < kWarps; ++v) {
      pre[v] = tot;
      tot += sc.count[v * kBins + t];
    }
    uint32_t incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) sc.warp_sum[w] = incl;
    __syncthreads();
    uint32_t off = incl - tot;
#pragma unroll
    for (int v = 0; v < kWarps; ++v)
      if (v < w) off += sc.warp_sum[v];
#pragma unroll
    for (int v = 0; v < kWarps; ++v) sc.count[v * kBins + t] = off + pre[v];
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (first + 32 * r + lane < n) dst[cw[digit(k[r], hi, base, shift)] + rank[r]] = k[r];
  __syncthreads();
}

// Sorts the n (1 < n <= 256 R) keys at g in place with the whole CTA; a and b are shared buffers
// of at least n keys, sc.match must be zero (it is again on return). All threads call it.
template <int R>
__device__ __forceinline__ void block_sort(unsigned long long* g, int n, unsigned long long* a, unsigned long long* b,
                                           BlockScratch& sc) {
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    sc.range[0] = 0xFFFFFFFFu;
    sc.range[1] = 0u;
    sc.range[2] = 0xFFFFFFFFu;
    sc.range[3] = 0u;
  }
  __syncthreads();
  uint32_t hmin = 0xFFFFFFFFu, hmax = 0u, lmin = 0xFFFFFFFFu, lmax = 0u;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int pos = r * kThreads + (int)threadIdx.x;
    if (pos < n) {
      const unsigned long long k = g[pos];
      a[pos] = k;
      hmin = min(hmin, key_word(k, true));
      hmax = max(hmax, key_word(k, true));
      lmin = min(lmin, key_word(k, false));
      lmax = max(lmax, key_word(k, false));
    }
  }
  hmin = __reduce_min_sync(kFull, hmin);
  hmax = __reduce_max_sync(kFull, hmax);
  lmin = __reduce_min_sync(kFull, lmin);
  lmax = __reduce_max_sync(kFull, lmax);
  if (lane == 0) {
    atomicMin(&sc.range[0], hmin);
    atomicMax(&sc.range[1], hmax);
    atomicMin(&sc.range[2], lmin);
    atomicMax(&sc.range[3], lmax);
  }
  __syncthreads();
  const uint32_t h0 = sc.range[0], l0 = sc.range[2];
  const int bh = bits_of(sc.range[1] - h0), bl = bits_of(sc.range[3] - l0);
  int np = 0;  // passes so far: the keys are in b after an odd number, in a otherwise
  for (int s = 0; s < bh; s += 8, ++np) block_pass<R>(np & 1 ? b : a, np & 1 ? a : b, n, true, h0, s, sc);
  bool tie = bh == 0;
  if (!tie) {
    const unsigned long long* r = np & 1 ? b : a;
    bool t = false;
    for (int pos = (int)threadIdx.x + 1; pos < n; pos += kThreads)
      t |= key_word(r[pos], true) == key_word(r[pos - 1], true);
    tie = __syncthreads_or(t) != 0;
  }
  if (tie && bh > 0) {  // uniform over the CTA: try the runs of equal depths by transposition
    unsigned long long* r = np & 1 ? b : a;
    bool fixed = false;
    for (int round = 0; round < kTieRounds && !fixed; ++round) {
      bool sw = false;
#pragma unroll
      for (int phase = 0; phase < 2; ++phase) {
        for (int pos = 2 * (int)threadIdx.x + phase; pos + 1 < n; pos += 2 * kThreads) {
          const unsigned long long x = r[pos], y = r[pos + 1];
          if (x > y) {
            r[pos] = y;
            r[pos + 1] = x;
            sw = true;
          }
        }
        __syncthreads();
      }
      fixed = __syncthreads_or(sw) == 0;
    }
    if (fixed) {
      for (int pos = threadIdx.x; pos < n; pos += kThreads) g[pos] = r[pos];
      __syncthreads();
      return;
    }
  }
  if (tie) {  // uniform over the CTA
    for (int s = 0; s < bl; s += 8, ++np) block_pass<R>(np & 1 ? b : a, np & 1 ? a : b, n, false, l0, s, sc);
    for (int s = 0; s < bh; s += 8, ++np) block_pass<R>(np & 1 ? b : a, np & 1 ? a : b, n, true, h0, s, sc);
  }
  const unsigned long long* r = np & 1 ? b : a;
  for (int pos = threadIdx.x; pos < n; pos += kThreads) g[pos] = r[pos];
  __syncthreads();
}

}  // namespace radix
}  // namespace icgs
