// blend.cu -- the per-tile front-to-back walks (Eq. 2, Eq. 4-6), one CTA per 16x16 screen tile:
// 256 threads with one pixel each, or (the kernels named ...2, for up to 3 or 4 channels) 128
// threads with two pixels each.
//
//   k_blend_accumulate  colorize: for every (pixel, Gaussian) blend weight w = alpha T (Eq. 4)
//   (2: <= 3 channels)  accumulate V = sum w (Eq. 5) and S_k = sum w t_k (Eq. 6 numerator). The
//                       tile's pixels are reduced per Gaussian inside each warp (a halving
//                       butterfly that leaves value v's warp sum in lane v * 32/NP) and across
//                       warps with shared-memory atomics; then ONE global atomic group per
//                       (Gaussian, tile) lands in the per-(camera, Gaussian) accumulator.
//   k_blend_render      render: img_k = sum w C_k (Eq. 1-3) with C from the payload.
//   (2: <= 4 channels)
//   k_blend_adjoint     gradient: dL/dt_k = sum w a_k and, per Gaussian, dL/do = sum over pixels of
//   (2: <= 4 channels)  (g T - sum_{n>m} g_n w_n / (1-alpha)) * alpha/o with g = beta + a . t.
//
// Warp w of a CTA covers the 8x4 pixel block ((w&1)*8, (w>>1)*4) of the tile (8x8 blocks at
// ((w&1)*8, (w>>1)*8) in the two-pixel walks). A warp skips a Gaussian whose padded support box
// misses its block (a warp-uniform ballot; the accumulate and adjoint walks then also test the
// ellipse against the block), and skips a whole batch once all its pixels stopped. Every walk
// takes its decisions through blend_step(), written with explicit round-to-nearest intrinsics, so
// all walks take the same threshold decisions for the same inputs.
#include <cuda_runtime.h>

#include "icgs_device.cuh"
#include "icgs_internal.h"
#include "walk.cuh"

namespace icgs {

namespace {

using namespace walk;

template <int N>
struct Log2 {
  static constexpr int value = 1 + Log2<N / 2>::value;
};
template <>
struct Log2<1> {
  static constexpr int value = 0;
};

template <int N>
struct NextPow2 {
  static constexpr int value = N <= 1 ? 1 : N <= 2 ? 2 : N <= 4 ? 4 : N <= 8 ? 8 : N <= 16 ? 16 : 32;
};

// Warp sums of NP values (NP a power of two <= 32) with NP - 1 + 5 - log2(NP) shuffles and no
// selects, for values held in lane-permuted slots: slot i of lane l holds value index i ^ m(l),
// m(l) = (l >> (5 - log2 NP)) & (NP - 1). At each level a lane keeps its lower half of slots and
// adds its partner's upper half, which holds the same value indices (the partner's m differs in
// exactly that level's bit). Lane l returns the warp sum of value m(l). The caller permutes its
// per-pixel factors once (they do not change during the walk).
template <int NP>
__device__ __forceinline__ float warp_permuted_reduce(float (&v)[NP]) {
  constexpr int P = Log2<NP>::value;
#pragma unroll
  for (int lvl = 0; lvl < P; ++lvl) {
    const int off = 16 >> lvl;
    const int half = NP >> (lvl + 1);
#pragma unroll
    for (int i = 0; i < half; ++i) v[i] += __shfl_xor_sync(kFull, v[i + half], off);
  }
  float r = v[0];
#pragma unroll
  for (int off = 16 >> P; off > 0; off >>= 1) r += __shfl_xor_sync(kFull, r, off);
  return r;
}
// ------------------------------------------------------------------------------------------
// colorize: V and S per (camera, Gaussian)
// ------------------------------------------------------------------------------------------
template <int KC>
__global__ void __launch_bounds__(kThreads, KC <= 8 ? 5 : 4) k_blend_accumulate(
    const uint32_t* __restrict__ tile_off, const uint64_t* __restrict__ entries, uint32_t capacity,
    const ProjRec* __restrict__ rec, int64_t n, int width, int height, int tiles_x, int tiles,
    const void* __restrict__ targets, int dtype, int K, int k0, int cam0, const float* __restrict__ sub_img,
    float* __restrict__ acc, int RS, int64_t acc_cam_stride, DevStatus* status) {
  static_assert(KC >= 4, "up to 3 channels take the two-pixel walk");
  constexpr int NV = KC + 1;                      // V and S_0..S_{KC-1}
  // 16 channels reduce V on its own, so that the sums fill a 16-value reduction instead of a
  // 32-value one padded with 15 zeros; otherwise V is value 0 of the reduction.
  constexpr bool kSplitV = KC == 16;
  constexpr int NS = kSplitV ? KC : NV;           // values in the warp reduction
  constexpr int NP = NextPow2<NS>::value;
  constexpr int SHIFT = 5 - Log2<NP>::value;      // lane l returns the sum of value l >> SHIFT
  __shared__ float4 s_geo[kBatch], s_aux[kBatch];
  __shared__ float2 s_half[kBatch];
  __shared__ uint32_t s_id[kBatch];
  __shared__ float s_acc[kBatch][NV];
  const TileCtx c = tile_ctx(tile_off, capacity, tiles, tiles_x, width, height);
  const unsigned long long* list = tile_list(entries, c.b);
  const int lane = threadIdx.x & 31;
  float tv[KC];
#pragma unroll
  for (int k = 0; k < KC; ++k) tv[k] = 0.0f;
  if (c.inside) {
    const int64_t base = (((int64_t)(cam0 + c.j) * height + c.py) * width + c.px) * K + k0;
#pragma unroll
    for (int k = 0; k < KC; ++k)
      if (k0 + k < K) tv[k] = load_target(targets, base + k, dtype);
    check_finite(tv, status);
    if (sub_img) {  // refinement: residual targets t - img, img of this pass's cameras
      const int64_t ib = (((int64_t)c.j * height + c.py) * width + c.px) * K + k0;
#pragma unroll
      for (int k = 0; k < KC; ++k)
        if (k0 + k < K) tv[k] -= sub_img[ib + k];
    }
  }
  for (int k = threadIdx.x; k < kBatch * NV; k += kThreads) (&s_acc[0][0])[k] = 0.0f;
  const ProjRec* rec_cam = rec + (int64_t)c.j * n;
  float* acc_cam = acc + (int64_t)c.j * acc_cam_stride;
  const int my_value = lane >> SHIFT;
  const bool reducer = (lane & ((1 << SHIFT) - 1)) == 0 && my_value < NS;
  const int my_col = (kSplitV ? 1 : 0) + my_value;  // the s_acc column of this lane's sum
  // Value q of a hit is w u[q], u = (1, t_0, .., t_{KC-1}, 0, ..), or the channels alone when V is
  // reduced on its own. This lane keeps value q in slot q ^ my_value (warp_permuted_reduce), so u
  // is permuted here once, by one conditional swap per bit of my_value.
  float u[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    const int k = q - (kSplitV ? 0 : 1);
    u[q] = k < 0 ? 1.0f : (k < KC ? tv[k >= 0 && k < KC ? k : 0] : 0.0f);
  }
#pragma unroll
  for (int bit = 1; bit < NP; bit <<= 1) {
    const bool sw = (my_value & bit) != 0;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      if (q & bit) continue;
      const float x = u[q], y = u[q | bit];
      u[q] = sw ? y : x;
      u[q | bit] = sw ? x : y;
    }
  }
  float T = 1.0f;
  bool done = !c.inside;
  uint32_t npairs = 0;
  for (uint32_t start = 0; start < c.len; start += kBatch) {
    const int nb = (int)min((uint32_t)kBatch, c.len - start);
    __syncthreads();
    load_batch(list, start, nb, rec_cam, n, c.ox, c.oy, s_geo, s_aux, s_half, s_id);
    __syncthreads();
    if (!__all_sync(kFull, done)) {
#pragma unroll
      for (int half = 0; half < kBatch / 32; ++half) {
        uint32_t bits = warp_hit_bits<true>(s_geo, s_aux, s_half, half * 32, nb, c);
        while (bits) {  // only the Gaussians whose box touches this warp's block, in depth order
          const int g = half * 32 + __ffs(bits) - 1;
          bits &= bits - 1;
          const float w = blend_weight<true>(s_geo[g], s_aux[g], c.pxf, c.pyf, T, done, npairs);
          if (__any_sync(kFull, w > 0.0f)) {
            float v[NP];
#pragma unroll
            for (int q = 0; q < NP; ++q) v[q] = __fmul_rn(w, u[q]);
            const float r = warp_permuted_reduce<NP>(v);
            if (reducer) atomicAdd(&s_acc[g][my_col], r);
            if constexpr (kSplitV) {
              float ws = w;
#pragma unroll
              for (int off = 16; off > 0; off >>= 1) ws += __shfl_xor_sync(kFull, ws, off);
              if (lane == 1) atomicAdd(&s_acc[g][0], ws);
            }
          }
        }
      }
    }
    __syncthreads();
    if ((int)threadIdx.x < nb) {
      const int g = threadIdx.x;
      if (s_acc[g][0] > 0.0f) {
        float* dst = acc_cam + (int64_t)s_id[g] * RS;
        if (k0 == 0) atomicAdd(dst, s_acc[g][0]);
#pragma unroll
        for (int k = 0; k < KC; ++k)
          if (k0 + k < K) atomicAdd(dst + 1 + k0 + k, s_acc[g][k + 1]);
#pragma unroll
        for (int k = 0; k < NV; ++k) s_acc[g][k] = 0.0f;
      }
    }
    if (__syncthreads_and(done)) break;
  }
  if (k0 == 0) add_pair_count(npairs, status);
}

// The same accumulation for up to 3 channels with two pixels per thread: CTAs of 128 threads, each
// warp covering an 8x8 block, 10 CTAs (48 registers a thread) per SM. A hit's fixed costs (the ballot loop, the shared loads, the vote, the
// warp reduction and the shared atomic) are shared by 64 pixels instead of 32: each thread adds its
// two pixels' contributions before the reduction. The pixels of a thread are walked independently
// (own transmittance, own stop), in the same depth order, through the same blend_step().
constexpr int kThreads2 = kThreads / 2;

template <int KC>
__global__ void __launch_bounds__(kThreads2, 10) k_blend_accumulate2(
    const uint32_t* __restrict__ tile_off, const uint64_t* __restrict__ entries, uint32_t capacity,
    const ProjRec* __restrict__ rec, int64_t n, int width, int height, int tiles_x, int tiles,
    const void* __restrict__ targets, int dtype, int K, int k0, int cam0, const float* __restrict__ sub_img,
    float* __restrict__ acc, int RS, int64_t acc_cam_stride, DevStatus* status) {
  static_assert(KC <= 3, "two pixels per thread: up to 3 channels");
  constexpr int NV = KC + 1;
  constexpr int NP = NextPow2<NV>::value;
  constexpr int NP2 = 2 * NP;                     // two hits per reduction
  constexpr int SHIFT2 = 5 - Log2<NP2>::value;
  __shared__ float4 s_geo[kBatch], s_aux[kBatch];
  __shared__ float2 s_half[kBatch];
  __shared__ uint32_t s_id[kBatch];
  __shared__ float s_acc[kBatch][NV];
  const TileCtx c = tile_ctx<2>(tile_off, capacity, tiles, tiles_x, width, height);
  const unsigned long long* list = tile_list(entries, c.b);
  const int lane = threadIdx.x & 31;
  const bool inside1 = c.inside && c.py + 4 < height;
  const float pyf1 = c.pyf + 4.0f;
  float tv0[KC], tv1[KC];
#pragma unroll
  for (int k = 0; k < KC; ++k) tv0[k] = tv1[k] = 0.0f;
  const int64_t row = (int64_t)width * K;
  if (c.inside) {
    const int64_t base = (((int64_t)(cam0 + c.j) * height + c.py) * width + c.px) * K + k0;
    const int64_t ib = (((int64_t)c.j * height + c.py) * width + c.px) * K + k0;
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      if (k0 + k < K) {
        tv0[k] = load_target(targets, base + k, dtype);
        if (sub_img) tv0[k] -= sub_img[ib + k];  // refinement: residual targets t - img
        if (inside1) {
          tv1[k] = load_target(targets, base + 4 * row + k, dtype);
          if (sub_img) tv1[k] -= sub_img[ib + 4 * row + k];
        }
      }
    }
    check_finite(tv0, status);
    check_finite(tv1, status);
  }
  // Value h NP + k of a hit pair is hit h's weights times u[k], u = (1, t_0, .., t_{KC-1}, 0, ..),
  // summed over the thread's two pixels. This lane keeps it in slot (h NP + k) ^ m
  // (warp_permuted_reduce), so u is permuted here once, by one conditional swap per bit of mk, and
  // the pair's two hits trade places when mh is set.
  const int m = lane >> SHIFT2;
  const bool mh = (m & NP) != 0;
  const int mk = m & (NP - 1);
  float u0[NP], u1[NP];
  u0[0] = u1[0] = 1.0f;
#pragma unroll
  for (int k = 1; k < NP; ++k) {
    u0[k] = k <= KC ? tv0[k <= KC ? k - 1 : 0] : 0.0f;
    u1[k] = k <= KC ? tv1[k <= KC ? k - 1 : 0] : 0.0f;
  }
#pragma unroll
  for (int bit = 1; bit < NP; bit <<= 1) {
    const bool sw = (mk & bit) != 0;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      if (k & bit) continue;
      const float x0 = u0[k], y0 = u0[k | bit], x1 = u1[k], y1 = u1[k | bit];
      u0[k] = sw ? y0 : x0;
      u0[k | bit] = sw ? x0 : y0;
      u1[k] = sw ? y1 : x1;
      u1[k | bit] = sw ? x1 : y1;
    }
  }
  for (int k = threadIdx.x; k < kBatch * NV; k += kThreads2) (&s_acc[0][0])[k] = 0.0f;
  const ProjRec* rec_cam = rec + (int64_t)c.j * n;
  float* acc_cam = acc + (int64_t)c.j * acc_cam_stride;
  float T0 = 1.0f, T1 = 1.0f;
  bool done0 = !c.inside, done1 = !inside1;
  uint32_t npairs = 0;
  for (uint32_t start = 0; start < c.len; start += kBatch) {
    const int nb = (int)min((uint32_t)kBatch, c.len - start);
    __syncthreads();
    load_batch(list, start, nb, rec_cam, n, c.ox, c.oy, s_geo, s_aux, s_half, s_id);
    __syncthreads();
    if (!__all_sync(kFull, done0 && done1)) {
#pragma unroll
      for (int half = 0; half < kBatch / 32; ++half) {
        uint32_t bits = warp_hit_bits<true>(s_geo, s_aux, s_half, half * 32, nb, c);
        while (bits) {
          const int g1 = half * 32 + __ffs(bits) - 1;
          bits &= bits - 1;
          const int g2 = bits ? half * 32 + __ffs(bits) - 1 : -1;
          bits &= bits - 1;
          float w20 = 0.0f, w21 = 0.0f;
          const float4 geo1 = s_geo[g1], aux1 = s_aux[g1];
          const float w10 = blend_weight<true>(geo1, aux1, c.pxf, c.pyf, T0, done0, npairs);
          const float w11 = blend_weight<true>(geo1, aux1, c.pxf, pyf1, T1, done1, npairs);
          if (g2 >= 0) {
            const float4 geo = s_geo[g2], aux = s_aux[g2];
            w20 = blend_weight<true>(geo, aux, c.pxf, c.pyf, T0, done0, npairs);
            w21 = blend_weight<true>(geo, aux, c.pxf, pyf1, T1, done1, npairs);
          }
          const float w1 = __fadd_rn(w10, w11), w2 = __fadd_rn(w20, w21);
          if (__any_sync(kFull, w1 > 0.0f || w2 > 0.0f)) {
            const float a0 = mh ? w20 : w10, a1 = mh ? w21 : w11;
            const float c0 = mh ? w10 : w20, c1 = mh ? w11 : w21;
            float v[NP2];
#pragma unroll
            for (int k = 0; k < NP; ++k) {
              v[k] = __fmaf_rn(a0, u0[k], __fmul_rn(a1, u1[k]));
              v[NP + k] = __fmaf_rn(c0, u0[k], __fmul_rn(c1, u1[k]));
            }
            const float r = warp_permuted_reduce<NP2>(v);  // the warp sum of value index m
            const int gg = mh ? g2 : g1;
            if ((lane & ((1 << SHIFT2) - 1)) == 0 && mk < NV && gg >= 0) atomicAdd(&s_acc[gg][mk], r);
          }
        }
      }
    }
    __syncthreads();
    if ((int)threadIdx.x < nb) {
      const int g = threadIdx.x;
      if (s_acc[g][0] > 0.0f) {
        float* dst = acc_cam + (int64_t)s_id[g] * RS;
        if (KC == 3 && K == 3) {
          atomicAdd(reinterpret_cast<float4*>(dst), make_float4(s_acc[g][0], s_acc[g][1], s_acc[g][2], s_acc[g][3]));
        } else {
          if (k0 == 0) atomicAdd(dst, s_acc[g][0]);
#pragma unroll
          for (int k = 0; k < KC; ++k)
            if (k0 + k < K) atomicAdd(dst + 1 + k0 + k, s_acc[g][k + 1]);
        }
#pragma unroll
        for (int k = 0; k < NV; ++k) s_acc[g][k] = 0.0f;
      }
    }
    if (__syncthreads_and(done0 && done1)) break;
  }
  if (k0 == 0) add_pair_count(npairs, status);
}

// ------------------------------------------------------------------------------------------
// render: img = sum w C
// ------------------------------------------------------------------------------------------
template <int KC>
__global__ void __launch_bounds__(kThreads) k_blend_render(
    const uint32_t* __restrict__ tile_off, const uint64_t* __restrict__ entries, uint32_t capacity,
    const ProjRec* __restrict__ rec, int64_t n, int width, int height, int tiles_x, int tiles,
    const float* __restrict__ payload, int K, int k0, int cam0, float* __restrict__ images) {
  __shared__ float4 s_geo[kBatch], s_aux[kBatch];
  __shared__ float2 s_half[kBatch];
  __shared__ uint32_t s_id[kBatch];
  __shared__ float s_col[kBatch][KC];
  const TileCtx c = tile_ctx(tile_off, capacity, tiles, tiles_x, width, height);
  const unsigned long long* list = tile_list(entries, c.b);
  const ProjRec* rec_cam = rec + (int64_t)c.j * n;
  const float* pay_cam = payload + (int64_t)c.j * n * K;
  float img[KC];
#pragma unroll
  for (int k = 0; k < KC; ++k) img[k] = 0.0f;
  float T = 1.0f;
  bool done = !c.inside;
  for (uint32_t start = 0; start < c.len; start += kBatch) {
    const int nb = (int)min((uint32_t)kBatch, c.len - start);
    __syncthreads();
    load_batch(list, start, nb, rec_cam, n, c.ox, c.oy, s_geo, s_aux, s_half, s_id);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nb * KC; idx += kThreads) {
      const int g = idx / KC, k = idx - g * KC;
      s_col[g][k] = k0 + k < K ? pay_cam[(int64_t)s_id[g] * K + k0 + k] : 0.0f;
    }
    __syncthreads();
    if (!__all_sync(kFull, done)) {
#pragma unroll
      for (int half = 0; half < kBatch / 32; ++half) {
        uint32_t bits = warp_hit_bits(s_geo, s_aux, s_half, half * 32, nb, c);
        while (bits && !done) {
          const int g = half * 32 + __ffs(bits) - 1;
          bits &= bits - 1;
          float al, ex;
          bool cap;
          const float w = blend_step(s_geo[g], s_aux[g], c.pxf, c.pyf, T, done, al, ex, cap);
          if (w > 0.0f) {
#pragma unroll
            for (int k = 0; k < KC; ++k) img[k] = fmaf(w, s_col[g][k], img[k]);
          }
        }
      }
    }
    if (__syncthreads_and(done)) break;
  }
  if (c.inside) {
    float* dst = images + (((int64_t)(cam0 + c.j) * height + c.py) * width + c.px) * K + k0;
#pragma unroll
    for (int k = 0; k < KC; ++k)
      if (k0 + k < K) dst[k] = img[k];
  }
}

// The render with two pixels per thread (up to 4 channels): CTAs of 128 threads, each warp
// covering an 8x8 block; the pixels (x, y) and (x, y + 4) of a thread are walked independently.
// A hit costs little here (no reduction), so the warp keeps the plain box test.
template <int KC>
__global__ void __launch_bounds__(kThreads2, 10) k_blend_render2(
    const uint32_t* __restrict__ tile_off, const uint64_t* __restrict__ entries, uint32_t capacity,
    const ProjRec* __restrict__ rec, int64_t n, int width, int height, int tiles_x, int tiles,
    const float* __restrict__ payload, int K, int k0, int cam0, float* __restrict__ images) {
  static_assert(KC <= 4, "two pixels per thread: up to 4 channels");
  __shared__ float4 s_geo[kBatch], s_aux[kBatch];
  __shared__ float2 s_half[kBatch];
  __shared__ uint32_t s_id[kBatch];
  __shared__ float s_col[kBatch][KC];
  const TileCtx c = tile_ctx<2>(tile_off, capacity, tiles, tiles_x, width, height);
  const unsigned long long* list = tile_list(entries, c.b);
  const bool inside1 = c.inside && c.py + 4 < height;
  const float pyf1 = c.pyf + 4.0f;
  const ProjRec* rec_cam = rec + (int64_t)c.j * n;
  const float* pay_cam = payload + (int64_t)c.j * n * K;
  float img0[KC], img1[KC];
#pragma unroll
  for (int k = 0; k < KC; ++k) img0[k] = img1[k] = 0.0f;
  float T0 = 1.0f, T1 = 1.0f;
  bool done0 = !c.inside, done1 = !inside1;
  for (uint32_t start = 0; start < c.len; start += kBatch) {
    const int nb = (int)min((uint32_t)kBatch, c.len - start);
    __syncthreads();
    load_batch(list, start, nb, rec_cam, n, c.ox, c.oy, s_geo, s_aux, s_half, s_id);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nb * KC; idx += kThreads2) {
      const int g = idx / KC, k = idx - g * KC;
      s_col[g][k] = k0 + k < K ? pay_cam[(int64_t)s_id[g] * K + k0 + k] : 0.0f;
    }
    __syncthreads();
    if (!__all_sync(kFull, done0 && done1)) {
#pragma unroll
      for (int half = 0; half < kBatch / 32; ++half) {
        uint32_t bits = warp_hit_bits(s_geo, s_aux, s_half, half * 32, nb, c);
        while (bits && !(done0 && done1)) {
          const int g = half * 32 + __ffs(bits) - 1;
          bits &= bits - 1;
          const float4 geo = s_geo[g], aux = s_aux[g];
          float al, ex;
          bool cap;
          if (!done0) {
            const float w = blend_step(geo, aux, c.pxf, c.pyf, T0, done0, al, ex, cap);
            if (w > 0.0f) {
#pragma unroll
              for (int k = 0; k < KC; ++k) img0[k] = fmaf(w, s_col[g][k], img0[k]);
            }
          }
          if (!done1) {
            const float w = blend_step(geo, aux, c.pxf, pyf1, T1, done1, al, ex, cap);
            if (w > 0.0f) {
#pragma unroll
              for (int k = 0; k < KC; ++k) img1[k] = fmaf(w, s_col[g][k], img1[k]);
            }
          }
        }
      }
    }
    if (__syncthreads_and(done0 && done1)) break;
  }
  if (c.inside) {
    float* dst = images + (((int64_t)(cam0 + c.j) * height + c.py) * width + c.px) * K + k0;
#pragma unroll
    for (int k = 0; k < KC; ++k)
      if (k0 + k < K) dst[k] = img0[k];
    if (inside1) {
      dst += 4 * (int64_t)width * K;
#pragma unroll
      for (int k = 0; k < KC; ++k)
        if (k0 + k < K) dst[k] = img1[k];
    }
  }
}

// ------------------------------------------------------------------------------------------
// adjoint: dL/dt and dL/do. Payload per (camera, Gaussian) = (a_0..a_{K-1}, beta).
// ------------------------------------------------------------------------------------------
template <int KC, int NT = kThreads>
__device__ __forceinline__ void load_payload(const float* __restrict__ pay_cam, int nb, int K, const uint32_t* s_id,
                                             float (*s_pay)[KC + 1]) {
  for (int idx = threadIdx.x; idx < nb * (KC + 1); idx += NT) {
    const int g = idx / (KC + 1), k = idx - g * (KC + 1);
    float v = 0.0f;
    if (k < KC) {
      if (k < K) v = pay_cam[(int64_t)s_id[g] * (K + 1) + k];
    } else {
      v = pay_cam[(int64_t)s_id[g] * (K + 1) + K];
    }
    s_pay[g][k] = v;
  }
}

template <int KC>
__global__ void __launch_bounds__(kThreads, KC <= 4 ? 6 : (KC <= 16 ? 4 : (KC <= 32 ? 2 : 1))) k_blend_adjoint(
    const uint32_t* __restrict__ tile_off, const uint64_t* __restrict__ entries, uint32_t capacity,
    const ProjRec* __restrict__ rec, int64_t n, int width, int height, int tiles_x, int tiles,
    const void* __restrict__ targets, int dtype, const float* __restrict__ payload, int K, int cam0,
    float* __restrict__ grad_t, float* __restrict__ grad_o) {
  __shared__ float4 s_geo[kBatch], s_aux[kBatch];
  __shared__ float2 s_half[kBatch];
  __shared__ uint32_t s_id[kBatch];
  __shared__ float s_pay[kBatch][KC + 1];
  __shared__ float s_go[kBatch];
  const TileCtx c = tile_ctx(tile_off, capacity, tiles, tiles_x, width, height);
  const unsigned long long* list = tile_list(entries, c.b);
  const int lane = threadIdx.x & 31;
  const ProjRec* rec_cam = rec + (int64_t)c.j * n;
  const float* pay_cam = payload + (int64_t)c.j * n * (K + 1);
  float tv[KC], gt[KC];
#pragma unroll
  for (int k = 0; k < KC; ++k) { tv[k] = 0.0f; gt[k] = 0.0f; }
  const int64_t pix = ((int64_t)(cam0 + c.j) * height + c.py) * width + c.px;
  if (c.inside) {
#pragma unroll
    for (int k = 0; k < KC; ++k)
      if (k < K) tv[k] = load_target(targets, pix * K + k, dtype);
  }
  // pass 1: F = sum_n g_n w_n and dL/dt = sum_n w_n a_n
  float F = 0.0f;
  {
    float T = 1.0f;
    bool done = !c.inside;
    for (uint32_t start = 0; start < c.len; start += kBatch) {
      const int nb = (int)min((uint32_t)kBatch, c.len - start);
      __syncthreads();
      load_batch(list, start, nb, rec_cam, n, c.ox, c.oy, s_geo, s_aux, s_half, s_id);
      __syncthreads();
      load_payload<KC>(pay_cam, nb, K, s_id, s_pay);
      __syncthreads();
      if (!__all_sync(kFull, done)) {
#pragma unroll
        for (int half = 0; half < kBatch / 32; ++half) {
          uint32_t bits = warp_hit_bits(s_geo, s_aux, s_half, half * 32, nb, c);
          while (bits && !done) {
            const int g = half * 32 + __ffs(bits) - 1;
            bits &= bits - 1;
            float al, ex;
            bool cap;
            const float w = blend_step(s_geo[g], s_aux[g], c.pxf, c.pyf, T, done, al, ex, cap);
            if (w > 0.0f) {
              float gg = s_pay[g][KC];
#pragma unroll
              for (int k = 0; k < KC; ++k) {
                gg = fmaf(s_pay[g][k], tv[k], gg);
                gt[k] = fmaf(w, s_pay[g][k], gt[k]);
              }
              F = fmaf(gg, w, F);
            }
          }
        }
      }
      if (__syncthreads_and(done)) break;
    }
  }
  if (grad_t && c.inside) {
#pragma unroll
    for (int k = 0; k < KC; ++k)
      if (k < K) grad_t[pix * K + k] = gt[k];
  }
  if (!grad_o) return;
  // pass 2: dL/dalpha_m = g_m T_m - (F - P_m) / (1 - alpha_m), P_m = sum_{n<=m} g_n w_n
  for (int k = threadIdx.x; k < kBatch; k += kThreads) s_go[k] = 0.0f;
  float T = 1.0f, P = 0.0f;
  bool done = !c.inside;
  for (uint32_t start = 0; start < c.len; start += kBatch) {
    const int nb = (int)min((uint32_t)kBatch, c.len - start);
    __syncthreads();
    load_batch(list, start, nb, rec_cam, n, c.ox, c.oy, s_geo, s_aux, s_half, s_id);
    __syncthreads();
    load_payload<KC>(pay_cam, nb, K, s_id, s_pay);
    __syncthreads();
    if (!__all_sync(kFull, done)) {
#pragma unroll
      for (int half = 0; half < kBatch / 32; ++half) {
       uint32_t bits = warp_hit_bits(s_geo, s_aux, s_half, half * 32, nb, c);
       // dL/dalpha_m of one hit for this pixel (0 when skipped or capped); updates T and P
       auto d_opacity = [&](int g) -> float {
         if (done) return 0.0f;
         const float Tm = T;
         float al = 0.0f, ex = 0.0f;
         bool cap = false;
         const float w = blend_step(s_geo[g], s_aux[g], c.pxf, c.pyf, T, done, al, ex, cap);
         if (!(w > 0.0f)) return 0.0f;
         float gg = s_pay[g][KC];
#pragma unroll
         for (int k = 0; k < KC; ++k) gg = fmaf(s_pay[g][k], tv[k], gg);
         P = fmaf(gg, w, P);
         const float dalpha = gg * Tm - __fdividef(F - P, 1.0f - al);
         return cap ? 0.0f : dalpha * ex;
       };
       // two consecutive hits (in depth order) share one warp reduction of their two values
       while (bits) {
        const int g1 = half * 32 + __ffs(bits) - 1;
        bits &= bits - 1;
        const int g2 = bits ? half * 32 + __ffs(bits) - 1 : -1;
        bits &= bits - 1;
        const float d1 = d_opacity(g1);
        const float d2 = g2 >= 0 ? d_opacity(g2) : 0.0f;
        if (__any_sync(kFull, d1 != 0.0f || d2 != 0.0f)) {
          // lanes < 16 end with the sum of d1, lanes >= 16 with the sum of d2
          const bool upper = (lane & 16) != 0;
          float r = (upper ? d2 : d1) + __shfl_xor_sync(kFull, upper ? d1 : d2, 16);
#pragma unroll
          for (int o = 8; o > 0; o >>= 1) r += __shfl_xor_sync(kFull, r, o);
          if (lane == 0) atomicAdd(&s_go[g1], r);
          if (lane == 16 && g2 >= 0) atomicAdd(&s_go[g2], r);
        }
       }
      }
    }
    __syncthreads();
    if ((int)threadIdx.x < nb) {
      const float v = s_go[threadIdx.x];
      if (v != 0.0f) {
        atomicAdd(grad_o + s_id[threadIdx.x], v);
        s_go[threadIdx.x] = 0.0f;
      }
    }
    if (__syncthreads_and(done)) break;
  }
}

// Pass 1 of the adjoint walk for one pixel and one staged Gaussian: F += g w and dL/dt += w a,
// with g = a . t + beta.
template <int KC>
__device__ __forceinline__ void adjoint_gather(const float4 geo, const float4 aux, const float* pay,
                                               const float (&tv)[KC], float pxf, float pyf, float& T, bool& done,
                                               float& F, float (&gt)[KC]) {
  float al, ex;
  bool cap;
  const float w = blend_step(geo, aux, pxf, pyf, T, done, al, ex, cap);
  if (w > 0.0f) {
    float gg = pay[KC];
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      gg = fmaf(pay[k], tv[k], gg);
      gt[k] = fmaf(w, pay[k], gt[k]);
    }
    F = fmaf(gg, w, F);
  }
}

// Pass 2 for one pixel and one staged Gaussian m: dL/dalpha_m = g_m T_m - (F - P_m) / (1 - alpha_m),
// returned times dalpha/do = exp(-q/2) (0 when skipped or when alpha was capped); advances T and P.
template <int KC>
__device__ __forceinline__ float adjoint_step(const float4 geo, const float4 aux, const float* pay,
                                              const float (&tv)[KC], float pxf, float pyf, float F, float& T,
                                              float& P, bool& done) {
  if (done) return 0.0f;
  const float Tm = T;
  float al = 0.0f, ex = 0.0f;
  bool cap = false;
  const float w = blend_step(geo, aux, pxf, pyf, T, done, al, ex, cap);
  if (!(w > 0.0f)) return 0.0f;
  float gg = pay[KC];
#pragma unroll
  for (int k = 0; k < KC; ++k) gg = fmaf(pay[k], tv[k], gg);
  P = fmaf(gg, w, P);
  const float dalpha = gg * Tm - __fdividef(F - P, 1.0f - al);
  return cap ? 0.0f : dalpha * ex;
}

// The adjoint walk with two pixels per thread (up to 4 channels): CTAs of 128 threads, each warp
// covering an 8x8 block. Pass 2 adds a thread's two pixels before the warp reduction, so one
// reduction of a hit pair serves 64 pixels.
template <int KC>
__global__ void __launch_bounds__(kThreads2, KC <= 2 ? 10 : 8) k_blend_adjoint2(
    const uint32_t* __restrict__ tile_off, const uint64_t* __restrict__ entries, uint32_t capacity,
    const ProjRec* __restrict__ rec, int64_t n, int width, int height, int tiles_x, int tiles,
    const void* __restrict__ targets, int dtype, const float* __restrict__ payload, int K, int cam0,
    float* __restrict__ grad_t, float* __restrict__ grad_o) {
  static_assert(KC <= 4, "two pixels per thread: up to 4 channels");
  __shared__ float4 s_geo[kBatch], s_aux[kBatch];
  __shared__ float2 s_half[kBatch];
  __shared__ uint32_t s_id[kBatch];
  __shared__ float s_pay[kBatch][KC + 1];
  __shared__ float s_go[kBatch];
  const TileCtx c = tile_ctx<2>(tile_off, capacity, tiles, tiles_x, width, height);
  const unsigned long long* list = tile_list(entries, c.b);
  const int lane = threadIdx.x & 31;
  const bool inside1 = c.inside && c.py + 4 < height;
  const float pyf1 = c.pyf + 4.0f;
  const ProjRec* rec_cam = rec + (int64_t)c.j * n;
  const float* pay_cam = payload + (int64_t)c.j * n * (K + 1);
  float tv0[KC], tv1[KC];
#pragma unroll
  for (int k = 0; k < KC; ++k) tv0[k] = tv1[k] = 0.0f;
  const int64_t pix0 = ((int64_t)(cam0 + c.j) * height + c.py) * width + c.px;
  const int64_t pix1 = pix0 + 4 * (int64_t)width;
  if (c.inside) {
#pragma unroll
    for (int k = 0; k < KC; ++k)
      if (k < K) {
        tv0[k] = load_target(targets, pix0 * K + k, dtype);
        if (inside1) tv1[k] = load_target(targets, pix1 * K + k, dtype);
      }
  }
  // pass 1: F = sum_n g_n w_n and dL/dt = sum_n w_n a_n, per pixel
  float F0 = 0.0f, F1 = 0.0f;
  {
    float gt0[KC], gt1[KC];
#pragma unroll
    for (int k = 0; k < KC; ++k) gt0[k] = gt1[k] = 0.0f;
    float T0 = 1.0f, T1 = 1.0f;
    bool done0 = !c.inside, done1 = !inside1;
    for (uint32_t start = 0; start < c.len; start += kBatch) {
      const int nb = (int)min((uint32_t)kBatch, c.len - start);
      __syncthreads();
      load_batch(list, start, nb, rec_cam, n, c.ox, c.oy, s_geo, s_aux, s_half, s_id);
      __syncthreads();
      load_payload<KC, kThreads2>(pay_cam, nb, K, s_id, s_pay);
      __syncthreads();
      if (!__all_sync(kFull, done0 && done1)) {
#pragma unroll
        for (int half = 0; half < kBatch / 32; ++half) {
          uint32_t bits = warp_hit_bits<true>(s_geo, s_aux, s_half, half * 32, nb, c);
          while (bits && !(done0 && done1)) {
            const int g = half * 32 + __ffs(bits) - 1;
            bits &= bits - 1;
            const float4 geo = s_geo[g], aux = s_aux[g];
            if (!done0) adjoint_gather<KC>(geo, aux, s_pay[g], tv0, c.pxf, c.pyf, T0, done0, F0, gt0);
            if (!done1) adjoint_gather<KC>(geo, aux, s_pay[g], tv1, c.pxf, pyf1, T1, done1, F1, gt1);
          }
        }
      }
      if (__syncthreads_and(done0 && done1)) break;
    }
    if (grad_t && c.inside) {
#pragma unroll
      for (int k = 0; k < KC; ++k)
        if (k < K) {
          grad_t[pix0 * K + k] = gt0[k];
          if (inside1) grad_t[pix1 * K + k] = gt1[k];
        }
    }
  }
  if (!grad_o) return;
  // pass 2: dL/dalpha_m = g_m T_m - (F - P_m) / (1 - alpha_m), P_m = sum_{n<=m} g_n w_n
  for (int k = threadIdx.x; k < kBatch; k += kThreads2) s_go[k] = 0.0f;
  float T0 = 1.0f, T1 = 1.0f, P0 = 0.0f, P1 = 0.0f;
  bool done0 = !c.inside, done1 = !inside1;
  for (uint32_t start = 0; start < c.len; start += kBatch) {
    const int nb = (int)min((uint32_t)kBatch, c.len - start);
    __syncthreads();
    load_batch(list, start, nb, rec_cam, n, c.ox, c.oy, s_geo, s_aux, s_half, s_id);
    __syncthreads();
    load_payload<KC, kThreads2>(pay_cam, nb, K, s_id, s_pay);
    __syncthreads();
    if (!__all_sync(kFull, done0 && done1)) {
#pragma unroll
      for (int half = 0; half < kBatch / 32; ++half) {
        uint32_t bits = warp_hit_bits<true>(s_geo, s_aux, s_half, half * 32, nb, c);
        // two consecutive hits (in depth order) share one warp reduction of their two values
        while (bits) {
          const int g1 = half * 32 + __ffs(bits) - 1;
          bits &= bits - 1;
          const int g2 = bits ? half * 32 + __ffs(bits) - 1 : -1;
          bits &= bits - 1;
          float d1, d2 = 0.0f;
          {
            const float4 geo = s_geo[g1], aux = s_aux[g1];
            d1 = adjoint_step<KC>(geo, aux, s_pay[g1], tv0, c.pxf, c.pyf, F0, T0, P0, done0) +
                 adjoint_step<KC>(geo, aux, s_pay[g1], tv1, c.pxf, pyf1, F1, T1, P1, done1);
          }
          if (g2 >= 0) {
            const float4 geo = s_geo[g2], aux = s_aux[g2];
            d2 = adjoint_step<KC>(geo, aux, s_pay[g2], tv0, c.pxf, c.pyf, F0, T0, P0, done0) +
                 adjoint_step<KC>(geo, aux, s_pay[g2], tv1, c.pxf, pyf1, F1, T1, P1, done1);
          }
          if (__any_sync(kFull, d1 != 0.0f || d2 != 0.0f)) {
            // lanes < 16 end with the sum of d1, lanes >= 16 with the sum of d2
            const bool upper = (lane & 16) != 0;
            float r = (upper ? d2 : d1) + __shfl_xor_sync(kFull, upper ? d1 : d2, 16);
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) r += __shfl_xor_sync(kFull, r, o);
            if (lane == 0) atomicAdd(&s_go[g1], r);
            if (lane == 16 && g2 >= 0) atomicAdd(&s_go[g2], r);
          }
        }
      }
    }
    __syncthreads();
    if ((int)threadIdx.x < nb) {
      const float v = s_go[threadIdx.x];
      if (v != 0.0f) {
        atomicAdd(grad_o + s_id[threadIdx.x], v);
        s_go[threadIdx.x] = 0.0f;
      }
    }
    if (__syncthreads_and(done0 && done1)) break;
  }
}

// One refinement walk (Alg. 1 lines 8-9) for up to 3 channels, two pixels per thread: pass 1
// renders the current colours of the thread's pixels (as k_blend_render2), pass 2 accumulates the
// residual targets t - img (as k_blend_accumulate2 with a rendered image subtracted), over the tile
// list sorted once. Same arithmetic as the two separate walks, without the image round trip.
template <int KC>
__global__ void __launch_bounds__(kThreads2, 10) k_blend_refine2(
    const uint32_t* __restrict__ tile_off, const uint64_t* __restrict__ entries, uint32_t capacity,
    const ProjRec* __restrict__ rec, int64_t n, int width, int height, int tiles_x, int tiles,
    const void* __restrict__ targets, int dtype, int K, int cam0, const float* __restrict__ payload,
    float* __restrict__ acc, int RS, int64_t acc_cam_stride, DevStatus* status) {
  static_assert(KC <= 3, "two pixels per thread: up to 3 channels");
  constexpr int NV = KC + 1;
  constexpr int NP = NextPow2<NV>::value;
  constexpr int NP2 = 2 * NP;
  constexpr int SHIFT2 = 5 - Log2<NP2>::value;
  __shared__ float4 s_geo[kBatch], s_aux[kBatch];
  __shared__ float2 s_half[kBatch];
  __shared__ uint32_t s_id[kBatch];
  __shared__ float s_acc[kBatch][NV];
  __shared__ float s_col[kBatch][KC];
  const TileCtx c = tile_ctx<2>(tile_off, capacity, tiles, tiles_x, width, height);
  const unsigned long long* list = tile_list(entries, c.b);
  const int lane = threadIdx.x & 31;
  const bool inside1 = c.inside && c.py + 4 < height;
  const float pyf1 = c.pyf + 4.0f;
  const ProjRec* rec_cam = rec + (int64_t)c.j * n;
  const float* pay_cam = payload + (int64_t)c.j * n * K;
  // pass 1: the current render of both pixels
  float img0[KC], img1[KC];
#pragma unroll
  for (int k = 0; k < KC; ++k) img0[k] = img1[k] = 0.0f;
  {
    float T0 = 1.0f, T1 = 1.0f;
    bool done0 = !c.inside, done1 = !inside1;
    for (uint32_t start = 0; start < c.len; start += kBatch) {
      const int nb = (int)min((uint32_t)kBatch, c.len - start);
      __syncthreads();
      load_batch(list, start, nb, rec_cam, n, c.ox, c.oy, s_geo, s_aux, s_half, s_id);
      __syncthreads();
      for (int idx = threadIdx.x; idx < nb * KC; idx += kThreads2) {
        const int g = idx / KC, k = idx - g * KC;
        s_col[g][k] = k < K ? pay_cam[(int64_t)s_id[g] * K + k] : 0.0f;
      }
      __syncthreads();
      if (!__all_sync(kFull, done0 && done1)) {
#pragma unroll
        for (int half = 0; half < kBatch / 32; ++half) {
          uint32_t bits = warp_hit_bits(s_geo, s_aux, s_half, half * 32, nb, c);
          while (bits && !(done0 && done1)) {
            const int g = half * 32 + __ffs(bits) - 1;
            bits &= bits - 1;
            const float4 geo = s_geo[g], aux = s_aux[g];
            float al, ex;
            bool cap;
            if (!done0) {
              const float w = blend_step(geo, aux, c.pxf, c.pyf, T0, done0, al, ex, cap);
              if (w > 0.0f) {
#pragma unroll
                for (int k = 0; k < KC; ++k) img0[k] = fmaf(w, s_col[g][k], img0[k]);
              }
            }
            if (!done1) {
              const float w = blend_step(geo, aux, c.pxf, pyf1, T1, done1, al, ex, cap);
              if (w > 0.0f) {
#pragma unroll
                for (int k = 0; k < KC; ++k) img1[k] = fmaf(w, s_col[g][k], img1[k]);
              }
            }
          }
        }
      }
      if (__syncthreads_and(done0 && done1)) break;
    }
  }
  // residual targets t - img
  float tv0[KC], tv1[KC];
#pragma unroll
  for (int k = 0; k < KC; ++k) tv0[k] = tv1[k] = 0.0f;
  if (c.inside) {
    const int64_t base = (((int64_t)(cam0 + c.j) * height + c.py) * width + c.px) * K;
    const int64_t row = (int64_t)width * K;
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      if (k < K) {
        tv0[k] = load_target(targets, base + k, dtype) - img0[k];
        if (inside1) tv1[k] = load_target(targets, base + 4 * row + k, dtype) - img1[k];
      }
    }
    check_finite(tv0, status);
    check_finite(tv1, status);
  }
  // pass 2: the accumulate walk of k_blend_accumulate2 on the residuals
  const int m = lane >> SHIFT2;
  const bool mh = (m & NP) != 0;
  const int mk = m & (NP - 1);
  float u0[NP], u1[NP];
  u0[0] = u1[0] = 1.0f;
#pragma unroll
  for (int k = 1; k < NP; ++k) {
    u0[k] = k <= KC ? tv0[k <= KC ? k - 1 : 0] : 0.0f;
    u1[k] = k <= KC ? tv1[k <= KC ? k - 1 : 0] : 0.0f;
  }
#pragma unroll
  for (int bit = 1; bit < NP; bit <<= 1) {  // u[k] <- u[k ^ mk], one conditional swap per bit of mk
    const bool sw = (mk & bit) != 0;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      if (k & bit) continue;
      const float x0 = u0[k], y0 = u0[k | bit], x1 = u1[k], y1 = u1[k | bit];
      u0[k] = sw ? y0 : x0;
      u0[k | bit] = sw ? x0 : y0;
      u1[k] = sw ? y1 : x1;
      u1[k | bit] = sw ? x1 : y1;
    }
  }
  for (int k = threadIdx.x; k < kBatch * NV; k += kThreads2) (&s_acc[0][0])[k] = 0.0f;
  float* acc_cam = acc + (int64_t)c.j * acc_cam_stride;
  float T0 = 1.0f, T1 = 1.0f;
  bool done0 = !c.inside, done1 = !inside1;
  uint32_t npairs = 0;
  for (uint32_t start = 0; start < c.len; start += kBatch) {
    const int nb = (int)min((uint32_t)kBatch, c.len - start);
    __syncthreads();
    load_batch(list, start, nb, rec_cam, n, c.ox, c.oy, s_geo, s_aux, s_half, s_id);
    __syncthreads();
    if (!__all_sync(kFull, done0 && done1)) {
#pragma unroll
      for (int half = 0; half < kBatch / 32; ++half) {
        uint32_t bits = warp_hit_bits<true>(s_geo, s_aux, s_half, half * 32, nb, c);
        while (bits) {
          const int g1 = half * 32 + __ffs(bits) - 1;
          bits &= bits - 1;
          const int g2 = bits ? half * 32 + __ffs(bits) - 1 : -1;
          bits &= bits - 1;
          float w20 = 0.0f, w21 = 0.0f;
          const float4 geo1 = s_geo[g1], aux1 = s_aux[g1];
          const float w10 = blend_weight<true>(geo1, aux1, c.pxf, c.pyf, T0, done0, npairs);
          const float w11 = blend_weight<true>(geo1, aux1, c.pxf, pyf1, T1, done1, npairs);
          if (g2 >= 0) {
            const float4 geo = s_geo[g2], aux = s_aux[g2];
            w20 = blend_weight<true>(geo, aux, c.pxf, c.pyf, T0, done0, npairs);
            w21 = blend_weight<true>(geo, aux, c.pxf, pyf1, T1, done1, npairs);
          }
          const float w1 = __fadd_rn(w10, w11), w2 = __fadd_rn(w20, w21);
          if (__any_sync(kFull, w1 > 0.0f || w2 > 0.0f)) {
            const float a0 = mh ? w20 : w10, a1 = mh ? w21 : w11;
            const float c0 = mh ? w10 : w20, c1 = mh ? w11 : w21;
            float v[NP2];
#pragma unroll
            for (int k = 0; k < NP; ++k) {
              v[k] = __fmaf_rn(a0, u0[k], __fmul_rn(a1, u1[k]));
              v[NP + k] = __fmaf_rn(c0, u0[k], __fmul_rn(c1, u1[k]));
            }
            const float r = warp_permuted_reduce<NP2>(v);  // the warp sum of value index m
            const int gg = mh ? g2 : g1;
            if ((lane & ((1 << SHIFT2) - 1)) == 0 && mk < NV && gg >= 0) atomicAdd(&s_acc[gg][mk], r);
          }
        }
      }
    }
    __syncthreads();
    if ((int)threadIdx.x < nb) {
      const int g = threadIdx.x;
      if (s_acc[g][0] > 0.0f) {
        float* dst = acc_cam + (int64_t)s_id[g] * RS;
        if (KC == 3 && K == 3) {
          atomicAdd(reinterpret_cast<float4*>(dst), make_float4(s_acc[g][0], s_acc[g][1], s_acc[g][2], s_acc[g][3]));
        } else {
          atomicAdd(dst, s_acc[g][0]);
#pragma unroll
          for (int k = 0; k < KC; ++k)
            if (k < K) atomicAdd(dst + 1 + k, s_acc[g][k + 1]);
        }
#pragma unroll
        for (int k = 0; k < NV; ++k) s_acc[g][k] = 0.0f;
      }
    }
    if (__syncthreads_and(done0 && done1)) break;
  }
  add_pair_count(npairs, status);
}

template <int KC>
void accumulate_chunk(const Problem& p, int cb, int cam0, const void* targets, int dtype, int k0,
                      const float* sub_img, const Workspace& ws, cudaStream_t s) {
  const int64_t stride = p.L == 0 ? 0 : p.n * (int64_t)p.acc_stride;
  if constexpr (KC <= 3) {
    k_blend_accumulate2<KC><<<cb * p.tiles, kThreads2, 0, s>>>(ws.tile_off, ws.entries, p.capacity, ws.rec, p.n,
                                                               p.width, p.height, p.tiles_x, p.tiles, targets, dtype,
                                                               p.K, k0, cam0, sub_img, ws.acc, p.acc_stride, stride,
                                                               ws.status);
  } else {
    k_blend_accumulate<KC><<<cb * p.tiles, kThreads, 0, s>>>(ws.tile_off, ws.entries, p.capacity, ws.rec, p.n,
                                                              p.width, p.height, p.tiles_x, p.tiles, targets, dtype,
                                                              p.K, k0, cam0, sub_img, ws.acc, p.acc_stride, stride,
                                                              ws.status);
  }
  note_launches(1);
}

template <int KC>
void render_chunk(const Problem& p, int cb, int cam0, int k0, const Workspace& ws, float* images,
                  cudaStream_t s) {
  if constexpr (KC <= 4) {
    k_blend_render2<KC><<<cb * p.tiles, kThreads2, 0, s>>>(ws.tile_off, ws.entries, p.capacity, ws.rec, p.n,
                                                           p.width, p.height, p.tiles_x, p.tiles, ws.payload, p.K,
                                                           k0, cam0, images);
  } else {
    k_blend_render<KC><<<cb * p.tiles, kThreads, 0, s>>>(ws.tile_off, ws.entries, p.capacity, ws.rec, p.n,
                                                          p.width, p.height, p.tiles_x, p.tiles, ws.payload, p.K,
                                                          k0, cam0, images);
  }
  note_launches(1);
}

}  // namespace

// Channels are processed in chunks of at most 16 per walk; the chunk width is the smallest
// instantiated width that covers the remaining channels (1+KC values are reduced per Gaussian,
// padded to a power of two).
void launch_blend_accumulate(const Problem& p, int cb, int cam0, const void* targets, int dtype,
                             const float* sub_img, const Workspace& ws, cudaStream_t s) {
  if (!sub_img && tc_accumulate_applies(p, dtype)) {
    launch_blend_accumulate_tc(p, cb, cam0, targets, dtype, ws, s);
    return;
  }
  for (int k0 = 0; k0 < p.K; k0 += 16) {
    const int kc = p.K - k0;
    if (kc == 1) accumulate_chunk<1>(p, cb, cam0, targets, dtype, k0, sub_img, ws, s);
    else if (kc == 2) accumulate_chunk<2>(p, cb, cam0, targets, dtype, k0, sub_img, ws, s);
    else if (kc == 3) accumulate_chunk<3>(p, cb, cam0, targets, dtype, k0, sub_img, ws, s);
    else if (kc <= 7) accumulate_chunk<7>(p, cb, cam0, targets, dtype, k0, sub_img, ws, s);
    else if (kc <= 15) accumulate_chunk<15>(p, cb, cam0, targets, dtype, k0, sub_img, ws, s);
    else accumulate_chunk<16>(p, cb, cam0, targets, dtype, k0, sub_img, ws, s);
  }
}

void launch_blend_render(const Problem& p, int cb, int cam0, const Workspace& ws, float* images,
                         cudaStream_t s) {
  for (int k0 = 0; k0 < p.K; k0 += 16) {
    const int kc = p.K - k0;
    if (kc == 1) render_chunk<1>(p, cb, cam0, k0, ws, images, s);
    else if (kc == 2) render_chunk<2>(p, cb, cam0, k0, ws, images, s);
    else if (kc == 3) render_chunk<3>(p, cb, cam0, k0, ws, images, s);
    else if (kc == 4) render_chunk<4>(p, cb, cam0, k0, ws, images, s);
    else if (kc <= 8) render_chunk<8>(p, cb, cam0, k0, ws, images, s);
    else render_chunk<16>(p, cb, cam0, k0, ws, images, s);
  }
}

// The refinement walk (render of the current colours, then accumulation of the residual targets)
// in one kernel for up to 3 channels; returns false when the channel count needs the two walks.
bool launch_blend_refine(const Problem& p, int cb, int cam0, const void* targets, int dtype, const Workspace& ws,
                         cudaStream_t s) {
  if (p.K > 3) return false;
  const int64_t stride = p.L == 0 ? 0 : p.n * (int64_t)p.acc_stride;
#define ICGS_REF(KC)                                                                                         \
  k_blend_refine2<KC><<<cb * p.tiles, kThreads2, 0, s>>>(ws.tile_off, ws.entries, p.capacity, ws.rec, p.n,     \
                                                          p.width, p.height, p.tiles_x, p.tiles, targets, dtype, \
                                                          p.K, cam0, ws.payload, ws.acc, p.acc_stride, stride,   \
                                                          ws.status)
  if (p.K == 1) ICGS_REF(1);
  else if (p.K == 2) ICGS_REF(2);
  else ICGS_REF(3);
#undef ICGS_REF
  note_launches(1);
  return true;
}

void launch_blend_adjoint(const Problem& p, int cb, int cam0, const void* targets, int dtype,
                          const Workspace& ws, float* grad_targets, bool want_grad_o, cudaStream_t s) {
  float* go = want_grad_o ? ws.grad_o_acc : nullptr;
#define ICGS_ADJ(KC)                                                                                       \
  k_blend_adjoint<KC><<<cb * p.tiles, kThreads, 0, s>>>(ws.tile_off, ws.entries, p.capacity, ws.rec, p.n,  \
                                                         p.width, p.height, p.tiles_x, p.tiles, targets,     \
                                                         dtype, ws.payload, p.K, cam0, grad_targets, go)
#define ICGS_ADJ2(KC)                                                                                        \
  k_blend_adjoint2<KC><<<cb * p.tiles, kThreads2, 0, s>>>(ws.tile_off, ws.entries, p.capacity, ws.rec, p.n,  \
                                                           p.width, p.height, p.tiles_x, p.tiles, targets,     \
                                                           dtype, ws.payload, p.K, cam0, grad_targets, go)
  if (p.K == 1) ICGS_ADJ2(1);
  else if (p.K == 2) ICGS_ADJ2(2);
  else if (p.K == 3) ICGS_ADJ2(3);
  else if (p.K == 4) ICGS_ADJ2(4);
  else if (p.K <= 8) ICGS_ADJ(8);
  else if (p.K <= 16) ICGS_ADJ(16);
  else if (p.K <= 32) ICGS_ADJ(32);
  else ICGS_ADJ(64);
#undef ICGS_ADJ
#undef ICGS_ADJ2
  note_launches(1);
}

}  // namespace icgs
