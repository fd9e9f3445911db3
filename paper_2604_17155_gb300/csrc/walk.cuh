// walk.cuh -- the per-pixel front-to-back step shared by every tile walk (Eq. 2, Eq. 4): the CUDA-core
// accumulate / render / adjoint kernels and the tensor-core accumulate kernel all take their
// threshold decisions through these functions, so they agree for the same inputs.
#pragma once

#include <cuda_runtime.h>

#include "icgs_device.cuh"
#include "icgs_internal.h"

namespace icgs {
namespace walk {

constexpr int kThreads = 256;
constexpr int kBatch = 64;
constexpr unsigned kFull = 0xFFFFFFFFu;

// Pixel coordinates in the walk are relative to the tile origin (ox, oy): the staged means are
// tile-relative too (load_batch), so dx = pixel centre - mean is formed from two small numbers and
// keeps the precision of the float-float mean that the projection wrote.
struct TileCtx {
  int j, t, px, py;
  bool inside;
  float ox, oy;              // tile origin in image pixels (exact integers)
  float pxf, pyf;            // this thread's pixel centre, tile-relative
  float wx0, wx1, wy0, wy1;  // pixel-centre rectangle of this thread's warp block, tile-relative
  uint32_t b, len;
};

// ROWS = 1: CTAs of 256 threads, warp w covers the 8x4 block ((w&1)*8, (w>>1)*4) with one pixel
// per lane. ROWS = 2: CTAs of 128 threads, warp w covers the 8x8 block ((w&1)*8, (w>>1)*8) and lane
// l the two pixels (l&7, l>>3) and (l&7, (l>>3) + 4) of it; px, py, pyf and inside then describe
// the first of the two (the second is 4 rows below).
template <int ROWS = 1>
__device__ __forceinline__ TileCtx tile_ctx(const uint32_t* tile_off, uint32_t capacity, int tiles,
                                            int tiles_x, int width, int height) {
  TileCtx c;
  const int bid = blockIdx.x;
  c.j = bid / tiles;
  c.t = bid - c.j * tiles;
  const int tyi = c.t / tiles_x, txi = c.t - tyi * tiles_x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ox = txi * kTile, oy = tyi * kTile;
  const int bx = (warp & 1) * 8, by = (warp >> 1) * 4 * ROWS;  // warp block, tile-relative
  c.px = ox + bx + (lane & 7);
  c.py = oy + by + (lane >> 3);
  c.inside = c.px < width && c.py < height;
  c.ox = (float)ox;
  c.oy = (float)oy;
  c.pxf = (float)(bx + (lane & 7)) + 0.5f;
  c.pyf = (float)(by + (lane >> 3)) + 0.5f;
  c.wx0 = (float)bx + 0.5f;
  c.wx1 = (float)bx + 7.5f;
  c.wy0 = (float)by + 0.5f;
  c.wy1 = (float)(by + 4 * ROWS) - 0.5f;
  const uint32_t b = min(tile_off[bid], capacity);
  uint32_t e = min(tile_off[bid + 1], capacity);
  if (e < b) e = b;
  c.b = b;
  c.len = e - b;
  return c;
}

// The tile's depth-ordered list: its slot range in global memory, sorted by the tile sort before
// the walk. Keys are unique ((depth bits << 32) | index), so the ascending order is depth order
// with ties in index order.
__device__ __forceinline__ const unsigned long long* tile_list(const uint64_t* __restrict__ entries, uint32_t b) {
  return reinterpret_cast<const unsigned long long*>(entries) + b;
}

// A Gaussian of the current batch as the walk evaluates it, staged in shared memory:
//   geo  = (mean_x - ox, mean_y - oy, A, Bc)
//   aux  = (C, opacity, E_thr, packed half-sizes: the record's box.w, unused by the step)
//   half = (half-width, half-height) of the support box (read by the warp ballot only)
// with the conic (a, b, c) scaled by -log2(e)/2: A = -a log2(e)/2, Bc = -b log2(e), C = -c log2(e)/2,
// so that E = A dx^2 + Bc dx dy + C dy^2 = -q log2(e)/2 and exp(-q/2) = 2^E. E_thr is the fast-reject
// threshold 2 ln(255 o) in the same units (E < E_thr => alpha < 1/255 for certain).
constexpr float kHalfLog2e = 0.72134752044448170f;  // log2(e) / 2

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Does the Gaussian's padded support box touch the warp's pixel block? (warp-uniform)
__device__ __forceinline__ bool warp_hits(const float4 geo, const float2 half, const TileCtx& c) {
  return geo.x + half.x >= c.wx0 && geo.x - half.x <= c.wx1 && geo.y + half.y >= c.wy0 && geo.y - half.y <= c.wy1;
}

// Can blend_step take the Gaussian at some pixel centre of the warp's block, i.e. can
// E = A dx^2 + Bc dx dy + C dy^2 reach E_thr there? E is concave with its peak (0) at the mean. Over
// the rectangle R of the block's pixel centres it peaks at the mean if the mean lies in R, else on
// the edge of R that faces the mean: x = the nearer x-edge when the mean lies outside R in x, or
// y = the nearer y-edge when it lies outside in y (from a point of R off those edges, a small step
// toward the mean stays in R and raises E), at the optimum of E along that edge, clamped to it.
// The test rejects only when that peak falls short of E_thr by more than a rounding margin
// (1e-5 of the terms' magnitude), far above the float32 error of the peak and of the per-pixel E,
// so it never drops a Gaussian that some pixel's blend_step would take.
__device__ __forceinline__ bool ellipse_reaches_block(const float4 geo, const float4 aux, const TileCtx& c) {
  const float x0 = c.wx0 - geo.x, x1 = c.wx1 - geo.x;  // dx over the block
  const float y0 = c.wy0 - geo.y, y1 = c.wy1 - geo.y;  // dy over the block
  const bool out_x = x0 > 0.0f || x1 < 0.0f, out_y = y0 > 0.0f || y1 < 0.0f;
  if (!out_x && !out_y) return true;
  const float A = geo.z, Bc = geo.w, C = aux.x;  // A, C < 0
  float best = -INFINITY, mag = 0.0f;
  if (out_x) {
    const float dx = x0 > 0.0f ? x0 : x1;
    const float dy = fminf(fmaxf(__fdividef(-Bc * dx, 2.0f * C), y0), y1);
    best = (A * dx + Bc * dy) * dx + C * dy * dy;
    mag = (fabsf(A * dx) + fabsf(Bc * dy)) * fabsf(dx) + fabsf(C * dy) * fabsf(dy);
  }
  if (out_y) {
    const float dy = y0 > 0.0f ? y0 : y1;
    const float dx = fminf(fmaxf(__fdividef(-Bc * dy, 2.0f * A), x0), x1);
    const float e = (A * dx + Bc * dy) * dx + C * dy * dy;
    const float m = (fabsf(A * dx) + fabsf(Bc * dy)) * fabsf(dx) + fabsf(C * dy) * fabsf(dy);
    best = fmaxf(best, e);
    mag = fmaxf(mag, m);
  }
  return best + 1e-5f * mag + 1e-6f >= aux.z;
}

// Hit masks of this warp for the batch's Gaussians [base, base + 32): bit i is set when
// Gaussian base + i (< nb) touches the warp's pixel block: its box, and with ELLIPSE also its
// ellipse. One Gaussian per lane, one ballot; iterating the set bits in ascending order keeps the
// depth order. The ellipse test removes about 15% of the box hits of an 8x8 block; it pays in the
// issue-bound accumulate walks and costs latency in the tensor-core walk, so each walk chooses.
template <bool ELLIPSE = false>
__device__ __forceinline__ uint32_t warp_hit_bits(const float4* s_geo, const float4* s_aux, const float2* s_half,
                                                  int base, int nb, const TileCtx& c) {
  const int g = base + (int)(threadIdx.x & 31);
  bool h = false;
  if (g < nb) {
    const float4 geo = s_geo[g];
    h = warp_hits(geo, s_half[g], c);
    if constexpr (ELLIPSE) h = h && ellipse_reaches_block(geo, s_aux[g], c);
  }
  return __ballot_sync(kFull, h);
}

// One step of the walk for a staged Gaussian (geo, aux) at the tile-relative pixel centre
// (pxf, pyf). Returns the weight w = alpha T (0 if skipped); sets `done` when the pixel stops here.
// e_out receives exp(-q/2) and capped whether alpha hit 0.99 (both only meaningful if w > 0).
__device__ __forceinline__ float blend_step(const float4 geo, const float4 aux, float pxf, float pyf, float& T,
                                            bool& done, float& alpha_out, float& e_out, bool& capped) {
  const float dx = __fsub_rn(pxf, geo.x), dy = __fsub_rn(pyf, geo.y);
  // E = (A dx + Bc dy) dx + (C dy) dy
  const float E = __fmaf_rn(__fmaf_rn(geo.z, dx, __fmul_rn(geo.w, dy)), dx, __fmul_rn(__fmul_rn(aux.x, dy), dy));
  // beyond the support threshold (with margin) alpha < 1/255 for certain: skip the exponential
  if (!(E >= aux.z)) return 0.0f;
  const float e = ex2_approx(E);
  const float oe = __fmul_rn(aux.y, e);
  const float alpha = fminf(kAlphaMax, oe);
  if (!(alpha >= kAlphaMin)) return 0.0f;
  const float tT = __fmul_rn(T, __fsub_rn(1.0f, alpha));
  if (tT < kTMin) {
    done = true;
    return 0.0f;
  }
  const float w = __fmul_rn(alpha, T);
  T = tT;
  alpha_out = alpha;
  e_out = e;
  capped = !(oe < kAlphaMax);
  return w;
}

// blend_step without branches, for walks that only need w: the same decisions (the fast reject,
// alpha >= 1/255, the stop when T (1 - alpha) < 1e-4) taken as predicates on values that every
// lane computes, so a warp whose lanes disagree does not split. blend_alpha is the part that does
// not depend on T; blend_take applies one alpha to the pixel's transmittance and returns w (0 if
// skipped), counting a taken step in npairs. With LIVE a pixel already done takes nothing (for walks
// that call it on every pixel). With TEXP the walk carries T scaled by 2^TEXP (from 2^TEXP down), so
// that w comes out scaled by 2^TEXP too; the stop compares with the threshold scaled the same way.
// Scaling by a power of two commutes with rounding for these normal values, so the decisions and
// the scaled weights are exactly those of the unscaled step.
struct StepAlpha {
  float alpha;
  bool ok;  // past the fast reject and alpha >= 1/255
};
__device__ __forceinline__ StepAlpha blend_alpha(const float4 geo, const float4 aux, float pxf, float pyf) {
  const float dx = __fsub_rn(pxf, geo.x), dy = __fsub_rn(pyf, geo.y);
  const float E = __fmaf_rn(__fmaf_rn(geo.z, dx, __fmul_rn(geo.w, dy)), dx, __fmul_rn(__fmul_rn(aux.x, dy), dy));
  const float alpha = fminf(kAlphaMax, __fmul_rn(aux.y, ex2_approx(E)));
  return {alpha, E >= aux.z && alpha >= kAlphaMin};
}
// blend_alpha without the fast reject, for walks that compute alpha for every step anyway: the
// reject only ever drops steps whose alpha is below 1/255 (E < E_thr implies o 2^E < 1/255 by its
// margin), so alpha >= 1/255 alone takes the same decisions. Alpha is clamped by a select, which
// keeps a NaN product NaN so that it fails the test, as it failed the reject. aux.z is not read.
__device__ __forceinline__ StepAlpha blend_alpha_noreject(const float4 geo, const float4 aux, float pxf, float pyf) {
  const float dx = __fsub_rn(pxf, geo.x), dy = __fsub_rn(pyf, geo.y);
  const float E = __fmaf_rn(__fmaf_rn(geo.z, dx, __fmul_rn(geo.w, dy)), dx, __fmul_rn(__fmul_rn(aux.x, dy), dy));
  const float oe = __fmul_rn(aux.y, ex2_approx(E));
  const float alpha = oe > kAlphaMax ? kAlphaMax : oe;
  return {alpha, alpha >= kAlphaMin};
}

template <bool LIVE = false, int TEXP = 0>
__device__ __forceinline__ float blend_take(const StepAlpha a, float& T, bool& done, uint32_t& npairs) {
  constexpr float kTMinScaled = kTMin * (float)(1 << TEXP);
  const float tT = __fmul_rn(T, __fsub_rn(1.0f, a.alpha));
  const bool take = (!LIVE || !done) && a.ok;
  const bool stop = take && tT < kTMinScaled;
  const bool keep = take && !stop;
  npairs += keep ? 1u : 0u;
  const float w = keep ? __fmul_rn(a.alpha, T) : 0.0f;
  T = keep ? tT : T;
  done = done || stop;
  return w;
}
template <bool LIVE = false>
__device__ __forceinline__ float blend_weight(const float4 geo, const float4 aux, float pxf, float pyf, float& T,
                                              bool& done, uint32_t& npairs) {
  return blend_take<LIVE>(blend_alpha(geo, aux, pxf, pyf), T, done, npairs);
}

// Slot ranges are only fully written when the pass fit its capacity; an overflowed pass (reported
// to the caller as ICGS_ERR_CAPACITY) may leave stale slots, so indices are clamped to the scene.
// The staged mean is relative to the tile origin (ox, oy): the record's hi and lo parts are
// combined there, where the result is small and float32 holds it closely. The fast-reject
// threshold is 2 ln(255 o) with a relative margin of 1e-4 (and 1e-4 absolute), beyond which
// alpha < 1/255 holds by more than the float32 error of alpha.
// The staged geometry of one record: the tile-relative mean and the scaled conic (A, Bc).
__device__ __forceinline__ float4 stage_geo(const ProjRec& r, float ox, float oy) {
  const float2 lo = unpack_half2(r.box.z);
  return make_float4(__fadd_rn(__fsub_rn(r.box.x, ox), __fmul_rn(lo.x, kMeanLoScaleInv)),
                     __fadd_rn(__fsub_rn(r.box.y, oy), __fmul_rn(lo.y, kMeanLoScaleInv)), -kHalfLog2e * r.par.x,
                     -2.0f * kHalfLog2e * r.par.y);
}

// The staged (geo, aux) of one record; aux.w carries the record's packed support half-sizes.
__device__ __forceinline__ void stage_record(const ProjRec& r, float ox, float oy, float4& geo, float4& aux) {
  const float qthr = __fmaf_rn(2.0f * logf(255.0f * r.par.w), 1.0001f, 1e-4f);
  geo = stage_geo(r, ox, oy);
  aux = make_float4(-kHalfLog2e * r.par.z, r.par.w, -kHalfLog2e * qthr, r.box.w);
}

__device__ __forceinline__ void load_batch(const unsigned long long* list, uint32_t first, int nb,
                                           const ProjRec* __restrict__ rec_cam, int64_t n, float ox, float oy,
                                           float4* s_geo, float4* s_aux, float2* s_half, uint32_t* s_id) {
  if ((int)threadIdx.x < nb) {
    const uint32_t id = min((uint32_t)list[first + threadIdx.x], (uint32_t)(n - 1));
    const ProjRec r = rec_cam[id];
    float4 geo, aux;
    stage_record(r, ox, oy, geo, aux);
    s_id[threadIdx.x] = id;
    s_geo[threadIdx.x] = geo;
    s_aux[threadIdx.x] = aux;
    s_half[threadIdx.x] = unpack_half2(r.box.w);
  }
}

// load_batch without the separate half-size array: the ballot reads the half-sizes from aux.w
// (warp_hit_bits_packed).
__device__ __forceinline__ void load_batch_packed(const unsigned long long* list, uint32_t first, int nb,
                                                  const ProjRec* __restrict__ rec_cam, int64_t n, float ox, float oy,
                                                  float4* s_geo, float4* s_aux, uint32_t* s_id) {
  if ((int)threadIdx.x < nb) {
    const uint32_t id = min((uint32_t)list[first + threadIdx.x], (uint32_t)(n - 1));
    const ProjRec r = rec_cam[id];
    float4 geo, aux;
    stage_record(r, ox, oy, geo, aux);
    s_id[threadIdx.x] = id;
    s_geo[threadIdx.x] = geo;
    s_aux[threadIdx.x] = aux;
  }
}

// warp_hit_bits (box test only) for batches staged by load_batch_packed.
__device__ __forceinline__ uint32_t warp_hit_bits_packed(const float4* s_geo, const float4* s_aux, int base, int nb,
                                                         const TileCtx& c) {
  const int g = base + (int)(threadIdx.x & 31);
  bool h = false;
  if (g < nb) h = warp_hits(s_geo[g], unpack_half2(s_aux[g].w), c);
  return __ballot_sync(kFull, h);
}

// Flags a non-finite target value in the status block (the call then fails with
// ICGS_ERR_NONFINITE_INPUT); the atomic runs only on that rare path.
template <int N>
__device__ __forceinline__ void check_finite(const float (&v)[N], DevStatus* status) {
  bool bad = false;
#pragma unroll
  for (int k = 0; k < N; ++k) bad |= !isfinite(v[k]);
  if (bad) atomicOr(&status->flags, kFlagNonfinite);
}

__device__ __forceinline__ void add_pair_count(uint32_t npairs, DevStatus* status) {
  const uint32_t warp_sum = __reduce_add_sync(kFull, npairs);
  if ((threadIdx.x & 31) == 0 && warp_sum) atomicAdd((unsigned long long*)&status->contrib_pairs, (unsigned long long)warp_sum);
}

}  // namespace walk
}  // namespace icgs
