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

struct TileCtx {
  int j, t, px, py;
  bool inside;
  float pxf, pyf;
  float wx0, wx1, wy0, wy1;  // pixel-centre rectangle of this thread's warp block
  uint32_t b, len;
};

__device__ __forceinline__ TileCtx tile_ctx(const uint32_t* tile_off, uint32_t capacity, int tiles,
                                            int tiles_x, int width, int height) {
  TileCtx c;
  const int bid = blockIdx.x;
  c.j = bid / tiles;
  c.t = bid - c.j * tiles;
  const int tyi = c.t / tiles_x, txi = c.t - tyi * tiles_x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int bx = txi * kTile + (warp & 1) * 8, by = tyi * kTile + (warp >> 1) * 4;
  c.px = bx + (lane & 7);
  c.py = by + (lane >> 3);
  c.inside = c.px < width && c.py < height;
  c.pxf = (float)c.px + 0.5f;
  c.pyf = (float)c.py + 0.5f;
  c.wx0 = (float)bx + 0.5f;
  c.wx1 = (float)bx + 7.5f;
  c.wy0 = (float)by + 0.5f;
  c.wy1 = (float)by + 3.5f;
  const uint32_t b = min(tile_off[bid], capacity);
  uint32_t e = min(tile_off[bid + 1], capacity);
  if (e < b) e = b;
  c.b = b;
  c.len = e - b;
  return c;
}

// Does the Gaussian's padded support box touch the warp's pixel block? (warp-uniform)
__device__ __forceinline__ bool warp_hits(const float4 box, const TileCtx& c) {
  return box.x + box.z >= c.wx0 && box.x - box.z <= c.wx1 && box.y + box.w >= c.wy0 && box.y - box.w <= c.wy1;
}

// Box-hit masks of this warp for the batch's Gaussians [base, base + 32): bit i is set when
// Gaussian base + i (< nb) touches the warp's pixel block. One Gaussian per lane, one ballot;
// iterating the set bits in ascending order keeps the depth order.
__device__ __forceinline__ uint32_t warp_hit_bits(const float4* s_box, int base, int nb, const TileCtx& c) {
  const int g = base + (int)(threadIdx.x & 31);
  const bool h = g < nb && warp_hits(s_box[g], c);
  return __ballot_sync(kFull, h);
}

// One step of the walk for a Gaussian (box, par, q threshold) at pixel centre (pxf, pyf).
// Returns the weight w = alpha T (0 if skipped); sets `done` when the pixel stops here.
// e_out receives exp(-q/2) and capped whether alpha hit 0.99 (both only meaningful if w > 0).
__device__ __forceinline__ float blend_step(const float4 box, const float4 par, float qthr, float pxf, float pyf,
                                            float& T, bool& done, float& alpha_out, float& e_out,
                                            bool& capped) {
  const float dx = __fsub_rn(pxf, box.x), dy = __fsub_rn(pyf, box.y);
  // q = a dx^2 + 2 b dx dy + c dy^2
  const float q = __fmaf_rn(__fmul_rn(par.x, dx), dx,
                            __fmaf_rn(__fmul_rn(__fmul_rn(2.0f, par.y), dx), dy, __fmul_rn(__fmul_rn(par.z, dy), dy)));
  // beyond the support threshold (with margin) alpha < 1/255 for certain: skip the exponential
  if (!(q <= qthr)) return 0.0f;
  const float e = __expf(__fmul_rn(-0.5f, q));
  const float oe = __fmul_rn(par.w, e);
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

// Slot ranges are only fully written when the pass fit its capacity; an overflowed pass (reported
// to the caller as ICGS_ERR_CAPACITY) may leave stale slots, so indices are clamped to the scene.
// The fast-reject threshold is 2 ln(255 o) with a relative margin of 1e-4 (and 1e-4 absolute),
// beyond which alpha < 1/255 holds by more than the float32 error of alpha.
__device__ __forceinline__ void load_batch(const uint64_t* __restrict__ entries, uint32_t first, int nb,
                                           const ProjRec* __restrict__ rec_cam, int64_t n, float4* s_box,
                                           float4* s_par, float* s_thr, uint32_t* s_id) {
  if ((int)threadIdx.x < nb) {
    const uint32_t id = min((uint32_t)entries[first + threadIdx.x], (uint32_t)(n - 1));
    const ProjRec r = rec_cam[id];
    s_id[threadIdx.x] = id;
    s_box[threadIdx.x] = r.box;
    s_par[threadIdx.x] = r.par;
    s_thr[threadIdx.x] = __fmaf_rn(2.0f * logf(255.0f * r.par.w), 1.0001f, 1e-4f);
  }
}

__device__ __forceinline__ void add_pair_count(uint32_t npairs, DevStatus* status) {
  const uint32_t warp_sum = __reduce_add_sync(kFull, npairs);
  if ((threadIdx.x & 31) == 0 && warp_sum) atomicAdd((unsigned long long*)&status->contrib_pairs, (unsigned long long)warp_sum);
}

}  // namespace walk
}  // namespace icgs
