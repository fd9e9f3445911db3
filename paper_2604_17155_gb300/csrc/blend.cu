// blend.cu -- the per-tile front-to-back walks (Eq. 2, Eq. 4-6), one CTA of 256 threads per
// 16x16 screen tile and one pixel per thread.
//
//   k_blend_accumulate  colorize: for every (pixel, Gaussian) blend weight w = alpha T (Eq. 4)
//                       accumulate V = sum w (Eq. 5) and S_k = sum w t_k (Eq. 6 numerator). The
//                       tile's pixels are reduced per Gaussian with warp shuffles and shared-memory
//                       atomics, then ONE global atomic group per (Gaussian, tile) lands in the
//                       per-(camera, Gaussian) accumulator.
//   k_blend_render      render: img_k = sum w C_k (Eq. 1-3) with C from the payload.
//   k_blend_adjoint     gradient: dL/dt_k = sum w a_k and, per Gaussian, dL/do = sum over pixels of
//                       (g T - sum_{n>m} g_n w_n / (1-alpha)) * alpha/o with g = beta + a . t.
//
// Warp w of a CTA covers the 8x4 pixel block ((w&1)*8, (w>>1)*4) of the tile, so a small Gaussian
// touches few warps; warps whose pixels all stopped skip the batch. Every kernel evaluates
// alpha and the transmittance update through blend_step(), written with explicit round-to-nearest
// intrinsics so that all walks take the same threshold decisions for the same inputs.
#include <cuda_runtime.h>

#include "icgs_device.cuh"
#include "icgs_internal.h"

namespace icgs {

namespace {

constexpr int kThreads = 256;
constexpr int kBatch = 64;
constexpr unsigned kFull = 0xFFFFFFFFu;

struct TileCtx {
  int j, t, px, py;
  bool inside;
  float pxf, pyf;
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
  c.px = txi * kTile + (warp & 1) * 8 + (lane & 7);
  c.py = tyi * kTile + (warp >> 1) * 4 + (lane >> 3);
  c.inside = c.px < width && c.py < height;
  c.pxf = (float)c.px + 0.5f;
  c.pyf = (float)c.py + 0.5f;
  const uint32_t b = min(tile_off[bid], capacity);
  uint32_t e = min(tile_off[bid + 1], capacity);
  if (e < b) e = b;
  c.b = b;
  c.len = e - b;
  return c;
}

// One step of the walk for Gaussian record (A, Bv) at pixel centre (pxf, pyf).
// Returns the weight w = alpha T (0 if skipped); sets `done` when the pixel stops here.
// e_out receives exp(-q/2) and capped whether alpha hit 0.99 (both only meaningful if w > 0).
__device__ __forceinline__ float blend_step(const float4 A, const float4 Bv, float pxf, float pyf,
                                            float& T, bool& done, float& alpha_out, float& e_out,
                                            bool& capped) {
  const float dx = __fsub_rn(pxf, A.x), dy = __fsub_rn(pyf, A.y);
  // q = a dx^2 + 2 b dx dy + c dy^2
  const float q = __fmaf_rn(__fmul_rn(A.z, dx), dx,
                            __fmaf_rn(__fmul_rn(__fmul_rn(2.0f, A.w), dx), dy, __fmul_rn(__fmul_rn(Bv.x, dy), dy)));
  // beyond the support threshold (with margin) alpha < 1/255 for certain: skip the exponential
  if (!(q <= __fmaf_rn(Bv.z, 1.0001f, 1e-4f))) return 0.0f;
  const float e = __expf(__fmul_rn(-0.5f, q));
  const float oe = __fmul_rn(Bv.y, e);
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
__device__ __forceinline__ void load_batch(const uint64_t* __restrict__ entries, uint32_t first, int nb,
                                           const ProjRec* __restrict__ rec_cam, int64_t n, float4* s_a,
                                           float4* s_b, uint32_t* s_id) {
  if ((int)threadIdx.x < nb) {
    const uint32_t id = min((uint32_t)entries[first + threadIdx.x], (uint32_t)(n - 1));
    const ProjRec r = rec_cam[id];
    s_id[threadIdx.x] = id;
    s_a[threadIdx.x] = r.a;
    s_b[threadIdx.x] = r.b;
  }
}

__device__ __forceinline__ void add_pair_count(uint32_t npairs, DevStatus* status) {
  const uint32_t warp_sum = __reduce_add_sync(kFull, npairs);
  if ((threadIdx.x & 31) == 0 && warp_sum) atomicAdd((unsigned long long*)&status->contrib_pairs, (unsigned long long)warp_sum);
}

// ------------------------------------------------------------------------------------------
// colorize: V and S per (camera, Gaussian)
// ------------------------------------------------------------------------------------------
template <int KC>
__global__ void __launch_bounds__(kThreads) k_blend_accumulate(
    const uint32_t* __restrict__ tile_off, const uint64_t* __restrict__ entries, uint32_t capacity,
    const ProjRec* __restrict__ rec, int64_t n, int width, int height, int tiles_x, int tiles,
    const void* __restrict__ targets, int dtype, int K, int k0, int cam0, float* __restrict__ acc,
    int64_t acc_cam_stride, DevStatus* status) {
  __shared__ float4 s_a[kBatch], s_b[kBatch];
  __shared__ uint32_t s_id[kBatch];
  __shared__ float s_acc[kBatch][KC + 1];
  const TileCtx c = tile_ctx(tile_off, capacity, tiles, tiles_x, width, height);
  const int lane = threadIdx.x & 31;
  float tv[KC];
#pragma unroll
  for (int k = 0; k < KC; ++k) tv[k] = 0.0f;
  if (c.inside) {
    const int64_t base = (((int64_t)(cam0 + c.j) * height + c.py) * width + c.px) * K + k0;
#pragma unroll
    for (int k = 0; k < KC; ++k)
      if (k0 + k < K) tv[k] = load_target(targets, base + k, dtype);
  }
  for (int k = threadIdx.x; k < kBatch * (KC + 1); k += kThreads) (&s_acc[0][0])[k] = 0.0f;
  const ProjRec* rec_cam = rec + (int64_t)c.j * n;
  float* acc_cam = acc + (int64_t)c.j * acc_cam_stride;
  float T = 1.0f;
  bool done = !c.inside;
  uint32_t npairs = 0;
  for (uint32_t start = 0; start < c.len; start += kBatch) {
    const int nb = (int)min((uint32_t)kBatch, c.len - start);
    __syncthreads();
    load_batch(entries, c.b + start, nb, rec_cam, n, s_a, s_b, s_id);
    __syncthreads();
    if (!__all_sync(kFull, done)) {
      for (int g = 0; g < nb; ++g) {
        float w = 0.0f, al, ex;
        bool cap;
        if (!done) w = blend_step(s_a[g], s_b[g], c.pxf, c.pyf, T, done, al, ex, cap);
        if (__any_sync(kFull, w > 0.0f)) {
          npairs += w > 0.0f;
          float v[KC + 1];
          v[0] = w;
#pragma unroll
          for (int k = 0; k < KC; ++k) v[k + 1] = w * tv[k];
#pragma unroll
          for (int k = 0; k <= KC; ++k) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(kFull, v[k], o);
          }
          if (lane == 0) {
#pragma unroll
            for (int k = 0; k <= KC; ++k) atomicAdd(&s_acc[g][k], v[k]);
          }
        }
      }
    }
    __syncthreads();
    if ((int)threadIdx.x < nb) {
      const int g = threadIdx.x;
      if (s_acc[g][0] > 0.0f) {
        float* dst = acc_cam + (int64_t)s_id[g] * (1 + K);
        if constexpr (KC == 3) {
          if (K == 3) {
            atomicAdd(reinterpret_cast<float4*>(dst), make_float4(s_acc[g][0], s_acc[g][1], s_acc[g][2], s_acc[g][3]));
          } else {
            if (k0 == 0) atomicAdd(dst, s_acc[g][0]);
            for (int k = 0; k < KC && k0 + k < K; ++k) atomicAdd(dst + 1 + k0 + k, s_acc[g][k + 1]);
          }
        } else {
          if (k0 == 0) atomicAdd(dst, s_acc[g][0]);
#pragma unroll
          for (int k = 0; k < KC; ++k)
            if (k0 + k < K) atomicAdd(dst + 1 + k0 + k, s_acc[g][k + 1]);
        }
#pragma unroll
        for (int k = 0; k <= KC; ++k) s_acc[g][k] = 0.0f;
      }
    }
    if (__syncthreads_and(done)) break;
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
  __shared__ float4 s_a[kBatch], s_b[kBatch];
  __shared__ uint32_t s_id[kBatch];
  __shared__ float s_col[kBatch][KC];
  const TileCtx c = tile_ctx(tile_off, capacity, tiles, tiles_x, width, height);
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
    load_batch(entries, c.b + start, nb, rec_cam, n, s_a, s_b, s_id);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nb * KC; idx += kThreads) {
      const int g = idx / KC, k = idx - g * KC;
      s_col[g][k] = k0 + k < K ? pay_cam[(int64_t)s_id[g] * K + k0 + k] : 0.0f;
    }
    __syncthreads();
    if (!__all_sync(kFull, done)) {
      for (int g = 0; g < nb && !done; ++g) {
        float al, ex;
        bool cap;
        const float w = blend_step(s_a[g], s_b[g], c.pxf, c.pyf, T, done, al, ex, cap);
        if (w > 0.0f) {
#pragma unroll
          for (int k = 0; k < KC; ++k) img[k] = fmaf(w, s_col[g][k], img[k]);
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

// ------------------------------------------------------------------------------------------
// adjoint: dL/dt and dL/do. Payload per (camera, Gaussian) = (a_0..a_{K-1}, beta).
// ------------------------------------------------------------------------------------------
template <int KC>
__global__ void __launch_bounds__(kThreads) k_blend_adjoint(
    const uint32_t* __restrict__ tile_off, const uint64_t* __restrict__ entries, uint32_t capacity,
    const ProjRec* __restrict__ rec, int64_t n, int width, int height, int tiles_x, int tiles,
    const void* __restrict__ targets, int dtype, const float* __restrict__ payload, int K, int cam0,
    float* __restrict__ grad_t, float* __restrict__ grad_o) {
  __shared__ float4 s_a[kBatch], s_b[kBatch];
  __shared__ uint32_t s_id[kBatch];
  __shared__ float s_pay[kBatch][KC + 1];
  __shared__ float s_go[kBatch];
  const TileCtx c = tile_ctx(tile_off, capacity, tiles, tiles_x, width, height);
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
      load_batch(entries, c.b + start, nb, rec_cam, n, s_a, s_b, s_id);
      __syncthreads();
      for (int idx = threadIdx.x; idx < nb * (KC + 1); idx += kThreads) {
        const int g = idx / (KC + 1), k = idx - g * (KC + 1);
        float v = 0.0f;
        if (k < KC) { if (k < K) v = pay_cam[(int64_t)s_id[g] * (K + 1) + k]; }
        else v = pay_cam[(int64_t)s_id[g] * (K + 1) + K];
        s_pay[g][k] = v;
      }
      __syncthreads();
      if (!__all_sync(kFull, done)) {
        for (int g = 0; g < nb && !done; ++g) {
          float al, ex;
          bool cap;
          const float w = blend_step(s_a[g], s_b[g], c.pxf, c.pyf, T, done, al, ex, cap);
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
    load_batch(entries, c.b + start, nb, rec_cam, n, s_a, s_b, s_id);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nb * (KC + 1); idx += kThreads) {
      const int g = idx / (KC + 1), k = idx - g * (KC + 1);
      float v = 0.0f;
      if (k < KC) { if (k < K) v = pay_cam[(int64_t)s_id[g] * (K + 1) + k]; }
      else v = pay_cam[(int64_t)s_id[g] * (K + 1) + K];
      s_pay[g][k] = v;
    }
    __syncthreads();
    if (!__all_sync(kFull, done)) {
      for (int g = 0; g < nb; ++g) {
        float d_o = 0.0f;
        if (!done) {
          const float Tm = T;
          float al = 0.0f, ex = 0.0f;
          bool cap = false;
          const float w = blend_step(s_a[g], s_b[g], c.pxf, c.pyf, T, done, al, ex, cap);
          if (w > 0.0f) {
            float gg = s_pay[g][KC];
#pragma unroll
            for (int k = 0; k < KC; ++k) gg = fmaf(s_pay[g][k], tv[k], gg);
            P = fmaf(gg, w, P);
            const float dalpha = gg * Tm - (F - P) / (1.0f - al);
            if (!cap) d_o = dalpha * ex;
          }
        }
        if (__any_sync(kFull, d_o != 0.0f)) {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) d_o += __shfl_xor_sync(kFull, d_o, o);
          if (lane == 0) atomicAdd(&s_go[g], d_o);
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

template <int KC>
void accumulate_chunk(const Problem& p, int cb, int cam0, const void* targets, int dtype, int k0,
                      const Workspace& ws, cudaStream_t s) {
  const int64_t stride = p.L == 0 ? 0 : p.n * (int64_t)(1 + p.K);
  k_blend_accumulate<KC><<<cb * p.tiles, kThreads, 0, s>>>(ws.tile_off, ws.entries, p.capacity, ws.rec, p.n,
                                                            p.width, p.height, p.tiles_x, p.tiles, targets, dtype,
                                                            p.K, k0, cam0, ws.acc, stride, ws.status);
  note_launches(1);
}

template <int KC>
void render_chunk(const Problem& p, int cb, int cam0, int k0, const Workspace& ws, float* images,
                  cudaStream_t s) {
  k_blend_render<KC><<<cb * p.tiles, kThreads, 0, s>>>(ws.tile_off, ws.entries, p.capacity, ws.rec, p.n,
                                                        p.width, p.height, p.tiles_x, p.tiles, ws.payload, p.K,
                                                        k0, cam0, images);
  note_launches(1);
}

}  // namespace

// Channels are processed in chunks of at most 16 per walk; the chunk width is the smallest
// instantiated width that covers the remaining channels.
void launch_blend_accumulate(const Problem& p, int cb, int cam0, const void* targets, int dtype,
                             const Workspace& ws, cudaStream_t s) {
  for (int k0 = 0; k0 < p.K; k0 += 16) {
    const int kc = p.K - k0;
    if (kc == 1) accumulate_chunk<1>(p, cb, cam0, targets, dtype, k0, ws, s);
    else if (kc == 2) accumulate_chunk<2>(p, cb, cam0, targets, dtype, k0, ws, s);
    else if (kc == 3) accumulate_chunk<3>(p, cb, cam0, targets, dtype, k0, ws, s);
    else if (kc == 4) accumulate_chunk<4>(p, cb, cam0, targets, dtype, k0, ws, s);
    else if (kc <= 8) accumulate_chunk<8>(p, cb, cam0, targets, dtype, k0, ws, s);
    else accumulate_chunk<16>(p, cb, cam0, targets, dtype, k0, ws, s);
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

void launch_blend_adjoint(const Problem& p, int cb, int cam0, const void* targets, int dtype,
                          const Workspace& ws, float* grad_targets, bool want_grad_o, cudaStream_t s) {
  float* go = want_grad_o ? ws.grad_o_acc : nullptr;
#define ICGS_ADJ(KC)                                                                                       \
  k_blend_adjoint<KC><<<cb * p.tiles, kThreads, 0, s>>>(ws.tile_off, ws.entries, p.capacity, ws.rec, p.n,  \
                                                         p.width, p.height, p.tiles_x, p.tiles, targets,     \
                                                         dtype, ws.payload, p.K, cam0, grad_targets, go)
  if (p.K == 1) ICGS_ADJ(1);
  else if (p.K == 2) ICGS_ADJ(2);
  else if (p.K == 3) ICGS_ADJ(3);
  else if (p.K == 4) ICGS_ADJ(4);
  else if (p.K <= 8) ICGS_ADJ(8);
  else if (p.K <= 16) ICGS_ADJ(16);
  else if (p.K <= 32) ICGS_ADJ(32);
  else ICGS_ADJ(64);
#undef ICGS_ADJ
  note_launches(1);
}

}  // namespace icgs
