// project.cu -- projection of every (camera, Gaussian) pair and binning into 16x16 screen tiles.
//
// Per pair (Eq. 1 with the 3DGS EWA model the paper renders with): camera-space mean, culling at
// the near plane, 2D covariance J W Sigma W^T J^T + 0.3 I, its inverse (the conic), the projected
// mean, the support threshold q <= 2 ln(255 o) (alpha >= 1/255), and the rectangle of tiles whose
// pixel centres can fall inside that support. The depth used for ordering and for the near-plane
// test is the float32 key fma(W22, z, fma(W21, y, fma(W20, x, W23))), three correctly rounded fused
// multiply-adds, so it is a well-defined function of the inputs that any IEEE implementation
// reproduces bit for bit. No step of the projection uses FP64 (about 1/64 of the FP32 rate here).
//
// Precision. alpha = o exp(-q/2) is sensitive to the offset between a pixel centre and the mean:
// for a one-pixel Gaussian an error of 1e-4 px in the mean moves alpha by about 1e-4 relative,
// and a float32 mean near x = 400 is already rounded by 1.5e-5 px. The projected mean is therefore
// evaluated in float-float arithmetic (error-free products and sums, Dekker/Knuth) and stored as
// hi + lo; the walk subtracts it from tile-relative pixel centres. The conic is formed from
// P = T M (T = J W, Sigma = M M^T), with det(P P^T + 0.3 I) = sum of the squared 2x2 minors of P
// + 0.3 tr(P P^T) + 0.09 (Cauchy-Binet): a sum of non-negative terms, where the textbook
// a c - b^2 cancels for thin projected Gaussians.
//
// Binning is a counting sort: k_project_hist counts instances per tile, an exclusive scan turns
// counts into offsets, and k_scatter_hist writes (depth key << 32 | index) into each tile's slot
// range. Both work on CTAs of 2048 Gaussians of one camera that count in a shared-memory
// histogram of the camera's tiles, so a global atomic is issued per (CTA, touched tile) rather
// than per instance. The order inside a tile is fixed later by the per-tile sort.
#include <cuda_runtime.h>

#include <algorithm>

#include "icgs_device.cuh"
#include "icgs_internal.h"

namespace icgs {

namespace {

// error-free transformations: s + e = a + b exactly (Knuth), p + e = a b exactly (FMA)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// a x + b y + c z + d as hi + lo (float-float; relative error near 2^-44 of the largest term)
__device__ __forceinline__ float affine_ff(float a, float b, float c, float d, float x, float y, float z, float& lo) {
  float p0, e0, p1, e1, p2, e2, s, t0, t1, t2;
  two_prod(a, x, p0, e0);
  two_prod(b, y, p1, e1);
  two_prod(c, z, p2, e2);
  two_sum(p0, p1, s, t0);
  two_sum(s, p2, s, t1);
  two_sum(s, d, s, t2);
  const float l = __fadd_rn(__fadd_rn(__fadd_rn(e0, e1), __fadd_rn(e2, t0)), __fadd_rn(t1, t2));
  const float hi = __fadd_rn(s, l);
  lo = __fsub_rn(l, __fsub_rn(hi, s));
  return hi;
}

// f (uh + ul) / (zh + zl) + c as hi + lo; iz is a float32 reciprocal of zh. The quotient's
// correction comes from the remainder uh - qh zh, which one FMA gives exactly.
__device__ __forceinline__ float pixel_ff(float f, float c, float uh, float ul, float zh, float zl, float iz,
                                          float& lo) {
  const float qh = __fmul_rn(uh, iz);
  const float r = __fadd_rn(__fmaf_rn(-qh, zh, uh), __fsub_rn(ul, __fmul_rn(qh, zl)));
  const float ql = __fmul_rn(r, iz);
  float ph, pe, sh, se;
  two_prod(f, qh, ph, pe);
  pe = __fmaf_rn(f, ql, pe);
  two_sum(ph, c, sh, se);
  se = __fadd_rn(se, pe);
  const float hi = __fadd_rn(sh, se);
  lo = __fsub_rn(se, __fsub_rn(hi, sh));
  return hi;
}

// The depth ordering key (see the file comment).
__device__ __forceinline__ float depth_key(const DevCam& c, float x, float y, float z) {
  return __fmaf_rn(c.w[10], z, __fmaf_rn(c.w[9], y, __fmaf_rn(c.w[8], x, c.w[11])));
}

// The smallest float32 >= 1/255: for a float32 opacity o, o >= kOpacityMin exactly when o * 255 >= 1.
constexpr float kOpacityMin = 0x1.010102p-8f;

// Projects Gaussian i into camera c, writes its record and tile rectangle at slot ji and returns
// the rectangle (tx0, ty0, tx1, ty1); tx0 > tx1 when the Gaussian has no pixel in the image.
// The parameters of one Gaussian as the projection reads them: mo = (mean, opacity),
// sq = (scale, quaternion w), qv = (quaternion x, y, z, unused); loaded by the caller (which may
// fetch them ahead of use). The record goes to rec[ji] (indexed by camera and Gaussian), the tile
// rectangle to rect[jp] (indexed by camera and processing position).
__device__ __forceinline__ int4 project_pair(const float4 mo, const float4 sq, const float4 qv, const DevCam& c,
                                             int width, int height, float near_z, int64_t ji, int64_t jp,
                                             ProjRec* __restrict__ rec, uint4* __restrict__ rect) {
  const int4 none = make_int4(1, 0, 0, 0);
  const float mx3 = mo.x, my3 = mo.y, mz3 = mo.z;
  const float o = mo.w;
  const float key = depth_key(c, mx3, my3, mz3);
  if (!(key > near_z) || !isfinite(key) || !(o >= kOpacityMin) || !isfinite(o)) {
    rect[jp] = make_uint4(0xFFFFFFFFu, 0u, 0u, 0u);
    return none;
  }
  float tz_lo, tx_lo, ty_lo;
  const float tz = affine_ff(c.w[8], c.w[9], c.w[10], c.w[11], mx3, my3, mz3, tz_lo);
  const float tx = affine_ff(c.w[0], c.w[1], c.w[2], c.w[3], mx3, my3, mz3, tx_lo);
  const float ty = affine_ff(c.w[4], c.w[5], c.w[6], c.w[7], mx3, my3, mz3, ty_lo);
  const float iz = 1.0f / tz;
  const float qthr = 2.0f * logf(255.0f * o);
  const float sx = sq.x, sy = sq.y, sz = sq.z;
  // a non-finite scale would give an unbounded support (NaN and zero quaternions fail the
  // determinant test below)
  if (!(isfinite(sx) && isfinite(sy) && isfinite(sz))) {
    rect[jp] = make_uint4(0xFFFFFFFFu, 0u, 0u, 0u);
    return none;
  }
  {
    // Early cull. Sigma'_xx = |T_0 M|^2 + 0.3 <= |J_0|^2 |R|^2 s_max^2 + 0.3 with
    // |J_0| <= (f/z) sqrt(1 + lim^2) (the Jacobian's clamp), so the support half-width is at most
    // sqrt(qthr (that bound)). A mean farther outside the image than this (plus a pixel) has no
    // pixel centre in its support: the box test below would reject it after the full covariance.
    const float smax = fmaxf(fmaxf(sx, sy), sz);
    const float fz = fmaxf(c.fx, c.fy) * iz;
    const float jb = 1.0f + fmaxf(c.limx * c.limx, c.limy * c.limy);
    const float hmax = sqrtf(fmaxf(qthr, 0.0f) * (fz * fz * jb * c.rnorm2 * smax * smax + 0.3f)) * 1.001f + 1.0f;
    const float mxa = fmaf(c.fx, tx * iz, c.cx), mya = fmaf(c.fy, ty * iz, c.cy);
    if (mxa + hmax < 0.0f || mxa - hmax > (float)width || mya + hmax < 0.0f || mya - hmax > (float)height) {
      rect[jp] = make_uint4(0xFFFFFFFFu, 0u, 0u, 0u);
      return none;
    }
  }

  // 3D covariance Sigma = M M^T with M = R(q) diag(s)
  float qw = sq.w, qx = qv.x, qy = qv.y, qz = qv.z;
  const float qn = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
  qw *= qn; qx *= qn; qy *= qn; qz *= qn;
  const float r00 = 1.f - 2.f * (qy * qy + qz * qz), r01 = 2.f * (qx * qy - qw * qz), r02 = 2.f * (qx * qz + qw * qy);
  const float r10 = 2.f * (qx * qy + qw * qz), r11 = 1.f - 2.f * (qx * qx + qz * qz), r12 = 2.f * (qy * qz - qw * qx);
  const float r20 = 2.f * (qx * qz - qw * qy), r21 = 2.f * (qy * qz + qw * qx), r22 = 1.f - 2.f * (qx * qx + qy * qy);
  const float m00 = r00 * sx, m01 = r01 * sy, m02 = r02 * sz;
  const float m10 = r10 * sx, m11 = r11 * sy, m12 = r12 * sz;
  const float m20 = r20 * sx, m21 = r21 * sy, m22 = r22 * sz;

  // EWA: T = J W (2x3), J at the clamped camera-space mean
  const float ux = fminf(c.limx, fmaxf(-c.limx, tx * iz));
  const float uy = fminf(c.limy, fmaxf(-c.limy, ty * iz));
  const float j00 = c.fx * iz, j02 = -c.fx * ux * iz;
  const float j11 = c.fy * iz, j12 = -c.fy * uy * iz;
  const float t00 = j00 * c.w[0] + j02 * c.w[8], t01 = j00 * c.w[1] + j02 * c.w[9], t02 = j00 * c.w[2] + j02 * c.w[10];
  const float t10 = j11 * c.w[4] + j12 * c.w[8], t11 = j11 * c.w[5] + j12 * c.w[9], t12 = j11 * c.w[6] + j12 * c.w[10];
  // Sigma' = P P^T + 0.3 I with P = T M (2x3)
  const float p00 = t00 * m00 + t01 * m10 + t02 * m20, p01 = t00 * m01 + t01 * m11 + t02 * m21;
  const float p02 = t00 * m02 + t01 * m12 + t02 * m22;
  const float p10 = t10 * m00 + t11 * m10 + t12 * m20, p11 = t10 * m01 + t11 * m11 + t12 * m21;
  const float p12 = t10 * m02 + t11 * m12 + t12 * m22;
  const float n0 = p00 * p00 + p01 * p01 + p02 * p02, n1 = p10 * p10 + p11 * p11 + p12 * p12;
  const float ca2 = n0 + 0.3f;
  const float cb2 = p00 * p10 + p01 * p11 + p02 * p12;
  const float cc2 = n1 + 0.3f;
  const float d01 = fmaf(p00, p11, -p01 * p10), d02 = fmaf(p00, p12, -p02 * p10), d12 = fmaf(p01, p12, -p02 * p11);
  const float det = (d01 * d01 + d02 * d02 + d12 * d12) + 0.3f * (n0 + n1) + 0.09f;
  float mx_lo, my_lo;
  const float mx = pixel_ff(c.fx, c.cx, tx, tx_lo, tz, tz_lo, iz, mx_lo);
  const float my = pixel_ff(c.fy, c.cy, ty, ty_lo, tz, tz_lo, iz, my_lo);
  if (!(det > 0.0f) || !isfinite(mx) || !isfinite(my)) {
    rect[jp] = make_uint4(0xFFFFFFFFu, 0u, 0u, 0u);
    return none;
  }
  const float idet = 1.0f / det;
  // x-extent of {q <= qthr} is sqrt(qthr * Sigma'_xx); pad so the box contains every pixel centre
  // that the blend kernel's own float32 alpha test can accept.
  const float hx = sqrtf(fmaxf(qthr, 0.0f) * ca2) * 1.0001f + 0.01f;
  const float hy = sqrtf(fmaxf(qthr, 0.0f) * cc2) * 1.0001f + 0.01f;
  const float fx0 = fmaxf(ceilf(mx - hx - 0.5f), 0.0f), fx1 = fminf(floorf(mx + hx - 0.5f), (float)(width - 1));
  const float fy0 = fmaxf(ceilf(my - hy - 0.5f), 0.0f), fy1 = fminf(floorf(my + hy - 0.5f), (float)(height - 1));
  if (!(fx0 <= fx1) || !(fy0 <= fy1)) {
    rect[jp] = make_uint4(0xFFFFFFFFu, 0u, 0u, 0u);
    return none;
  }
  const int tx0 = (int)fx0 / kTile, tx1 = (int)fx1 / kTile;
  const int ty0 = (int)fy0 / kTile, ty1 = (int)fy1 / kTile;
  ProjRec r;
  const bool lo_ok = fabsf(mx) < 1048576.0f && fabsf(my) < 1048576.0f;  // fp16 holds lo * 2^8 there
  r.box = make_float4(mx, my,
                      pack_half2(__float2half_rn(lo_ok ? mx_lo * kMeanLoScale : 0.0f),
                                 __float2half_rn(lo_ok ? my_lo * kMeanLoScale : 0.0f)),
                      pack_half2(__float2half_ru(hx), __float2half_ru(hy)));
  r.par = make_float4(cc2 * idet, -cb2 * idet, ca2 * idet, o);
  rec[ji] = r;
  rect[jp] = make_uint4((uint32_t)tx0 | ((uint32_t)ty0 << 16), (uint32_t)tx1 | ((uint32_t)ty1 << 16),
                        __float_as_uint(key), 0u);
  return make_int4(tx0, ty0, tx1, ty1);
}

// Gaussians per thread in the histogram kernels (a CTA takes 256 PT Gaussians of one camera). Each
// CTA zeroes and flushes one histogram bin per tile, so large tile grids take more Gaussians a
// thread, which spreads that per-CTA cost; smaller ones take fewer, which keeps more CTAs in flight.
// Measured choices: the projection 8 / 32 and the scatter 4 / 16 Gaussians a thread below / from
// 4,096 tiles.
constexpr int kBigTileGrid = 4096;
__host__ __device__ constexpr int hist_per_cta(int per_thread) { return 256 * per_thread; }
constexpr int kHistTiles = 12288;             // largest tile grid the shared-memory histograms take

// One CTA per (camera, 256 PT Gaussians): counts the CTA's instances per tile in shared memory, then
// adds each nonzero bin to the global count with one atomic. The camera is the fast index of the
// 1-D grid, so the CTAs of one chunk of Gaussians run together and read its parameters from DRAM
// once (a scene larger than L2 would otherwise be re-read for every camera).
template <int PT>
__global__ void __launch_bounds__(256, 4) k_project_hist(
    const float4* __restrict__ packed, const uint32_t* __restrict__ order, int64_t n, const DevCam* __restrict__ cams,
    int j0, int cbl, int width, int height, float near_z, int tiles_x, int tiles, ProjRec* __restrict__ rec,
    uint4* __restrict__ rect, uint32_t* __restrict__ tile_count) {
  extern __shared__ uint32_t s_hist[];
  const int64_t chunk = blockIdx.x / cbl;
  const int j = j0 + (int)(blockIdx.x - chunk * cbl);
  const DevCam& c = cams[j];
  for (int t = threadIdx.x; t < tiles; t += 256) s_hist[t] = 0u;
  __syncthreads();
  const int64_t p0 = chunk * hist_per_cta(PT);
  // the Gaussian at processing position q and its mean and opacity, fetched one step ahead
  int64_t i_next = 0;
  float4 mo_next = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  if (p0 + threadIdx.x < n) {
    i_next = order[p0 + threadIdx.x];
    mo_next = packed[3 * (p0 + threadIdx.x)];
  }
  for (int r = 0; r < PT; ++r) {
    const int64_t q = p0 + r * 256 + threadIdx.x;
    if (q >= n) break;
    const float4 mo = mo_next;
    const int64_t i = i_next;
    if (r + 1 < PT && q + 256 < n) {
      i_next = order[q + 256];
      mo_next = packed[3 * (q + 256)];
    }
    const int4 tr = project_pair(mo, packed[3 * q + 1], packed[3 * q + 2], c, width, height, near_z,
                                 (int64_t)j * n + i, (int64_t)j * n + q, rec, rect);
    for (int ty = tr.y; ty <= tr.w; ++ty)
      for (int tx = tr.x; tx <= tr.z; ++tx) atomicAdd(&s_hist[ty * tiles_x + tx], 1u);
  }
  __syncthreads();
  uint32_t* base = tile_count + (int64_t)j * tiles;
  for (int t = threadIdx.x; t < tiles; t += 256)
    if (s_hist[t]) atomicAdd(base + t, s_hist[t]);
}

// Fallback for tile grids beyond kHistTiles: one global atomic per instance.
__global__ void __launch_bounds__(256) k_project(
    const float4* __restrict__ packed, const uint32_t* __restrict__ order, int64_t n,
    const DevCam* __restrict__ cams, int width, int height, float near_z, int tiles_x, int tiles,
    ProjRec* __restrict__ rec, uint4* __restrict__ rect, uint32_t* __restrict__ tile_count) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (q >= n) return;
  const int64_t i = order[q];
  const int4 tr = project_pair(packed[3 * q], packed[3 * q + 1], packed[3 * q + 2], cams[j], width, height, near_z,
                               (int64_t)j * n + i, (int64_t)j * n + q, rec, rect);
  uint32_t* base = tile_count + (int64_t)j * tiles;
  for (int ty = tr.y; ty <= tr.w; ++ty)
    for (int tx = tr.x; tx <= tr.z; ++tx) atomicAdd(base + ty * tiles_x + tx, 1u);
}

__global__ void __launch_bounds__(256) k_scatter(
    int64_t n, const uint4* __restrict__ rect, const uint32_t* __restrict__ order, int tiles_x, int tiles,
    const uint32_t* __restrict__ tile_off, uint32_t* __restrict__ tile_cur, uint64_t* __restrict__ entries,
    uint32_t capacity, DevStatus* status) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (q >= n) return;
  const uint4 rc = rect[(int64_t)j * n + q];
  const int tx0 = rc.x & 0xFFFF, ty0 = rc.x >> 16, tx1 = rc.y & 0xFFFF, ty1 = rc.y >> 16;
  if (rc.x == 0xFFFFFFFFu) return;
  const uint64_t key = ((uint64_t)rc.z << 32) | (uint64_t)order[q];
  bool overflow = false;
  for (int ty = ty0; ty <= ty1; ++ty)
    for (int tx = tx0; tx <= tx1; ++tx) {
      const int64_t t = (int64_t)j * tiles + ty * tiles_x + tx;
      const uint32_t pos = atomicAdd(tile_cur + t, 1u);
      const uint64_t slot = (uint64_t)tile_off[t] + pos;
      if (slot < capacity) entries[slot] = key;
      else overflow = true;
    }
  if (overflow) atomicOr(&status->flags, kFlagOverflow);
}

// Same CTA tiling as k_project_hist (processing positions, rectangles indexed by position): the
// CTA counts its instances per tile, reserves one contiguous run per tile with a single global
// atomic, then places its instances with shared-memory cursors.
template <int PT>
__global__ void __launch_bounds__(256) k_scatter_hist(
    int64_t n, const uint4* __restrict__ rect, const uint32_t* __restrict__ order, int tiles_x, int tiles,
    const uint32_t* __restrict__ tile_off,
    uint32_t* __restrict__ tile_cur, uint64_t* __restrict__ entries, uint32_t capacity, DevStatus* status) {
  extern __shared__ uint32_t s_mem[];
  uint32_t* s_cnt = s_mem;          // [tiles] count, then running cursor
  uint32_t* s_base = s_mem + tiles;  // [tiles] start of the CTA's run in the tile's slot range
  const int j = blockIdx.y;
  for (int t = threadIdx.x; t < tiles; t += 256) s_cnt[t] = 0u;
  __syncthreads();
  // The rectangles are read kGroup at a time (all loads in flight before the first is used), and
  // the per-tile reservations kFlush tiles at a time, so that global round trips overlap.
  constexpr int kGroup = 4, kFlush = 8;
  static_assert(PT % kGroup == 0, "whole groups of rectangles");
  const int64_t i0 = (int64_t)blockIdx.x * hist_per_cta(PT);
  const uint4* rect_j = rect + (int64_t)j * n;
  for (int r0 = 0; r0 < PT; r0 += kGroup) {
    uint4 rcs[kGroup];
#pragma unroll
    for (int u = 0; u < kGroup; ++u) {
      const int64_t q = i0 + (r0 + u) * 256 + threadIdx.x;
      rcs[u] = q < n ? rect_j[q] : make_uint4(0xFFFFFFFFu, 0u, 0u, 0u);
    }
#pragma unroll
    for (int u = 0; u < kGroup; ++u) {
      const uint4 rc = rcs[u];
      if (rc.x == 0xFFFFFFFFu) continue;
      const int tx0 = rc.x & 0xFFFF, ty0 = rc.x >> 16, tx1 = rc.y & 0xFFFF, ty1 = rc.y >> 16;
      for (int ty = ty0; ty <= ty1; ++ty)
        for (int tx = tx0; tx <= tx1; ++tx) atomicAdd(&s_cnt[ty * tiles_x + tx], 1u);
    }
  }
  __syncthreads();
  const int64_t tj = (int64_t)j * tiles;
  for (int t0 = threadIdx.x; t0 < tiles; t0 += 256 * kFlush) {
    uint32_t cnt[kFlush], old[kFlush], off[kFlush];
#pragma unroll
    for (int u = 0; u < kFlush; ++u) {
      const int t = t0 + 256 * u;
      cnt[u] = t < tiles ? s_cnt[t] : 0u;
    }
#pragma unroll
    for (int u = 0; u < kFlush; ++u) {
      const int t = t0 + 256 * u;
      old[u] = 0u;
      off[u] = 0u;
      if (cnt[u]) {
        old[u] = atomicAdd(tile_cur + tj + t, cnt[u]);
        off[u] = tile_off[tj + t];
      }
    }
#pragma unroll
    for (int u = 0; u < kFlush; ++u) {
      const int t = t0 + 256 * u;
      if (t < tiles) {
        s_base[t] = off[u] + old[u];
        s_cnt[t] = 0u;
      }
    }
  }
  __syncthreads();
  bool overflow = false;
  for (int r0 = 0; r0 < PT; r0 += kGroup) {
    uint4 rcs[kGroup];
    uint32_t ids[kGroup];
#pragma unroll
    for (int u = 0; u < kGroup; ++u) {
      const int64_t q = i0 + (r0 + u) * 256 + threadIdx.x;
      rcs[u] = q < n ? rect_j[q] : make_uint4(0xFFFFFFFFu, 0u, 0u, 0u);
      ids[u] = q < n ? order[q] : 0u;
    }
#pragma unroll
    for (int u = 0; u < kGroup; ++u) {
      const uint4 rc = rcs[u];
      if (rc.x == 0xFFFFFFFFu) continue;
      const int tx0 = rc.x & 0xFFFF, ty0 = rc.x >> 16, tx1 = rc.y & 0xFFFF, ty1 = rc.y >> 16;
      const uint64_t key = ((uint64_t)rc.z << 32) | (uint64_t)ids[u];
      for (int ty = ty0; ty <= ty1; ++ty)
        for (int tx = tx0; tx <= tx1; ++tx) {
          const int t = ty * tiles_x + tx;
          const uint64_t slot = (uint64_t)s_base[t] + atomicAdd(&s_cnt[t], 1u);
          if (slot < capacity) entries[slot] = key;
          else overflow = true;
        }
    }
  }
  if (overflow) atomicOr(&status->flags, kFlagOverflow);
}

// ---- processing order: the Gaussians by cell of a 64^3 grid over the scene's bounding box, cells
// in Morton order. The CTAs of the projection and the scatter take consecutive positions of this
// order, so that each covers a compact part of the scene and touches few screen tiles (one global
// atomic per touched tile). Results do not depend on the order. ----
constexpr int kCellBits = 6;
constexpr int kCells = 1 << (3 * kCellBits);

// float <-> unsigned key with the same order (finite values)
__device__ __forceinline__ uint32_t f2key(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key2f(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// box[0..2] = min keys of x, y, z (initialised to 0xFFFFFFFF), box[3..5] = max keys (initialised to 0),
// over the finite means
__global__ void __launch_bounds__(256) k_bounds(const float* __restrict__ means, int64_t n, uint32_t* __restrict__ box) {
  uint32_t lo[3] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu}, hi[3] = {0u, 0u, 0u};
  for (int64_t i = blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
    const float x = means[3 * i], y = means[3 * i + 1], z = means[3 * i + 2];
    if (!(isfinite(x) && isfinite(y) && isfinite(z))) continue;
    const uint32_t k[3] = {f2key(x), f2key(y), f2key(z)};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      lo[a] = min(lo[a], k[a]);
      hi[a] = max(hi[a], k[a]);
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = __reduce_min_sync(0xFFFFFFFFu, lo[a]);
    hi[a] = __reduce_max_sync(0xFFFFFFFFu, hi[a]);
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      atomicMin(box + a, lo[a]);
      atomicMax(box + 3 + a, hi[a]);
    }
  }
}

__device__ __forceinline__ uint32_t spread3(uint32_t x) {  // bit b of x to bit 3 b
  uint32_t r = 0u;
#pragma unroll
  for (int b = 0; b < kCellBits; ++b) r |= ((x >> b) & 1u) << (3 * b);
  return r;
}

// Morton cell of Gaussian i (cell 0 for a non-finite mean, or before any finite mean was seen)
__device__ __forceinline__ uint32_t cell_of(const float* __restrict__ means, int64_t i, const uint32_t* __restrict__ box) {
  uint32_t code = 0u;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float x = means[3 * i + a];
    if (!isfinite(x) || box[a] > box[3 + a]) return 0u;
    const float lo = key2f(box[a]), hi = key2f(box[3 + a]);
    const float t = (hi > lo) ? (x - lo) / (hi - lo) * (float)(1 << kCellBits) : 0.0f;
    const uint32_t c = (uint32_t)fminf(fmaxf(t, 0.0f), (float)((1 << kCellBits) - 1));
    code |= spread3(c) << a;
  }
  return code;
}

__global__ void __launch_bounds__(256) k_cell_count(const float* __restrict__ means, int64_t n,
                                                    const uint32_t* __restrict__ box, uint32_t* __restrict__ count) {
  const int64_t i = blockIdx.x * (int64_t)256 + threadIdx.x;
  if (i < n) atomicAdd(count + cell_of(means, i, box), 1u);
}

__global__ void __launch_bounds__(256) k_cell_place(const float* __restrict__ means, int64_t n,
                                                    const uint32_t* __restrict__ box, const uint32_t* __restrict__ off,
                                                    uint32_t* __restrict__ cur, uint32_t* __restrict__ order) {
  const int64_t i = blockIdx.x * (int64_t)256 + threadIdx.x;
  if (i >= n) return;
  const uint32_t cell = cell_of(means, i, box);
  order[off[cell] + atomicAdd(cur + cell, 1u)] = (uint32_t)i;
}

// The parameters of the Gaussian at each processing position, packed as three float4:
// (mean, opacity), (scale, quaternion w), (quaternion x, y, z, 0).
__global__ void __launch_bounds__(256) k_pack_params(const float* __restrict__ means, const float* __restrict__ scales,
                                                     const float* __restrict__ quats, const float* __restrict__ opac,
                                                     const uint32_t* __restrict__ order, int64_t n,
                                                     float4* __restrict__ packed) {
  const int64_t q = blockIdx.x * (int64_t)256 + threadIdx.x;
  if (q >= n) return;
  const int64_t i = order[q];
  packed[3 * q] = make_float4(means[3 * i], means[3 * i + 1], means[3 * i + 2], opac[i]);
  packed[3 * q + 1] = make_float4(scales[3 * i], scales[3 * i + 1], scales[3 * i + 2], quats[4 * i]);
  packed[3 * q + 2] = make_float4(quats[4 * i + 1], quats[4 * i + 2], quats[4 * i + 3], 0.0f);
}

// ---- exclusive scan of uint32 counts (reduce, scan the block sums, add) ----
constexpr int kScanBlock = 1024;

__global__ void __launch_bounds__(kScanBlock) k_scan_reduce(const uint32_t* __restrict__ in, int64_t m,
                                                            uint32_t* __restrict__ sums) {
  __shared__ uint32_t warp_sums[kScanBlock / 32];
  const int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
  uint32_t v = i < m ? in[i] : 0u;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t s = warp_sums[threadIdx.x];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    if (threadIdx.x == 0) sums[blockIdx.x] = s;
  }
}

// One CTA scans the block sums in place (exclusive) and records the 64-bit total.
__global__ void __launch_bounds__(kScanBlock) k_scan_sums(uint32_t* __restrict__ sums, int nblocks,
                                                          DevStatus* status, uint32_t* __restrict__ total_out) {
  __shared__ unsigned long long warp_tot[kScanBlock / 32];
  __shared__ unsigned long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int base = 0; base < nblocks; base += kScanBlock) {
    const int i = base + threadIdx.x;
    unsigned long long v = i < nblocks ? sums[i] : 0ull;
    unsigned long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
      unsigned long long w = warp_tot[lane];
      unsigned long long z = w;
      for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, z, o);
        if (lane >= o) z += y;
      }
      warp_tot[lane] = z - w;  // exclusive prefix of warp totals
    }
    __syncthreads();
    const unsigned long long excl = carry + warp_tot[wid] + x - v;
    if (i < nblocks) sums[i] = (uint32_t)excl;
    __syncthreads();
    if (threadIdx.x == kScanBlock - 1) carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const unsigned long long tot = carry;
    *total_out = tot > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)tot;
    if (status) {  // the instance counts of a binning pass
      if (tot > status->instances_needed) status->instances_needed = tot;
      status->instances_total += tot;
    }
  }
}

__global__ void __launch_bounds__(kScanBlock) k_scan_apply(uint32_t* __restrict__ data, int64_t m,
                                                           const uint32_t* __restrict__ sums) {
  __shared__ uint32_t warp_tot[kScanBlock / 32];
  const int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t v = i < m ? data[i] : 0u;
  uint32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t w = warp_tot[lane];
    uint32_t z = w;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xFFFFFFFFu, z, o);
      if (lane >= o) z += y;
    }
    warp_tot[lane] = z - w;
  }
  __syncthreads();
  if (i < m) data[i] = sums[blockIdx.x] + warp_tot[wid] + x - v;
}

}  // namespace

void launch_project(const Problem& p, const float* means, const float* scales, const float* quats,
                    const float* opac, int cb, const Workspace& ws, cudaStream_t s) {
  if (p.tiles <= kHistTiles) {
    const size_t smem = sizeof(uint32_t) * (size_t)p.tiles;
    const bool big = p.tiles >= kBigTileGrid;
    auto kern = big ? k_project_hist<32> : k_project_hist<8>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int per_cta = hist_per_cta(big ? 32 : 8);
    const int64_t chunks = (p.n + per_cta - 1) / per_cta;
    // cameras per launch so that the 1-D grid stays below 2^31 CTAs
    const int per = (int)std::min<int64_t>(cb, std::max<int64_t>(1, 0x7FFFFFFF / std::max<int64_t>(chunks, 1)));
    for (int j0 = 0; j0 < cb; j0 += per) {
      const int cbl = std::min(per, cb - j0);
      kern<<<(unsigned)(chunks * cbl), 256, smem, s>>>(ws.packed, ws.order, p.n, ws.cams, j0, cbl, p.width,
                                                       p.height, p.near_z, p.tiles_x, p.tiles, ws.rec, ws.rect,
                                                       ws.tile_off);
      note_launches(1);
    }
    return;
  }
  dim3 grid((unsigned)((p.n + 255) / 256), (unsigned)cb);
  k_project<<<grid, 256, 0, s>>>(ws.packed, ws.order, p.n, ws.cams, p.width, p.height, p.near_z,
                                 p.tiles_x, p.tiles, ws.rec, ws.rect, ws.tile_off);
  note_launches(1);
}

void launch_scan(const Problem& p, int cb, const Workspace& ws, cudaStream_t s) {
  const int64_t m = (int64_t)cb * p.tiles;
  const int nblocks = (int)((m + kScanBlock - 1) / kScanBlock);
  k_scan_reduce<<<nblocks, kScanBlock, 0, s>>>(ws.tile_off, m, ws.scan_tmp);
  k_scan_sums<<<1, kScanBlock, 0, s>>>(ws.scan_tmp, nblocks, ws.status, ws.tile_off + m);
  k_scan_apply<<<nblocks, kScanBlock, 0, s>>>(ws.tile_off, m, ws.scan_tmp);
  note_launches(3);
}

int spatial_cells() { return kCells; }

void launch_spatial_order(const Problem& p, const float* means, const float* scales, const float* quats,
                          const float* opac, const Workspace& ws, cudaStream_t s) {
  if (p.n == 0) return;
  cudaMemsetAsync(ws.cell_box, 0xFF, 3 * sizeof(uint32_t), s);
  cudaMemsetAsync(ws.cell_box + 3, 0, 3 * sizeof(uint32_t), s);
  cudaMemsetAsync(ws.cell_off, 0, sizeof(uint32_t) * (size_t)(kCells + 1), s);
  cudaMemsetAsync(ws.cell_cur, 0, sizeof(uint32_t) * (size_t)kCells, s);
  const unsigned grid = (unsigned)((p.n + 255) / 256);
  k_bounds<<<std::min(grid, 152u * 8u), 256, 0, s>>>(means, p.n, ws.cell_box);
  k_cell_count<<<grid, 256, 0, s>>>(means, p.n, ws.cell_box, ws.cell_off);
  const int nblocks = (kCells + kScanBlock - 1) / kScanBlock;
  k_scan_reduce<<<nblocks, kScanBlock, 0, s>>>(ws.cell_off, kCells, ws.cell_tmp);
  k_scan_sums<<<1, kScanBlock, 0, s>>>(ws.cell_tmp, nblocks, nullptr, ws.cell_off + kCells);
  k_scan_apply<<<nblocks, kScanBlock, 0, s>>>(ws.cell_off, kCells, ws.cell_tmp);
  k_cell_place<<<grid, 256, 0, s>>>(means, p.n, ws.cell_box, ws.cell_off, ws.cell_cur, ws.order);
  k_pack_params<<<grid, 256, 0, s>>>(means, scales, quats, opac, ws.order, p.n, ws.packed);
  note_launches(7);
}

void launch_scatter(const Problem& p, int cb, const Workspace& ws, cudaStream_t s) {
  if (p.tiles <= kHistTiles) {
    const size_t smem = 2 * sizeof(uint32_t) * (size_t)p.tiles;
    const bool big = p.tiles >= kBigTileGrid;
    auto kern = big ? k_scatter_hist<16> : k_scatter_hist<4>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int per_cta = hist_per_cta(big ? 16 : 4);
    dim3 grid((unsigned)((p.n + per_cta - 1) / per_cta), (unsigned)cb);
    kern<<<grid, 256, smem, s>>>(p.n, ws.rect, ws.order, p.tiles_x, p.tiles, ws.tile_off, ws.tile_cur, ws.entries,
                                 p.capacity, ws.status);
    note_launches(1);
    return;
  }
  dim3 grid((unsigned)((p.n + 255) / 256), (unsigned)cb);
  k_scatter<<<grid, 256, 0, s>>>(p.n, ws.rect, ws.order, p.tiles_x, p.tiles, ws.tile_off, ws.tile_cur,
                                 ws.entries, p.capacity, ws.status);
  note_launches(1);
}

}  // namespace icgs
