// solve.cu -- the normal equations and the batched regularised solve (Eq. 12-14, Alg. 1 lines 5-6).
//
//   k_fold          G_i += sum_j V_ij Y_ij Y_ij^T, b_i += sum_j Y_ij S_ij^T, w_i += sum_j V_ij over the
//                   cameras of one pass (L > 0). One 8-lane group per Gaussian: lane r forms wrapped
//                   diagonal r of the symmetric G_i and rows r, r + 8 of b_i. MIXED forms every
//                   product exactly (TwoProduct) and keeps a TwoSum compensation term per entry.
//   k_solve         A_i = G_i + w_i Lambda; Cholesky with the rows in registers of the group (pivots
//                   and columns exchanged by shuffles); forward and back substitution per channel.
//                   MIXED: the FP32 solution is refined in float-float against the compensated sums;
//                   a Gaussian whose smallest pivot ratio d_k / A_kk is below refold_tau is first
//                   re-folded exactly from the resident per-camera sums (single pass), one below
//                   cond_tau (or with a non-positive pivot) is solved in FP64.
//   k_solve_l0      L = 0: c = b / (G + w lambda) with G = V / (4 pi), b = S / sqrt(4 pi).
//   k_adjoint_prep  u_i = A_i^-1 dL/dc_i from the stored factor, reg_i = sum lambda_m u_mk c_mk.
//   k_payload_*     per (camera, Gaussian): C = Y . c (render) or (a = Y . u, beta) (adjoint).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "icgs_device.cuh"
#include "icgs_internal.h"

namespace icgs {

namespace {

constexpr int kGroup = 16;
constexpr int kSolveThreads = 128;  // 8 Gaussians per CTA
constexpr float kY0 = 0.28209479177387814f;

// Shuffles name only the 16 lanes of the caller's group, so a neighbouring group that has
// finished (or never started) in the same warp does not take part.
__device__ __forceinline__ unsigned group_mask() {
  return 0xFFFFu << (threadIdx.x & 16u);
}
template <typename F>
__device__ __forceinline__ F group_sum(F v) {
  const unsigned m = group_mask();
#pragma unroll
  for (int o = kGroup / 2; o > 0; o >>= 1) v += __shfl_xor_sync(m, v, o, kGroup);
  return v;
}

// ------------------------------------------------------------------------------------------
// fold
// ------------------------------------------------------------------------------------------
// One 8-lane group per Gaussian. G is symmetric, so the group forms only its B (B + 1) / 2 unique
// unique entries only, by wrapped diagonals: lane r accumulates diagonal r, the entries
// ((c + r) mod B, c) for c = 0..B-1, and for even B also the entry (r + B/2, r) of the half
// diagonal B/2. Diagonals 0..ceil(B/2)-1 and that half diagonal hold every unordered pair {row, col}
// exactly once. Per camera the column factor Y[c] is a compile-time index (a broadcast float4
// load) and the row factor v Y[(c + r) mod B] is read from a doubled copy of the v Y row at the
// lane's own offset r, so an entry costs one FMA. b rows r, r + 8 belong to lane r. G is written
// out in full (both triangles), row-major like the sums of the single-camera-group layout.
constexpr int kFoldGroup = 8;

__device__ __forceinline__ unsigned fold_group_mask() {
  return 0xFFu << (threadIdx.x & 24u);
}

template <int B, int KC, bool MIXED>
__global__ void __launch_bounds__(kSolveThreads) k_fold(
    const float* __restrict__ means, int64_t n, const DevCam* __restrict__ cams, int cb,
    const float* __restrict__ acc, int K, int RS, int k0, bool first, bool want_gram, float* __restrict__ G,
    float* __restrict__ Glo, float* __restrict__ bvec, float* __restrict__ blo,
    float* __restrict__ wsum, float* __restrict__ wlo) {
  constexpr int GS = kFoldGroup;
  constexpr int ND = (B + 1) / 2;              // full wrapped diagonals (lanes 0..ND-1)
  constexpr bool kHalf = (B % 2) == 0;         // even B: lanes 0..B/2-1 also take one entry of diagonal B/2
  constexpr int NG = B + (kHalf ? 1 : 0);      // Gram slots of a lane
  constexpr int NR = (B + GS - 1) / GS;        // b rows of a lane: r, r + 8
  constexpr int kYStride = (B + 3) / 4 * 4 + 4;
  constexpr int kVStride = 2 * B + 1;          // odd: the four groups' rows fall in distinct banks
  static_assert(ND <= GS, "one diagonal per lane");
  __shared__ __align__(16) float s_Y[kSolveThreads][kYStride];
  __shared__ float s_vY[kSolveThreads][kVStride];
  __shared__ float s_vYl[MIXED ? kSolveThreads : 1][MIXED ? kVStride : 1];  // lo parts of v Y (MIXED)
  const int64_t i = (blockIdx.x * (int64_t)kSolveThreads + threadIdx.x) / GS;
  const int r = threadIdx.x % GS;
  if (i >= n) return;  // whole groups exit together
  const bool diag = r < ND;
  const bool do_gram = k0 == 0 && want_gram;  // G (skipped by refinement, whose Gram is fixed)
  const bool do_w = k0 == 0;
  float* Gi = G + i * B * B;
  float* Gli = MIXED ? Glo + i * B * B : nullptr;
  float g[NG], gl[NG], bb[NR][KC], bl[NR][KC];
  float w = 0.0f, wl = 0.0f;
#pragma unroll
  for (int s = 0; s < NG; ++s) { g[s] = 0.0f; gl[s] = 0.0f; }
#pragma unroll
  for (int m = 0; m < NR; ++m)
#pragma unroll
    for (int k = 0; k < KC; ++k) { bb[m][k] = 0.0f; bl[m][k] = 0.0f; }
  // slot s < B: entry ((s + r) mod B, s); slot B (even B): entry (r + B/2, r)
  auto entry = [&](int s) -> int {
    if (s < B) { const int row = s + r < B ? s + r : s + r - B; return row * B + s; }
    return (r + B / 2) * B + r;
  };
  const bool half_slot = kHalf && r < B / 2;
  if (!first) {
    if (do_gram && diag) {
#pragma unroll
      for (int s = 0; s < NG; ++s) {
        if (s == B && !half_slot) continue;
        g[s] = Gi[entry(s)];
        if (MIXED) gl[s] = Gli[entry(s)];
      }
    }
    if (do_w) {
      w = wsum[i];
      if (MIXED) wl = wlo[i];
    }
#pragma unroll
    for (int m = 0; m < NR; ++m) {
      const int row = r + GS * m;
      if (row < B) {
#pragma unroll
        for (int k = 0; k < KC; ++k)
          if (k0 + k < K) {
            bb[m][k] = bvec[(i * B + row) * K + k0 + k];
            if (MIXED) bl[m][k] = blo[(i * B + row) * K + k0 + k];
          }
      }
    }
  }
  const float mu[3] = {means[3 * i], means[3 * i + 1], means[3 * i + 2]};
  const int64_t stride = n * (int64_t)RS;
  // MIXED: every product is exact in float-float (v Y_r split by an FMA, then each entry's product
  // split again) and every addition a TwoSum into the running (hi, lo) pair, so G, b and w are the
  // sums of the float32 basis to about 2^-44 relative -- the same basis the adjoint's payload uses
  const unsigned gm = fold_group_mask();
  const int gbase = threadIdx.x & ~(GS - 1);
  // 8 cameras at a time: lane q loads camera jb + q's row (V, S), evaluates its basis Y into s_Y
  // and v Y (twice) into s_vY; the group shares V, S by shuffles and reads the rows back
  for (int jb = 0; jb < cb; jb += GS) {
    float lv = 0.0f, ls[KC];
#pragma unroll
    for (int k = 0; k < KC; ++k) ls[k] = 0.0f;
    if (jb + r < cb) {
      const float* a = acc + (int64_t)(jb + r) * stride + i * RS;
      lv = a[0];
#pragma unroll
      for (int k = 0; k < KC; ++k)
        if (k0 + k < K) ls[k] = a[1 + k0 + k];
    }
    if (lv > 0.0f) {
      const float3 d = view_dir(mu, cams[jb + r]);
      float Yl[kYStride];
      sh_basis<B>(d.x, d.y, d.z, Yl);
#pragma unroll
      for (int c4 = 0; c4 < (B + 3) / 4; ++c4)
        reinterpret_cast<float4*>(s_Y[threadIdx.x])[c4] =
            make_float4(Yl[4 * c4], 4 * c4 + 1 < B ? Yl[4 * c4 + 1] : 0.0f, 4 * c4 + 2 < B ? Yl[4 * c4 + 2] : 0.0f,
                        4 * c4 + 3 < B ? Yl[4 * c4 + 3] : 0.0f);
      if (do_gram) {
#pragma unroll
        for (int c = 0; c < B; ++c) {
          const float vy = lv * Yl[c];
          s_vY[threadIdx.x][c] = vy;
          s_vY[threadIdx.x][c + B] = vy;
          if constexpr (MIXED) {
            const float vyl = fmaf(lv, Yl[c], -vy);
            s_vYl[threadIdx.x][c] = vyl;
            s_vYl[threadIdx.x][c + B] = vyl;
          }
        }
      }
    }
    __syncwarp(gm);
    const int nj = min(GS, cb - jb);
    for (int q = 0; q < nj; ++q) {
      const int j = jb + q;
      const float v = __shfl_sync(gm, lv, q, GS);
      float sv[KC];
#pragma unroll
      for (int k = 0; k < KC; ++k) sv[k] = __shfl_sync(gm, ls[k], q, GS);
      if (v > 0.0f) {
        const float* Yq = s_Y[gbase + q];
        if (do_gram && diag) {
          float Y[(B + 3) / 4 * 4];
#pragma unroll
          for (int c4 = 0; c4 < (B + 3) / 4; ++c4) {
            const float4 y4 = reinterpret_cast<const float4*>(Yq)[c4];
            Y[4 * c4] = y4.x; Y[4 * c4 + 1] = y4.y; Y[4 * c4 + 2] = y4.z; Y[4 * c4 + 3] = y4.w;
          }
          const float* vq = s_vY[gbase + q] + r;  // vq[c] = v Y[(c + r) mod B]
          const float* vql = s_vYl[MIXED ? gbase + q : 0] + (MIXED ? r : 0);
#pragma unroll
          for (int s = 0; s < B; ++s) {
            if constexpr (MIXED) {
              const float p = vq[s] * Y[s];
              const float e = fmaf(vq[s], Y[s], -p) + vql[s] * Y[s];
              two_sum_acc(g[s], gl[s], p);
              gl[s] += e;
            } else {
              g[s] = fmaf(vq[s], Y[s], g[s]);
            }
          }
          if constexpr (kHalf) {
            if (half_slot) {  // entry (r + B/2, r): v Y[r + B/2] Y[r]
              if constexpr (MIXED) {
                const float p = vq[B / 2] * Yq[r];
                const float e = fmaf(vq[B / 2], Yq[r], -p) + vql[B / 2] * Yq[r];
                two_sum_acc(g[B], gl[B], p);
                gl[B] += e;
              } else {
                g[B] = fmaf(vq[B / 2], Yq[r], g[B]);
              }
            }
          }
        }
        if (do_w) {
          if constexpr (MIXED) two_sum_acc(w, wl, v);
          else w += v;
        }
#pragma unroll
        for (int m = 0; m < NR; ++m) {
          const int row = r + GS * m;
          const float Yr = row < B ? Yq[row] : 0.0f;
#pragma unroll
          for (int k = 0; k < KC; ++k)
            if (k0 + k < K) {
              if constexpr (MIXED) {
                const float p = Yr * sv[k];
                two_sum_acc(bb[m][k], bl[m][k], p);
                bl[m][k] += fmaf(Yr, sv[k], -p);
              } else {
                bb[m][k] = fmaf(Yr, sv[k], bb[m][k]);
              }
            }
        }
      }
    }
    __syncwarp(gm);
  }
  if (do_gram && diag) {
#pragma unroll
    for (int s = 0; s < NG; ++s) {
      if (s == B && !half_slot) continue;
      const int e = entry(s);
      const int row = e / B, col = e - row * B;
      Gi[e] = g[s];
      if (MIXED) Gli[e] = gl[s];
      if (row != col) {  // the mirrored entry
        Gi[col * B + row] = g[s];
        if (MIXED) Gli[col * B + row] = gl[s];
      }
    }
  }
  if (do_w && r == 0) {
    wsum[i] = w;
    if (MIXED) wlo[i] = wl;
  }
#pragma unroll
  for (int m = 0; m < NR; ++m) {
    const int row = r + GS * m;
    if (row < B) {
#pragma unroll
      for (int k = 0; k < KC; ++k)
        if (k0 + k < K) {
          bvec[(i * B + row) * K + k0 + k] = bb[m][k];
          if (MIXED) blo[(i * B + row) * K + k0 + k] = bl[m][k];
        }
    }
  }
}

// ------------------------------------------------------------------------------------------
// Cholesky in a 16-lane group: lane r holds row r of A (a[0..B-1]); on return a[0..r] is row r of
// the lower factor L. Returns the smallest pivot ratio d_k / A_kk (<= 0 if a pivot was not
// positive; such pivots are replaced by 1 so the arithmetic stays finite).
// ------------------------------------------------------------------------------------------
template <int B, typename F>
__device__ __forceinline__ F group_cholesky(F (&a)[B], int r) {
  F diag0 = 0;
#pragma unroll
  for (int c = 0; c < B; ++c)
    if (c == r) diag0 = a[c];
  F minratio = 1;
  const unsigned m = group_mask();
#pragma unroll
  for (int k = 0; k < B; ++k) {
    F d = __shfl_sync(m, a[k], k, kGroup);
    const F d0 = __shfl_sync(m, diag0, k, kGroup);
    const F ratio = d / d0;
    if (!(ratio >= minratio)) minratio = ratio;  // also catches NaN
    if (!(d > 0)) d = 1;
    const F lkk = sqrt(d);
    const F inv = F(1) / lkk;
    const F lrk = r > k ? a[k] * inv : (r == k ? lkk : F(0));
    a[k] = lrk;
#pragma unroll
    for (int c = k + 1; c < B; ++c) {
      const F lck = __shfl_sync(m, lrk, c, kGroup);
      if (r >= c) a[c] -= lrk * lck;
    }
  }
  return minratio;
}

// Solve L L^T x = rhs for one right-hand side; lane r holds rhs_r in x and L's row r in a.
template <int B, typename F>
__device__ __forceinline__ void group_chol_solve(const F (&a)[B], int r, F& x) {
  F lrr = 1;
#pragma unroll
  for (int c = 0; c < B; ++c)
    if (c == r) lrr = a[c];
  const F inv_rr = F(1) / lrr;
  const unsigned m = group_mask();
  // forward: L y = rhs
#pragma unroll
  for (int k = 0; k < B; ++k) {
    if (r == k) x *= inv_rr;
    const F yk = __shfl_sync(m, x, k, kGroup);
    if (r > k && r < B) x -= a[k] * yk;
  }
  // backward: L^T x = y; at step k subtract sum_{m>k} L_mk x_m, held by lanes m > k
#pragma unroll
  for (int k = B - 1; k >= 0; --k) {
    const F part = (r > k && r < B) ? a[k] * x : F(0);
    const F s = group_sum(part);
    if (r == k) x = (x - s) * inv_rr;
  }
}

// Solves L L^T x_q = rhs_q for NR right-hand sides at once: lane r holds rhs_q,r in x[q] and row r
// of L in a; s_L holds the same rows (s_L[k (B + 1) + c] = L_kc). Both substitutions go by
// columns, one broadcast shuffle per step and right-hand side: the forward one reads L_rk from a,
// the backward one the column entry L_kr from s_L.
template <int B, int NR>
__device__ __forceinline__ void group_chol_solve_rows(const float (&a)[B], int r, float (&x)[NR],
                                                      const float* s_L) {
  float lrr = 1.0f;
#pragma unroll
  for (int c = 0; c < B; ++c)
    if (c == r) lrr = a[c];
  const float inv_rr = 1.0f / lrr;
  const unsigned m = group_mask();
#pragma unroll
  for (int k = 0; k < B; ++k) {  // L y = rhs
    if (r == k) {
#pragma unroll
      for (int q = 0; q < NR; ++q) x[q] *= inv_rr;
    }
    float yk[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) yk[q] = __shfl_sync(m, x[q], k, kGroup);
    if (r > k && r < B) {
#pragma unroll
      for (int q = 0; q < NR; ++q) x[q] -= a[k] * yk[q];
    }
  }
#pragma unroll
  for (int k = B - 1; k >= 0; --k) {  // L^T x = y: x_k final, then x_j -= L_kj x_k for j < k
    if (r == k) {
#pragma unroll
      for (int q = 0; q < NR; ++q) x[q] *= inv_rr;
    }
    float xk[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) xk[q] = __shfl_sync(m, x[q], k, kGroup);
    if (r < k) {
      const float l = s_L[k * (B + 1) + r];
#pragma unroll
      for (int q = 0; q < NR; ++q) x[q] -= l * xk[q];
    }
  }
}

constexpr int kRefineSteps = 2;
constexpr int kRefineStepsRefold = 4;  // re-folded Gaussians: pivot ratio below refold_tau
// A re-folded Gaussian's sums are exact to float-float, so the refined FP32 solve converges down to
// much smaller pivot ratios; FP64 takes over below cond_tau * kRefoldFp64Scale.
constexpr float kRefoldFp64Scale = 1e-2f;

// Residual b - A x of row r with A = G_hi + G_lo + (w_hi + w_lo) Lambda and b = b_hi + b_lo,
// evaluated in float-float: every product is split exactly with an FMA (TwoProduct) and summed
// with TwoSum, so the residual is accurate even though A x and b agree to FP32 rounding.
template <int B>
__device__ __forceinline__ float refine_residual(const float (&ghi)[B], const float (&glo)[B], float wl_r,
                                                 float wl_lo, float bh, float bl, float x, int r) {
  const unsigned m = group_mask();
  float s = 0.0f, comp = 0.0f;
#pragma unroll
  for (int c = 0; c < B; ++c) {
    const float xc = __shfl_sync(m, x, c, kGroup);
    const float p = ghi[c] * xc;
    const float e = fmaf(ghi[c], xc, -p);
    two_sum_acc(s, comp, p);
    comp += e + glo[c] * xc;
  }
  const float p = wl_r * x;
  two_sum_acc(s, comp, p);
  comp += fmaf(wl_r, x, -p) + wl_lo * x;
  return r < B ? (bh - s) + (bl - comp) : 0.0f;
}

// Exact float-float fold of one Gaussian's row r from the per-camera sums still resident in acc:
// every product split with an FMA (TwoProduct) and every addition with TwoSum, so (hi + lo) holds
// sum_j V_j Y_j Y_j^T (and sum_j Y_j S_j for channels k0..k0+3, and w) to about 2^-44 relative.
// The basis stays float32: a consistent perturbation of the directions barely moves the solution,
// whereas the independent rounding of each product in the fast fold is amplified by the condition
// number. Lane q evaluates camera jb + q's basis into s_Y; the group then walks the 16 cameras.
// Group-collective (all 16 lanes).
template <int B>
__device__ __forceinline__ void exact_fold(const float* __restrict__ acc, int64_t cam_stride, int64_t i, int RS,
                                           int n_cams, const DevCam* __restrict__ cams, const float* mu, int r,
                                           bool gram, int k0, int K, float (&gh)[B], float (&gl)[B], float& wh,
                                           float& wl, float (&bh)[4], float (&bl)[4], float (*s_Y)[B + 1]) {
  const unsigned gm = group_mask();
  const int gbase = threadIdx.x & ~(kGroup - 1);
  const bool row = r < B;
  for (int jb = 0; jb < n_cams; jb += kGroup) {
    const int jq = jb + r;
    float vq = 0.0f, sq[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (jq < n_cams) {
      const float* a = acc + jq * cam_stride + i * RS;
      vq = a[0];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (k0 + q < K) sq[q] = a[1 + k0 + q];
    }
    if (vq > 0.0f) {
      const float3 d = view_dir(mu, cams[jq]);
      sh_basis<B>(d.x, d.y, d.z, s_Y[threadIdx.x]);
    }
    __syncwarp(gm);
    const int nj = min(kGroup, n_cams - jb);
    for (int q = 0; q < nj; ++q) {
      const float v = __shfl_sync(gm, vq, q, kGroup);
      float sv[4];
#pragma unroll
      for (int qq = 0; qq < 4; ++qq) sv[qq] = __shfl_sync(gm, sq[qq], q, kGroup);
      if (!(v > 0.0f)) continue;  // uniform in the group
      const float* yq = s_Y[gbase + q];
      const float Yr = row ? yq[r] : 0.0f;
      if (gram) {
        const float vh = v * Yr, vl = fmaf(v, Yr, -vh);
#pragma unroll
        for (int c = 0; c < B; ++c) {
          const float y = yq[c];
          const float p = vh * y;
          const float e = fmaf(vh, y, -p);
          two_sum_acc(gh[c], gl[c], p);
          gl[c] += fmaf(vl, y, e);
        }
        two_sum_acc(wh, wl, v);
      }
#pragma unroll
      for (int qq = 0; qq < 4; ++qq)
        if (k0 + qq < K) {
          const float p = Yr * sv[qq];
          const float e = fmaf(Yr, sv[qq], -p);
          two_sum_acc(bh[qq], bl[qq], p);
          bl[qq] += e;
        }
    }
    __syncwarp(gm);
  }
}

// MIXED: every Gaussian is factorised in FP32 from the fold's G_hi. When all cameras were
// accumulated in one pass (n_acc_cams > 0) and the smallest pivot ratio is below refold_tau, the
// row is re-folded exactly from the resident per-camera sums (exact_fold) and refactorised; the
// FP32 solution is then refined in float-float against (G_hi + G_lo, b_hi + b_lo) for
// kRefineStepsRefold steps. Below cond_tau (cond_tau * kRefoldFp64Scale after a re-fold), or with
// a non-positive pivot, the Gaussian is solved in FP64.
// NR: right-hand sides solved together (3 for RGB, else 4; the last group is padded with zeros)
template <int B, bool MIXED, int NR>
__global__ void __launch_bounds__(kSolveThreads, 5) k_solve(
    int64_t n, int K, const float* __restrict__ G, const float* __restrict__ Glo,
    const float* __restrict__ bvec, const float* __restrict__ blo, const float* __restrict__ wsum,
    const float* __restrict__ wlo, const float* __restrict__ lam, float cond_tau, float refold_tau,
    float* __restrict__ coeffs, uint8_t* __restrict__ status_out, float* __restrict__ chol,
    DevStatus* status, const float* __restrict__ acc, int RS, int n_acc_cams,
    const DevCam* __restrict__ cams, const float* __restrict__ means) {
  __shared__ float s_Y[MIXED ? kSolveThreads : 1][B + 1];  // per lane: basis of its camera (re-fold)
  __shared__ float s_L[(kSolveThreads / kGroup) * B * (B + 1)];  // per group: the rows of L
  const int64_t i = (blockIdx.x * (int64_t)kSolveThreads + threadIdx.x) / kGroup;
  const int r = threadIdx.x % kGroup;
  if (i >= n) return;
  const bool row = r < B;
  float w = wsum[i];
  const float lam_r = row ? lam[r] : 0.0f;
  constexpr int P = B * (B + 1) / 2;
  float* rec = chol ? chol + i * solve_record_floats(B) : nullptr;
  if (!(w > 0.0f)) {
    if (row) {
      for (int k = 0; k < K; ++k) coeffs[(i * B + r) * K + k] = 0.0f;
      if (rec)
        for (int c = 0; c <= r; ++c) {  // no register array
          const int e = r * (r + 1) / 2 + c;
          rec[e] = 0.0f;
          rec[P + e] = 0.0f;
          rec[2 * P + e] = 0.0f;
        }
    }
    if (r == 0 && status_out) status_out[i] = kGaussUnseen;
    return;
  }
  float a[B];
#pragma unroll
  for (int c = 0; c < B; ++c) {
    a[c] = row ? G[(i * B + r) * B + c] : 0.0f;
    if (c == r) a[c] += w * lam_r;
  }
  if (!MIXED && rec && row) {  // PLAIN: A in FP32 (no compensation term)
#pragma unroll
    for (int c = 0; c < B; ++c)
      if (c <= r) {
        rec[P + r * (r + 1) / 2 + c] = a[c];
        rec[2 * P + r * (r + 1) / 2 + c] = 0.0f;
      }
  }
  float minratio = group_cholesky<B, float>(a, r);
  // MIXED: rows of G_hi, G_lo (and w_lo) for the residuals of the refinement
  float ghi[B], glo[B];
  float wl = 0.0f;
  bool refold = false;
  float rb_h[4] = {0.0f, 0.0f, 0.0f, 0.0f}, rb_l[4] = {0.0f, 0.0f, 0.0f, 0.0f};  // re-fold: b, channels 0-3
  // the mean is read only by the exact re-fold, which needs the resident per-camera sums (callers
  // without them pass no means)
  const bool have_sums = n_acc_cams > 0 && means != nullptr;
  float mu[3] = {0.0f, 0.0f, 0.0f};
  if (have_sums) {
    mu[0] = means[3 * i];
    mu[1] = means[3 * i + 1];
    mu[2] = means[3 * i + 2];
  }
  const int64_t cam_stride = n * (int64_t)RS;
  if constexpr (MIXED) {
    refold = have_sums && !(minratio >= refold_tau);
    if (refold) {
#pragma unroll
      for (int c = 0; c < B; ++c) { ghi[c] = 0.0f; glo[c] = 0.0f; }
      w = 0.0f;
      exact_fold<B>(acc, cam_stride, i, RS, n_acc_cams, cams, mu, r, true, 0, K, ghi, glo, w, wl, rb_h, rb_l, s_Y);
#pragma unroll
      for (int c = 0; c < B; ++c) {
        a[c] = row ? ghi[c] : 0.0f;
        if (c == r) a[c] += w * lam_r;
      }
      minratio = group_cholesky<B, float>(a, r);
      if (r == 0) atomicAdd(&status->refold_count, 1u);
    } else {
      wl = wlo[i];
#pragma unroll
      for (int c = 0; c < B; ++c) {
        ghi[c] = row ? G[(i * B + r) * B + c] : 0.0f;
        glo[c] = row ? Glo[(i * B + r) * B + c] : 0.0f;
      }
    }
  }
  if (MIXED && rec && row) {  // A = (G_hi + G_lo) + (w_hi + w_lo) Lambda in float-float
#pragma unroll
    for (int c = 0; c < B; ++c)
      if (c <= r) {
        float hi = ghi[c], lo = glo[c];
        if (c == r) {
          const float p = w * lam_r;
          two_sum_acc(hi, lo, p);
          lo += fmaf(w, lam_r, -p) + wl * lam_r;
        }
        rec[P + r * (r + 1) / 2 + c] = hi;
        rec[2 * P + r * (r + 1) / 2 + c] = lo;
      }
  }
  const bool fp64 = MIXED && !(minratio >= (refold ? cond_tau * kRefoldFp64Scale : cond_tau));
  if (!fp64) {
    const float wl_r = w * lam_r;
    const float wl_lo = MIXED ? wl * lam_r : 0.0f;
    const int steps = refold ? kRefineStepsRefold : kRefineSteps;
    float* s_Lg = s_L + (threadIdx.x / kGroup) * (B * (B + 1));
    if (row) {
#pragma unroll
      for (int c = 0; c < B; ++c)
        if (c <= r) s_Lg[r * (B + 1) + c] = a[c];
    }
    __syncwarp(group_mask());
    for (int k0 = 0; k0 < K; k0 += NR) {
      float bh[4] = {0.0f, 0.0f, 0.0f, 0.0f}, bl[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      if (refold && k0 == 0) {
#pragma unroll
        for (int q = 0; q < NR; ++q) { bh[q] = rb_h[q]; bl[q] = rb_l[q]; }
      } else if (refold) {
        float gdummy[B], gldummy[B], wdummy = 0.0f, wldummy = 0.0f;
        exact_fold<B>(acc, cam_stride, i, RS, n_acc_cams, cams, mu, r, false, k0, K, gdummy, gldummy, wdummy,
                      wldummy, bh, bl, s_Y);
      } else {
#pragma unroll
        for (int q = 0; q < NR; ++q)
          if (k0 + q < K && row) {
            bh[q] = bvec[(i * B + r) * K + k0 + q];
            if (MIXED) bl[q] = blo[(i * B + r) * K + k0 + q];
          }
      }
      // NR channels at once (padding channels carry zeros)
      float x[NR];
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        if (!(row && k0 + q < K)) { bh[q] = 0.0f; bl[q] = 0.0f; }
        x[q] = bh[q];
      }
      group_chol_solve_rows<B, NR>(a, r, x, s_Lg);
      if constexpr (MIXED) {
#pragma unroll 1
        for (int it = 0; it < steps; ++it) {
          float res[NR];
#pragma unroll
          for (int q = 0; q < NR; ++q) res[q] = refine_residual<B>(ghi, glo, wl_r, wl_lo, bh[q], bl[q], x[q], r);
          group_chol_solve_rows<B, NR>(a, r, res, s_Lg);
#pragma unroll
          for (int q = 0; q < NR; ++q) x[q] += res[q];
        }
      }
#pragma unroll
      for (int q = 0; q < NR; ++q)
        if (row && k0 + q < K) coeffs[(i * B + r) * K + k0 + q] = x[q];
    }
    if (chol && row) {
#pragma unroll
      for (int c = 0; c < B; ++c)
        if (c <= r) chol[i * solve_record_floats(B) + r * (r + 1) / 2 + c] = a[c];
    }
    if (r == 0 && status_out) status_out[i] = kGaussOk;
    return;
  }
  // FP64 from (G_hi + G_lo, b_hi + b_lo): the exact re-fold when it ran, else the fold's
  // compensated sums
  double ad[B];
  const double wd = (double)w + (double)wl;
#pragma unroll
  for (int c = 0; c < B; ++c) {
    ad[c] = row ? (double)ghi[c] + (double)glo[c] : 0.0;
    if (c == r) ad[c] += wd * (double)lam_r;
  }
  group_cholesky<B, double>(ad, r);
  for (int k0 = 0; k0 < K; k0 += NR) {
    float bh[4] = {0.0f, 0.0f, 0.0f, 0.0f}, bl[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (refold && k0 == 0) {
#pragma unroll
      for (int q = 0; q < NR; ++q) { bh[q] = rb_h[q]; bl[q] = rb_l[q]; }
    } else if (refold) {
      float gdummy[B], gldummy[B], wdummy = 0.0f, wldummy = 0.0f;
      exact_fold<B>(acc, cam_stride, i, RS, n_acc_cams, cams, mu, r, false, k0, K, gdummy, gldummy, wdummy,
                    wldummy, bh, bl, s_Y);
    } else {
#pragma unroll
      for (int q = 0; q < NR; ++q)
        if (k0 + q < K && row) {
          bh[q] = bvec[(i * B + r) * K + k0 + q];
          bl[q] = blo[(i * B + r) * K + k0 + q];
        }
    }
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      if (k0 + q >= K) break;
      double x = row ? (double)bh[q] + (double)bl[q] : 0.0;
      group_chol_solve<B, double>(ad, r, x);
      if (row) coeffs[(i * B + r) * K + k0 + q] = (float)x;
    }
  }
  if (chol && row) {
#pragma unroll
    for (int c = 0; c < B; ++c)
      if (c <= r) chol[i * solve_record_floats(B) + r * (r + 1) / 2 + c] = (float)ad[c];
  }
  if (r == 0) {
    if (status_out) status_out[i] = kGaussFp64;
    atomicAdd(&status->fp64_count, 1u);
  }
}

// L = 0: acc[i] = (V, S_0..S_{K-1}) summed over every camera. keep (nullable) receives, per
// Gaussian and channel, whether the colour c Y_0 reaches tau (the segmentation threshold; 0 for
// Gaussians no camera sees).
__global__ void k_solve_l0(int64_t n, int K, int RS, const float* __restrict__ acc, float lam0,
                           float* __restrict__ coeffs, uint8_t* __restrict__ status_out,
                           float* __restrict__ chol, float tau, uint8_t* __restrict__ keep) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n * (int64_t)K) return;
  const int64_t i = idx / K;
  const int k = (int)(idx - i * K);
  const float V = acc[i * RS];
  float c = 0.0f;
  if (V > 0.0f) {
    // (Y0^2 V + V lambda) c = Y0 S
    const float y = kY0 * kY0 + lam0;
    const float A = V * y;
    c = kY0 * acc[i * RS + 1 + k] / A;
    if (k == 0 && chol) {  // record: sqrt(A), then A = V y exactly as hi + lo
      chol[3 * i] = sqrtf(A);
      chol[3 * i + 1] = A;
      chol[3 * i + 2] = fmaf(V, y, -A);
    }
  } else if (k == 0 && chol) {
    chol[3 * i] = 0.0f;
    chol[3 * i + 1] = 0.0f;
    chol[3 * i + 2] = 0.0f;
  }
  coeffs[i * K + k] = c;
  if (keep) keep[i * K + k] = (V > 0.0f && c * kY0 >= tau) ? 1 : 0;
  if (k == 0 && status_out) status_out[i] = V > 0.0f ? kGaussOk : kGaussUnseen;
}

// ------------------------------------------------------------------------------------------
// adjoint preparation: u = A^-1 g from the factor, reg = sum_mk lambda_m u_mk c_mk
// ------------------------------------------------------------------------------------------
// The FP32 solve with the stored factor is refined twice in float-float against A = A_hi + A_lo of
// the record (the same sums the forward solve used), so u carries the forward's accuracy instead of
// the factor's rounding amplified by the condition number.
constexpr int kAdjointRefineSteps = 2;

// Residual g - (A_hi + A_lo)(x_hi + x_lo) of row r in float-float (TwoProduct / TwoSum), for an
// iterate that is itself float-float.
template <int B>
__device__ __forceinline__ float residual_ff(const float (&ahi)[B], const float (&alo)[B], float g, float x_hi,
                                            float x_lo, int r) {
  const unsigned m = group_mask();
  float s = 0.0f, comp = 0.0f;
#pragma unroll
  for (int c = 0; c < B; ++c) {
    const float xh = __shfl_sync(m, x_hi, c, kGroup);
    const float xl = __shfl_sync(m, x_lo, c, kGroup);
    const float p = ahi[c] * xh;
    const float e = fmaf(ahi[c], xh, -p);
    two_sum_acc(s, comp, p);
    comp += e + alo[c] * xh + ahi[c] * xl;
  }
  return r < B ? (g - s) - comp : 0.0f;
}

template <int B>
__global__ void __launch_bounds__(kSolveThreads) k_adjoint_prep(
    int64_t n, int K, const float* __restrict__ chol, const float* __restrict__ grad_c,
    const float* __restrict__ coeffs, const float* __restrict__ lam, float* __restrict__ u,
    float* __restrict__ u_lo, float* __restrict__ reg) {
  constexpr int P = B * (B + 1) / 2;
  const int64_t i = (blockIdx.x * (int64_t)kSolveThreads + threadIdx.x) / kGroup;
  const int r = threadIdx.x % kGroup;
  if (i >= n) return;
  const bool row = r < B;
  const float* rec = chol + i * solve_record_floats(B);
  float a[B], ahi[B], alo[B];
#pragma unroll
  for (int c = 0; c < B; ++c) {
    a[c] = (row && c <= r) ? rec[r * (r + 1) / 2 + c] : 0.0f;
    const int hi = r > c ? r : c, lo = r > c ? c : r;  // row r of the symmetric A from its lower triangle
    ahi[c] = row ? rec[P + hi * (hi + 1) / 2 + lo] : 0.0f;
    alo[c] = row ? rec[2 * P + hi * (hi + 1) / 2 + lo] : 0.0f;
  }
  const float l00 = __shfl_sync(group_mask(), a[0], 0, kGroup);
  const bool seen = l00 > 0.0f;
  double rg = 0.0;  // sum lambda_m u_mk c_mk: large u terms can cancel, so in double (per Gaussian only)
  for (int k = 0; k < K; ++k) {
    const float g = row ? grad_c[(i * B + r) * K + k] : 0.0f;
    float xh = 0.0f, xl = 0.0f;
    if (seen) {
      xh = g;
      group_chol_solve<B, float>(a, r, xh);
#pragma unroll 1
      for (int it = 0; it < kAdjointRefineSteps; ++it) {
        float d = residual_ff<B>(ahi, alo, g, xh, xl, r);
        group_chol_solve<B, float>(a, r, d);
        float e = 0.0f;
        two_sum_acc(xh, e, d);  // (xh, e) = xh + d exactly
        xl += e;
        const float t = xh + xl;  // renormalise the pair
        xl = xl - (t - xh);
        xh = t;
      }
    }
    if (row) {
      u[(i * B + r) * K + k] = xh;
      u_lo[(i * B + r) * K + k] = xl;
      rg += (double)lam[r] * (double)coeffs[(i * B + r) * K + k] * ((double)xh + (double)xl);
    }
  }
  const unsigned m = group_mask();
#pragma unroll
  for (int o = kGroup / 2; o > 0; o >>= 1) rg += __shfl_xor_sync(m, rg, o, kGroup);
  if (r == 0) reg[i] = (float)rg;
}

__global__ void k_adjoint_prep_l0(int64_t n, int K, const float* __restrict__ chol,
                                  const float* __restrict__ grad_c, const float* __restrict__ coeffs,
                                  float lam0, float* __restrict__ u, float* __restrict__ u_lo,
                                  float* __restrict__ reg) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float A = chol[3 * i + 1], A_lo = chol[3 * i + 2];  // record: sqrt(A), A_hi, A_lo
  float rg = 0.0f;
  for (int k = 0; k < K; ++k) {
    const float g = grad_c[i * K + k];
    float x = 0.0f, xl = 0.0f;
    if (A > 0.0f) {
      x = g / A;
      xl = (fmaf(-A, x, g) - A_lo * x) / A;  // one float-float correction, kept as the lo part
    }
    u[i * K + k] = x;
    u_lo[i * K + k] = xl;
    rg = fmaf(lam0 * (x + xl), coeffs[i * K + k], rg);
  }
  reg[i] = rg;
}

// ------------------------------------------------------------------------------------------
// refinement update (Alg. 1 line 10): c <- c + A^-1 (b - w Lambda c), A from its stored factor
// ------------------------------------------------------------------------------------------
template <int B, bool MIXED>
__global__ void __launch_bounds__(kSolveThreads) k_refine_update(
    int64_t n, int K, const float* __restrict__ chol, const float* __restrict__ bvec,
    const float* __restrict__ blo, const float* __restrict__ wsum, const float* __restrict__ wlo,
    const float* __restrict__ lam, float* __restrict__ coeffs) {
  const int64_t i = (blockIdx.x * (int64_t)kSolveThreads + threadIdx.x) / kGroup;
  const int r = threadIdx.x % kGroup;
  if (i >= n) return;
  const bool row = r < B;
  float a[B];
#pragma unroll
  for (int c = 0; c < B; ++c) a[c] = (row && c <= r) ? chol[i * solve_record_floats(B) + r * (r + 1) / 2 + c] : 0.0f;
  const float l00 = __shfl_sync(group_mask(), a[0], 0, kGroup);
  if (!(l00 > 0.0f)) return;  // unseen: the coefficients stay 0 (whole group)
  const float w = wsum[i] + (MIXED ? wlo[i] : 0.0f);
  const float wl = row ? w * lam[r] : 0.0f;
  for (int k = 0; k < K; ++k) {
    float x = 0.0f;
    if (row) {
      const float b = bvec[(i * B + r) * K + k] + (MIXED ? blo[(i * B + r) * K + k] : 0.0f);
      x = b - wl * coeffs[(i * B + r) * K + k];
    }
    group_chol_solve<B, float>(a, r, x);
    if (row) coeffs[(i * B + r) * K + k] += x;
  }
}

// L = 0: b = S / sqrt(4 pi) and A = w (1/(4 pi) + lambda) from acc, summed over every camera.
__global__ void k_refine_update_l0(int64_t n, int K, int RS, const float* __restrict__ acc, float lam0,
                                   float* __restrict__ coeffs) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n * (int64_t)K) return;
  const int64_t i = idx / K;
  const int k = (int)(idx - i * K);
  const float V = acc[i * RS];
  if (!(V > 0.0f)) return;
  const float A = V * (kY0 * kY0 + lam0);
  const float c = coeffs[i * K + k];
  coeffs[i * K + k] = c + (kY0 * acc[i * RS + 1 + k] - V * lam0 * c) / A;
}

// ------------------------------------------------------------------------------------------
// per (camera, Gaussian) payloads
// ------------------------------------------------------------------------------------------
// Payload kernels. A CTA takes G consecutive Gaussians (G = 64 when their coefficient rows fit):
// the rows (contiguous in global memory) are staged in shared memory with coalesced loads, at an
// odd row stride RW so that the threads' row reads fall in distinct banks. The 256 threads are G
// Gaussians x (256 / G) camera lanes; a lane loops over its cameras, and the threads of a warp
// write consecutive payload rows of one camera.
constexpr int kPayThreads = 256;

__device__ __forceinline__ void stage_rows(const float* __restrict__ src, int64_t i0, int gcount, int BK, int RW,
                                           float* dst) {
  const float* base = src + i0 * BK;
  for (int e = threadIdx.x; e < gcount * BK; e += kPayThreads) {
    const int g = e / BK;
    dst[g * RW + (e - g * BK)] = base[e];
  }
}

template <int B>
__global__ void __launch_bounds__(kPayThreads) k_payload_render(int64_t n, int K, int G, const float* __restrict__ means,
                                                                const DevCam* __restrict__ cams, int cb,
                                                                const float* __restrict__ coeffs,
                                                                float* __restrict__ payload) {
  extern __shared__ float s_rows[];
  const int BK = B * K, RW = BK | 1;
  const int64_t i0 = blockIdx.x * (int64_t)G;
  const int gcount = (int)min((int64_t)G, n - i0);
  stage_rows(coeffs, i0, gcount, BK, RW, s_rows);
  __syncthreads();
  const int g = threadIdx.x % G, lanes = kPayThreads / G, cl = threadIdx.x / G;
  if (g >= gcount) return;
  const int64_t i = i0 + g;
  const float mu[3] = {means[3 * i], means[3 * i + 1], means[3 * i + 2]};
  const float* ci = s_rows + g * RW;
  for (int j = cl; j < cb; j += lanes) {
    const float3 d = view_dir(mu, cams[j]);
    float Y[B];
    sh_basis<B>(d.x, d.y, d.z, Y);
    float* out = payload + ((int64_t)j * n + i) * K;
    for (int k = 0; k < K; ++k) {
      float acc = 0.0f;
#pragma unroll
      for (int m = 0; m < B; ++m) acc = fmaf(Y[m], ci[m * K + k], acc);
      out[k] = acc;
    }
  }
}

// a = Y . u and Y . c per (camera, Gaussian) in float-float: for an ill-conditioned A, u = A^-1 g
// is large along directions that the basis of the well-weighted cameras nearly annihilates, so the
// dot products cancel heavily; with u = u_hi + u_lo from the refined solve and the same float32
// basis the fold used, they keep the accuracy of the forward solve.
template <int B>
__global__ void __launch_bounds__(kPayThreads) k_payload_adjoint(int64_t n, int K, int G, const float* __restrict__ means,
                                                                 const DevCam* __restrict__ cams, int cb,
                                                                 const float* __restrict__ coeffs,
                                                                 const float* __restrict__ u,
                                                                 const float* __restrict__ u_lo,
                                                                 const float* __restrict__ reg,
                                                                 float* __restrict__ payload) {
  extern __shared__ float s_rows[];
  const int BK = B * K, RW = BK | 1;
  const int64_t i0 = blockIdx.x * (int64_t)G;
  const int gcount = (int)min((int64_t)G, n - i0);
  stage_rows(coeffs, i0, gcount, BK, RW, s_rows);
  stage_rows(u, i0, gcount, BK, RW, s_rows + G * RW);
  stage_rows(u_lo, i0, gcount, BK, RW, s_rows + 2 * G * RW);
  __syncthreads();
  const int g = threadIdx.x % G, lanes = kPayThreads / G, cl = threadIdx.x / G;
  if (g >= gcount) return;
  const int64_t i = i0 + g;
  const float mu[3] = {means[3 * i], means[3 * i + 1], means[3 * i + 2]};
  const float* ci = s_rows + g * RW;
  const float* ui = s_rows + (G + g) * RW;
  const float* li = s_rows + (2 * G + g) * RW;
  const float rg = reg[i];
  for (int j = cl; j < cb; j += lanes) {
    const float3 d = view_dir(mu, cams[j]);
    float Y[B];
    sh_basis<B>(d.x, d.y, d.z, Y);
    float* out = payload + ((int64_t)j * n + i) * (K + 1);
    float beta = -rg, beta_c = 0.0f;
    for (int k = 0; k < K; ++k) {
      float a = 0.0f, a_c = 0.0f, yc = 0.0f, yc_c = 0.0f;
#pragma unroll
      for (int m = 0; m < B; ++m) {
        const float uh = ui[m * K + k], cm = ci[m * K + k];
        const float p = Y[m] * uh, q = Y[m] * cm;
        two_sum_acc(a, a_c, p);
        a_c += fmaf(Y[m], uh, -p) + Y[m] * li[m * K + k];
        two_sum_acc(yc, yc_c, q);
        yc_c += fmaf(Y[m], cm, -q);
      }
      a += a_c;
      yc += yc_c;
      out[k] = a;
      const float pb = -a * yc;
      two_sum_acc(beta, beta_c, pb);
      beta_c += fmaf(-a, yc, -pb);
    }
    out[K] = beta + beta_c;
  }
}

// Gaussians per payload CTA: the largest power of two <= 64 whose staged rows (arrays of them)
// fit in 48 KB of shared memory.
int payload_group(int B, int K, int arrays) {
  const size_t row = (size_t)((B * K) | 1) * sizeof(float) * arrays;
  int G = 64;
  while (G > 1 && (size_t)G * row > 48 * 1024) G >>= 1;
  return G;
}

template <int B, bool MIXED>
void fold_b(const Problem& p, const float* means, int cb, const Workspace& ws, bool first, bool want_gram,
            cudaStream_t s) {
  const unsigned grid = (unsigned)((p.n * kFoldGroup + kSolveThreads - 1) / kSolveThreads);
  if (p.K == 3) {  // RGB: one launch of three channels (no zero fourth channel)
    k_fold<B, 3, MIXED><<<grid, kSolveThreads, 0, s>>>(means, p.n, ws.cams, cb, ws.acc, p.K, p.acc_stride, 0, first,
                                                        want_gram, ws.G, ws.Glo, ws.bvec, ws.blo, ws.wsum, ws.wlo);
    note_launches(1);
    return;
  }
  for (int k0 = 0; k0 < p.K; k0 += 4) {
    k_fold<B, 4, MIXED><<<grid, kSolveThreads, 0, s>>>(means, p.n, ws.cams, cb, ws.acc, p.K, p.acc_stride, k0, first,
                                                        want_gram, ws.G, ws.Glo, ws.bvec, ws.blo, ws.wsum, ws.wlo);
    note_launches(1);
  }
}

template <int B, bool MIXED>
void solve_b(const Problem& p, const float* lam_dev, const Workspace& ws, float* coeffs, uint8_t* st,
             float* chol, const float* means, int n_acc_cams, cudaStream_t s) {
  const unsigned grid = (unsigned)((p.n * kGroup + kSolveThreads - 1) / kSolveThreads);
  if (p.K == 3)
    k_solve<B, MIXED, 3><<<grid, kSolveThreads, 0, s>>>(p.n, p.K, ws.G, ws.Glo, ws.bvec, ws.blo, ws.wsum, ws.wlo,
                                                         lam_dev, p.cond_tau, p.refold_tau, coeffs, st, chol,
                                                         ws.status, ws.acc,
                                                         p.acc_stride, n_acc_cams, ws.cams, means);
  else
    k_solve<B, MIXED, 4><<<grid, kSolveThreads, 0, s>>>(p.n, p.K, ws.G, ws.Glo, ws.bvec, ws.blo, ws.wsum, ws.wlo,
                                                         lam_dev, p.cond_tau, p.refold_tau, coeffs, st, chol,
                                                         ws.status, ws.acc,
                                                         p.acc_stride, n_acc_cams, ws.cams, means);
  note_launches(1);
}

}  // namespace

// The first pass of a call writes G, b, w; later passes add to them.
void launch_fold(const Problem& p, const float* means, int cb, bool first, bool want_gram, const Workspace& ws,
                 cudaStream_t s) {
  const bool mixed = p.precision == 1;
#define ICGS_FOLD(B)                                                    \
  if (mixed) fold_b<B, true>(p, means, cb, ws, first, want_gram, s);   \
  else fold_b<B, false>(p, means, cb, ws, first, want_gram, s)
  if (p.B == 4) { ICGS_FOLD(4); }
  else if (p.B == 9) { ICGS_FOLD(9); }
  else { ICGS_FOLD(16); }
#undef ICGS_FOLD
}

// ------------------------------------------------------------------------------------------
// normal equations in and out (camera sharding): per Gaussian R = P + B K + 1 doubles, P = B(B+1)/2:
// the upper triangle of G row by row (r <= c), then b [B,K], then w; hi + lo combined in double
// ------------------------------------------------------------------------------------------
namespace {

constexpr double kY0d = 0.28209479177387814;

// (r, c) of packed upper-triangle entry k of a B x B matrix (rows r = 0..B-1 hold c = r..B-1)
__device__ __forceinline__ void packed_rc(int k, int B, int& r, int& c) {
  r = 0;
  while (k >= B - r) {
    k -= B - r;
    ++r;
  }
  c = r + k;
}
__device__ __forceinline__ int packed_index(int r, int c, int B) {  // r <= c
  return r * B - r * (r - 1) / 2 + (c - r);
}

__global__ void k_export_packed(int64_t n, int B, int K, const float* __restrict__ G, const float* __restrict__ Glo,
                                const float* __restrict__ b, const float* __restrict__ blo,
                                const float* __restrict__ w, const float* __restrict__ wlo, double* __restrict__ out) {
  const int P = B * (B + 1) / 2, R = P + B * K + 1;
  const int64_t total = n * (int64_t)R, stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += stride) {
    const int64_t i = e / R;
    const int k = (int)(e - i * R);
    double v;
    if (k < P) {
      int r, c;
      packed_rc(k, B, r, c);
      const int64_t idx = (i * B + r) * B + c;
      v = (double)G[idx] + (Glo ? (double)Glo[idx] : 0.0);
    } else if (k < P + B * K) {
      const int64_t idx = i * B * K + (k - P);
      v = (double)b[idx] + (blo ? (double)blo[idx] : 0.0);
    } else {
      v = (double)w[i] + (wlo ? (double)wlo[i] : 0.0);
    }
    out[e] = v;
  }
}

// L = 0: acc[i] = (V, S_0..S_{K-1}) gives G = Y0^2 V, b = Y0 S, w = V
__global__ void k_export_packed_l0(int64_t n, int K, int RS, const float* __restrict__ acc, double* __restrict__ out) {
  const int R = K + 2;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * (int64_t)R) return;
  const int64_t i = e / R;
  const int k = (int)(e - i * R);
  const double V = (double)acc[i * RS];
  out[e] = k == 0 ? kY0d * kY0d * V : (k <= K ? kY0d * (double)acc[i * RS + k] : V);
}

__device__ __forceinline__ void split_double(double x, float& hi, float& lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}

__global__ void k_import_packed(int64_t n, int B, int K, const double* __restrict__ in, float* __restrict__ G,
                                float* __restrict__ Glo, float* __restrict__ b, float* __restrict__ blo,
                                float* __restrict__ w, float* __restrict__ wlo) {
  const int P = B * (B + 1) / 2, R = P + B * K + 1, E = B * B + B * K + 1;
  const int64_t total = n * (int64_t)E, stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += stride) {
    const int64_t i = e / E;
    const int k = (int)(e - i * E);
    const double* row = in + i * R;
    float hi, lo;
    if (k < B * B) {
      const int r = k / B, c = k - r * B;
      split_double(row[r <= c ? packed_index(r, c, B) : packed_index(c, r, B)], hi, lo);
      G[i * B * B + k] = hi;
      if (Glo) Glo[i * B * B + k] = lo;
    } else if (k < B * B + B * K) {
      const int kk = k - B * B;
      split_double(row[P + kk], hi, lo);
      b[i * B * K + kk] = hi;
      if (blo) blo[i * B * K + kk] = lo;
    } else {
      split_double(row[R - 1], hi, lo);
      w[i] = hi;
      if (wlo) wlo[i] = lo;
    }
  }
}

// L = 0: back to acc[i] = (V, S) with V = w, S = b / Y0
__global__ void k_import_packed_l0(int64_t n, int K, int RS, const double* __restrict__ in, float* __restrict__ acc) {
  const int R = K + 2;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * (int64_t)(K + 1)) return;
  const int64_t i = e / (K + 1);
  const int k = (int)(e - i * (K + 1));
  const double* row = in + i * R;
  if (k == K) acc[i * RS] = (float)row[R - 1];
  else acc[i * RS + 1 + k] = (float)(row[1 + k] / kY0d);
}

}  // namespace

void launch_export_normal(const Problem& p, const Workspace& ws, double* sums, cudaStream_t s) {
  if (p.B == 1) {
    const int64_t m = p.n * (int64_t)(p.K + 2);
    k_export_packed_l0<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(p.n, p.K, p.acc_stride, ws.acc, sums);
  } else {
    const bool mixed = p.precision == 1;
    k_export_packed<<<1216, 256, 0, s>>>(p.n, p.B, p.K, ws.G, mixed ? ws.Glo : nullptr, ws.bvec,
                                         mixed ? ws.blo : nullptr, ws.wsum, mixed ? ws.wlo : nullptr, sums);
  }
  note_launches(1);
}

void launch_import_normal(const Problem& p, const Workspace& ws, const double* sums, cudaStream_t s) {
  if (p.B == 1) {
    const int64_t m = p.n * (int64_t)(p.K + 1);
    k_import_packed_l0<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(p.n, p.K, p.acc_stride, sums, ws.acc);
  } else {
    const bool mixed = p.precision == 1;
    k_import_packed<<<1216, 256, 0, s>>>(p.n, p.B, p.K, sums, ws.G, mixed ? ws.Glo : nullptr, ws.bvec,
                                         mixed ? ws.blo : nullptr, ws.wsum, mixed ? ws.wlo : nullptr);
  }
  note_launches(1);
}

// Merges one target set's accumulator rows into the combined rows: S_0..S_{Ks-1} of the set into
// columns 1 + col0.., and V (column 0) from the first set only.
__global__ void k_merge_set(int64_t rows, int Ks, int RSs, const float* __restrict__ src, int RS, int col0,
                            float* __restrict__ dst) {
  const int W = Ks + 1;
  const int64_t total = rows * W, stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += stride) {
    const int64_t r = e / W;
    const int k = (int)(e - r * W);
    if (k == 0) {
      if (col0 == 0) dst[r * RS] = src[r * RSs];
    } else {
      dst[r * RS + col0 + k] = src[r * RSs + k];
    }
  }
}

void launch_merge_set(int64_t rows, int Ks, int RSs, const float* src, int RS, int col0, float* dst, cudaStream_t s) {
  const int64_t m = rows * (int64_t)(Ks + 1);
  const unsigned grid = (unsigned)std::min<int64_t>((m + 255) / 256, 152 * 16);
  k_merge_set<<<grid, 256, 0, s>>>(rows, Ks, RSs, src, RS, col0, dst);
  note_launches(1);
}

void launch_solve(const Problem& p, const float* lam_dev, const float* lam_host, const Workspace& ws,
                  float* coeffs, uint8_t* status, float* chol, const float* means, int n_acc_cams,
                  cudaStream_t s, float tau, uint8_t* keep) {
  if (p.B == 1) {
    const int64_t m = p.n * (int64_t)p.K;
    k_solve_l0<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(p.n, p.K, p.acc_stride, ws.acc, lam_host[0], coeffs, status, chol,
                                                           tau, keep);
    note_launches(1);
    return;
  }
  const bool mixed = p.precision == 1;
#define ICGS_SOLVE(B)                                                                              \
  if (mixed) solve_b<B, true>(p, lam_dev, ws, coeffs, status, chol, means, n_acc_cams, s);       \
  else solve_b<B, false>(p, lam_dev, ws, coeffs, status, chol, means, n_acc_cams, s)
  if (p.B == 4) { ICGS_SOLVE(4); }
  else if (p.B == 9) { ICGS_SOLVE(9); }
  else { ICGS_SOLVE(16); }
#undef ICGS_SOLVE
}

void launch_refine_update(const Problem& p, const float* lam_dev, const float* lam_host, const float* chol,
                          const Workspace& ws, float* coeffs, cudaStream_t s) {
  if (p.B == 1) {
    const int64_t m = p.n * (int64_t)p.K;
    k_refine_update_l0<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(p.n, p.K, p.acc_stride, ws.acc, lam_host[0], coeffs);
    note_launches(1);
    return;
  }
  const unsigned grid = (unsigned)((p.n * kGroup + kSolveThreads - 1) / kSolveThreads);
  const bool mixed = p.precision == 1;
#define ICGS_REF(B)                                                                                           \
  if (mixed)                                                                                                  \
    k_refine_update<B, true><<<grid, kSolveThreads, 0, s>>>(p.n, p.K, chol, ws.bvec, ws.blo, ws.wsum, ws.wlo,  \
                                                             lam_dev, coeffs);                                 \
  else                                                                                                        \
    k_refine_update<B, false><<<grid, kSolveThreads, 0, s>>>(p.n, p.K, chol, ws.bvec, ws.blo, ws.wsum, ws.wlo, \
                                                              lam_dev, coeffs)
  if (p.B == 4) { ICGS_REF(4); }
  else if (p.B == 9) { ICGS_REF(9); }
  else { ICGS_REF(16); }
#undef ICGS_REF
  note_launches(1);
}

void launch_payload_render(const Problem& p, const float* means, const float* coeffs, int cb,
                           const Workspace& ws, cudaStream_t s) {
  const int G = payload_group(p.B, p.K, 1);
  const unsigned grid = (unsigned)((p.n + G - 1) / G);
  const size_t smem = (size_t)G * ((p.B * p.K) | 1) * sizeof(float);
  if (p.B == 1) k_payload_render<1><<<grid, kPayThreads, smem, s>>>(p.n, p.K, G, means, ws.cams, cb, coeffs, ws.payload);
  else if (p.B == 4) k_payload_render<4><<<grid, kPayThreads, smem, s>>>(p.n, p.K, G, means, ws.cams, cb, coeffs, ws.payload);
  else if (p.B == 9) k_payload_render<9><<<grid, kPayThreads, smem, s>>>(p.n, p.K, G, means, ws.cams, cb, coeffs, ws.payload);
  else k_payload_render<16><<<grid, kPayThreads, smem, s>>>(p.n, p.K, G, means, ws.cams, cb, coeffs, ws.payload);
  note_launches(1);
}

void launch_adjoint_prepare(const Problem& p, const float* lam_dev, const float* lam_host,
                                const float* coeffs, const float* chol, const float* grad_coeffs,
                                const Workspace& ws, cudaStream_t s) {
  if (p.B == 1) {
    k_adjoint_prep_l0<<<(unsigned)((p.n + 255) / 256), 256, 0, s>>>(p.n, p.K, chol, grad_coeffs, coeffs,
                                                                     lam_host[0], ws.u, ws.u_lo, ws.reg);
    note_launches(1);
    return;
  }
  const unsigned grid = (unsigned)((p.n * kGroup + kSolveThreads - 1) / kSolveThreads);
  if (p.B == 4)
    k_adjoint_prep<4><<<grid, kSolveThreads, 0, s>>>(p.n, p.K, chol, grad_coeffs, coeffs, lam_dev, ws.u, ws.u_lo,
                                                      ws.reg);
  else if (p.B == 9)
    k_adjoint_prep<9><<<grid, kSolveThreads, 0, s>>>(p.n, p.K, chol, grad_coeffs, coeffs, lam_dev, ws.u, ws.u_lo,
                                                      ws.reg);
  else
    k_adjoint_prep<16><<<grid, kSolveThreads, 0, s>>>(p.n, p.K, chol, grad_coeffs, coeffs, lam_dev, ws.u, ws.u_lo,
                                                      ws.reg);
  note_launches(1);
}

void launch_payload_adjoint(const Problem& p, const float* means, const float* coeffs, int cb,
                            const Workspace& ws, cudaStream_t s) {
  const int G = payload_group(p.B, p.K, 3);
  const unsigned grid = (unsigned)((p.n + G - 1) / G);
  const size_t smem = 3 * (size_t)G * ((p.B * p.K) | 1) * sizeof(float);
#define ICGS_PAYADJ(BB)                                                                              \
  k_payload_adjoint<BB><<<grid, kPayThreads, smem, s>>>(p.n, p.K, G, means, ws.cams, cb, coeffs, ws.u, \
                                                        ws.u_lo, ws.reg, ws.payload)
  if (p.B == 1) ICGS_PAYADJ(1);
  else if (p.B == 4) ICGS_PAYADJ(4);
  else if (p.B == 9) ICGS_PAYADJ(9);
  else ICGS_PAYADJ(16);
#undef ICGS_PAYADJ
  note_launches(1);
}

}  // namespace icgs
