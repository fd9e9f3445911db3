// icgs_device.cuh -- device helpers shared by the CUDA kernels of libicgs.so.
#pragma once

#include <cstdint>

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "icgs_internal.h"

namespace icgs {

constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;

// The lo part of a float-float projected mean is at most half an ulp of its hi part; scaled by
// 2^8 it is below 1/2 for |mean| < 2^16 pixels and fp16 keeps it to about 2^-27 of a pixel there.
constexpr float kMeanLoScale = 256.0f;
constexpr float kMeanLoScaleInv = 1.0f / 256.0f;

__device__ __forceinline__ float pack_half2(__half a, __half b) {
  return __uint_as_float((uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16));
}
__device__ __forceinline__ float2 unpack_half2(float v) {
  const uint32_t u = __float_as_uint(v);
  return make_float2(__half2float(__ushort_as_half((unsigned short)(u & 0xFFFFu))),
                     __half2float(__ushort_as_half((unsigned short)(u >> 16))));
}

// Real orthonormal spherical harmonics (Eq. 3) of a unit direction (x, y, z), degree 0..3, index
// l*l + l + m. These are the Cartesian forms of sqrt(2) N_lm P_l^|m|(cos th) {cos, sin}(|m| ph)
// without the Condon-Shortley phase; the normalisation constants are
// N = 1/(2 sqrt(pi)), sqrt(3/(4 pi)), (1/2)sqrt(15/pi), (1/4)sqrt(5/pi), (1/4)sqrt(15/pi),
// (1/4)sqrt(35/(2 pi)), (1/2)sqrt(105/pi), (1/4)sqrt(21/(2 pi)), (1/4)sqrt(7/pi), (1/4)sqrt(105/pi).
template <int B, typename T = float>
__device__ __forceinline__ void sh_basis(T x, T y, T z, T* Y) {
  Y[0] = T(0.28209479177387814);
  if constexpr (B > 1) {
    const T c1 = T(0.48860251190291987);
    Y[1] = c1 * y;
    Y[2] = c1 * z;
    Y[3] = c1 * x;
  }
  if constexpr (B > 4) {
    const T xx = x * x, yy = y * y, zz = z * z;
    Y[4] = T(1.0925484305920792) * (x * y);
    Y[5] = T(1.0925484305920792) * (y * z);
    Y[6] = T(0.31539156525252005) * (T(3) * zz - T(1));
    Y[7] = T(1.0925484305920792) * (x * z);
    Y[8] = T(0.54627421529603959) * (xx - yy);
    if constexpr (B > 9) {
      Y[9] = T(0.59004358992664352) * y * (T(3) * xx - yy);
      Y[10] = T(2.8906114426405538) * (x * y) * z;
      Y[11] = T(0.45704579946446572) * y * (T(5) * zz - T(1));
      Y[12] = T(0.37317633259011540) * z * (T(5) * zz - T(3));
      Y[13] = T(0.45704579946446572) * x * (T(5) * zz - T(1));
      Y[14] = T(1.4453057213202769) * z * (xx - yy);
      Y[15] = T(0.59004358992664352) * x * (xx - T(3) * yy);
    }
  }
}

// Unit direction from the camera centre to the Gaussian mean.
__device__ __forceinline__ float3 view_dir(const float* mean, const DevCam& c) {
  float dx = mean[0] - c.centre[0], dy = mean[1] - c.centre[1], dz = mean[2] - c.centre[2];
  float r = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
  return make_float3(dx * r, dy * r, dz * r);
}

// Knuth's branch-free TwoSum: s + c += x with the rounding error of the sum kept in c.
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float x) {
  float t = s + x;
  float bp = t - s;
  float err = (s - (t - bp)) + (x - bp);
  s = t;
  c += err;
}

__device__ __forceinline__ float load_target(const void* base, int64_t idx, int dtype) {
  if (dtype == 0) return __ldg(reinterpret_cast<const float*>(base) + idx);
  unsigned short h = __ldg(reinterpret_cast<const unsigned short*>(base) + idx);
  if (dtype == 1) return __uint_as_float(static_cast<uint32_t>(h) << 16);  // bf16
  return __half2float(__ushort_as_half(h));                                 // f16
}

}  // namespace icgs
