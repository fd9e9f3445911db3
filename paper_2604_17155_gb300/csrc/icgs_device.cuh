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

// Real orthonormal spherical harmonics (Eq. 3) of a unit direction (x, y, z), degree 0..3, index
// l*l + l + m. These are the Cartesian forms of sqrt(2) N_lm P_l^|m|(cos th) {cos, sin}(|m| ph)
// without the Condon-Shortley phase; the normalisation constants are
// N = 1/(2 sqrt(pi)), sqrt(3/(4 pi)), (1/2)sqrt(15/pi), (1/4)sqrt(5/pi), (1/4)sqrt(15/pi),
// (1/4)sqrt(35/(2 pi)), (1/2)sqrt(105/pi), (1/4)sqrt(21/(2 pi)), (1/4)sqrt(7/pi), (1/4)sqrt(105/pi).
template <int B>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float* Y) {
  Y[0] = 0.28209479177387814f;
  if constexpr (B > 1) {
    const float c1 = 0.48860251190291987f;
    Y[1] = c1 * y;
    Y[2] = c1 * z;
    Y[3] = c1 * x;
  }
  if constexpr (B > 4) {
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = 1.0925484305920792f * (x * y);
    Y[5] = 1.0925484305920792f * (y * z);
    Y[6] = 0.31539156525252005f * (3.0f * zz - 1.0f);
    Y[7] = 1.0925484305920792f * (x * z);
    Y[8] = 0.54627421529603959f * (xx - yy);
    if constexpr (B > 9) {
      Y[9] = 0.59004358992664352f * y * (3.0f * xx - yy);
      Y[10] = 2.8906114426405538f * (x * y) * z;
      Y[11] = 0.45704579946446572f * y * (5.0f * zz - 1.0f);
      Y[12] = 0.37317633259011540f * z * (5.0f * zz - 3.0f);
      Y[13] = 0.45704579946446572f * x * (5.0f * zz - 1.0f);
      Y[14] = 1.4453057213202769f * z * (xx - yy);
      Y[15] = 0.59004358992664352f * x * (xx - 3.0f * yy);
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
