// Row-scaled BF16 planes of the operands of the mixed exchange (B rows, C^T rows, X rows):
//   p0 = sigma 2^-7 RN(x 2^7 / sigma), sigma the power of two just above the row's max |x|,
//        so p0 is an integer in [-128, 128] on a grid fixed along the row;
//   p1, p2, p3 = RN_bf16 of what the planes before leave of x.
// Products of two p0 rows sum exactly in an FP32 accumulator (integers on one grid); the
// residual planes keep about 24 bits of |x| itself for elements far below the row max.
#pragma once
#include <cuda_bf16.h>

namespace dfscf {

constexpr int kPlanesMax = 4;

// Power of two strictly above amax (0 for amax = 0).
__device__ __forceinline__ double row_scale(double amax) {
  if (!(amax > 0.0)) return 0.0;
  int e;
  frexp(amax, &e);  // amax = f 2^e, f in [0.5, 1)
  return ldexp(1.0, e);
}

__device__ __forceinline__ float row_scale_f(float amax) {
  if (!(amax > 0.0f)) return 0.0f;
  int e;
  frexpf(amax, &e);
  return ldexpf(1.0f, e);
}

// Residuals in FP64.
__device__ __forceinline__ void split_row_value(double x, double sig, __nv_bfloat16 (&q)[kPlanesMax]) {
  double h = 0.0;
  if (sig > 0.0) h = rint(x * (128.0 / sig)) * (sig * (1.0 / 128.0));
  q[0] = __double2bfloat16(h);  // exact: at most 8 significant bits
  double r = x - h;
#pragma unroll
  for (int j = 1; j < kPlanesMax; ++j) {
    q[j] = __double2bfloat16(r);
    r -= (double)__bfloat162float(q[j]);
  }
}

// FP32 version for the half-transformed X (x exact in FP32; every residual is exact).
__device__ __forceinline__ void split_row_value_f(float x, float sig, __nv_bfloat16 (&q)[kPlanesMax]) {
  float h = 0.0f;
  if (sig > 0.0f) h = rintf(x * (128.0f / sig)) * (sig * (1.0f / 128.0f));
  q[0] = __float2bfloat16_rn(h);
  float r = x - h;
#pragma unroll
  for (int j = 1; j < kPlanesMax; ++j) {
    q[j] = __float2bfloat16_rn(r);
    r -= __bfloat162float(q[j]);
  }
}

}  // namespace dfscf
