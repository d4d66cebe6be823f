// Row-scaled BF16 planes of the operands of the mixed exchange (B rows, C^T rows, X rows).
// With sigma the power of two just above the row's max |x|:
//   p0 = x rounded to the grid sigma 2^-7   (an integer in [-128, 128] times sigma 2^-7),
//   p1 = x - p0 rounded to the grid sigma 2^-15 (again an integer in [-128, 128]),
//   p2, p3, ... = RN_bf16 of what the planes before leave.
// Products of the two fixed-point planes of two rows are integers on grids fixed along the
// contraction, so the exchange sums them exactly in FP32 accumulators of their own; only
// the contributions of elements far below the row max (under 2^-16 of it) pass through the
// floating planes, whose FP32 sums round.
#pragma once
#include <cuda_bf16.h>

namespace dfscf {

constexpr int kPlanesMax = 5;

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
  double h0 = 0.0, h1 = 0.0;
  if (sig > 0.0) {
    h0 = rint(x * (128.0 / sig)) * (sig * (1.0 / 128.0));
    h1 = rint((x - h0) * (32768.0 / sig)) * (sig * (1.0 / 32768.0));
  }
  q[0] = __double2bfloat16(h0);  // exact: at most 8 significant bits
  q[1] = __double2bfloat16(h1);
  double r = (x - h0) - h1;
#pragma unroll
  for (int j = 2; j < kPlanesMax; ++j) {
    q[j] = __double2bfloat16(r);
    r -= (double)__bfloat162float(q[j]);
  }
}

// X held as an unevaluated FP32 pair x = hi + lo (the half-transform's two accumulators).
// The fixed-point planes round the pair's sum to their grids, so they carry the leading bits
// of x whichever accumulator holds them; each remainder is formed exactly with two TwoSums
// (Knuth), and every floating plane rounds the remainder's sum to BF16 and keeps what is
// left as a pair.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void split_row_pair(float hi, float lo, float sig, __nv_bfloat16 (&q)[kPlanesMax]) {
  float rh = hi, rl = lo;
#pragma unroll
  for (int j = 0; j < 2; ++j) {  // the two fixed-point planes
    const float g = j == 0 ? 128.0f : 32768.0f;
    float h = 0.0f;
    if (sig > 0.0f) h = rintf((rh + rl) * (g / sig)) * (sig / g);
    q[j] = __float2bfloat16_rn(h);
    float s1, e1, e2;
    two_sum(rh, -h, s1, e1);  // rh - h = s1 + e1
    two_sum(s1, rl, rh, e2);  // s1 + rl = rh + e2
    rl = e1 + e2;             // below 2^-24 of the remainder: its rounding is negligible
  }
#pragma unroll
  for (int j = 2; j < kPlanesMax; ++j) {
    float sum, err;
    two_sum(rh, rl, sum, err);
    q[j] = __float2bfloat16_rn(sum);
    rh = sum - __bfloat162float(q[j]);  // exact: q[j] is sum rounded to 8 bits
    rl = err;
  }
}

}  // namespace dfscf
