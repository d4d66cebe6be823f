// Order-zero Boys function F0(t) = int_0^1 exp(-t u^2) du on the GPU.
//
// Every s-type Coulomb integral of the density-fitting path ((P|Q), (Q|mn), and the
// nuclear attraction) reduces to a prefactor times F0 of a scaled squared distance.
// One lane evaluates one integral; the three regimes below are chosen per lane and the
// far regime (most pairs of a large molecule) needs only one square root and division.
//   t < 1e-3 : Maclaurin series sum_k (-t)^k / (k! (2k+1)), seven terms (truncation
//              error below 1e-22);
//   t > 40   : erf(sqrt t) equals 1 in double precision, F0 = (sqrt(pi)/2) / sqrt(t);
//   otherwise: F0 = (sqrt(pi)/2) erf(sqrt t) / sqrt t, with CUDA's erf.
#pragma once

__device__ __forceinline__ double boys_f0(double t) {
  const double half_sqrt_pi = 0.88622692545275801365;
  if (t < 1e-3) {
    // coefficients 1/(k! (2k+1)) with alternating signs, Horner in t
    double r = 1.0 / 9360.0;
    r = fma(r, -t, 1.0 / 1320.0);
    r = fma(r, -t, 1.0 / 216.0);
    r = fma(r, -t, 1.0 / 42.0);
    r = fma(r, -t, 1.0 / 10.0);
    r = fma(r, -t, 1.0 / 3.0);
    return fma(r, -t, 1.0);
  }
  double s = sqrt(t);
  if (t > 40.0) return half_sqrt_pi / s;
  return half_sqrt_pi * erf(s) / s;
}
