// Density-fitting error diagnostics on the GPU (arXiv 2506.06661):
//   Section "Density fitting", Lehtola's diagonal error
//       Delta = sum_mn [(mn|mn) - sum_P T_{P,mn} T_{P,mn}];
//   Section "Automatic Differentiation", the residual of the auxiliary-basis fit
//       sigma_mn = (mn|mn) - sum_PQ (P|mn) (M^-1)_PQ (Q|mn)
//   and its Jacobian with respect to the auxiliary exponents, which the paper obtains by
//   automatic differentiation and this file writes out for s primitives:
//       d sigma_mn / d alpha_P = -2 C_{P,mn} [d(P|mn)/d alpha_P - sum_Q m1_{PQ} C_{Q,mn}],
//   C = M^-1 (P|mn) = L^-T T (the fitting coefficients), m1_{PQ} = d(P|Q)/d alpha_P with
//   alpha_Q fixed.  The Jacobian is contracted on the GPU with d alpha_P / d theta_t for a
//   few parameters theta (for an even-tempered set: ln alpha_min and ln beta), so the output
//   is npair x ntheta, not npair x naux.
// Exponent derivatives of the normalised closed forms (product rule):
//   d ln(N_c / (c sqrt(c + x))) / dc = 3/(4c) - 1/c - 1/(2(c + x)),
//   d/dc [c x R^2 / (c + x)] = x^2 R^2 / (c + x)^2,   F0'(t) = -F1(t).
#include "boys.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace dfscf {

namespace {

__device__ __forceinline__ double norm_s_(double a) {
  double x = 2.0 * a / kPi;
  return sqrt(x * sqrt(x));
}

// F1(t) = int_0^1 u^2 exp(-t u^2) du = (F0(t) - exp(-t)) / (2t); Maclaurin series
// sum_k (-t)^k / (k! (2k+3)) below t = 1e-2 (eight terms, truncation below 1e-20).
__device__ __forceinline__ double boys_f1(double t, double f0) {
  if (t < 1e-2) {
    double r = 1.0 / (40320.0 * 19.0);
    r = fma(r, -t, 1.0 / (5040.0 * 17.0));
    r = fma(r, -t, 1.0 / (720.0 * 15.0));
    r = fma(r, -t, 1.0 / (120.0 * 13.0));
    r = fma(r, -t, 1.0 / (24.0 * 11.0));
    r = fma(r, -t, 1.0 / (6.0 * 9.0));
    r = fma(r, -t, 1.0 / (2.0 * 7.0));
    r = fma(r, -t, 1.0 / 5.0);
    return fma(r, -t, 1.0 / 3.0);
  }
  return (f0 - exp(-t)) / (2.0 * t);
}

// m1[c][d] = d (c|d) / d alpha_c with alpha_d fixed.
__global__ void int2c_dexp_kernel(const double* __restrict__ xyz, const double* __restrict__ ex, int naux,
                                  double* __restrict__ m1) {
  const int c = blockIdx.y;
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= naux) return;
  const double ec = ex[c], ed = ex[d];
  const double dx = xyz[3 * c] - xyz[3 * d], dy = xyz[3 * c + 1] - xyz[3 * d + 1], dz = xyz[3 * c + 2] - xyz[3 * d + 2];
  const double r2 = dx * dx + dy * dy + dz * dz;
  const double pre = norm_s_(ec) * norm_s_(ed) * 2.0 * kPi * kPi * sqrt(kPi) / (ec * ed * sqrt(ec + ed));
  const double t = ec * ed / (ec + ed) * r2;
  const double f0 = boys_f0(t), f1 = boys_f1(t, f0);
  m1[(size_t)c * naux + d] =
      pre * f0 * (0.75 / ec - 1.0 / ec - 0.5 / (ec + ed)) - pre * f1 * ed * ed / ((ec + ed) * (ec + ed)) * r2;
}

// dv[Q][mn] = d (Q|mn) / d alpha_Q from the pair table of launch_int3c (padding zero).
__global__ void int3c_dexp_kernel(const double* __restrict__ pp, const double* __restrict__ px,
                                  const double* __restrict__ py, const double* __restrict__ pz,
                                  const double* __restrict__ pk, long npair, long ld,
                                  const double* __restrict__ axyz, const double* __restrict__ aex,
                                  double* __restrict__ dv) {
  const int q = blockIdx.y;
  const long ij = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (ij >= ld) return;
  double* row = dv + (size_t)q * ld;
  if (ij >= npair) {
    row[ij] = 0.0;
    return;
  }
  const double c = aex[q];
  const double p = pp[ij];
  const double dx = px[ij] - axyz[3 * q], dy = py[ij] - axyz[3 * q + 1], dz = pz[ij] - axyz[3 * q + 2];
  const double r2 = dx * dx + dy * dy + dz * dz;
  const double inv = 1.0 / (p + c);
  const double t = p * c * inv * r2;
  const double pre = pk[ij] * norm_s_(c) / c * sqrt(inv);
  const double f0 = boys_f0(t), f1 = boys_f1(t, f0);
  row[ij] = pre * f0 * (0.75 / c - 1.0 / c - 0.5 * inv) - pre * f1 * p * p * inv * inv * r2;
}

// sigma_mn = (mn|mn) - sum_P T_{P,mn}^2, with (ab|ab) = K_ab^2 / (2 pi^(5/2) sqrt(2p)) from
// the pair table (K_ab = N_a N_b e^{-mu R^2} 2 pi^(5/2) / p).  One lane per packed pair.
__global__ void residual_kernel(const double* __restrict__ pp, const double* __restrict__ pk, long npair,
                                const double* __restrict__ T, long ld, int naux, double* __restrict__ sigma) {
  const long ij = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (ij >= npair) return;
  double s = 0.0;
  for (int P = 0; P < naux; ++P) {
    const double b = T[DF_IX((size_t)P * ld + ij, (size_t)naux * ld)];
    s = fma(b, b, s);
  }
  const double k = pk[ij];
  const double diag = k * k / (2.0 * kPi * kPi * sqrt(kPi) * sqrt(2.0 * pp[ij]));
  sigma[ij] = diag - s;
}

// Delta over ordered pairs (weight 2 off the diagonal), one CTA.
__global__ void delta_kernel(const double* __restrict__ sigma, int nao, double* __restrict__ out) {
  __shared__ double sh[32];
  const long npair = (long)nao * (nao + 1) / 2;
  double t = 0.0;
  for (long ij = threadIdx.x; ij < npair; ij += blockDim.x) {
    int m, n;
    unpack_pair(ij, m, n);
    t += (m == n ? 1.0 : 2.0) * sigma[ij];
  }
  t = block_sum(t, sh);
  if (threadIdx.x == 0) *out = t;
}

constexpr int kMaxTheta = 8;

// jac[mn][t] = sum_P -2 C[P][mn] (dv[P][mn] - G[P][mn]) dalpha[P][t].
__global__ void jac_theta_kernel(const double* __restrict__ C, const double* __restrict__ dv,
                                 const double* __restrict__ G, long ld, long npair, int naux,
                                 const double* __restrict__ dalpha, int ntheta, double* __restrict__ jac) {
  const long ij = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (ij >= npair) return;
  double acc[kMaxTheta];
#pragma unroll
  for (int t = 0; t < kMaxTheta; ++t) acc[t] = 0.0;
  for (int P = 0; P < naux; ++P) {
    const size_t o = DF_IX((size_t)P * ld + ij, (size_t)naux * ld);
    const double g = -2.0 * C[o] * (dv[o] - G[o]);
#pragma unroll
    for (int t = 0; t < kMaxTheta; ++t)
      if (t < ntheta) acc[t] = fma(g, dalpha[(size_t)P * ntheta + t], acc[t]);
  }
  for (int t = 0; t < ntheta; ++t) jac[DF_IX(ij * ntheta + t, npair * ntheta)] = acc[t];
}

__global__ void identity_kernel(double* __restrict__ A, int n) {
  const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < (long)n * n) A[q] = (q / n == q % n) ? 1.0 : 0.0;
}

struct FitWork {
  double *L, *Linv, *m1, *pair_tab, *T, *C, *dv, *G, *maxdiag, *delta;
  int* status;
};

void fit_layout(int nao, int naux, bool jac, Arena* a, Sizer* z, FitWork* w) {
  const long ld = B_ld(nao);
  const size_t big = (size_t)naux * ld;
#define TAKE(T_, ptr, count) \
  if (a) ptr = a->take<T_>(count); else z->take<T_>(count);
  TAKE(double, w->L, (size_t)naux * naux);
  TAKE(double, w->pair_tab, 5 * (size_t)npair_of(nao));
  TAKE(double, w->T, big);
  TAKE(double, w->maxdiag, 1);
  TAKE(double, w->delta, 1);
  TAKE(int, w->status, 1);
  if (jac) {
    TAKE(double, w->Linv, (size_t)naux * naux);
    TAKE(double, w->m1, (size_t)naux * naux);
    TAKE(double, w->C, big);
    TAKE(double, w->dv, big);
    TAKE(double, w->G, big);
  }
#undef TAKE
}

}  // namespace

}  // namespace dfscf

using namespace dfscf;

extern "C" size_t df_fit_residual_work_bytes(int nao, int naux, int with_jacobian) {
  if (nao <= 0 || naux <= 0) return 0;
  Sizer z;
  FitWork w{};
  fit_layout(nao, naux, with_jacobian != 0, nullptr, &z, &w);
  return z.used;
}

extern "C" int df_fit_residual(const double* ao_xyz, const double* ao_exp, int nao, const double* aux_xyz,
                               const double* aux_exp, int naux, const double* dalpha, int ntheta, double* sigma,
                               double* jac, double* delta, void* work, size_t work_bytes, cudaStream_t s) {
  clear_error();
  DF_REQUIRE(nao > 0 && naux > 0 && ao_xyz && ao_exp && aux_xyz && aux_exp && sigma, DF_ERR_ARG,
             "df_fit_residual: bad arguments");
  const bool want_jac = jac != nullptr;
  DF_REQUIRE(!want_jac || (dalpha && ntheta >= 1 && ntheta <= kMaxTheta), DF_ERR_ARG,
             "df_fit_residual: the Jacobian needs dalpha and 1 <= ntheta <= %d", kMaxTheta);
  const size_t need = df_fit_residual_work_bytes(nao, naux, want_jac);
  DF_REQUIRE(work && work_bytes >= need, DF_ERR_NOMEM, "df_fit_residual: workspace of %zu bytes < %zu", work_bytes,
             need);
  DF_REQUIRE(naux <= 65535, DF_ERR_ARG, "df_fit_residual: naux > 65535");
  Arena a(work, work_bytes);
  FitWork w{};
  fit_layout(nao, naux, want_jac, &a, nullptr, &w);
  const long ld = B_ld(nao), npair = npair_of(nao);
  DF_REQUIRE(ld < (1L << 31), DF_ERR_ARG, "df_fit_residual: too many orbital pairs");
  // metric and its Cholesky factor (pivot check as in df_metric_chol)
  DF_TRY(launch_int2c(aux_xyz, aux_exp, naux, w.L, s));
  DF_TRY(cholesky_inplace(w.L, naux, w.status, w.maxdiag, 1e-14, s));
  int h_status = -1;
  DF_CUDA(cudaMemcpyAsync(&h_status, w.status, sizeof(int), cudaMemcpyDeviceToHost, s));
  DF_CUDA(cudaStreamSynchronize(s));
  DF_REQUIRE(h_status < 0, DF_ERR_NOT_SPD, "df_fit_residual: auxiliary metric not positive definite at pivot %d",
             h_status);
  // T = L^-1 (P|mn), then sigma and Delta
  DF_TRY(launch_int3c(ao_xyz, ao_exp, nao, aux_xyz, aux_exp, naux, w.T, ld, w.pair_tab, s));
  const double* pp = w.pair_tab;
  const double* px = pp + npair;
  const double* py = px + npair;
  const double* pz = py + npair;
  const double* pk = pz + npair;
  DF_TRY(forward_substitution(w.T, ld, ld, w.L, naux, s));
  residual_kernel<<<(unsigned)((npair + 255) / 256), 256, 0, s>>>(pp, pk, npair, w.T, ld, naux, sigma);
  DF_LAUNCHED("residual_kernel");
  delta_kernel<<<1, 1024, 0, s>>>(sigma, nao, w.delta);
  DF_LAUNCHED("delta_kernel");
  if (want_jac) {
    // C = M^-1 (P|mn) = L^-T L^-1 (P|mn): L^-1 explicitly, then C = (L^-1)^T T
    identity_kernel<<<(unsigned)(((long)naux * naux + 255) / 256), 256, 0, s>>>(w.Linv, naux);
    DF_LAUNCHED("identity_kernel");
    DF_TRY(forward_substitution(w.Linv, naux, naux, w.L, naux, s));
    DF_TRY(dgemm(true, false, naux, (int)ld, naux, 1.0, w.Linv, naux, 0, w.T, ld, 0, 0.0, w.C, ld, 0, 1, s, 0, 0));
    dim3 g3((unsigned)((ld + 255) / 256), (unsigned)naux);
    int3c_dexp_kernel<<<g3, 256, 0, s>>>(pp, px, py, pz, pk, npair, ld, aux_xyz, aux_exp, w.dv);
    DF_LAUNCHED("int3c_dexp_kernel");
    dim3 g2((unsigned)((naux + 127) / 128), (unsigned)naux);
    int2c_dexp_kernel<<<g2, 128, 0, s>>>(aux_xyz, aux_exp, naux, w.m1);
    DF_LAUNCHED("int2c_dexp_kernel");
    DF_TRY(dgemm(false, false, naux, (int)ld, naux, 1.0, w.m1, naux, 0, w.C, ld, 0, 0.0, w.G, ld, 0, 1, s, 0, 0));
    jac_theta_kernel<<<(unsigned)((npair + 127) / 128), 128, 0, s>>>(w.C, w.dv, w.G, ld, npair, naux, dalpha, ntheta,
                                                                      jac);
    DF_LAUNCHED("jac_theta_kernel");
  }
  if (delta) {
    DF_CUDA(cudaMemcpyAsync(delta, w.delta, sizeof(double), cudaMemcpyDeviceToHost, s));
    DF_CUDA(cudaStreamSynchronize(s));
  }
  return DF_OK;
}

DF_BOUNDS_READER(bounds_read_dferr)
