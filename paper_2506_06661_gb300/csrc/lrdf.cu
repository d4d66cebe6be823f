// Long-range density fitting (LRDF) for J and K (arXiv 2506.06661, Section "Density
// fitting", the LRDF paragraphs):
//   1/r = erf(w r)/r + erfc(w r)/r,
//   (mn|kl) ~ (mn|kl)^SR + sum_P T_{P,mn} T_{P,kl},  M^LR = L L^T,  T = L^-1 (Q|mn)^LR.
// The long-range tensor T uses the ordinary B layout (FP64 packed rows), so df_jk builds its
// J and K; the short-range part is computed exactly here by direct four-centre kernels.
// For s primitives with pair exponents p, q (rho = pq/(p+q)) and pair factors
// K_ab = N_a N_b exp(-ab/p R_AB^2) 2 pi^(5/2) / p (the pair table of launch_int3c):
//   (ab|cd)       = K_ab K_cd / (2 pi^(5/2) sqrt(p + q)) F0(rho R^2),
//   (ab|cd)^LR    = the same with sqrt(f) F0(f rho R^2), f = w^2 / (rho + w^2),
//   (ab|cd)^SR    = (ab|cd) - (ab|cd)^LR
//                 = K_ab K_cd / (2 pi^(5/2) sqrt(p + q)) (sqrt(pi)/2) [erfc(sqrt(f rho) R) -
//                   erfc(sqrt(rho) R)] / (sqrt(rho) R)   for rho R^2 >= 1e-3,
// which keeps its accuracy where both terms are nearly equal (large R); below 1e-3 the two
// Boys values come from their series.  Quartets whose pair factors multiply to less than
// 1e-16 of the largest are skipped (their integrals are below that times the largest).
#include <cmath>

#include "boys.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace dfscf {

namespace {

constexpr int LR_TILE = 256;

__device__ __forceinline__ double sr_kernel(double p, double q, double R2, double omega) {
  const double rho = p * q / (p + q);
  const double f = omega * omega / (rho + omega * omega);
  const double x = rho * R2;
  if (x < 1e-3) return boys_f0(x) - sqrt(f) * boys_f0(f * x);
  const double R = sqrt(R2), sr = sqrt(rho);
  return 0.88622692545275801365 * (erfc(sqrt(f) * sr * R) - erfc(sr * R)) / (sr * R);
}

// Jsr[ij] = sum_kl w_kl D_kl (ij|kl)^SR over packed pairs (w = 2 off the diagonal); one lane
// per pair ij, the kl pairs streamed through shared memory in tiles.
__global__ void __launch_bounds__(LR_TILE) jsr_kernel(const double* __restrict__ pp, const double* __restrict__ px,
                                                      const double* __restrict__ py, const double* __restrict__ pz,
                                                      const double* __restrict__ pk, const double* __restrict__ Dw,
                                                      long npair, double omega, double cut,
                                                      double* __restrict__ J) {
  __shared__ double sp[LR_TILE], sx[LR_TILE], sy[LR_TILE], sz[LR_TILE], sk[LR_TILE];
  const long ij = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = ij < npair;
  const double p = live ? pp[ij] : 1.0, x = live ? px[ij] : 0.0, y = live ? py[ij] : 0.0, z = live ? pz[ij] : 0.0;
  const double k1 = live ? pk[ij] : 0.0;
  double acc = 0.0;
  for (long t0 = 0; t0 < npair; t0 += LR_TILE) {
    __syncthreads();
    const long kl = t0 + threadIdx.x;
    if (kl < npair) {
      sp[threadIdx.x] = pp[kl];
      sx[threadIdx.x] = px[kl];
      sy[threadIdx.x] = py[kl];
      sz[threadIdx.x] = pz[kl];
      sk[threadIdx.x] = pk[kl] * Dw[kl];
    }
    __syncthreads();
    const int n = (int)min((long)LR_TILE, npair - t0);
    for (int u = 0; u < n; ++u) {
      const double kk = k1 * sk[u];
      if (fabs(kk) < cut) continue;
      const double q = sp[u], dx = x - sx[u], dy = y - sy[u], dz = z - sz[u];
      acc += kk / sqrt(p + q) * sr_kernel(p, q, dx * dx + dy * dy + dz * dz, omega);
    }
  }
  if (live) J[ij] = acc * (1.0 / (2.0 * kPi * kPi * sqrt(kPi)));
}

__device__ __forceinline__ long pair_index(int a, int b) {
  return a >= b ? (long)a * (a + 1) / 2 + b : (long)b * (b + 1) / 2 + a;
}

// Ksr[m][n] = sum_kl (mk|nl)^SR Pm_kl for m >= n (mirrored); one CTA per (m, n) pair, lanes
// over k, a loop over l.
__global__ void __launch_bounds__(128) ksr_kernel(const double* __restrict__ pp, const double* __restrict__ px,
                                                  const double* __restrict__ py, const double* __restrict__ pz,
                                                  const double* __restrict__ pk, const double* __restrict__ Pm,
                                                  int nao, double omega, double pkmax, double cut,
                                                  double* __restrict__ K) {
  __shared__ double sh[32];
  long mn = blockIdx.x;
  int m, n;
  unpack_pair(mn, m, n);
  double acc = 0.0;
  for (int k = threadIdx.x; k < nao; k += blockDim.x) {
    const long a = DF_IX(pair_index(m, k), (long)nao * (nao + 1) / 2);
    const double p = pp[a], ka = pk[a];
    if (fabs(ka) * pkmax < cut) continue;  // no pair (n, l) can lift this one above the cut
    const double xa = px[a], ya = py[a], za = pz[a];
    for (int l = 0; l < nao; ++l) {
      const long b = DF_IX(pair_index(n, l), (long)nao * (nao + 1) / 2);
      const double kk = ka * pk[b] * Pm[DF_IX((size_t)k * nao + l, (size_t)nao * nao)];
      if (fabs(ka * pk[b]) < cut) continue;
      const double q = pp[b], dx = xa - px[b], dy = ya - py[b], dz = za - pz[b];
      acc += kk / sqrt(p + q) * sr_kernel(p, q, dx * dx + dy * dy + dz * dz, omega);
    }
  }
  acc = block_sum(acc, sh) * (1.0 / (2.0 * kPi * kPi * sqrt(kPi)));
  if (threadIdx.x == 0) {
    K[(size_t)m * nao + n] = acc;
    K[(size_t)n * nao + m] = acc;
  }
}

// Dw_mn = w_mn (D_mn + D_nm)/2 over packed pairs (w = 2 off the diagonal).
__global__ void lr_weighted_density_kernel(const double* __restrict__ D, int nao, long npair, double* __restrict__ Dw) {
  const long ij = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (ij >= npair) return;
  int m, n;
  unpack_pair(ij, m, n);
  Dw[ij] = (m == n ? 1.0 : 2.0) * 0.5 * (D[(size_t)m * nao + n] + D[(size_t)n * nao + m]);
}

// J = Jsr unpacked + Jlr (in place: J holds Jlr on entry).
__global__ void add_packed_kernel(const double* __restrict__ Jsr, int nao, double* __restrict__ J) {
  const long ij = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (ij >= (long)nao * (nao + 1) / 2) return;
  int m, n;
  unpack_pair(ij, m, n);
  J[(size_t)m * nao + n] += Jsr[ij];
  if (m != n) J[(size_t)n * nao + m] += Jsr[ij];
}

__global__ void add_kernel(double* __restrict__ y, const double* __restrict__ x, long n) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += x[i];
}

__global__ void absmax_pk_kernel(const double* __restrict__ pk, long n, double* __restrict__ out) {
  __shared__ double sh[32];
  double m = 0.0;
  for (long i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(pk[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = fmax(t, sh[i]);
    *out = t;
  }
}

struct LrWork {
  double *pair_tab, *Dw, *Jsr, *Pm, *Ksr, *pkmax;
};

void lr_layout(int nao, Arena* a, Sizer* z, LrWork* w) {
  const long np = npair_of(nao);
  const size_t nn = (size_t)nao * nao;
#define TAKE(T_, ptr, count) \
  if (a) ptr = a->take<T_>(count); else z->take<T_>(count);
  TAKE(double, w->pair_tab, 5 * (size_t)np);
  TAKE(double, w->Dw, np);
  TAKE(double, w->Jsr, np);
  TAKE(double, w->Pm, nn);
  TAKE(double, w->Ksr, nn);
  TAKE(double, w->pkmax, 1);
#undef TAKE
}

}  // namespace
}  // namespace dfscf

using namespace dfscf;

extern "C" size_t df_lrdf_build_work_bytes(int nao, int naux) {
  if (nao <= 0 || naux <= 0) return 0;
  Sizer z;
  z.take<double>((size_t)naux * naux);
  z.take<int>(1);
  z.take<double>(1);
  z.take<double>(5 * (size_t)npair_of(nao));
  return z.used;
}

extern "C" int df_lrdf_build(const double* ao_xyz, const double* ao_exp, int nao, const double* aux_xyz,
                             const double* aux_exp, int naux, double omega, void* B, size_t B_bytes, void* work,
                             size_t work_bytes, cudaStream_t s) {
  clear_error();
  DF_REQUIRE(nao > 0 && naux > 0 && ao_xyz && ao_exp && aux_xyz && aux_exp && B, DF_ERR_ARG,
             "df_lrdf_build: bad arguments");
  DF_REQUIRE(omega > 0.0 && std::isfinite(omega), DF_ERR_ARG, "df_lrdf_build: omega must be positive and finite");
  DF_REQUIRE(B_bytes >= df_B_bytes(nao, naux, DF_FP64), DF_ERR_NOMEM, "df_lrdf_build: B buffer of %zu bytes < %zu",
             B_bytes, df_B_bytes(nao, naux, DF_FP64));
  DF_REQUIRE(work && work_bytes >= df_lrdf_build_work_bytes(nao, naux), DF_ERR_NOMEM,
             "df_lrdf_build: workspace too small");
  Arena a(work, work_bytes);
  double* L = a.take<double>((size_t)naux * naux);
  int* status = a.take<int>(1);
  double* maxdiag = a.take<double>(1);
  double* pair_tab = a.take<double>(5 * (size_t)npair_of(nao));
  DF_TRY(launch_int2c(aux_xyz, aux_exp, naux, L, s, omega));
  DF_TRY(cholesky_inplace(L, naux, status, maxdiag, 1e-14, s));
  int h = -1;
  DF_CUDA(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s));
  DF_CUDA(cudaStreamSynchronize(s));
  DF_REQUIRE(h < 0, DF_ERR_NOT_SPD, "df_lrdf_build: long-range metric not positive definite at pivot %d", h);
  const long ld = B_ld(nao);
  double* B64 = (double*)B;
  DF_TRY(launch_int3c(ao_xyz, ao_exp, nao, aux_xyz, aux_exp, naux, B64, ld, pair_tab, s, omega));
  DF_TRY(forward_substitution(B64, ld, ld, L, naux, s));
  return DF_OK;
}

extern "C" size_t df_lrdf_jk_work_bytes(int nao, int naux, int nocc) {
  if (nao <= 0 || naux <= 0 || nocc < 0) return 0;
  Sizer z;
  LrWork w{};
  lr_layout(nao, nullptr, &z, &w);
  return z.used + df_jk_work_bytes(nao, naux, nocc, DF_FP64) + 256;
}

extern "C" int df_lrdf_jk(const void* B_lr, const double* ao_xyz, const double* ao_exp, int nao, int naux, double omega,
                          const double* D, const double* C, int nocc, double* J, double* K, void* work,
                          size_t work_bytes, cudaStream_t s) {
  clear_error();
  DF_REQUIRE(B_lr && ao_xyz && ao_exp && nao > 0 && naux > 0, DF_ERR_ARG, "df_lrdf_jk: bad arguments");
  DF_REQUIRE(omega > 0.0 && std::isfinite(omega), DF_ERR_ARG, "df_lrdf_jk: omega must be positive and finite");
  DF_REQUIRE(!J || D, DF_ERR_ARG, "df_lrdf_jk: J requested without D");
  DF_REQUIRE(!K || (C && nocc > 0), DF_ERR_ARG, "df_lrdf_jk: K requested without C / nocc");
  DF_REQUIRE(work && work_bytes >= df_lrdf_jk_work_bytes(nao, naux, nocc), DF_ERR_NOMEM,
             "df_lrdf_jk: workspace too small");
  Arena a(work, work_bytes);
  LrWork w{};
  lr_layout(nao, &a, nullptr, &w);
  void* jkw = (char*)work + align_up(a.used, 256);
  const size_t jkw_bytes = work_bytes - align_up(a.used, 256);
  // long-range part: ordinary DF J/K on the long-range tensor
  DF_TRY(df_jk(B_lr, nao, naux, DF_FP64, D, C, nocc, J, K, jkw, jkw_bytes, s));
  clear_error();
  // short-range part: direct four-centre sums over the orbital pair table
  const long np = npair_of(nao), nn = (long)nao * nao;
  double* pp = w.pair_tab;
  DF_TRY(launch_pair_table(ao_xyz, ao_exp, nao, w.pair_tab, s));
  absmax_pk_kernel<<<1, 1024, 0, s>>>(pp + 4 * np, np, w.pkmax);
  DF_LAUNCHED("absmax_pk_kernel");
  double pkmax = 0.0;
  DF_CUDA(cudaMemcpyAsync(&pkmax, w.pkmax, sizeof(double), cudaMemcpyDeviceToHost, s));
  DF_CUDA(cudaStreamSynchronize(s));
  const double cut = 1e-16 * pkmax * pkmax;
  if (J) {
    lr_weighted_density_kernel<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(D, nao, np, w.Dw);
    DF_LAUNCHED("lr_weighted_density_kernel");
    jsr_kernel<<<(unsigned)((np + LR_TILE - 1) / LR_TILE), LR_TILE, 0, s>>>(pp, pp + np, pp + 2 * np, pp + 3 * np,
                                                                           pp + 4 * np, w.Dw, np, omega, cut, w.Jsr);
    DF_LAUNCHED("jsr_kernel");
    add_packed_kernel<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(w.Jsr, nao, J);
    DF_LAUNCHED("add_packed_kernel");
  }
  if (K) {
    DF_TRY(dgemm(false, true, nao, nao, nocc, 1.0, C, nocc, 0, C, nocc, 0, 0.0, w.Pm, nao, 0, 1, s, 0, 0));
    DF_REQUIRE(np < (1L << 31), DF_ERR_ARG, "df_lrdf_jk: too many orbital pairs");
    ksr_kernel<<<(unsigned)np, 128, 0, s>>>(pp, pp + np, pp + 2 * np, pp + 3 * np, pp + 4 * np, w.Pm, nao, omega,
                                             pkmax, cut, w.Ksr);
    DF_LAUNCHED("ksr_kernel");
    add_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(K, w.Ksr, nn);
    DF_LAUNCHED("add_kernel");
  }
  return DF_OK;
}

DF_BOUNDS_READER(bounds_read_lrdf)
