/*
 * CPU oracle for density-fitted Hartree-Fock with s-type Gaussians.
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously-correct FP64 loops that the test
 * suite, the package's smoke check and the bench's CPU baseline compare the CUDA path
 * against.  It shares no code, header or constant table with the CUDA library and is
 * never called by the product path.
 *
 * Conventions (all arrays row-major, double precision):
 *   primitive   phi_a(r) = N_a exp(-a |r-A|^2),  N_a = (2a/pi)^(3/4)  (L2-normalised)
 *   packed pair ij = i(i+1)/2 + j for i >= j;  npair = nao(nao+1)/2
 *
 * Paper passages followed (arXiv 2506.06661):
 *   density fitting, Eq. (eq:df:eri) and the metric / whitening equations that follow it
 *     (Section "Density fitting"): (mn|kl) ~ sum_P T_{P,mn} T_{P,kl},
 *     M_PQ = (P|Q) = L L^T,  T_{P,mn} = sum_Q (L^-1)_{PQ} (Q|mn);
 *   Gaussian product theorem (Section "Numba JIT compilation", the overlap example):
 *     theta = a b/(a+b), X_p = (a X_a + b X_b)/(a+b);
 *   the Lehtola diagonal error Delta = sum_mn [(mn|mn) - sum_P T_{P,mn}^2].
 * The closed forms of the s-type integrals are textbook results of the product theorem;
 * the paper does not print them.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846

/* ------------------------------------------------------------------------------------ */
/* Boys function of order zero: F0(t) = int_0^1 exp(-t u^2) du.                          */
/* Closed form 0.5 sqrt(pi/t) erf(sqrt t); below t = 1e-3 the Maclaurin series            */
/* sum_k (-t)^k / (k! (2k+1)), ten terms, avoids 0/0 at t = 0.                            */
/* ------------------------------------------------------------------------------------ */
double oracle_boys_f0(double t) {
  if (t < 1e-3) {
    double term = 1.0, sum = 0.0;
    for (int k = 0; k < 10; ++k) {
      sum += term / (2.0 * k + 1.0);
      term *= -t / (k + 1.0);
    }
    return sum;
  }
  double s = sqrt(t);
  return 0.5 * sqrt(ORACLE_PI / t) * erf(s);
}

void oracle_boys_f0_vec(const double* t, long n, double* out) {
  for (long i = 0; i < n; ++i) out[i] = oracle_boys_f0(t[i]);
}

static double norm_s(double a) { return pow(2.0 * a / ORACLE_PI, 0.75); }

static double dist2(const double* A, const double* B) {
  double dx = A[0] - B[0], dy = A[1] - B[1], dz = A[2] - B[2];
  return dx * dx + dy * dy + dz * dz;
}

/* ------------------------------------------------------------------------------------ */
/* One-electron integrals over normalised s primitives (product theorem: p = a+b,         */
/* mu = ab/p, P = (aA+bB)/p):                                                             */
/*   S_ab = N_a N_b (pi/p)^(3/2) exp(-mu R_AB^2)                                          */
/*   T_ab = mu (3 - 2 mu R_AB^2) S_ab                                                     */
/*   V_ab = - sum_C Z_C N_a N_b (2 pi/p) exp(-mu R_AB^2) F0(p |P-C|^2)                    */
/* ------------------------------------------------------------------------------------ */
void oracle_int1e(const double* xyz, const double* ex, int nao, const double* nuc_xyz, const double* nuc_z,
                  int natm, double* S, double* T, double* V) {
#pragma omp parallel for schedule(dynamic)
  for (int a = 0; a < nao; ++a) {
    for (int b = 0; b < nao; ++b) {
      double ea = ex[a], eb = ex[b];
      double p = ea + eb, mu = ea * eb / p;
      double r2 = dist2(xyz + 3 * a, xyz + 3 * b);
      double nab = norm_s(ea) * norm_s(eb);
      double s = nab * pow(ORACLE_PI / p, 1.5) * exp(-mu * r2);
      double P[3];
      for (int x = 0; x < 3; ++x) P[x] = (ea * xyz[3 * a + x] + eb * xyz[3 * b + x]) / p;
      double v = 0.0;
      for (int c = 0; c < natm; ++c) {
        v -= nuc_z[c] * nab * (2.0 * ORACLE_PI / p) * exp(-mu * r2) * oracle_boys_f0(p * dist2(P, nuc_xyz + 3 * c));
      }
      if (S) S[(size_t)a * nao + b] = s;
      if (T) T[(size_t)a * nao + b] = mu * (3.0 - 2.0 * mu * r2) * s;
      if (V) V[(size_t)a * nao + b] = v;
    }
  }
}

double oracle_nuclear_repulsion(const double* nuc_xyz, const double* nuc_z, int natm) {
  double e = 0.0;
  for (int a = 0; a < natm; ++a)
    for (int b = 0; b < a; ++b) e += nuc_z[a] * nuc_z[b] / sqrt(dist2(nuc_xyz + 3 * a, nuc_xyz + 3 * b));
  return e;
}

/* ------------------------------------------------------------------------------------ */
/* Coulomb metric M_PQ = (chi_P|chi_Q) (two-centre):                                      */
/*   (c|d) = N_c N_d 2 pi^(5/2) / (c d sqrt(c+d)) F0(cd/(c+d) R_CD^2)                     */
/* ------------------------------------------------------------------------------------ */
void oracle_int2c(const double* xyz, const double* ex, int naux, double* M) {
#pragma omp parallel for schedule(dynamic)
  for (int c = 0; c < naux; ++c) {
    for (int d = 0; d < naux; ++d) {
      double ec = ex[c], ed = ex[d];
      double r2 = dist2(xyz + 3 * c, xyz + 3 * d);
      double pre = norm_s(ec) * norm_s(ed) * 2.0 * pow(ORACLE_PI, 2.5) / (ec * ed * sqrt(ec + ed));
      M[(size_t)c * naux + d] = pre * oracle_boys_f0(ec * ed / (ec + ed) * r2);
    }
  }
}

/* ------------------------------------------------------------------------------------ */
/* Three-centre integrals (Q|mn) for packed pairs m >= n:                                 */
/*   (c|ab) = N_c N_a N_b 2 pi^(5/2) / (p c sqrt(p+c)) exp(-mu R_AB^2)                    */
/*            * F0(p c/(p+c) |P-C|^2)                                                     */
/* R is [naux][npair].                                                                    */
/* ------------------------------------------------------------------------------------ */
void oracle_int3c(const double* ao_xyz, const double* ao_ex, int nao, const double* aux_xyz, const double* aux_ex,
                  int naux, double* R) {
  size_t npair = (size_t)nao * (nao + 1) / 2;
#pragma omp parallel for schedule(dynamic)
  for (int q = 0; q < naux; ++q) {
    double ec = aux_ex[q];
    const double* C = aux_xyz + 3 * q;
    for (int a = 0; a < nao; ++a) {
      for (int b = 0; b <= a; ++b) {
        double ea = ao_ex[a], eb = ao_ex[b];
        double p = ea + eb, mu = ea * eb / p;
        double r2 = dist2(ao_xyz + 3 * a, ao_xyz + 3 * b);
        double P[3];
        for (int x = 0; x < 3; ++x) P[x] = (ea * ao_xyz[3 * a + x] + eb * ao_xyz[3 * b + x]) / p;
        double pre = norm_s(ec) * norm_s(ea) * norm_s(eb) * 2.0 * pow(ORACLE_PI, 2.5) / (p * ec * sqrt(p + ec));
        size_t ij = (size_t)a * (a + 1) / 2 + b;
        R[(size_t)q * npair + ij] = pre * exp(-mu * r2) * oracle_boys_f0(p * ec / (p + ec) * dist2(P, C));
      }
    }
  }
}

/* ------------------------------------------------------------------------------------ */
/* Rows of the three-centre tensor: (Q|r n) for the listed orbital rows r and every n,    */
/* out [naux][nrows][nao] (unpacked).  The same closed form as oracle_int3c, evaluated    */
/* with the larger index first so that every value equals the packed one bit for bit;    */
/* it lets tests sample a few rows of B at sizes where the full tensor is too large.      */
/* ------------------------------------------------------------------------------------ */
void oracle_int3c_rows(const double* ao_xyz, const double* ao_ex, int nao, const double* aux_xyz,
                       const double* aux_ex, int naux, const int* rows, int nrows, double* out) {
#pragma omp parallel for schedule(dynamic)
  for (int q = 0; q < naux; ++q) {
    double ec = aux_ex[q];
    const double* C = aux_xyz + 3 * q;
    for (int t = 0; t < nrows; ++t) {
      for (int n = 0; n < nao; ++n) {
        int a = rows[t] > n ? rows[t] : n, b = rows[t] > n ? n : rows[t];
        double ea = ao_ex[a], eb = ao_ex[b];
        double p = ea + eb, mu = ea * eb / p;
        double r2 = dist2(ao_xyz + 3 * a, ao_xyz + 3 * b);
        double P[3];
        for (int x = 0; x < 3; ++x) P[x] = (ea * ao_xyz[3 * a + x] + eb * ao_xyz[3 * b + x]) / p;
        double pre = norm_s(ec) * norm_s(ea) * norm_s(eb) * 2.0 * pow(ORACLE_PI, 2.5) / (p * ec * sqrt(p + ec));
        out[((size_t)q * nrows + t) * nao + n] = pre * exp(-mu * r2) * oracle_boys_f0(p * ec / (p + ec) * dist2(P, C));
      }
    }
  }
}

/* ------------------------------------------------------------------------------------ */
/* Four-centre integrals (ab|cd), full nao^4 tensor (brute-force checks only):            */
/*   (ab|cd) = N_a N_b N_c N_d 2 pi^(5/2) / (p q sqrt(p+q))                               */
/*             exp(-mu_ab R_AB^2) exp(-mu_cd R_CD^2) F0(p q/(p+q) |P-Q|^2)                */
/* ------------------------------------------------------------------------------------ */
void oracle_int4c(const double* xyz, const double* ex, int nao, double* eri) {
  size_t n = (size_t)nao;
#pragma omp parallel for schedule(dynamic)
  for (int a = 0; a < nao; ++a)
    for (int b = 0; b < nao; ++b) {
      double p = ex[a] + ex[b], mab = ex[a] * ex[b] / p;
      double P[3];
      for (int x = 0; x < 3; ++x) P[x] = (ex[a] * xyz[3 * a + x] + ex[b] * xyz[3 * b + x]) / p;
      double kab = norm_s(ex[a]) * norm_s(ex[b]) * exp(-mab * dist2(xyz + 3 * a, xyz + 3 * b));
      for (int c = 0; c < nao; ++c)
        for (int d = 0; d < nao; ++d) {
          double q = ex[c] + ex[d], mcd = ex[c] * ex[d] / q;
          double Q[3];
          for (int x = 0; x < 3; ++x) Q[x] = (ex[c] * xyz[3 * c + x] + ex[d] * xyz[3 * d + x]) / q;
          double kcd = norm_s(ex[c]) * norm_s(ex[d]) * exp(-mcd * dist2(xyz + 3 * c, xyz + 3 * d));
          double val = kab * kcd * 2.0 * pow(ORACLE_PI, 2.5) / (p * q * sqrt(p + q)) *
                       oracle_boys_f0(p * q / (p + q) * dist2(P, Q));
          eri[((a * n + b) * n + c) * n + d] = val;
        }
    }
}

/* ------------------------------------------------------------------------------------ */
/* Textbook Cholesky M = L L^T (lower).  Returns -1 on success, else the index of the     */
/* first pivot that is <= tol * max_i M_ii (the factor is then incomplete).               */
/* ------------------------------------------------------------------------------------ */
int oracle_cholesky(const double* M, int n, double* L, double tol) {
  double dmax = 0.0;
  for (int i = 0; i < n; ++i)
    if (M[(size_t)i * n + i] > dmax) dmax = M[(size_t)i * n + i];
  memset(L, 0, sizeof(double) * (size_t)n * n);
  for (int j = 0; j < n; ++j) {
    double s = M[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) s -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
    if (!(s > tol * dmax)) return j;
    double ljj = sqrt(s);
    L[(size_t)j * n + j] = ljj;
#pragma omp parallel for
    for (int i = j + 1; i < n; ++i) {
      double t = M[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) t -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
      L[(size_t)i * n + j] = t / ljj;
    }
  }
  return -1;
}

/* ------------------------------------------------------------------------------------ */
/* Whitening T = L^-1 R by forward substitution, independently for every column          */
/* (packed pair) of R [naux][ncol]; done in place.                                        */
/* ------------------------------------------------------------------------------------ */
void oracle_whiten(const double* L, int naux, double* R, long ncol) {
#pragma omp parallel for schedule(static)
  for (long c = 0; c < ncol; ++c) {
    for (int p = 0; p < naux; ++p) {
      double s = R[(size_t)p * ncol + c];
      for (int q = 0; q < p; ++q) s -= L[(size_t)p * naux + q] * R[(size_t)q * ncol + c];
      R[(size_t)p * ncol + c] = s / L[(size_t)p * naux + p];
    }
  }
}

/* ------------------------------------------------------------------------------------ */
/* DF Coulomb matrix: d_P = sum_{m>=n} w_mn B_{P,mn} D_mn  (w = 2 off-diagonal, 1 on it)  */
/* and J_mn = sum_P d_P B_{P,mn}; J returned as a full symmetric nao x nao matrix.        */
/* B is packed [naux][npair] (row stride ldb >= npair); D is full and symmetric.          */
/* ------------------------------------------------------------------------------------ */
void oracle_df_j(const double* B, long ldb, int naux, int nao, const double* D, double* J) {
  size_t npair = (size_t)nao * (nao + 1) / 2;
  double* d = (double*)calloc((size_t)naux, sizeof(double));
#pragma omp parallel for
  for (int P = 0; P < naux; ++P) {
    double s = 0.0;
    for (int m = 0; m < nao; ++m)
      for (int n = 0; n <= m; ++n) {
        double w = (m == n) ? 1.0 : 2.0;
        s += w * B[(size_t)P * ldb + (size_t)m * (m + 1) / 2 + n] * D[(size_t)m * nao + n];
      }
    d[P] = s;
  }
#pragma omp parallel for
  for (long ij = 0; ij < (long)npair; ++ij) {
    double s = 0.0;
    for (int P = 0; P < naux; ++P) s += d[P] * B[(size_t)P * ldb + ij];
    /* unpack ij -> (m, n) */
    int m = (int)((sqrt(8.0 * (double)ij + 1.0) - 1.0) / 2.0);
    while ((long)m * (m + 1) / 2 > ij) --m;
    while ((long)(m + 1) * (m + 2) / 2 <= ij) ++m;
    int n = (int)(ij - (long)m * (m + 1) / 2);
    J[(size_t)m * nao + n] = s;
    J[(size_t)n * nao + m] = s;
  }
  free(d);
}

static double packed_at(const double* row, int m, int n) {
  int a = m > n ? m : n, b = m > n ? n : m;
  return row[(size_t)a * (a + 1) / 2 + b];
}

/* ------------------------------------------------------------------------------------ */
/* DF exchange matrix from occupied coefficients C [nao][nocc]:                           */
/*   X_{P,mi} = sum_n B_P[m,n] C_ni,   K_mn = sum_P sum_i X_{P,mi} X_{P,ni}.               */
/* ------------------------------------------------------------------------------------ */
void oracle_df_k(const double* B, long ldb, int naux, int nao, const double* C, int nocc, double* K) {
  memset(K, 0, sizeof(double) * (size_t)nao * nao);
  int nthreads = 1;
#ifdef _OPENMP
  nthreads = omp_get_max_threads();
#endif
  double* Kt = (double*)calloc((size_t)nthreads * nao * nao, sizeof(double));
#pragma omp parallel
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double* X = (double*)malloc(sizeof(double) * (size_t)nao * nocc);
    double* Kl = Kt + (size_t)tid * nao * nao;
#pragma omp for schedule(dynamic)
    for (int P = 0; P < naux; ++P) {
      const double* row = B + (size_t)P * ldb;
      for (int m = 0; m < nao; ++m)
        for (int i = 0; i < nocc; ++i) {
          double s = 0.0;
          for (int n = 0; n < nao; ++n) s += packed_at(row, m, n) * C[(size_t)n * nocc + i];
          X[(size_t)m * nocc + i] = s;
        }
      for (int m = 0; m < nao; ++m)
        for (int n = 0; n < nao; ++n) {
          double s = 0.0;
          for (int i = 0; i < nocc; ++i) s += X[(size_t)m * nocc + i] * X[(size_t)n * nocc + i];
          Kl[(size_t)m * nao + n] += s;
        }
    }
    free(X);
  }
  for (int t = 0; t < nthreads; ++t)
    for (size_t e = 0; e < (size_t)nao * nao; ++e) K[e] += Kt[(size_t)t * nao * nao + e];
  free(Kt);
}

/* Brute-force four-centre J_mn = sum_kl (mn|kl) D_kl and K_mn = sum_kl (mk|nl) P_kl.   */
void oracle_jk_4c(const double* eri, int nao, const double* D, const double* Pm, double* J, double* K) {
  size_t n = (size_t)nao;
  for (size_t m = 0; m < n; ++m)
    for (size_t v = 0; v < n; ++v) {
      double j = 0.0, k = 0.0;
      for (size_t a = 0; a < n; ++a)
        for (size_t b = 0; b < n; ++b) {
          j += eri[((m * n + v) * n + a) * n + b] * D[a * n + b];
          k += eri[((m * n + a) * n + v) * n + b] * Pm[a * n + b];
        }
      J[m * n + v] = j;
      K[m * n + v] = k;
    }
}

/* Diagonal (mn|mn) for packed pairs (same closed form as oracle_int4c with cd = ab).    */
void oracle_eri_diag(const double* xyz, const double* ex, int nao, double* diag) {
#pragma omp parallel for schedule(dynamic)
  for (int a = 0; a < nao; ++a)
    for (int b = 0; b <= a; ++b) {
      double p = ex[a] + ex[b], mab = ex[a] * ex[b] / p;
      double kab = norm_s(ex[a]) * norm_s(ex[b]) * exp(-mab * dist2(xyz + 3 * a, xyz + 3 * b));
      diag[(size_t)a * (a + 1) / 2 + b] = kab * kab * 2.0 * pow(ORACLE_PI, 2.5) / (p * p * sqrt(2.0 * p));
    }
}

/* K[Dm]_mn = sum_P sum_kl B_P[m,k] Dm_kl B_P[l,n] for a general symmetric Dm:            */
/* for every P form T = Dm B_P, then K += B_P T.                                          */
void oracle_df_k_dm(const double* B, long ldb, int naux, int nao, const double* Dm, double* K) {
  memset(K, 0, sizeof(double) * (size_t)nao * nao);
  double* T = (double*)malloc(sizeof(double) * (size_t)nao * nao);
  for (int P = 0; P < naux; ++P) {
    const double* row = B + (size_t)P * ldb;
#pragma omp parallel for
    for (int k = 0; k < nao; ++k)
      for (int n = 0; n < nao; ++n) {
        double t = 0.0;
        for (int l = 0; l < nao; ++l) t += Dm[(size_t)k * nao + l] * packed_at(row, l, n);
        T[(size_t)k * nao + n] = t;
      }
#pragma omp parallel for
    for (int m = 0; m < nao; ++m)
      for (int n = 0; n < nao; ++n) {
        double s = 0.0;
        for (int k = 0; k < nao; ++k) s += packed_at(row, m, k) * T[(size_t)k * nao + n];
        K[(size_t)m * nao + n] += s;
      }
  }
  free(T);
}
