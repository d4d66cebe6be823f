// FP64 symmetric eigensolver for the SCF (orthogonalisation of S and the Fock
// diagonalisation F'C' = C' eps).  One CTA per matrix, so a batch of molecules is one
// launch with one CTA each:
//   1. Householder reduction A -> Q^T A Q = tridiag(d, e), reflectors kept in A;
//   2. explicit Q by backward accumulation of the reflectors;
//   3. implicit QL iterations with Wilkinson shifts on (d, e); each sweep's Givens
//      rotations are generated serially by one lane and applied by all lanes to the
//      eigenvector rows (vectors stored as rows, so the updates are coalesced);
//   4. ascending sort of (eigenvalue, vector).
// All three phases are textbook algorithms (Householder 1958; QL with implicit shifts as
// in Bowdler, Martin, Reinsch and Wilkinson 1968) written here for a thread block.
#include <cfloat>

#include "common.cuh"
#include "kernels.cuh"

namespace dfscf {

struct EigShared {
  double red[32];
  double scal[4];
  int flag;
};

__device__ double cta_sum(double v, EigShared& sh) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh.red[wid] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < nw; ++i) t += sh.red[i];
  __syncthreads();
  return t;
}

// Householder reduction of the symmetric A [n][n] (full storage) to tridiag(d, e): reflector
// k (k = 0..n-3) is H_k = I - beta[k] v v^T with v stored in column k below the diagonal.
__device__ void tridiagonalize_cta(double* __restrict__ A, int n, double* __restrict__ d, double* __restrict__ e,
                                   double* __restrict__ beta, double* __restrict__ v, double* __restrict__ cs,
                                   double* __restrict__ sn, EigShared& sh) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int k = 0; k + 2 < n; ++k) {
    int len = n - k - 1;                      // x = A[k+1..n)[k]
    double part = 0.0;
    for (int i = tid + 1; i < len; i += nt) {
      double x = A[(size_t)(k + 1 + i) * n + k];
      part += x * x;
    }
    double sigma = cta_sum(part, sh);         // sum of x_1..x_{len-1} squared
    double x0 = A[(size_t)(k + 1) * n + k];
    double alpha, b;
    if (sigma == 0.0) {
      alpha = x0;
      b = 0.0;
    } else {
      double nrm = sqrt(x0 * x0 + sigma);
      alpha = (x0 >= 0.0) ? -nrm : nrm;
      double v0 = x0 - alpha;
      b = 2.0 / (v0 * v0 + sigma);
    }
    for (int i = tid; i < len; i += nt) v[i] = (i == 0) ? (x0 - alpha) : A[(size_t)(k + 1 + i) * n + k];
    __syncthreads();
    d[k] = A[(size_t)k * n + k];
    e[k] = alpha;
    if (tid == 0) beta[k] = b;
    if (b != 0.0) {
      // p = b * A22 v  (one warp per row)
      int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
      for (int i = wid; i < len; i += nw) {
        const double* row = A + (size_t)(k + 1 + i) * n + k + 1;
        double s = 0.0;
        for (int j = lane; j < len; j += 32) s += row[j] * v[j];
        s = warp_sum(s);
        if (lane == 0) cs[i] = b * s;
      }
      __syncthreads();
      double pv = 0.0;
      for (int i = tid; i < len; i += nt) pv += cs[i] * v[i];
      double K = 0.5 * b * cta_sum(pv, sh);
      for (int i = tid; i < len; i += nt) sn[i] = cs[i] - K * v[i];  // w
      __syncthreads();
      for (long q = tid; q < (long)len * len; q += nt) {
        int i = (int)(q / len), j = (int)(q % len);
        A[(size_t)(k + 1 + i) * n + k + 1 + j] -= v[i] * sn[j] + sn[i] * v[j];
      }
    }
    // keep the reflector in column k below the diagonal
    for (int i = tid; i < len; i += nt) A[(size_t)(k + 1 + i) * n + k] = v[i];
    __syncthreads();
  }
  if (n >= 2) {
    if (tid == 0) {
      d[n - 2] = A[(size_t)(n - 2) * n + n - 2];
      e[n - 2] = A[(size_t)(n - 1) * n + n - 2];
    }
  }
  if (tid == 0) {
    d[n - 1] = A[(size_t)(n - 1) * n + n - 1];
    e[n - 1] = 0.0;
  }
  __syncthreads();
}

// A [n][n] symmetric (full storage), overwritten.  Outputs w [n] ascending and
// ZT [n][n] with eigenvector k in row k.  Scratch: d, e, beta, v (n each), cs, sn (n each).
__device__ int eigh_cta(double* __restrict__ A, int n, double* __restrict__ w, double* __restrict__ ZT,
                        double* __restrict__ d, double* __restrict__ e, double* __restrict__ beta,
                        double* __restrict__ v, double* __restrict__ cs, double* __restrict__ sn, EigShared& sh) {
  const int tid = threadIdx.x, nt = blockDim.x;
  // ---- 1. tridiagonalisation --------------------------------------------------------
  tridiagonalize_cta(A, n, d, e, beta, v, cs, sn, sh);
  // ---- 2. Q = H_0 H_1 ... H_{n-3}, built as rows ZT = Q^T -----------------------------
  // Work on Q directly in ZT's storage as Q[i][j] = ZT[j][i] would be strided; instead build
  // Q (row-major) and transpose in place at the end of this phase.
  for (long q = tid; q < (long)n * n; q += nt) ZT[q] = ((q / n) == (q % n)) ? 1.0 : 0.0;
  __syncthreads();
  for (int k = n - 3; k >= 0; --k) {
    double b = beta[k];
    if (b == 0.0) continue;
    int len = n - k - 1;
    // u_j = b * sum_i v_i Q[k+1+i][k+1+j]
    for (int j = tid; j < len; j += nt) {
      double s = 0.0;
      for (int i = 0; i < len; ++i) s += A[(size_t)(k + 1 + i) * n + k] * ZT[(size_t)(k + 1 + i) * n + k + 1 + j];
      cs[j] = b * s;
    }
    __syncthreads();
    for (long q = tid; q < (long)len * len; q += nt) {
      int i = (int)(q / len), j = (int)(q % len);
      ZT[(size_t)(k + 1 + i) * n + k + 1 + j] -= A[(size_t)(k + 1 + i) * n + k] * cs[j];
    }
    __syncthreads();
  }
  // transpose Q -> rows are the columns of Q
  for (long q = tid; q < (long)n * n; q += nt) {
    int i = (int)(q / n), j = (int)(q % n);
    if (j > i) {
      double t = ZT[(size_t)i * n + j];
      ZT[(size_t)i * n + j] = ZT[(size_t)j * n + i];
      ZT[(size_t)j * n + i] = t;
    }
  }
  __syncthreads();
  // ---- 3. implicit QL ---------------------------------------------------------------
  // An off-diagonal element is negligible when it is below eps relative to its two
  // diagonal neighbours, or below eps relative to the whole matrix (needed for clusters of
  // zero eigenvalues, where the neighbours themselves vanish).
  if (tid == 0) {
    double t = 0.0;
    for (int i = 0; i < n; ++i) t = fmax(t, fabs(d[i]) + fabs(e[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0));
    sh.scal[3] = t;
  }
  __syncthreads();
  const double tnorm = sh.scal[3];
  int fail = 0;
  for (int l = 0; l < n; ++l) {
    int iter = 0;
    while (true) {
      // lane 0 runs the scalar recurrence of one sweep and records its rotations
      if (tid == 0) {
        int m = l;
        for (; m < n - 1; ++m) {
          double dd = fabs(d[m]) + fabs(d[m + 1]);
          if (fabs(e[m]) <= DBL_EPSILON * dd || fabs(e[m]) <= DBL_EPSILON * tnorm) break;
        }
        int lo = l, hi = l - 1;   // rotations cs/sn[i] for i in [lo, hi], applied from hi down to lo
        if (m != l) {
          if (iter++ >= 60) {
            sh.flag = -1;
          } else {
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double r = hypot(g, 1.0);
            g = d[m] - d[l] + e[l] / (g + copysign(r, g));
            double s = 1.0, c = 1.0, p = 0.0;
            int i = m - 1;
            bool early = false;
            for (; i >= l; --i) {
              double f = s * e[i], bb = c * e[i];
              r = hypot(f, g);
              e[i + 1] = r;
              if (r == 0.0) {
                d[i + 1] -= p;
                e[m] = 0.0;
                early = true;
                break;
              }
              s = f / r;
              c = g / r;
              g = d[i + 1] - p;
              r = (d[i] - g) * s + 2.0 * c * bb;
              p = s * r;
              d[i + 1] = g + p;
              g = c * r - bb;
              cs[i] = c;
              sn[i] = s;
            }
            lo = early ? i + 1 : l;
            hi = m - 1;
            if (!early) {
              d[l] -= p;
              e[l] = g;
              e[m] = 0.0;
            }
            sh.flag = 1;
          }
        } else {
          sh.flag = 0;
        }
        sh.scal[0] = lo;
        sh.scal[1] = hi;
      }
      __syncthreads();
      int flag = sh.flag;
      int lo = (int)sh.scal[0], hi = (int)sh.scal[1];
      __syncthreads();
      if (flag == 0) break;
      if (flag < 0) {
        fail = 1;
        break;
      }
      // apply rotations hi, hi-1, ..., lo to vector rows (i, i+1), element-parallel
      // (the updated row i is the next rotation's row i+1: carry it in a register)
      for (int col = tid; col < n; col += nt) {
        if (hi < lo) break;
        double carry = ZT[(size_t)(hi + 1) * n + col];
        for (int i = hi; i >= lo; --i) {
          double zi = ZT[(size_t)i * n + col];
          double c = cs[i], s_ = sn[i];
          ZT[(size_t)(i + 1) * n + col] = s_ * zi + c * carry;
          carry = c * zi - s_ * carry;
        }
        ZT[(size_t)lo * n + col] = carry;
      }
      __syncthreads();
    }
    if (fail) break;
  }
  if (fail) return 1;
  // ---- 4. ascending selection sort --------------------------------------------------
  for (int i = 0; i < n - 1; ++i) {
    if (tid == 0) {
      int kmin = i;
      for (int j = i + 1; j < n; ++j)
        if (d[j] < d[kmin]) kmin = j;
      sh.scal[2] = kmin;
      if (kmin != i) {
        double t = d[i];
        d[i] = d[kmin];
        d[kmin] = t;
      }
    }
    __syncthreads();
    int kmin = (int)sh.scal[2];
    if (kmin != i) {
      for (int c = tid; c < n; c += nt) {
        double t = ZT[(size_t)i * n + c];
        ZT[(size_t)i * n + c] = ZT[(size_t)kmin * n + c];
        ZT[(size_t)kmin * n + c] = t;
      }
    }
    __syncthreads();
  }
  for (int i = tid; i < n; i += nt) w[i] = d[i];
  __syncthreads();
  return 0;
}

__global__ void __launch_bounds__(1024) eigh_batched_kernel(double* A, int n, long sA, double* w, long sw, double* ZT,
                                                            long sZ, double* scratch, long sS, int* status) {
  __shared__ EigShared sh;
  int b = blockIdx.x;
  double* s = scratch + (size_t)b * sS;
  int rc = eigh_cta(A + (size_t)b * sA, n, w + (size_t)b * sw, ZT + (size_t)b * sZ, s, s + n, s + 2 * n, s + 3 * n,
                    s + 4 * n, s + 5 * n, sh);
  if (threadIdx.x == 0 && status) status[b] = rc;
}

// ---- k lowest eigenpairs --------------------------------------------------------------------
// The SCF needs only the occupied orbitals and the LUMO.  After the same Householder
// reduction, eigenvalues come from Sturm-sequence bisection (one lane per eigenvalue),
// eigenvectors of the tridiagonal matrix from inverse iteration with a partially pivoted
// LU of T - lambda I (one lane per vector), then the reflectors are applied to those k
// vectors only (one warp per vector) and the vectors are re-orthonormalised by classical
// Gram-Schmidt applied twice.  Cost O(n^3) for the reduction plus O(n^2 k), instead of the
// O(n^3) vector updates of the full QL sweep.

// Eigenvalues of tridiag(d, e) that are < x (count of negative pivots of T - x I).
__device__ int sturm_count(const double* __restrict__ d, const double* __restrict__ e, int n, double x,
                           double pivmin) {
  int c = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  c += q < 0.0;
  for (int i = 1; i < n; ++i) {
    q = d[i] - x - e[i - 1] * e[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    c += q < 0.0;
  }
  return c;
}

// Lane t: inverse iteration for eigenvalue lam of tridiag(d, e) into x (interleaved
// storage: element i of lane t at [i * kk + t]).  dl, dd, du, du2, pv: LU workspace.
__device__ bool inverse_iteration(const double* __restrict__ d, const double* __restrict__ e, int n, double lam,
                                  double tnorm, int t, int kk, double* __restrict__ dl, double* __restrict__ dd,
                                  double* __restrict__ du, double* __restrict__ du2, double* __restrict__ pv,
                                  double* __restrict__ x) {
#define IX(a, i) a[(size_t)(i) * kk + t]
  const double small = DBL_EPSILON * tnorm + 1e-300;
  // LU with partial pivoting of T - lam I (rows i, i+1 interchanged when |sub| > |diag|)
  for (int i = 0; i < n; ++i) {
    IX(dd, i) = d[i] - lam;
    if (i + 1 < n) {
      IX(dl, i) = e[i];
      IX(du, i) = e[i];
    }
    if (i + 2 < n) IX(du2, i) = 0.0;
  }
  for (int i = 0; i + 1 < n; ++i) {
    double di = IX(dd, i), li = IX(dl, i);
    if (fabs(di) >= fabs(li)) {
      IX(pv, i) = 0.0;
      double f = (di != 0.0) ? li / di : 0.0;
      IX(dl, i) = f;
      IX(dd, i + 1) -= f * IX(du, i);
    } else {
      IX(pv, i) = 1.0;
      double f = di / li;
      IX(dd, i) = li;
      IX(dl, i) = f;
      double tmp = IX(du, i);
      IX(du, i) = IX(dd, i + 1);
      IX(dd, i + 1) = tmp - f * IX(dd, i + 1);
      if (i + 2 < n) {
        IX(du2, i) = IX(du, i + 1);
        IX(du, i + 1) = -f * IX(du, i + 1);
      }
    }
  }
  for (int i = 0; i < n; ++i)
    if (fabs(IX(dd, i)) < small) IX(dd, i) = copysign(small, IX(dd, i) == 0.0 ? 1.0 : IX(dd, i));
  // deterministic start vector with all components non-zero
  for (int i = 0; i < n; ++i) IX(x, i) = 1.0 + 0.5 * sin(0.7 * i + 1.3 * t + 0.1);
  for (int it = 0; it < 4; ++it) {
    for (int i = 0; i + 1 < n; ++i) {
      if (IX(pv, i) == 0.0) {
        IX(x, i + 1) -= IX(dl, i) * IX(x, i);
      } else {
        double tmp = IX(x, i);
        IX(x, i) = IX(x, i + 1);
        IX(x, i + 1) = tmp - IX(dl, i) * IX(x, i + 1);
      }
    }
    IX(x, n - 1) /= IX(dd, n - 1);
    if (n >= 2) IX(x, n - 2) = (IX(x, n - 2) - IX(du, n - 2) * IX(x, n - 1)) / IX(dd, n - 2);
    for (int i = n - 3; i >= 0; --i)
      IX(x, i) = (IX(x, i) - IX(du, i) * IX(x, i + 1) - IX(du2, i) * IX(x, i + 2)) / IX(dd, i);
    double mx = 0.0;
    for (int i = 0; i < n; ++i) mx = fmax(mx, fabs(IX(x, i)));
    if (!(mx > 0.0) || !isfinite(mx)) return false;
    double s2 = 0.0;
    for (int i = 0; i < n; ++i) {
      double v = IX(x, i) / mx;
      IX(x, i) = v;
      s2 += v * v;
    }
    double inv = 1.0 / sqrt(s2);
    for (int i = 0; i < n; ++i) IX(x, i) *= inv;
  }
  return true;
#undef IX
}

// A [n][n] (destroyed); outputs w [k] ascending and ZT [k][n] (eigenvector rows).
// Scratch: 4 n + 6 n k doubles.  Returns 0 on success.
__device__ int eigh_lowest_cta(double* __restrict__ A, int n, int k, double* __restrict__ w, double* __restrict__ ZT,
                               double* __restrict__ scr, EigShared& sh) {
  const int tid = threadIdx.x, nt = blockDim.x;
  double* d = scr;
  double* e = d + n;
  double* beta = e + n;
  double* v = beta + n;
  double* lu = v + n;  // 6 n k
  tridiagonalize_cta(A, n, d, e, beta, v, lu, lu + n, sh);
  // reflector k into row k of the (now unused) upper triangle, for coalesced reads
  for (long q = tid; q < (long)n * n; q += nt) {
    int i = (int)(q / n), j = (int)(q % n);
    if (j > i + 0) A[(size_t)i * n + j] = A[(size_t)j * n + i];
  }
  if (tid == 0) sh.flag = 0;
  __syncthreads();
  // Gershgorin interval and ||T||
  double glo = INFINITY, ghi = -INFINITY, emax2 = 0.0;
  for (int i = 0; i < n; ++i) {
    double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0);
    glo = fmin(glo, d[i] - r);
    ghi = fmax(ghi, d[i] + r);
    if (i + 1 < n) emax2 = fmax(emax2, e[i] * e[i]);
  }
  const double tnorm = fmax(fabs(glo), fabs(ghi));
  const double pivmin = DBL_MIN * fmax(1.0, emax2);
  double* x = lu + 5 * (size_t)n * k;
  for (int t = tid; t < k; t += nt) {
    double lo = glo - 2.0 * DBL_EPSILON * tnorm, hi = ghi + 2.0 * DBL_EPSILON * tnorm;
    for (int it = 0; it < 200; ++it) {
      double mid = 0.5 * (lo + hi);
      if (sturm_count(d, e, n, mid, pivmin) > t) hi = mid;
      else lo = mid;
      if (hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + pivmin) break;
    }
    double lam = 0.5 * (lo + hi);
    w[t] = lam;
    bool ok = inverse_iteration(d, e, n, lam, tnorm, t, k, lu, lu + (size_t)n * k, lu + 2 * (size_t)n * k,
                                lu + 3 * (size_t)n * k, lu + 4 * (size_t)n * k, x);
    if (!ok) atomicExch(&sh.flag, 1);
  }
  __syncthreads();
  if (sh.flag) return 1;
  // back-transform: z <- H_0 H_1 ... H_{n-3} z, one warp per vector
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  for (int t = wid; t < k; t += nw) {
    double* z = ZT + (size_t)t * n;
    for (int i = lane; i < n; i += 32) z[i] = x[(size_t)i * k + t];
    __syncwarp();
    for (int r = n - 3; r >= 0; --r) {
      double b = beta[r];
      if (b == 0.0) continue;
      const double* vr = A + (size_t)r * n + r + 1;
      double s = 0.0;
      for (int i = lane; i < n - r - 1; i += 32) s += vr[i] * z[r + 1 + i];
      s = b * warp_sum(s);
      for (int i = lane; i < n - r - 1; i += 32) z[r + 1 + i] -= s * vr[i];
      __syncwarp();
    }
  }
  __syncthreads();
  // classical Gram-Schmidt, twice, row by row; coefficients in lu (k doubles)
  double* coef = lu;
  for (int a = 0; a < k; ++a) {
    double* za = ZT + (size_t)a * n;
    for (int pass = 0; pass < 2; ++pass) {
      for (int b = wid; b < a; b += nw) {
        const double* zb = ZT + (size_t)b * n;
        double s = 0.0;
        for (int i = lane; i < n; i += 32) s += zb[i] * za[i];
        s = warp_sum(s);
        if (lane == 0) coef[b] = s;
      }
      __syncthreads();
      for (int i = tid; i < n; i += nt) {
        double s = za[i];
        for (int b = 0; b < a; ++b) s -= coef[b] * ZT[(size_t)b * n + i];
        za[i] = s;
      }
      __syncthreads();
    }
    double s2 = 0.0;
    for (int i = tid; i < n; i += nt) s2 += za[i] * za[i];
    s2 = cta_sum(s2, sh);
    if (!(s2 > 1e-20)) return 2;
    double inv = 1.0 / sqrt(s2);
    for (int i = tid; i < n; i += nt) za[i] *= inv;
    __syncthreads();
  }
  return 0;
}

__global__ void __launch_bounds__(1024) eigh_lowest_kernel(double* A, int n, int k, double* w, double* ZT,
                                                           double* scratch, int* status) {
  __shared__ EigShared sh;
  int rc = eigh_lowest_cta(A, n, k, w, ZT, scratch, sh);
  if (threadIdx.x == 0 && status) *status = rc;
}

// ---- k lowest eigenpairs on many SMs -------------------------------------------------------
// Same algorithm as eigh_lowest_cta with the O(n^3) reduction spread over G co-resident CTAs
// (cooperative launch): in step k every CTA recomputes the Householder vector of column k
// itself (same data, same reduction order, so the same bits), updates p = beta A22 v for
// its share of rows (row r belongs to CTA (r - k - 1) mod G), and after a grid barrier
// applies the rank-2 update to those rows.  Two grid barriers per column.  Barrier waits
// are bounded; a timeout sets the error flag and every CTA returns.
struct GridBarrier {
  unsigned count;
  unsigned gen;
  int err;
};

__device__ bool grid_sync(GridBarrier* b, unsigned nblocks) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &b->gen;
    volatile int* verr = &b->err;
    unsigned g = *vgen;
    __threadfence();
    if (atomicAdd(&b->count, 1u) == nblocks - 1) {
      b->count = 0;
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      for (unsigned it = 0; *vgen == g; ++it) {
        if (it > (1u << 24) || *verr) {
          atomicExch(&b->err, 1);
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    ok = (*verr == 0);
  }
  __syncthreads();
  return ok != 0;
}

__global__ void __launch_bounds__(256) eigh_lowest_coop_kernel(double* __restrict__ A, int n, int k,
                                                                double* __restrict__ w, double* __restrict__ ZT,
                                                                double* __restrict__ scr, double* __restrict__ pbuf,
                                                                GridBarrier* bar, int* status) {
  extern __shared__ double smem_d[];
  __shared__ EigShared sh;
  const unsigned G = gridDim.x;
  const int cta = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  double* v = smem_d;       // n
  double* wv = smem_d + n;  // n
  double* d = scr;
  double* e = d + n;
  double* beta = e + n;
  double* lu = beta + 2 * n;  // 6 n k (after one spare n)
  // ---- 1. tridiagonalisation -------------------------------------------------------------
  for (int kk = 0; kk + 2 < n; ++kk) {
    const int len = n - kk - 1;
    double part = 0.0;
    for (int i = tid + 1; i < len; i += nt) {
      double x = A[(size_t)(kk + 1 + i) * n + kk];
      part += x * x;
    }
    double sigma = cta_sum(part, sh);
    double x0 = A[(size_t)(kk + 1) * n + kk];
    double alpha, b;
    if (sigma == 0.0) {
      alpha = x0;
      b = 0.0;
    } else {
      double nrm = sqrt(x0 * x0 + sigma);
      alpha = (x0 >= 0.0) ? -nrm : nrm;
      double v0 = x0 - alpha;
      b = 2.0 / (v0 * v0 + sigma);
    }
    for (int i = tid; i < len; i += nt) v[i] = (i == 0) ? (x0 - alpha) : A[(size_t)(kk + 1 + i) * n + kk];
    if (cta == 0 && tid == 0) {
      d[kk] = A[(size_t)kk * n + kk];
      e[kk] = alpha;
      beta[kk] = b;
    }
    __syncthreads();
    if (b != 0.0) {
      for (int i = cta + (int)G * wid; i < len; i += (int)G * nw) {
        const double* row = A + (size_t)(kk + 1 + i) * n + kk + 1;
        double s = 0.0;
        for (int j = lane; j < len; j += 32) s += row[j] * v[j];
        s = warp_sum(s);
        if (lane == 0) pbuf[i] = b * s;
      }
    }
    if (!grid_sync(bar, G)) break;
    if (b != 0.0) {
      double pv = 0.0;
      for (int i = tid; i < len; i += nt) {
        double p = pbuf[i];
        wv[i] = p;
        pv += p * v[i];
      }
      double Kf = 0.5 * b * cta_sum(pv, sh);
      for (int i = tid; i < len; i += nt) wv[i] -= Kf * v[i];
      __syncthreads();
      for (int i = cta + (int)G * wid; i < len; i += (int)G * nw) {
        double* row = A + (size_t)(kk + 1 + i) * n + kk + 1;
        const double vi = v[i], wi = wv[i];
        for (int j = lane; j < len; j += 32) row[j] -= vi * wv[j] + wi * v[j];
      }
    }
    // reflector into column kk, rows owned by this CTA
    for (int i = cta + (int)G * tid; i < len; i += (int)G * nt) A[(size_t)(kk + 1 + i) * n + kk] = v[i];
    if (!grid_sync(bar, G)) break;
  }
  if (bar->err) {
    if (cta == 0 && tid == 0) *status = 3;
    return;
  }
  if (cta == 0 && tid == 0) {
    if (n >= 2) {
      d[n - 2] = A[(size_t)(n - 2) * n + n - 2];
      e[n - 2] = A[(size_t)(n - 1) * n + n - 2];
    }
    d[n - 1] = A[(size_t)(n - 1) * n + n - 1];
    e[n - 1] = 0.0;
  }
  // reflectors into the upper triangle rows for coalesced reads
  for (long q = (long)cta * nt + tid; q < (long)n * n; q += (long)G * nt) {
    int i = (int)(q / n), j = (int)(q % n);
    if (j > i) A[(size_t)i * n + j] = A[(size_t)j * n + i];
  }
  if (!grid_sync(bar, G)) {
    if (cta == 0 && tid == 0) *status = 3;
    return;
  }
  // ---- 2. bisection and inverse iteration, one lane per eigenvalue ---------------------------
  double glo = INFINITY, ghi = -INFINITY, emax2 = 0.0;
  for (int i = 0; i < n; ++i) {
    double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0);
    glo = fmin(glo, d[i] - r);
    ghi = fmax(ghi, d[i] + r);
    if (i + 1 < n) emax2 = fmax(emax2, e[i] * e[i]);
  }
  const double tnorm = fmax(fabs(glo), fabs(ghi));
  const double pivmin = DBL_MIN * fmax(1.0, emax2);
  double* x = lu + 5 * (size_t)n * k;
  for (int t = cta * nt + tid; t < k; t += (int)G * nt) {
    double lo = glo - 2.0 * DBL_EPSILON * tnorm, hi = ghi + 2.0 * DBL_EPSILON * tnorm;
    for (int it = 0; it < 200; ++it) {
      double mid = 0.5 * (lo + hi);
      if (sturm_count(d, e, n, mid, pivmin) > t) hi = mid;
      else lo = mid;
      if (hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + pivmin) break;
    }
    double lam = 0.5 * (lo + hi);
    w[t] = lam;
    if (!inverse_iteration(d, e, n, lam, tnorm, t, k, lu, lu + (size_t)n * k, lu + 2 * (size_t)n * k,
                           lu + 3 * (size_t)n * k, lu + 4 * (size_t)n * k, x))
      atomicExch(&bar->err, 2);
  }
  if (!grid_sync(bar, G)) {
    if (cta == 0 && tid == 0) *status = 1;
    return;
  }
  // ---- 3. back-transformation, one warp per vector -------------------------------------------
  for (int t = cta * nw + wid; t < k; t += (int)G * nw) {
    double* z = ZT + (size_t)t * n;
    for (int i = lane; i < n; i += 32) z[i] = x[(size_t)i * k + t];
    __syncwarp();
    for (int r = n - 3; r >= 0; --r) {
      double bb = beta[r];
      if (bb == 0.0) continue;
      const double* vr = A + (size_t)r * n + r + 1;
      double s = 0.0;
      for (int i = lane; i < n - r - 1; i += 32) s += vr[i] * z[r + 1 + i];
      s = bb * warp_sum(s);
      for (int i = lane; i < n - r - 1; i += 32) z[r + 1 + i] -= s * vr[i];
      __syncwarp();
    }
  }
  if (!grid_sync(bar, G)) {
    if (cta == 0 && tid == 0) *status = 3;
    return;
  }
  if (cta != 0) return;
  // ---- 4. classical Gram-Schmidt twice (one CTA) -------------------------------------------
  double* coef = lu;
  for (int a = 0; a < k; ++a) {
    double* za = ZT + (size_t)a * n;
    for (int pass = 0; pass < 2; ++pass) {
      for (int bI = wid; bI < a; bI += nw) {
        const double* zb = ZT + (size_t)bI * n;
        double s = 0.0;
        for (int i = lane; i < n; i += 32) s += zb[i] * za[i];
        s = warp_sum(s);
        if (lane == 0) coef[bI] = s;
      }
      __syncthreads();
      for (int i = tid; i < n; i += nt) {
        double s = za[i];
        for (int bI = 0; bI < a; ++bI) s -= coef[bI] * ZT[(size_t)bI * n + i];
        za[i] = s;
      }
      __syncthreads();
    }
    double s2 = 0.0;
    for (int i = tid; i < n; i += nt) s2 += za[i] * za[i];
    s2 = cta_sum(s2, sh);
    if (!(s2 > 1e-20)) {
      if (tid == 0) *status = 2;
      return;
    }
    double inv = 1.0 / sqrt(s2);
    for (int i = tid; i < n; i += nt) za[i] *= inv;
    __syncthreads();
  }
  if (tid == 0) *status = 0;
}

__global__ void transpose_kernel(const double* __restrict__ in, int rows, int cols, double* __restrict__ out) {
  __shared__ double t[32][33];
  int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += 8) {
    int r = by + j, c = bx + threadIdx.x;
    if (r < rows && c < cols) t[j][threadIdx.x] = in[(size_t)r * cols + c];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += 8) {
    int r = bx + j, c = by + threadIdx.x;  // out is cols x rows
    if (r < cols && c < rows) out[(size_t)r * rows + c] = t[threadIdx.x][j];
  }
}

int transpose(const double* in, int rows, int cols, double* out, cudaStream_t s) {
  dim3 grid((cols + 31) / 32, (rows + 31) / 32);
  transpose_kernel<<<grid, dim3(32, 8), 0, s>>>(in, rows, cols, out);
  DF_LAUNCHED("transpose_kernel");
  return DF_OK;
}

size_t eigh_scratch_doubles(int n) { return (size_t)6 * n; }

size_t eigh_lowest_scratch_doubles(int n, int k) { return (size_t)4 * n + (size_t)6 * n * std::max(k, 1); }

size_t eigh_coop_aux_bytes(int n) { return align_up(sizeof(double) * (size_t)n, 256) + 256; }

// Number of CTAs for the multi-SM path (0: use one CTA).  Knob "eig_ctas" overrides.
static int coop_ctas(int n) {
  int forced = knob("eig_ctas");
  if (forced == 1) return 0;
  if (forced == 0 && n < 160) return 0;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  size_t smem = 2 * sizeof(double) * (size_t)n;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(eigh_lowest_coop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, eigh_lowest_coop_kernel, 256, smem) != cudaSuccess)
    return 0;
  int cap = sms * std::max(per_sm, 0);
  int want = forced > 1 ? forced : std::min(sms, std::max(8, n / 16));
  return std::min(want, cap);
}

// aux: coop_aux_bytes(n) of scratch for the multi-SM path (p vector and grid barrier).
int eigh_lowest_rows(double* A, int n, int k, double* w, double* ZT, double* scratch, int* status, cudaStream_t s,
                     void* aux) {
  int G = aux ? coop_ctas(n) : 0;
  if (G >= 2) {
    double* pbuf = (double*)aux;
    GridBarrier* bar = (GridBarrier*)((char*)aux + align_up(sizeof(double) * (size_t)n, 256));
    DF_CUDA(cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 2 * sizeof(double) * (size_t)n;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    DF_CUDA(cudaLaunchKernelEx(&cfg, eigh_lowest_coop_kernel, A, n, k, w, ZT, scratch, pbuf, bar, status));
    return DF_OK;
  }
  eigh_lowest_kernel<<<1, 1024, 0, s>>>(A, n, k, w, ZT, scratch, status);
  DF_LAUNCHED("eigh_lowest_kernel");
  return DF_OK;
}

int eigh_rows(double* A, int n, double* w, double* ZT, double* scratch, int* status, cudaStream_t s) {
  eigh_batched_kernel<<<1, 1024, 0, s>>>(A, n, 0, w, 0, ZT, 0, scratch, 0, status);
  DF_LAUNCHED("eigh_batched_kernel");
  return DF_OK;
}

}  // namespace dfscf

using namespace dfscf;

extern "C" size_t df_eigh_work_bytes(int n) {
  if (n <= 0) return 0;
  Sizer z;
  z.take<double>(eigh_scratch_doubles(n));
  z.take<double>((size_t)n * n);
  z.take<int>(1);
  return z.used;
}

extern "C" int df_eigh(double* A, int n, double* w, double* Z, void* work, size_t work_bytes, cudaStream_t s) {
  clear_error();
  DF_REQUIRE(A && w && Z && n > 0, DF_ERR_ARG, "df_eigh: bad arguments");
  DF_REQUIRE(work && work_bytes >= df_eigh_work_bytes(n), DF_ERR_NOMEM, "df_eigh: workspace too small");
  Arena a(work, work_bytes);
  double* scratch = a.take<double>(eigh_scratch_doubles(n));
  double* ZT = a.take<double>((size_t)n * n);
  int* status = a.take<int>(1);
  DF_TRY(eigh_rows(A, n, w, ZT, scratch, status, s));
  DF_TRY(transpose(ZT, n, n, Z, s));
  int h = 0;
  DF_CUDA(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s));
  DF_CUDA(cudaStreamSynchronize(s));
  DF_REQUIRE(h == 0, DF_ERR_NOCONV, "df_eigh: QL iteration did not converge");
  return DF_OK;
}

extern "C" size_t df_eigh_lowest_work_bytes(int n, int k) {
  if (n <= 0 || k <= 0 || k > n) return 0;
  Sizer z;
  z.take<double>(eigh_lowest_scratch_doubles(n, k));
  z.take<double>((size_t)n * k);
  z.take<int>(1);
  z.take<char>(eigh_coop_aux_bytes(n));
  return z.used;
}

extern "C" int df_eigh_lowest(double* A, int n, int k, double* w, double* Z, void* work, size_t work_bytes,
                              cudaStream_t s) {
  clear_error();
  DF_REQUIRE(A && w && Z && n > 0 && k > 0 && k <= n, DF_ERR_ARG, "df_eigh_lowest: bad arguments");
  DF_REQUIRE(work && work_bytes >= df_eigh_lowest_work_bytes(n, k), DF_ERR_NOMEM, "df_eigh_lowest: workspace too small");
  Arena a(work, work_bytes);
  double* scratch = a.take<double>(eigh_lowest_scratch_doubles(n, k));
  double* ZT = a.take<double>((size_t)n * k);
  int* status = a.take<int>(1);
  void* aux = a.take<char>(eigh_coop_aux_bytes(n));
  DF_TRY(eigh_lowest_rows(A, n, k, w, ZT, scratch, status, s, aux));
  DF_TRY(transpose(ZT, k, n, Z, s));
  int h = 0;
  DF_CUDA(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s));
  DF_CUDA(cudaStreamSynchronize(s));
  DF_REQUIRE(h == 0, DF_ERR_NOCONV, "df_eigh_lowest: inverse iteration or re-orthogonalisation failed (%d)", h);
  return DF_OK;
}
