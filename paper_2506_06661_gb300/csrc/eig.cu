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
  double bsum, bmax;  // broadcast slots of cta_sum / cta_max
  int flag;
};

// CTA-wide sum, the same value (and the same bits in every CTA of a grid) for every thread:
// warp sums, then warp 0 reduces the partials and broadcasts through shared memory (FP64
// issues slowly on this part, so no warp repeats the partials' sum).
__device__ double cta_sum(double v, EigShared& sh) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh.red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double t = lane < nw ? sh.red[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) sh.bsum = t;
  }
  __syncthreads();
  return sh.bsum;
}

__device__ double cta_max(double v, EigShared& sh) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) sh.red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double t = lane < nw ? sh.red[lane] : -INFINITY;
    for (int o = 16; o; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
    if (lane == 0) sh.bmax = t;
  }
  __syncthreads();
  return sh.bmax;
}

// Gershgorin interval [glo, ghi] of tridiag(d, e) and max e^2, reduced over the CTA.
__device__ void gershgorin_cta(const double* __restrict__ d, const double* __restrict__ e, int n, double& glo,
                               double& ghi, double& emax2, EigShared& sh) {
  double lo = INFINITY, hi = -INFINITY, em = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0);
    lo = fmin(lo, d[i] - r);
    hi = fmax(hi, d[i] + r);
    if (i + 1 < n) em = fmax(em, e[i] * e[i]);
  }
  glo = -cta_max(-lo, sh);
  ghi = cta_max(hi, sh);
  emax2 = cta_max(em, sh);
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
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    if (b != 0.0) {
      // p = b * A22 v, one thread per entry: A22 is symmetric (kept so by the full rank-2
      // updates), so thread i walks column i, coalesced across the warp and with no
      // reduction between lanes; four partial sums for independent FMA chains
      for (int i = tid; i < len; i += nt) {
        const double* col = A + (size_t)(k + 1) * n + k + 1 + i;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int j = 0;
        for (; j + 3 < len; j += 4) {
          s0 += col[(size_t)j * n] * v[j];
          s1 += col[(size_t)(j + 1) * n] * v[j + 1];
          s2 += col[(size_t)(j + 2) * n] * v[j + 2];
          s3 += col[(size_t)(j + 3) * n] * v[j + 3];
        }
        for (; j < len; ++j) s0 += col[(size_t)j * n] * v[j];
        cs[i] = b * ((s0 + s1) + (s2 + s3));
      }
      __syncthreads();
      double pv = 0.0;
      for (int i = tid; i < len; i += nt) pv += cs[i] * v[i];
      double K = 0.5 * b * cta_sum(pv, sh);
      for (int i = tid; i < len; i += nt) sn[i] = cs[i] - K * v[i];  // w
      __syncthreads();
      // rank-2 update, one warp per row, lanes along the row
      for (int i = wid; i < len; i += nw) {
        double* row = A + (size_t)(k + 1 + i) * n + k + 1;
        const double vi = v[i], wi = sn[i];
        for (int j = lane; j < len; j += 32) row[j] -= vi * sn[j] + wi * v[j];
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

// Eigenvalues of tridiag(d, e) that are < x (count of negative pivots of T - x I);
// ee[i] = e[i]^2.
__device__ int sturm_count(const double* __restrict__ d, const double* __restrict__ ee, int n, double x,
                           double pivmin) {
  int c = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  c += q < 0.0;
  for (int i = 1; i < n; ++i) {
    q = (d[i] - x) - ee[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    c += q < 0.0;
  }
  return c;
}

// Deterministic start component in [1, 1.5) from an integer hash of (i, t): every
// component non-zero, no transcendental FP64 work.
__device__ __forceinline__ double start_component(int i, int t) {
  unsigned h = (unsigned)i * 0x9E3779B1u ^ ((unsigned)t + 0x7F4A7C15u) * 0x85EBCA77u;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  return 1.0 + (double)(h >> 8) * (0.5 / 16777216.0);
}

// Lane t: inverse iteration for eigenvalue lam of tridiag(d, e) into x (interleaved storage:
// element i of lane t at [i * kk + t]).  T - lam I = P L U with partial pivoting (rows i and
// i+1 interchanged when |sub| > |diag|); the factors are stored as L (multipliers), piv,
// ru0 = 1/U(i,i) (pivots below eps ||T|| raised to it), u1 = U(i,i+1), u2 = U(i,i+2).  The
// elimination and both triangular sweeps carry their recurrences in registers, so the only
// dependent chain is the FP64 arithmetic itself.  Each solve's result is divided by its
// max-norm on the next sweep (no overflow); three solves, then a 2-norm normalisation.
__device__ bool inverse_iteration(const double* __restrict__ d, const double* __restrict__ e, int n, double lam,
                                  double tnorm, int t, int kk, double* __restrict__ L, double* __restrict__ ru0,
                                  double* __restrict__ u1, double* __restrict__ u2, double* __restrict__ piv,
                                  double* __restrict__ x) {
#define IX(a, i) a[(size_t)(i) * kk + t]
  const double small = DBL_EPSILON * tnorm + 1e-300;
  double di = d[0] - lam;
  double ui = n > 1 ? e[0] : 0.0;
  for (int i = 0; i + 1 < n; ++i) {
    const double li = e[i], dn = d[i + 1] - lam, un = i + 2 < n ? e[i + 1] : 0.0;
    double piv_d, f;
    if (fabs(di) >= fabs(li)) {
      f = di != 0.0 ? li / di : 0.0;
      piv_d = di;
      IX(piv, i) = 0.0;
      IX(u1, i) = ui;
      IX(u2, i) = 0.0;
      di = dn - f * ui;
      ui = un;
    } else {
      f = di / li;
      piv_d = li;
      IX(piv, i) = 1.0;
      IX(u1, i) = dn;
      IX(u2, i) = un;
      di = ui - f * dn;
      ui = -f * un;
    }
    IX(L, i) = f;
    if (fabs(piv_d) < small) piv_d = copysign(small, piv_d == 0.0 ? 1.0 : piv_d);
    IX(ru0, i) = 1.0 / piv_d;
  }
  if (fabs(di) < small) di = copysign(small, di == 0.0 ? 1.0 : di);
  IX(ru0, n - 1) = 1.0 / di;
  if (n >= 1) {
    IX(u1, n - 1) = 0.0;
    IX(u2, n - 1) = 0.0;
  }
  if (n >= 2) IX(u2, n - 2) = 0.0;
  double scale = 1.0;
  for (int it = 0; it < 3; ++it) {
    // forward: apply P and L^-1 to scale * x (the start vector on the first solve)
    double xi = it == 0 ? start_component(0, t) : scale * IX(x, 0);
    for (int i = 0; i + 1 < n; ++i) {
      const double xn = it == 0 ? start_component(i + 1, t) : scale * IX(x, i + 1);
      const double f = IX(L, i);
      double out, carry;
      if (IX(piv, i) == 0.0) {
        out = xi;
        carry = xn - f * xi;
      } else {
        out = xn;
        carry = xi - f * xn;
      }
      IX(x, i) = out;
      xi = carry;
    }
    IX(x, n - 1) = xi;
    // backward: U^-1, tracking the max-norm
    double x1 = 0.0, x2 = 0.0, mx = 0.0;
    for (int i = n - 1; i >= 0; --i) {
      const double v = (IX(x, i) - IX(u1, i) * x1 - IX(u2, i) * x2) * IX(ru0, i);
      IX(x, i) = v;
      mx = fmax(mx, fabs(v));
      x2 = x1;
      x1 = v;
    }
    if (!(mx > 0.0) || !isfinite(mx)) return false;
    scale = 1.0 / mx;
  }
  double s2 = 0.0;
  for (int i = 0; i < n; ++i) {
    const double v = IX(x, i) * scale;
    s2 += v * v;
  }
  const double inv = scale / sqrt(s2);
  for (int i = 0; i < n; ++i) IX(x, i) *= inv;
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
  double glo, ghi, emax2;
  gershgorin_cta(d, e, n, glo, ghi, emax2, sh);
  const double tnorm = fmax(fabs(glo), fabs(ghi));
  const double pivmin = DBL_MIN * fmax(1.0, emax2);
  double* x = lu + 5 * (size_t)n * k;
  double* ee = v;  // the reduction's work vector is free now
  for (int i = tid; i + 1 < n; i += nt) ee[i] = e[i] * e[i];
  __syncthreads();
  // eigenvalues: groups of G lanes per eigenvalue split the bracket (G+1)-way per round; G is
  // chosen so that about four warps work (one per FP64 pipe of the SM)
  int G = 1;
  while (G < 32 && k * (2 * G) <= 128) G *= 2;
  {
    const int lane = tid & 31, sub = tid % G, base = lane - sub;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << base);
    for (int t0 = tid / G; t0 - (lane / G) < k; t0 += nt / G) {  // every lane of a warp iterates together
      const int t = t0;
      const bool live = t < k;
      double lo = glo - 2.0 * DBL_EPSILON * tnorm, hi = ghi + 2.0 * DBL_EPSILON * tnorm;
      bool done = !live;
      for (int round = 0; round < 200; ++round) {
        if (!done && hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + pivmin) done = true;
        if (__all_sync(0xffffffffu, done)) break;
        const double h = (hi - lo) / (double)(G + 1);
        const double xj = fmin(lo + (double)(sub + 1) * h, hi);
        const bool up = live && sturm_count(d, ee, n, xj, pivmin) > t;
        const unsigned above = (__ballot_sync(0xffffffffu, up) & gmask) >> base;
        const double xlast = __shfl_sync(0xffffffffu, xj, base + G - 1);
        const int j = above ? __ffs(above) - 1 : 0;
        const double xhi = __shfl_sync(0xffffffffu, xj, base + j);
        const double xlo = __shfl_sync(0xffffffffu, xj, base + (j > 0 ? j - 1 : 0));
        if (!done) {
          if (above == 0u) {
            lo = xlast;
          } else {
            if (j > 0) lo = xlo;
            hi = xhi;
          }
        }
      }
      if (live && sub == 0) w[t] = 0.5 * (lo + hi);
    }
  }
  __syncthreads();
  // eigenvectors of T: inverse iteration, one lane per eigenvalue
  for (int t = tid; t < k; t += nt) {
    bool ok = inverse_iteration(d, e, n, w[t], tnorm, t, k, lu, lu + (size_t)n * k, lu + 2 * (size_t)n * k,
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
// Same algorithm as eigh_lowest_cta spread over G co-resident CTAs (cooperative launch).
// FP64 issues at a small fraction of the FP32 rate on this GPU, so every serial FP64 chain
// is spread over as many SMs as possible:
//   1. reduction: in step k every CTA recomputes the Householder vector of column k itself
//      (same data, same reduction order, so the same bits), updates p = beta A22 v for its
//      share of rows (row r belongs to CTA (r - k - 1) mod G), and after a grid barrier
//      applies the rank-2 update to those rows (two grid barriers per column);
//   2. eigenvalues: one warp per eigenvalue, consecutive eigenvalues on different CTAs; each
//      round evaluates 32 Sturm counts at the interior points of a 33-way split of the
//      bracket (the interval shrinks 33-fold per round instead of 2-fold);
//   3. inverse iteration: one lane per eigenvalue, 32 per warp, warps on different CTAs;
//   4. back-transformation: one warp per vector with the vector staged in shared memory;
//   5. classical Gram-Schmidt twice, each projection spread over the whole grid.
// Barrier waits are bounded; a timeout sets the error flag and every CTA returns.
struct GridBarrier {
  unsigned count;  // arrivals since launch (monotone; zeroed before the launch)
  unsigned extra;  // arrivals expected beyond the grid's own CTAs: 0, except in the test of
                   // the bounded wait (knob "eig_barrier_extra"), where no barrier can complete
  int err;         // 1: a wait gave up; 2: inverse iteration failed
  unsigned limit;  // polls before a wait gives up (knob "eig_barrier_polls")
};

// Set up the barrier record on the stream (graph-capturable, unlike a host write).
__global__ void grid_barrier_init_kernel(GridBarrier* b, unsigned limit, unsigned extra) {
  if (threadIdx.x != 0) return;
  b->count = 0;
  b->extra = extra;
  b->err = 0;
  b->limit = limit;
}

// Grid barrier on a monotone arrival counter: the b-th barrier completes when the counter
// reaches b * (G + extra).  Thread 0 of each CTA arrives after a device-scope fence and polls
// with acquire loads; after `limit` polls (2^22 by default, about a second) it raises the
// error flag, every other CTA sees the flag within 256 polls, and all of them return.
__device__ bool grid_sync(GridBarrier* b, unsigned G) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned Ge = G + b->extra;
    const unsigned limit = b->limit;
    const unsigned old = atomicAdd(&b->count, 1u);
    const unsigned target = (old / Ge + 1u) * Ge;
    unsigned cur = old + 1u;
    volatile int* verr = &b->err;
    for (unsigned it = 0; (int)(cur - target) < 0; ++it) {
      if (it > limit) {
        atomicCAS(&b->err, 0, 1);
        break;
      }
      if ((it & 255u) == 0u && *verr) break;
      asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(cur) : "l"(&b->count) : "memory");
    }
    __threadfence();
    ok = (*verr == 0);
  }
  __syncthreads();
  return ok != 0;
}

// aux layout (eigh_coop_aux_bytes): p vector [n], Gram-Schmidt coefficients [n], per-CTA
// partial sums [kCoopMaxCtas], barrier.
constexpr int kCoopMaxCtas = 1024;

// Phases 2-5 on the tridiagonal form (d, e, beta; reflector r in row r of A, columns
// r+1..n-1), shared by both reductions.  zsm: zw * n doubles of shared memory.
__device__ void coop_tail(const double* __restrict__ A, int n, int k, double* __restrict__ w, double* __restrict__ ZT,
                          double* __restrict__ d, double* __restrict__ e, double* __restrict__ beta,
                          double* __restrict__ ee, double* __restrict__ lu, double* __restrict__ coef,
                          double* __restrict__ part, int zw, double* zsm, GridBarrier* bar, int* status,
                          EigShared& sh) {
  const unsigned G = gridDim.x;
  const int cta = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  // ---- 2. eigenvalues: 33-way multisection, one warp per eigenvalue -----------------------
  double glo, ghi, emax2;
  gershgorin_cta(d, e, n, glo, ghi, emax2, sh);
  for (int i = cta * nt + tid; i + 1 < n; i += (int)G * nt) ee[i] = e[i] * e[i];
  if (!grid_sync(bar, G)) {
    if (cta == 0 && tid == 0) *status = 3;
    return;
  }
  const double tnorm = fmax(fabs(glo), fabs(ghi));
  const double pivmin = DBL_MIN * fmax(1.0, emax2);
  for (int t = wid * (int)G + cta; t < k; t += (int)G * nw) {
    double lo = glo - 2.0 * DBL_EPSILON * tnorm, hi = ghi + 2.0 * DBL_EPSILON * tnorm;
    for (int round = 0; round < 64; ++round) {
      if (hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + pivmin) break;
      const double h = (hi - lo) * (1.0 / 33.0);
      const double xj = fmin(lo + (double)(lane + 1) * h, hi);
      const unsigned above = __ballot_sync(0xffffffffu, sturm_count(d, ee, n, xj, pivmin) > t);
      if (above == 0u) {
        lo = __shfl_sync(0xffffffffu, xj, 31);
      } else {
        const int j = __ffs(above) - 1;
        const double xhi = __shfl_sync(0xffffffffu, xj, j);
        const double xlo = __shfl_sync(0xffffffffu, xj, j > 0 ? j - 1 : 0);
        if (j > 0) lo = xlo;
        hi = xhi;
      }
    }
    if (lane == 0) w[t] = 0.5 * (lo + hi);
  }
  if (!grid_sync(bar, G)) {
    if (cta == 0 && tid == 0) *status = 3;
    return;
  }
  // ---- 3. inverse iteration, one lane per eigenvalue, warps on different CTAs ---------------
  double* x = lu + 5 * (size_t)n * k;
  for (int t = (wid * (int)G + cta) * 32 + lane; t - lane < k; t += (int)G * nw * 32) {
    if (t < k &&
        !inverse_iteration(d, e, n, w[t], tnorm, t, k, lu, lu + (size_t)n * k, lu + 2 * (size_t)n * k,
                           lu + 3 * (size_t)n * k, lu + 4 * (size_t)n * k, x))
      atomicExch(&bar->err, 2);
  }
  if (!grid_sync(bar, G)) {
    if (cta == 0 && tid == 0) *status = bar->err == 2 ? 1 : 3;
    return;
  }
  // ---- 4. back-transformation, one warp per vector staged in shared memory ------------------
  if (wid < zw) {
    double* zs = zsm + (size_t)wid * n;
    for (int t = wid * (int)G + cta; t < k; t += (int)G * zw) {
      for (int i = lane; i < n; i += 32) zs[i] = x[(size_t)i * k + t];
      __syncwarp();
      for (int r = n - 3; r >= 0; --r) {
        const double bb = beta[r];
        if (bb == 0.0) continue;
        const double* vr = A + (size_t)r * n + r + 1;
        double* zr = zs + r + 1;
        const int len = n - r - 1;
        double s = 0.0;
        for (int i = lane; i < len; i += 32) s += vr[i] * zr[i];
        s = bb * warp_sum(s);
        for (int i = lane; i < len; i += 32) zr[i] -= s * vr[i];
        __syncwarp();
      }
      double* z = ZT + (size_t)t * n;
      for (int i = lane; i < n; i += 32) z[i] = zs[i];
      __syncwarp();
    }
  }
  if (!grid_sync(bar, G)) {
    if (cta == 0 && tid == 0) *status = 3;
    return;
  }
  // ---- 5. classical Gram-Schmidt twice over the grid ----------------------------------------
  const int gw = wid * (int)G + cta, ngw = (int)G * nw;
  const int gt = cta * nt + tid, ngt = (int)G * nt;
  for (int a = 0; a < k; ++a) {
    double* za = ZT + (size_t)a * n;
    for (int pass = 0; a > 0 && pass < 2; ++pass) {
      for (int b = gw; b < a; b += ngw) {
        const double* zb = ZT + (size_t)b * n;
        double s = 0.0;
        for (int i = lane; i < n; i += 32) s += zb[i] * za[i];
        s = warp_sum(s);
        if (lane == 0) coef[b] = s;
      }
      if (!grid_sync(bar, G)) break;
      for (int i = gt; i < n; i += ngt) {
        double s = za[i];
        for (int b = 0; b < a; ++b) s -= coef[b] * ZT[(size_t)b * n + i];
        za[i] = s;
      }
      if (!grid_sync(bar, G)) break;
    }
    if (bar->err) break;
    double s2 = 0.0;
    for (int i = gt; i < n; i += ngt) s2 += za[i] * za[i];
    s2 = cta_sum(s2, sh);
    if (tid == 0) part[cta] = s2;
    if (!grid_sync(bar, G)) break;
    double tot = 0.0;
    for (unsigned c = 0; c < G; ++c) tot += part[c];  // same order in every CTA
    if (!(tot > 1e-20)) {
      if (cta == 0 && tid == 0) *status = 2;
      return;
    }
    const double inv = 1.0 / sqrt(tot);
    for (int i = gt; i < n; i += ngt) za[i] *= inv;
    if (!grid_sync(bar, G)) break;
  }
  if (cta == 0 && tid == 0) *status = bar->err ? 3 : 0;
}

// Reduction with the trailing matrix in global memory (any n).  Dynamic shared memory:
// v, w [n] for the reduction, then zw vectors [n] for the back-transformation.
__global__ void __launch_bounds__(256, 1) eigh_lowest_coop_kernel(double* __restrict__ A, int n, int k,
                                                                double* __restrict__ w, double* __restrict__ ZT,
                                                                double* __restrict__ scr, double* __restrict__ pbuf,
                                                                double* __restrict__ coef, double* __restrict__ part,
                                                                int zw, GridBarrier* bar, int* status) {
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
  double* ee = beta + n;
  double* lu = beta + 2 * n;  // 6 n k
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
  coop_tail(A, n, k, w, ZT, d, e, beta, ee, lu, coef, part, zw, smem_d + 2 * (size_t)n, bar, status, sh);
}

// Reduction with the rows of the trailing matrix in shared memory: row r lives in CTA
// r mod G at slot r / G (R = ceil(n / G) slots of n doubles).  Every CTA keeps the current
// column x = A[kk+1.., kk] and recomputes the reflector (v, beta) from it; the owners of the
// rows compute p = beta A22 v and publish p together with the old column kk+1; after the one
// grid barrier of the step every CTA forms w = p - (beta p.v / 2) v, updates its rows and
// derives the next column from the old one with the same rank-2 formula, so all CTAs hold
// the same bits.  Exchange buffers are double-buffered by step parity.  The reflector goes to
// row kk of A (global) for the back-transformation.  Dynamic shared memory: 4 n + max(R, zw) n
// doubles (the back-transformation's vectors reuse the row slots).
__device__ __forceinline__ double rank2(double vi, double wj, double wi, double vj) {
  return __fma_rn(vi, wj, __dmul_rn(wi, vj));
}

__global__ void __launch_bounds__(256, 1) eigh_lowest_coop_smem_kernel(double* __restrict__ A, int n, int k,
                                                                     double* __restrict__ w, double* __restrict__ ZT,
                                                                     double* __restrict__ scr,
                                                                     double* __restrict__ xbuf, int R,
                                                                     double* __restrict__ coef,
                                                                     double* __restrict__ part, int zw,
                                                                     GridBarrier* bar, int* status) {
  extern __shared__ double smem_d[];
  __shared__ EigShared sh;
  const unsigned G = gridDim.x;
  const int cta = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  double* v = smem_d;            // n: reflector
  double* wv = smem_d + n;       // n: p, then w
  double* x = smem_d + 2 * n;    // n: current column below the diagonal
  double* c = smem_d + 3 * n;    // n: old next column
  double* rows = smem_d + 4 * n; // R n
  double* d = scr;
  double* e = d + n;
  double* beta = e + n;
  double* ee = beta + n;
  double* lu = beta + 2 * n;  // 6 n k
  // owned rows into shared memory; column 0 below the diagonal into x
  for (int s = 0; s < R; ++s) {
    const int r = s * (int)G + cta;
    if (r >= n) break;
    for (int j = tid; j < n; j += nt) rows[(size_t)s * n + j] = A[(size_t)r * n + j];
  }
  for (int i = tid; i + 1 < n; i += nt) x[i] = A[(size_t)(i + 1) * n];
  // all CTAs have read A before any reflector is written back into it
  if (!grid_sync(bar, G)) {
    if (cta == 0 && tid == 0) *status = 3;
    return;
  }
  // ---- 1. tridiagonalisation -------------------------------------------------------------
  for (int kk = 0; kk + 2 < n; ++kk) {
    const int len = n - kk - 1;  // x = A[kk+1..n)[kk]
    double part_s = 0.0;
    for (int i = tid + 1; i < len; i += nt) part_s += x[i] * x[i];
    const double sigma = cta_sum(part_s, sh);
    const double x0 = x[0];
    double alpha, b;
    if (sigma == 0.0) {
      alpha = x0;
      b = 0.0;
    } else {
      const double nrm = sqrt(x0 * x0 + sigma);
      alpha = (x0 >= 0.0) ? -nrm : nrm;
      const double v0 = x0 - alpha;
      b = 2.0 / (v0 * v0 + sigma);
    }
    for (int i = tid; i < len; i += nt) v[i] = (i == 0) ? (x0 - alpha) : x[i];
    if (cta == 0 && tid == 0) {
      e[kk] = alpha;
      beta[kk] = b;
    }
    if (kk % (int)G == cta && tid == 0) d[kk] = rows[(size_t)(kk / (int)G) * n + kk];
    __syncthreads();
    // p for the owned rows of the trailing block, and their entries in column kk+1
    double* pg = xbuf + (size_t)(kk & 1) * 2 * n;
    double* cg = pg + n;
    {
      const int s0 = (kk + 1 - cta + (int)G - 1) / (int)G;  // first slot with row > kk
      for (int s = s0 + wid; s < R; s += nw) {
        const int r = s * (int)G + cta;
        if (r >= n) break;
        const double* row = rows + (size_t)s * n + kk + 1;
        double acc = 0.0;
        if (b != 0.0)
          for (int j = lane; j < len; j += 32) acc += row[j] * v[j];
        acc = warp_sum(acc);
        if (lane == 0) {
          pg[r - kk - 1] = b * acc;
          cg[r - kk - 1] = row[0];
        }
      }
    }
    // the reflector, for the back-transformation
    if (kk % (int)G == cta)
      for (int i = tid; i < len; i += nt) A[(size_t)kk * n + kk + 1 + i] = v[i];
    if (!grid_sync(bar, G)) break;
    double pv = 0.0;
    for (int i = tid; i < len; i += nt) {
      const double pi = pg[i];
      wv[i] = pi;
      c[i] = cg[i];
      pv += pi * v[i];
    }
    const double Kf = 0.5 * b * cta_sum(pv, sh);
    for (int i = tid; i < len; i += nt) wv[i] -= Kf * v[i];
    __syncthreads();
    // next column x' = A'[kk+2.., kk+1] from the old column and the same rank-2 formula
    const double v0 = v[0], w0 = wv[0];
    for (int i = tid; i + 1 < len; i += nt) x[i] = c[i + 1] - rank2(v[i + 1], w0, wv[i + 1], v0);
    if (b != 0.0) {
      const int s0 = (kk + 1 - cta + (int)G - 1) / (int)G;
      for (int s = s0 + wid; s < R; s += nw) {
        const int r = s * (int)G + cta;
        if (r >= n) break;
        const int i = r - kk - 1;
        double* row = rows + (size_t)s * n + kk + 1;
        const double vi = v[i], wi = wv[i];
        for (int j = lane; j < len; j += 32) row[j] -= rank2(vi, wv[j], wi, v[j]);
      }
    }
    __syncthreads();
  }
  if (bar->err) {
    if (cta == 0 && tid == 0) *status = 3;
    return;
  }
  if (n >= 2) {
    if ((n - 2) % (int)G == cta && tid == 0) d[n - 2] = rows[(size_t)((n - 2) / (int)G) * n + n - 2];
    if (cta == 0 && tid == 0) e[n - 2] = x[0];
  }
  if ((n - 1) % (int)G == cta && tid == 0) d[n - 1] = rows[(size_t)((n - 1) / (int)G) * n + n - 1];
  if (cta == 0 && tid == 0) e[n - 1] = 0.0;
  if (!grid_sync(bar, G)) {
    if (cta == 0 && tid == 0) *status = 3;
    return;
  }
  coop_tail(A, n, k, w, ZT, d, e, beta, ee, lu, coef, part, zw, rows, bar, status, sh);
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

size_t eigh_coop_aux_bytes(int n) {
  return align_up(4 * sizeof(double) * (size_t)n, 256) + align_up(sizeof(double) * (size_t)n, 256) +
         align_up(sizeof(double) * kCoopMaxCtas, 256) + 256;
}

namespace {
constexpr size_t kSmemMax = 227 * 1024;

// Warps per CTA that hold a vector in the back-transformation.
int coop_zw(int k, int G) { return std::min(8, std::max(1, (k + G - 1) / G)); }

struct CoopPlan {
  int G = 0;         // CTAs (0: one-CTA kernel)
  bool rows = false; // trailing rows in shared memory
  int R = 0;         // row slots per CTA
  int zw = 0;
  size_t smem = 0;
};

size_t plan_smem(int n, int k, int G, bool rows) {
  const int zw = coop_zw(k, G);
  if (rows) return sizeof(double) * (size_t)n * (4 + std::max((n + G - 1) / G, zw));
  return sizeof(double) * (size_t)n * (2 + zw);
}

bool fits(const void* kern, size_t smem, int G, int sms) {
  if (smem > kSmemMax) return false;
  if (smem > 48 * 1024 && cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                              cudaSuccess)
    return false;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem) != cudaSuccess) return false;
  return G <= sms * per_sm;
}

// Multi-SM plan (G = 0: use one CTA).  Knob "eig_ctas" overrides the CTA count; the default
// takes up to one CTA per SM once n is large enough for the reduction to gain from it, and
// keeps the trailing rows in shared memory whenever they fit.
CoopPlan coop_plan(int n, int k) {
  CoopPlan P;
  int forced = knob("eig_ctas");
  if (forced == 1) return P;
  if (forced == 0 && n < 160) return P;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return P;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int G = forced > 1 ? forced : std::min(sms, std::max(32, n / 8));
  G = std::min(G, kCoopMaxCtas);
  if (G < 2) return P;
  size_t sm_rows = plan_smem(n, k, G, true);
  if (fits((const void*)eigh_lowest_coop_smem_kernel, sm_rows, G, sms)) {
    P.G = G;
    P.rows = true;
    P.R = (n + G - 1) / G;
    P.zw = coop_zw(k, G);
    P.smem = sm_rows;
    return P;
  }
  size_t sm_glob = plan_smem(n, k, G, false);
  if (fits((const void*)eigh_lowest_coop_kernel, sm_glob, G, sms)) {
    P.G = G;
    P.zw = coop_zw(k, G);
    P.smem = sm_glob;
  }
  return P;
}
}  // namespace

// aux: coop_aux_bytes(n) of scratch for the multi-SM path.
int eigh_lowest_rows(double* A, int n, int k, double* w, double* ZT, double* scratch, int* status, cudaStream_t s,
                     void* aux) {
  CoopPlan P;
  if (aux) P = coop_plan(n, k);
  if (P.G >= 2) {
    char* p = (char*)aux;
    double* xbuf = (double*)p;
    p += align_up(4 * sizeof(double) * (size_t)n, 256);
    double* coef = (double*)p;
    p += align_up(sizeof(double) * (size_t)n, 256);
    double* part = (double*)p;
    p += align_up(sizeof(double) * kCoopMaxCtas, 256);
    GridBarrier* bar = (GridBarrier*)p;
    grid_barrier_init_kernel<<<1, 32, 0, s>>>(bar, (unsigned)knob("eig_barrier_polls"),
                                              (unsigned)knob("eig_barrier_extra"));
    DF_LAUNCHED("grid_barrier_init_kernel");
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(P.G);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = P.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (P.rows)
      DF_CUDA(cudaLaunchKernelEx(&cfg, eigh_lowest_coop_smem_kernel, A, n, k, w, ZT, scratch, xbuf, P.R, coef, part,
                                 P.zw, bar, status));
    else
      DF_CUDA(cudaLaunchKernelEx(&cfg, eigh_lowest_coop_kernel, A, n, k, w, ZT, scratch, xbuf, coef, part, P.zw, bar,
                                 status));
    return DF_OK;
  }
  eigh_lowest_kernel<<<1, 1024, 0, s>>>(A, n, k, w, ZT, scratch, status);
  DF_LAUNCHED("eigh_lowest_kernel");
  return DF_OK;
}

size_t eigh_full_scratch_doubles(int n) {
  return std::max(eigh_scratch_doubles(n), eigh_lowest_scratch_doubles(n, n));
}

// Full spectrum: the multi-SM solver with k = n where it applies (aux given, n large enough),
// else one CTA with implicit QL.  scratch: eigh_full_scratch_doubles(n).
int eigh_full_rows(double* A, int n, double* w, double* ZT, double* scratch, int* status, cudaStream_t s,
                   void* aux) {
  if (aux && coop_plan(n, n).G >= 2) return eigh_lowest_rows(A, n, n, w, ZT, scratch, status, s, aux);
  return eigh_rows(A, n, w, ZT, scratch, status, s);
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
  z.take<double>(eigh_full_scratch_doubles(n));
  z.take<double>((size_t)n * n);
  z.take<int>(1);
  z.take<char>(eigh_coop_aux_bytes(n));
  return z.used;
}

extern "C" int df_eigh(double* A, int n, double* w, double* Z, void* work, size_t work_bytes, cudaStream_t s) {
  clear_error();
  DF_REQUIRE(A && w && Z && n > 0, DF_ERR_ARG, "df_eigh: bad arguments");
  DF_REQUIRE(work && work_bytes >= df_eigh_work_bytes(n), DF_ERR_NOMEM, "df_eigh: workspace too small");
  Arena a(work, work_bytes);
  double* scratch = a.take<double>(eigh_full_scratch_doubles(n));
  double* ZT = a.take<double>((size_t)n * n);
  int* status = a.take<int>(1);
  void* aux = a.take<char>(eigh_coop_aux_bytes(n));
  DF_TRY(eigh_full_rows(A, n, w, ZT, scratch, status, s, aux));
  DF_TRY(transpose(ZT, n, n, Z, s));
  int h = 0;
  DF_CUDA(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s));
  DF_CUDA(cudaStreamSynchronize(s));
  DF_REQUIRE(h != 3, DF_ERR_TIMEOUT, "df_eigh: a grid barrier of the multi-SM eigensolver timed out");
  DF_REQUIRE(h == 0, DF_ERR_NOCONV, "df_eigh: eigensolver failed (status %d)", h);
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
  DF_REQUIRE(h != 3, DF_ERR_TIMEOUT, "df_eigh_lowest: a grid barrier of the multi-SM eigensolver timed out");
  DF_REQUIRE(h == 0, DF_ERR_NOCONV, "df_eigh_lowest: inverse iteration or re-orthogonalisation failed (%d)", h);
  return DF_OK;
}

DF_BOUNDS_READER(bounds_read_eig)
