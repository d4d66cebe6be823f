// Restricted Hartree-Fock SCF over the DF Fock build, with Pulay DIIS and the
// mixed -> FP64 precision switch, for one molecule (scf_run) or a batch of molecules of
// uneven size (scf_run_batch).  The paper (arXiv 2506.06661) uses DF mean-field methods
// (Section "Density fitting") and names DIIS as the default accelerator (Section
// "Second-Order Self-Consistent Field"); the formulas are the textbook ones:
//   F = h + J[D] - K,  K = K[C_occ] = 1/2 K[D] for D = 2 C_occ C_occ^T,
//   E = 1/2 tr(D (h + F)) + E_nuc,
//   e = X^T (F D S - S D F) X,  X = U s^-1/2 over eigenvalues s > lindep of S,
//   Fbar = sum_i c_i F_i with [[B, -1], [-1, 0]] [c, lam] = [0, -1], B_ij = <e_i, e_j>.
// DIIS works in the orthogonal basis of X: it keeps F' = X^T F X, whose error is
// F' D' - D' F' for D = X D' X^T, and diagonalises the extrapolated F' directly.
// One iteration is a fixed sequence of device work with no host decision inside it: the
// DIIS ring (slot choice, ageing, restart on a singular system) lives in device memory,
// so the iteration is captured once per precision into a CUDA graph and replayed.  The
// host reads one small pinned status block per iteration to decide convergence and the
// precision switch.  A starting density dm0 need not be idempotent (Section "Initial
// Guess for Mean-field Methods"); its exchange matrix is formed from the eigen-
// decomposition dm0 = sum_k n_k u_k u_k^T as K[C+] - K[C-] in an eager first iteration.
#include <algorithm>
#include <chrono>
#include <cstdint>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace dfscf {

constexpr int DIIS_MAX = 16;
constexpr int kDavidsonMax = 24;  // subspace of the stability analysis (vectors)

struct ScfStatus {
  double energy;
  double emax;
  double trDS;
  double idem;   // ||D S D - 2 D||_F / ||D||_F
  double homo, lumo;
  int singular;  // DIIS system had no usable pivot this iteration
  int nonfinite;
  int eig_fail;   // eigensolver status: 0 ok, 3 a grid barrier timed out, else a breakdown
  int tc_timeout; // a bounded wait of the tensor-core exchange gave up in this iteration
  double inc_min_cos2;  // smallest cos^2 of the principal angles between the occupied spaces
                        // of the accumulated K and of the next density (incremental exchange)
  double inc_ssum;      // sum of the sines of those angles (size of the projector change)
  int inc_fail;         // the small eigensolver of the incremental exchange failed
  int pad;
};

struct DiisState {
  int valid[DIIS_MAX];
  long age[DIIS_MAX];
  long tick;
  int nvalid;
  int slot;
  int space;
};

// ---- elementwise / reduction kernels ----------------------------------------------------
// F = h + J - K; status.energy = 1/2 sum D (h + F) + enuc; nonfinite flag.
__global__ void fock_energy_kernel(const double* __restrict__ h, const double* __restrict__ J,
                                   const double* __restrict__ K, const double* __restrict__ D, long nn,
                                   const double* __restrict__ enuc, double* __restrict__ F, ScfStatus* st) {
  __shared__ double sh[32];
  double e = 0.0;
  int bad = 0;
  for (long i = threadIdx.x; i < nn; i += blockDim.x) {
    double f = h[i] + J[i] - K[i];
    F[i] = f;
    e += D[i] * (h[i] + f);
    bad |= !isfinite(f);
  }
  e = block_sum(e, sh);
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    st->energy = 0.5 * e + *enuc;
    st->nonfinite = bad || !isfinite(e);
  }
}

// out = T - T^T (T = F D S), i.e. F D S - S D F.
__global__ void antisym_kernel(const double* __restrict__ T, int n, double* __restrict__ out) {
  long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long)n * n) return;
  int i = (int)(q / n), j = (int)(q % n);
  out[q] = T[q] - T[(size_t)j * n + i];
}

__global__ void absmax_kernel(const double* __restrict__ x, long n, double* out) {
  __shared__ double sh[32];
  double m = 0.0;
  for (long i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(x[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = fmax(t, sh[i]);
    *out = t;
  }
}

// ---- DIIS on device ------------------------------------------------------------------------
__global__ void diis_reset_kernel(DiisState* d, int space) {
  if (threadIdx.x != 0) return;
  for (int k = 0; k < DIIS_MAX; ++k) {
    d->valid[k] = 0;
    d->age[k] = 0;
  }
  d->tick = 0;
  d->nvalid = 0;
  d->slot = 0;
  d->space = space;
}

// Slot for the new (F, e) pair: a free one, else the oldest (at most `space` vectors kept).
__global__ void diis_select_kernel(DiisState* d) {
  if (threadIdx.x != 0) return;
  int slot = -1;
  for (int k = 0; k < d->space; ++k)
    if (!d->valid[k]) {
      slot = k;
      break;
    }
  if (slot < 0) {
    slot = 0;
    for (int k = 1; k < d->space; ++k)
      if (d->age[k] < d->age[slot]) slot = k;
  } else {
    d->nvalid++;
  }
  d->valid[slot] = 1;
  d->age[slot] = ++d->tick;
  d->slot = slot;
}

// Keep only the newest vector (a restart of the extrapolation).
__global__ void diis_keep_newest_kernel(DiisState* d) {
  if (threadIdx.x != 0) return;
  for (int k = 0; k < d->space; ++k) d->valid[k] = (k == d->slot);
  d->nvalid = 1;
}

// Fhist[slot] = F, Ehist[slot] = E (E holds ne = nmo*nmo entries).
// Slot stride nn; F and E both hold ne = nmo^2 entries (orthogonal basis).
__global__ void diis_store_kernel(const DiisState* __restrict__ d, const double* __restrict__ F,
                                  const double* __restrict__ E, double* __restrict__ Fh, double* __restrict__ Eh,
                                  long nn, long ne) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  int slot = d->slot;
  if (i < ne) {
    Fh[DF_IX((size_t)slot * nn + i, (size_t)DIIS_MAX * nn)] = F[i];
    Eh[DF_IX((size_t)slot * nn + i, (size_t)DIIS_MAX * nn)] = E[i];
  }
}

// G[slot][j] = G[j][slot] = <E[slot], E[j]> for valid slots j.
__global__ void diis_gram_kernel(const DiisState* __restrict__ d, const double* __restrict__ Eh, long nn, long ne,
                                 double* __restrict__ G) {
  __shared__ double sh[32];
  int j = blockIdx.x;
  if (j >= d->space || !d->valid[j]) return;
  int slot = d->slot;
  const double* a = Eh + (size_t)slot * nn;
  const double* b = Eh + (size_t)j * nn;
  double s = 0.0;
  for (long i = threadIdx.x; i < ne; i += blockDim.x) s += a[i] * b[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) {
    G[slot * DIIS_MAX + j] = s;
    G[j * DIIS_MAX + slot] = s;
  }
}

// Solve the bordered Pulay system over the valid slots (one lane).  With fewer than two
// vectors, or when no pivot exceeds 1e-14 of the largest entry, the newest vector gets
// coefficient 1; in the singular case the history restarts from the newest vector.
__global__ void diis_solve_kernel(DiisState* d, const double* __restrict__ G, double* __restrict__ coef,
                                  ScfStatus* st) {
  if (threadIdx.x != 0) return;
  int order[DIIS_MAX];
  int m = 0;
  for (int k = 0; k < d->space; ++k)
    if (d->valid[k]) order[m++] = k;
  for (int i = 0; i < DIIS_MAX; ++i) coef[i] = 0.0;
  st->singular = 0;
  if (m < 2) {
    coef[d->slot] = 1.0;
    return;
  }
  double A[DIIS_MAX + 1][DIIS_MAX + 2];
  int dim = m + 1;
  double scale = 0.0;
  for (int i = 0; i < m; ++i) scale = fmax(scale, fabs(G[order[i] * DIIS_MAX + order[i]]));
  if (!(scale > 0.0)) scale = 1.0;
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j < m; ++j) A[i][j] = G[order[i] * DIIS_MAX + order[j]] / scale;
    A[i][m] = -1.0;
    A[m][i] = -1.0;
    A[i][dim] = 0.0;
  }
  A[m][m] = 0.0;
  A[m][dim] = -1.0;
  double amax = 0.0;
  for (int i = 0; i < dim; ++i)
    for (int j = 0; j < dim; ++j) amax = fmax(amax, fabs(A[i][j]));
  bool ok = true;
  for (int c = 0; c < dim && ok; ++c) {
    int p = c;
    for (int r = c + 1; r < dim; ++r)
      if (fabs(A[r][c]) > fabs(A[p][c])) p = r;
    if (!(fabs(A[p][c]) > 1e-14 * amax)) {
      ok = false;
      break;
    }
    if (p != c)
      for (int k = 0; k <= dim; ++k) {
        double t = A[c][k];
        A[c][k] = A[p][k];
        A[p][k] = t;
      }
    for (int r = c + 1; r < dim; ++r) {
      double f = A[r][c] / A[c][c];
      for (int k = c; k <= dim; ++k) A[r][k] -= f * A[c][k];
    }
  }
  if (ok) {
    double x[DIIS_MAX + 1];
    for (int r = dim - 1; r >= 0; --r) {
      double s = A[r][dim];
      for (int k = r + 1; k < dim; ++k) s -= A[r][k] * x[k];
      x[r] = s / A[r][r];
    }
    for (int i = 0; i < m; ++i) {
      if (!isfinite(x[i])) ok = false;
      coef[order[i]] = x[i];
    }
  }
  if (!ok) {
    for (int i = 0; i < DIIS_MAX; ++i) coef[i] = 0.0;
    coef[d->slot] = 1.0;
    for (int k = 0; k < DIIS_MAX; ++k) d->valid[k] = (k == d->slot);
    d->nvalid = 1;
    st->singular = 1;
  }
}

// out = sum_k coef[k] Fh[k] over valid slots.
// out[i] = sum_k c_k Fh[k][i] for i < ne (slot stride nn).
__global__ void diis_combine_kernel(const DiisState* __restrict__ d, const double* __restrict__ Fh, long nn, long ne,
                                    const double* __restrict__ coef, double* __restrict__ out) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ne) return;
  double s = 0.0;
  for (int k = 0; k < d->space; ++k)
    if (d->valid[k]) s += coef[k] * Fh[DF_IX((size_t)k * nn + i, (size_t)DIIS_MAX * nn)];
  out[i] = s;
}

// ---- orbitals ---------------------------------------------------------------------------------
// X[:, j] = U[:, n - nmo + j] / sqrt(s[n - nmo + j]) with U given as rows UT (eigenvector rows).
__global__ void canonical_x_kernel(const double* __restrict__ UT, const double* __restrict__ s, int n, int nmo,
                                   double* __restrict__ X) {
  long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long)n * nmo) return;
  int i = (int)(q / nmo), j = (int)(q % nmo);
  int k = n - nmo + j;
  X[q] = UT[(size_t)k * n + i] / sqrt(s[k]);
}

// C'_occ [nmo][nocc] from eigenvector rows ZT [nmo][nmo] (lowest nocc rows).
__global__ void occ_columns_kernel(const double* __restrict__ ZT, int nmo, int nocc, double* __restrict__ Cp) {
  long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long)nmo * nocc) return;
  int i = (int)(q / nocc), j = (int)(q % nocc);
  Cp[q] = ZT[(size_t)j * nmo + i];
}

// HOMO / LUMO of the last diagonalisation, its eigensolver status and the tensor-core
// exchange's timeout flag (tc_err may be null: an FP64 iteration) into the status block.
__global__ void orbital_status_kernel(const double* __restrict__ eps, int nmo, int nocc, const int* eig_status,
                                      const int* tc_err, ScfStatus* st) {
  if (threadIdx.x != 0) return;
  st->homo = nocc > 0 ? eps[nocc - 1] : 0.0;
  st->lumo = nocc < nmo ? eps[nocc] : 0.0;
  st->eig_fail = *eig_status;
  st->tc_timeout = tc_err ? *tc_err : 0;
}

__global__ void axpy_kernel(double* __restrict__ y, const double* __restrict__ x, long n, double a) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += a * x[i];
}

// For a density Dx in an orthonormal basis (n x n) and T = Dx Dx:
// trDS = tr(Dx) (= tr(D S)), idem = ||Dx Dx - 2 Dx||_F / ||Dx||_F (the same in every
// orthonormal basis).
__global__ void guess_check_kernel(const double* __restrict__ Dx, const double* __restrict__ T, int n,
                                   ScfStatus* st) {
  __shared__ double sh[32];
  double tr = 0.0, r2 = 0.0, d2 = 0.0;
  for (long i = threadIdx.x; i < (long)n * n; i += blockDim.x) {
    if (i / n == i % n) tr += Dx[i];
    double r = T[i] - 2.0 * Dx[i];
    r2 += r * r;
    d2 += Dx[i] * Dx[i];
  }
  tr = block_sum(tr, sh);
  r2 = block_sum(r2, sh);
  d2 = block_sum(d2, sh);
  if (threadIdx.x == 0) {
    st->trDS = tr;
    st->idem = d2 > 0.0 ? sqrt(r2 / d2) : INFINITY;
  }
}

// Columns idx[0..cnt) of eigenvector rows ZT scaled by sqrt(|w|/2): dm0/2 = C+ C+^T - C- C-^T.
__global__ void split_density_kernel(const double* __restrict__ ZT, const double* __restrict__ w, int n,
                                     const int* __restrict__ idx, int cnt, double* __restrict__ Cout) {
  long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long)n * cnt) return;
  int i = (int)(q / cnt), j = (int)(q % cnt);
  int k = idx[j];
  Cout[q] = ZT[(size_t)k * n + i] * sqrt(fabs(w[k]) * 0.5);
}

// ---- incremental mixed-precision exchange -----------------------------------------------
// K is linear in the density, so K[P_new] = K[P_base] + K[P_new - P_base] for the occupied
// projectors P = C' C'^T (orthonormal basis).  The change is factorised as
// U+ U+^T - U- U-^T with factors whose squared norm is about twice the sum of the sines of
// the principal angles between the two occupied spaces: the mixed-precision error of the
// update then shrinks with the change, and the accumulated K keeps the accuracy of the FP64
// build it started from.  Principal vectors: with M = C'_base^T C'_new and
// M^T M = W diag(cos^2) W^T, B = C'_new W and A = C'_base M W (column norms cos) pair up
// column by column.  For unit vectors a, b, the rank-2 matrix b b^T - a a^T equals
// s (p m^T + m p^T) with p = (b + a)/|b + a|, m = (b - a)/|b - a| and s = |b - a||b + a|/2
// the sine of their angle, i.e. u+ u+^T - u- u-^T with u+- = sqrt(s/2) (p +- m).  |b - a|
// is formed from the difference vector itself, so small angles keep FP64 accuracy.

// One CTA per column j of A, B [nmo][k]: U+, U- columns and the sine s_j.
__global__ void principal_pairs_kernel(const double* __restrict__ A, const double* __restrict__ B, int nmo, int k,
                                       double* __restrict__ Up, double* __restrict__ Um, double* __restrict__ sv) {
  __shared__ double sh[32];
  const int j = blockIdx.x;
  double aa = 0.0, bb = 0.0;
  for (int i = threadIdx.x; i < nmo; i += blockDim.x) {
    const double a = A[DF_IX((size_t)i * k + j, (size_t)nmo * k)], b = B[DF_IX((size_t)i * k + j, (size_t)nmo * k)];
    aa += a * a;
    bb += b * b;
  }
  aa = block_sum(aa, sh);
  bb = block_sum(bb, sh);
  const double ia = aa > 0.0 ? 1.0 / sqrt(aa) : 0.0, ib = bb > 0.0 ? 1.0 / sqrt(bb) : 0.0;
  double mm = 0.0, pp = 0.0;
  for (int i = threadIdx.x; i < nmo; i += blockDim.x) {
    const double a = A[(size_t)i * k + j] * ia, b = B[(size_t)i * k + j] * ib;
    mm += (b - a) * (b - a);
    pp += (b + a) * (b + a);
  }
  mm = block_sum(mm, sh);
  pp = block_sum(pp, sh);
  const double nm = sqrt(mm), np = sqrt(pp);
  const bool live = aa > 0.0 && bb > 0.0 && nm > 1e-300 && np > 1e-300;
  const double sj = live ? 0.5 * nm * np : 0.0;
  const double f = sqrt(0.5 * sj), inm = live ? 1.0 / nm : 0.0, inp = live ? 1.0 / np : 0.0;
  for (int i = threadIdx.x; i < nmo; i += blockDim.x) {
    const double a = A[(size_t)i * k + j] * ia, b = B[(size_t)i * k + j] * ib;
    const double pv = (b + a) * inp, mv = (b - a) * inm;
    Up[DF_IX((size_t)i * k + j, (size_t)nmo * k)] = f * (pv + mv);
    Um[DF_IX((size_t)i * k + j, (size_t)nmo * k)] = f * (pv - mv);
  }
  if (threadIdx.x == 0) sv[j] = sj;
}

// K += Kp - Km.
__global__ void kacc_kernel(double* __restrict__ K, const double* __restrict__ Kp, const double* __restrict__ Km,
                            long n) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) K[i] += Kp[i] - Km[i];
}

// Smallest cos^2 (ascending eigenvalues c2) and sum of the sines of the principal angles into
// the status block, with the small eigensolver's status.
__global__ void inc_status_kernel(const double* __restrict__ c2, int k, const int* __restrict__ eig_status,
                                  ScfStatus* st) {
  __shared__ double sh[32];
  double t = 0.0;
  for (int j = threadIdx.x; j < k; j += blockDim.x) t += sqrt(fmax(0.0, 1.0 - fmin(1.0, c2[j])));
  t = block_sum(t, sh);
  if (threadIdx.x == 0) {
    st->inc_min_cos2 = k > 0 ? c2[0] : 1.0;
    st->inc_ssum = t;
    st->inc_fail = *eig_status;
  }
}

// ---- second-order SCF (Newton steps on the orbital rotation) ----------------------------
// The paper's SOSCF section: after DIIS has stalled, an exact-gradient Newton solver with an
// approximate orbital Hessian converges where DIIS oscillates.  Closed-shell form in the
// orthonormal basis of X, with the full orbital set C' = [C'_o, C'_v] and the Fock matrix
// F_mo = C'^T F' C': gradient F_vo (the energy gradient divided by 4), Hessian product
//   (H v)_ai = (F_vv v - v F_oo)_ai + (C_v^T dF[v] C_o)_ai,  dF = J[dD] - 1/2 K[dD],
//   dD = 2 (L R^T + R L^T),  L = X C'_v v,  R = X C'_o = C_occ,
// solved for H kappa = -F_vo by preconditioned conjugate gradients (diagonal
// F_aa - F_ii, floored at 0.05) from kappa = 0 with device-side scalars, truncated as in
// Steihaug's method at a trust radius |kappa| <= 0.5 or at non-positive curvature (near a
// saddle point the step then follows the downhill direction).  K[dD] comes from
// two ordinary exchange builds: F+- = L/t +- t R, F+ F+^T - F- F-^T = 2 (L R^T + R L^T), with
// t = (|L| / |R|)^(1/2) so that both factors are of the size of the change.  The step is
// capped at 0.3 rad per element, and the orbitals rotate exactly by exp([[0, -k^T], [k, 0]]):
// with k^T k = V diag(s^2) V^T,
//   C'_o <- C'_o V cos(s) V^T + C'_v k V sinc(s) V^T,
//   C'_v <- C'_v (1 + k V ((cos(s) - 1)/s^2) V^T k^T) - C'_o V sinc(s) V^T k^T.

// g = F_vo and the preconditioner h_ai = max(F_aa - F_ii, 0.05), both [nvir][nocc].
__global__ void soscf_grad_kernel(const double* __restrict__ Fmo, int nmo, int nocc, double* __restrict__ g,
                                  double* __restrict__ h) {
  const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int nvir = nmo - nocc;
  if (q >= (long)nvir * nocc) return;
  const int a = (int)(q / nocc), i = (int)(q % nocc);
  g[q] = Fmo[DF_IX((size_t)(nocc + a) * nmo + i, (size_t)nmo * nmo)];
  h[q] = fmax(Fmo[DF_IX((size_t)(nocc + a) * nmo + nocc + a, (size_t)nmo * nmo)] -
                  Fmo[DF_IX((size_t)i * nmo + i, (size_t)nmo * nmo)], 0.05);
}

// *out = <a, b> over n entries (one CTA).
__global__ void dot_kernel(const double* __restrict__ a, const double* __restrict__ b, long n,
                           double* __restrict__ out) {
  __shared__ double sh[32];
  double t = 0.0;
  for (long i = threadIdx.x; i < n; i += blockDim.x) t += a[i] * b[i];
  t = block_sum(t, sh);
  if (threadIdx.x == 0) *out = t;
}

// CG start from x = 0: r = -g, z = r / h, p = z.
__global__ void cg_start_kernel(double* __restrict__ x, double* __restrict__ r, double* __restrict__ z,
                                double* __restrict__ p, const double* __restrict__ g, const double* __restrict__ h,
                                long n) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  x[i] = 0.0;
  r[i] = -g[i];
  z[i] = -g[i] / h[i];
  p[i] = z[i];
}

// Steihaug's truncated CG inside the trust region |x| <= Delta (2-norm): the step length is
// alpha = rz / pAp, unless the curvature along p is not positive or the step would leave the
// region; then x moves along p to the boundary and the iteration stops (later steps add
// nothing).  sc: [0] rz, [1] pAp, [6] x.x, [7] x.p, [8] p.p, [9] stopped, [10] Delta,
// [11] the step length used.
__global__ void cg_decide_kernel(double* __restrict__ sc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (sc[9] != 0.0) {
    sc[11] = 0.0;
    return;
  }
  const double rz = sc[0], pAp = sc[1], xx = sc[6], xp = sc[7], pp = sc[8], D = sc[10];
  const double alpha = pAp > 0.0 ? rz / pAp : 0.0;
  if (pAp > 0.0 && xx + 2.0 * alpha * xp + alpha * alpha * pp <= D * D) {
    sc[11] = alpha;
    return;
  }
  // boundary: |x + tau p| = Delta, tau >= 0
  double tau = 0.0;
  if (pp > 0.0) tau = (-xp + sqrt(fmax(xp * xp - pp * (xx - D * D), 0.0))) / pp;
  sc[11] = tau;
  sc[9] = 1.0;
}

// x += a p; r -= a Ap; z = r / h with a = sc[11].
__global__ void cg_step_kernel(double* __restrict__ x, double* __restrict__ r, double* __restrict__ z,
                               const double* __restrict__ p, const double* __restrict__ Ap,
                               const double* __restrict__ h, long n, const double* __restrict__ sc) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double alpha = sc[11];
  x[i] += alpha * p[i];
  const double ri = r[i] - alpha * Ap[i];
  r[i] = ri;
  z[i] = ri / h[i];
}

// Start of a Newton step's CG: not stopped, trust radius Delta.
__global__ void cg_reset_kernel(double* __restrict__ sc, double Delta) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  sc[9] = 0.0;
  sc[10] = Delta;
}

// p = z + beta p, beta = rz_new / rz (sc[2] / sc[0]).
__global__ void cg_dir_kernel(double* __restrict__ p, const double* __restrict__ z, long n,
                              const double* __restrict__ sc) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double beta = sc[0] > 0.0 ? sc[2] / sc[0] : 0.0;
  p[i] = z[i] + beta * p[i];
}

__global__ void copy_scalar_kernel(double* __restrict__ dst, const double* __restrict__ src) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *dst = *src;
}

// F+- = L / t +- t R with t = (|L|^2 / |R|^2)^(1/4) (sc[3] = |L|^2, sc[4] = |R|^2).
__global__ void pm_factors_kernel(const double* __restrict__ L, const double* __restrict__ R, long n,
                                  const double* __restrict__ sc, double* __restrict__ Fp, double* __restrict__ Fm) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double t = (sc[3] > 0.0 && sc[4] > 0.0) ? sqrt(sqrt(sc[3] / sc[4])) : 1.0;
  const double a = L[i] / t, b = t * R[i];
  Fp[i] = a + b;
  Fm[i] = a - b;
}

// out = 2 (T + T^T) for n x n T.
__global__ void sym2_kernel(const double* __restrict__ T, int n, double* __restrict__ out) {
  const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long)n * n) return;
  const int i = (int)(q / n), j = (int)(q % n);
  out[q] = 2.0 * (T[q] + T[(size_t)j * n + i]);
}

// dF = dJ - 1/2 (dK+ - dK-), in place of dJ.
__global__ void response_fock_kernel(double* __restrict__ dJ, const double* __restrict__ dKp,
                                     const double* __restrict__ dKm, long n) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dJ[i] -= 0.5 * (dKp[i] - dKm[i]);
}

// Cap the step: x *= cap / max|x| when max|x| (sc[5]) exceeds cap.
__global__ void cap_step_kernel(double* __restrict__ x, long n, const double* __restrict__ sc, double cap) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && sc[5] > cap) x[i] *= cap / sc[5];
}

// Pc = V cos(s) V^T, Ps = V sinc(s) V^T, Pd = V ((cos(s) - 1)/s^2) V^T from the eigenvector
// rows Vrow [k][k] and eigenvalues s^2 of k^T k (series below s = 1e-4).
__global__ void rotation_mats_kernel(const double* __restrict__ Vrow, const double* __restrict__ s2, int k,
                                     double* __restrict__ Pc, double* __restrict__ Ps, double* __restrict__ Pd) {
  const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long)k * k) return;
  const int a = (int)(q / k), b = (int)(q % k);
  double c = 0.0, sn = 0.0, d = 0.0;
  for (int j = 0; j < k; ++j) {
    const double sq = fmax(s2[j], 0.0), sg = sqrt(sq);
    double fc, fs, fd;
    if (sg < 1e-4) {
      fc = 1.0 - 0.5 * sq;
      fs = 1.0 - sq / 6.0;
      fd = -0.5 + sq / 24.0;
    } else {
      fc = cos(sg);
      fs = sin(sg) / sg;
      fd = (fc - 1.0) / sq;
    }
    const double vv = Vrow[DF_IX((size_t)j * k + a, (size_t)k * k)] * Vrow[DF_IX((size_t)j * k + b, (size_t)k * k)];
    c += vv * fc;
    sn += vv * fs;
    d += vv * fd;
  }
  Pc[q] = c;
  Ps[q] = sn;
  Pd[q] = d;
}

__global__ void add_identity_kernel(double* __restrict__ A, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) A[(size_t)i * n + i] += 1.0;
}

// HOMO / LUMO estimates (diagonal of F_mo) and statuses after a Newton step.
__global__ void soscf_status_kernel(const double* __restrict__ Fmo, int nmo, int nocc, const int* k_status,
                                    const int* tc_err, ScfStatus* st) {
  if (threadIdx.x != 0) return;
  double homo = -INFINITY, lumo = INFINITY;
  for (int i = 0; i < nocc; ++i) homo = fmax(homo, Fmo[(size_t)i * nmo + i]);
  for (int a = nocc; a < nmo; ++a) lumo = fmin(lumo, Fmo[(size_t)a * nmo + a]);
  st->homo = homo;
  st->lumo = nocc < nmo ? lumo : 0.0;
  st->eig_fail = *k_status;
  st->tc_timeout = tc_err ? *tc_err : 0;
}

static unsigned blocks_for(long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// ---- per-molecule workspace --------------------------------------------------------------
struct ScfWork {
  double *L, *pair_tab, *S, *h, *V, *X, *F, *Fo, *Cp, *J, *K, *D, *Dprev, *Cocc, *Cprev, *Cchunk, *T1, *T2, *E, *Fp,
      *ZT, *eps, *Fhist, *Ehist, *G, *coef, *eig_scratch, *enuc, *maxdiag;
  int *eig_status, *chol_status, *idx;
  // incremental mixed exchange: C' the accumulated K belongs to, M = C'_base^T C'_new, the
  // eigen-decomposition of M^T M (rows of Winc, ascending cos^2 in cinc), the principal
  // vectors A, B and the two factors of the projector change (orthonormal basis, then AO)
  double *Cbase, *Minc, *Tinc, *Winc, *cinc, *MW, *Ainc, *Binc, *Up, *Um, *Uao_p, *Uao_m, *sinc;
  int* inc_status;
  // second-order SCF: the full orbital set C'_all (columns; occupied first), its Fock matrix,
  // the extrapolated F' kept for the switch, CG vectors over (virtual, occupied) pairs, the
  // trial-density response and the small matrices of the exact rotation exp(kappa)
  double *Fbar, *Call, *Call2, *Fmo, *Lv, *cg_g, *cg_h, *cg_x, *cg_r, *cg_z, *cg_p, *cg_Ap, *Lf, *Lfp, *Lfm, *dD,
      *dJ, *dK1, *dK2, *cg_s, *kk, *kVrow, *ksig, *Pc, *Ps, *Pd, *ktmp, *KPdK;
  int* k_status;
  double* dav;  // Davidson subspace of the stability analysis: V, H V [kDavidsonMax][nvir * nocc], G, scalars
  char* guess_ws;      // learned-guess prediction (guess_density), 5 basis functions per centre
  size_t guess_bytes;
  void* eig_aux;  // p vector and grid barrier of the multi-SM eigensolver
  ScfStatus* st;
  DiisState* diis;
  void* B;
  JKWork jk;
};

static void scf_layout(int nao, int naux, int nocc, int precision, Arena* a, Sizer* z, ScfWork* w) {
  size_t nn = (size_t)nao * nao;
#define TAKE(T, ptr, count) \
  if (a) ptr = a->take<T>(count); else z->take<T>(count);
  TAKE(double, w->L, (size_t)naux * naux);
  // learned starting density from the geometry (scf_opts.guess_params), 5 functions per centre
  w->guess_bytes = nao % 5 == 0 ? guess_density_work_bytes(nao / 5) : 0;
  w->guess_ws = nullptr;
  if (w->guess_bytes) TAKE(char, w->guess_ws, w->guess_bytes);
  TAKE(double, w->pair_tab, 5 * (size_t)npair_of(nao));
  TAKE(double, w->S, nn);
  TAKE(double, w->h, nn);
  TAKE(double, w->V, nn);
  TAKE(double, w->X, nn);
  TAKE(double, w->F, nn);
  TAKE(double, w->Fo, nn);
  TAKE(double, w->Cp, (size_t)nao * std::max(nocc, 1));
  TAKE(double, w->J, nn);
  TAKE(double, w->K, nn);
  TAKE(double, w->D, nn);
  TAKE(double, w->Dprev, nn);
  TAKE(double, w->Cocc, (size_t)nao * nocc);
  TAKE(double, w->Cprev, (size_t)nao * nocc);
  TAKE(double, w->Cchunk, (size_t)nao * nocc);
  TAKE(double, w->T1, nn);
  TAKE(double, w->T2, nn);
  TAKE(double, w->E, nn);
  TAKE(double, w->Fp, nn);
  TAKE(double, w->ZT, nn);
  TAKE(double, w->eps, nao);
  TAKE(double, w->Fhist, DIIS_MAX * nn);
  TAKE(double, w->Ehist, DIIS_MAX * nn);
  TAKE(double, w->G, DIIS_MAX * DIIS_MAX);
  TAKE(double, w->coef, DIIS_MAX);
  TAKE(double, w->eig_scratch, eigh_full_scratch_doubles(nao));
  TAKE(double, w->enuc, 1);
  TAKE(double, w->maxdiag, 1);
  TAKE(int, w->eig_status, 1);
  TAKE(char, w->eig_aux, eigh_coop_aux_bytes(nao));
  TAKE(int, w->chol_status, 1);
  TAKE(int, w->idx, nao);
  {
    const size_t oc = (size_t)std::max(nocc, 1);
    TAKE(double, w->Cbase, (size_t)nao * oc);
    TAKE(double, w->Minc, oc * oc);
    TAKE(double, w->Tinc, oc * oc);
    TAKE(double, w->Winc, oc * oc);
    TAKE(double, w->cinc, oc);
    TAKE(double, w->MW, oc * oc);
    TAKE(double, w->Ainc, (size_t)nao * oc);
    TAKE(double, w->Binc, (size_t)nao * oc);
    TAKE(double, w->Up, (size_t)nao * oc);
    TAKE(double, w->Um, (size_t)nao * oc);
    TAKE(double, w->Uao_p, (size_t)nao * oc);
    TAKE(double, w->Uao_m, (size_t)nao * oc);
    TAKE(double, w->sinc, oc);
    TAKE(int, w->inc_status, 1);
    const size_t vo = (size_t)nao * oc;  // (virtual, occupied) pairs: at most nao * nocc
    TAKE(double, w->Fbar, nn);
    TAKE(double, w->Call, nn);
    TAKE(double, w->Call2, nn);
    TAKE(double, w->Fmo, nn);
    TAKE(double, w->Lv, nn);
    TAKE(double, w->cg_g, vo);
    TAKE(double, w->cg_h, vo);
    TAKE(double, w->cg_x, vo);
    TAKE(double, w->cg_r, vo);
    TAKE(double, w->cg_z, vo);
    TAKE(double, w->cg_p, vo);
    TAKE(double, w->cg_Ap, vo);
    TAKE(double, w->Lf, vo);
    TAKE(double, w->Lfp, vo);
    TAKE(double, w->Lfm, vo);
    TAKE(double, w->dD, nn);
    TAKE(double, w->dJ, nn);
    TAKE(double, w->dK1, nn);
    TAKE(double, w->dK2, nn);
    TAKE(double, w->cg_s, 32);
    TAKE(double, w->kk, oc * oc);
    TAKE(double, w->kVrow, oc * oc);
    TAKE(double, w->ksig, oc);
    TAKE(double, w->Pc, oc * oc);
    TAKE(double, w->Ps, oc * oc);
    TAKE(double, w->Pd, oc * oc);
    TAKE(double, w->ktmp, vo);
    TAKE(double, w->KPdK, nn);
    TAKE(int, w->k_status, 1);
    TAKE(double, w->dav, (size_t)2 * kDavidsonMax * vo + (size_t)kDavidsonMax * kDavidsonMax + 8);
  }
  TAKE(ScfStatus, w->st, 1);
  TAKE(DiisState, w->diis, 1);
  if (a) w->B = a->take<char>(df_B_bytes(nao, naux, precision)); else z->take<char>(df_B_bytes(nao, naux, precision));
#undef TAKE
  w->jk = jk_work_layout(nao, naux, nocc, precision, a, z, true);
}

static int eig_rows(double* A, int n, double* w, double* ZT, ScfWork& W, cudaStream_t s) {
  return eigh_full_rows(A, n, w, ZT, W.eig_scratch, W.eig_status, s, W.eig_aux);
}

// Occupied orbitals of the orthogonal-basis Fock matrix W.Fp [nmo][nmo] (destroyed):
// C'_occ into W.Cp [nmo][nocc], C_occ = X C'_occ, D = 2 C C^T.
static int diagonalize_orth(int nao, int nmo, int nocc, ScfWork& W, cudaStream_t s) {
  // only the occupied orbitals and the LUMO are needed: k lowest eigenpairs when k << nmo
  const int k = std::min(nocc + 1, nmo);
  {
    ProfScope ps("scf_eigensolver", s);
    if (nmo >= 16 && 2 * k <= nmo)
      DF_TRY(eigh_lowest_rows(W.Fp, nmo, k, W.eps, W.ZT, W.eig_scratch, W.eig_status, s, W.eig_aux));
    else
      DF_TRY(eig_rows(W.Fp, nmo, W.eps, W.ZT, W, s));
  }
  occ_columns_kernel<<<blocks_for((long)nmo * nocc), 256, 0, s>>>(W.ZT, nmo, nocc, W.Cp);
  DF_LAUNCHED("occ_columns_kernel");
  DF_TRY(dgemm(false, false, nao, nocc, nmo, 1.0, W.X, nmo, 0, W.Cp, nocc, 0, 0.0, W.Cocc, nocc, 0, 1, s, 0, 0));
  DF_TRY(dgemm(false, true, nao, nao, nocc, 2.0, W.Cocc, nocc, 0, W.Cocc, nocc, 0, 0.0, W.D, nao, 0, 1, s, 0, 0));
  return DF_OK;
}

// F' = X^T Fm X into `out` [nmo][nmo] (T1 as scratch).
static int to_orth(const double* Fm, int nao, int nmo, ScfWork& W, double* out, cudaStream_t s) {
  DF_TRY(dgemm(false, false, nao, nmo, nao, 1.0, Fm, nao, 0, W.X, nmo, 0, 0.0, W.T1, nmo, 0, 1, s, 0, 0));
  DF_TRY(dgemm(true, false, nmo, nmo, nao, 1.0, W.X, nmo, 0, W.T1, nmo, 0, 0.0, out, nmo, 0, 1, s, 0, 0));
  return DF_OK;
}

// Occupied coefficients from an AO-basis Fock-like matrix.
static int diagonalize_fock(const double* Fm, int nao, int nmo, int nocc, ScfWork& W, cudaStream_t s) {
  DF_TRY(to_orth(Fm, nao, nmo, W, W.Fp, s));
  return diagonalize_orth(nao, nmo, nocc, W, s);
}

// ---- one molecule's SCF state machine ----------------------------------------------------------
// Host state of the stability analysis (Davidson; see dav_begin / dav_advance).
struct DavState {
  enum Stage { OFF, RITZ } stage = OFF;
  int m = 0, have = 0, row0 = 0, products = 0, kmax = 0, max_products = 0;
  bool added = false;    // the newest vector came from a correction (its norm is checked)
  bool have_rr = false;  // the read-back carries the residual of the previous Ritz pair
  double theta = NAN, mode_scale = 0.0;
  std::vector<double> Hs, y;
};

struct ScfMol {
  df_molecule mol{};
  scf_opts opt{};
  int nao = 0, naux = 0, nocc = 0, nmo = 0;
  ScfWork W{};
  cudaStream_t s = nullptr;
  ScfStatus* hst = nullptr;   // pinned host mirror of W.st
  int prec = DF_FP64;
  bool switched = false;
  bool first_dm0 = false;
  int fp64_done = 0;
  double e_old = 0.0;
  bool have_old = false;
  double best_err = INFINITY;  // smallest max|e| of the mixed phase so far
  int stall = 0;               // mixed iterations without a 10% gain on best_err
  // Incremental mixed exchange (mixed precision with the knob "mixed_incremental"): full
  // mixed builds until max|e| < 1e-3 (or the switch rules), one FP64 build as the base of
  // the accumulated K, updates from the change of the occupied projector until converged,
  // then n_fp64_final FP64 iterations.  A base is rebuilt when the occupied space turned by
  // more than 60 degrees in one step or the updates stall.
  bool inc = false;
  // Second-order steps (knob "soscf"): once the DIIS error has not improved by 10% for 12
  // iterations with an accurate Fock matrix, every later iteration takes a Newton step
  // instead of the DIIS extrapolation and diagonalisation.
  bool soscf_on = false;      // enabled for this molecule (F' is kept for the switch)
  bool soscf = false;         // Newton steps active
  bool soscf_pending = false; // switch before the next launch
  double d_best = INFINITY;
  int d_stall = 0;
  enum KPhase { KP_FULL, KP_BASE, KP_INCR, KP_FINAL } kp = KP_FULL;
  int rebases = 0;
  double inc_best = INFINITY;
  int inc_stall = 0;
  bool done = false;
  int iter_limit = 0;         // iterations allowed so far (max_cycle, renewed by a saddle escape)
  int rc = DF_OK;
  cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};
  scf_result res{};
  const double* dm0 = nullptr;
  double* D_out = nullptr;
  double* C_out = nullptr;
  double* mo_out = nullptr;
  // Set-up runs as asynchronous phases so that a batch never blocks on one molecule:
  // SETUP (integrals, metric, B, eig(S) enqueued) -> ORTHO (host reads eig(S)) ->
  // GUESS_CHECK (only with dm0) -> READY -> ITER (an iteration is in flight) -> [STAB (the
  // stability analysis, knob "stability"; back to ITER after a saddle escape)] -> DONE.
  enum Phase { SETUP, GUESS_CHECK, READY, DM0_EIG, ITER, STAB, DONE } phase = SETUP;
  bool outputs_done = false;  // outputs already written for the current solution
  double* h_eps = nullptr;  // pinned: eigenvalues of S, then E_nuc (nao + 1 doubles); then of dm0
  int* h_ints = nullptr;    // pinned: [0] eigensolver status, [1] Cholesky status
  double* h_dav = nullptr;  // pinned: read-backs of the stability analysis
  DavState dav;
  std::vector<int> dm0_ids; // eigenvalue indices of the dm0 split (source of an async copy)

  ~ScfMol() {
    for (auto& g : graph)
      if (g) cudaGraphExecDestroy(g);
  }
};

// Phase SETUP: enqueue integrals, metric Cholesky, B and eig(S), plus asynchronous copies of
// what the host needs next.  Does not synchronise.
static int setup_launch(ScfMol& M) {
  const df_molecule* mol = &M.mol;
  cudaStream_t s = M.s;
  ScfWork& W = M.W;
  const int nao = M.nao, naux = M.naux;
  const long nn = (long)nao * nao;
  memset(&M.res, 0, sizeof(M.res));
  DF_TRY(umma_prepare());
  DF_TRY(launch_int1e(mol->ao_xyz, mol->ao_exp, nao, mol->xyz, mol->charges, mol->natm, W.S, W.h, W.V, s));
  axpy_kernel<<<blocks_for(nn), 256, 0, s>>>(W.h, W.V, nn, 1.0);
  DF_LAUNCHED("axpy_kernel");
  DF_TRY(launch_enuc(mol->xyz, mol->charges, mol->natm, W.enuc, s));
  DF_TRY(launch_int2c(mol->aux_xyz, mol->aux_exp, naux, W.L, s));
  DF_TRY(cholesky_inplace(W.L, naux, W.chol_status, W.maxdiag, 1e-14, s));
  DF_TRY(build_B(mol->ao_xyz, mol->ao_exp, nao, mol->aux_xyz, mol->aux_exp, naux, W.L, M.opt.precision, W.B,
                 W.pair_tab, s));
  DF_CUDA(cudaMemcpyAsync(W.T1, W.S, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
  DF_TRY(eig_rows(W.T1, nao, W.eps, W.ZT, W, s));
  DF_CUDA(cudaMemcpyAsync(M.h_eps, W.eps, sizeof(double) * nao, cudaMemcpyDeviceToHost, s));
  DF_CUDA(cudaMemcpyAsync(M.h_ints, W.eig_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  DF_CUDA(cudaMemcpyAsync(M.h_ints + 1, W.chol_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  DF_CUDA(cudaMemcpyAsync(M.h_eps + nao, W.enuc, sizeof(double), cudaMemcpyDeviceToHost, s));
  M.phase = ScfMol::SETUP;
  return DF_OK;
}

// use_dm0 with an idempotent dm0 (orbitals): start from its occupied orbitals.  With
// P = Dx / 2 (Dx = X^T S dm0 S X, left in W.Fp by the guess check) and H = X^T h X, the matrix
//   A = -2 P + delta (H - P H - H P + 2 P H P),   delta = 1 / (2 ||H||_F),
// commutes with P; its occupied eigenvalues lie in -2 + delta spec(H) and its virtual ones in
// delta spec(H), at least 1 apart, so its nocc lowest eigenvectors span range(P) exactly.
// The core-Hamiltonian term splits the nocc-fold eigenvalue of -Dx (a degenerate cluster
// that inverse iteration resolves only to ~1e-8) into distinct ones.  The first iteration
// is then an ordinary one.  A general dm0 keeps the eager first iteration with the exchange
// of its eigen-decomposition.
__global__ void frobenius_kernel(const double* __restrict__ A, long n, double* __restrict__ out) {
  __shared__ double sh[32];
  double t = 0.0;
  for (long i = threadIdx.x; i < n; i += blockDim.x) t += A[i] * A[i];
  t = block_sum(t, sh);
  if (threadIdx.x == 0) *out = sqrt(t);
}

// A (in place of Dx) = -Dx + delta (H - PH - (PH)^T + 2 PHP), P = Dx / 2.
__global__ void shifted_projector_kernel(double* __restrict__ Dx, const double* __restrict__ H,
                                         const double* __restrict__ PH, const double* __restrict__ PHP, int n,
                                         const double* __restrict__ hnorm) {
  long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long)n * n) return;
  const int i = (int)(q / n), j = (int)(q % n);
  const double delta = 0.5 / fmax(*hnorm, 1e-300);
  Dx[q] = -Dx[q] + delta * (H[q] - PH[q] - PH[(size_t)j * n + i] + 2.0 * PHP[q]);
}

static int orbitals_from_determinant(ScfMol& M) {
  ScfWork& W = M.W;
  cudaStream_t s = M.s;
  const int nao = M.nao, nmo = M.nmo;
  const long ne = (long)nmo * nmo;
  DF_TRY(to_orth(W.h, nao, nmo, W, W.E, s));
  DF_TRY(dgemm(false, false, nmo, nmo, nmo, 0.5, W.Fp, nmo, 0, W.E, nmo, 0, 0.0, W.J, nmo, 0, 1, s, 0, 0));
  DF_TRY(dgemm(false, false, nmo, nmo, nmo, 0.5, W.J, nmo, 0, W.Fp, nmo, 0, 0.0, W.K, nmo, 0, 1, s, 0, 0));
  frobenius_kernel<<<1, 1024, 0, s>>>(W.E, ne, W.coef);
  DF_LAUNCHED("frobenius_kernel");
  shifted_projector_kernel<<<blocks_for(ne), 256, 0, s>>>(W.Fp, W.E, W.J, W.K, nmo, W.coef);
  DF_LAUNCHED("shifted_projector_kernel");
  return diagonalize_orth(nao, nmo, M.nocc, W, s);
}

static int finish_guess(ScfMol& M, bool use_dm0, bool orbitals) {
  ScfWork& W = M.W;
  const long nn = (long)M.nao * M.nao;
  if (use_dm0 && orbitals) {
    DF_TRY(orbitals_from_determinant(M));
    use_dm0 = false;
  } else if (use_dm0) {
    DF_CUDA(cudaMemcpyAsync(W.D, M.dm0, sizeof(double) * nn, cudaMemcpyDeviceToDevice, M.s));
  } else {
    DF_TRY(diagonalize_fock(W.h, M.nao, M.nmo, M.nocc, W, M.s));
  }
  diis_reset_kernel<<<1, 32, 0, M.s>>>(W.diis, M.opt.diis_space);
  DF_LAUNCHED("diis_reset_kernel");
  M.inc = M.opt.precision == DF_MIXED && knob("mixed_incremental") != 0;
  M.soscf_on = knob("soscf") != 0 && M.nocc < M.nmo;
  if (M.inc) DF_CUDA(cudaMemsetAsync(W.Cbase, 0, sizeof(double) * (size_t)M.nmo * M.nocc, M.s));
  M.first_dm0 = use_dm0;
  M.prec = M.opt.precision;
  M.switched = (M.prec == DF_FP64);
  M.phase = ScfMol::READY;
  return DF_OK;
}

// After SETUP completed on the stream: canonical orthogonalisation, then either the core
// guess (-> READY) or the enqueued dm0 checks (-> GUESS_CHECK).
static int setup_orthogonalize(ScfMol& M) {
  ScfWork& W = M.W;
  cudaStream_t s = M.s;
  const int nao = M.nao, nocc = M.nocc;
  const long nn = (long)nao * nao;
  M.res.e_nuc = M.h_eps[nao];
  DF_REQUIRE(M.h_ints[1] < 0, DF_ERR_NOT_SPD, "scf: auxiliary metric not positive definite at pivot %d", M.h_ints[1]);
  DF_REQUIRE(M.h_ints[0] != 3, DF_ERR_TIMEOUT, "scf: a grid barrier of the eigensolver timed out on S");
  DF_REQUIRE(M.h_ints[0] == 0, DF_ERR_NOCONV, "scf: eigensolver failed on S");
  int nmo = 0;
  for (int i = 0; i < nao; ++i) nmo += M.h_eps[i] > M.opt.lindep;
  DF_REQUIRE(nmo >= nocc, DF_ERR_ARG, "scf: only %d orbitals above lindep for %d occupied", nmo, nocc);
  M.nmo = nmo;
  M.res.nmo = nmo;
  canonical_x_kernel<<<blocks_for((long)nao * nmo), 256, 0, s>>>(W.ZT, W.eps, nao, nmo, W.X);
  DF_LAUNCHED("canonical_x_kernel");
  if (!M.dm0 && M.opt.guess_params && W.guess_bytes && 5 * M.mol.natm == nao) {
    // learned starting density: S^-1/2 from the eigen-decomposition of S above (the same
    // eigenvalues as X), the network's Loewdin-basis blocks, dm0 = S^-1/2 Dt S^-1/2 in W.J;
    // then the same checks as a caller's dm0
    DF_TRY(lowdin_power(W.ZT, W.eps, nao, M.opt.lindep, -0.5, W.T1, W.K, s));
    DF_TRY(guess_density(M.opt.guess_params, M.mol.xyz, M.mol.natm, M.mol.nelec, W.K, W.J, W.guess_ws,
                         W.guess_bytes, s));
    M.dm0 = W.J;
  }
  if (!M.dm0) return finish_guess(M, false, false);
  // dm0 in the orthonormal basis X: Dx = X^T S dm0 S X; then the checks on Dx and Dx Dx
  DF_TRY(dgemm(false, false, nao, nao, nao, 1.0, W.S, nao, 0, M.dm0, nao, 0, 0.0, W.T1, nao, 0, 1, s, 0, 0));
  DF_TRY(dgemm(false, false, nao, nao, nao, 1.0, W.T1, nao, 0, W.S, nao, 0, 0.0, W.T2, nao, 0, 1, s, 0, 0));
  DF_TRY(dgemm(false, false, nao, nmo, nao, 1.0, W.T2, nao, 0, W.X, nmo, 0, 0.0, W.T1, nmo, 0, 1, s, 0, 0));
  DF_TRY(dgemm(true, false, nmo, nmo, nao, 1.0, W.X, nmo, 0, W.T1, nmo, 0, 0.0, W.Fp, nmo, 0, 1, s, 0, 0));
  DF_TRY(dgemm(false, false, nmo, nmo, nmo, 1.0, W.Fp, nmo, 0, W.Fp, nmo, 0, 0.0, W.T2, nmo, 0, 1, s, 0, 0));
  guess_check_kernel<<<1, 1024, 0, s>>>(W.Fp, W.T2, nmo, W.st);
  DF_LAUNCHED("guess_check_kernel");
  (void)nn;
  DF_CUDA(cudaMemcpyAsync(M.hst, W.st, sizeof(ScfStatus), cudaMemcpyDeviceToHost, s));
  M.phase = ScfMol::GUESS_CHECK;
  return DF_OK;
}

// After GUESS_CHECK completed: accept dm0 when its electron count is within 5% and its
// idempotency error in the orthonormal basis, ||Dx Dx - 2 Dx|| / ||Dx||, is below
// knob "guess_idem_max" / 100 (default 2); else fall back to the core guess.
static int setup_guess(ScfMol& M) {
  const ScfStatus& h = *M.hst;
  int ne = M.mol.nelec;
  bool use = std::isfinite(h.trDS) && fabs(h.trDS - ne) / ne < 0.05 && h.idem < knob("guess_idem_max") / 100.0;
  M.res.guess = use ? 1 : 2;
  // an idempotent dm0 (the learned guess is one): start from its orbitals
  return finish_guess(M, use, use && h.idem < 1e-6);
}

// Whole set-up for one molecule, synchronising between the phases.
static int scf_setup(ScfMol& M) {
  DF_TRY(setup_launch(M));
  DF_CUDA(cudaStreamSynchronize(M.s));
  DF_TRY(setup_orthogonalize(M));
  if (M.phase == ScfMol::GUESS_CHECK) {
    DF_CUDA(cudaStreamSynchronize(M.s));
    DF_TRY(setup_guess(M));
  }
  return DF_OK;
}

// J and K for a general starting density (first iteration with dm0), eager launches.
// First iteration from a non-idempotent dm0, in two halves so that a batch never blocks
// on it.  dm0_launch enqueues J(dm0) and the eigen-decomposition of dm0 with an asynchronous
// read-back of its eigenvalues; dm0_finish (once the stream has drained) splits
// dm0/2 = C+ C+^T - C- C-^T over the non-negligible eigenvalues and enqueues
// K = K(C+) - K(C-) in chunks of nocc columns, then the rest of the iteration.
static int dm0_launch(ScfMol& M) {
  ScfWork& W = M.W;
  cudaStream_t s = M.s;
  const int nao = M.nao;
  const long nn = (long)nao * nao;
  DF_CUDA(cudaMemcpyAsync(W.Dprev, W.D, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
  DF_TRY(run_jk(W.B, nao, M.naux, M.prec, W.D, nullptr, 0, W.J, nullptr, W.jk, s));
  DF_CUDA(cudaMemcpyAsync(W.T1, W.D, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
  DF_TRY(eig_rows(W.T1, nao, W.eps, W.ZT, W, s));
  DF_CUDA(cudaMemcpyAsync(M.h_eps, W.eps, sizeof(double) * nao, cudaMemcpyDeviceToHost, s));
  DF_CUDA(cudaMemcpyAsync(M.h_ints, W.eig_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  return DF_OK;
}

static int dm0_finish(ScfMol& M) {
  ScfWork& W = M.W;
  cudaStream_t s = M.s;
  const int nao = M.nao, naux = M.naux, nocc = M.nocc;
  const long nn = (long)nao * nao;
  DF_REQUIRE(M.h_ints[0] != 3, DF_ERR_TIMEOUT, "scf: a grid barrier of the eigensolver timed out on dm0");
  DF_REQUIRE(M.h_ints[0] == 0, DF_ERR_NOCONV, "scf: eigensolver failed on the starting density");
  double wmax = 0.0;
  for (int k = 0; k < nao; ++k) wmax = fmax(wmax, fabs(M.h_eps[k]));
  // natural occupations below 10^-dm0_eig_cut of the largest are dropped (default 10^-12:
  // the exact exchange of dm0; a coarser cut trades exactness of the first exchange for
  // fewer columns)
  const double cut = pow(10.0, -(double)std::max(1, knob("dm0_eig_cut"))) * wmax;
  // positive eigenvalues first, then negative ones; one copy of all indices to the device
  M.dm0_ids.clear();
  for (int k = 0; k < nao; ++k)
    if (M.h_eps[k] > cut) M.dm0_ids.push_back(k);
  const size_t npos = M.dm0_ids.size();
  for (int k = 0; k < nao; ++k)
    if (-M.h_eps[k] > cut) M.dm0_ids.push_back(k);
  DF_CUDA(cudaMemsetAsync(W.K, 0, sizeof(double) * nn, s));
  if (!M.dm0_ids.empty())
    DF_CUDA(cudaMemcpyAsync(W.idx, M.dm0_ids.data(), sizeof(int) * M.dm0_ids.size(), cudaMemcpyHostToDevice, s));
  for (int part = 0; part < 2; ++part) {
    const size_t b = part == 0 ? 0 : npos, e = part == 0 ? npos : M.dm0_ids.size();
    for (size_t c0 = b; c0 < e; c0 += nocc) {
      int cnt = (int)std::min((size_t)nocc, e - c0);
      split_density_kernel<<<blocks_for((long)nao * cnt), 256, 0, s>>>(W.ZT, W.eps, nao, W.idx + c0, cnt, W.Cchunk);
      DF_LAUNCHED("split_density_kernel");
      DF_TRY(run_jk(W.B, nao, naux, M.prec, nullptr, W.Cchunk, cnt, nullptr, W.T2, W.jk, s));
      axpy_kernel<<<blocks_for(nn), 256, 0, s>>>(W.K, W.T2, nn, part == 0 ? 1.0 : -1.0);
      DF_LAUNCHED("axpy_kernel");
    }
  }
  return DF_OK;
}

// Principal angles between the occupied space of the accumulated K (C'_base) and the new
// one (C'): M = C'_base^T C', eigen-decomposition of M^T M on one CTA, summary into the status.
static int incremental_prep(ScfMol& M) {
  ScfWork& W = M.W;
  cudaStream_t s = M.s;
  const int nmo = M.nmo, nocc = M.nocc;
  ProfScope ps_inc("scf_incremental_prep", s);
  DF_TRY(dgemm(true, false, nocc, nocc, nmo, 1.0, W.Cbase, nocc, 0, W.Cp, nocc, 0, 0.0, W.Minc, nocc, 0, 1, s, 0, 0));
  DF_TRY(dgemm(true, false, nocc, nocc, nocc, 1.0, W.Minc, nocc, 0, W.Minc, nocc, 0, 0.0, W.Tinc, nocc, 0, 1, s, 0, 0));
  DF_TRY(eigh_rows(W.Tinc, nocc, W.cinc, W.Winc, W.eig_scratch, W.inc_status, s));
  inc_status_kernel<<<1, 256, 0, s>>>(W.cinc, nocc, W.inc_status, W.st);
  DF_LAUNCHED("inc_status_kernel");
  return DF_OK;
}

// C_occ = X C'_o, D = 2 C_occ C_occ^T from the occupied columns of C'_all.
static int occupied_from_all(ScfMol& M) {
  ScfWork& W = M.W;
  cudaStream_t s = M.s;
  const int nao = M.nao, nmo = M.nmo, nocc = M.nocc;
  DF_CUDA(cudaMemcpy2DAsync(W.Cp, sizeof(double) * nocc, W.Call, sizeof(double) * nmo, sizeof(double) * nocc, nmo,
                            cudaMemcpyDeviceToDevice, s));
  DF_TRY(dgemm(false, false, nao, nocc, nmo, 1.0, W.X, nmo, 0, W.Cp, nocc, 0, 0.0, W.Cocc, nocc, 0, 1, s, 0, 0));
  DF_TRY(dgemm(false, true, nao, nao, nocc, 2.0, W.Cocc, nocc, 0, W.Cocc, nocc, 0, 0.0, W.D, nao, 0, 1, s, 0, 0));
  return DF_OK;
}

// Switch to Newton steps: the full orbital set from the extrapolated F' that produced the
// current occupied orbitals (kept in Fbar by the last DIIS step), so that the occupied
// space is unchanged.
static int soscf_init(ScfMol& M) {
  ScfWork& W = M.W;
  cudaStream_t s = M.s;
  const int nmo = M.nmo;
  const long ne = (long)nmo * nmo;
  DF_CUDA(cudaMemcpyAsync(W.Fp, W.Fbar, sizeof(double) * ne, cudaMemcpyDeviceToDevice, s));
  DF_TRY(eigh_full_rows(W.Fp, nmo, W.eps, W.ZT, W.eig_scratch, W.eig_status, s, W.eig_aux));
  DF_TRY(transpose(W.ZT, nmo, nmo, W.Call, s));
  DF_TRY(occupied_from_all(M));
  if (M.inc) DF_TRY(incremental_prep(M));
  return DF_OK;
}

// Av = H v for v [nvir][nocc] (see the head of the Newton-step kernels).
static int soscf_hessian(ScfMol& M, const double* v, double* Av, int hprec) {
  ScfWork& W = M.W;
  cudaStream_t s = M.s;
  const int nao = M.nao, nmo = M.nmo, nocc = M.nocc, nvir = nmo - nocc;
  const long nn = (long)nao * nao, no = (long)nao * nocc;
  DF_TRY(dgemm(false, false, nvir, nocc, nvir, 1.0, W.Fmo + (size_t)nocc * nmo + nocc, nmo, 0, v, nocc, 0, 0.0, Av,
               nocc, 0, 1, s, 0, 0));
  DF_TRY(dgemm(false, false, nvir, nocc, nocc, -1.0, v, nocc, 0, W.Fmo, nmo, 0, 1.0, Av, nocc, 0, 1, s, 0, 0));
  // L = X C'_v v, dD = 2 (L R^T + R L^T)
  DF_TRY(dgemm(false, false, nao, nocc, nvir, 1.0, W.Lv, nvir, 0, v, nocc, 0, 0.0, W.Lf, nocc, 0, 1, s, 0, 0));
  DF_TRY(dgemm(false, true, nao, nao, nocc, 1.0, W.Lf, nocc, 0, W.Cocc, nocc, 0, 0.0, W.dK1, nao, 0, 1, s, 0, 0));
  sym2_kernel<<<blocks_for(nn), 256, 0, s>>>(W.dK1, nao, W.dD);
  DF_LAUNCHED("sym2_kernel");
  DF_TRY(run_jk(W.B, nao, M.naux, hprec, W.dD, nullptr, 0, W.dJ, nullptr, W.jk, s));
  dot_kernel<<<1, 1024, 0, s>>>(W.Lf, W.Lf, no, W.cg_s + 3);
  DF_LAUNCHED("dot_kernel");
  dot_kernel<<<1, 1024, 0, s>>>(W.Cocc, W.Cocc, no, W.cg_s + 4);
  DF_LAUNCHED("dot_kernel");
  pm_factors_kernel<<<blocks_for(no), 256, 0, s>>>(W.Lf, W.Cocc, no, W.cg_s, W.Lfp, W.Lfm);
  DF_LAUNCHED("pm_factors_kernel");
  DF_TRY(run_jk(W.B, nao, M.naux, hprec, nullptr, W.Lfp, nocc, nullptr, W.dK1, W.jk, s));
  DF_TRY(run_jk(W.B, nao, M.naux, hprec, nullptr, W.Lfm, nocc, nullptr, W.dK2, W.jk, s));
  response_fock_kernel<<<blocks_for(nn), 256, 0, s>>>(W.dJ, W.dK1, W.dK2, nn);
  DF_LAUNCHED("response_fock_kernel");
  // Av += (X C'_v)^T dF C_occ
  DF_TRY(dgemm(false, false, nao, nocc, nao, 1.0, W.dJ, nao, 0, W.Cocc, nocc, 0, 0.0, W.Lf, nocc, 0, 1, s, 0, 0));
  DF_TRY(dgemm(true, false, nvir, nocc, nao, 1.0, W.Lv, nvir, 0, W.Lf, nocc, 0, 1.0, Av, nocc, 0, 1, s, 0, 0));
  return DF_OK;
}

static int rotate_orbitals(ScfMol& M);

// One Newton step from the Fock matrix F' (W.Fo) of the current orbitals C'_all: CG on
// H kappa = -F_vo, capped step, exact rotation of C'_all, new C_occ and D.
static int soscf_step(ScfMol& M) {
  ScfWork& W = M.W;
  cudaStream_t s = M.s;
  const int nao = M.nao, nmo = M.nmo, nocc = M.nocc, nvir = nmo - nocc;
  const long nvo = (long)nvir * nocc;
  const int hprec = M.opt.precision;  // the approximate Hessian uses the mixed exchange when B has its planes
  ProfScope ps("scf_newton_step", s);
  DF_TRY(dgemm(false, false, nmo, nmo, nmo, 1.0, W.Fo, nmo, 0, W.Call, nmo, 0, 0.0, W.T1, nmo, 0, 1, s, 0, 0));
  DF_TRY(dgemm(true, false, nmo, nmo, nmo, 1.0, W.Call, nmo, 0, W.T1, nmo, 0, 0.0, W.Fmo, nmo, 0, 1, s, 0, 0));
  soscf_grad_kernel<<<blocks_for(nvo), 256, 0, s>>>(W.Fmo, nmo, nocc, W.cg_g, W.cg_h);
  DF_LAUNCHED("soscf_grad_kernel");
  DF_TRY(dgemm(false, false, nao, nvir, nmo, 1.0, W.X, nmo, 0, W.Call + nocc, nmo, 0, 0.0, W.Lv, nvir, 0, 1, s, 0, 0));
  cg_start_kernel<<<blocks_for(nvo), 256, 0, s>>>(W.cg_x, W.cg_r, W.cg_z, W.cg_p, W.cg_g, W.cg_h, nvo);
  DF_LAUNCHED("cg_start_kernel");
  cg_reset_kernel<<<1, 32, 0, s>>>(W.cg_s, 0.5);
  DF_LAUNCHED("cg_reset_kernel");
  dot_kernel<<<1, 1024, 0, s>>>(W.cg_r, W.cg_z, nvo, W.cg_s + 0);
  DF_LAUNCHED("dot_kernel");
  const int ncg = std::max(1, knob("soscf_cg"));
  for (int it = 0; it < ncg; ++it) {
    DF_TRY(soscf_hessian(M, W.cg_p, W.cg_Ap, hprec));
    dot_kernel<<<1, 1024, 0, s>>>(W.cg_p, W.cg_Ap, nvo, W.cg_s + 1);
    DF_LAUNCHED("dot_kernel");
    dot_kernel<<<1, 1024, 0, s>>>(W.cg_x, W.cg_x, nvo, W.cg_s + 6);
    DF_LAUNCHED("dot_kernel");
    dot_kernel<<<1, 1024, 0, s>>>(W.cg_x, W.cg_p, nvo, W.cg_s + 7);
    DF_LAUNCHED("dot_kernel");
    dot_kernel<<<1, 1024, 0, s>>>(W.cg_p, W.cg_p, nvo, W.cg_s + 8);
    DF_LAUNCHED("dot_kernel");
    cg_decide_kernel<<<1, 32, 0, s>>>(W.cg_s);
    DF_LAUNCHED("cg_decide_kernel");
    cg_step_kernel<<<blocks_for(nvo), 256, 0, s>>>(W.cg_x, W.cg_r, W.cg_z, W.cg_p, W.cg_Ap, W.cg_h, nvo, W.cg_s);
    DF_LAUNCHED("cg_step_kernel");
    if (it + 1 == ncg) break;
    dot_kernel<<<1, 1024, 0, s>>>(W.cg_r, W.cg_z, nvo, W.cg_s + 2);
    DF_LAUNCHED("dot_kernel");
    cg_dir_kernel<<<blocks_for(nvo), 256, 0, s>>>(W.cg_p, W.cg_z, nvo, W.cg_s);
    DF_LAUNCHED("cg_dir_kernel");
    copy_scalar_kernel<<<1, 32, 0, s>>>(W.cg_s + 0, W.cg_s + 2);
    DF_LAUNCHED("copy_scalar_kernel");
  }
  absmax_kernel<<<1, 1024, 0, s>>>(W.cg_x, nvo, W.cg_s + 5);
  DF_LAUNCHED("absmax_kernel");
  cap_step_kernel<<<blocks_for(nvo), 256, 0, s>>>(W.cg_x, nvo, W.cg_s, 0.3);
  DF_LAUNCHED("cap_step_kernel");
  return rotate_orbitals(M);
}

// C'_all <- C'_all exp(A) with A = [[0, -k^T], [k, 0]] and k = W.cg_x [nvir][nocc] (exact, from
// the eigen-decomposition of k^T k), then the new C_occ and D.
static int rotate_orbitals(ScfMol& M) {
  ScfWork& W = M.W;
  cudaStream_t s = M.s;
  const int nmo = M.nmo, nocc = M.nocc, nvir = nmo - nocc;
  const long ne = (long)nmo * nmo;
  DF_TRY(dgemm(true, false, nocc, nocc, nvir, 1.0, W.cg_x, nocc, 0, W.cg_x, nocc, 0, 0.0, W.kk, nocc, 0, 1, s, 0, 0));
  DF_TRY(eigh_rows(W.kk, nocc, W.ksig, W.kVrow, W.eig_scratch, W.k_status, s));
  rotation_mats_kernel<<<blocks_for((long)nocc * nocc), 256, 0, s>>>(W.kVrow, W.ksig, nocc, W.Pc, W.Ps, W.Pd);
  DF_LAUNCHED("rotation_mats_kernel");
  // occupied: C'_o Pc + C'_v (k Ps)
  DF_TRY(dgemm(false, false, nvir, nocc, nocc, 1.0, W.cg_x, nocc, 0, W.Ps, nocc, 0, 0.0, W.ktmp, nocc, 0, 1, s, 0, 0));
  DF_TRY(dgemm(false, false, nmo, nocc, nocc, 1.0, W.Call, nmo, 0, W.Pc, nocc, 0, 0.0, W.Call2, nmo, 0, 1, s, 0, 0));
  DF_TRY(dgemm(false, false, nmo, nocc, nvir, 1.0, W.Call + nocc, nmo, 0, W.ktmp, nocc, 0, 1.0, W.Call2, nmo, 0, 1, s,
               0, 0));
  // virtual: C'_v (1 + k Pd k^T) - C'_o (Ps k^T)
  if (nvir > 0) {
    DF_TRY(dgemm(false, false, nvir, nocc, nocc, 1.0, W.cg_x, nocc, 0, W.Pd, nocc, 0, 0.0, W.ktmp, nocc, 0, 1, s, 0,
                 0));
    DF_TRY(dgemm(false, true, nvir, nvir, nocc, 1.0, W.ktmp, nocc, 0, W.cg_x, nocc, 0, 0.0, W.KPdK, nvir, 0, 1, s, 0,
                 0));
    add_identity_kernel<<<blocks_for(nvir), 256, 0, s>>>(W.KPdK, nvir);
    DF_LAUNCHED("add_identity_kernel");
    DF_TRY(dgemm(false, false, nmo, nvir, nvir, 1.0, W.Call + nocc, nmo, 0, W.KPdK, nvir, 0, 0.0, W.Call2 + nocc, nmo,
                 0, 1, s, 0, 0));
    DF_TRY(dgemm(false, true, nocc, nvir, nocc, 1.0, W.Ps, nocc, 0, W.cg_x, nocc, 0, 0.0, W.ktmp, nvir, 0, 1, s, 0,
                 0));
    DF_TRY(dgemm(false, false, nmo, nvir, nocc, -1.0, W.Call, nmo, 0, W.ktmp, nvir, 0, 1.0, W.Call2 + nocc, nmo, 0, 1,
                 s, 0, 0));
  }
  DF_CUDA(cudaMemcpyAsync(W.Call, W.Call2, sizeof(double) * ne, cudaMemcpyDeviceToDevice, s));
  return occupied_from_all(M);
}

// ---- stability analysis ---------------------------------------------------------------------
// The lowest eigenvalue of the orbital Hessian at a converged solution (the operator of the
// Newton steps, in units of the gradient F_vo): positive at a local minimum of the energy over
// closed-shell determinants, negative at a saddle point.  Davidson's method on the canonical
// orbitals of the last Fock matrix (the converged ones: F and D commute there): the subspace
// holds the search vectors V and their products H V; the Rayleigh-Ritz matrix V^T H V is
// diagonalised on the host (cyclic Jacobi, at most kDavidsonMax rows); the correction is the
// residual divided by (eps_a - eps_i - theta), the diagonal of the Hessian's one-electron part.
// The start block is the unit vectors of the smallest eps_a - eps_i and one fixed
// pseudo-random vector (so that a mode of another symmetry than the lowest excitations is
// still reached).  A full subspace collapses onto the current Ritz vector.


__global__ void scale_copy_kernel(const double* __restrict__ x, double* __restrict__ y, long n,
                                  const double* __restrict__ nrm2) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = *nrm2 > 0.0 ? x[i] / sqrt(*nrm2) : 0.0;
}

// w -= c v with c = *cp (device scalar).
__global__ void axpy_dev_kernel(double* __restrict__ w, const double* __restrict__ v, long n,
                                const double* __restrict__ cp) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) w[i] -= (*cp) * v[i];
}

// t = r / (eps_a - eps_i - theta), the denominator kept at least 1e-3 away from zero.
__global__ void davidson_precond_kernel(const double* __restrict__ Fmo, int nmo, int nocc,
                                        const double* __restrict__ r, double theta, double* __restrict__ t) {
  const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int nvir = nmo - nocc;
  if (q >= (long)nvir * nocc) return;
  const int a = (int)(q / nocc), i = (int)(q % nocc);
  double d = Fmo[DF_IX((size_t)(nocc + a) * nmo + nocc + a, (size_t)nmo * nmo)] -
             Fmo[DF_IX((size_t)i * nmo + i, (size_t)nmo * nmo)] - theta;
  if (fabs(d) < 1e-3) d = d < 0.0 ? -1e-3 : 1e-3;
  t[q] = r[q] / d;
}

// eps_a - eps_i for every (virtual, occupied) pair.
__global__ void excitation_diag_kernel(const double* __restrict__ Fmo, int nmo, int nocc, double* __restrict__ d) {
  const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int nvir = nmo - nocc;
  if (q >= (long)nvir * nocc) return;
  const int a = (int)(q / nocc), i = (int)(q % nocc);
  d[q] = Fmo[DF_IX((size_t)(nocc + a) * nmo + nocc + a, (size_t)nmo * nmo)] -
         Fmo[DF_IX((size_t)i * nmo + i, (size_t)nmo * nmo)];
}

// Lowest eigenpair of a symmetric k x k matrix (row-major, k <= kDavidsonMax) by cyclic
// Jacobi rotations.
static double sym_lowest(std::vector<double> T, int k, std::vector<double>& vec) {
  std::vector<double> V((size_t)k * k, 0.0);
  for (int i = 0; i < k; ++i) V[(size_t)i * k + i] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int p = 0; p < k; ++p) {
      diag += T[(size_t)p * k + p] * T[(size_t)p * k + p];
      for (int q = p + 1; q < k; ++q) off += T[(size_t)p * k + q] * T[(size_t)p * k + q];
    }
    if (off <= 1e-30 * std::max(diag, 1e-300)) break;
    for (int p = 0; p < k; ++p)
      for (int q = p + 1; q < k; ++q) {
        const double apq = T[(size_t)p * k + q];
        if (apq == 0.0) continue;
        const double theta = (T[(size_t)q * k + q] - T[(size_t)p * k + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
        for (int r = 0; r < k; ++r) {  // T <- T G (columns p, q)
          const double tp = T[(size_t)r * k + p], tq = T[(size_t)r * k + q];
          T[(size_t)r * k + p] = c * tp - sn * tq;
          T[(size_t)r * k + q] = sn * tp + c * tq;
        }
        for (int r = 0; r < k; ++r) {  // T <- G^T T (rows p, q)
          const double tp = T[(size_t)p * k + r], tq = T[(size_t)q * k + r];
          T[(size_t)p * k + r] = c * tp - sn * tq;
          T[(size_t)q * k + r] = sn * tp + c * tq;
        }
        for (int r = 0; r < k; ++r) {  // V <- V G
          const double vp = V[(size_t)r * k + p], vq = V[(size_t)r * k + q];
          V[(size_t)r * k + p] = c * vp - sn * vq;
          V[(size_t)r * k + q] = sn * vp + c * vq;
        }
      }
  }
  int lo = 0;
  for (int i = 1; i < k; ++i)
    if (T[(size_t)i * k + i] < T[(size_t)lo * k + lo]) lo = i;
  vec.resize(k);
  for (int r = 0; r < k; ++r) vec[r] = V[(size_t)r * k + lo];
  return T[(size_t)lo * k + lo];
}

// Index of the smallest d[i] (ties: the smaller index), skipping i == *skip when skip is set;
// written as a double to *out (one CTA).
__global__ void dav_argmin_kernel(const double* __restrict__ d, long n, const double* __restrict__ skip,
                                  double* __restrict__ out) {
  __shared__ double sv[1024];
  __shared__ long si[1024];
  const long excl = skip ? (long)*skip : -1;
  double bv = INFINITY;
  long bi = -1;
  for (long i = threadIdx.x; i < n; i += blockDim.x)
    if (i != excl && (d[i] < bv || (d[i] == bv && (bi < 0 || i < bi)))) {
      bv = d[i];
      bi = i;
    }
  sv[threadIdx.x] = bv;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      const double ov = sv[threadIdx.x + h];
      const long oi = si[threadIdx.x + h];
      if (oi >= 0 && (si[threadIdx.x] < 0 || ov < sv[threadIdx.x] || (ov == sv[threadIdx.x] && oi < si[threadIdx.x]))) {
        sv[threadIdx.x] = ov;
        si[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = (double)(si[0] < 0 ? 0 : si[0]);
}

// v = unit vector at index *at.
__global__ void dav_unit_kernel(double* __restrict__ v, long n, const double* __restrict__ at) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = i == (long)*at ? 1.0 : 0.0;
}

// SplitMix64 of i + 1 mapped to [-1/2, 1/2): the fixed pseudo-random direction of the start
// block and of the sign convention of the Ritz vector.
__device__ __forceinline__ double splitmix_unit(long i) {
  unsigned long long z = 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
}

__global__ void dav_splitmix_kernel(double* __restrict__ v, long n) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = splitmix_unit(i);
}

// *out = sum_i x[i] h(i) with h the SplitMix direction (one CTA).
__global__ void dav_dot_splitmix_kernel(const double* __restrict__ x, long n, double* __restrict__ out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (long i = threadIdx.x; i < n; i += blockDim.x) acc += x[i] * splitmix_unit(i);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = (int)threadIdx.x < (int)(blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) *out = acc;
  }
}

// x *= a * sign(*sdot) (a zero dot counts as positive).
__global__ void dav_scale_signed_kernel(double* __restrict__ x, long n, double a, const double* __restrict__ sdot) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] *= (*sdot < 0.0 ? -a : a);
}

// Orthonormalise w against V[0..m) (classical Gram-Schmidt, two passes, device scalars) and
// store it normalised as V[m]; its squared norm before the normalisation stays in *n2.
static int davidson_store(ScfMol& M, double* w, double* V, int m, long nvo, double* n2, double* scratch) {
  cudaStream_t s = M.s;
  for (int pass = 0; pass < 2; ++pass)
    for (int i = 0; i < m; ++i) {
      dot_kernel<<<1, 1024, 0, s>>>(V + (size_t)i * nvo, w, nvo, scratch);
      DF_LAUNCHED("dot_kernel");
      axpy_dev_kernel<<<blocks_for(nvo), 256, 0, s>>>(w, V + (size_t)i * nvo, nvo, scratch);
      DF_LAUNCHED("axpy_dev_kernel");
    }
  dot_kernel<<<1, 1024, 0, s>>>(w, w, nvo, n2);
  DF_LAUNCHED("dot_kernel");
  scale_copy_kernel<<<blocks_for(nvo), 256, 0, s>>>(w, V + (size_t)m * nvo, nvo, n2);
  DF_LAUNCHED("scale_copy_kernel");
  return DF_OK;
}

// Device layout of the Davidson workspace W.dav: V, H V, the Rayleigh-Ritz entries G (row j
// holds V_i . H V_j, i <= j) and scalars (|r|^2 of the last Ritz pair, |t|^2 of the newest
// vector, sign dot, two start indices, scratch).  One host round trip per iteration: the step
// that forms the residual r of a Ritz pair also forms the next correction and its product, and
// the read-back of their entries carries |r|^2, so convergence is judged one iteration late (an
// extra product at the end; forming |r|^2 from the Gram matrix of H V instead would cancel
// catastrophically when |H| is large).
struct DavPtrs {
  double *V, *AV, *G, *misc;
};
static DavPtrs dav_ptrs(ScfMol& M) {
  const long nvo = (long)(M.nmo - M.nocc) * M.nocc;
  DavPtrs p;
  p.V = M.W.dav;
  p.AV = p.V + (size_t)kDavidsonMax * nvo;
  p.G = p.AV + (size_t)kDavidsonMax * nvo;
  p.misc = p.G + (size_t)kDavidsonMax * kDavidsonMax;
  return p;
}
constexpr int kDavHost = kDavidsonMax * kDavidsonMax + 8;  // pinned doubles per molecule: G, scalars
constexpr double kDavTol = 1e-5;                                // residual of the converged Ritz pair

// Products H V_j for the vectors without one, their entries of G and Q, and an asynchronous
// read-back of the new rows with the squared norm of the newest vector.
static int dav_products(ScfMol& M) {
  DavState& d = M.dav;
  const long nvo = (long)(M.nmo - M.nocc) * M.nocc;
  DavPtrs p = dav_ptrs(M);
  d.row0 = d.have;
  for (; d.have < d.m; ++d.have) {
    DF_TRY(soscf_hessian(M, p.V + (size_t)d.have * nvo, p.AV + (size_t)d.have * nvo, M.opt.precision));
    d.products++;
    for (int i = 0; i <= d.have; ++i) {
      dot_kernel<<<1, 1024, 0, M.s>>>(p.V + (size_t)i * nvo, p.AV + (size_t)d.have * nvo, nvo,
                                      p.G + (size_t)d.have * kDavidsonMax + i);
      DF_LAUNCHED("dot_kernel");
    }
  }
  const size_t rows = (size_t)kDavidsonMax * (d.have - d.row0), at = (size_t)d.row0 * kDavidsonMax;
  DF_CUDA(cudaMemcpyAsync(M.h_dav + at, p.G + at, sizeof(double) * rows, cudaMemcpyDeviceToHost, M.s));
  DF_CUDA(cudaMemcpyAsync(M.h_dav + kDavidsonMax * kDavidsonMax, p.misc, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                          M.s));
  d.stage = DavState::RITZ;
  return DF_OK;
}

// Start of the stability analysis of a converged solution (enqueued only; the host continues
// with dav_advance once the stream has drained).  mode_scale > 0: the finished analysis
// leaves mode_scale times the unit Ritz vector of the lowest eigenvalue in W.cg_x, in the
// (virtual, occupied) basis of the canonical orbitals left in C'_all, with the sign that makes
// its dot with the SplitMix direction non-negative (so that both precisions turn the same way).
static int dav_begin(ScfMol& M, double mode_scale) {
  ScfWork& W = M.W;
  cudaStream_t s = M.s;
  const int nao = M.nao, nmo = M.nmo, nocc = M.nocc, nvir = nmo - nocc;
  const long ne = (long)nmo * nmo, nvo = (long)nvir * nocc;
  DavState& d = M.dav;
  d = DavState();
  M.res.hess_min = NAN;
  if (nvo <= 0) return DF_OK;  // stage stays OFF: nothing to analyse
  // canonical orbitals of the last Fock matrix F' (W.Fo)
  DF_CUDA(cudaMemcpyAsync(W.Fp, W.Fo, sizeof(double) * ne, cudaMemcpyDeviceToDevice, s));
  DF_TRY(eigh_full_rows(W.Fp, nmo, W.eps, W.ZT, W.eig_scratch, W.eig_status, s, W.eig_aux));
  DF_TRY(transpose(W.ZT, nmo, nmo, W.Call, s));
  DF_TRY(occupied_from_all(M));
  DF_TRY(dgemm(false, false, nmo, nmo, nmo, 1.0, W.Fo, nmo, 0, W.Call, nmo, 0, 0.0, W.T1, nmo, 0, 1, s, 0, 0));
  DF_TRY(dgemm(true, false, nmo, nmo, nmo, 1.0, W.Call, nmo, 0, W.T1, nmo, 0, 0.0, W.Fmo, nmo, 0, 1, s, 0, 0));
  DF_TRY(dgemm(false, false, nao, nvir, nmo, 1.0, W.X, nmo, 0, W.Call + nocc, nmo, 0, 0.0, W.Lv, nvir, 0, 1, s, 0, 0));
  d.kmax = (int)std::min<long>(kDavidsonMax, nvo);
  d.max_products = std::max(2, knob("stability_steps"));
  d.mode_scale = mode_scale;
  d.Hs.assign((size_t)kDavidsonMax * kDavidsonMax, 0.0);
  DavPtrs p = dav_ptrs(M);
  // start block: the unit vectors of the two smallest eps_a - eps_i, then the SplitMix
  // direction orthonormalised against them
  excitation_diag_kernel<<<blocks_for(nvo), 256, 0, s>>>(W.Fmo, nmo, nocc, W.cg_h);
  DF_LAUNCHED("excitation_diag_kernel");
  dav_argmin_kernel<<<1, 1024, 0, s>>>(W.cg_h, nvo, nullptr, p.misc + 3);
  DF_LAUNCHED("dav_argmin_kernel");
  dav_unit_kernel<<<blocks_for(nvo), 256, 0, s>>>(p.V, nvo, p.misc + 3);
  DF_LAUNCHED("dav_unit_kernel");
  d.m = 1;
  if (nvo >= 2) {
    dav_argmin_kernel<<<1, 1024, 0, s>>>(W.cg_h, nvo, p.misc + 3, p.misc + 4);
    DF_LAUNCHED("dav_argmin_kernel");
    dav_unit_kernel<<<blocks_for(nvo), 256, 0, s>>>(p.V + nvo, nvo, p.misc + 4);
    DF_LAUNCHED("dav_unit_kernel");
    d.m = 2;
  }
  if (nvo >= 3 && d.kmax >= 3) {
    dav_splitmix_kernel<<<blocks_for(nvo), 256, 0, s>>>(W.cg_Ap, nvo);
    DF_LAUNCHED("dav_splitmix_kernel");
    DF_TRY(davidson_store(M, W.cg_Ap, p.V, 2, nvo, p.misc + 1, p.misc + 5));
    d.m = 3;
  }
  d.added = false;  // start vectors are checked by construction
  d.have_rr = false;
  return dav_products(M);
}

// One host step of the analysis after the stream has drained; *finished once hess_min is set
// (and, with a mode scale, the scaled Ritz vector is enqueued into W.cg_x).
static int dav_advance(ScfMol& M, bool* finished) {
  ScfWork& W = M.W;
  cudaStream_t s = M.s;
  DavState& d = M.dav;
  const int nmo = M.nmo, nocc = M.nocc;
  const long nvo = (long)(nmo - nocc) * nocc;
  DavPtrs p = dav_ptrs(M);
  double* x = W.cg_x;
  double* r = W.cg_r;
  double* wv = W.cg_Ap;
  *finished = false;
  if (d.stage == DavState::OFF) {
    *finished = true;
    return DF_OK;
  }
  const double* hG = M.h_dav;
  const double rr_prev = M.h_dav[kDavidsonMax * kDavidsonMax];      // |r|^2 of the previous Ritz pair
  const double n2 = M.h_dav[kDavidsonMax * kDavidsonMax + 1];       // |t|^2 of the newest vector
  // Ritz vector x = V y of the current (theta, y)
  auto ritz_vector = [&]() -> int {
    DF_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * nvo, s));
    for (int i = 0; i < d.m; ++i) {
      axpy_kernel<<<blocks_for(nvo), 256, 0, s>>>(x, p.V + (size_t)i * nvo, nvo, d.y[i]);
      DF_LAUNCHED("axpy_kernel");
    }
    return DF_OK;
  };
  auto finish = [&]() -> int {
    M.res.hess_min = d.theta;
    d.stage = DavState::OFF;
    *finished = true;
    if (d.mode_scale > 0.0) {  // x is a unit vector (orthonormal V, unit y)
      DF_TRY(ritz_vector());
      dav_dot_splitmix_kernel<<<1, 1024, 0, s>>>(x, nvo, p.misc + 2);
      DF_LAUNCHED("dav_dot_splitmix_kernel");
      dav_scale_signed_kernel<<<blocks_for(nvo), 256, 0, s>>>(x, nvo, d.mode_scale, p.misc + 2);
      DF_LAUNCHED("dav_scale_signed_kernel");
    }
    return DF_OK;
  };
  if (d.added && !(n2 > 1e-24)) {
    // the last correction lay in the subspace: drop it and keep the previous Ritz pair
    d.m--;
    d.have--;
    return finish();
  }
  const double theta_prev = d.theta;
  for (int j = d.row0; j < d.have; ++j)
    for (int i = 0; i <= j; ++i)
      d.Hs[(size_t)i * kDavidsonMax + j] = d.Hs[(size_t)j * kDavidsonMax + i] = hG[(size_t)j * kDavidsonMax + i];
  std::vector<double> T((size_t)d.m * d.m);
  for (int i = 0; i < d.m; ++i)
    for (int j = 0; j < d.m; ++j) T[(size_t)i * d.m + j] = d.Hs[(size_t)i * kDavidsonMax + j];
  d.theta = sym_lowest(T, d.m, d.y);
  if (M.opt.verbose)
    printf("stability: %d products, theta %.10f, previous |r| %.3e\n", d.products, d.theta,
           d.have_rr ? sqrt(std::max(0.0, rr_prev)) : -1.0);
  // converged when the previous pair's residual was below the tolerance (this pair is at
  // least as good: Rayleigh-Ritz on a larger subspace)
  if (d.have_rr && sqrt(std::max(0.0, rr_prev)) < kDavTol * std::max(1.0, fabs(theta_prev))) return finish();
  if (d.products >= d.max_products || d.m == nvo) return finish();
  // x = V y, r = AV y - theta x and |r|^2 (read back with the next entries)
  DF_TRY(ritz_vector());
  DF_CUDA(cudaMemsetAsync(r, 0, sizeof(double) * nvo, s));
  for (int i = 0; i < d.m; ++i) {
    axpy_kernel<<<blocks_for(nvo), 256, 0, s>>>(r, p.AV + (size_t)i * nvo, nvo, d.y[i]);
    DF_LAUNCHED("axpy_kernel");
  }
  if (d.m == d.kmax) {  // collapse the subspace onto the Ritz vector and its product
    DF_CUDA(cudaMemcpyAsync(p.V, x, sizeof(double) * nvo, cudaMemcpyDeviceToDevice, s));
    DF_CUDA(cudaMemcpyAsync(p.AV, r, sizeof(double) * nvo, cudaMemcpyDeviceToDevice, s));  // H x
    std::fill(d.Hs.begin(), d.Hs.end(), 0.0);
    d.Hs[0] = d.theta;
    d.y.assign(1, 1.0);  // the Ritz vector in the collapsed basis
    d.m = d.have = 1;
  }
  axpy_kernel<<<blocks_for(nvo), 256, 0, s>>>(r, x, nvo, -d.theta);
  DF_LAUNCHED("axpy_kernel");
  dot_kernel<<<1, 1024, 0, s>>>(r, r, nvo, p.misc + 0);
  DF_LAUNCHED("dot_kernel");
  d.have_rr = true;
  davidson_precond_kernel<<<blocks_for(nvo), 256, 0, s>>>(W.Fmo, nmo, nocc, r, d.theta, wv);
  DF_LAUNCHED("davidson_precond_kernel");
  DF_TRY(davidson_store(M, wv, p.V, d.m, nvo, p.misc + 1, p.misc + 5));
  d.m++;
  d.added = true;
  return dav_products(M);
}

// The whole analysis for one molecule, waiting on its stream between the host steps.
static int stability_analysis(ScfMol& M, double mode_scale) {
  DF_TRY(dav_begin(M, mode_scale));
  bool fin = false;
  while (!fin) {
    DF_CUDA(cudaStreamSynchronize(M.s));
    DF_TRY(dav_advance(M, &fin));
  }
  return DF_OK;
}

// Escape from a saddle point (knob "stability" = 2): with the Ritz vector u of the negative
// Hessian eigenvalue in W.cg_x (scaled to the rotation angle), turn the canonical orbitals by
// exp(u) (the energy falls as 2 hess_min |u|^2 to second order, in Eh) and restart the
// iterations there with Newton steps (or DIIS from an empty history when they are switched
// off), in FP64, with a fresh iteration budget.
constexpr double kSaddleTol = -1e-4;  // hess_min below this is a saddle, not noise
constexpr double kEscapeAngle = 0.3;  // |u| of the escape rotation (radians)
constexpr int kMaxEscapes = 3;

static int escape_saddle(ScfMol& M) {
  DF_TRY(rotate_orbitals(M));
  diis_reset_kernel<<<1, 32, 0, M.s>>>(M.W.diis, M.opt.diis_space);
  DF_LAUNCHED("diis_reset_kernel");
  M.res.converged = 0;
  M.res.stability_restarts++;
  M.done = false;
  M.have_old = false;
  M.fp64_done = 0;
  M.prec = DF_FP64;
  M.switched = true;
  if (M.inc) M.kp = ScfMol::KP_FINAL;
  M.soscf = M.soscf_on;
  M.soscf_pending = false;
  M.iter_limit = M.res.iterations + M.opt.max_cycle;
  return DF_OK;
}

// Everything after J and K: Fock, energy, DIIS error and extrapolation, diagonalisation,
// status readback.  No host decisions: capturable.
static int iteration_tail(ScfMol& M, int prec) {
  ScfWork& W = M.W;
  cudaStream_t s = M.s;
  const int nao = M.nao, nmo = M.nmo, nocc = M.nocc;
  const long nn = (long)nao * nao, ne = (long)nmo * nmo;
  {
    ProfScope ps("scf_fock_energy", s);
    fock_energy_kernel<<<1, 1024, 0, s>>>(W.h, W.J, W.K, W.D, nn, W.enuc, W.F, W.st);
    DF_LAUNCHED("fock_energy_kernel");
  }
  {
    // DIIS in the orthogonal basis of X (X^T S X = 1): F' = X^T F X and, for D = X D' X^T,
    // e = X^T (F D S - S D F) X = F' D' - D' F'.  With D' = 2 C' C'^T (C' the occupied
    // columns of the last diagonalisation) e = M - M^T, M = 2 (F' C') C'^T: O(nmo^2 nocc)
    // work instead of four O(nao^3) products; the extrapolated F' is diagonalised as it is.
    ProfScope ps("scf_diis_error", s);
    DF_TRY(to_orth(W.F, nao, nmo, W, W.Fo, s));
    if (M.first_dm0) {
      // a starting density need not lie in the span of X C': AO-basis commutator
      DF_TRY(dgemm(false, false, nao, nao, nao, 1.0, W.F, nao, 0, W.D, nao, 0, 0.0, W.T1, nao, 0, 1, s, 0, 0));
      DF_TRY(dgemm(false, false, nao, nao, nao, 1.0, W.T1, nao, 0, W.S, nao, 0, 0.0, W.T2, nao, 0, 1, s, 0, 0));
      antisym_kernel<<<blocks_for(nn), 256, 0, s>>>(W.T2, nao, W.T1);
      DF_LAUNCHED("antisym_kernel");
      DF_TRY(dgemm(false, false, nao, nmo, nao, 1.0, W.T1, nao, 0, W.X, nmo, 0, 0.0, W.T2, nmo, 0, 1, s, 0, 0));
      DF_TRY(dgemm(true, false, nmo, nmo, nao, 1.0, W.X, nmo, 0, W.T2, nmo, 0, 0.0, W.E, nmo, 0, 1, s, 0, 0));
    } else {
      DF_TRY(dgemm(false, false, nmo, nocc, nmo, 1.0, W.Fo, nmo, 0, W.Cp, nocc, 0, 0.0, W.T1, nocc, 0, 1, s, 0, 0));
      DF_TRY(dgemm(false, true, nmo, nmo, nocc, 2.0, W.T1, nocc, 0, W.Cp, nocc, 0, 0.0, W.T2, nmo, 0, 1, s, 0, 0));
      antisym_kernel<<<blocks_for(ne), 256, 0, s>>>(W.T2, nmo, W.E);
      DF_LAUNCHED("antisym_kernel");
    }
    absmax_kernel<<<1, 1024, 0, s>>>(W.E, ne, &W.st->emax);
    DF_LAUNCHED("absmax_kernel");
  }
  ProfScope ps_diis("scf_diis_and_diagonalize", s);
  diis_select_kernel<<<1, 32, 0, s>>>(W.diis);
  DF_LAUNCHED("diis_select_kernel");
  diis_store_kernel<<<blocks_for(ne), 256, 0, s>>>(W.diis, W.Fo, W.E, W.Fhist, W.Ehist, nn, ne);
  DF_LAUNCHED("diis_store_kernel");
  diis_gram_kernel<<<DIIS_MAX, 256, 0, s>>>(W.diis, W.Ehist, nn, ne, W.G);
  DF_LAUNCHED("diis_gram_kernel");
  diis_solve_kernel<<<1, 32, 0, s>>>(W.diis, W.G, W.coef, W.st);
  DF_LAUNCHED("diis_solve_kernel");
  diis_combine_kernel<<<blocks_for(ne), 256, 0, s>>>(W.diis, W.Fhist, nn, ne, W.coef, W.Fp);
  DF_LAUNCHED("diis_combine_kernel");
  if (M.soscf_on) DF_CUDA(cudaMemcpyAsync(W.Fbar, W.Fp, sizeof(double) * ne, cudaMemcpyDeviceToDevice, s));
  DF_TRY(diagonalize_orth(nao, nmo, nocc, W, s));
  if (M.inc) DF_TRY(incremental_prep(M));
  orbital_status_kernel<<<1, 32, 0, s>>>(W.eps, nmo, nocc, W.eig_status, prec == DF_MIXED ? W.jk.mk.err : nullptr,
                                         W.st);
  DF_LAUNCHED("orbital_status_kernel");
  DF_CUDA(cudaMemcpyAsync(M.hst, W.st, sizeof(ScfStatus), cudaMemcpyDeviceToHost, s));
  return DF_OK;
}

// Tail of a Newton iteration: Fock and energy, the orthogonal-basis error of the density
// that was built (for the convergence test), then a Newton step instead of DIIS and the
// diagonalisation.
static int iteration_tail_soscf(ScfMol& M, int prec) {
  ScfWork& W = M.W;
  cudaStream_t s = M.s;
  const int nao = M.nao, nmo = M.nmo, nocc = M.nocc;
  const long nn = (long)nao * nao, ne = (long)nmo * nmo;
  fock_energy_kernel<<<1, 1024, 0, s>>>(W.h, W.J, W.K, W.D, nn, W.enuc, W.F, W.st);
  DF_LAUNCHED("fock_energy_kernel");
  DF_TRY(to_orth(W.F, nao, nmo, W, W.Fo, s));
  DF_TRY(dgemm(false, false, nmo, nocc, nmo, 1.0, W.Fo, nmo, 0, W.Cp, nocc, 0, 0.0, W.T1, nocc, 0, 1, s, 0, 0));
  DF_TRY(dgemm(false, true, nmo, nmo, nocc, 2.0, W.T1, nocc, 0, W.Cp, nocc, 0, 0.0, W.T2, nmo, 0, 1, s, 0, 0));
  antisym_kernel<<<blocks_for(ne), 256, 0, s>>>(W.T2, nmo, W.E);
  DF_LAUNCHED("antisym_kernel");
  absmax_kernel<<<1, 1024, 0, s>>>(W.E, ne, &W.st->emax);
  DF_LAUNCHED("absmax_kernel");
  DF_TRY(soscf_step(M));
  if (M.inc) DF_TRY(incremental_prep(M));
  soscf_status_kernel<<<1, 32, 0, s>>>(W.Fmo, nmo, nocc, W.k_status, prec == DF_MIXED ? W.jk.mk.err : nullptr, W.st);
  DF_LAUNCHED("soscf_status_kernel");
  DF_CUDA(cudaMemcpyAsync(M.hst, W.st, sizeof(ScfStatus), cudaMemcpyDeviceToHost, s));
  return DF_OK;
}

// Body of a regular iteration: keep the incoming density, build J/K, then the tail.
static int iteration_body(ScfMol& M, int prec) {
  ScfWork& W = M.W;
  const long nn = (long)M.nao * M.nao;
  DF_CUDA(cudaMemcpyAsync(W.Dprev, W.D, sizeof(double) * nn, cudaMemcpyDeviceToDevice, M.s));
  DF_CUDA(cudaMemcpyAsync(W.Cprev, W.Cocc, sizeof(double) * M.nao * M.nocc, cudaMemcpyDeviceToDevice, M.s));
  DF_TRY(run_jk(W.B, M.nao, M.naux, prec, W.D, W.Cocc, M.nocc, W.J, W.K, W.jk, M.s));
  if (M.inc)  // a full build: the accumulated K now belongs to this density
    DF_CUDA(cudaMemcpyAsync(W.Cbase, W.Cp, sizeof(double) * M.nmo * M.nocc, cudaMemcpyDeviceToDevice, M.s));
  return M.soscf ? iteration_tail_soscf(M, prec) : iteration_tail(M, prec);
}

// Body of an incremental iteration: J in FP64 as always; K += K[U+] - K[U-] with the
// factors of P_new - P_base in mixed precision (the principal-angle decomposition above,
// from the eigen-decomposition the previous tail left in Winc / cinc).
static int iteration_body_incremental(ScfMol& M) {
  ScfWork& W = M.W;
  cudaStream_t s = M.s;
  const int nao = M.nao, nmo = M.nmo, nocc = M.nocc;
  const long nn = (long)nao * nao;
  DF_CUDA(cudaMemcpyAsync(W.Dprev, W.D, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
  DF_CUDA(cudaMemcpyAsync(W.Cprev, W.Cocc, sizeof(double) * nao * nocc, cudaMemcpyDeviceToDevice, s));
  DF_TRY(run_jk(W.B, nao, M.naux, DF_MIXED, W.D, nullptr, 0, W.J, nullptr, W.jk, s));
  {
    ProfScope ps("scf_incremental_factors", s);
    // MW = M W, A = C'_base M W, B = C' W (W = Winc^T: eigenvectors as rows)
    DF_TRY(dgemm(false, true, nocc, nocc, nocc, 1.0, W.Minc, nocc, 0, W.Winc, nocc, 0, 0.0, W.MW, nocc, 0, 1, s, 0, 0));
    DF_TRY(dgemm(false, false, nmo, nocc, nocc, 1.0, W.Cbase, nocc, 0, W.MW, nocc, 0, 0.0, W.Ainc, nocc, 0, 1, s, 0, 0));
    DF_TRY(dgemm(false, true, nmo, nocc, nocc, 1.0, W.Cp, nocc, 0, W.Winc, nocc, 0, 0.0, W.Binc, nocc, 0, 1, s, 0, 0));
    principal_pairs_kernel<<<nocc, 256, 0, s>>>(W.Ainc, W.Binc, nmo, nocc, W.Up, W.Um, W.sinc);
    DF_LAUNCHED("principal_pairs_kernel");
    DF_TRY(dgemm(false, false, nao, nocc, nmo, 1.0, W.X, nmo, 0, W.Up, nocc, 0, 0.0, W.Uao_p, nocc, 0, 1, s, 0, 0));
    DF_TRY(dgemm(false, false, nao, nocc, nmo, 1.0, W.X, nmo, 0, W.Um, nocc, 0, 0.0, W.Uao_m, nocc, 0, 1, s, 0, 0));
  }
  DF_TRY(run_jk(W.B, nao, M.naux, DF_MIXED, nullptr, W.Uao_p, nocc, nullptr, W.T2, W.jk, s));
  DF_TRY(run_jk(W.B, nao, M.naux, DF_MIXED, nullptr, W.Uao_m, nocc, nullptr, W.T1, W.jk, s));
  kacc_kernel<<<blocks_for(nn), 256, 0, s>>>(W.K, W.T2, W.T1, nn);
  DF_LAUNCHED("kacc_kernel");
  DF_CUDA(cudaMemcpyAsync(W.Cbase, W.Cp, sizeof(double) * nmo * nocc, cudaMemcpyDeviceToDevice, s));
  return M.soscf ? iteration_tail_soscf(M, DF_MIXED) : iteration_tail(M, DF_MIXED);
}

// Second half of the first iteration from a non-idempotent dm0 (after dm0_launch drained).
static int scf_dm0_finish(ScfMol& M) {
  DF_TRY(dm0_finish(M));
  DF_TRY(iteration_tail(M, M.prec));
  M.first_dm0 = false;
  return DF_OK;
}

// Launch one iteration asynchronously.  The first iteration from a non-idempotent dm0 only
// enqueues its first half here (phase DM0_EIG): scf_dm0_finish completes it.
static int scf_iter_launch(ScfMol& M, bool use_graphs) {
  if (M.first_dm0) return dm0_launch(M);
  if (M.soscf_pending) {
    DF_TRY(soscf_init(M));
    M.soscf = true;
    M.soscf_pending = false;
  }
  const bool incr = M.inc && M.kp == ScfMol::KP_INCR;
  int gi = M.prec == DF_FP64 ? 0 : (incr ? 2 : 1);
  auto body = [&]() { return incr ? iteration_body_incremental(M) : iteration_body(M, M.prec); };
  // Newton iterations run eagerly (their launch count varies with the CG length knob)
  if (!use_graphs || prof_on() || M.soscf) return body();
  if (!M.graph[gi]) {
    cudaGraph_t g = nullptr;
    DF_CUDA(cudaStreamBeginCapture(M.s, cudaStreamCaptureModeThreadLocal));
    int rc = body();
    cudaError_t ce = cudaStreamEndCapture(M.s, &g);
    if (rc != DF_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    DF_REQUIRE(ce == cudaSuccess, DF_ERR_CUDA, "scf: graph capture failed: %s", cudaGetErrorString(ce));
    cudaError_t ie = cudaGraphInstantiate(&M.graph[gi], g, 0);
    cudaGraphDestroy(g);
    DF_REQUIRE(ie == cudaSuccess, DF_ERR_CUDA, "scf: graph instantiation failed: %s", cudaGetErrorString(ie));
  }
  DF_CUDA(cudaGraphLaunch(M.graph[gi], M.s));
  return DF_OK;
}

// Phase logic of the incremental mixed exchange (after the checks common to every mode):
// FULL (mixed builds) -> BASE (one FP64 build) -> INCR (updates) -> FINAL (FP64 builds).
static bool scf_iter_finish_incremental(ScfMol& M, double de) {
  const ScfStatus& h = *M.hst;
  const scf_opts& o = M.opt;
  const bool crit = M.have_old && de < o.conv_tol && h.emax < o.conv_err;
  M.res.homo = h.homo;
  M.res.lumo = h.lumo;
  // the next update is safe when the small eigensolver worked and no principal angle
  // between the accumulated K's occupied space and the next one exceeds 60 degrees
  const bool update_ok = h.inc_fail == 0 && h.inc_min_cos2 >= 0.25;
  auto to_final = [&]() {
    M.kp = ScfMol::KP_FINAL;
    M.switched = true;
    M.prec = DF_FP64;
  };
  auto to_base = [&]() {
    M.kp = ScfMol::KP_BASE;
    M.prec = DF_FP64;
  };
  switch (M.kp) {
    case ScfMol::KP_FINAL:
      if (M.fp64_done + 1 >= o.n_fp64_final && crit) {
        M.res.converged = 1;
        return true;
      }
      M.fp64_done++;
      break;
    case ScfMol::KP_FULL: {
      if (h.emax < 0.9 * M.best_err) {
        M.best_err = h.emax;
        M.stall = 0;
      } else {
        M.stall++;
      }
      const bool stalled = (M.stall >= 10 && M.best_err < 1e-3) || 4 * M.res.iterations >= 3 * o.max_cycle;
      if (M.have_old && (h.emax < 1e-3 || de < o.switch_tol || h.emax < o.switch_err || stalled)) to_base();
      break;
    }
    case ScfMol::KP_BASE:
      // an FP64 iteration: when its error jumps well above the mixed phase's best, the mixed
      // vectors in the DIIS history do not describe the FP64 problem; restart from this one
      if (M.rebases == 0 && h.emax > 3.0 * M.best_err) {
        diis_keep_newest_kernel<<<1, 32, 0, M.s>>>(M.W.diis);
        if (cudaGetLastError() != cudaSuccess) {
          M.rc = DF_ERR_CUDA;
          set_error("scf: DIIS restart launch failed");
          return true;
        }
      }
      if (crit) {  // converged on the base build itself: it is the first final FP64 iteration
        to_final();
        M.fp64_done = 1;
        if (M.fp64_done >= o.n_fp64_final) {
          M.res.converged = 1;
          return true;
        }
      } else if (update_ok && M.rebases <= 3) {
        M.kp = ScfMol::KP_INCR;
        M.prec = DF_MIXED;
        M.inc_best = h.emax;
        M.inc_stall = 0;
      } else if (M.rebases > 3) {
        to_final();
      } else {
        M.rebases++;
      }
      break;
    case ScfMol::KP_INCR:
      if (crit || 4 * M.res.iterations >= 3 * o.max_cycle) {
        to_final();
        break;
      }
      if (h.emax < 0.9 * M.inc_best) {
        M.inc_best = h.emax;
        M.inc_stall = 0;
      } else {
        M.inc_stall++;
      }
      if (M.inc_stall >= 10 && update_ok && M.soscf_on && !M.soscf && M.rebases >= 1) {
        // still stalled after a fresh base: DIIS itself is stuck, take Newton steps
        M.soscf_pending = true;
        M.inc_stall = 0;
      } else if (!update_ok || (M.inc_stall >= 10 && !M.soscf_pending)) {
        // a large rotation, or updates that no longer reduce the error: rebuild the base
        M.rebases++;
        M.inc_stall = 0;
        if (M.rebases > 3) to_final();
        else to_base();
      }
      break;
  }
  M.e_old = h.energy;
  M.have_old = true;
  if (M.res.iterations >= M.iter_limit) {
    M.rc = DF_ERR_NOCONV;
    set_error("scf: not converged after %d iterations (dE %.3e, max|e| %.3e)", M.res.iterations, M.res.last_de,
              M.res.last_err);
    return true;
  }
  return false;
}

// After the stream has completed the iteration: convergence, precision switch.
// Returns true when the molecule is finished (converged, failed or out of iterations).
static bool scf_iter_finish(ScfMol& M) {
  const ScfStatus& h = *M.hst;
  M.res.iterations++;
  if (M.prec == DF_FP64) M.res.fp64_iterations++;
  if (h.nonfinite || !std::isfinite(h.emax)) {
    M.rc = DF_ERR_NUMERIC;
    set_error("scf: non-finite Fock matrix at iteration %d", M.res.iterations);
    return true;
  }
  if (h.tc_timeout) {
    M.rc = DF_ERR_TIMEOUT;
    set_error("scf: a bounded wait of the tensor-core exchange gave up at iteration %d", M.res.iterations);
    return true;
  }
  if (h.eig_fail == 3) {
    M.rc = DF_ERR_TIMEOUT;
    set_error("scf: a grid barrier of the eigensolver timed out at iteration %d", M.res.iterations);
    return true;
  }
  if (h.eig_fail) {
    M.rc = DF_ERR_NOCONV;
    set_error("scf: eigensolver failed at iteration %d", M.res.iterations);
    return true;
  }
  double de = M.have_old ? fabs(h.energy - M.e_old) : INFINITY;
  M.res.energy = h.energy;
  M.res.last_de = de;
  M.res.last_err = h.emax;
  if (M.opt.verbose)
    printf("scf iter %3d  %s  E = %.12f  dE = %.3e  max|e| = %.3e\n", M.res.iterations,
           M.prec == DF_FP64 ? "fp64 " : (M.inc && M.kp == ScfMol::KP_INCR ? "incr " : "mixed"), h.energy, de, h.emax);
  // DIIS progress, for the switch to Newton steps: with an accurate Fock matrix (FP64, or
  // the incremental updates) and no 10% gain on the best error for 12 iterations
  if (h.emax < 0.9 * M.d_best) {
    M.d_best = h.emax;
    M.d_stall = 0;
  } else {
    M.d_stall++;
  }
  const bool accurate_fock = M.prec == DF_FP64 || (M.inc && M.kp == ScfMol::KP_INCR);
  if (M.soscf_on && !M.soscf && !M.soscf_pending && accurate_fock && M.d_stall >= 12 && M.d_best < 0.1) {
    M.soscf_pending = true;
    M.inc_stall = 0;
  }
  if (M.inc) return scf_iter_finish_incremental(M, de);
  if (M.prec == DF_FP64 && M.switched && M.fp64_done + 1 >= M.opt.n_fp64_final && M.have_old &&
      de < M.opt.conv_tol && h.emax < M.opt.conv_err) {
    M.res.converged = 1;
    return true;
  }
  // First FP64 iteration after the switch: when its error jumps well above what the mixed
  // phase reached, the mixed-precision vectors in the DIIS history no longer describe the
  // FP64 problem (the mixed floor was high); restart the extrapolation from the new vector.
  if (M.opt.precision == DF_MIXED && M.prec == DF_FP64 && M.fp64_done == 0 && h.emax > 3.0 * M.best_err) {
    diis_keep_newest_kernel<<<1, 32, 0, M.s>>>(M.W.diis);
    if (cudaGetLastError() != cudaSuccess) {
      M.rc = DF_ERR_CUDA;
      set_error("scf: DIIS restart launch failed");
      return true;
    }
  }
  if (M.prec == DF_FP64) M.fp64_done++;
  // orbital energies of the diagonalisation that produced the next density
  M.res.homo = h.homo;
  M.res.lumo = h.lumo;
  // Mixed phase: switch on the thresholds; or when the DIIS error, already below 1e-3, has
  // not improved by 10% for 10 iterations (the floor of the mixed-precision Fock matrix; the
  // energy of the first iterations oscillates too much to judge by |dE|, and slowly
  // converging systems plateau for several iterations in FP64 too); or after three quarters
  // of the iteration budget.
  bool stalled = false;
  if (!M.switched) {
    if (h.emax < 0.9 * M.best_err) {
      M.best_err = h.emax;
      M.stall = 0;
    } else {
      M.stall++;
    }
    stalled = (M.stall >= 10 && M.best_err < 1e-3) || 4 * M.res.iterations >= 3 * M.opt.max_cycle;
  }
  if (!M.switched && M.have_old && (de < M.opt.switch_tol || h.emax < M.opt.switch_err || stalled)) {
    // The DIIS history is kept: the mixed-precision Fock matrices are close to the FP64
    // ones and keep the extrapolation informed; new FP64 vectors replace them as they age
    // (unless the first FP64 error shows they are not close, see above).
    M.switched = true;
    M.prec = DF_FP64;
  }
  M.e_old = h.energy;
  M.have_old = true;
  if (M.res.iterations >= M.iter_limit) {
    M.rc = DF_ERR_NOCONV;
    set_error("scf: not converged after %d iterations (dE %.3e, max|e| %.3e)", M.res.iterations, M.res.last_de,
              M.res.last_err);
    return true;
  }
  return false;
}

// The reported energy belongs to Dprev / Cprev, the density of the last Fock build.
static int scf_outputs(ScfMol& M) {
  ScfWork& W = M.W;
  const long nn = (long)M.nao * M.nao;
  if (M.D_out) DF_CUDA(cudaMemcpyAsync(M.D_out, W.Dprev, sizeof(double) * nn, cudaMemcpyDeviceToDevice, M.s));
  if (M.C_out)
    DF_CUDA(cudaMemcpyAsync(M.C_out, W.Cprev, sizeof(double) * M.nao * M.nocc, cudaMemcpyDeviceToDevice, M.s));
  if (M.mo_out)
    DF_CUDA(cudaMemcpyAsync(M.mo_out, W.eps, sizeof(double) * std::min(M.nmo, M.nocc + 1), cudaMemcpyDeviceToDevice,
                            M.s));
  return DF_OK;
}

static int check_molecule(const df_molecule* mol, const scf_opts& o) {
  DF_REQUIRE(mol, DF_ERR_ARG, "scf: null molecule");
  DF_REQUIRE(mol->nao > 0 && mol->naux > 0 && mol->natm > 0 && mol->nelec > 0 && mol->nelec % 2 == 0, DF_ERR_ARG,
             "scf: bad molecule sizes (nao %d naux %d natm %d nelec %d)", mol->nao, mol->naux, mol->natm, mol->nelec);
  DF_REQUIRE(mol->xyz && mol->charges && mol->ao_xyz && mol->ao_exp && mol->aux_xyz && mol->aux_exp, DF_ERR_ARG,
             "scf: null molecule array");
  DF_REQUIRE(o.precision == DF_FP64 || o.precision == DF_MIXED, DF_ERR_ARG, "scf: bad precision");
  DF_REQUIRE(o.diis_space >= 1 && o.diis_space <= DIIS_MAX, DF_ERR_ARG, "scf: diis_space must be in [1, 16]");
  DF_REQUIRE(o.max_cycle >= 1 && o.n_fp64_final >= 1, DF_ERR_ARG, "scf: bad iteration limits");
  DF_REQUIRE(mol->naux <= 65535, DF_ERR_ARG, "scf: naux > 65535");
  DF_REQUIRE(mol->nelec / 2 <= mol->nao, DF_ERR_ARG, "scf: more occupied orbitals than basis functions");
  DF_REQUIRE(o.precision == DF_FP64 || mol->nelec / 2 <= 256, DF_ERR_ARG,
             "scf: mixed precision supports at most 256 occupied orbitals");
  return DF_OK;
}

int scf_run_on(const df_molecule* mol, const scf_opts& o, const double* dm0, double* D_out, double* C_out,
               double* mo_energy, scf_result* res, void* work, size_t work_bytes, cudaStream_t s);

static int init_mol(ScfMol& M, const df_molecule* mol, const scf_opts& o, void* work, size_t work_bytes,
                    cudaStream_t s) {
  M.mol = *mol;
  M.opt = o;
  M.iter_limit = o.max_cycle;
  M.res.hess_min = NAN;
  M.nao = mol->nao;
  M.naux = mol->naux;
  M.nocc = mol->nelec / 2;
  M.s = s;
  Arena a(work, work_bytes);
  scf_layout(M.nao, M.naux, M.nocc, o.precision, &a, nullptr, &M.W);
  DF_REQUIRE(!a.overflow, DF_ERR_NOMEM, "scf: workspace overflow");
  return DF_OK;
}

}  // namespace dfscf

using namespace dfscf;

extern "C" void scf_default_opts(scf_opts* o) {
  if (!o) return;
  o->precision = DF_FP64;
  o->diis_space = 8;
  o->max_cycle = 100;
  o->n_fp64_final = 2;
  o->conv_tol = 1e-8;
  o->conv_err = 1e-5;
  o->lindep = 1e-8;
  o->switch_tol = 3e-8;
  o->switch_err = 3e-5;
  o->verbose = 0;
  o->guess_params = nullptr;
}

extern "C" size_t scf_work_bytes(int nao, int naux, int nocc, int precision) {
  if (nao <= 0 || naux <= 0 || nocc <= 0) return 0;
  Sizer z;
  ScfWork w;
  scf_layout(nao, naux, nocc, precision, nullptr, &z, &w);
  return z.used;
}

extern "C" int scf_run(const df_molecule* mol, const scf_opts* opt, const double* dm0, double* D_out, double* C_out,
                       double* mo_energy, scf_result* res, void* work, size_t work_bytes, cudaStream_t s) {
  clear_error();
  DF_REQUIRE(res, DF_ERR_ARG, "scf_run: null result");
  scf_opts o;
  if (opt) o = *opt; else scf_default_opts(&o);
  DF_TRY(check_molecule(mol, o));
  size_t need = scf_work_bytes(mol->nao, mol->naux, mol->nelec / 2, o.precision);
  DF_REQUIRE(work && work_bytes >= need, DF_ERR_NOMEM, "scf_run: workspace of %zu bytes < %zu", work_bytes, need);
  // The iterations are captured into CUDA graphs, which the legacy default stream does
  // not allow; run on a private stream ordered after the caller's and join back at the end.
  cudaStream_t ps = nullptr;
  cudaEvent_t ev = nullptr;
  DF_CUDA(cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking));
  DF_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  DF_CUDA(cudaEventRecord(ev, s));
  DF_CUDA(cudaStreamWaitEvent(ps, ev, 0));
  int rc_run = scf_run_on(mol, o, dm0, D_out, C_out, mo_energy, res, work, work_bytes, ps);
  cudaEventRecord(ev, ps);
  cudaStreamWaitEvent(s, ev, 0);
  cudaStreamSynchronize(ps);
  cudaEventDestroy(ev);
  cudaStreamDestroy(ps);
  return rc_run;
}

namespace dfscf {

int scf_run_on(const df_molecule* mol, const scf_opts& o, const double* dm0, double* D_out, double* C_out,
               double* mo_energy, scf_result* res, void* work, size_t work_bytes, cudaStream_t s) {
  ScfMol M;
  DF_TRY(init_mol(M, mol, o, work, work_bytes, s));
  ScfStatus* hst = nullptr;
  double* heps = nullptr;
  int* hints = nullptr;
  DF_CUDA(cudaMallocHost(&hst, sizeof(ScfStatus)));
  DF_CUDA(cudaMallocHost(&heps, sizeof(double) * (mol->nao + 1)));
  DF_CUDA(cudaMallocHost(&hints, sizeof(int) * 2));
  double* hdav = nullptr;
  DF_CUDA(cudaMallocHost(&hdav, sizeof(double) * kDavHost));
  M.h_dav = hdav;
  M.hst = hst;
  M.h_eps = heps;
  M.h_ints = hints;
  M.dm0 = dm0;
  M.D_out = D_out;
  M.C_out = C_out;
  M.mo_out = mo_energy;
  int rc = scf_setup(M);
  for (;;) {
    while (rc == DF_OK && !M.done) {
      const bool dm0_first = M.first_dm0;
      rc = scf_iter_launch(M, true);
      if (rc == DF_OK && dm0_first) {
        rc = cudaStreamSynchronize(s) == cudaSuccess ? scf_dm0_finish(M) : DF_ERR_CUDA;
        if (rc == DF_ERR_CUDA) set_error("scf_run: %s", cudaGetErrorString(cudaGetLastError()));
      }
      if (rc != DF_OK) break;
      cudaError_t e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        set_error("scf_run: %s", cudaGetErrorString(e));
        rc = DF_ERR_CUDA;
        break;
      }
      M.done = scf_iter_finish(M);
    }
    if (rc == DF_OK) rc = scf_outputs(M);
    if (rc == DF_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = DF_ERR_CUDA;
    M.res.hess_min = NAN;
    if (!(rc == DF_OK && M.rc == DF_OK && M.res.converged && knob("stability"))) break;
    const bool follow = knob("stability") >= 2 && M.res.stability_restarts < kMaxEscapes;
    rc = stability_analysis(M, follow ? kEscapeAngle : 0.0);
    if (rc != DF_OK || !follow || !(M.res.hess_min < kSaddleTol)) break;
    rc = escape_saddle(M);
  }
  *res = M.res;
  cudaFreeHost(hdav);
  cudaFreeHost(hst);
  cudaFreeHost(heps);
  cudaFreeHost(hints);
  return rc != DF_OK ? rc : M.rc;
}

}  // namespace dfscf

// ---- batch ---------------------------------------------------------------------------------------
extern "C" size_t scf_batch_work_bytes(const df_molecule* mols, int nmol, int precision, int slots) {
  if (!mols || nmol <= 0 || slots <= 0) return 0;
  size_t mx = 0;
  for (int i = 0; i < nmol; ++i)
    mx = std::max(mx, scf_work_bytes(mols[i].nao, mols[i].naux, std::max(1, mols[i].nelec / 2), precision));
  return align_up(mx, 256) * (size_t)std::min(slots, nmol);
}

// First-fit allocator over the batch workspace: molecules of uneven size take regions of
// their own size, so many small molecules run beside a few large ones.  Free regions are
// kept sorted by offset and merged with their neighbours when a region is released.
namespace dfscf {
class RegionPool {
 public:
  explicit RegionPool(size_t bytes) { free_.push_back({0, bytes}); }
  // offset of a region of `bytes` (256-byte aligned), or SIZE_MAX when none fits
  size_t take(size_t bytes) {
    bytes = align_up(bytes, 256);
    for (size_t i = 0; i < free_.size(); ++i)
      if (free_[i].size >= bytes) {
        const size_t off = free_[i].off;
        free_[i].off += bytes;
        free_[i].size -= bytes;
        if (free_[i].size == 0) free_.erase(free_.begin() + (long)i);
        return off;
      }
    return SIZE_MAX;
  }
  void give(size_t off, size_t bytes) {
    bytes = align_up(bytes, 256);
    size_t i = 0;
    while (i < free_.size() && free_[i].off < off) ++i;
    free_.insert(free_.begin() + (long)i, {off, bytes});
    if (i + 1 < free_.size() && free_[i].off + free_[i].size == free_[i + 1].off) {
      free_[i].size += free_[i + 1].size;
      free_.erase(free_.begin() + (long)i + 1);
    }
    if (i > 0 && free_[i - 1].off + free_[i - 1].size == free_[i].off) {
      free_[i - 1].size += free_[i].size;
      free_.erase(free_.begin() + (long)i);
    }
  }

 private:
  struct Region {
    size_t off, size;
  };
  std::vector<Region> free_;
};
}  // namespace dfscf

extern "C" int scf_run_batch(const df_molecule* mols, int nmol, const scf_opts* opt, const double* const* dm0s,
                             double* const* D_outs, scf_result* results, int slots, void* work, size_t work_bytes,
                             cudaStream_t s) {
  clear_error();
  DF_REQUIRE(mols && nmol > 0 && results && slots > 0, DF_ERR_ARG, "scf_run_batch: bad arguments");
  scf_opts o;
  if (opt) o = *opt; else scf_default_opts(&o);
  o.verbose = 0;
  for (int i = 0; i < nmol; ++i) DF_TRY(check_molecule(&mols[i], o));
  slots = std::min(slots, nmol);
  std::vector<size_t> bytes(nmol);
  size_t largest = 0;
  for (int i = 0; i < nmol; ++i) {
    bytes[i] = align_up(scf_work_bytes(mols[i].nao, mols[i].naux, mols[i].nelec / 2, o.precision), 256);
    largest = std::max(largest, bytes[i]);
  }
  DF_REQUIRE(work && work_bytes >= largest, DF_ERR_NOMEM,
             "scf_run_batch: workspace of %zu bytes cannot hold the largest molecule (%zu bytes)", work_bytes, largest);
  memset(results, 0, sizeof(scf_result) * nmol);
  // largest molecules first: the long runs start early and small ones fill the gaps
  std::vector<int> order(nmol);
  for (int i = 0; i < nmol; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return bytes[a] > bytes[b]; });
  RegionPool pool(work_bytes);
  // stream pool, ordered after the caller's stream
  std::vector<cudaStream_t> streams(slots, nullptr);
  cudaEvent_t start;
  DF_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
  DF_CUDA(cudaEventRecord(start, s));
  for (int k = 0; k < slots; ++k) {
    DF_CUDA(cudaStreamCreateWithFlags(&streams[k], cudaStreamNonBlocking));
    DF_CUDA(cudaStreamWaitEvent(streams[k], start, 0));
  }
  int max_nao = 0;
  for (int i = 0; i < nmol; ++i) max_nao = std::max(max_nao, mols[i].nao);
  ScfStatus* hst = nullptr;
  double* heps = nullptr;
  int* hints = nullptr;
  DF_CUDA(cudaMallocHost(&hst, sizeof(ScfStatus) * slots));
  DF_CUDA(cudaMallocHost(&heps, sizeof(double) * (size_t)(max_nao + 1) * slots));
  DF_CUDA(cudaMallocHost(&hints, sizeof(int) * 2 * slots));
  double* hdav = nullptr;
  DF_CUDA(cudaMallocHost(&hdav, sizeof(double) * kDavHost * slots));
  std::vector<ScfMol*> slot_mol(slots, nullptr);
  std::vector<int> slot_index(slots, -1);
  std::vector<size_t> slot_off(slots, 0);
  int next = 0, finished = 0, running = 0, rc = DF_OK;
  // Each running molecule holds a stream and a region of the workspace until it finishes.
  // The host polls the streams and advances whichever molecule's stream has drained: it
  // never blocks on one molecule while others could run.  A stream slot that frees up takes
  // the next molecule (in the size order above) as soon as its region fits.
  auto try_start = [&](int k) -> int {
    if (next >= nmol) return DF_OK;
    const int i = order[next];
    const size_t off = pool.take(bytes[i]);
    if (off == SIZE_MAX) return DF_OK;  // wait until a running molecule returns its region
    next++;
    ScfMol* M = new ScfMol();
    slot_mol[k] = M;
    slot_index[k] = i;
    slot_off[k] = off;
    running++;
    DF_TRY(init_mol(*M, &mols[i], o, (char*)work + off, bytes[i], streams[k]));
    // With several molecules in flight each diagonalises on one CTA: many one-CTA
    // eigensolvers fill the SMs in parallel, while cooperative grids from different streams
    // (one CTA per SM each) would contend for co-residency.
    if (slots > 1) M->W.eig_aux = nullptr;
    M->hst = hst + k;
    M->h_eps = heps + (size_t)(max_nao + 1) * k;
    M->h_ints = hints + 2 * k;
    M->h_dav = hdav + (size_t)kDavHost * k;
    M->dm0 = dm0s ? dm0s[i] : nullptr;
    M->D_out = D_outs ? D_outs[i] : nullptr;
    int r = setup_launch(*M);
    if (r != DF_OK) {
      M->rc = r;
      M->phase = ScfMol::DONE;
    }
    return DF_OK;
  };
  // Advance one molecule whose stream is idle; returns a fatal status.
  auto advance = [&](int k) -> int {
    ScfMol* M = slot_mol[k];
    int r = DF_OK;
    switch (M->phase) {
      case ScfMol::SETUP:
        r = setup_orthogonalize(*M);
        break;
      case ScfMol::GUESS_CHECK:
        r = setup_guess(*M);
        break;
      case ScfMol::READY:
        r = scf_iter_launch(*M, true);
        if (r == DF_OK) M->phase = M->first_dm0 ? ScfMol::DM0_EIG : ScfMol::ITER;
        break;
      case ScfMol::DM0_EIG:
        r = scf_dm0_finish(*M);
        if (r == DF_OK) M->phase = ScfMol::ITER;
        break;
      case ScfMol::ITER:
        if (scf_iter_finish(*M)) {
          M->phase = ScfMol::DONE;
          if (M->rc == DF_OK && M->res.converged && knob("stability")) {
            // outputs of this solution first (the analysis overwrites the orbitals), then the
            // analysis, advanced like the iterations whenever this stream is idle
            r = scf_outputs(*M);
            M->outputs_done = true;
            const bool follow = knob("stability") >= 2 && M->res.stability_restarts < kMaxEscapes;
            if (r == DF_OK) r = dav_begin(*M, follow ? kEscapeAngle : 0.0);
            if (r == DF_OK) M->phase = ScfMol::STAB;
          }
        } else {
          r = scf_iter_launch(*M, true);
        }
        break;
      case ScfMol::STAB: {
        bool fin = false;
        r = dav_advance(*M, &fin);
        if (r == DF_OK && fin) {
          const bool follow = knob("stability") >= 2 && M->res.stability_restarts < kMaxEscapes;
          if (follow && M->res.hess_min < kSaddleTol) {
            // a saddle point: turn along its mode and iterate on
            r = escape_saddle(*M);
            if (r == DF_OK) r = scf_iter_launch(*M, true);
            M->outputs_done = false;
            M->phase = ScfMol::ITER;
          } else {
            M->phase = ScfMol::DONE;
          }
        }
        break;
      }
      case ScfMol::DONE:
        break;
    }
    if (r != DF_OK) {
      // a per-molecule failure (metric, eigensolver, guess) ends that molecule only
      if (r == DF_ERR_CUDA) return r;
      M->rc = r;
      M->phase = ScfMol::DONE;
    }
    if (M->phase == ScfMol::DONE) {
      const int i = slot_index[k];
      if ((M->rc == DF_OK || M->rc == DF_ERR_NOCONV) && !M->outputs_done) DF_TRY(scf_outputs(*M));
      results[i] = M->res;
      // the region goes back to the pool only once this stream has finished with it: the
      // outputs above are its last work, so wait for them
      DF_CUDA(cudaStreamSynchronize(streams[k]));
      delete M;
      slot_mol[k] = nullptr;
      pool.give(slot_off[k], bytes[i]);
      finished++;
      running--;
    }
    return DF_OK;
  };
  while (rc == DF_OK && finished < nmol) {
    bool progressed = false;
    for (int k = 0; k < slots && rc == DF_OK; ++k) {
      if (!slot_mol[k]) {
        const int before = next;
        rc = try_start(k);
        if (next != before) progressed = true;
        continue;
      }
      cudaError_t q = cudaStreamQuery(streams[k]);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) {
        set_error("scf_run_batch: %s", cudaGetErrorString(q));
        rc = DF_ERR_CUDA;
        break;
      }
      progressed = true;
      rc = advance(k);
    }
    if (rc == DF_OK && running == 0 && next < nmol) {
      // nothing runs and the next molecule still does not fit: cannot happen while the
      // workspace holds the largest molecule, but never spin on it
      set_error("scf_run_batch: molecule %d does not fit in the workspace", order[next]);
      rc = DF_ERR_NOMEM;
    }
    if (!progressed && rc == DF_OK) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  for (int k = 0; k < slots; ++k) {
    cudaStreamSynchronize(streams[k]);
    delete slot_mol[k];
    cudaStreamDestroy(streams[k]);
  }
  cudaEventDestroy(start);
  cudaFreeHost(hdav);
  cudaFreeHost(hst);
  cudaFreeHost(heps);
  cudaFreeHost(hints);
  if (rc != DF_OK) return rc;
  for (int i = 0; i < nmol; ++i)
    if (!results[i].converged) {
      set_error("scf_run_batch: molecule %d did not converge", i);
      return DF_ERR_NOCONV;
    }
  return DF_OK;
}

// ---- core-Hamiltonian guess -------------------------------------------------------------
namespace dfscf {

static void guess_layout(int nao, int nocc, Arena* a, Sizer* z, ScfWork* w) {
  size_t nn = (size_t)nao * nao;
#define TAKE(T, ptr, count) \
  if (a) ptr = a->take<T>(count); else z->take<T>(count);
  TAKE(double, w->S, nn);
  TAKE(double, w->h, nn);
  TAKE(double, w->V, nn);
  TAKE(double, w->X, nn);
  TAKE(double, w->T1, nn);
  TAKE(double, w->T2, nn);
  TAKE(double, w->Fp, nn);
  TAKE(double, w->ZT, nn);
  TAKE(double, w->eps, nao);
  TAKE(double, w->eig_scratch, eigh_full_scratch_doubles(nao));
  TAKE(int, w->eig_status, 1);
  TAKE(char, w->eig_aux, eigh_coop_aux_bytes(nao));
  TAKE(double, w->Cocc, (size_t)nao * std::max(nocc, 1));
  TAKE(double, w->Cp, (size_t)nao * std::max(nocc, 1));
  TAKE(double, w->D, nn);
#undef TAKE
}

}  // namespace dfscf

extern "C" size_t df_core_guess_work_bytes(int nao, int nocc) {
  if (nao <= 0 || nocc < 0) return 0;
  Sizer z;
  ScfWork w;
  guess_layout(nao, nocc, nullptr, &z, &w);
  return z.used;
}

extern "C" int df_core_guess(const df_molecule* mol, double lindep, double* S_out, double* h_out, double* C_occ,
                             double* D_out, double* mo_energy, int* nmo_out, void* work, size_t work_bytes,
                             cudaStream_t s) {
  clear_error();
  DF_REQUIRE(mol && mol->nao > 0 && mol->natm > 0 && mol->nelec > 0 && mol->nelec % 2 == 0, DF_ERR_ARG,
             "df_core_guess: bad molecule");
  DF_REQUIRE(mol->ao_xyz && mol->ao_exp && mol->xyz && mol->charges, DF_ERR_ARG, "df_core_guess: null array");
  const int nao = mol->nao, nocc = mol->nelec / 2;
  DF_REQUIRE(nocc <= nao, DF_ERR_ARG, "df_core_guess: nocc > nao");
  size_t need = df_core_guess_work_bytes(nao, nocc);
  DF_REQUIRE(work && work_bytes >= need, DF_ERR_NOMEM, "df_core_guess: workspace of %zu bytes < %zu", work_bytes, need);
  Arena a(work, work_bytes);
  ScfWork W;
  guess_layout(nao, nocc, &a, nullptr, &W);
  const long nn = (long)nao * nao;
  DF_TRY(launch_int1e(mol->ao_xyz, mol->ao_exp, nao, mol->xyz, mol->charges, mol->natm, W.S, W.h, W.V, s));
  axpy_kernel<<<blocks_for(nn), 256, 0, s>>>(W.h, W.V, nn, 1.0);
  DF_LAUNCHED("axpy_kernel");
  DF_CUDA(cudaMemcpyAsync(W.T1, W.S, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
  DF_TRY(eig_rows(W.T1, nao, W.eps, W.ZT, W, s));
  std::vector<double> hs(nao);
  int bad = 0;
  DF_CUDA(cudaMemcpyAsync(hs.data(), W.eps, sizeof(double) * nao, cudaMemcpyDeviceToHost, s));
  DF_CUDA(cudaMemcpyAsync(&bad, W.eig_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  DF_CUDA(cudaStreamSynchronize(s));
  DF_REQUIRE(bad != 3, DF_ERR_TIMEOUT, "df_core_guess: a grid barrier of the eigensolver timed out on S");
  DF_REQUIRE(bad == 0, DF_ERR_NOCONV, "df_core_guess: eigensolver failed on S");
  int nmo = 0;
  for (int i = 0; i < nao; ++i) nmo += hs[i] > lindep;
  DF_REQUIRE(nmo >= nocc, DF_ERR_ARG, "df_core_guess: only %d orbitals above lindep", nmo);
  canonical_x_kernel<<<blocks_for((long)nao * nmo), 256, 0, s>>>(W.ZT, W.eps, nao, nmo, W.X);
  DF_LAUNCHED("canonical_x_kernel");
  DF_TRY(diagonalize_fock(W.h, nao, nmo, nocc, W, s));
  if (S_out) DF_CUDA(cudaMemcpyAsync(S_out, W.S, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
  if (h_out) DF_CUDA(cudaMemcpyAsync(h_out, W.h, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
  if (C_occ) DF_CUDA(cudaMemcpyAsync(C_occ, W.Cocc, sizeof(double) * nao * nocc, cudaMemcpyDeviceToDevice, s));
  if (D_out) DF_CUDA(cudaMemcpyAsync(D_out, W.D, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
  if (mo_energy)
    DF_CUDA(cudaMemcpyAsync(mo_energy, W.eps, sizeof(double) * std::min(nmo, nocc + 1), cudaMemcpyDeviceToDevice, s));
  bad = 0;
  DF_CUDA(cudaMemcpyAsync(&bad, W.eig_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  DF_CUDA(cudaStreamSynchronize(s));
  DF_REQUIRE(bad != 3, DF_ERR_TIMEOUT, "df_core_guess: a grid barrier of the eigensolver timed out");
  DF_REQUIRE(bad == 0, DF_ERR_NOCONV, "df_core_guess: eigensolver failed on the core Hamiltonian");
  if (nmo_out) *nmo_out = nmo;
  return DF_OK;
}

DF_BOUNDS_READER(bounds_read_scf)
