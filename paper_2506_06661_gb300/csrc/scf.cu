// Restricted Hartree-Fock SCF over the DF Fock build, with Pulay DIIS and the
// mixed -> FP64 precision switch.  The paper (arXiv 2506.06661) uses DF mean-field
// methods (Section "Density fitting") and names DIIS as the default accelerator
// (Section "Second-Order Self-Consistent Field"); the formulas are the textbook ones:
//   F = h + J[D] - K,  K = K[C_occ] = 1/2 K[D] for D = 2 C_occ C_occ^T,
//   E = 1/2 tr(D (h + F)) + E_nuc,
//   e = X^T (F D S - S D F) X,  X = U s^-1/2 over eigenvalues s > lindep of S,
//   Fbar = sum_i c_i F_i with [[B, -1], [-1, 0]] [c, lam] = [0, -1], B_ij = <e_i, e_j>.
// Every matrix operation runs on the GPU; the host only reads a 64-byte status block per
// iteration to decide convergence.  A starting density dm0 need not be idempotent
// (Section "Initial Guess for Mean-field Methods"); its exchange matrix is formed from
// the eigen-decomposition dm0 = sum_k n_k u_k u_k^T as K[C+] - K[C-].
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace dfscf {

struct ScfStatus {
  double energy;
  double emax;
  double trDS;
  double idem;   // ||D S D - 2 D||_F / ||D||_F
  int singular;  // DIIS system had no usable pivot
  int nonfinite;
};

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

// comm = T - T^T (T = F D S);  for the DIIS error this is F D S - S D F.
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

// G[slot][j] = G[j][slot] = <E[slot], E[j]> for the occupied history slots.
// E holds one nmo x nmo error matrix per slot (slot stride nn, ne = nmo*nmo entries used).
__global__ void diis_gram_kernel(const double* __restrict__ E, long nn, long ne, int space, int slot,
                                 const int* __restrict__ valid, double* __restrict__ G) {
  __shared__ double sh[32];
  int j = blockIdx.x;
  if (!valid[j]) return;
  const double* a = E + (size_t)slot * nn;
  const double* b = E + (size_t)j * nn;
  double s = 0.0;
  for (long i = threadIdx.x; i < ne; i += blockDim.x) s += a[i] * b[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) {
    G[slot * space + j] = s;
    G[j * space + slot] = s;
  }
}

// Solve the bordered Pulay system for the m valid slots (listed in order[]), one lane.
// On a singular system the newest vector gets coefficient 1 and st->singular is set.
__global__ void diis_solve_kernel(const double* __restrict__ G, int space, const int* __restrict__ order, int m,
                                  int newest, double* __restrict__ coef, ScfStatus* st) {
  if (threadIdx.x != 0) return;
  double A[17][18];
  int dim = m + 1;
  double scale = 0.0;
  for (int i = 0; i < m; ++i) scale = fmax(scale, fabs(G[order[i] * space + order[i]]));
  if (!(scale > 0.0)) scale = 1.0;
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j < m; ++j) A[i][j] = G[order[i] * space + order[j]] / scale;
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
  for (int i = 0; i < space; ++i) coef[i] = 0.0;
  if (ok) {
    double x[17];
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
    for (int i = 0; i < space; ++i) coef[i] = 0.0;
    coef[newest] = 1.0;
  }
  st->singular = ok ? 0 : 1;
}

// out = sum_s coef[s] Fh[s] over valid slots.
__global__ void diis_combine_kernel(const double* __restrict__ Fh, long nn, int space, const double* __restrict__ coef,
                                    const int* __restrict__ valid, double* __restrict__ out) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  double s = 0.0;
  for (int k = 0; k < space; ++k)
    if (valid[k]) s += coef[k] * Fh[(size_t)k * nn + i];
  out[i] = s;
}

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

__global__ void scale_kernel(double* __restrict__ x, long n, double a) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] *= a;
}

__global__ void axpy_kernel(double* __restrict__ y, const double* __restrict__ x, long n, double a) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += a * x[i];
}

// trDS = sum D S;  idem = ||D S D - 2 D||_F / ||D||_F  (T = D S D given).
__global__ void guess_check_kernel(const double* __restrict__ D, const double* __restrict__ S,
                                   const double* __restrict__ T, long nn, ScfStatus* st) {
  __shared__ double sh[32];
  double tr = 0.0, r2 = 0.0, d2 = 0.0;
  for (long i = threadIdx.x; i < nn; i += blockDim.x) {
    tr += D[i] * S[i];
    double r = T[i] - 2.0 * D[i];
    r2 += r * r;
    d2 += D[i] * D[i];
  }
  tr = block_sum(tr, sh);
  r2 = block_sum(r2, sh);
  d2 = block_sum(d2, sh);
  if (threadIdx.x == 0) {
    st->trDS = tr;
    st->idem = d2 > 0.0 ? sqrt(r2 / d2) : INFINITY;
  }
}

// Columns of eigenvector rows ZT [n][n] with eigenvalue w > thr (pos) or < -thr (neg),
// scaled by sqrt(|w|/2):  dm0 / 2 = C+ C+^T - C- C-^T.
__global__ void split_density_kernel(const double* __restrict__ ZT, const double* __restrict__ w, int n,
                                     const int* __restrict__ idx, int cnt, double* __restrict__ Cout) {
  long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long)n * cnt) return;
  int i = (int)(q / cnt), j = (int)(q % cnt);
  int k = idx[j];
  Cout[q] = ZT[(size_t)k * n + i] * sqrt(fabs(w[k]) * 0.5);
}

static unsigned blocks_for(long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

struct ScfWork {
  double *L, *pair_tab, *S, *h, *V, *X, *F, *Fbar, *J, *K, *D, *Cocc, *T1, *T2, *E, *Fp, *ZT, *eps, *Fhist, *Ehist,
      *G, *coef, *eig_scratch, *enuc, *Cchunk;
  int *valid, *order, *eig_status, *chol_status, *idx;
  double* maxdiag;
  ScfStatus* st;
  void* B;
  JKWork jk;
};

static void scf_layout(int nao, int naux, int nocc, int precision, Arena* a, Sizer* z, ScfWork* w) {
  size_t nn = (size_t)nao * nao;
  const int space = 16;
#define TAKE(T, ptr, count) \
  if (a) ptr = a->take<T>(count); else z->take<T>(count);
  TAKE(double, w->L, (size_t)naux * naux);
  TAKE(double, w->pair_tab, 5 * (size_t)npair_of(nao));
  TAKE(double, w->S, nn);
  TAKE(double, w->h, nn);
  TAKE(double, w->V, nn);
  TAKE(double, w->X, nn);
  TAKE(double, w->F, nn);
  TAKE(double, w->Fbar, nn);
  TAKE(double, w->J, nn);
  TAKE(double, w->K, nn);
  TAKE(double, w->D, nn);
  TAKE(double, w->Cocc, (size_t)nao * nocc);
  TAKE(double, w->Cchunk, (size_t)nao * nocc);
  TAKE(double, w->T1, nn);
  TAKE(double, w->T2, nn);
  TAKE(double, w->E, nn);
  TAKE(double, w->Fp, nn);
  TAKE(double, w->ZT, nn);
  TAKE(double, w->eps, nao);
  TAKE(double, w->Fhist, space * nn);
  TAKE(double, w->Ehist, space * nn);
  TAKE(double, w->G, space * space);
  TAKE(double, w->coef, space);
  TAKE(double, w->eig_scratch, eigh_scratch_doubles(nao));
  TAKE(double, w->enuc, 1);
  TAKE(double, w->maxdiag, 1);
  TAKE(int, w->valid, space);
  TAKE(int, w->order, space);
  TAKE(int, w->eig_status, 1);
  TAKE(int, w->chol_status, 1);
  TAKE(int, w->idx, nao);
  TAKE(ScfStatus, w->st, 1);
  if (a) w->B = a->take<char>(df_B_bytes(nao, naux, precision)); else z->take<char>(df_B_bytes(nao, naux, precision));
#undef TAKE
  w->jk = jk_work_layout(nao, naux, nocc, precision, a, z);
}

// Eigenpairs of the symmetric n x n matrix in `A` (destroyed): w ascending, rows ZT.
static int eig_sync(double* A, int n, double* w, double* ZT, ScfWork& W, cudaStream_t s) {
  DF_TRY(eigh_rows(A, n, w, ZT, W.eig_scratch, W.eig_status, s));
  return DF_OK;
}

// Occupied coefficients from a Fock-like matrix: C_occ = X C'_occ, D = 2 C C^T.
static int diagonalize_fock(const double* Fm, int nao, int nmo, int nocc, ScfWork& W, cudaStream_t s) {
  // Fp = X^T F X
  DF_TRY(dgemm(false, false, nao, nmo, nao, 1.0, Fm, nao, 0, W.X, nmo, 0, 0.0, W.T1, nmo, 0, 1, s, 0, 0));
  DF_TRY(dgemm(true, false, nmo, nmo, nao, 1.0, W.X, nmo, 0, W.T1, nmo, 0, 0.0, W.Fp, nmo, 0, 1, s, 0, 0));
  DF_TRY(eig_sync(W.Fp, nmo, W.eps, W.ZT, W, s));
  occ_columns_kernel<<<blocks_for((long)nmo * nocc), 256, 0, s>>>(W.ZT, nmo, nocc, W.T2);
  DF_LAUNCHED("occ_columns_kernel");
  DF_TRY(dgemm(false, false, nao, nocc, nmo, 1.0, W.X, nmo, 0, W.T2, nocc, 0, 0.0, W.Cocc, nocc, 0, 1, s, 0, 0));
  DF_TRY(dgemm(false, true, nao, nao, nocc, 2.0, W.Cocc, nocc, 0, W.Cocc, nocc, 0, 0.0, W.D, nao, 0, 1, s, 0, 0));
  return DF_OK;
}

int scf_driver(const df_molecule* mol, const scf_opts* o, const double* dm0, double* D_out, double* C_out,
               double* mo_energy, scf_result* res, ScfWork& W, cudaStream_t s) {
  const int nao = mol->nao, naux = mol->naux, nocc = mol->nelec / 2;
  const long nn = (long)nao * nao;
  const int space = o->diis_space;
  memset(res, 0, sizeof(*res));
  // ---- integrals, metric, B ----------------------------------------------------------
  DF_TRY(launch_int1e(mol->ao_xyz, mol->ao_exp, nao, mol->xyz, mol->charges, mol->natm, W.S, W.T1, W.V, s));
  axpy_kernel<<<blocks_for(nn), 256, 0, s>>>(W.T1, W.V, nn, 1.0);
  DF_LAUNCHED("axpy_kernel");
  DF_CUDA(cudaMemcpyAsync(W.h, W.T1, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
  DF_TRY(launch_enuc(mol->xyz, mol->charges, mol->natm, W.enuc, s));
  DF_TRY(launch_int2c(mol->aux_xyz, mol->aux_exp, naux, W.L, s));
  DF_TRY(cholesky_inplace(W.L, naux, W.chol_status, W.maxdiag, 1e-14, s));
  int chol_bad = -1;
  DF_CUDA(cudaMemcpyAsync(&chol_bad, W.chol_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  DF_CUDA(cudaStreamSynchronize(s));
  DF_REQUIRE(chol_bad < 0, DF_ERR_NOT_SPD, "scf_run: auxiliary metric not positive definite at pivot %d", chol_bad);
  DF_TRY(build_B(mol->ao_xyz, mol->ao_exp, nao, mol->aux_xyz, mol->aux_exp, naux, W.L, o->precision, W.B, W.pair_tab, s));
  // ---- canonical orthogonalisation ----------------------------------------------------
  DF_CUDA(cudaMemcpyAsync(W.T1, W.S, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
  DF_TRY(eig_sync(W.T1, nao, W.eps, W.ZT, W, s));
  std::vector<double> hs(nao);
  int eig_bad = 0;
  DF_CUDA(cudaMemcpyAsync(hs.data(), W.eps, sizeof(double) * nao, cudaMemcpyDeviceToHost, s));
  DF_CUDA(cudaMemcpyAsync(&eig_bad, W.eig_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  DF_CUDA(cudaMemcpyAsync(&res->e_nuc, W.enuc, sizeof(double), cudaMemcpyDeviceToHost, s));
  DF_CUDA(cudaStreamSynchronize(s));
  DF_REQUIRE(eig_bad == 0, DF_ERR_NOCONV, "scf_run: eigensolver failed on S");
  int nmo = 0;
  for (int i = 0; i < nao; ++i) nmo += hs[i] > o->lindep;
  DF_REQUIRE(nmo >= nocc + 1 || (nmo >= nocc && nocc > 0), DF_ERR_ARG, "scf_run: only %d orbitals after lindep", nmo);
  res->nmo = nmo;
  canonical_x_kernel<<<blocks_for((long)nao * nmo), 256, 0, s>>>(W.ZT, W.eps, nao, nmo, W.X);
  DF_LAUNCHED("canonical_x_kernel");
  // ---- guess ---------------------------------------------------------------------------
  bool use_dm0 = false;
  if (dm0) {
    DF_TRY(dgemm(false, false, nao, nao, nao, 1.0, dm0, nao, 0, W.S, nao, 0, 0.0, W.T1, nao, 0, 1, s, 0, 0));
    DF_TRY(dgemm(false, false, nao, nao, nao, 1.0, W.T1, nao, 0, dm0, nao, 0, 0.0, W.T2, nao, 0, 1, s, 0, 0));
    guess_check_kernel<<<1, 1024, 0, s>>>(dm0, W.S, W.T2, nn, W.st);
    DF_LAUNCHED("guess_check_kernel");
    ScfStatus hst;
    DF_CUDA(cudaMemcpyAsync(&hst, W.st, sizeof(hst), cudaMemcpyDeviceToHost, s));
    DF_CUDA(cudaStreamSynchronize(s));
    use_dm0 = std::isfinite(hst.trDS) && fabs(hst.trDS - mol->nelec) / mol->nelec < 0.05 && hst.idem < 0.5;
    res->guess = use_dm0 ? 1 : 2;
  }
  if (use_dm0) {
    DF_CUDA(cudaMemcpyAsync(W.D, dm0, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
  } else {
    DF_TRY(diagonalize_fock(W.h, nao, nmo, nocc, W, s));
  }
  // ---- iterations ----------------------------------------------------------------------
  std::vector<int> hvalid(space, 0), horder(space, 0);
  std::vector<long> age(space, 0);
  int nvalid = 0;
  long tick = 0;
  DF_CUDA(cudaMemsetAsync(W.valid, 0, sizeof(int) * space, s));
  int prec = o->precision;
  bool switched = (prec == DF_FP64);
  int fp64_done = 0;
  double e_old = 0.0;
  bool have_old = false;
  bool first_dm0 = use_dm0;
  ScfStatus hst{};
  int it = 0;
  for (it = 1; it <= o->max_cycle; ++it) {
    // ---- J, K -------------------------------------------------------------------------
    if (first_dm0) {
      // K for a general density from its eigen-decomposition (dm0/2 = C+ C+^T - C- C-^T)
      DF_TRY(run_jk(W.B, nao, naux, prec, W.D, nullptr, 0, W.J, nullptr, W.jk, s));
      DF_CUDA(cudaMemcpyAsync(W.T1, W.D, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
      DF_TRY(eig_sync(W.T1, nao, W.eps, W.ZT, W, s));
      std::vector<double> wv(nao);
      DF_CUDA(cudaMemcpyAsync(wv.data(), W.eps, sizeof(double) * nao, cudaMemcpyDeviceToHost, s));
      DF_CUDA(cudaStreamSynchronize(s));
      double wmax = 0.0;
      for (double x : wv) wmax = fmax(wmax, fabs(x));
      DF_CUDA(cudaMemsetAsync(W.K, 0, sizeof(double) * nn, s));
      for (int sign = 1; sign >= -1; sign -= 2) {
        std::vector<int> ids;
        for (int k = 0; k < nao; ++k)
          if (sign * wv[k] > 1e-12 * wmax) ids.push_back(k);
        for (size_t c0 = 0; c0 < ids.size(); c0 += nocc) {
          int cnt = (int)std::min((size_t)nocc, ids.size() - c0);
          DF_CUDA(cudaMemcpyAsync(W.idx, ids.data() + c0, sizeof(int) * cnt, cudaMemcpyHostToDevice, s));
          split_density_kernel<<<blocks_for((long)nao * cnt), 256, 0, s>>>(W.ZT, W.eps, nao, W.idx, cnt, W.Cchunk);
          DF_LAUNCHED("split_density_kernel");
          DF_TRY(run_jk(W.B, nao, naux, prec, nullptr, W.Cchunk, cnt, nullptr, W.T2, W.jk, s));
          axpy_kernel<<<blocks_for(nn), 256, 0, s>>>(W.K, W.T2, nn, (double)sign);
          DF_LAUNCHED("axpy_kernel");
          DF_CUDA(cudaStreamSynchronize(s));  // host vector ids is reused
        }
      }
      first_dm0 = false;
    } else {
      DF_TRY(run_jk(W.B, nao, naux, prec, W.D, W.Cocc, nocc, W.J, W.K, W.jk, s));
    }
    // ---- Fock, energy, DIIS error -------------------------------------------------------
    fock_energy_kernel<<<1, 1024, 0, s>>>(W.h, W.J, W.K, W.D, nn, W.enuc, W.F, W.st);
    DF_LAUNCHED("fock_energy_kernel");
    DF_TRY(dgemm(false, false, nao, nao, nao, 1.0, W.F, nao, 0, W.D, nao, 0, 0.0, W.T1, nao, 0, 1, s, 0, 0));
    DF_TRY(dgemm(false, false, nao, nao, nao, 1.0, W.T1, nao, 0, W.S, nao, 0, 0.0, W.T2, nao, 0, 1, s, 0, 0));
    antisym_kernel<<<blocks_for(nn), 256, 0, s>>>(W.T2, nao, W.T1);
    DF_LAUNCHED("antisym_kernel");
    DF_TRY(dgemm(false, false, nao, nmo, nao, 1.0, W.T1, nao, 0, W.X, nmo, 0, 0.0, W.T2, nmo, 0, 1, s, 0, 0));
    // slot for the new vector: a free one, else the oldest
    int slot = -1;
    for (int k = 0; k < space; ++k)
      if (!hvalid[k]) { slot = k; break; }
    if (slot < 0) {
      slot = 0;
      for (int k = 1; k < space; ++k)
        if (age[k] < age[slot]) slot = k;
    }
    double* Eslot = W.Ehist + (size_t)slot * nn;
    DF_TRY(dgemm(true, false, nmo, nmo, nao, 1.0, W.X, nmo, 0, W.T2, nmo, 0, 0.0, Eslot, nmo, 0, 1, s, 0, 0));
    absmax_kernel<<<1, 1024, 0, s>>>(Eslot, (long)nmo * nmo, &W.st->emax);
    DF_LAUNCHED("absmax_kernel");
    DF_CUDA(cudaMemcpyAsync(&hst, W.st, sizeof(hst), cudaMemcpyDeviceToHost, s));
    DF_CUDA(cudaStreamSynchronize(s));
    res->iterations = it;
    if (prec == DF_FP64) res->fp64_iterations++;
    DF_REQUIRE(!hst.nonfinite && std::isfinite(hst.emax), DF_ERR_NUMERIC, "scf_run: non-finite Fock matrix at iteration %d", it);
    double de = have_old ? fabs(hst.energy - e_old) : INFINITY;
    res->energy = hst.energy;
    res->last_de = de;
    res->last_err = hst.emax;
    if (o->verbose)
      printf("scf iter %3d  %s  E = %.12f  dE = %.3e  max|e| = %.3e\n", it, prec == DF_FP64 ? "fp64 " : "mixed", hst.energy,
             de, hst.emax);
    if (prec == DF_FP64 && switched && fp64_done + 1 >= o->n_fp64_final && have_old && de < o->conv_tol &&
        hst.emax < o->conv_err) {
      res->converged = 1;
      break;
    }
    if (prec == DF_FP64) fp64_done++;
    // ---- DIIS ---------------------------------------------------------------------------
    DF_CUDA(cudaMemcpyAsync(W.Fhist + (size_t)slot * nn, W.F, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
    if (!hvalid[slot]) nvalid++;
    hvalid[slot] = 1;
    age[slot] = ++tick;
    if (nvalid > space) nvalid = space;
    // keep at most diis_space vectors: drop the oldest beyond that
    while (nvalid > o->diis_space) {
      int old = -1;
      for (int k = 0; k < space; ++k)
        if (hvalid[k] && (old < 0 || age[k] < age[old])) old = k;
      hvalid[old] = 0;
      nvalid--;
    }
    DF_CUDA(cudaMemcpyAsync(W.valid, hvalid.data(), sizeof(int) * space, cudaMemcpyHostToDevice, s));
    // Gram row of the new vector (E stored with leading dimension nmo, nmo*nmo entries)
    diis_gram_kernel<<<space, 256, 0, s>>>(W.Ehist, nn, (long)nmo * nmo, space, slot, W.valid, W.G);
    DF_LAUNCHED("diis_gram_kernel");
    const double* Fuse = W.F;
    if (nvalid >= 2) {
      int m = 0;
      for (int k = 0; k < space; ++k)
        if (hvalid[k]) horder[m++] = k;
      DF_CUDA(cudaMemcpyAsync(W.order, horder.data(), sizeof(int) * m, cudaMemcpyHostToDevice, s));
      diis_solve_kernel<<<1, 32, 0, s>>>(W.G, space, W.order, m, slot, W.coef, W.st);
      DF_LAUNCHED("diis_solve_kernel");
      diis_combine_kernel<<<blocks_for(nn), 256, 0, s>>>(W.Fhist, nn, space, W.coef, W.valid, W.Fbar);
      DF_LAUNCHED("diis_combine_kernel");
      Fuse = W.Fbar;
    }
    DF_TRY(diagonalize_fock(Fuse, nao, nmo, nocc, W, s));
    if (nvalid >= 2) {
      int sing = 0;
      DF_CUDA(cudaMemcpyAsync(&sing, &W.st->singular, sizeof(int), cudaMemcpyDeviceToHost, s));
      DF_CUDA(cudaStreamSynchronize(s));
      if (sing) {  // restart the history from the newest vector
        for (int k = 0; k < space; ++k) hvalid[k] = (k == slot);
        nvalid = 1;
      }
    }
    // ---- mixed -> FP64 switch --------------------------------------------------------------
    if (!switched && have_old && (de < o->switch_tol || hst.emax < o->switch_err)) {
      switched = true;
      prec = DF_FP64;
      for (int k = 0; k < space; ++k) hvalid[k] = 0;
      nvalid = 0;
    }
    e_old = hst.energy;
    have_old = true;
  }
  // orbital energies of the last diagonalisation
  std::vector<double> he(nmo);
  DF_CUDA(cudaMemcpyAsync(he.data(), W.eps, sizeof(double) * nmo, cudaMemcpyDeviceToHost, s));
  DF_CUDA(cudaStreamSynchronize(s));
  res->homo = nocc > 0 ? he[nocc - 1] : 0.0;
  res->lumo = nocc < nmo ? he[nocc] : 0.0;
  if (D_out) DF_CUDA(cudaMemcpyAsync(D_out, W.D, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
  if (C_out) DF_CUDA(cudaMemcpyAsync(C_out, W.Cocc, sizeof(double) * nao * nocc, cudaMemcpyDeviceToDevice, s));
  if (mo_energy) DF_CUDA(cudaMemcpyAsync(mo_energy, W.eps, sizeof(double) * std::min(nmo, nocc + 1), cudaMemcpyDeviceToDevice, s));
  DF_CUDA(cudaStreamSynchronize(s));
  if (!res->converged) {
    set_error("scf_run: not converged after %d iterations (dE %.3e, max|e| %.3e)", res->iterations, res->last_de,
              res->last_err);
    return DF_ERR_NOCONV;
  }
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
  o->switch_tol = 1e-7;
  o->switch_err = 1e-4;
  o->verbose = 0;
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
  DF_REQUIRE(mol && res, DF_ERR_ARG, "scf_run: null molecule or result");
  scf_opts o;
  if (opt) o = *opt; else scf_default_opts(&o);
  DF_REQUIRE(mol->nao > 0 && mol->naux > 0 && mol->natm > 0 && mol->nelec > 0 && mol->nelec % 2 == 0, DF_ERR_ARG,
             "scf_run: bad molecule sizes (nao %d naux %d natm %d nelec %d)", mol->nao, mol->naux, mol->natm, mol->nelec);
  DF_REQUIRE(mol->xyz && mol->charges && mol->ao_xyz && mol->ao_exp && mol->aux_xyz && mol->aux_exp, DF_ERR_ARG,
             "scf_run: null molecule array");
  DF_REQUIRE(o.precision == DF_FP64 || o.precision == DF_MIXED, DF_ERR_ARG, "scf_run: bad precision");
  DF_REQUIRE(o.diis_space >= 1 && o.diis_space <= 16, DF_ERR_ARG, "scf_run: diis_space must be in [1, 16]");
  DF_REQUIRE(o.max_cycle >= 1 && o.n_fp64_final >= 1, DF_ERR_ARG, "scf_run: bad iteration limits");
  DF_REQUIRE(mol->naux <= 65535, DF_ERR_ARG, "scf_run: naux > 65535");
  int nocc = mol->nelec / 2;
  DF_REQUIRE(nocc <= mol->nao, DF_ERR_ARG, "scf_run: more occupied orbitals than basis functions");
  size_t need = scf_work_bytes(mol->nao, mol->naux, nocc, o.precision);
  DF_REQUIRE(work && work_bytes >= need, DF_ERR_NOMEM, "scf_run: workspace of %zu bytes < %zu", work_bytes, need);
  Arena a(work, work_bytes);
  ScfWork w;
  scf_layout(mol->nao, mol->naux, nocc, o.precision, &a, nullptr, &w);
  DF_REQUIRE(!a.overflow, DF_ERR_NOMEM, "scf_run: workspace overflow");
  return scf_driver(mol, &o, dm0, D_out, C_out, mo_energy, res, w, s);
}
