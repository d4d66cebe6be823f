/*
 * dfscf.h - C ABI of the GB300 (sm_103a) density-fitted Hartree-Fock library.
 *
 * Method: density fitting of the four-centre Coulomb integrals as stated in
 * arXiv 2506.06661, Section "Density fitting":
 *     (mn|kl) ~ sum_P T_{P,mn} T_{P,kl},   M_PQ = (chi_P|chi_Q) = L L^T,
 *     T_{P,mn} = sum_Q (L^-1)_{PQ} (chi_Q|mn)                 (this library calls T "B"),
 * used to build the Coulomb matrix J = sum_P B_P (B_P . D) and the exchange matrix
 * K = sum_P (B_P C)(B_P C)^T inside a restricted Hartree-Fock SCF loop with DIIS.
 * The get_jk call shape (J and K for a given density) follows the paper's description
 * of get_jk in PySCF and GPU4PySCF (Sections "PySCF" and "GPU4PySCF").
 *
 * Basis: s-type primitives phi_a(r) = N_a exp(-a |r - A|^2), N_a = (2a/pi)^(3/4), for
 * both the orbital and the auxiliary set.  Orbital pairs are packed m >= n with
 * index mn = m(m+1)/2 + n; npair = nao(nao+1)/2.
 *
 * Conventions for every call:
 *   - all matrices are row-major; all array arguments are DEVICE pointers unless the
 *     parameter is documented as host memory;
 *   - the caller owns every buffer.  Calls that need scratch take (work, work_bytes);
 *     the matching *_work_bytes() query gives the size.  The library never allocates
 *     device memory;
 *   - every call is asynchronous on stream `s` unless documented otherwise; results are
 *     valid once the stream has synchronised;
 *   - every call returns DF_OK or one of the error codes below and, on error, records a
 *     thread-local message readable with df_last_error().  Argument errors are detected
 *     on the host before anything is launched.
 *   - there is no CPU fallback: a missing or failing GPU yields DF_ERR_CUDA.
 */
#ifndef DFSCF_H
#define DFSCF_H

#include <stddef.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------- */
#define DF_OK 0
#define DF_ERR_ARG 1         /* null pointer, bad size, workspace too small, ...        */
#define DF_ERR_CUDA 2        /* a CUDA runtime call or kernel launch failed             */
#define DF_ERR_NOT_SPD 3     /* Cholesky pivot <= tol * max diagonal                    */
#define DF_ERR_NOCONV 4      /* SCF did not converge within max_cycle                   */
#define DF_ERR_TIMEOUT 5     /* a bounded device-side wait gave up                      */
#define DF_ERR_NOMEM 6       /* the caller's buffer is smaller than the query says      */
#define DF_ERR_NUMERIC 7     /* NaN/Inf detected in an SCF quantity                     */

/* ---- precision modes -------------------------------------------------------------- */
#define DF_FP64 0            /* every contraction in FP64                               */
#define DF_MIXED 1           /* K contractions as split-BF16 GEMMs on tcgen05 tensor
                                cores.  Every operand row (of B_P, of C^T, of X) is held
                                as NP BF16 planes, NP = the knob "mixed_planes" (3, 4 or
                                5; default 5).  With sigma the power of two just above
                                the row's max |x|: p0 = x rounded to the grid
                                sigma 2^-7 and p1 = (x - p0) rounded to sigma 2^-15 are
                                fixed-point planes (integers in [-128, 128] on grids
                                fixed along the contraction); p2.. p(NP-1) are the BF16
                                roundings of what is left.  Plane products pa*qb with
                                a + b < NP (6, 10 or 15 of them) accumulate in FP32
                                tensor memory.  In the exchange SYRK the products of
                                the two fixed-point planes, (0,0), (0,1)+(1,0) and
                                (1,1), each sum integers on one grid in an accumulator
                                of their own and are exact; every product with a
                                floating plane goes to a fourth.  J is the FP64
                                streaming pass in both modes.  An FP32 J, or products
                                summed in a single FP32 accumulator, leaves an error in
                                F that the orthogonal-basis DIIS commutator amplifies to
                                ~1e-3 on ill-conditioned bases, where the mixed SCF
                                then stalls. */

/* Message describing the last error on the calling thread ("" if none). */
const char* df_last_error(void);

/* Library version, major*10000 + minor*100 + patch. */
int df_version(void);

/* ---- a1: Boys function -------------------------------------------------------------
 * out[i] = F0(t[i]) = int_0^1 exp(-t u^2) du for n values (t >= 0).  The order-zero
 * Boys function is the radial factor of every s-type Coulomb integral implied by the
 * paper's DF integrals (chi_P|chi_Q) and (chi_Q|mn).  One GPU lane per value.        */
int df_boys_f0(const double* t, long n, double* out, cudaStream_t s);

/* ---- one-electron integrals ---------------------------------------------------------
 * S, T, V (each [nao][nao]; any may be NULL) for s primitives at ao_xyz [nao][3] with
 * exponents ao_exp [nao]; V sums the attraction of natm point nuclei nuc_xyz [natm][3]
 * with charges nuc_z [natm].  Products of primitives use the Gaussian product theorem
 * of the paper's overlap example (Section "Numba JIT compilation").                  */
int df_int1e(const double* ao_xyz, const double* ao_exp, int nao, const double* nuc_xyz,
             const double* nuc_z, int natm, double* S, double* T, double* V, cudaStream_t s);

/* Nuclear repulsion sum_{A<B} Z_A Z_B / R_AB of natm nuclei, written to the device
 * double *e_nuc.                                                                      */
int df_nuclear_repulsion(const double* nuc_xyz, const double* nuc_z, int natm, double* e_nuc,
                         cudaStream_t s);

/* ---- a2: Coulomb metric and its Cholesky factor ------------------------------------
 * M_PQ = (chi_P|chi_Q) for naux auxiliary s primitives, then M = L L^T
 * (Section "Density fitting", metric equation).  L is [naux][naux], lower triangle
 * filled, strict upper triangle set to zero.  Optionally M is also written to M_out
 * ([naux][naux], may be NULL).
 * Synchronises the stream once to read the pivot status.  If a pivot is <= 1e-14 times
 * the largest diagonal element of M, returns DF_ERR_NOT_SPD and stores the 0-based
 * pivot index in the HOST int *bad_pivot (otherwise *bad_pivot = -1).
 * work: df_metric_chol_work_bytes(naux) bytes.                                         */
size_t df_metric_chol_work_bytes(int naux);
int df_metric_chol(const double* aux_xyz, const double* aux_exp, int naux, double* L, double* M_out,
                   int* bad_pivot, void* work, size_t work_bytes, cudaStream_t s);

/* ---- a3 + a4: three-centre integrals and whitening ---------------------------------
 * B_{P,mn} = sum_Q (L^-1)_{PQ} (chi_Q|mn) for all packed pairs (Section "Density
 * fitting", whitened three-index tensor), computed in FP64 by blocked forward
 * substitution.  B is one caller-owned buffer of df_B_bytes(nao, naux, precision) bytes
 * holding, in this order:
 *   [0]  FP64 packed rows: naux rows of df_B_ld(nao) doubles, entry mn at m(m+1)/2+n,
 *        padding zero;
 *   [1]  (DF_MIXED only) NP BF16 planes p0 .. p(NP-1) of the full symmetric B_P (the
 *        row-scaled planes described at DF_MIXED), each naux x npad x npad with
 *        npad = df_nao_pad(nao), padding zero; NP is the knob "mixed_planes" when
 *        df_B_bytes is called, and df_build_B must see the same value.  A later mixed
 *        df_jk needs NP at least its own "mixed_planes" (checked: DF_ERR_ARG otherwise).
 * L is the factor from df_metric_chol.  work: df_build_B_work_bytes(...) bytes.         */
long df_B_ld(int nao);
int df_nao_pad(int nao);
size_t df_B_bytes(int nao, int naux, int precision);
size_t df_build_B_work_bytes(int nao, int naux);
int df_build_B(const double* ao_xyz, const double* ao_exp, int nao, const double* aux_xyz,
               const double* aux_exp, int naux, const double* L, int precision, void* B,
               size_t B_bytes, void* work, size_t work_bytes, cudaStream_t s);

/* Copy the FP64 packed row P of B (npair doubles) to `row` (device).  For tests.      */
int df_B_get_packed(const void* B, int nao, int naux, int P, double* row, cudaStream_t s);

/* ---- a5..a8: Coulomb and exchange matrices ------------------------------------------
 * J[D]_mn = sum_P d_P B_{P,mn}, d_P = sum_{kl} B_{P,kl} D_kl   (J = sum_P B_P (B_P . D))
 * K_mn    = sum_P sum_i (B_P C)_{mi} (B_P C)_{ni}               (K = K[C C^T])
 * D: [nao][nao] symmetric density; C: [nao][nocc] occupied coefficients.  For an RHF
 * density D = 2 C C^T the Fock matrix is F = h + J - K.  J or K may be NULL to skip it
 * (then D or C may be NULL too).  precision DF_MIXED requires B built with DF_MIXED.
 * The tensor-core kernels of the mixed exchange bound every wait; if one gives up, K is
 * filled with NaN and, unless the stream is being captured into a graph, df_jk (which then
 * synchronises the stream once to read the flag) returns DF_ERR_TIMEOUT.  A mixed df_jk
 * outside a capture therefore returns with the stream drained.
 * work: df_jk_work_bytes(nao, naux, nocc, precision) bytes.                           */
size_t df_jk_work_bytes(int nao, int naux, int nocc, int precision);
int df_jk(const void* B, int nao, int naux, int precision, const double* D, const double* C,
          int nocc, double* J, double* K, void* work, size_t work_bytes, cudaStream_t s);

/* ---- a11: symmetric eigensolver ----------------------------------------------------
 * Eigenvalues w[0..n) ascending and eigenvectors (columns of Z, [n][n]) of the
 * symmetric matrix A [n][n] (A is overwritten).  Householder tridiagonalisation, then
 * implicit QL on one thread block (n < 160), or for larger n the multi-SM path of
 * df_eigh_lowest with k = n (Sturm multisection, inverse iteration, back-transformation,
 * two Gram-Schmidt passes).  Synchronises the stream; DF_ERR_NOCONV if the solver breaks
 * down, DF_ERR_TIMEOUT if a grid barrier of the multi-SM path gave up waiting (every CTA
 * then returns; the context stays usable).  work: df_eigh_work_bytes(n).                 */
size_t df_eigh_work_bytes(int n);
int df_eigh(double* A, int n, double* w, double* Z, void* work, size_t work_bytes, cudaStream_t s);

/* The k lowest eigenpairs only (w [k] ascending, Z [n][k] columns), as the SCF needs for
 * the occupied orbitals and the LUMO: Householder reduction, Sturm bisection, inverse
 * iteration on the tridiagonal matrix, back-transformation of the k vectors and
 * re-orthonormalisation.  A is overwritten.  work: df_eigh_lowest_work_bytes(n, k).
 * Returns DF_ERR_NOCONV if inverse iteration or re-orthonormalisation breaks down and
 * DF_ERR_TIMEOUT if a grid barrier of the multi-SM path gave up waiting.                  */
size_t df_eigh_lowest_work_bytes(int n, int k);
int df_eigh_lowest(double* A, int n, int k, double* w, double* Z, void* work, size_t work_bytes, cudaStream_t s);

/* ---- a9..a12: restricted Hartree-Fock SCF --------------------------------------------
 * Mean-field DF-RHF ("density_fit()" mean-field in the paper's DF section) with Pulay
 * DIIS (named as PySCF's default accelerator in the paper's SOSCF section):
 *   F = h + J[D] - 1/2 K[D],  E = 1/2 tr(D (h + F)) + E_nuc,
 *   e = X^T (F D S - S D F) X with canonical orthogonalisation X = U s^-1/2 (s > lindep),
 *   extrapolation over <= diis_space vectors, aufbau occupation of nocc = nelec/2.
 * Converged when |dE| < conv_tol and max|e| < conv_err.  In DF_MIXED mode the loop runs
 * with mixed-precision K until max|e| < 1e-3, |dE| < switch_tol or max|e| < switch_err, or
 * until max|e|, once below 1e-3, has not improved by 10% for 10 iterations (the
 * mixed-precision floor), or for three quarters of max_cycle.  With the knob
 * "mixed_incremental" (default 1) one FP64 Fock build then becomes the base of K, and later
 * iterations update K += K[U+] - K[U-] in mixed precision, U+ U+^T - U- U-^T being the change
 * of the occupied projector (factorised over the principal angles between the two occupied
 * spaces, so the mixed error shrinks with the change); a new base is built when the occupied
 * space turns by more than 60 degrees in one step or the updates stall.  With the knob at 0
 * the iterations switch to FP64 instead.  Either way at least n_fp64_final FP64 iterations
 * end the run and the reported energy is the FP64 one.
 * Newton steps (knob "soscf", default 1; the paper's Section "Second-Order Self-Consistent
 * Field"): once max|e| has not improved by 10% for 12 iterations with an accurate Fock
 * matrix, each later iteration replaces the DIIS extrapolation and diagonalisation by a
 * Newton step on the orbital rotation, solved by "soscf_cg" preconditioned conjugate-
 * gradient iterations whose Hessian products use the exchange of the SCF's precision (mixed
 * in DF_MIXED mode: an approximate Hessian with the exact gradient, so the converged result
 * is unchanged).
 * dm0 (device [nao][nao], may be NULL): initial density; it need not be idempotent nor
 * have the right electron count (paper, Section "Initial Guess for Mean-field Methods").
 * If dm0 fails the checks |tr(dm0 S) - nelec| / nelec < 0.05 and
 * ||Dx Dx - 2 Dx||_F / ||Dx||_F < g with Dx = X^T S dm0 S X (dm0 in the orthonormal basis
 * of X; g = knob "guess_idem_max" / 100, default 2) the core-Hamiltonian guess is used
 * instead.  An accepted dm0 with
 * ||Dx Dx - 2 Dx||_F / ||Dx||_F < 1e-6 (a determinant) starts from its occupied orbitals,
 * which span the nocc leading eigenvectors of Dx; any other accepted dm0 runs a first
 * iteration whose exchange uses the eigen-decomposition of dm0 (scf_run_batch advances the
 * other molecules while that decomposition runs).  With dm0 NULL and opt->guess_params set
 * (the learned guess's parameters, guess_mlp_create layout) the SCF predicts dm0 itself during
 * set-up (guess_density with S^-1/2 from the overlap eigen-decomposition it computes for X;
 * molecules whose nao is not 5 natm use the core guess), then applies the same checks;
 * res.guess reports 1 (used) or 2 (rejected).
 * Outputs (device, may be NULL): D_out [nao][nao], C_out [nao][nocc], mo_energy [nocc+1].
 * res is HOST memory.  The host loop reads one small status block per iteration.       */
typedef struct {
  int natm;
  const double* xyz;      /* [natm][3] */
  const double* charges;  /* [natm]    */
  int nao;
  const double* ao_xyz;   /* [nao][3]  */
  const double* ao_exp;   /* [nao]     */
  int naux;
  const double* aux_xyz;  /* [naux][3] */
  const double* aux_exp;  /* [naux]    */
  int nelec;              /* even */
} df_molecule;

typedef struct {
  int precision;      /* DF_FP64 or DF_MIXED                  (default DF_FP64) */
  int diis_space;     /* DIIS history length                   (8)              */
  int max_cycle;      /* Fock builds before DF_ERR_NOCONV      (100)            */
  int n_fp64_final;   /* FP64 iterations after the mixed phase (2)              */
  double conv_tol;    /* |dE| threshold                         (1e-8)          */
  double conv_err;    /* max|e| threshold                       (1e-5)          */
  double lindep;      /* canonical orthogonalisation cut        (1e-8)          */
  double switch_tol;  /* mixed -> FP64 switch on |dE|           (3e-8)          */
  double switch_err;  /* mixed -> FP64 switch on max|e|         (3e-5)          */
  int verbose;        /* print one line per iteration to stdout (0)             */
  const float* guess_params; /* device parameters of the learned-guess network
                                (guess_mlp_create); with dm0 NULL the starting density
                                is predicted from the geometry (NULL: core guess)   */
} scf_opts;

typedef struct {
  double energy;        /* total energy (Hartree)                                 */
  double e_nuc;         /* nuclear repulsion                                      */
  double homo, lumo;    /* orbital energies of the last diagonalisation           */
  double last_de;       /* |dE| of the final iteration                            */
  double last_err;      /* max|e| of the final iteration                          */
  int iterations;       /* Fock builds in total                                   */
  int fp64_iterations;  /* Fock builds done in FP64                               */
  int converged;        /* 1 if both thresholds were met                          */
  int guess;            /* 0 core guess, 1 dm0 used, 2 dm0 rejected -> core guess */
  int nmo;              /* orbitals kept by canonical orthogonalisation           */
  double hess_min;      /* lowest orbital-Hessian eigenvalue at the solution (knob
                           "stability" >= 1; NaN otherwise): > 0 a local minimum over
                           closed-shell determinants, < 0 a saddle point          */
  int stability_restarts; /* saddle points left along their negative mode (knob
                           "stability" = 2)                                       */
} scf_result;

void scf_default_opts(scf_opts* opt);
size_t scf_work_bytes(int nao, int naux, int nocc, int precision);
int scf_run(const df_molecule* mol, const scf_opts* opt, const double* dm0, double* D_out,
            double* C_out, double* mo_energy, scf_result* res, void* work, size_t work_bytes,
            cudaStream_t s);

/* ---- a13: batched SCF -------------------------------------------------------------------
 * Runs scf_run's algorithm for nmol molecules of uneven size.  At most `slots` molecules
 * are in flight at once, each with its own stream (created by the library, ordered after
 * `s`) and a region of the workspace of its own size (scf_work_bytes of that molecule),
 * handed out first-fit: many small molecules run beside a few large ones.  Molecules start
 * largest first; a molecule that finishes returns its region and stream to the next one.
 * The workspace may have any size that holds the largest molecule; more bytes allow more
 * molecules in flight.  scf_batch_work_bytes(mols, nmol, precision, slots) is the size that
 * holds `slots` copies of the largest molecule (always enough for `slots` in flight).
 * Each molecule's iteration is captured once per precision into a CUDA graph and replayed
 * (Newton iterations run eagerly).  dm0s (may be NULL; entries may be NULL): device starting
 * densities; D_outs (may be NULL; entries may be NULL): device [nao][nao] outputs; results:
 * HOST array of nmol.  Returns DF_ERR_NOCONV if any molecule did not converge (all results
 * are still filled), DF_ERR_NOMEM if the workspace cannot hold the largest molecule.
 * Blocks until done.                                                                     */
size_t scf_batch_work_bytes(const df_molecule* mols, int nmol, int precision, int slots);
int scf_run_batch(const df_molecule* mols, int nmol, const scf_opts* opt, const double* const* dm0s,
                  double* const* D_outs, scf_result* results, int slots, void* work, size_t work_bytes,
                  cudaStream_t s);

/* ---- a14: learned initial guess --------------------------------------------------------
 * A starting density for scf_run / scf_run_batch (dm0), predicted from geometry.  The
 * paper lets dm0 be any density, idempotent or not (Section "Initial Guess for Mean-field
 * Methods"); scf_run falls back to the core guess when the trace or idempotency check
 * fails.  Centres carry 5 orbital functions each (the workload's basis).
 *   features: for every centre pair p = A(A+1)/2 + B (A >= B), 65 inputs: 32 Gaussian
 *     radial-basis values exp(-gamma (R - r_k)^2), r_k = 12k/31, gamma = (31/12)^2, and the
 *     environment env_A = 1/8 sum_{C != A, R_AC <= 12} rbf(R_AC): off-diagonal pairs
 *     [rbf(R_AB), env_A + env_B, 0], diagonal pairs [0, 2 env_A, 1]; mask[p] = 0 for pairs
 *     more than 12 bohr apart (their block stays zero).
 *   network: 65 -> 256 -> 256 -> 256 -> 15, SiLU hidden activations; params is one float
 *     array of guess_mlp_param_count() values, per layer W [out][in] then b [out].
 *   outputs: the 15 upper-triangle entries (a <= b, row-major) of a symmetric 5x5 block.
 * All pointers are device memory; n is the number of pair samples.                        */
size_t guess_mlp_param_count(void);
size_t guess_mlp_work_bytes(int n);
/* Model lifecycle.  guess_mlp_create initialises params [param_count] (device) with
 * Uniform(-sqrt(3/fan_in), +sqrt(3/fan_in)) weights drawn from a counter-based generator
 * (SplitMix64 of seed and parameter index) and zero biases, and zeroes the Adam moments
 * adam_m, adam_v (each may be NULL).
 * guess_mlp_save writes the model to the HOST buffer blob of guess_mlp_blob_bytes(m) bytes,
 * m = 1 when adam_m and adam_v are given (both or neither): a header (magic "DFSCFMLP",
 * format version, the layer shapes, the Adam step, the parameter count and an FNV-1a 64
 * checksum of the payload) followed by params, then adam_m and adam_v, as FP32.
 * guess_mlp_load checks magic, version, layer shapes, size and checksum (DF_ERR_ARG on any
 * mismatch, nothing copied) and fills params (and adam_m, adam_v, zeroed when the blob holds
 * no moments) and the HOST int *step (may be NULL; 0 without moments).  Both synchronise s. */
int guess_mlp_create(unsigned long long seed, float* params, float* adam_m, float* adam_v, cudaStream_t s);
size_t guess_mlp_blob_bytes(int with_moments);
int guess_mlp_save(const float* params, const float* adam_m, const float* adam_v, int step, void* blob,
                   size_t blob_bytes, cudaStream_t s);
int guess_mlp_load(const void* blob, size_t blob_bytes, float* params, float* adam_m, float* adam_v, int* step,
                   cudaStream_t s);
/* feat [natm(natm+1)/2][65], mask [natm(natm+1)/2]; work >= 128*natm bytes.               */
int guess_features(const double* xyz, int natm, float* feat, float* mask, void* work, size_t work_bytes,
                   cudaStream_t s);
/* Y [npairs][15]: symmetrised 5x5 blocks 1/2 (D_AB + D_AB^T) of a converged D [nao][nao]. */
int guess_targets(const double* D, int natm, float* Y, cudaStream_t s);
/* out [n][15]; bf16 != 0 runs the BF16 inference path (BF16 weights and activations, FP32
 * accumulation), else FP32.                                                               */
int guess_mlp_forward(const float* params, const float* X, int n, float* out, int bf16, void* work,
                      size_t work_bytes, cudaStream_t s);
/* loss = sum_p mask_p |out_p - Y_p|^2 / (nvalid * 15) (device float) and its gradient
 * grad [param_count] in FP32.                                                              */
int guess_mlp_loss_grad(const float* params, const float* X, const float* Y, const float* mask, int n,
                        float nvalid, float* loss, float* grad, void* work, size_t work_bytes, cudaStream_t s);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected with step >= 1) on the
 * mini-batch's loss; adam_m / adam_v [param_count] are the moment buffers; loss may be NULL. */
int guess_mlp_train_step(float* params, float* adam_m, float* adam_v, int step, float lr, const float* X,
                         const float* Y, const float* mask, int n, float nvalid, float* loss, void* work,
                         size_t work_bytes, cudaStream_t s);
/* The network's targets are the blocks of the Loewdin-orthogonalised density
 * Dt = S^1/2 D S^1/2 (its blocks are well conditioned; those of D are not in a strongly
 * non-orthogonal basis).  guess_density assembles Dt from the predicted blocks (BF16
 * inference), scales it to tr(Dt) = nelec when nelec > 0 (nelec = 0 keeps the raw
 * assembly; a non-positive trace is left unscaled), and returns
 * dm0 = S^-1/2 Dt S^-1/2 [5 natm][5 natm].  Since tr(dm0 S) = tr(Dt) for a full-rank S,
 * the scaled guess carries the right electron count (the paper's Section "Initial Guess
 * for Mean-field Methods" allows dm0 with any count; the scaling only removes the
 * network's systematic overshoot, which the electron-count check would otherwise reject). */
size_t guess_density_work_bytes(int natm);
int guess_density(const float* params, const double* xyz, int natm, int nelec, const double* Sinvhalf,
                  double* D0, void* work, size_t work_bytes, cudaStream_t s);
/* S^1/2 and S^-1/2 (either may be NULL) of the orbital overlap, over eigenvalues above
 * lindep (pseudo-inverse below).  Synchronises the stream to check the eigensolver.      */
size_t df_lowdin_work_bytes(int nao);
int df_lowdin_factors(const double* ao_xyz, const double* ao_exp, int nao, double lindep, double* Shalf,
                      double* Sinvhalf, void* work, size_t work_bytes, cudaStream_t s);
/* out = M A M for n x n matrices (M symmetric), e.g. Dt = S^1/2 D S^1/2.                  */
size_t df_congruence_work_bytes(int n);
int df_congruence(const double* M, const double* A, int n, double* out, void* work, size_t work_bytes,
                  cudaStream_t s);

/* ---- density-fitting error diagnostics (NEXT-3) ------------------------------------------
 * Lehtola's diagonal error of the paper's Section "Density fitting",
 *     Delta = sum_mn [(mn|mn) - sum_P T_{P,mn}^2]   (ordered pairs: packed pairs off the
 *                                                    diagonal count twice),
 * and the residual of the auxiliary-basis fit of Section "Automatic Differentiation",
 *     sigma_mn = (mn|mn) - sum_PQ (P|mn) (M^-1)_PQ (Q|mn)   (>= 0 for the Coulomb metric),
 * for every packed pair mn (sigma [npair], device).  With jac (device [npair][ntheta], may be
 * NULL) the Jacobian is also formed, contracted with dalpha (device [naux][ntheta],
 * d alpha_P / d theta_t, 1 <= ntheta <= 8): jac[mn][t] = sum_P (d sigma_mn / d alpha_P)
 * dalpha[P][t], from the closed-form exponent derivatives of the s-type integrals (the paper
 * differentiates automatically).  For an even-tempered set alpha_P = a beta^k_P on every
 * centre, theta = (ln a, ln beta) gives dalpha[P] = (alpha_P, k_P alpha_P).  *delta (HOST,
 * may be NULL) receives Delta.  Synchronises the stream (pivot check of the metric's
 * Cholesky factor: DF_ERR_NOT_SPD).  The Jacobian needs O(naux^2 npair) work and
 * 4 naux npair doubles of workspace: meant for small molecules or single atoms, as in the
 * paper's basis optimisation.  work: df_fit_residual_work_bytes(nao, naux, jac != NULL).   */
size_t df_fit_residual_work_bytes(int nao, int naux, int with_jacobian);
int df_fit_residual(const double* ao_xyz, const double* ao_exp, int nao, const double* aux_xyz,
                    const double* aux_exp, int naux, const double* dalpha, int ntheta, double* sigma, double* jac,
                    double* delta, void* work, size_t work_bytes, cudaStream_t s);

/* ---- long-range density fitting (NEXT-1) -----------------------------------------------
 * The LRDF scheme of the paper's Section "Density fitting": 1/r = erf(w r)/r + erfc(w r)/r,
 * the long-range part density fitted with the long-range metric M^LR = L L^T and
 * T = L^-1 (Q|mn)^LR, the short-range part computed exactly:
 *     (mn|kl) ~ (mn|kl)^SR + sum_P T_{P,mn} T_{P,kl}.
 * df_lrdf_build writes T (omega > 0) into B in the DF_FP64 layout of df_build_B
 * (df_B_bytes(nao, naux, DF_FP64) bytes), synchronising once for the metric's pivot check
 * (DF_ERR_NOT_SPD).  df_lrdf_jk returns J[D] and K[C C^T] (either may be NULL) as the
 * long-range DF part (df_jk on T) plus the short-range four-centre part, summed directly over
 * orbital pairs (quartets whose pair factors multiply to less than 1e-16 of the largest are
 * skipped).  The short-range sums cost O(npair^2) for J and O(nao^4) for K: meant for
 * molecules of up to a few hundred basis functions.  Both synchronise the stream once.
 * works: df_lrdf_build_work_bytes(nao, naux), df_lrdf_jk_work_bytes(nao, naux, nocc).       */
size_t df_lrdf_build_work_bytes(int nao, int naux);
int df_lrdf_build(const double* ao_xyz, const double* ao_exp, int nao, const double* aux_xyz, const double* aux_exp,
                  int naux, double omega, void* B, size_t B_bytes, void* work, size_t work_bytes, cudaStream_t s);
size_t df_lrdf_jk_work_bytes(int nao, int naux, int nocc);
int df_lrdf_jk(const void* B_lr, const double* ao_xyz, const double* ao_exp, int nao, int naux, double omega,
               const double* D, const double* C, int nocc, double* J, double* K, void* work, size_t work_bytes,
               cudaStream_t s);

/* ---- core-Hamiltonian guess ------------------------------------------------------------
 * S, h = T + V, canonical orthogonalisation X (eigenvalues of S above lindep), the
 * nocc = nelec/2 lowest eigenvectors C_occ = X C' of X^T h X and D = 2 C_occ C_occ^T: the
 * default starting point of the SCF (the paper's initial-guess section).  Outputs are
 * device buffers and may be NULL except C_occ and D; *nmo_out (HOST, may be NULL) gets the
 * number of orbitals kept.  Synchronises the stream.
 * work: df_core_guess_work_bytes(nao, nocc) bytes.                                       */
size_t df_core_guess_work_bytes(int nao, int nocc);
int df_core_guess(const df_molecule* mol, double lindep, double* S_out, double* h_out, double* C_occ,
                  double* D_out, double* mo_energy, int* nmo_out, void* work, size_t work_bytes,
                  cudaStream_t s);

/* ---- Coulomb build without a caller workspace ------------------------------------------
 * The paper has no counterpart of this entry point; it exists for callers that cannot
 * allocate device memory for a workspace (plugins whose host framework owns every device
 * allocation, and latency-critical services that forbid allocation once running).
 * Computes exactly what df_jk computes for J in DF_FP64 mode (K is not available here):
 * J[D]_mn = sum_P d_P B_{P,mn}, d_P = sum_{kl} B_{P,kl} D_kl, from the FP64 packed rows of
 * a B built by df_build_B in either precision.  B, D [nao][nao] and J [nao][nao] are
 * device pointers owned by the caller.
 * Scratch comes from one fixed device array of df_j_noalloc_capacity() bytes (8 MiB)
 * that the library reserves on every GPU that loads it, until the process exits.  The
 * call allocates nothing and returns DF_ERR_ARG when (nao, naux) need more than that
 * (for example nao <= 400 with naux <= 1200 always fits; nao 1500 does not).
 * Each call made outside a stream capture looks up the array's device address (with the
 * calling thread's current device); a call inside a capture reuses the address of the
 * last such call on that device, so make one call on each device before capturing (a first
 * call inside a capture returns DF_ERR_ARG).  Every call shares the array and it keeps the
 * last call's contents: calls whose GPU work overlaps (other streams or threads on the same
 * device) race and must be ordered by the caller.                                        */
size_t df_j_noalloc_capacity(void);
int df_j_noalloc(const void* B, int nao, int naux, const double* D, double* J, cudaStream_t s);

/* ---- tuning knobs ------------------------------------------------------------------------
 * Launch parameters chosen by the autotuner (paper_2506_06661_gb300/tune.py): "umma_max_stages"
 * (2..8, the largest shared-memory ring depth of the tensor-core GEMM; as many stages as fit
 * up to that), "syrk_pair" (0, the default: one CTA per 128 x 128 tile of the exchange
 * SYRK; 1: 256 x 128 blocks on CTA pairs, tcgen05 cta_group::2, each CTA staging its own A rows
 * and half of B), "syrk_bk" (one-CTA SYRK only: 32, or 16 for K boxes of 16 elements, so that
 * twice as many narrower stages are in flight), "syrk_split" and "fp64_syrk_split"
 * (K-dimension splits of the exchange SYRK, 0 = built-in heuristic), "jpass2_rows" (32..512,
 * auxiliary rows per CTA slice of J's second pass), "eig_ctas" (CTAs of the multi-SM
 * eigensolver: 0 automatic, 1 a single CTA) and "mixed_planes" (3..5 BF16 planes per operand of
 * the mixed exchange: 6, 10 or 15 plane products; it also sizes a mixed B).
 * Tile shapes: "fp64_ht_cols" (0 automatic, 16 or 32 occupied columns per FP64 half-transform
 * CTA), "ht_n" (0: the widest tcgen05 half-transform tile that fits; else a cap, a multiple
 * of 16), "jpass1_rows" (1, 2, 4 or 8 auxiliary rows per CTA of J's first pass) and
 * "j_fp64_fma" (1: J's passes with FP64 FMAs instead of double-float products).
 * "mixed_incremental" (0 or 1), "soscf" (0 or 1) and "soscf_cg" (1..64) shape the SCF as
 * described at scf_run; "stability" (0, 1 or 2) finds the lowest eigenvalue of
 * the orbital Hessian of every converged solution by Davidson's method with the
 * eps_a - eps_i preconditioner, to a residual below 1e-5 or at most "stability_steps"
 * (2..400, default 60) Hessian products (scf_result.hess_min; the products use the SCF's
 * precision, one J and two exchange builds each); with 2, a solution whose
 * hess_min is below -1e-4 (a saddle point) is turned by 0.3 rad along the Ritz vector of that
 * eigenvalue and the SCF goes on from there in FP64 (Newton steps when "soscf" is on) with a
 * fresh max_cycle budget, at most three times (scf_result.stability_restarts); "dm0_eig_cut" (1..16, default 12) drops natural occupations of a
 * non-idempotent dm0 below 10^-cut of the largest from its first exchange; "guess_idem_max"
 * (1..1000, default 200) is the largest idempotency error of an accepted dm0, in hundredths.
 * Two more knobs bound the multi-SM eigensolver's grid barriers:
 * "eig_barrier_polls" (256..2^30 polls before a wait gives up with DF_ERR_TIMEOUT; default 2^22, about a second) and "eig_barrier_extra"
 * (0 or 1; 1 makes every barrier wait for one arrival that never comes, so that a test can
 * watch the bounded wait run out; leave it 0).  Host-side process-wide state: change
 * knobs only between calls and re-query *_work_bytes afterwards (split counts size the
 * workspaces).  df_tune_set returns DF_ERR_ARG for an unknown name or an out-of-range value;
 * df_tune_get returns -1 for an unknown name; df_tune_reset puts every knob back to its
 * built-in value.                                                                           */
int df_tune_set(const char* name, int value);
int df_tune_get(const char* name);
void df_tune_reset(void);

/* ---- bounds-checking build -------------------------------------------------------------
 * A build of this library with -DDFSCF_BOUNDS_CHECK (libdfscf_bounds.so) checks the global
 * index of the kernels' computed accesses against their buffer's extent; a bad index is
 * counted, the first one is recorded with its bound and source line, and the access is
 * redirected to element 0 so that the run continues without a fault (it stands in for a
 * memory checker).  df_bounds_checked() is 1 in that build, 0 otherwise.
 * df_bounds_violations synchronises the device, writes the number of bad indices since the
 * last call to the HOST *count and the first one's location to where (HOST, may be NULL),
 * and clears the records (always 0 in the normal build).                                   */
int df_bounds_checked(void);
int df_bounds_violations(unsigned long long* count, char* where, size_t where_bytes);

/* ---- phase profiler ------------------------------------------------------------------
 * When enabled, the J/K builds bracket each kernel phase with CUDA events on the
 * launching stream.  df_profile_count() synchronises those events and returns the number
 * of distinct phases; name / total milliseconds / number of launches per phase follow.
 * Host-side state, not thread-safe; off by default.                                      */
void df_profile_enable(int on);
void df_profile_reset(void);
int df_profile_count(void);
const char* df_profile_name(int i);
double df_profile_ms(int i);
long df_profile_calls(int i);

#ifdef __cplusplus
}
#endif
#endif /* DFSCF_H */
