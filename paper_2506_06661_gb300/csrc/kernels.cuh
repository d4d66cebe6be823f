// Internal launchers shared between the library's translation units.
#pragma once
#include <cstddef>
#include <vector>
#include <algorithm>

#include "common.cuh"

namespace dfscf {

// ---- integrals (integrals.cu) ------------------------------------------------------
int launch_int1e(const double* ao_xyz, const double* ao_exp, int nao, const double* nuc_xyz, const double* nuc_z,
                 int natm, double* S, double* T, double* V, cudaStream_t s);
// Per packed orbital pair: exponent p, centre (x, y, z) and factor K_ab = N_a N_b e^{-mu R^2}
// 2 pi^{5/2} / p, as five arrays of npair doubles in pair_tab.
int launch_pair_table(const double* ao_xyz, const double* ao_exp, int nao, double* pair_tab, cudaStream_t s);
// omega > 0: the long-range operator erf(omega r)/r instead of 1/r (LRDF)
int launch_int2c(const double* xyz, const double* ex, int naux, double* M, cudaStream_t s, double omega = 0.0);
int launch_int3c(const double* ao_xyz, const double* ao_exp, int nao, const double* aux_xyz, const double* aux_exp,
                 int naux, double* R, long ld, double* pair_tab, cudaStream_t s, double omega = 0.0);
int launch_enuc(const double* xyz, const double* z, int natm, double* out, cudaStream_t s);

// ---- FP64 linear algebra (linalg.cu) -----------------------------------------------
int dgemm(bool ta, bool tb, int M, int N, int K, double alpha, const double* A, long lda, long sA, const double* B,
          long ldb, long sB, double beta, double* C, long ldc, long sC, int batch, cudaStream_t s, long kchunk,
          int lower_only);
int cholesky_inplace(double* A, int n, int* d_status, double* d_maxdiag, double tol, cudaStream_t s);
int forward_substitution(double* R, long ld, long ncol, const double* L, int naux, cudaStream_t s);

// ---- eigensolver (eig.cu) ------------------------------------------------------------
size_t eigh_scratch_doubles(int n);
int eigh_rows(double* A, int n, double* w, double* ZT, double* scratch, int* status, cudaStream_t s);
size_t eigh_lowest_scratch_doubles(int n, int k);
size_t eigh_coop_aux_bytes(int n);
size_t eigh_full_scratch_doubles(int n);
int eigh_full_rows(double* A, int n, double* w, double* ZT, double* scratch, int* status, cudaStream_t s, void* aux);
// S^p over the eigenvalues of S above lindep, from its eigenvector rows ZT and eigenvalues (lowdin.cu).
int lowdin_power(const double* ZT, const double* s_eig, int n, double lindep, double power, double* scratch,
                 double* out, cudaStream_t s);
int eigh_lowest_rows(double* A, int n, int k, double* w, double* ZT, double* scratch, int* status, cudaStream_t s,
                     void* aux);
int transpose(const double* in, int rows, int cols, double* out, cudaStream_t s);

// ---- B layout and J/K (jk.cu, umma.cu) --------------------------------------------------
// Most BF16 planes a mixed-precision B can hold; a B keeps as many as the knob "mixed_planes"
// asked for when it was sized and built (3, 4 or 5).
constexpr int kMixedPlanes = 5;

struct BLayout {
  long ld;       // packed row stride (elements)
  int npad;      // padded orbital dimension of the BF16 planes
  int planes;    // BF16 planes held (0 for DF_FP64)
  size_t off64, offp[kMixedPlanes], bytes;
};

struct MixedKWork {
  void* Cp[kMixedPlanes];  // bf16 [ncpad][npad]  planes of C^T
  void* Xp[kMixedPlanes];  // bf16 [npad][naux * ncpad]  planes of X (row m, column P*ncpad + i)
  float* X32;              // fp32 [2][npad][naux * ncpad]  X from the half transform as a pair
                           //   (order-0 accumulator, higher-order accumulator)
  unsigned* xmax;          // [npad] max |X| of row m (FP32 bits)
  float* Kpart;            // fp32 [nsplit][npad][npad] partial K tiles
  int* err;                // device error flag of the tensor-core kernels
  int ncpad;               // padded occupied count (multiple of 16, >= 16)
  int nsplit;              // K-dimension splits of the exchange contraction
  int planes;              // BF16 planes per operand (3, 4, 5: 6, 10, 15 plane products)
};

struct JKWork {
  double* Dw;
  double* d;
  double* Jpart;
  double* X;
  double* Kpart;
  int nsplit_j, nsplit_k;
  MixedKWork mk;
};

long B_ld(int nao);
int nao_pad(int nao);
// planes: BF16 planes of a mixed B (ignored for DF_FP64); plane j sits at the same offset
// whatever the count, so a B with more planes serves an exchange that uses fewer.
BLayout B_layout(int nao, int naux, int precision, int planes);
int mixed_planes();
// Host-side record of the plane count each mixed B was built with (keyed by its address),
// checked before an exchange reads the planes; -1 if the address was never recorded.
void record_B_planes(const void* B, int planes);
int recorded_B_planes(const void* B);
JKWork jk_work_layout(int nao, int naux, int nocc, int precision, Arena* a, Sizer* z, bool fp64_k);
int umma_prepare();
void mixed_k_work_layout(int nao, int naux, int nocc, Arena* a, Sizer* z, MixedKWork* w);
int build_K_mixed(const void* B, const BLayout& L, int nao, int naux, const double* C, int nocc, double* K,
                  const MixedKWork& w, cudaStream_t s);
int build_J(const void* Bbuf, const BLayout& L, int nao, int naux, int precision, const double* D, double* J,
            const JKWork& w, cudaStream_t s);
int run_jk(const void* B, int nao, int naux, int precision, const double* D, const double* C, int nocc, double* J,
           double* K, const JKWork& w, cudaStream_t s);
int build_B(const double* ao_xyz, const double* ao_exp, int nao, const double* aux_xyz, const double* aux_exp,
            int naux, const double* Lfac, int precision, void* Bbuf, double* pair_tab, cudaStream_t s);

// Bounds-check records of the translation units with kernels (checking build; all zero
// otherwise).
int bounds_read_dferr(BoundsRecord*);
int bounds_read_eig(BoundsRecord*);
int bounds_read_integrals(BoundsRecord*);
int bounds_read_jk(BoundsRecord*);
int bounds_read_linalg(BoundsRecord*);
int bounds_read_lowdin(BoundsRecord*);
int bounds_read_lrdf(BoundsRecord*);
int bounds_read_mlp(BoundsRecord*);
int bounds_read_scf(BoundsRecord*);
int bounds_read_umma(BoundsRecord*);

}  // namespace dfscf
