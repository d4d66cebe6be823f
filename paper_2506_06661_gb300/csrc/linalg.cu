// FP64 dense linear algebra on CUDA cores: a register-tiled GEMM (batched, split-K,
// lower-triangle-only), the blocked Cholesky factorisation of the Coulomb metric
// M = L L^T and the blocked forward substitution B = L^-1 R of the density-fitting
// whitening (arXiv 2506.06661, Section "Density fitting").  On this GPU FP64 runs at
// about 1.9 FMA/clk/SM, so these kernels are FP64-ALU bound by design; they only need
// coalesced loads and enough independent FMAs per thread.
#include "common.cuh"
#include "kernels.cuh"

namespace dfscf {

constexpr int GB_M = 64, GB_N = 64, GB_K = 16;

// C = alpha * op(A) op(B) + beta * C.
//   op(A)(m,k) = TA ? A[k*lda + m] : A[m*lda + k];  op(B)(k,n) = TB ? B[n*ldb + k] : B[k*ldb + n].
// blockIdx.z: batch index (strides sA, sB, sC) or, when kchunk > 0, a split of the K range
// [z*kchunk, min(K, (z+1)*kchunk)) with output slice C + z*sC.
// lower_only: tiles strictly above the diagonal are skipped.
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) dgemm_kernel(int M, int N, int K, double alpha, const double* __restrict__ A,
                                                    long lda, long sA, const double* __restrict__ B, long ldb, long sB,
                                                    double beta, double* __restrict__ C, long ldc, long sC,
                                                    long kchunk, int lower_only) {
  int mt = blockIdx.y, nt = blockIdx.x;
  if (lower_only && mt < nt) return;
  __shared__ double As[GB_K][GB_M + 1];
  __shared__ double Bs[GB_K][GB_N + 1];
  long k_begin = 0, k_end = K;
  if (kchunk > 0) {
    k_begin = (long)blockIdx.z * kchunk;
    k_end = min((long)K, k_begin + kchunk);
    C += (size_t)blockIdx.z * sC;
  } else {
    A += (size_t)blockIdx.z * sA;
    B += (size_t)blockIdx.z * sB;
    C += (size_t)blockIdx.z * sC;
  }
  int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  int m0 = mt * GB_M, n0 = nt * GB_N;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (long k0 = k_begin; k0 < k_end; k0 += GB_K) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int idx = threadIdx.x + 256 * r;
      int mm, kk;
      if (TA) { kk = idx >> 6; mm = idx & 63; } else { mm = idx >> 4; kk = idx & 15; }
      long gk = k0 + kk;
      int gm = m0 + mm;
      double v = 0.0;
      if (gm < M && gk < k_end) v = TA ? A[gk * lda + gm] : A[(long)gm * lda + gk];
      As[kk][mm] = v;
      int nn;
      if (TB) { nn = idx >> 4; kk = idx & 15; } else { kk = idx >> 6; nn = idx & 63; }
      gk = k0 + kk;
      int gn = n0 + nn;
      v = 0.0;
      if (gn < N && gk < k_end) v = TB ? B[(long)gn * ldb + gk] : B[gk * ldb + gn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GB_K; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      double* c = C + (long)gm * ldc + gn;
      *c = (beta == 0.0) ? alpha * acc[i][j] : fma(alpha, acc[i][j], beta * *c);
    }
  }
}

int dgemm(bool ta, bool tb, int M, int N, int K, double alpha, const double* A, long lda, long sA, const double* B,
          long ldb, long sB, double beta, double* C, long ldc, long sC, int batch, cudaStream_t s, long kchunk,
          int lower_only) {
  if (M <= 0 || N <= 0 || batch <= 0) return DF_OK;
  dim3 grid((N + GB_N - 1) / GB_N, (M + GB_M - 1) / GB_M, batch);
  DF_REQUIRE(grid.y <= 65535 && grid.z <= 65535, DF_ERR_ARG, "dgemm: grid too large (M=%d batch=%d)", M, batch);
  if (!ta && !tb)
    dgemm_kernel<false, false><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, kchunk, lower_only);
  else if (!ta && tb)
    dgemm_kernel<false, true><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, kchunk, lower_only);
  else if (ta && !tb)
    dgemm_kernel<true, false><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, kchunk, lower_only);
  else
    dgemm_kernel<true, true><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, kchunk, lower_only);
  DF_LAUNCHED("dgemm_kernel");
  return DF_OK;
}

// ---- Cholesky ----------------------------------------------------------------------
constexpr int CH_NB = 64;

__global__ void chol_init_kernel(const double* __restrict__ A, int n, double* maxdiag, int* status) {
  __shared__ double sh[32];
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, A[(size_t)i * n + i]);
  // block max via warp shuffles
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = fmax(t, sh[i]);
    *maxdiag = t;
    *status = -1;
  }
}

// Factor the b x b diagonal block at (k0, k0) in shared memory (right-looking, one CTA).
__global__ void __launch_bounds__(256) chol_diag_kernel(double* __restrict__ A, int n, int k0, int b,
                                                        const double* maxdiag, int* status, double tol) {
  __shared__ double T[CH_NB][CH_NB + 1];
  __shared__ int fail;
  if (*status >= 0) return;
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    int i = e / b, j = e % b;
    T[i][j] = A[(size_t)(k0 + i) * n + k0 + j];
  }
  if (threadIdx.x == 0) fail = -1;
  __syncthreads();
  double thr = tol * *maxdiag;
  for (int j = 0; j < b; ++j) {
    if (threadIdx.x == 0) {
      double piv = T[j][j];
      if (!(piv > thr)) fail = j;
      else T[j][j] = sqrt(piv);
    }
    __syncthreads();
    if (fail >= 0) break;
    double ljj = T[j][j];
    for (int i = j + 1 + threadIdx.x; i < b; i += blockDim.x) T[i][j] /= ljj;
    __syncthreads();
    int rem = b - j - 1;
    for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
      int i = j + 1 + e / rem, c = j + 1 + e % rem;
      if (c <= i) T[i][c] -= T[i][j] * T[c][j];
    }
    __syncthreads();
  }
  if (fail >= 0) {
    if (threadIdx.x == 0) atomicCAS(status, -1, k0 + fail);
    return;
  }
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    int i = e / b, j = e % b;
    A[(size_t)(k0 + i) * n + k0 + j] = (j <= i) ? T[i][j] : 0.0;
  }
}

// Panel below the diagonal block: L[i, k0:k0+b] = A[i, k0:k0+b] L_kk^-T, one lane per row.
__global__ void chol_panel_kernel(double* __restrict__ A, int n, int k0, int b, const int* status) {
  __shared__ double Lk[CH_NB][CH_NB + 1];
  if (*status >= 0) return;
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    int i = e / b, j = e % b;
    Lk[i][j] = A[(size_t)(k0 + i) * n + k0 + j];
  }
  __syncthreads();
  int i = k0 + b + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double* row = A + (size_t)i * n + k0;
  for (int j = 0; j < b; ++j) {
    double x = row[j];
    for (int m = 0; m < j; ++m) x -= row[m] * Lk[j][m];
    row[j] = x / Lk[j][j];
  }
}

__global__ void zero_upper_kernel(double* __restrict__ A, int n) {
  long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)n * n) return;
  int i = (int)(e / n), j = (int)(e % n);
  if (j > i) A[e] = 0.0;
}

int cholesky_inplace(double* A, int n, int* d_status, double* d_maxdiag, double tol, cudaStream_t s) {
  chol_init_kernel<<<1, 1024, 0, s>>>(A, n, d_maxdiag, d_status);
  DF_LAUNCHED("chol_init_kernel");
  for (int k0 = 0; k0 < n; k0 += CH_NB) {
    int b = min(CH_NB, n - k0);
    chol_diag_kernel<<<1, 256, 0, s>>>(A, n, k0, b, d_maxdiag, d_status, tol);
    DF_LAUNCHED("chol_diag_kernel");
    int rest = n - k0 - b;
    if (rest <= 0) break;
    chol_panel_kernel<<<(rest + 127) / 128, 128, 0, s>>>(A, n, k0, b, d_status);
    DF_LAUNCHED("chol_panel_kernel");
    int k1 = k0 + b;
    DF_TRY(dgemm(false, true, rest, rest, b, -1.0, A + (size_t)k1 * n + k0, n, 0, A + (size_t)k1 * n + k0, n, 0, 1.0,
                 A + (size_t)k1 * n + k1, n, 0, 1, s, 0, 1));
  }
  long nn = (long)n * n;
  zero_upper_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(A, n);
  DF_LAUNCHED("zero_upper_kernel");
  return DF_OK;
}

// ---- forward substitution B = L^-1 R ---------------------------------------------------
// Rows k0..k0+b of R are solved against the diagonal block of L, one lane per column.
template <int NB>
__global__ void __launch_bounds__(128) trsm_diag_kernel(double* __restrict__ R, long ld, long ncol,
                                                        const double* __restrict__ L, int naux, int k0) {
  __shared__ double Lk[NB][NB];
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    int i = e / NB, j = e % NB;
    Lk[i][j] = (j <= i) ? L[(size_t)(k0 + i) * naux + k0 + j] : 0.0;
  }
  __syncthreads();
  long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncol) return;
  double x[NB];
#pragma unroll
  for (int p = 0; p < NB; ++p) x[p] = R[(size_t)(k0 + p) * ld + c];
#pragma unroll
  for (int p = 0; p < NB; ++p) {
    double v = x[p];
#pragma unroll
    for (int q = 0; q < p; ++q) v = fma(-Lk[p][q], x[q], v);
    x[p] = v / Lk[p][p];
  }
#pragma unroll
  for (int p = 0; p < NB; ++p) R[(size_t)(k0 + p) * ld + c] = x[p];
}

__global__ void trsm_diag_generic_kernel(double* __restrict__ R, long ld, long ncol, const double* __restrict__ L,
                                         int naux, int k0, int b) {
  long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncol) return;
  for (int p = 0; p < b; ++p) {
    double v = R[(size_t)(k0 + p) * ld + c];
    for (int q = 0; q < p; ++q) v -= L[(size_t)(k0 + p) * naux + k0 + q] * R[(size_t)(k0 + q) * ld + c];
    R[(size_t)(k0 + p) * ld + c] = v / L[(size_t)(k0 + p) * naux + k0 + p];
  }
}

int forward_substitution(double* R, long ld, long ncol, const double* L, int naux, cudaStream_t s) {
  constexpr int NB = 32;
  for (int k0 = 0; k0 < naux; k0 += NB) {
    int b = min(NB, naux - k0);
    unsigned blocks = (unsigned)((ncol + 127) / 128);
    if (b == NB)
      trsm_diag_kernel<NB><<<blocks, 128, 0, s>>>(R, ld, ncol, L, naux, k0);
    else
      trsm_diag_generic_kernel<<<blocks, 128, 0, s>>>(R, ld, ncol, L, naux, k0, b);
    DF_LAUNCHED("trsm_diag_kernel");
    int rest = naux - k0 - b;
    if (rest <= 0) break;
    // R[k0+b:, :] -= L[k0+b:, k0:k0+b] R[k0:k0+b, :], in column chunks (grid.x limit is ample)
    DF_TRY(dgemm(false, false, rest, (int)ncol, b, -1.0, L + (size_t)(k0 + b) * naux + k0, naux, 0,
                 R + (size_t)k0 * ld, ld, 0, 1.0, R + (size_t)(k0 + b) * ld, ld, 0, 1, s, 0, 0));
  }
  return DF_OK;
}

}  // namespace dfscf

using namespace dfscf;

extern "C" size_t df_metric_chol_work_bytes(int naux) {
  (void)naux;
  return 512;
}

extern "C" int df_metric_chol(const double* aux_xyz, const double* aux_exp, int naux, double* L, double* M_out,
                              int* bad_pivot, void* work, size_t work_bytes, cudaStream_t s) {
  clear_error();
  DF_REQUIRE(naux > 0 && aux_xyz && aux_exp && L && bad_pivot, DF_ERR_ARG, "df_metric_chol: bad arguments");
  DF_REQUIRE(work && work_bytes >= df_metric_chol_work_bytes(naux), DF_ERR_NOMEM,
             "df_metric_chol: workspace of %zu bytes is smaller than %zu", work_bytes, df_metric_chol_work_bytes(naux));
  *bad_pivot = -1;
  int* d_status = (int*)work;
  double* d_maxdiag = (double*)((char*)work + 256);
  DF_TRY(launch_int2c(aux_xyz, aux_exp, naux, L, s));
  if (M_out) DF_CUDA(cudaMemcpyAsync(M_out, L, sizeof(double) * naux * naux, cudaMemcpyDeviceToDevice, s));
  DF_TRY(cholesky_inplace(L, naux, d_status, d_maxdiag, 1e-14, s));
  int h_status = -1;
  DF_CUDA(cudaMemcpyAsync(&h_status, d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  DF_CUDA(cudaStreamSynchronize(s));
  if (h_status >= 0) {
    *bad_pivot = h_status;
    set_error("df_metric_chol: metric not positive definite at pivot %d", h_status);
    return DF_ERR_NOT_SPD;
  }
  return DF_OK;
}

DF_BOUNDS_READER(bounds_read_linalg)
