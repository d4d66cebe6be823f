// Loewdin factors S^1/2, S^-1/2 and the congruence M A M, used by the learned guess: its
// network predicts centre-pair blocks of the orthonormalised density Dt = S^1/2 D S^1/2,
// and the starting density handed to the SCF is D0 = S^-1/2 Dt S^-1/2.
#include <cmath>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace dfscf {

// W[k][j] = ZT[k][j] * s_k^power for s_k > lindep, 0 otherwise (eigenvector rows ZT).
__global__ void scaled_rows_kernel(const double* __restrict__ ZT, const double* __restrict__ s, int n, double lindep,
                                   double power, double* __restrict__ W) {
  long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long)n * n) return;
  int k = (int)(q / n);
  double f = s[k] > lindep ? pow(s[k], power) : 0.0;
  W[q] = ZT[q] * f;
}

static unsigned nblk(long n) { return (unsigned)((n + 255) / 256); }

// S^p = ZT^T diag(s^p) ZT over the eigenvalues above lindep, from eigenvector rows ZT and
// eigenvalues s of S (scratch: n x n).
int lowdin_power(const double* ZT, const double* s_eig, int n, double lindep, double power, double* scratch,
                 double* out, cudaStream_t s) {
  const long nn = (long)n * n;
  scaled_rows_kernel<<<nblk(nn), 256, 0, s>>>(ZT, s_eig, n, lindep, power, scratch);
  DF_LAUNCHED("scaled_rows_kernel");
  return dgemm(true, false, n, n, n, 1.0, ZT, n, 0, scratch, n, 0, 0.0, out, n, 0, 1, s, 0, 0);
}

}  // namespace dfscf

using namespace dfscf;

extern "C" size_t df_lowdin_work_bytes(int nao) {
  if (nao <= 0) return 0;
  Sizer z;
  z.take<double>((size_t)nao * nao);  // S
  z.take<double>((size_t)nao * nao);  // eigenvector rows
  z.take<double>((size_t)nao * nao);  // scaled rows
  z.take<double>(nao);                // eigenvalues
  z.take<double>(eigh_full_scratch_doubles(nao));
  z.take<int>(1);
  z.take<char>(eigh_coop_aux_bytes(nao));
  return z.used;
}

extern "C" int df_lowdin_factors(const double* ao_xyz, const double* ao_exp, int nao, double lindep, double* Shalf,
                                 double* Sinvhalf, void* work, size_t work_bytes, cudaStream_t s) {
  clear_error();
  DF_REQUIRE(ao_xyz && ao_exp && nao > 0 && (Shalf || Sinvhalf), DF_ERR_ARG, "df_lowdin_factors: bad arguments");
  DF_REQUIRE(work && work_bytes >= df_lowdin_work_bytes(nao), DF_ERR_NOMEM, "df_lowdin_factors: workspace too small");
  Arena a(work, work_bytes);
  double* S = a.take<double>((size_t)nao * nao);
  double* ZT = a.take<double>((size_t)nao * nao);
  double* W = a.take<double>((size_t)nao * nao);
  double* w = a.take<double>(nao);
  double* scr = a.take<double>(eigh_full_scratch_doubles(nao));
  int* status = a.take<int>(1);
  void* aux = a.take<char>(eigh_coop_aux_bytes(nao));
  const long nn = (long)nao * nao;
  DF_TRY(launch_int1e(ao_xyz, ao_exp, nao, nullptr, nullptr, 0, S, nullptr, nullptr, s));
  DF_TRY(eigh_full_rows(S, nao, w, ZT, scr, status, s, aux));
  // S^p = sum_k u_k s_k^p u_k^T = ZT^T diag(s^p) ZT
  if (Shalf) {
    scaled_rows_kernel<<<nblk(nn), 256, 0, s>>>(ZT, w, nao, lindep, 0.5, W);
    DF_LAUNCHED("scaled_rows_kernel");
    DF_TRY(dgemm(true, false, nao, nao, nao, 1.0, ZT, nao, 0, W, nao, 0, 0.0, Shalf, nao, 0, 1, s, 0, 0));
  }
  if (Sinvhalf) {
    scaled_rows_kernel<<<nblk(nn), 256, 0, s>>>(ZT, w, nao, lindep, -0.5, W);
    DF_LAUNCHED("scaled_rows_kernel");
    DF_TRY(dgemm(true, false, nao, nao, nao, 1.0, ZT, nao, 0, W, nao, 0, 0.0, Sinvhalf, nao, 0, 1, s, 0, 0));
  }
  int h = 0;
  DF_CUDA(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s));
  DF_CUDA(cudaStreamSynchronize(s));
  DF_REQUIRE(h != 3, DF_ERR_TIMEOUT, "df_lowdin_factors: a grid barrier of the eigensolver timed out");
  DF_REQUIRE(h == 0, DF_ERR_NOCONV, "df_lowdin_factors: eigensolver failed on S");
  return DF_OK;
}

extern "C" size_t df_congruence_work_bytes(int n) { return n > 0 ? align_up(sizeof(double) * (size_t)n * n, 256) : 0; }

extern "C" int df_congruence(const double* M, const double* A, int n, double* out, void* work, size_t work_bytes,
                             cudaStream_t s) {
  clear_error();
  DF_REQUIRE(M && A && out && n > 0 && out != A && out != M, DF_ERR_ARG, "df_congruence: bad arguments");
  DF_REQUIRE(work && work_bytes >= df_congruence_work_bytes(n), DF_ERR_NOMEM, "df_congruence: workspace too small");
  double* T = (double*)work;
  DF_TRY(dgemm(false, false, n, n, n, 1.0, A, n, 0, M, n, 0, 0.0, T, n, 0, 1, s, 0, 0));
  DF_TRY(dgemm(false, false, n, n, n, 1.0, M, n, 0, T, n, 0, 0.0, out, n, 0, 1, s, 0, 0));
  return DF_OK;
}

DF_BOUNDS_READER(bounds_read_lowdin)
