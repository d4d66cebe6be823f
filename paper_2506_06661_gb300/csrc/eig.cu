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

// A [n][n] symmetric (full storage), overwritten.  Outputs w [n] ascending and
// ZT [n][n] with eigenvector k in row k.  Scratch: d, e, beta, v (n each), cs, sn (n each).
__device__ int eigh_cta(double* __restrict__ A, int n, double* __restrict__ w, double* __restrict__ ZT,
                        double* __restrict__ d, double* __restrict__ e, double* __restrict__ beta,
                        double* __restrict__ v, double* __restrict__ cs, double* __restrict__ sn, EigShared& sh) {
  const int tid = threadIdx.x, nt = blockDim.x;
  // ---- 1. tridiagonalisation --------------------------------------------------------
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
  int fail = 0;
  for (int l = 0; l < n; ++l) {
    int iter = 0;
    while (true) {
      // lane 0 runs the scalar recurrence of one sweep and records its rotations
      if (tid == 0) {
        int m = l;
        for (; m < n - 1; ++m) {
          double dd = fabs(d[m]) + fabs(d[m + 1]);
          if (fabs(e[m]) <= DBL_EPSILON * dd) break;
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
      for (int col = tid; col < n; col += nt) {
        for (int i = hi; i >= lo; --i) {
          double zi = ZT[(size_t)i * n + col], zi1 = ZT[(size_t)(i + 1) * n + col];
          ZT[(size_t)(i + 1) * n + col] = sn[i] * zi + cs[i] * zi1;
          ZT[(size_t)i * n + col] = cs[i] * zi - sn[i] * zi1;
        }
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
