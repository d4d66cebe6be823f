// Whitened three-index tensor B and the DF Coulomb / exchange builds
// (arXiv 2506.06661, Section "Density fitting"):
//   B_{P,mn} = sum_Q (L^-1)_{PQ} (Q|mn)
//   J_mn = sum_P d_P B_{P,mn},  d_P = sum_{kl} B_{P,kl} D_kl       (J = sum_P B_P (B_P . D))
//   K_mn = sum_P sum_i X_{P,mi} X_{P,ni},  X_P = B_P C
//
// B layout (one caller-owned buffer):
//   FP64 packed rows        naux x ld doubles,  ld = npair rounded up to 32 (256-byte rows)
//   BF16 planes 0..NP-1     naux x npad x npad  (mixed mode; full symmetric B_P, npad = nao
//                                                rounded up to 128, zero padding; NP = 3..5)
// With sigma the power of two just above the row's max |x|, planes 0 and 1 are fixed-point
// (x on the grid sigma 2^-7, then the remainder on sigma 2^-15) and planes 2..NP-1 are BF16
// roundings of what is left (planes.cuh).  J streams the FP64 packed rows in both modes
// (each symmetric pair stored once, weight 2 off the diagonal); the mixed K reads the BF16
// planes through TMA as plain K-major GEMM operands.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>
#include <unordered_map>

#include "common.cuh"
#include "kernels.cuh"
#include "planes.cuh"

namespace dfscf {

long B_ld(int nao) { return (long)align_up((size_t)npair_of(nao), 32); }
int nao_pad(int nao) { return (int)align_up((size_t)nao, 128); }

BLayout B_layout(int nao, int naux, int precision, int planes) {
  BLayout L{};
  L.ld = B_ld(nao);
  L.npad = nao_pad(nao);
  L.planes = precision == DF_MIXED ? std::min(kMixedPlanes, std::max(3, planes)) : 0;
  size_t off = 0;
  L.off64 = off;
  off += align_up(sizeof(double) * (size_t)naux * L.ld, 256);
  for (int j = 0; j < L.planes; ++j) {
    L.offp[j] = off;
    off += align_up(sizeof(__nv_bfloat16) * (size_t)naux * L.npad * L.npad, 256);
  }
  L.bytes = off;
  return L;
}

static std::mutex g_bplanes_mutex;
static std::unordered_map<uintptr_t, int> g_bplanes;

void record_B_planes(const void* B, int planes) {
  std::lock_guard<std::mutex> lock(g_bplanes_mutex);
  g_bplanes[(uintptr_t)B] = planes;
}

int recorded_B_planes(const void* B) {
  std::lock_guard<std::mutex> lock(g_bplanes_mutex);
  auto it = g_bplanes.find((uintptr_t)B);
  return it == g_bplanes.end() ? -1 : it->second;
}

// ---- BF16 planes of B ------------------------------------------------------------------
// Row (P, m) of the full symmetric B_P (over n) as `planes` row-scaled planes (planes.cuh;
// residuals in FP64).  One CTA per row; padding (m or n >= nao) is zero.
struct PlaneOut {
  __nv_bfloat16* p[kMixedPlanes];
  int planes;
};

__global__ void __launch_bounds__(128) b_to_planes_kernel(const double* __restrict__ B64, long ld, int nao, int npad,
                                                          PlaneOut out) {
  __shared__ double sh[4];
  const int m = blockIdx.x, P = blockIdx.y;
  const double* row = B64 + (size_t)P * ld;
  auto load = [&](int n) -> double {
    if (m >= nao || n >= nao) return 0.0;
    int a = max(m, n), b = min(m, n);
    return row[DF_IX((size_t)a * (a + 1) / 2 + b, ld)];
  };
  double amax = 0.0;
  for (int n = threadIdx.x; n < npad; n += blockDim.x) amax = fmax(amax, fabs(load(n)));
  for (int o = 16; o; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = amax;
  __syncthreads();
  const double sig = row_scale(fmax(fmax(sh[0], sh[1]), fmax(sh[2], sh[3])));
  const size_t o = ((size_t)P * npad + m) * npad;
  for (int n = threadIdx.x; n < npad; n += blockDim.x) {
    __nv_bfloat16 q[kPlanesMax];
    split_row_value(load(n), sig, q);
#pragma unroll
    for (int j = 0; j < kMixedPlanes; ++j)
      if (j < out.planes) out.p[j][DF_IX(o + n, (size_t)gridDim.y * npad * npad)] = q[j];
  }
}

// ---- J --------------------------------------------------------------------------------
// Dw_mn = w_mn D_mn for packed m >= n (w = 2 off the diagonal, 1 on it); padding zero.
__global__ void weighted_packed_density_kernel(const double* __restrict__ D, int nao, long npair, long ld,
                                               double* __restrict__ Dw) {
  long ij = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (ij >= ld) return;
  if (ij >= npair) {
    Dw[ij] = 0.0;
    return;
  }
  int m, n;
  unpack_pair(ij, m, n);
  double w = (m == n) ? 1.0 : 2.0;
  Dw[ij] = w * 0.5 * (D[(size_t)m * nao + n] + D[(size_t)n * nao + m]);
}

// d_P = sum_ij B[P][ij] Dw[ij]; one CTA per row, 128-bit loads.
__global__ void __launch_bounds__(512) jpass1_fp64_kernel(const double* __restrict__ B, long ld,
                                                          const double* __restrict__ Dw, double* __restrict__ d) {
  __shared__ double sh[16];
  const double2* row = reinterpret_cast<const double2*>(B + (size_t)blockIdx.x * ld);
  const double2* dw = reinterpret_cast<const double2*>(Dw);
  long n2 = ld / 2;
  double acc0 = 0.0, acc1 = 0.0;
  long i = threadIdx.x;
  for (; i + 3 * 512 < n2; i += 4 * 512) {
    double2 b0 = __ldcs(row + i), b1 = __ldcs(row + i + 512), b2 = __ldcs(row + i + 1024), b3 = __ldcs(row + i + 1536);
    double2 w0 = dw[i], w1 = dw[i + 512], w2 = dw[i + 1024], w3 = dw[i + 1536];
    acc0 = fma(b0.x, w0.x, acc0); acc1 = fma(b0.y, w0.y, acc1);
    acc0 = fma(b1.x, w1.x, acc0); acc1 = fma(b1.y, w1.y, acc1);
    acc0 = fma(b2.x, w2.x, acc0); acc1 = fma(b2.y, w2.y, acc1);
    acc0 = fma(b3.x, w3.x, acc0); acc1 = fma(b3.y, w3.y, acc1);
  }
  for (; i < n2; i += 512) {
    double2 b0 = __ldcs(row + i), w0 = dw[i];
    acc0 = fma(b0.x, w0.x, acc0); acc1 = fma(b0.y, w0.y, acc1);
  }
  double t = block_sum(acc0 + acc1, sh);
  if (threadIdx.x == 0) d[blockIdx.x] = t;
}

// ---- J in double-float arithmetic -------------------------------------------------------
// FP64 issues at about 0.6e12 FMA/s on this GPU, below the one FMA per 8-byte element that
// J's two passes would need at full HBM speed, so the passes below keep FP64 out of their
// inner loops.  Each FP64 element x of B is split with integer operations into an unevaluated
// pair of floats x = hi + lo: hi holds the sign, exponent and top 23 fraction bits (x
// truncated to 24 significant bits), lo the remaining 29 fraction bits rounded to 24 (so the
// pair is x to 2^-48 relative; |x| below 2^-126 counts as zero).  Products with the density
// (or fitting coefficient) pair (h, l) keep h*hi exactly as p + e (e = fma(h, hi, -p)) and add
// the cross terms h*lo + l*hi to e; sums accumulate as float pairs with Knuth's TwoSum and are
// combined in FP64 once per thread.  The result matches the FP64 passes to ~1e-13 relative.
__device__ __forceinline__ void split_f64_bits(double x, float& hi, float& lo) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned int uh = (unsigned int)(u >> 32), ul = (unsigned int)u;
  const unsigned int sign = uh & 0x80000000u;
  const int e11 = (int)((uh >> 20) & 0x7FFu);
  const int e8 = e11 - 1023 + 127;                  // biased float exponent of x
  const bool normal = e8 > 0 && e8 < 255;
  const unsigned int frac23 = ((uh & 0xFFFFFu) << 3) | (ul >> 29);
  hi = normal ? __uint_as_float(sign | ((unsigned int)e8 << 23) | frac23) : (e11 == 0x7FF ? __int_as_float(0x7fc00000) : 0.0f);
  const int es = e11 - 1075 + 127;                  // biased exponent of 2^(e - 52)
  const float scale = (normal && es > 0) ? __uint_as_float((unsigned int)es << 23) : 0.0f;
  const float r = __uint2float_rn(ul & 0x1FFFFFFFu) * scale;
  lo = __uint_as_float(__float_as_uint(r) | sign);
}

__device__ __forceinline__ void split_f64_arith(double x, float& hi, float& lo) {
  hi = __double2float_rn(x);
  lo = __double2float_rn(x - (double)hi);
}

// (sh, sl) += x * (h + l), x = xh + xl.
__device__ __forceinline__ void df_madd(float xh, float xl, float h, float l, float& sh, float& sl) {
  const float p = xh * h;
  float e = fmaf(xh, h, -p);
  e = fmaf(xh, l, e);
  e = fmaf(xl, h, e);
  const float s = sh + p;
  const float bp = s - sh;
  const float t = (sh - (s - bp)) + (p - bp);
  sl += t + e;
  sh = s;
}

// Dw2[ij] = (hi, lo) of w_mn D_mn (packed, padding zero).
__global__ void weighted_packed_density_df_kernel(const double* __restrict__ D, int nao, long npair, long ld,
                                                  float2* __restrict__ Dw2) {
  long ij = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (ij >= ld) return;
  if (ij >= npair) {
    Dw2[ij] = make_float2(0.0f, 0.0f);
    return;
  }
  int m, n;
  unpack_pair(ij, m, n);
  const double w = (m == n) ? 1.0 : 2.0;
  float h, l;
  split_f64_arith(w * 0.5 * (D[DF_IX((size_t)m * nao + n, (size_t)nao * nao)] + D[DF_IX((size_t)n * nao + m, (size_t)nao * nao)]),
                  h, l);
  Dw2[ij] = make_float2(h, l);
}

// d_P = sum_ij B[P][ij] Dw[ij] for R rows per CTA: every load of the density pair (from L2)
// serves R rows of B (from HBM), so the density is re-read naux / R times instead of naux
// times.  128-bit loads, double-float products, one FP64 block sum per row.
template <int R, int NT>
__global__ void __launch_bounds__(NT) jpass1_df_kernel(const double* __restrict__ B, long ld, int naux,
                                                       const float4* __restrict__ Dw4, double* __restrict__ d) {
  __shared__ double sh[NT / 32];
  const int p0 = blockIdx.x * R;
  const long n2 = ld / 2;
  const double2* rows[R];
#pragma unroll
  for (int r = 0; r < R; ++r)
    rows[r] = reinterpret_cast<const double2*>(B) + DF_IX((size_t)min(p0 + r, naux - 1) * n2, (size_t)naux * n2);
  float ah[R], al[R];
#pragma unroll
  for (int r = 0; r < R; ++r) ah[r] = al[r] = 0.0f;
  long i = threadIdx.x;
  for (; i + NT < n2; i += 2 * NT) {
    const float4 w0 = Dw4[DF_IX(i, n2)], w1 = Dw4[DF_IX(i + NT, n2)];
    double2 b0[R], b1[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      b0[r] = __ldcs(rows[r] + DF_IX(i, n2));
      b1[r] = __ldcs(rows[r] + DF_IX(i + NT, n2));
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float xh, xl, yh, yl;
      split_f64_bits(b0[r].x, xh, xl);
      split_f64_bits(b0[r].y, yh, yl);
      df_madd(xh, xl, w0.x, w0.y, ah[r], al[r]);
      df_madd(yh, yl, w0.z, w0.w, ah[r], al[r]);
      split_f64_bits(b1[r].x, xh, xl);
      split_f64_bits(b1[r].y, yh, yl);
      df_madd(xh, xl, w1.x, w1.y, ah[r], al[r]);
      df_madd(yh, yl, w1.z, w1.w, ah[r], al[r]);
    }
  }
  for (; i < n2; i += NT) {
    const float4 w0 = Dw4[i];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const double2 b0 = __ldcs(rows[r] + i);
      float xh, xl, yh, yl;
      split_f64_bits(b0.x, xh, xl);
      split_f64_bits(b0.y, yh, yl);
      df_madd(xh, xl, w0.x, w0.y, ah[r], al[r]);
      df_madd(yh, yl, w0.z, w0.w, ah[r], al[r]);
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const double t = block_sum((double)ah[r] + (double)al[r], sh);
    if (threadIdx.x == 0 && p0 + r < naux) d[p0 + r] = t;
  }
}

constexpr int JP2_MAX_ROWS = 512;  // largest P slice of pass 2 (shared-memory copy of d)

// Jpart[split][ij] = sum_{P in split} d_P B[P][ij]; one lane per two packed columns,
// double-float products and sums.
__global__ void __launch_bounds__(256) jpass2_df_kernel(const double* __restrict__ B, long ld, int naux, int rows,
                                                        const double* __restrict__ d, double* __restrict__ Jpart) {
  __shared__ float2 sd[JP2_MAX_ROWS];
  const int p0 = blockIdx.y * rows;
  const int np = min(rows, naux - p0);
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    float h, l;
    split_f64_arith(d[p0 + i], h, l);
    sd[i] = make_float2(h, l);
  }
  __syncthreads();
  const long c2 = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c2 * 2 >= ld) return;
  const long st = ld / 2;
  const double2* col = reinterpret_cast<const double2*>(B) + (size_t)p0 * st + c2;
  float xh = 0.0f, xl = 0.0f, yh = 0.0f, yl = 0.0f;
  int p = 0;
  for (; p + 3 < np; p += 4) {
    double2 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      v[u] = __ldcs(col + DF_IX((size_t)(p0 + p + u) * st + c2, (size_t)naux * st) - (size_t)p0 * st - c2);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float2 w = sd[p + u];
      float ah, al, bh, bl;
      split_f64_bits(v[u].x, ah, al);
      split_f64_bits(v[u].y, bh, bl);
      df_madd(ah, al, w.x, w.y, xh, xl);
      df_madd(bh, bl, w.x, w.y, yh, yl);
    }
  }
  for (; p < np; ++p) {
    const double2 v0 = __ldcs(col + (size_t)p * st);
    const float2 w = sd[p];
    float ah, al, bh, bl;
    split_f64_bits(v0.x, ah, al);
    split_f64_bits(v0.y, bh, bl);
    df_madd(ah, al, w.x, w.y, xh, xl);
    df_madd(bh, bl, w.x, w.y, yh, yl);
  }
  reinterpret_cast<double2*>(Jpart)[DF_IX((size_t)blockIdx.y * st + c2, (size_t)gridDim.y * st)] =
      make_double2((double)xh + (double)xl, (double)yh + (double)yl);
}

// Jpart[split][ij] = sum_{P in split} d_P B[P][ij]; one lane per two packed columns.
__global__ void __launch_bounds__(256) jpass2_fp64_kernel(const double* __restrict__ B, long ld, int naux, int rows,
                                                          const double* __restrict__ d, double* __restrict__ Jpart) {
  __shared__ double sd[JP2_MAX_ROWS];
  int p0 = blockIdx.y * rows;
  int np = min(rows, naux - p0);
  for (int i = threadIdx.x; i < np; i += blockDim.x) sd[i] = d[p0 + i];
  __syncthreads();
  long c2 = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c2 * 2 >= ld) return;
  const double2* col = reinterpret_cast<const double2*>(B + (size_t)p0 * ld) + c2;
  long st = ld / 2;
  double ax = 0.0, ay = 0.0, bx = 0.0, by = 0.0;
  int p = 0;
  for (; p + 1 < np; p += 2) {
    double2 v0 = __ldcs(col + (size_t)p * st), v1 = __ldcs(col + (size_t)(p + 1) * st);
    ax = fma(sd[p], v0.x, ax); ay = fma(sd[p], v0.y, ay);
    bx = fma(sd[p + 1], v1.x, bx); by = fma(sd[p + 1], v1.y, by);
  }
  if (p < np) {
    double2 v0 = __ldcs(col + (size_t)p * st);
    ax = fma(sd[p], v0.x, ax); ay = fma(sd[p], v0.y, ay);
  }
  reinterpret_cast<double2*>(Jpart + (size_t)blockIdx.y * ld)[c2] = make_double2(ax + bx, ay + by);
}

// J[m][n] = J[n][m] = sum_split Jpart[split][mn].
__global__ void jreduce_unpack_kernel(const double* __restrict__ Jpart, int nsplit, long ld, int nao,
                                      double* __restrict__ J) {
  long ij = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (ij >= (long)nao * (nao + 1) / 2) return;
  double s = 0.0;
  for (int k = 0; k < nsplit; ++k) s += Jpart[DF_IX((size_t)k * ld + ij, (size_t)nsplit * ld)];
  int m, n;
  unpack_pair(ij, m, n);
  J[DF_IX((size_t)m * nao + n, (size_t)nao * nao)] = s;
  J[DF_IX((size_t)n * nao + m, (size_t)nao * nao)] = s;
}

// ---- FP64 K ---------------------------------------------------------------------------
// X[m][P][i] = sum_n B_P[m][n] C[n][i]; B_P gathered from the packed row.
// CTA tile 64 (m) x 16 CI (i), 256 lanes with 4 x CI outputs each (CI = 2: 32 columns, for
// wide occupied spaces; CI = 1: 16 columns, less padding for small ones; knob
// "fp64_ht_cols").
template <int CI>
__global__ void __launch_bounds__(256) k_halftransform_fp64_kernel(const double* __restrict__ B, long ld, int nao,
                                                                   int naux, const double* __restrict__ C, int nocc,
                                                                   double* __restrict__ X) {
  constexpr int TN = 16 * CI;
  __shared__ double As[16][65];
  __shared__ double Cs[16][TN + 1];
  int P = blockIdx.z;
  int m0 = blockIdx.y * 64, i0 = blockIdx.x * TN;
  const double* row = B + (size_t)P * ld;
  int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // tx -> i (CI each, stride 16), ty -> m (4 each, stride 16)
  double acc[4][CI];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < CI; ++v) acc[u][v] = 0.0;
  for (int n0 = 0; n0 < nao; n0 += 16) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int idx = threadIdx.x + 256 * r;
      int mm = idx >> 4, nn = idx & 15;
      int gm = m0 + mm, gn = n0 + nn;
      double v = 0.0;
      if (gm < nao && gn < nao) {
        int a = max(gm, gn), b = min(gm, gn);
        v = row[DF_IX((size_t)a * (a + 1) / 2 + b, ld)];
      }
      As[nn][mm] = v;
    }
#pragma unroll
    for (int r = 0; r < CI; ++r) {
      int idx = threadIdx.x + 256 * r;
      int nn = idx / TN, ii = idx % TN;
      int gn = n0 + nn, gi = i0 + ii;
      Cs[nn][ii] = (gn < nao && gi < nocc) ? C[DF_IX((size_t)gn * nocc + gi, (size_t)nao * nocc)] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      double a[4], c[CI];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = As[k][ty + 16 * u];
#pragma unroll
      for (int v = 0; v < CI; ++v) c[v] = Cs[k][tx + 16 * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < CI; ++v) acc[u][v] = fma(a[u], c[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    int gm = m0 + ty + 16 * u;
    if (gm >= nao) continue;
#pragma unroll
    for (int v = 0; v < CI; ++v) {
      int gi = i0 + tx + 16 * v;
      if (gi < nocc) X[DF_IX(((size_t)gm * naux + P) * nocc + gi, (size_t)nao * naux * nocc)] = acc[u][v];
    }
  }
}

// K[m][n] = K[n][m] = sum_split Kpart[split][m][n] over the lower triangle m >= n.
__global__ void ksum_mirror_kernel(const double* __restrict__ Kpart, int nsplit, int nao, double* __restrict__ K) {
  long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)nao * nao) return;
  int m = (int)(e / nao), n = (int)(e % nao);
  if (n > m) return;
  double s = 0.0;
  for (int k = 0; k < nsplit; ++k) s += Kpart[DF_IX((size_t)k * nao * nao + e, (size_t)nsplit * nao * nao)];
  K[(size_t)m * nao + n] = s;
  K[(size_t)n * nao + m] = s;
}

int ksplit_count(int nao, long kdim) {
  // enough CTAs for ~4 waves on 152 SMs over the lower-triangle tiles
  long tiles = (long)((nao + 63) / 64) * ((nao + 63) / 64 + 1) / 2;
  long want = (4L * 152 * 4 + tiles - 1) / tiles;
  long maxs = max(1L, kdim / 512);
  int forced = knob("fp64_syrk_split");
  if (forced > 0) return (int)max(1L, min((long)forced, max(1L, kdim / 16)));
  return (int)max(1L, min(want, min(maxs, 64L)));
}

// fp64_k: also carve the FP64 exchange buffers when precision is DF_MIXED (an SCF that
// switches from mixed to FP64 iterations needs both).
JKWork jk_work_layout(int nao, int naux, int nocc, int precision, Arena* a, Sizer* z, bool fp64_k) {
  JKWork w{};
  long ld = B_ld(nao);
  int rows = max(32, min(JP2_MAX_ROWS, knob("jpass2_rows")));
  int nsplit_j = (naux + rows - 1) / rows;
  int nsplit_k = ksplit_count(nao, (long)naux * max(nocc, 1));
  w.nsplit_j = nsplit_j;
  w.nsplit_k = nsplit_k;
#define TAKE(T, ptr, count) \
  if (a) ptr = a->take<T>(count); else z->take<T>(count);
  TAKE(double, w.Dw, ld);
  TAKE(double, w.d, naux);
  TAKE(double, w.Jpart, (size_t)nsplit_j * ld);
  if (precision == DF_FP64 || fp64_k) {
    TAKE(double, w.X, (size_t)nao * naux * max(nocc, 1));
    TAKE(double, w.Kpart, (size_t)nsplit_k * nao * nao);
  }
  if (precision == DF_MIXED) mixed_k_work_layout(nao, naux, nocc, a, z, &w.mk);
#undef TAKE
  return w;
}

int build_J(const void* Bbuf, const BLayout& L, int nao, int naux, int precision, const double* D, double* J,
            const JKWork& w, cudaStream_t s) {
  long npair = npair_of(nao), ld = L.ld;
  const char* base = (const char*)Bbuf;
  const int rows = (naux + w.nsplit_j - 1) / w.nsplit_j;  // P rows per slice of pass 2
  DF_REQUIRE(rows <= JP2_MAX_ROWS, DF_ERR_ARG, "J: %d auxiliary rows per slice exceed %d", rows, JP2_MAX_ROWS);
  unsigned g = (unsigned)((ld + 255) / 256);
  unsigned gp = (unsigned)((npair + 255) / 256);
  (void)precision;  // J streams the FP64 rows in both modes
  const double* B64 = (const double*)(base + L.off64);
  const dim3 grid2((unsigned)((ld / 2 + 255) / 256), (unsigned)w.nsplit_j);
  if (knob("j_fp64_fma") == 0) {
    // double-float passes (the Dw buffer holds ld float pairs: the same bytes as ld doubles)
    weighted_packed_density_df_kernel<<<g, 256, 0, s>>>(D, nao, npair, ld, (float2*)w.Dw);
    DF_LAUNCHED("weighted_packed_density_df_kernel");
    {
      ProfScope ps("j_pass1", s);
      // rows per CTA: each density load from L2 serves R rows of B (knob "jpass1_rows")
      const int R = knob("jpass1_rows");
      const float4* Dw4 = (const float4*)w.Dw;
      if (R >= 8)
        jpass1_df_kernel<8, 512><<<(unsigned)((naux + 7) / 8), 512, 0, s>>>(B64, ld, naux, Dw4, w.d);
      else if (R >= 4)
        jpass1_df_kernel<4, 256><<<(unsigned)((naux + 3) / 4), 256, 0, s>>>(B64, ld, naux, Dw4, w.d);
      else if (R >= 2)
        jpass1_df_kernel<2, 256><<<(unsigned)((naux + 1) / 2), 256, 0, s>>>(B64, ld, naux, Dw4, w.d);
      else
        jpass1_df_kernel<1, 512><<<(unsigned)naux, 512, 0, s>>>(B64, ld, naux, Dw4, w.d);
      DF_LAUNCHED("jpass1_df_kernel");
    }
    {
      ProfScope ps("j_pass2", s);
      jpass2_df_kernel<<<grid2, 256, 0, s>>>(B64, ld, naux, rows, w.d, w.Jpart);
      DF_LAUNCHED("jpass2_df_kernel");
    }
  } else {
    weighted_packed_density_kernel<<<g, 256, 0, s>>>(D, nao, npair, ld, w.Dw);
    DF_LAUNCHED("weighted_packed_density_kernel");
    {
      ProfScope ps("j_pass1", s);
      jpass1_fp64_kernel<<<naux, 512, 0, s>>>(B64, ld, w.Dw, w.d);
      DF_LAUNCHED("jpass1_fp64_kernel");
    }
    {
      ProfScope ps("j_pass2", s);
      jpass2_fp64_kernel<<<grid2, 256, 0, s>>>(B64, ld, naux, rows, w.d, w.Jpart);
      DF_LAUNCHED("jpass2_fp64_kernel");
    }
  }
  jreduce_unpack_kernel<<<gp, 256, 0, s>>>(w.Jpart, w.nsplit_j, ld, nao, J);
  DF_LAUNCHED("jreduce_unpack_kernel");
  return DF_OK;
}

int build_K_fp64(const double* B64, long ld, int nao, int naux, const double* C, int nocc, double* K, const JKWork& w,
                 cudaStream_t s) {
  {
    ProfScope ps("k_halftransform_fp64", s);
    const int forced = knob("fp64_ht_cols");
    const int cols = forced == 16 || forced == 32 ? forced : (nocc <= 16 ? 16 : 32);
    if (cols == 16) {
      dim3 grid((nocc + 15) / 16, (nao + 63) / 64, naux);
      k_halftransform_fp64_kernel<1><<<grid, 256, 0, s>>>(B64, ld, nao, naux, C, nocc, w.X);
    } else {
      dim3 grid((nocc + 31) / 32, (nao + 63) / 64, naux);
      k_halftransform_fp64_kernel<2><<<grid, 256, 0, s>>>(B64, ld, nao, naux, C, nocc, w.X);
    }
    DF_LAUNCHED("k_halftransform_fp64_kernel");
  }
  long kdim = (long)naux * nocc;
  long kchunk = (kdim + w.nsplit_k - 1) / w.nsplit_k;
  kchunk = (kchunk + 15) / 16 * 16;
  int nsplit = (int)((kdim + kchunk - 1) / kchunk);
  {
    ProfScope ps("k_syrk_fp64", s);
    DF_TRY(dgemm(false, true, nao, nao, (int)kdim, 1.0, w.X, kdim, 0, w.X, kdim, 0, 0.0, w.Kpart, nao,
                 (long)nao * nao, nsplit, s, kchunk, 1));
  }
  long nn = (long)nao * nao;
  ksum_mirror_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(w.Kpart, nsplit, nao, K);
  DF_LAUNCHED("ksum_mirror_kernel");
  return DF_OK;
}

int run_jk(const void* B, int nao, int naux, int precision, const double* D, const double* C, int nocc, double* J,
           double* K, const JKWork& w, cudaStream_t s) {
  BLayout L = B_layout(nao, naux, precision, w.mk.planes);
  if (precision == DF_MIXED && K) {
    const int built = recorded_B_planes(B);
    DF_REQUIRE(built < 0 || built >= w.mk.planes, DF_ERR_ARG,
               "mixed exchange with %d BF16 planes on a B built with %d (set the knob mixed_planes before sizing "
               "and building B, and keep it while B is used)", w.mk.planes, built);
  }
  if (J) DF_TRY(build_J(B, L, nao, naux, precision, D, J, w, s));
  if (K) {
    if (precision == DF_FP64) {
      DF_REQUIRE(w.X && w.Kpart, DF_ERR_ARG, "FP64 exchange requested with a workspace laid out for mixed precision");
      DF_TRY(build_K_fp64((const double*)((const char*)B + L.off64), L.ld, nao, naux, C, nocc, K, w, s));
    } else {
      DF_REQUIRE(w.mk.Xp[0] && w.mk.Kpart, DF_ERR_ARG, "mixed exchange requested with a workspace laid out for FP64");
      DF_TRY(build_K_mixed(B, L, nao, naux, C, nocc, K, w.mk, s));
    }
  }
  return DF_OK;
}

int build_B(const double* ao_xyz, const double* ao_exp, int nao, const double* aux_xyz, const double* aux_exp,
            int naux, const double* Lfac, int precision, void* Bbuf, double* pair_tab, cudaStream_t s) {
  BLayout L = B_layout(nao, naux, precision, mixed_planes());
  double* B64 = (double*)((char*)Bbuf + L.off64);
  DF_TRY(launch_int3c(ao_xyz, ao_exp, nao, aux_xyz, aux_exp, naux, B64, L.ld, pair_tab, s));
  DF_TRY(forward_substitution(B64, L.ld, L.ld, Lfac, naux, s));
  if (precision == DF_MIXED) {
    DF_REQUIRE(naux <= 65535, DF_ERR_ARG, "naux too large");
    PlaneOut po{};
    po.planes = L.planes;
    for (int j = 0; j < L.planes; ++j) po.p[j] = (__nv_bfloat16*)((char*)Bbuf + L.offp[j]);
    record_B_planes(Bbuf, L.planes);
    b_to_planes_kernel<<<dim3((unsigned)L.npad, (unsigned)naux), 128, 0, s>>>(B64, L.ld, nao, L.npad, po);
    DF_LAUNCHED("b_to_planes_kernel");
  }
  return DF_OK;
}

}  // namespace dfscf

using namespace dfscf;

extern "C" long df_B_ld(int nao) { return nao > 0 ? B_ld(nao) : 0; }
extern "C" int df_nao_pad(int nao) { return nao > 0 ? nao_pad(nao) : 0; }

extern "C" size_t df_B_bytes(int nao, int naux, int precision) {
  if (nao <= 0 || naux <= 0 || (precision != DF_FP64 && precision != DF_MIXED)) return 0;
  return B_layout(nao, naux, precision, mixed_planes()).bytes;
}

extern "C" size_t df_build_B_work_bytes(int nao, int naux) {
  (void)naux;
  return nao > 0 ? align_up(sizeof(double) * 5 * (size_t)npair_of(nao), 256) : 0;
}

extern "C" int df_build_B(const double* ao_xyz, const double* ao_exp, int nao, const double* aux_xyz,
                          const double* aux_exp, int naux, const double* L, int precision, void* B, size_t B_bytes,
                          void* work, size_t work_bytes, cudaStream_t s) {
  clear_error();
  DF_REQUIRE(nao > 0 && naux > 0, DF_ERR_ARG, "df_build_B: bad sizes nao=%d naux=%d", nao, naux);
  DF_REQUIRE(precision == DF_FP64 || precision == DF_MIXED, DF_ERR_ARG, "df_build_B: bad precision %d", precision);
  DF_REQUIRE(ao_xyz && ao_exp && aux_xyz && aux_exp && L && B, DF_ERR_ARG, "df_build_B: null pointer");
  DF_REQUIRE(B_bytes >= df_B_bytes(nao, naux, precision), DF_ERR_NOMEM, "df_build_B: B buffer of %zu bytes < %zu",
             B_bytes, df_B_bytes(nao, naux, precision));
  DF_REQUIRE(work && work_bytes >= df_build_B_work_bytes(nao, naux), DF_ERR_NOMEM,
             "df_build_B: workspace of %zu bytes < %zu", work_bytes, df_build_B_work_bytes(nao, naux));
  DF_REQUIRE(precision == DF_FP64 || naux <= 65535, DF_ERR_ARG, "df_build_B: naux > 65535 in mixed mode");
  return build_B(ao_xyz, ao_exp, nao, aux_xyz, aux_exp, naux, L, precision, B, (double*)work, s);
}

extern "C" int df_B_get_packed(const void* B, int nao, int naux, int P, double* row, cudaStream_t s) {
  clear_error();
  DF_REQUIRE(B && row && nao > 0 && P >= 0 && P < naux, DF_ERR_ARG, "df_B_get_packed: bad arguments");
  long ld = B_ld(nao);
  DF_CUDA(cudaMemcpyAsync(row, (const double*)B + (size_t)P * ld, sizeof(double) * npair_of(nao),
                          cudaMemcpyDeviceToDevice, s));
  return DF_OK;
}

extern "C" size_t df_jk_work_bytes(int nao, int naux, int nocc, int precision) {
  if (nao <= 0 || naux <= 0 || nocc < 0) return 0;
  Sizer z;
  jk_work_layout(nao, naux, nocc, precision, nullptr, &z, false);
  return z.used;
}

extern "C" int df_jk(const void* B, int nao, int naux, int precision, const double* D, const double* C, int nocc,
                     double* J, double* K, void* work, size_t work_bytes, cudaStream_t s) {
  clear_error();
  DF_REQUIRE(B && nao > 0 && naux > 0, DF_ERR_ARG, "df_jk: bad B or sizes");
  DF_REQUIRE(precision == DF_FP64 || precision == DF_MIXED, DF_ERR_ARG, "df_jk: bad precision %d", precision);
  DF_REQUIRE(!J || D, DF_ERR_ARG, "df_jk: J requested without D");
  DF_REQUIRE(!K || (C && nocc > 0), DF_ERR_ARG, "df_jk: K requested without C / nocc");
  DF_REQUIRE(naux <= 65535, DF_ERR_ARG, "df_jk: naux > 65535");
  size_t need = df_jk_work_bytes(nao, naux, nocc, precision);
  DF_REQUIRE(work && work_bytes >= need, DF_ERR_NOMEM, "df_jk: workspace of %zu bytes < %zu", work_bytes, need);
  Arena a(work, work_bytes);
  JKWork w = jk_work_layout(nao, naux, nocc, precision, &a, nullptr, false);
  DF_REQUIRE(!a.overflow, DF_ERR_NOMEM, "df_jk: workspace overflow");
  DF_TRY(run_jk(B, nao, naux, precision, D, C, nocc, J, K, w, s));
  if (K && precision == DF_MIXED) {
    // The tensor-core kernels flag a bounded wait that gave up (K is then NaN).  Outside a
    // stream capture the flag is read back here, which synchronises the stream.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    DF_CUDA(cudaStreamIsCapturing(s, &cs));
    if (cs == cudaStreamCaptureStatusNone) {
      int err = 0;
      DF_CUDA(cudaMemcpyAsync(&err, w.mk.err, sizeof(int), cudaMemcpyDeviceToHost, s));
      DF_CUDA(cudaStreamSynchronize(s));
      DF_REQUIRE(err == 0, DF_ERR_TIMEOUT, "df_jk: a bounded wait of the tensor-core exchange gave up; K is NaN");
    }
  }
  return DF_OK;
}

DF_BOUNDS_READER(bounds_read_jk)
