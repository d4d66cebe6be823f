// Learned initial guess: geometry -> per-centre-pair 5x5 density blocks -> dm0.
//
// The paper allows any starting density for a mean-field calculation, idempotent or not
// and with any electron count (arXiv 2506.06661, Section "Initial Guess for Mean-field
// Methods").  This file produces such a density from geometry with a small network that
// is trained on densities the SCF itself converges:
//   features  32 Gaussian radial-basis values exp(-gamma (R - r_k)^2), r_k = 12 k / 31,
//             gamma = (31/12)^2, plus the environment env_A = 1/8 sum_{C != A, R <= 12}
//             rbf(R_AC):  off-diagonal pair (A > B): [rbf(R_AB), env_A + env_B, 0],
//             diagonal pair (A, A): [0, 2 env_A, 1]; pairs beyond 12 bohr are masked out;
//   network   65 -> 256 -> 256 -> 256 -> 15 with SiLU on the hidden layers; the 15 outputs
//             are the upper triangle (a <= b, row-major) of a symmetric 5x5 block;
//   training  mean squared error against the symmetrised converged blocks, Adam, FP32
//             weights and FP32 arithmetic on CUDA cores;
//   inference the same network with BF16 weights and activations and FP32 accumulation, on
//             the tensor cores (tcgen05, one CTA per 128 pairs, below).
// Parameters are one float array: for each layer, W [out][in] then b [out].
#include <cuda_bf16.h>

#include <cstdint>
#include <cstring>

#include "common.cuh"
#include "kernels.cuh"
#include "tcgen05.cuh"

namespace dfscf {
namespace mlp {

constexpr int NRBF = 32, NIN = 65, NHID = 256, NOUT = 15, NBF = 5;
constexpr float RCUT = 12.0f;
constexpr int NLAYER = 4;
__host__ __device__ constexpr int layer_in(int l) { return l == 0 ? NIN : NHID; }
__host__ __device__ constexpr int layer_out(int l) { return l == NLAYER - 1 ? NOUT : NHID; }
__host__ __device__ constexpr size_t w_offset(int l) {
  size_t o = 0;
  for (int k = 0; k < l; ++k) o += (size_t)layer_in(k) * layer_out(k) + layer_out(k);
  return o;
}
__host__ __device__ constexpr size_t b_offset(int l) { return w_offset(l) + (size_t)layer_in(l) * layer_out(l); }
constexpr size_t NPARAM = w_offset(NLAYER);

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }
template <typename T> __device__ __forceinline__ T from_f(float x);
template <> __device__ __forceinline__ float from_f<float>(float x) { return x; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

__device__ __forceinline__ float rbf(float r, int k) {
  const float dr = RCUT / (NRBF - 1);
  float x = (r - dr * k) / dr;
  return __expf(-x * x);
}

// ---- SIMT GEMM with FP32 accumulation ---------------------------------------------------------
// C[M][N] = alpha * op(A) op(B) + beta * C;  op(A)(m,k) = TA ? A[k*lda+m] : A[m*lda+k];
// op(B)(k,n) = TB ? B[n*ldb+k] : B[k*ldb+n].  64x64 tiles, 256 lanes with 4x4 outputs.
template <bool TA, bool TB, typename T>
__global__ void __launch_bounds__(256) sgemm_kernel(int M, int N, int K, float alpha, const T* __restrict__ A, int lda,
                                                    const T* __restrict__ B, int ldb, float beta, float* __restrict__ C,
                                                    int ldc) {
  __shared__ float As[16][65];
  __shared__ float Bs[16][65];
  int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int idx = threadIdx.x + 256 * r;
      int mm, kk;
      if (TA) { kk = idx >> 6; mm = idx & 63; } else { mm = idx >> 4; kk = idx & 15; }
      int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < K) ? to_f(TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk]) : 0.f;
      int nn;
      if (TB) { nn = idx >> 4; kk = idx & 15; } else { kk = idx >> 6; nn = idx & 63; }
      int gn = n0 + nn;
      gk = k0 + kk;
      Bs[kk][nn] = (gn < N && gk < K) ? to_f(TB ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn]) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
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
      float* c = C + (size_t)gm * ldc + gn;
      *c = beta == 0.f ? alpha * acc[i][j] : fmaf(alpha, acc[i][j], beta * *c);
    }
  }
}

template <bool TA, bool TB, typename T>
static int sgemm(int M, int N, int K, float alpha, const T* A, int lda, const T* B, int ldb, float beta, float* C,
                 int ldc, cudaStream_t s) {
  if (M <= 0 || N <= 0) return DF_OK;
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  DF_REQUIRE(grid.y <= 65535, DF_ERR_ARG, "mlp: batch too large for one GEMM (%d rows)", M);
  sgemm_kernel<TA, TB, T><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  DF_LAUNCHED("sgemm_kernel");
  return DF_OK;
}

// Z += b (broadcast over rows), H = act(Z) in type T (SiLU when act != 0).
template <typename T>
__global__ void bias_act_kernel(float* __restrict__ Z, const float* __restrict__ b, int rows, int cols, int act,
                                T* __restrict__ H) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)rows * cols) return;
  float z = Z[i] + b[i % cols];
  Z[i] = z;
  float h = act ? z / (1.f + __expf(-z)) : z;
  H[i] = from_f<T>(h);
}

// G = 2 (out - Y) mask / (nvalid * 15); loss partial sums atomically into loss[0].
__global__ void mse_grad_kernel(const float* __restrict__ out, const float* __restrict__ Y,
                                const float* __restrict__ mask, int n, float inv_count, float* __restrict__ G,
                                float* __restrict__ loss) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (i < (long)n * NOUT) {
    float m = mask ? mask[i / NOUT] : 1.f;
    float d = (out[i] - Y[i]) * m;
    G[i] = 2.f * d * inv_count;
    l = d * d * inv_count;
  }
  l = warp_sumf(l);
  if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, l);
}

// dZ = dA * silu'(Z), silu'(z) = s (1 + z (1 - s)), s = sigmoid(z).
__global__ void silu_backward_kernel(const float* __restrict__ Z, float* __restrict__ dA, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float z = Z[i];
  float s = 1.f / (1.f + __expf(-z));
  dA[i] *= s * (1.f + z * (1.f - s));
}

// db[c] = sum_r G[r][c]
__global__ void column_sum_kernel(const float* __restrict__ G, int rows, int cols, float* __restrict__ db) {
  int c = blockIdx.x;
  float s = 0.f;
  for (int r = threadIdx.x; r < rows; r += blockDim.x) s += G[(size_t)r * cols + c];
  s = warp_sumf(s);
  __shared__ float sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
    db[c] = t;
  }
}

// Adam (Kingma & Ba): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long n, float lr, float b1, float b2, float eps, float c1, float c2) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = g[i];
  float mi = b1 * m[i] + (1.f - b1) * gi;
  float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ---- features, targets, density ------------------------------------------------------------
// env[A][k] = 1/8 sum_{C != A, R_AC <= 12} rbf_k(R_AC)
__global__ void env_kernel(const double* __restrict__ xyz, int natm, float* __restrict__ env) {
  int a = blockIdx.x;
  int k = threadIdx.x;  // 32 lanes, one radial function each
  if (k >= NRBF) return;
  float s = 0.f;
  for (int c = 0; c < natm; ++c) {
    if (c == a) continue;
    double dx = xyz[3 * a] - xyz[3 * c], dy = xyz[3 * a + 1] - xyz[3 * c + 1], dz = xyz[3 * a + 2] - xyz[3 * c + 2];
    float r = (float)sqrt(dx * dx + dy * dy + dz * dz);
    if (r <= RCUT) s += rbf(r, k);
  }
  env[a * NRBF + k] = s * 0.125f;
}

// Pair p = A(A+1)/2 + B (A >= B): features [p][65] and mask [p] (0 beyond the cutoff).
template <typename T>
__global__ void pair_feature_kernel(const double* __restrict__ xyz, int natm, const float* __restrict__ env,
                                    T* __restrict__ feat, float* __restrict__ mask) {
  long p = blockIdx.x;
  int k = threadIdx.x;  // 65 lanes
  int A, B;
  unpack_pair(p, A, B);
  double dx = xyz[3 * A] - xyz[3 * B], dy = xyz[3 * A + 1] - xyz[3 * B + 1], dz = xyz[3 * A + 2] - xyz[3 * B + 2];
  float r = (float)sqrt(dx * dx + dy * dy + dz * dz);
  bool diag = A == B;
  float v = 0.f;
  if (k < NRBF) v = diag ? 0.f : rbf(r, k);
  else if (k < 2 * NRBF) v = diag ? 2.f * env[A * NRBF + k - NRBF] : env[A * NRBF + k - NRBF] + env[B * NRBF + k - NRBF];
  else if (k == 2 * NRBF) v = diag ? 1.f : 0.f;
  if (k < NIN) feat[p * NIN + k] = from_f<T>(v);
  if (k == 0) mask[p] = (diag || r <= RCUT) ? 1.f : 0.f;
}

// Y[p][t] = entries (a <= b) of the symmetrised block 1/2 (D_AB + D_AB^T).
__global__ void block_targets_kernel(const double* __restrict__ D, int natm, float* __restrict__ Y) {
  long p = blockIdx.x;
  int t = threadIdx.x;
  if (t >= NOUT) return;
  int A, B;
  unpack_pair(p, A, B);
  int a = 0, b = 0, q = t;
  for (a = 0; a < NBF; ++a) {
    int len = NBF - a;
    if (q < len) {
      b = a + q;
      break;
    }
    q -= len;
  }
  int nao = NBF * natm;
  double x = 0.5 * (D[(size_t)(NBF * A + a) * nao + NBF * B + b] + D[(size_t)(NBF * A + b) * nao + NBF * B + a]);
  Y[p * NOUT + t] = (float)x;
}

// dm0 from predicted blocks (masked pairs stay zero).  D must be zeroed beforehand.
__global__ void assemble_density_kernel(const float* __restrict__ out, const float* __restrict__ mask, int natm,
                                        double* __restrict__ D) {
  long p = blockIdx.x;
  int t = threadIdx.x;
  if (t >= NOUT || mask[p] == 0.f) return;
  int A, B;
  unpack_pair(p, A, B);
  int a = 0, b = 0, q = t;
  for (a = 0; a < NBF; ++a) {
    int len = NBF - a;
    if (q < len) {
      b = a + q;
      break;
    }
    q -= len;
  }
  int nao = NBF * natm;
  double v = out[p * NOUT + t];
  D[(size_t)(NBF * A + a) * nao + NBF * B + b] = v;
  D[(size_t)(NBF * A + b) * nao + NBF * B + a] = v;
  D[(size_t)(NBF * B + b) * nao + NBF * A + a] = v;
  D[(size_t)(NBF * B + a) * nao + NBF * A + b] = v;
}

// Factor that brings tr(Dt) to nelec (one block); a non-positive trace gives 1 and the
// validity gate then rejects the guess.
__global__ void trace_scale_kernel(const double* __restrict__ D, int nao, int nelec, double* __restrict__ scale) {
  __shared__ double sh[32];
  double t = 0.0;
  for (int i = threadIdx.x; i < nao; i += blockDim.x) t += D[(size_t)i * nao + i];
  t = block_sum(t, sh);
  if (threadIdx.x == 0) *scale = t > 0.0 ? (double)nelec / t : 1.0;
}

__global__ void scale_kernel(double* __restrict__ D, size_t n, const double* __restrict__ scale) {
  const double c = *scale;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) D[k] *= c;
}

// ---- workspace -------------------------------------------------------------------------------
struct Work {
  float* Z[NLAYER];   // pre-activations
  float* H[NLAYER];   // activations (H[3] = output)
  float* G;           // gradient of the current layer's pre-activation
  float* dA;          // gradient w.r.t. the previous activation
  float* grad;        // parameter gradient (NPARAM)
  float* loss;
  __nv_bfloat16* Wp;  // BF16 weights of the tensor-core inference, zero-padded per layer
  int* err;           // bounded wait of the inference kernel gave up
};

static void layout(int n, Arena* a, Sizer* z, Work* w) {
#define TAKE(T, ptr, count) \
  if (a) ptr = a->take<T>(count); else z->take<T>(count);
  for (int l = 0; l < NLAYER; ++l) {
    TAKE(float, w->Z[l], (size_t)n * layer_out(l));
    TAKE(float, w->H[l], (size_t)n * layer_out(l));
  }
  TAKE(float, w->G, (size_t)n * NHID);
  TAKE(float, w->dA, (size_t)n * NHID);
  TAKE(float, w->grad, NPARAM);
  TAKE(float, w->loss, 1);
  TAKE(__nv_bfloat16, w->Wp, (size_t)(2 * NHID * NHID + 128 * NHID + 16 * NHID));
  TAKE(int, w->err, 1);
#undef TAKE
}

// Inference only (forward_bf16): the output H[3], the packed BF16 weights and the error flag.
static void layout_infer(int n, Arena* a, Sizer* z, Work* w) {
#define TAKE(T, ptr, count) \
  if (a) ptr = a->take<T>(count); else z->take<T>(count);
  TAKE(float, w->H[NLAYER - 1], (size_t)n * NOUT);
  TAKE(__nv_bfloat16, w->Wp, (size_t)(2 * NHID * NHID + 128 * NHID + 16 * NHID));
  TAKE(int, w->err, 1);
#undef TAKE
}

static unsigned nb(long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// FP32 forward: H[3] = network(X).
static int forward_fp32(const float* P, const float* X, int n, Work& w, cudaStream_t s) {
  const float* in = X;
  for (int l = 0; l < NLAYER; ++l) {
    int fi = layer_in(l), fo = layer_out(l);
    DF_TRY((sgemm<false, true, float>(n, fo, fi, 1.f, in, fi, P + w_offset(l), fi, 0.f, w.Z[l], fo, s)));
    bias_act_kernel<float><<<nb((long)n * fo), 256, 0, s>>>(w.Z[l], P + b_offset(l), n, fo, l < NLAYER - 1, w.H[l]);
    DF_LAUNCHED("bias_act_kernel");
    in = w.H[l];
  }
  return DF_OK;
}

// ---- BF16 inference on the tensor cores (tcgen05) ---------------------------------------------
// One CTA runs the whole network for 128 pair rows: the activations of a layer stay in shared
// memory as the A operand of the next (BF16, K-major, 128-byte swizzle: row r's 16-byte unit u of
// a 64-element K chunk sits at unit u ^ (r mod 8)), each layer's BF16 weights [out][in] arrive by
// TMA as the B operand, and one thread issues M = 128, N = 256 (16 for the output layer), K = 16
// MMAs into an FP32 accumulator in TMEM; the four warps read it back row by row, add the bias
// and apply SiLU in FP32, and store the BF16 activation (or the FP32 output).  Layer 0's K is
// padded from 65 to 128 and the output layer's N from 15 to 16 with zeros.
namespace tc {

constexpr int THREADS = 128;
constexpr int KPAD0 = 128, NOUTP = 16;
__host__ __device__ constexpr int kpad(int l) { return l == 0 ? KPAD0 : NHID; }
__host__ __device__ constexpr int npad(int l) { return l == NLAYER - 1 ? NOUTP : NHID; }
__host__ __device__ constexpr size_t wp_offset(int l) {
  size_t o = 0;
  for (int k = 0; k < l; ++k) o += (size_t)kpad(k) * npad(k);
  return o;
}
constexpr size_t WP_COUNT = wp_offset(NLAYER);
static_assert(WP_COUNT == 2 * NHID * NHID + 128 * NHID + 16 * NHID, "workspace of the packed weights");
constexpr uint32_t A_CHUNK = 128 * 64 * 2;       // 128 rows x 64 bf16
constexpr uint32_t A_BYTES = 4 * A_CHUNK;        // K up to 256
constexpr uint32_t W_BYTES = NHID * NHID * 2;    // largest layer
constexpr size_t SMEM = A_BYTES + W_BYTES + 1024;

struct Maps {
  CUtensorMap w[NLAYER];
};

// BF16 copies of the weights, zero-padded to [npad(l)][kpad(l)].
__global__ void pack_weights_kernel(const float* __restrict__ P, __nv_bfloat16* __restrict__ Wp) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)WP_COUNT) return;
  int l = 0;
  while (l + 1 < NLAYER && (size_t)i >= wp_offset(l + 1)) ++l;
  const long j = i - (long)wp_offset(l);
  const int o = (int)(j / kpad(l)), k = (int)(j % kpad(l));
  const float v = (o < layer_out(l) && k < layer_in(l)) ? P[w_offset(l) + (size_t)o * layer_in(l) + k] : 0.f;
  Wp[i] = __float2bfloat16_rn(v);
}

// Store 8 consecutive BF16 values of row r, K elements k0 .. k0 + 7 (k0 a multiple of 8), into
// the swizzled A operand.
__device__ __forceinline__ void store_a8(uint8_t* A, int r, int k0, const float* v) {
  __align__(16) __nv_bfloat16 h[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) h[e] = __float2bfloat16_rn(v[e]);
  const int c = k0 >> 6, u = (k0 & 63) >> 3;
  *reinterpret_cast<uint4*>(A + (size_t)c * A_CHUNK + (size_t)r * 128 + (size_t)((u ^ (r & 7)) << 4)) =
      *reinterpret_cast<const uint4*>(h);
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__global__ void __launch_bounds__(THREADS, 1) mlp_forward_kernel(const __grid_constant__ Maps maps,
                                                                 const float* __restrict__ X, int n,
                                                                 const float* __restrict__ P, float* __restrict__ out,
                                                                 int* __restrict__ err) {
  using namespace umma;
  extern __shared__ uint8_t dyn_smem[];
  __shared__ uint64_t wbar, mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  uint32_t base = smem_u32(dyn_smem);
  uint8_t* A = dyn_smem + ((1024u - (base & 1023u)) & 1023u);
  uint8_t* W = A + A_BYTES;
  const int r = threadIdx.x, warp = r >> 5;
  const long g = (long)blockIdx.x * 128 + r;
  if (r == 0) {
    mbar_init(&wbar, 1);
    mbar_init(&mbar, 1);
    abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == 0) {
    __syncwarp();  // lane 0 initialised the barriers above: the allocation is warp-collective
    tmem_alloc(&tmem_base, NHID);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  auto load_weights = [&](int l) {
    mbar_arrive_expect_tx(&wbar, (uint32_t)(kpad(l) * npad(l) * 2));
    for (int c = 0; c < kpad(l) / 64; ++c) tma_load_2d(W + (size_t)c * npad(l) * 128, &maps.w[l], &wbar, c * 64, 0);
  };
  if (r == 0) load_weights(0);
  // layer 0's A operand: the features of this CTA's rows (zero past n and past 65)
  for (int k0 = 0; k0 < KPAD0; k0 += 8) {
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = (g < n && k0 + e < NIN) ? X[g * NIN + k0 + e] : 0.f;
    store_a8(A, r, k0, v);
  }
  fence_async_smem();
  __syncthreads();
  int loads = 1;
  bool ok = true;
  for (int l = 0; l < NLAYER && ok; ++l) {
    const uint32_t ph = (uint32_t)l & 1u;
    if (r == 0) {
      if (!mbar_wait(&wbar, ph, &abort_flag)) {
        abort_flag = 1;
      } else {
        tc_fence_after();
        const uint32_t idesc = idesc_bf16(128, npad(l));
        const uint32_t sa = smem_u32(A), sw = smem_u32(W);
        for (int c = 0; c < kpad(l) / 64; ++c)
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t off = (uint64_t)(kk * 32) >> 4;
            umma_bf16(tmem, desc_sw<64>(sa + c * A_CHUNK) + off, desc_sw<64>(sw + (uint32_t)(c * npad(l) * 128)) + off,
                      idesc, (c > 0 || kk > 0) ? 1u : 0u);
          }
        umma_commit(&mbar);
      }
    }
    __syncthreads();
    if (!abort_flag && !mbar_wait(&mbar, ph, &abort_flag)) abort_flag = 1;
    tc_fence_after();
    __syncthreads();  // every thread has seen the MMAs complete (or the abort): W and A may be overwritten
    if (abort_flag) {  // the same shared value for every thread after the barrier
      ok = false;
      break;
    }
    if (r == 0 && l + 1 < NLAYER) {
      load_weights(l + 1);
      loads++;
    }
    const float* bias = P + b_offset(l);
    for (int c0 = 0; c0 < npad(l); c0 += 16) {
      uint32_t v[16];
      tmem_ld_x16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      tmem_wait_ld();
      float h[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int col = c0 + j;
        const float z = __uint_as_float(v[j]) + (col < layer_out(l) ? bias[col] : 0.f);
        h[j] = l + 1 < NLAYER ? z / (1.f + __expf(-z)) : z;
      }
      if (l + 1 < NLAYER) {
        store_a8(A, r, c0, h);
        store_a8(A, r, c0 + 8, h + 8);
      } else if (g < n) {
#pragma unroll
        for (int j = 0; j < NOUT; ++j) out[g * NOUT + j] = h[j];
      }
    }
    tc_fence_before();
    fence_async_smem();
    __syncthreads();
  }
  if (!ok) {  // no result: NaN rows, the flag, and the weights still in flight
    if (g < n)
      for (int j = 0; j < NOUT; ++j) out[g * NOUT + j] = __int_as_float(0x7fc00000);
    if (r == 0) {
      atomicExch(err, 1);
      mbar_wait(&wbar, (uint32_t)(loads - 1) & 1u, nullptr);  // completes the last armed phase
    }
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, NHID);
  }
}

}  // namespace tc

// BF16 inference on the tensor cores: output in H[3] (FP32, n x 15).
static int forward_bf16(const float* P, const float* X, int n, Work& w, cudaStream_t s) {
  tc::pack_weights_kernel<<<nb((long)tc::WP_COUNT), 256, 0, s>>>(P, w.Wp);
  DF_LAUNCHED("pack_weights_kernel");
  tc::Maps maps;
  for (int l = 0; l < NLAYER; ++l)
    DF_TRY(make_map(&maps.w[l], w.Wp + tc::wp_offset(l), tc::kpad(l), tc::npad(l), tc::kpad(l), tc::npad(l), 64));
  static bool attr = false;
  if (!attr) {
    DF_CUDA(cudaFuncSetAttribute(tc::mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::SMEM));
    attr = true;
  }
  DF_CUDA(cudaMemsetAsync(w.err, 0, sizeof(int), s));
  tc::mlp_forward_kernel<<<(unsigned)((n + 127) / 128), tc::THREADS, tc::SMEM, s>>>(maps, X, n, P, w.H[NLAYER - 1],
                                                                                  w.err);
  DF_LAUNCHED("mlp_forward_kernel");
  return DF_OK;
}

// Loss and full parameter gradient (into w.grad) for a batch; loss accumulated into w.loss.
static int loss_grad(const float* P, const float* X, const float* Y, const float* mask, int n, float nvalid, Work& w,
                     cudaStream_t s) {
  DF_TRY(forward_fp32(P, X, n, w, s));
  DF_CUDA(cudaMemsetAsync(w.loss, 0, sizeof(float), s));
  float inv = 1.f / (fmaxf(nvalid, 1.f) * NOUT);
  mse_grad_kernel<<<nb((long)n * NOUT), 256, 0, s>>>(w.H[NLAYER - 1], Y, mask, n, inv, w.G, w.loss);
  DF_LAUNCHED("mse_grad_kernel");
  for (int l = NLAYER - 1; l >= 0; --l) {
    int fi = layer_in(l), fo = layer_out(l);
    const float* Ain = l == 0 ? X : w.H[l - 1];
    // dW = G^T A_in  [fo][fi];  db = column sums of G
    DF_TRY((sgemm<true, false, float>(fo, fi, n, 1.f, w.G, fo, Ain, fi, 0.f, w.grad + w_offset(l), fi, s)));
    column_sum_kernel<<<fo, 256, 0, s>>>(w.G, n, fo, w.grad + b_offset(l));
    DF_LAUNCHED("column_sum_kernel");
    if (l == 0) break;
    // dA = G W  [n][fi]; then G = dA * silu'(Z_{l-1})
    DF_TRY((sgemm<false, false, float>(n, fi, fo, 1.f, w.G, fo, P + w_offset(l), fi, 0.f, w.dA, fi, s)));
    silu_backward_kernel<<<nb((long)n * fi), 256, 0, s>>>(w.Z[l - 1], w.dA, (long)n * fi);
    DF_LAUNCHED("silu_backward_kernel");
    std::swap(w.G, w.dA);
  }
  return DF_OK;
}

}  // namespace mlp
}  // namespace dfscf

using namespace dfscf;
using namespace dfscf::mlp;

extern "C" size_t guess_mlp_param_count(void) { return NPARAM; }

extern "C" size_t guess_mlp_work_bytes(int batch) {
  if (batch <= 0) return 0;
  Sizer z;
  Work w;
  layout(batch, nullptr, &z, &w);
  return z.used;
}

extern "C" int guess_features(const double* xyz, int natm, float* feat, float* mask, void* work, size_t work_bytes,
                              cudaStream_t s) {
  clear_error();
  DF_REQUIRE(xyz && feat && mask && natm > 0, DF_ERR_ARG, "guess_features: bad arguments");
  DF_REQUIRE(work && work_bytes >= sizeof(float) * NRBF * (size_t)natm, DF_ERR_NOMEM, "guess_features: workspace");
  float* env = (float*)work;
  env_kernel<<<natm, 32, 0, s>>>(xyz, natm, env);
  DF_LAUNCHED("env_kernel");
  long npairs = (long)natm * (natm + 1) / 2;
  pair_feature_kernel<float><<<(unsigned)npairs, 96, 0, s>>>(xyz, natm, env, feat, mask);
  DF_LAUNCHED("pair_feature_kernel");
  return DF_OK;
}

extern "C" int guess_targets(const double* D, int natm, float* Y, cudaStream_t s) {
  clear_error();
  DF_REQUIRE(D && Y && natm > 0, DF_ERR_ARG, "guess_targets: bad arguments");
  long npairs = (long)natm * (natm + 1) / 2;
  block_targets_kernel<<<(unsigned)npairs, 32, 0, s>>>(D, natm, Y);
  DF_LAUNCHED("block_targets_kernel");
  return DF_OK;
}

extern "C" int guess_mlp_forward(const float* params, const float* X, int n, float* out, int bf16, void* work,
                                 size_t work_bytes, cudaStream_t s) {
  clear_error();
  DF_REQUIRE(params && X && out && n > 0, DF_ERR_ARG, "guess_mlp_forward: bad arguments");
  DF_REQUIRE(work && work_bytes >= guess_mlp_work_bytes(n), DF_ERR_NOMEM, "guess_mlp_forward: workspace too small");
  Arena a(work, work_bytes);
  Work w;
  layout(n, &a, nullptr, &w);
  if (bf16) DF_TRY(forward_bf16(params, X, n, w, s));
  else DF_TRY(forward_fp32(params, X, n, w, s));
  DF_CUDA(cudaMemcpyAsync(out, w.H[NLAYER - 1], sizeof(float) * n * NOUT, cudaMemcpyDeviceToDevice, s));
  return DF_OK;
}

extern "C" int guess_mlp_loss_grad(const float* params, const float* X, const float* Y, const float* mask, int n,
                                   float nvalid, float* loss, float* grad, void* work, size_t work_bytes,
                                   cudaStream_t s) {
  clear_error();
  DF_REQUIRE(params && X && Y && n > 0 && loss && grad, DF_ERR_ARG, "guess_mlp_loss_grad: bad arguments");
  DF_REQUIRE(work && work_bytes >= guess_mlp_work_bytes(n), DF_ERR_NOMEM, "guess_mlp_loss_grad: workspace too small");
  Arena a(work, work_bytes);
  Work w;
  layout(n, &a, nullptr, &w);
  DF_TRY(loss_grad(params, X, Y, mask, n, nvalid, w, s));
  DF_CUDA(cudaMemcpyAsync(loss, w.loss, sizeof(float), cudaMemcpyDeviceToDevice, s));
  DF_CUDA(cudaMemcpyAsync(grad, w.grad, sizeof(float) * NPARAM, cudaMemcpyDeviceToDevice, s));
  return DF_OK;
}

extern "C" int guess_mlp_train_step(float* params, float* adam_m, float* adam_v, int step, float lr, const float* X,
                                    const float* Y, const float* mask, int n, float nvalid, float* loss, void* work,
                                    size_t work_bytes, cudaStream_t s) {
  clear_error();
  DF_REQUIRE(params && adam_m && adam_v && X && Y && n > 0 && step >= 1, DF_ERR_ARG, "guess_mlp_train_step: bad args");
  DF_REQUIRE(work && work_bytes >= guess_mlp_work_bytes(n), DF_ERR_NOMEM, "guess_mlp_train_step: workspace too small");
  Arena a(work, work_bytes);
  Work w;
  layout(n, &a, nullptr, &w);
  DF_TRY(loss_grad(params, X, Y, mask, n, nvalid, w, s));
  const float b1 = 0.9f, b2 = 0.999f;
  float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<nb((long)NPARAM), 256, 0, s>>>(params, w.grad, adam_m, adam_v, (long)NPARAM, lr, b1, b2, 1e-8f, c1, c2);
  DF_LAUNCHED("adam_kernel");
  if (loss) DF_CUDA(cudaMemcpyAsync(loss, w.loss, sizeof(float), cudaMemcpyDeviceToDevice, s));
  return DF_OK;
}

extern "C" size_t guess_density_work_bytes(int natm) {
  if (natm <= 0) return 0;
  long np = (long)natm * (natm + 1) / 2;
  Sizer z;
  z.take<float>((size_t)NRBF * natm);
  z.take<float>((size_t)np * NIN);
  z.take<float>((size_t)np);
  z.take<double>((size_t)NBF * natm * NBF * natm);
  z.take<double>((size_t)NBF * natm * NBF * natm);
  z.take<double>(1);
  Work w;
  layout_infer((int)np, nullptr, &z, &w);
  return z.used;
}

extern "C" int guess_density(const float* params, const double* xyz, int natm, int nelec, const double* Sinvhalf,
                             double* D0, void* work, size_t work_bytes, cudaStream_t s) {
  clear_error();
  DF_REQUIRE(params && xyz && D0 && Sinvhalf && natm > 0 && nelec >= 0, DF_ERR_ARG, "guess_density: bad arguments");
  DF_REQUIRE(work && work_bytes >= guess_density_work_bytes(natm), DF_ERR_NOMEM, "guess_density: workspace too small");
  long np = (long)natm * (natm + 1) / 2;
  DF_REQUIRE(np < 65535L * 64, DF_ERR_ARG, "guess_density: too many centres");
  const int nao = NBF * natm;
  Arena a(work, work_bytes);
  float* env = a.take<float>((size_t)NRBF * natm);
  float* feat = a.take<float>((size_t)np * NIN);
  float* mask = a.take<float>((size_t)np);
  double* Dt = a.take<double>((size_t)nao * nao);
  double* T = a.take<double>((size_t)nao * nao);
  double* scale = a.take<double>(1);
  size_t rest = work_bytes - a.used;
  void* mw = (char*)work + a.used;
  env_kernel<<<natm, 32, 0, s>>>(xyz, natm, env);
  DF_LAUNCHED("env_kernel");
  pair_feature_kernel<float><<<(unsigned)np, 96, 0, s>>>(xyz, natm, env, feat, mask);
  DF_LAUNCHED("pair_feature_kernel");
  Arena b(mw, rest);
  Work w;
  layout_infer((int)np, &b, nullptr, &w);
  DF_REQUIRE(!b.overflow, DF_ERR_NOMEM, "guess_density: workspace too small");
  DF_TRY(forward_bf16(params, feat, (int)np, w, s));
  // orthonormal-basis density from the predicted blocks, then D0 = S^-1/2 Dt S^-1/2
  DF_CUDA(cudaMemsetAsync(Dt, 0, sizeof(double) * nao * nao, s));
  assemble_density_kernel<<<(unsigned)np, 32, 0, s>>>(w.H[NLAYER - 1], mask, natm, Dt);
  DF_LAUNCHED("assemble_density_kernel");
  if (nelec > 0) {
    trace_scale_kernel<<<1, 1024, 0, s>>>(Dt, nao, nelec, scale);
    DF_LAUNCHED("trace_scale_kernel");
    scale_kernel<<<nb((long)nao * nao), 256, 0, s>>>(Dt, (size_t)nao * nao, scale);
    DF_LAUNCHED("scale_kernel");
  }
  DF_TRY(dgemm(false, false, nao, nao, nao, 1.0, Dt, nao, 0, Sinvhalf, nao, 0, 0.0, T, nao, 0, 1, s, 0, 0));
  DF_TRY(dgemm(false, false, nao, nao, nao, 1.0, Sinvhalf, nao, 0, T, nao, 0, 0.0, D0, nao, 0, 1, s, 0, 0));
  return DF_OK;
}

// ---- model lifecycle: create, save, load ---------------------------------------------------
// The network's parameters (and Adam's moments) live in caller-owned device arrays; these
// entry points initialise them and move them to and from a self-describing host blob:
//   header  magic "DFSCFMLP", format version, layer count, each layer's (in, out), Adam step,
//           a flag for the moments, the parameter count and an FNV-1a 64-bit checksum of the
//           payload;
//   payload params [NPARAM], then (if flagged) adam_m [NPARAM] and adam_v [NPARAM], FP32.
namespace dfscf {
namespace mlp {

struct BlobHeader {
  char magic[8];
  uint32_t version;
  uint32_t nlayer;
  uint32_t in[NLAYER];
  uint32_t out[NLAYER];
  int32_t step;
  uint32_t has_moments;
  uint64_t nparam;
  uint64_t checksum;
};
constexpr uint32_t kBlobVersion = 1;

static uint64_t fnv1a(const unsigned char* p, size_t n) {
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

// Uniform(-sqrt(3 / fan_in), +sqrt(3 / fan_in)) weights from a counter-based generator
// (SplitMix64 of seed and index), zero biases.
__global__ void init_params_kernel(float* __restrict__ P, unsigned long long seed) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)NPARAM) return;
  int l = 0;
  while (l + 1 < NLAYER && (size_t)i >= w_offset(l + 1)) ++l;
  if ((size_t)i >= b_offset(l)) {
    P[i] = 0.0f;
    return;
  }
  unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);  // [0, 1)
  const double bound = sqrt(3.0 / (double)layer_in(l));
  P[i] = (float)((2.0 * u - 1.0) * bound);
}

}  // namespace mlp
}  // namespace dfscf

extern "C" int guess_mlp_create(unsigned long long seed, float* params, float* adam_m, float* adam_v, cudaStream_t s) {
  clear_error();
  DF_REQUIRE(params, DF_ERR_ARG, "guess_mlp_create: null params");
  init_params_kernel<<<nb((long)NPARAM), 256, 0, s>>>(params, seed);
  DF_LAUNCHED("init_params_kernel");
  if (adam_m) DF_CUDA(cudaMemsetAsync(adam_m, 0, sizeof(float) * NPARAM, s));
  if (adam_v) DF_CUDA(cudaMemsetAsync(adam_v, 0, sizeof(float) * NPARAM, s));
  return DF_OK;
}

extern "C" size_t guess_mlp_blob_bytes(int with_moments) {
  return sizeof(BlobHeader) + sizeof(float) * NPARAM * (with_moments ? 3 : 1);
}

extern "C" int guess_mlp_save(const float* params, const float* adam_m, const float* adam_v, int step, void* blob,
                              size_t blob_bytes, cudaStream_t s) {
  clear_error();
  DF_REQUIRE(params && blob && step >= 0, DF_ERR_ARG, "guess_mlp_save: bad arguments");
  DF_REQUIRE((adam_m == nullptr) == (adam_v == nullptr), DF_ERR_ARG, "guess_mlp_save: give both Adam moments or neither");
  const int moments = adam_m != nullptr;
  DF_REQUIRE(blob_bytes >= guess_mlp_blob_bytes(moments), DF_ERR_NOMEM, "guess_mlp_save: blob of %zu bytes < %zu",
             blob_bytes, guess_mlp_blob_bytes(moments));
  BlobHeader h{};
  memcpy(h.magic, "DFSCFMLP", 8);
  h.version = kBlobVersion;
  h.nlayer = NLAYER;
  for (int l = 0; l < NLAYER; ++l) {
    h.in[l] = (uint32_t)layer_in(l);
    h.out[l] = (uint32_t)layer_out(l);
  }
  h.step = step;
  h.has_moments = (uint32_t)moments;
  h.nparam = NPARAM;
  unsigned char* payload = (unsigned char*)blob + sizeof(BlobHeader);
  DF_CUDA(cudaMemcpyAsync(payload, params, sizeof(float) * NPARAM, cudaMemcpyDefault, s));
  if (moments) {
    DF_CUDA(cudaMemcpyAsync(payload + sizeof(float) * NPARAM, adam_m, sizeof(float) * NPARAM, cudaMemcpyDefault, s));
    DF_CUDA(cudaMemcpyAsync(payload + 2 * sizeof(float) * NPARAM, adam_v, sizeof(float) * NPARAM, cudaMemcpyDefault, s));
  }
  DF_CUDA(cudaStreamSynchronize(s));
  h.checksum = fnv1a(payload, sizeof(float) * NPARAM * (moments ? 3 : 1));
  memcpy(blob, &h, sizeof(h));
  return DF_OK;
}

extern "C" int guess_mlp_load(const void* blob, size_t blob_bytes, float* params, float* adam_m, float* adam_v,
                              int* step, cudaStream_t s) {
  clear_error();
  DF_REQUIRE(blob && params, DF_ERR_ARG, "guess_mlp_load: bad arguments");
  DF_REQUIRE((adam_m == nullptr) == (adam_v == nullptr), DF_ERR_ARG, "guess_mlp_load: give both Adam moments or neither");
  DF_REQUIRE(blob_bytes >= sizeof(BlobHeader), DF_ERR_ARG, "guess_mlp_load: blob of %zu bytes has no header", blob_bytes);
  BlobHeader h;
  memcpy(&h, blob, sizeof(h));
  DF_REQUIRE(memcmp(h.magic, "DFSCFMLP", 8) == 0, DF_ERR_ARG, "guess_mlp_load: not a model blob (bad magic)");
  DF_REQUIRE(h.version == kBlobVersion, DF_ERR_ARG, "guess_mlp_load: format version %u, expected %u", h.version,
             kBlobVersion);
  bool shapes = h.nlayer == NLAYER && h.nparam == NPARAM;
  for (int l = 0; shapes && l < NLAYER; ++l) shapes = h.in[l] == (uint32_t)layer_in(l) && h.out[l] == (uint32_t)layer_out(l);
  DF_REQUIRE(shapes, DF_ERR_ARG, "guess_mlp_load: the blob's layer shapes differ from this library's network");
  const size_t payload_bytes = sizeof(float) * NPARAM * (h.has_moments ? 3 : 1);
  DF_REQUIRE(blob_bytes >= sizeof(BlobHeader) + payload_bytes, DF_ERR_ARG, "guess_mlp_load: blob truncated");
  const unsigned char* payload = (const unsigned char*)blob + sizeof(BlobHeader);
  DF_REQUIRE(fnv1a(payload, payload_bytes) == h.checksum, DF_ERR_ARG, "guess_mlp_load: checksum mismatch");
  DF_CUDA(cudaMemcpyAsync(params, payload, sizeof(float) * NPARAM, cudaMemcpyDefault, s));
  if (adam_m) {
    if (h.has_moments) {
      DF_CUDA(cudaMemcpyAsync(adam_m, payload + sizeof(float) * NPARAM, sizeof(float) * NPARAM, cudaMemcpyDefault, s));
      DF_CUDA(cudaMemcpyAsync(adam_v, payload + 2 * sizeof(float) * NPARAM, sizeof(float) * NPARAM, cudaMemcpyDefault,
                              s));
    } else {
      DF_CUDA(cudaMemsetAsync(adam_m, 0, sizeof(float) * NPARAM, s));
      DF_CUDA(cudaMemsetAsync(adam_v, 0, sizeof(float) * NPARAM, s));
    }
  }
  DF_CUDA(cudaStreamSynchronize(s));
  if (step) *step = h.has_moments ? h.step : 0;
  return DF_OK;
}

DF_BOUNDS_READER(bounds_read_mlp)
