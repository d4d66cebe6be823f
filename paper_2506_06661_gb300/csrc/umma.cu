// Mixed-precision DF exchange build on the 5th-generation tensor cores (tcgen05).
//
// K_mn = sum_P sum_i X_{P,mi} X_{P,ni},  X_P = B_P C   (arXiv 2506.06661, Section
// "Density fitting": the fitted integrals sum_P B_{P,mk} B_{P,nl} contracted with the
// occupied coefficients).  Both contractions run as split-BF16 GEMMs: every operand row is
// stored as NP BF16 planes; with sigma the power of two just above the row's max |x|,
// p0 = x rounded to the grid sigma 2^-7, p1 = (x - p0) rounded to sigma 2^-15, and
// p2 .. p(NP-1) = BF16 roundings of what is left.  A product is formed from the plane
// products pa*qb with a + b < NP in FP32 accumulators in tensor memory (TMEM).  p0 and p1
// are fixed-point (integers on grids fixed along each row, planes.cuh), so in the exchange SYRK the
// products (0,0), (0,1)+(1,0) and (1,1) each sum integers on one grid in an accumulator of
// their own and are exact; every product with a floating plane (the contributions of
// elements far below their row's max) goes to a fourth.  The half-transform uses two
// accumulators, (0,0) and the rest.  With a single accumulator, long FP32 sums of many
// small positive products lose their low bits and K of a 300-centre molecule comes out
// ~1e-5 low on the diagonal.  NP = 3, 4, 5: 6, 10, 15 products.
//
//   half-transform:  X[(P,m), i] = sum_n B[(P,m), n] C^T[i, n]     (A = B planes, B = C^T)
//   exchange SYRK:   K[m, n]     = sum_(P,i) X[m, (P,i)] X[n, (P,i)] (A = B = X, lower tiles)
//
// Both are "D = A B^T" with A and B K-major in global memory, so one kernel serves both:
// TMA (128-byte swizzle and 64-element K boxes; 64-byte swizzle and 32-element boxes for four
// or more planes, whose stages are wider) fills a multi-stage shared-memory ring, one
// elected lane issues tcgen05.mma (M = 128, N <= 256, K = 16 per instruction, one per
// plane product and K step), tcgen05.commit releases ring slots, and four epilogue warps read the
// accumulator with tcgen05.ld.  Every mbarrier wait is bounded; on a timeout the kernel
// raises a device error flag and returns after releasing its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "kernels.cuh"
#include "planes.cuh"
#include "tcgen05.cuh"

namespace dfscf {

namespace umma {

enum Mode { HALF_TRANSFORM = 0, SYRK = 1 };

struct Params {
  int mode;
  int N;             // tile columns (multiple of 16, <= 256)
  int num_kb;        // K blocks of bk_of(NP) in the whole K range
  int kb_per_split;  // K blocks per split (SYRK) or num_kb
  int stages;
  uint32_t stage_bytes;
  uint32_t b_bytes;  // bytes of one B tile (N x 128)
  // half-transform epilogue: X as the FP32 pair (order 0, higher orders) and the max |X|
  // of every row m
  int npad;          // rows per P in A
  long ldx;          // X row stride (elements)
  int ncx;           // X columns per P
  float* X32;        // [2][npad][ldx]
  long xsize;        // npad * ldx
  unsigned* xmax;    // FP32 bit patterns of max |X| per row m (non-negative: integer order)
  // SYRK epilogue
  float* Kpart;      // [split][npad][npad]
  int n_lower_tiles;
  int* err;
};

// Tile t of the lower triangle in row blocks of 128 and column blocks of 128 * wide: row
// block mt needs (mt + wide) / wide column blocks to reach its diagonal.
__host__ __device__ __forceinline__ int lower_tiles_in_row(int mt, int wide) { return (mt + wide) / wide; }
__device__ __forceinline__ void lower_tile(int t, int wide, int& mt, int& nt) {
  int m = 0;
  while (t >= lower_tiles_in_row(m, wide)) {
    t -= lower_tiles_in_row(m, wide);
    ++m;
  }
  mt = m;
  nt = t;
}

// Tensor maps of the operand planes (A planes, then B planes); entries >= NP unused.
struct Maps {
  CUtensorMap a[5];
  CUtensorMap b[5];
};

template <int NP, int BK>
__global__ void __launch_bounds__(THREADS, 1) split_bf16_gemm_kernel(const __grid_constant__ Maps maps,
                                                                      const Params p) {
  extern __shared__ uint8_t dyn_smem[];
  __shared__ uint64_t full_bar[MAX_STAGES];
  __shared__ uint64_t empty_bar[MAX_STAGES];
  __shared__ uint64_t accum_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // tile coordinates
  int row0, col0, kb0, nkb, split = 0;
  if (p.mode == HALF_TRANSFORM) {
    row0 = blockIdx.x * BM;
    col0 = blockIdx.y * p.N;
    kb0 = 0;
    nkb = p.num_kb;
  } else {
    int mt, nt;
    lower_tile(blockIdx.x, p.N / BM, mt, nt);
    row0 = mt * BM;
    col0 = nt * p.N;
    split = blockIdx.y;
    kb0 = split * p.kb_per_split;
    nkb = min(p.kb_per_split, p.num_kb - kb0);
  }
  // a wait of this build already gave up (flag set by another CTA): no work, no waits
  if (*(volatile const int*)p.err) nkb = 0;
  // 1024-byte aligned ring of stages: [A planes | B planes]
  uint32_t base = smem_u32(dyn_smem);
  uint32_t pad = (1024u - (base & 1023u)) & 1023u;
  uint8_t* ring = dyn_smem + pad;
  const uint32_t a_bytes = BM * BK * 2;
  const int nacc = p.mode == SYRK ? 4 : 2;  // accumulators of N columns
  uint32_t ncols = 32;
  while ((int)ncols < nacc * p.N) ncols <<= 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < p.stages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&accum_bar, 1);
    abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == 0 && lane == 0) {
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      tma_prefetch(&maps.a[j]);
      tma_prefetch(&maps.b[j]);
    }
  }
  if (warp == 1) {
    tmem_alloc(&tmem_base, ncols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  int issued = 0;  // k-blocks whose loads the producer has issued

  if (warp == 0 && lane == 0 && nkb > 0) {
    // ---- TMA producer ----------------------------------------------------------------
    for (int i = 0; i < nkb; ++i) {
      int s = i % p.stages;
      uint32_t ph = (uint32_t)(i / p.stages) & 1u;
      if (!mbar_wait(&empty_bar[s], ph ^ 1u, &abort_flag)) {
        abort_flag = 1;
        break;
      }
      uint8_t* st = ring + (size_t)s * p.stage_bytes;
      mbar_arrive_expect_tx(&full_bar[s], p.stage_bytes);
      int kx = (kb0 + i) * BK;
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        tma_load_2d(st + j * a_bytes, &maps.a[j], &full_bar[s], kx, row0);
        tma_load_2d(st + NP * a_bytes + j * p.b_bytes, &maps.b[j], &full_bar[s], kx, col0);
      }
      issued = i + 1;
    }
  } else if (warp == 1 && lane == 0 && nkb > 0) {
    // ---- MMA issuer ------------------------------------------------------------------
    const uint32_t idesc = idesc_bf16(BM, p.N);
    bool ok = true;
    for (int i = 0; i < nkb; ++i) {
      int s = i % p.stages;
      uint32_t ph = (uint32_t)(i / p.stages) & 1u;
      if (!mbar_wait(&full_bar[s], ph, &abort_flag)) {
        abort_flag = 1;
        ok = false;
        break;
      }
      tc_fence_after();
      uint32_t st = smem_u32(ring + (size_t)s * p.stage_bytes);
      uint64_t ad[NP], bd[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        ad[j] = desc_sw<BK>(st + j * a_bytes);
        bd[j] = desc_sw<BK>(st + NP * a_bytes + j * p.b_bytes);
      }
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        uint64_t off = (uint64_t)(kk * 32) >> 4;  // 16 bf16 = 32 bytes along K inside the swizzle row
        // plane products in order t = a + b; accumulator of (a, b): half-transform (0,0) -> 0,
        // rest -> 1; SYRK (0,0) -> 0, (0,1) (1,0) -> 1, (1,1) -> 2, rest -> 3.  The first
        // product issued into an accumulator (t = 0; t = 1, a = 0; SYRK t = 2, a <= 1)
        // overwrites it.
#pragma unroll
        for (int t = 0; t < NP; ++t)
#pragma unroll
          for (int a = 0; a <= t; ++a) {
            const int b = t - a;
            const int acc = p.mode == SYRK ? ((a <= 1 && b <= 1) ? t : 3) : (t > 0 ? 1 : 0);
            const bool first = t == 0 || (t == 1 && a == 0) || (p.mode == SYRK && t == 2 && a <= 1);
            umma_bf16(tmem + (uint32_t)(acc * p.N), ad[a] + off, bd[b] + off, idesc,
                      (i > 0 || kk > 0 || !first) ? 1u : 0u);
          }
      }
      umma_commit(&empty_bar[s]);  // slot reusable once these MMAs have read it
    }
    if (ok) umma_commit(&accum_bar);
  } else if (warp >= 2) {
    // ---- epilogue: TMEM -> registers -> global ----------------------------------------
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    const int r = q * 32 + lane;
    bool ok = (nkb > 0) && mbar_wait(&accum_bar, 0, &abort_flag);
    ok = __all_sync(0xffffffffu, ok);  // the TMEM loads below are warp-collective
    if (!ok && nkb > 0) abort_flag = 1;
    tc_fence_after();
    if (ok) {
      const int grow = row0 + r;
      float lmax = 0.0f;
      for (int c = 0; c < p.N; c += 16) {
        if (p.mode == HALF_TRANSFORM && col0 + c >= p.ncx) break;  // column tiles past ncpad
        if (p.mode == SYRK && col0 + c >= p.npad) break;            // last wide tile past npad
        uint32_t v[4][16];
        tmem_ld_x16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c, v[0]);
        tmem_ld_x16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(p.N + c), v[1]);
        if (nacc == 4) {
          tmem_ld_x16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(2 * p.N + c), v[2]);
          tmem_ld_x16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(3 * p.N + c), v[3]);
        }
        tmem_wait_ld();
        float x[16];
        if (nacc == 4) {
#pragma unroll
          for (int j = 0; j < 16; ++j)  // smallest first
            x[j] = ((__uint_as_float(v[3][j]) + __uint_as_float(v[2][j])) + __uint_as_float(v[1][j])) +
                   __uint_as_float(v[0][j]);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) x[j] = __uint_as_float(v[0][j]) + __uint_as_float(v[1][j]);
        }
        if (p.mode == HALF_TRANSFORM) {
          int P = grow / p.npad, m = grow % p.npad;
          const size_t o = DF_IXW((size_t)m * p.ldx + (size_t)P * p.ncx + col0 + c, 16, p.xsize);
          float4* d0 = reinterpret_cast<float4*>(p.X32 + o);
          float4* d1 = reinterpret_cast<float4*>(p.X32 + p.xsize + o);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            d0[j] = make_float4(__uint_as_float(v[0][4 * j]), __uint_as_float(v[0][4 * j + 1]),
                                __uint_as_float(v[0][4 * j + 2]), __uint_as_float(v[0][4 * j + 3]));
            d1[j] = make_float4(__uint_as_float(v[1][4 * j]), __uint_as_float(v[1][4 * j + 1]),
                                __uint_as_float(v[1][4 * j + 2]), __uint_as_float(v[1][4 * j + 3]));
            lmax = fmaxf(lmax, fmaxf(fmaxf(fabsf(x[4 * j]), fabsf(x[4 * j + 1])),
                                     fmaxf(fabsf(x[4 * j + 2]), fabsf(x[4 * j + 3]))));
          }
        } else {
          float4* dst = reinterpret_cast<float4*>(
              p.Kpart + DF_IXW(((size_t)split * p.npad + grow) * p.npad + col0 + c, 16,
                               (size_t)gridDim.y * p.npad * p.npad));
#pragma unroll
          for (int j = 0; j < 4; ++j) dst[j] = make_float4(x[4 * j], x[4 * j + 1], x[4 * j + 2], x[4 * j + 3]);
        }
      }
      if (p.mode == HALF_TRANSFORM) atomicMax(p.xmax + grow % p.npad, __float_as_uint(lmax));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (abort_flag && warp == 0 && lane == 0) {
    atomicExch(p.err, 1);
    // after a timeout, wait (bounded) for the loads still in flight into each ring slot
    // before the CTA's shared memory is released: the last k-block issued to slot s
    // completes phase ((i / stages) & 1) of full_bar[s]
    for (int s = 0; s < p.stages; ++s) {
      const int last = issued - 1 - ((issued - 1 - s) % p.stages + p.stages) % p.stages;
      if (issued > 0 && last >= 0 && last % p.stages == s)
        mbar_wait(&full_bar[s], (uint32_t)(last / p.stages) & 1u, nullptr);
    }
  }
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, ncols);
  }
}

// ---- exchange SYRK on CTA pairs ------------------------------------------------------------
// One cluster of two CTAs computes a 256 x 128 block of K (rows row_pair .. +255, columns
// col0 .. +127) with tcgen05.mma.cta_group::2 (M = 256, N = 128): each CTA stages its own 128
// rows of the A operand and 64 of the 128 rows of the shared B operand, and the leader CTA
// (rank 0) issues every MMA, which reads both CTAs' shared memory and writes rows 0..127 of the
// block into the leader's TMEM and rows 128..255 into the peer's.  Per MMA a CTA reads 4 KB of
// A and 2 KB of B from its shared memory instead of 4 + 4 KB for a one-CTA 128 x 128 tile, and
// a stage is 60 KB instead of 80 KB (three stages in flight instead of two).  The plane
// products and their four accumulators are those of split_bf16_gemm_kernel's SYRK mode.
//
// Blocks: double rows of 256 (row blocks 2 mp and 2 mp + 1) times column blocks of 128 up to
// and including the double row's diagonal, nt <= 2 mp + 1 (the block above the diagonal of
// row block 2 mp is formed too; the reduction reads m >= n only).  A double row past npad
// (odd npad / 128) loads zeros (TMA fill) and writes nothing.
//
// Barriers: full_bar[s] of the leader counts the bytes of both CTAs' loads of stage s (the
// peer's loads complete on it through their cluster address); the leader's commits arrive on
// empty_bar[s] and accum_bar of both CTAs.  Waits are bounded as in the one-CTA kernel.

__host__ __device__ __forceinline__ int pair_col_blocks(int mp, int nblk) { return min(2 * mp + 2, nblk); }

__device__ __forceinline__ void pair_block(int t, int nblk, int& mp, int& nt) {
  int m = 0;
  while (t >= pair_col_blocks(m, nblk)) {
    t -= pair_col_blocks(m, nblk);
    ++m;
  }
  mp = m;
  nt = t;
}

template <int NP, int BK>
__global__ void __launch_bounds__(THREADS, 1) syrk_pair_kernel(const __grid_constant__ Maps maps, const Params p) {
  extern __shared__ uint8_t dyn_smem[];
  __shared__ uint64_t full_bar[MAX_STAGES];
  __shared__ uint64_t empty_bar[MAX_STAGES];
  __shared__ uint64_t accum_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const int nblk = p.npad / BM;
  int mp, nt;
  pair_block((int)(blockIdx.x >> 1), nblk, mp, nt);
  const int row0 = mp * 2 * BM + (int)rank * BM;  // this CTA's rows of the block
  const int col0 = nt * BM;                       // the block's columns
  const int bcol = col0 + (int)rank * (BM / 2);   // this CTA's half of the B rows
  const int split = blockIdx.y;
  const int kb0 = split * p.kb_per_split;
  // a wait of this build already gave up (flag set by another CTA): no work; a peer that
  // read the flag before it was set gives up on its own waits after WAIT_NS
  const int nkb = *(volatile const int*)p.err ? 0 : min(p.kb_per_split, p.num_kb - kb0);

  uint32_t base = smem_u32(dyn_smem);
  uint32_t pad = (1024u - (base & 1023u)) & 1023u;
  uint8_t* ring = dyn_smem + pad;
  constexpr uint32_t a_bytes = BM * BK * 2;        // 128 rows
  constexpr uint32_t bh_bytes = (BM / 2) * BK * 2; // 64 rows
  constexpr uint32_t cta_stage = NP * (a_bytes + bh_bytes);
  constexpr uint32_t ncols = 4 * BM;               // four accumulators of 128 columns

  if (threadIdx.x == 0) {
    for (int s = 0; s < p.stages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&accum_bar, 1);
    abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == 0 && lane == 0) {
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      tma_prefetch(&maps.a[j]);
      tma_prefetch(&maps.b[j]);
    }
  }
  if (warp == 1) {
    tmem_alloc_pair(&tmem_base, ncols);
    tmem_relinquish_pair();
  }
  tc_fence_before();
  cluster_sync();  // both CTAs' barriers initialised and TMEM allocated before any remote use
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  int issued = 0;

  if (warp == 0 && lane == 0 && nkb > 0) {
    // ---- TMA producer (both CTAs) --------------------------------------------------------
    for (int i = 0; i < nkb; ++i) {
      const int s = i % p.stages;
      const uint32_t ph = (uint32_t)(i / p.stages) & 1u;
      if (!mbar_wait(&empty_bar[s], ph ^ 1u, &abort_flag)) {
        abort_flag = 1;
        break;
      }
      uint8_t* st = ring + (size_t)s * cta_stage;
      if (rank == 0) mbar_arrive_expect_tx(&full_bar[s], 2 * cta_stage);
      const uint32_t bar = mapa_rank(smem_u32(&full_bar[s]), 0);
      const int kx = (kb0 + i) * BK;
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        tma_load_2d_pair(st + j * a_bytes, &maps.a[j], bar, kx, row0);
        tma_load_2d_pair(st + NP * a_bytes + j * bh_bytes, &maps.b[j], bar, kx, bcol);
      }
      issued = i + 1;
    }
  } else if (warp == 1 && lane == 0 && rank == 0 && nkb > 0) {
    // ---- MMA issuer (leader only) -------------------------------------------------------
    const uint32_t idesc = idesc_bf16(2 * BM, BM);
    bool ok = true;
    for (int i = 0; i < nkb; ++i) {
      const int s = i % p.stages;
      const uint32_t ph = (uint32_t)(i / p.stages) & 1u;
      if (!mbar_wait(&full_bar[s], ph, &abort_flag)) {
        abort_flag = 1;
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t st = smem_u32(ring + (size_t)s * cta_stage);
      uint64_t ad[NP], bd[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        ad[j] = desc_sw<BK>(st + j * a_bytes);
        bd[j] = desc_sw<BK>(st + NP * a_bytes + j * bh_bytes);
      }
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        const uint64_t off = (uint64_t)(kk * 32) >> 4;
#pragma unroll
        for (int t = 0; t < NP; ++t)
#pragma unroll
          for (int a = 0; a <= t; ++a) {
            const int b = t - a;
            const int acc = (a <= 1 && b <= 1) ? t : 3;
            const bool first = t == 0 || (t == 1 && a == 0) || (t == 2 && a <= 1);
            umma_bf16_pair(tmem + (uint32_t)(acc * BM), ad[a] + off, bd[b] + off, idesc,
                           (i > 0 || kk > 0 || !first) ? 1u : 0u);
          }
      }
      umma_commit_pair(&empty_bar[s]);
    }
    if (ok) umma_commit_pair(&accum_bar);
  } else if (warp >= 2) {
    // ---- epilogue (both CTAs): this CTA's 128 rows from its own TMEM --------------------
    const int q = warp & 3;
    const int r = q * 32 + lane;
    bool ok = (nkb > 0) && mbar_wait(&accum_bar, 0, &abort_flag);
    ok = __all_sync(0xffffffffu, ok);  // the TMEM loads below are warp-collective
    if (!ok && nkb > 0) abort_flag = 1;
    tc_fence_after();
    const int grow = row0 + r;
    if (ok && row0 < p.npad) {
      for (int c = 0; c < BM; c += 16) {
        uint32_t v[4][16];
#pragma unroll
        for (int k = 0; k < 4; ++k) tmem_ld_x16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(k * BM + c), v[k]);
        tmem_wait_ld();
        float x[16];
#pragma unroll
        for (int j = 0; j < 16; ++j)  // smallest first
          x[j] = ((__uint_as_float(v[3][j]) + __uint_as_float(v[2][j])) + __uint_as_float(v[1][j])) +
                 __uint_as_float(v[0][j]);
        float4* dst = reinterpret_cast<float4*>(
            p.Kpart + DF_IXW(((size_t)split * p.npad + grow) * p.npad + col0 + c, 16,
                             (size_t)gridDim.y * p.npad * p.npad));
#pragma unroll
        for (int j = 0; j < 4; ++j) dst[j] = make_float4(x[4 * j], x[4 * j + 1], x[4 * j + 2], x[4 * j + 3]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (abort_flag && warp == 0 && lane == 0) {
    atomicExch(p.err, 1);
    // loads still in flight complete on the leader's full barriers: the leader waits
    // (bounded) for the last phase of every slot it armed
    if (rank == 0)
      for (int s = 0; s < p.stages; ++s) {
        const int last = issued - 1 - ((issued - 1 - s) % p.stages + p.stages) % p.stages;
        if (issued > 0 && last >= 0 && last % p.stages == s)
          mbar_wait(&full_bar[s], (uint32_t)(last / p.stages) & 1u, nullptr);
      }
  }
  cluster_sync();  // no CTA leaves while its peer may still signal its barriers or read its TMEM
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc_pair(tmem, ncols);
  }
}

}  // namespace umma

// ---- host side -------------------------------------------------------------------------

template <int NP, int BK>
static int launch_gemm(const umma::Maps& maps, umma::Params p, dim3 grid, cudaStream_t s) {
  p.b_bytes = (uint32_t)p.N * BK * 2;
  p.stage_bytes = NP * (umma::BM * BK * 2 + p.b_bytes);
  const uint32_t budget = 220 * 1024;
  p.stages = (int)std::min<uint32_t>(std::min(umma::MAX_STAGES, std::max(2, knob("umma_max_stages"))),
                                     budget / p.stage_bytes);
  DF_REQUIRE(p.stages >= 2, DF_ERR_ARG, "split-bf16 GEMM: tile too large for shared memory");
  size_t smem = (size_t)p.stages * p.stage_bytes + 1024;
  DF_REQUIRE(smem <= 220 * 1024 + 1024, DF_ERR_ARG, "split-bf16 GEMM: %zu bytes of shared memory requested", smem);
  DF_TRY(umma_prepare());
  umma::split_bf16_gemm_kernel<NP, BK><<<grid, umma::THREADS, smem, s>>>(maps, p);
  DF_LAUNCHED("split_bf16_gemm_kernel");
  return DF_OK;
}

// Double-row blocks of the CTA-pair SYRK for npad rows.
static int pair_blocks(int npad) {
  const int nblk = npad / umma::BM;
  int t = 0;
  for (int mp = 0; 2 * mp < nblk; ++mp) t += umma::pair_col_blocks(mp, nblk);
  return t;
}

// CTA-pair exchange SYRK: clusters of two CTAs along x (grid.x = 2 x double-row blocks).
template <int NP, int BK>
static int launch_syrk_pair(const umma::Maps& maps, umma::Params p, dim3 grid, cudaStream_t s) {
  p.b_bytes = (uint32_t)(umma::BM / 2) * BK * 2;
  p.stage_bytes = NP * (umma::BM * BK * 2 + p.b_bytes);
  const uint32_t budget = 220 * 1024;
  p.stages = (int)std::min<uint32_t>(std::min(umma::MAX_STAGES, std::max(2, knob("umma_max_stages"))),
                                     budget / p.stage_bytes);
  DF_REQUIRE(p.stages >= 2, DF_ERR_ARG, "pair SYRK: stage too large for shared memory");
  DF_REQUIRE(grid.x % 2 == 0, DF_ERR_ARG, "pair SYRK: odd grid");
  const size_t smem = (size_t)p.stages * p.stage_bytes + 1024;
  DF_TRY(umma_prepare());
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(umma::THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  DF_CUDA(cudaLaunchKernelEx(&cfg, umma::syrk_pair_kernel<NP, BK>, maps, p));
  DF_LAUNCHED("syrk_pair_kernel");
  return DF_OK;
}

struct PlanePtrs {
  __nv_bfloat16* p[5];
};

// C^T [ncpad][npad] as row-scaled planes (row i = column i of C over n); one CTA per row,
// zero padding.
__global__ void __launch_bounds__(256) pack_ct_kernel(const double* __restrict__ C, int nao, int nocc, int npad,
                                                      int planes, PlanePtrs out) {
  __shared__ double sh[8];
  const int i = blockIdx.x;
  double amax = 0.0;
  if (i < nocc)
    for (int n = threadIdx.x; n < nao; n += blockDim.x) amax = fmax(amax, fabs(C[DF_IX((size_t)n * nocc + i, (size_t)nao * nocc)]));
  for (int o = 16; o; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = amax;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < 8; ++w) t = fmax(t, sh[w]);
  const double sig = row_scale(t);
  for (int n = threadIdx.x; n < npad; n += blockDim.x) {
    const double x = (i < nocc && n < nao) ? C[(size_t)n * nocc + i] : 0.0;
    __nv_bfloat16 q[kPlanesMax];
    split_row_value(x, sig, q);
    const size_t e = DF_IX((size_t)i * npad + n, (size_t)gridDim.x * npad);
    for (int j = 0; j < planes; ++j) out.p[j][e] = q[j];
  }
}

// X [npad][kdim], held as the FP32 pair (X0, X1) = (order-0, higher-order accumulators), into
// row-scaled planes, the scale of row m from xmax[m].  Row m is blockIdx.y; four consecutive
// elements per thread (kdim is a multiple of 16).
template <int NP>
__global__ void __launch_bounds__(256) x_to_planes_kernel(const float* __restrict__ X0, const float* __restrict__ X1,
                                                          const unsigned* __restrict__ xmax, long kdim,
                                                          PlanePtrs out) {
  const int m = blockIdx.y;
  // the row max came from the rounded sum X0 + X1: a power of two above it by at least one
  // FP32 ulp covers the exact pair
  const float sig = row_scale_f(__uint_as_float(xmax[m]) * (1.0f + 1.2e-7f));
  const size_t row = (size_t)m * kdim;
  for (long c = ((long)blockIdx.x * blockDim.x + threadIdx.x) * 4; c < kdim; c += (long)gridDim.x * blockDim.x * 4) {
    const size_t at = DF_IXW(row + c, 4, (size_t)gridDim.y * kdim);
    const float4 a = *reinterpret_cast<const float4*>(X0 + at);
    const float4 b = *reinterpret_cast<const float4*>(X1 + at);
    const float hs[4] = {a.x, a.y, a.z, a.w}, ls[4] = {b.x, b.y, b.z, b.w};
    __align__(8) __nv_bfloat16 q[NP][4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      __nv_bfloat16 t[kPlanesMax];
      split_row_pair(hs[u], ls[u], sig, t);
#pragma unroll
      for (int j = 0; j < NP; ++j) q[j][u] = t[j];
    }
#pragma unroll
    for (int j = 0; j < NP; ++j) *reinterpret_cast<uint2*>(out.p[j] + at) = *reinterpret_cast<uint2*>(q[j]);
  }
}

// K[m][n] = K[n][m] = sum_split Kpart[split][m][n] (FP64 sum of FP32 partials), m >= n.
// When a bounded wait of the tensor-core kernels gave up (*err set), K is filled with NaN so
// that an incomplete exchange matrix can never pass for a result.
__global__ void kmixed_reduce_kernel(const float* __restrict__ Kpart, int nsplit, int npad, int nao,
                                     const int* __restrict__ err, double* __restrict__ K) {
  long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)nao * nao) return;
  int m = (int)(e / nao), n = (int)(e % nao);
  if (n > m) return;
  double s = 0.0;
  for (int k = 0; k < nsplit; ++k) s += (double)Kpart[DF_IX(((size_t)k * npad + m) * npad + n, (size_t)nsplit * npad * npad)];
  if (*err) s = __longlong_as_double(0x7ff8000000000000LL);
  K[(size_t)m * nao + n] = s;
  K[(size_t)n * nao + m] = s;
}

static int mixed_ncpad(int nocc) { return std::max(16, (nocc + 15) / 16 * 16); }

// Columns of an exchange SYRK tile: four accumulators of 128 columns fill TMEM.
static int syrk_n(int) { return 128; }

// Widest half-transform tile (multiple of 16, <= 256) whose stage fits twice in the ring.
static int ht_max_n(int planes) {
  const int bk = umma::bk_of(planes);
  const long budget = 220 * 1024 / 2;
  long n = (budget / planes - (long)umma::BM * bk * 2) / (bk * 2);
  return (int)std::min<long>(256, n / 16 * 16);
}

static int syrk_tiles(int npad, int planes) {
  int t = 0;
  for (int mt = 0; mt < npad / umma::BM; ++mt) t += umma::lower_tiles_in_row(mt, syrk_n(planes) / umma::BM);
  return t;
}

static int mixed_nsplit(int npad, int naux, int ncpad, int planes) {
  const int bk = umma::bk_of(planes);
  long kdim = (long)naux * ncpad;
  long nkb = (kdim + bk - 1) / bk;
  int tiles = syrk_tiles(npad, planes);
  // several waves of CTAs; splits of at most ~16k terms
  long want = std::max<long>((kdim + 16383) / 16384, (4L * 152 + tiles - 1) / tiles);
  if (knob("syrk_split") > 0) want = knob("syrk_split");
  return (int)std::max<long>(1, std::min<long>(want, std::min<long>(nkb, 1024)));
}

// Raise the tensor-core kernel's dynamic shared-memory limit once, before any launch can
// happen inside a stream capture.
int umma_prepare() {
  static bool done = false;
  if (!done) {
    const int lim = 220 * 1024 + 1024;
    DF_CUDA(cudaFuncSetAttribute(umma::syrk_pair_kernel<3, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    DF_CUDA(cudaFuncSetAttribute(umma::syrk_pair_kernel<4, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    DF_CUDA(cudaFuncSetAttribute(umma::syrk_pair_kernel<5, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    DF_CUDA(cudaFuncSetAttribute(umma::split_bf16_gemm_kernel<3, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    DF_CUDA(cudaFuncSetAttribute(umma::split_bf16_gemm_kernel<4, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    DF_CUDA(cudaFuncSetAttribute(umma::split_bf16_gemm_kernel<5, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    DF_CUDA(cudaFuncSetAttribute(umma::split_bf16_gemm_kernel<3, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    DF_CUDA(cudaFuncSetAttribute(umma::split_bf16_gemm_kernel<4, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    DF_CUDA(cudaFuncSetAttribute(umma::split_bf16_gemm_kernel<5, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    done = true;
  }
  return DF_OK;
}

// BF16 planes per operand of the mixed exchange (knob "mixed_planes": 3, 4 or 5).
int mixed_planes() { return std::min(5, std::max(3, knob("mixed_planes"))); }

void mixed_k_work_layout(int nao, int naux, int nocc, Arena* a, Sizer* z, MixedKWork* w) {
  int npad = nao_pad(nao);
  int ncpad = mixed_ncpad(std::max(nocc, 1));
  w->planes = mixed_planes();
  int nsplit = mixed_nsplit(npad, naux, ncpad, w->planes);
  w->ncpad = ncpad;
  w->nsplit = nsplit;
  size_t xsize = (size_t)npad * naux * ncpad;
  for (int j = 0; j < kMixedPlanes; ++j) {
    w->Cp[j] = nullptr;
    w->Xp[j] = nullptr;
  }
  for (int j = 0; j < w->planes; ++j) {
    if (a) w->Cp[j] = a->take<__nv_bfloat16>((size_t)ncpad * npad);
    else z->take<__nv_bfloat16>((size_t)ncpad * npad);
  }
  for (int j = 0; j < w->planes; ++j) {
    if (a) w->Xp[j] = a->take<__nv_bfloat16>(xsize);
    else z->take<__nv_bfloat16>(xsize);
  }
  if (a) {
    w->X32 = a->take<float>(2 * xsize);
    w->xmax = a->take<unsigned>((size_t)npad);
  } else {
    z->take<float>(2 * xsize);
    z->take<unsigned>((size_t)npad);
  }
  if (a) {
    w->Kpart = a->take<float>((size_t)nsplit * npad * npad);
    w->err = a->take<int>(1);
  } else {
    z->take<float>((size_t)nsplit * npad * npad);
    z->take<int>(1);
  }
}

int build_K_mixed(const void* B, const BLayout& L, int nao, int naux, const double* C, int nocc, double* K,
                  const MixedKWork& w, cudaStream_t s) {
  const int npad = L.npad, ncpad = w.ncpad, NP = w.planes;
  DF_REQUIRE(nocc <= ncpad, DF_ERR_ARG, "mixed K: workspace sized for %d occupied columns, got %d", ncpad, nocc);
  DF_REQUIRE(ncpad <= 256, DF_ERR_ARG, "mixed K: more than 256 occupied orbitals per call is not supported");
  DF_REQUIRE(NP >= 3 && NP <= 5, DF_ERR_ARG, "mixed K: %d planes", NP);
  DF_CUDA(cudaMemsetAsync(w.err, 0, sizeof(int), s));
  DF_CUDA(cudaMemsetAsync(w.xmax, 0, sizeof(unsigned) * (size_t)npad, s));
  PlanePtrs cpp{}, xpp{};
  for (int j = 0; j < NP; ++j) {
    cpp.p[j] = (__nv_bfloat16*)w.Cp[j];
    xpp.p[j] = (__nv_bfloat16*)w.Xp[j];
  }
  pack_ct_kernel<<<(unsigned)ncpad, 256, 0, s>>>(C, nao, nocc, npad, NP, cpp);
  DF_LAUNCHED("pack_ct_kernel");
  // column tiles of the half transform: two stages in the ring and two accumulators of N
  // columns in 512 TMEM columns
  // knob "ht_n" (a multiple of 16) caps the tile width below the widest that fits
  const int forced = knob("ht_n");
  const int maxN = forced >= 16 ? std::min(ht_max_n(NP), forced / 16 * 16) : ht_max_n(NP);
  const int ntc = (ncpad + maxN - 1) / maxN;
  const int Nht = ((ncpad + ntc - 1) / ntc + 15) / 16 * 16;
  const char* base = (const char*)B;
  umma::Maps maps{};
  // half transform: A = B planes [(P, m)][n], B = C^T [i][n]
  for (int j = 0; j < NP; ++j) {
    DF_TRY(make_map(&maps.a[j], base + L.offp[j], npad, (uint64_t)naux * npad, npad, umma::BM, umma::bk_of(NP)));
    DF_TRY(make_map(&maps.b[j], w.Cp[j], npad, ncpad, npad, Nht, umma::bk_of(NP)));
  }
  umma::Params p{};
  p.mode = umma::HALF_TRANSFORM;
  p.N = Nht;
  const int bk = umma::bk_of(NP);
  p.num_kb = npad / bk;
  p.kb_per_split = p.num_kb;
  p.npad = npad;
  p.ncx = ncpad;
  p.ldx = (long)naux * ncpad;
  p.X32 = w.X32;
  p.xsize = (long)npad * naux * ncpad;
  p.xmax = w.xmax;
  p.err = w.err;
  long mtiles = (long)naux * npad / umma::BM;
  DF_REQUIRE(mtiles < (1L << 31), DF_ERR_ARG, "mixed K: too many row tiles");
  {
    ProfScope ps("k_halftransform_tc", s);
    const dim3 grid((unsigned)mtiles, (unsigned)ntc);
    if (NP == 5) DF_TRY((launch_gemm<5, 32>(maps, p, grid, s)));
    else if (NP == 4) DF_TRY((launch_gemm<4, 32>(maps, p, grid, s)));
    else DF_TRY((launch_gemm<3, 64>(maps, p, grid, s)));
  }
  {
    const long kd = (long)naux * ncpad;
    DF_REQUIRE(npad <= 65535, DF_ERR_ARG, "mixed K: npad %d too large", npad);
    ProfScope ps("k_x_planes", s);
    dim3 grid((unsigned)std::min<long>((kd / 4 + 255) / 256, 64L), (unsigned)npad);
    const float* x0 = w.X32;
    const float* x1 = w.X32 + (size_t)npad * kd;
    if (NP == 5) x_to_planes_kernel<5><<<grid, 256, 0, s>>>(x0, x1, w.xmax, kd, xpp);
    else if (NP == 4) x_to_planes_kernel<4><<<grid, 256, 0, s>>>(x0, x1, w.xmax, kd, xpp);
    else x_to_planes_kernel<3><<<grid, 256, 0, s>>>(x0, x1, w.xmax, kd, xpp);
    DF_LAUNCHED("x_to_planes_kernel");
  }
  // exchange SYRK: A = B = X [m][(P, i)], lower tiles of 128 x syrk_n, split over (P, i).
  // Knob "syrk_bk" = 16: K boxes of 16 elements (32-byte swizzle), stages half as wide, so
  // twice as many k-blocks are in flight to hide the refills from L2.
  long kdim = (long)naux * ncpad;
  const int ns = syrk_n(NP);
  // knob "syrk_pair": 256 x 128 blocks on CTA pairs (cta_group::2), K boxes of bk
  const bool pair = knob("syrk_pair") != 0;
  const int sbk = !pair && knob("syrk_bk") == 16 ? 16 : bk;
  for (int j = 0; j < NP; ++j) {
    DF_TRY(make_map(&maps.a[j], w.Xp[j], kdim, npad, kdim, umma::BM, sbk));
    DF_TRY(make_map(&maps.b[j], w.Xp[j], kdim, npad, kdim, pair ? umma::BM / 2 : ns, sbk));
  }
  umma::Params q{};
  q.mode = umma::SYRK;
  q.N = ns;
  q.num_kb = (int)((kdim + sbk - 1) / sbk);
  q.kb_per_split = (q.num_kb + w.nsplit - 1) / w.nsplit;
  int nsplit = (q.num_kb + q.kb_per_split - 1) / q.kb_per_split;
  q.npad = npad;
  q.Kpart = w.Kpart;
  q.n_lower_tiles = syrk_tiles(npad, NP);
  q.err = w.err;
  if (pair) {
    ProfScope ps("k_syrk_tc", s);
    dim3 grid((unsigned)(2 * pair_blocks(npad)), (unsigned)nsplit);
    if (NP == 5) DF_TRY((launch_syrk_pair<5, 32>(maps, q, grid, s)));
    else if (NP == 4) DF_TRY((launch_syrk_pair<4, 32>(maps, q, grid, s)));
    else DF_TRY((launch_syrk_pair<3, 64>(maps, q, grid, s)));
  } else {
    ProfScope ps("k_syrk_tc", s);
    dim3 grid((unsigned)q.n_lower_tiles, (unsigned)nsplit);
    if (sbk == 16) {
      if (NP == 5) DF_TRY((launch_gemm<5, 16>(maps, q, grid, s)));
      else if (NP == 4) DF_TRY((launch_gemm<4, 16>(maps, q, grid, s)));
      else DF_TRY((launch_gemm<3, 16>(maps, q, grid, s)));
    } else {
      if (NP == 5) DF_TRY((launch_gemm<5, 32>(maps, q, grid, s)));
      else if (NP == 4) DF_TRY((launch_gemm<4, 32>(maps, q, grid, s)));
      else DF_TRY((launch_gemm<3, 64>(maps, q, grid, s)));
    }
  }
  long nn = (long)nao * nao;
  kmixed_reduce_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(w.Kpart, nsplit, npad, nao, w.err, K);
  DF_LAUNCHED("kmixed_reduce_kernel");
  return DF_OK;
}

}  // namespace dfscf

DF_BOUNDS_READER(bounds_read_umma)
