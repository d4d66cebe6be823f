// Shared helpers of the CUDA library: error reporting, launch checks, small math.
#pragma once
#include <cuda_runtime.h>
#include <cstdarg>
#include <cstddef>
#include <cstdint>
#include <cstdio>

#include "dfscf.h"

namespace dfscf {

void set_error(const char* fmt, ...);
void clear_error();

// Tuning knob value by name (api.cu); 0 for an unknown name.
int knob(const char* name);

// Phase profiler (api.cu): CUDA events around kernel phases when enabled.
bool prof_on();
void* prof_begin(const char* name, cudaStream_t s);
void prof_end(void* tok, cudaStream_t s);
struct ProfScope {
  void* tok;
  cudaStream_t s;
  ProfScope(const char* name, cudaStream_t st) : tok(prof_begin(name, st)), s(st) {}
  ~ProfScope() { prof_end(tok, s); }
};

constexpr double kPi = 3.14159265358979323846;

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
inline long npair_of(int nao) { return (long)nao * (nao + 1) / 2; }

// Bump allocator over a caller-owned workspace; every slice is 256-byte aligned.
struct Arena {
  char* base;
  size_t size;
  size_t used = 0;
  bool overflow = false;
  Arena(void* b, size_t s) : base((char*)b), size(s) {}
  template <typename T>
  T* take(size_t count) {
    size_t off = align_up(used, 256);
    size_t bytes = align_up(count * sizeof(T), 256);
    used = off + bytes;
    if (used > size || base == nullptr) {
      overflow = true;
      return nullptr;
    }
    return (T*)(base + off);
  }
};

// Size-only twin of Arena used by the *_work_bytes queries.
struct Sizer {
  size_t used = 0;
  template <typename T>
  void take(size_t count) {
    used = align_up(used, 256) + align_up(count * sizeof(T), 256);
  }
};

}  // namespace dfscf

#define DF_CUDA(expr)                                                                           \
  do {                                                                                          \
    cudaError_t e_ = (expr);                                                                    \
    if (e_ != cudaSuccess) {                                                                    \
      dfscf::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return DF_ERR_CUDA;                                                                       \
    }                                                                                           \
  } while (0)

#define DF_LAUNCHED(name)                                                                       \
  do {                                                                                          \
    cudaError_t e_ = cudaGetLastError();                                                        \
    if (e_ != cudaSuccess) {                                                                    \
      dfscf::set_error("launch of %s failed: %s (%s:%d)", name, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return DF_ERR_CUDA;                                                                       \
    }                                                                                           \
  } while (0)

#define DF_REQUIRE(cond, code, ...)   \
  do {                                \
    if (!(cond)) {                    \
      dfscf::set_error(__VA_ARGS__);  \
      return code;                    \
    }                                 \
  } while (0)

#define DF_TRY(expr)              \
  do {                            \
    int rc_ = (expr);             \
    if (rc_ != DF_OK) return rc_; \
  } while (0)

// ---- bounds-checked indexing (checking build) -------------------------------------------
// Built with -DDFSCF_BOUNDS_CHECK, DF_IX(i, n) checks 0 <= i < n.  A bad index is counted in
// this translation unit's record (the first one with its bound and source line is kept)
// and replaced by 0, so the access stays inside the buffer and the run goes on; the host
// reads the records with df_bounds_violations().  In the normal build DF_IX(i, n) is i.
namespace dfscf {
struct BoundsRecord {
  unsigned long long count;
  long long index, bound;
  int line, pad;
};
// Reads and clears this translation unit's record (all zero in the normal build).
typedef int (*BoundsReader)(BoundsRecord* out);
}  // namespace dfscf

#ifdef DFSCF_BOUNDS_CHECK
static __device__ dfscf::BoundsRecord g_df_bounds;
// An access of w consecutive elements starting at i: 0 <= i and i + w <= n.
__device__ __forceinline__ long long df_ixw(long long i, long long w, long long n, int line) {
  if (i >= 0 && i + w <= n) return i;
  if (atomicAdd(&g_df_bounds.count, 1ull) == 0ull) {
    g_df_bounds.index = i;
    g_df_bounds.bound = n;
    g_df_bounds.line = line;
  }
  return 0;
}
#define DF_IX(i, n) df_ixw((long long)(i), 1, (long long)(n), __LINE__)
#define DF_IXW(i, w, n) df_ixw((long long)(i), (long long)(w), (long long)(n), __LINE__)
#define DF_BOUNDS_READER(name)                                                            \
  namespace dfscf {                                                                       \
  int name(BoundsRecord* out) {                                                           \
    if (cudaMemcpyFromSymbol(out, g_df_bounds, sizeof(BoundsRecord)) != cudaSuccess) return DF_ERR_CUDA; \
    BoundsRecord zero{};                                                                  \
    if (cudaMemcpyToSymbol(g_df_bounds, &zero, sizeof(BoundsRecord)) != cudaSuccess) return DF_ERR_CUDA; \
    return DF_OK;                                                                         \
  }                                                                                       \
  }
#else
#define DF_IX(i, n) (i)
#define DF_IXW(i, w, n) (i)
#define DF_BOUNDS_READER(name)            \
  namespace dfscf {                       \
  int name(BoundsRecord* out) {           \
    *out = BoundsRecord{};                \
    return DF_OK;                         \
  }                                       \
  }
#endif

// ---- device helpers ----------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum; every thread gets the total.  `sh` needs blockDim.x/32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < nw; ++i) t += sh[i];
  return t;
}

// Unpack packed lower-triangle index ij = m(m+1)/2 + n (m >= n).
__device__ __forceinline__ void unpack_pair(long ij, int& m, int& n) {
  int mm = (int)((sqrt(8.0 * (double)ij + 1.0) - 1.0) * 0.5);
  while ((long)mm * (mm + 1) / 2 > ij) --mm;
  while ((long)(mm + 1) * (mm + 2) / 2 <= ij) ++mm;
  m = mm;
  n = (int)(ij - (long)mm * (mm + 1) / 2);
}
