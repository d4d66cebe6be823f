// Coulomb build with library-owned scratch: the allocation-free variant of df_jk's J.
//
// Some callers cannot hand this library a workspace: plugins hosted inside a framework
// that owns every device allocation through its own allocator, and long-running
// latency-critical services whose policy forbids device allocation (cudaMalloc may
// synchronise the whole device) once they are running.  df_j_noalloc serves them: it
// computes the same FP64 Coulomb matrix as df_jk, with its scratch (weighted packed
// density, fitting coefficients d_P, per-split partial J) in one fixed array that the
// library declares at file scope below.  Every GPU that loads the library reserves that
// array until the process exits.
//
// The array lives in device memory, so host code cannot use the symbol itself as an
// address; the device address is obtained with cudaGetSymbolAddress (with the device
// current) and passed to the kernels.  Outside a stream capture every call looks it up
// again, so a context torn down and recreated (cudaDeviceReset) gets its new address; inside
// a capture the call reuses the address of the last call on that device, so one call must
// come before the first capture.  All calls share the one
// array: two calls whose GPU work overlaps (different streams, or different host threads
// on the same device without ordering) race on it and give wrong results.  Nothing in the
// array needs to start at zero: every word a call reads was written earlier in that call.
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace dfscf {

constexpr size_t NOALLOC_DOUBLES = (size_t)1 << 20;  // 8 MiB of scratch per device

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

static std::mutex g_noalloc_mutex;
static double* g_noalloc_ptr[256];

// Device address of the scratch array on the current device: looked up on every call made
// outside a stream capture (and remembered), reused from the last such call inside one.
static int noalloc_scratch(cudaStream_t s, double** out) {
  int dev = 0;
  DF_CUDA(cudaGetDevice(&dev));
  DF_REQUIRE(dev >= 0 && dev < 256, DF_ERR_ARG, "df_j_noalloc: device index %d out of range", dev);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  DF_CUDA(cudaStreamIsCapturing(s, &cs));
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (cs == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    DF_REQUIRE(e == cudaSuccess && p, DF_ERR_CUDA, "df_j_noalloc: cudaGetSymbolAddress failed: %s",
               cudaGetErrorString(e));
    g_noalloc_ptr[dev] = (double*)p;
  }
  DF_REQUIRE(g_noalloc_ptr[dev], DF_ERR_ARG,
             "df_j_noalloc: first call on device %d made inside a stream capture; call it once before capturing",
             dev);
  *out = g_noalloc_ptr[dev];
  return DF_OK;
}

// Scratch doubles for one call: Dw (ld), d (naux), Jpart (splits x ld), each on 32-double
// (256-byte) boundaries; splits = ceil(naux / 256) as in df_jk's second J pass.
static size_t noalloc_need(int nao, int naux, long* ld_out, int* nsplit_out) {
  long ld = B_ld(nao);
  int nsplit = (naux + 255) / 256;
  *ld_out = ld;
  *nsplit_out = nsplit;
  return align_up((size_t)ld, 32) + align_up((size_t)naux, 32) + (size_t)nsplit * align_up((size_t)ld, 32);
}

}  // namespace dfscf

using namespace dfscf;

extern "C" size_t df_j_noalloc_capacity(void) { return NOALLOC_DOUBLES * sizeof(double); }

extern "C" int df_j_noalloc(const void* B, int nao, int naux, const double* D, double* J, cudaStream_t s) {
  clear_error();
  DF_REQUIRE(B && D && J && nao > 0 && naux > 0, DF_ERR_ARG, "df_j_noalloc: bad arguments");
  long ld = 0;
  int nsplit = 0;
  size_t need = noalloc_need(nao, naux, &ld, &nsplit);
  DF_REQUIRE(need <= NOALLOC_DOUBLES, DF_ERR_ARG,
             "df_j_noalloc: nao %d / naux %d need %zu bytes of scratch, more than the fixed %zu bytes "
             "(use df_jk with a caller workspace)",
             nao, naux, need * sizeof(double), NOALLOC_DOUBLES * sizeof(double));
  double* base = nullptr;
  DF_TRY(noalloc_scratch(s, &base));
  JKWork w{};
  w.Dw = base;
  w.d = base + align_up((size_t)ld, 32);
  w.Jpart = w.d + align_up((size_t)naux, 32);
  w.nsplit_j = nsplit;
  return build_J(B, B_layout(nao, naux, DF_FP64, 0), nao, naux, DF_FP64, D, J, w, s);
}
