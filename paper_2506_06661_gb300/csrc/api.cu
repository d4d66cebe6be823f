// Thread-local error text and version of the C ABI.
#include <cstdarg>
#include <cstdio>

#include "common.cuh"
#include "kernels.cuh"

namespace dfscf {

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

void clear_error() { g_err[0] = '\0'; }

}  // namespace dfscf

extern "C" const char* df_last_error(void) { return dfscf::g_err; }
extern "C" int df_version(void) { return 100; }

// ---- phase profiler ----------------------------------------------------------------
// When enabled, launch sites bracket their kernels with CUDA events on the launching
// stream; df_profile_* sum the elapsed times per phase name.
#include <cstring>
#include <string>
#include <vector>

namespace dfscf {

struct ProfEntry {
  std::string name;
  cudaEvent_t a, b;
};
static bool g_prof_on = false;
static std::vector<ProfEntry> g_prof;
static std::vector<std::pair<std::string, double>> g_prof_sum;
static std::vector<std::pair<std::string, long>> g_prof_cnt;

bool prof_on() { return g_prof_on; }

void* prof_begin(const char* name, cudaStream_t s) {
  if (!g_prof_on) return nullptr;
  ProfEntry e{name, nullptr, nullptr};
  cudaEventCreate(&e.a);
  cudaEventCreate(&e.b);
  cudaEventRecord(e.a, s);
  g_prof.push_back(e);
  return (void*)(g_prof.size());
}

void prof_end(void* tok, cudaStream_t s) {
  if (!g_prof_on || !tok) return;
  size_t i = (size_t)tok - 1;
  if (i < g_prof.size()) cudaEventRecord(g_prof[i].b, s);
}

static void prof_collect() {
  for (auto& e : g_prof) {
    cudaEventSynchronize(e.b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e.a, e.b);
    bool found = false;
    for (size_t k = 0; k < g_prof_sum.size(); ++k)
      if (g_prof_sum[k].first == e.name) {
        g_prof_sum[k].second += ms;
        g_prof_cnt[k].second += 1;
        found = true;
      }
    if (!found) {
      g_prof_sum.push_back({e.name, (double)ms});
      g_prof_cnt.push_back({e.name, 1});
    }
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  g_prof.clear();
}

}  // namespace dfscf

extern "C" void df_profile_enable(int on) {
  dfscf::prof_collect();
  dfscf::g_prof_on = on != 0;
}

extern "C" void df_profile_reset(void) {
  dfscf::prof_collect();
  dfscf::g_prof_sum.clear();
  dfscf::g_prof_cnt.clear();
}

extern "C" int df_profile_count(void) {
  dfscf::prof_collect();
  return (int)dfscf::g_prof_sum.size();
}

extern "C" const char* df_profile_name(int i) {
  if (i < 0 || i >= (int)dfscf::g_prof_sum.size()) return "";
  return dfscf::g_prof_sum[i].first.c_str();
}

extern "C" double df_profile_ms(int i) {
  if (i < 0 || i >= (int)dfscf::g_prof_sum.size()) return 0.0;
  return dfscf::g_prof_sum[i].second;
}

extern "C" long df_profile_calls(int i) {
  if (i < 0 || i >= (int)dfscf::g_prof_cnt.size()) return 0;
  return dfscf::g_prof_cnt[i].second;
}

// ---- tuning knobs ---------------------------------------------------------------------
// Launch parameters the autotuner may change between calls.  0 means "use the built-in
// heuristic" where that is allowed.
namespace dfscf {

struct Knob {
  const char* name;
  int value, lo, hi;
  int def = -1;  // the built-in value, recorded at the first df_tune_set / df_tune_reset
};
static Knob g_knobs[] = {
    {"umma_max_stages", 8, 2, 8},    // largest shared-memory ring depth of the tcgen05 GEMM (as many as fit)
    {"syrk_bk", 32, 16, 32},         // K box of the tcgen05 exchange SYRK: 32, or 16 for a deeper ring
    {"syrk_split", 0, 0, 4096},      // K-dimension splits of the tcgen05 exchange SYRK
    {"syrk_pair", 0, 0, 1},          // exchange SYRK on CTA pairs (cta_group::2, 256 x 128 blocks); 0: one CTA per 128 x 128 tile
    {"fp64_syrk_split", 0, 0, 4096}, // K-dimension splits of the FP64 exchange SYRK
    {"jpass2_rows", 256, 32, 512},   // auxiliary rows per CTA slice of J's second pass
    {"j_fp64_fma", 0, 0, 1},         // J passes: 0 double-float products on FP32 units, 1 FP64 FMAs
    {"jpass1_rows", 1, 1, 8},        // auxiliary rows per CTA of J's first pass (1, 2, 4 or 8)
    {"fp64_ht_cols", 0, 0, 32},      // FP64 half-transform tile columns: 0 auto, 16 or 32
    {"dm0_eig_cut", 12, 1, 16},      // first exchange of a fractional dm0: occupations below 10^-cut dropped
    {"guess_idem_max", 200, 1, 1000},// largest idempotency error of an accepted dm0, in hundredths
    {"ht_n", 0, 0, 256},             // tcgen05 half-transform tile columns: 0 widest that fits, else a cap
    {"eig_ctas", 0, 0, 4096},        // CTAs of the multi-SM eigensolver (0 auto, 1 single CTA)
    {"mixed_planes", 5, 3, 5},       // BF16 planes per operand of the mixed exchange (3, 4, 5: 6, 10, 15 products)
    {"mixed_incremental", 1, 0, 1},  // mixed SCF: update K from the change of the occupied projector
    {"soscf", 1, 0, 1},              // switch from DIIS to Newton steps when DIIS stalls
    {"soscf_cg", 6, 1, 64},          // conjugate-gradient iterations per Newton step
    {"stability", 0, 0, 2},          // lowest orbital-Hessian eigenvalue of every converged solution (2: leave saddles)
    {"stability_steps", 60, 2, 400}, // Hessian products allowed to that analysis (Davidson)
    {"eig_barrier_polls", 1 << 22, 256, 1 << 30},  // polls before a grid-barrier wait of the eigensolver gives up
    {"eig_barrier_extra", 0, 0, 1},  // test hook: 1 = every eigensolver grid barrier waits for one arrival
                                     // that never comes, so its bounded wait runs out
};

int knob(const char* name) {
  for (auto& k : g_knobs)
    if (strcmp(k.name, name) == 0) return k.value;
  return 0;
}

}  // namespace dfscf

namespace dfscf {
static void record_defaults() {
  static bool done = false;
  if (done) return;
  for (auto& k : g_knobs) k.def = k.value;
  done = true;
}
}  // namespace dfscf

extern "C" void df_tune_reset(void) {
  dfscf::record_defaults();
  for (auto& k : dfscf::g_knobs) k.value = k.def;
}

extern "C" int df_tune_set(const char* name, int value) {
  dfscf::clear_error();
  if (!name) return DF_ERR_ARG;
  dfscf::record_defaults();
  for (auto& k : dfscf::g_knobs)
    if (strcmp(k.name, name) == 0) {
      if (value < k.lo || value > k.hi) {
        dfscf::set_error("df_tune_set: %s = %d outside [%d, %d]", name, value, k.lo, k.hi);
        return DF_ERR_ARG;
      }
      k.value = value;
      return DF_OK;
    }
  dfscf::set_error("df_tune_set: unknown knob '%s'", name);
  return DF_ERR_ARG;
}

extern "C" int df_tune_get(const char* name) {
  if (!name) return -1;
  for (auto& k : dfscf::g_knobs)
    if (strcmp(k.name, name) == 0) return k.value;
  return -1;
}

// ---- bounds-check records -------------------------------------------------------------
extern "C" int df_bounds_checked(void) {
#ifdef DFSCF_BOUNDS_CHECK
  return 1;
#else
  return 0;
#endif
}

extern "C" int df_bounds_violations(unsigned long long* count, char* where, size_t where_bytes) {
  dfscf::clear_error();
  DF_REQUIRE(count, DF_ERR_ARG, "df_bounds_violations: null count");
  struct Unit {
    const char* name;
    dfscf::BoundsReader read;
  };
  const Unit units[] = {{"dferr.cu", dfscf::bounds_read_dferr},   {"eig.cu", dfscf::bounds_read_eig},
                        {"integrals.cu", dfscf::bounds_read_integrals}, {"jk.cu", dfscf::bounds_read_jk},
                        {"linalg.cu", dfscf::bounds_read_linalg}, {"lowdin.cu", dfscf::bounds_read_lowdin},
                        {"lrdf.cu", dfscf::bounds_read_lrdf},     {"mlp.cu", dfscf::bounds_read_mlp},
                        {"scf.cu", dfscf::bounds_read_scf},       {"umma.cu", dfscf::bounds_read_umma}};
  DF_CUDA(cudaDeviceSynchronize());
  *count = 0;
  if (where && where_bytes) where[0] = '\0';
  for (const Unit& u : units) {
    dfscf::BoundsRecord r{};
    DF_TRY(u.read(&r));
    if (r.count && *count == 0 && where && where_bytes)
      snprintf(where, where_bytes, "%s:%d index %lld outside [0, %lld)", u.name, r.line, r.index, r.bound);
    *count += r.count;
  }
  return DF_OK;
}
