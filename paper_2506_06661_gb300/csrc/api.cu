// Thread-local error text and version of the C ABI.
#include <cstdarg>
#include <cstdio>

#include "common.cuh"

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
