// Thread-local last-error message of the C ABI.
#include <cstdarg>
#include <cstdio>

#include "rift_ile_internal.h"

namespace {
thread_local char g_last_error[512] = "";
}

void rift_ile_set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
}

extern "C" const char* rift_ile_last_error(void) { return g_last_error; }
