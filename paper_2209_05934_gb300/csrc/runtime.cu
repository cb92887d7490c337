// Process-wide bookkeeping of the library (host side).
#include <stdarg.h>
#include <stdio.h>

#include <atomic>

#include "omm_internal.cuh"

namespace omm {
namespace {
std::atomic<int64_t> g_launches{0};
}
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }
void count_launch(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

namespace {
thread_local char g_err[512] = "";
}
void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
}  // namespace omm

extern "C" const char *omm_last_error(void) { return omm::g_err; }
