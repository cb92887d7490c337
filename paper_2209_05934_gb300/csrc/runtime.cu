// Process-wide bookkeeping of the library (host side).
#include <atomic>

#include "omm_internal.cuh"

namespace omm {
namespace {
std::atomic<int64_t> g_launches{0};
}
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }
void count_launch(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
}  // namespace omm
