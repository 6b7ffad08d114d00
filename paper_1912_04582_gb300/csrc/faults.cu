// Host-side fault injection: makes the library's error paths reachable in tests
// without any device fault.  Every injected failure happens on the host, at the
// point where the real failure would be detected: a device allocation reported
// as out of memory, the device error flag reported as set by a bulk-copy wait
// that ran out, or the serving loop's admission check reporting the budget as
// full.  Process-wide; each kind disarms itself after it has fired.
#include <atomic>

#include "dvm_internal.h"

namespace dvm {
namespace {
// operations of each kind to let through before the next one fails (-1: off)
std::atomic<int64_t> g_alloc{-1}, g_timeout{-1};
// admission checks still to be answered "budget full"
std::atomic<int64_t> g_admit{0};

bool countdown(std::atomic<int64_t> &c) {
  int64_t v = c.load();
  while (v >= 0)
    if (c.compare_exchange_weak(v, v - 1)) return v == 0;
  return false;
}
}  // namespace

bool fault_alloc() { return countdown(g_alloc); }
bool fault_timeout() { return countdown(g_timeout); }
bool fault_admit() {
  int64_t v = g_admit.load();
  while (v > 0)
    if (g_admit.compare_exchange_weak(v, v - 1)) return true;
  return false;
}
}  // namespace dvm

extern "C" int dvm_fault_inject(int32_t kind, int64_t count) {
  switch (kind) {
    case DVM_FAULT_NONE:
      dvm::g_alloc = -1;
      dvm::g_timeout = -1;
      dvm::g_admit = 0;
      return DVM_OK;
    case DVM_FAULT_ALLOC:
      dvm::g_alloc = count < 0 ? -1 : count;
      return DVM_OK;
    case DVM_FAULT_TIMEOUT:
      dvm::g_timeout = count < 0 ? -1 : count;
      return DVM_OK;
    case DVM_FAULT_ADMIT:
      dvm::g_admit = count < 0 ? 0 : count;
      return DVM_OK;
    default:
      dvm::set_error("dvm_fault_inject: unknown kind");
      return DVM_ERR_INVALID_ARG;
  }
}
