// ch_fault.cu -- host-side fault injection (ch_set_fault, environment variable CH_FAULT).
//
// Failures are made on the host, never on the device: an allocation of the library that
// reports failure without allocating, a NaN written into a member's field through an
// ordinary host-to-device copy, and a stall of the serving worker's host thread.  Each
// exercises the error path that a real failure takes (CH_ENOMEM with everything already
// allocated released, CH_ENONFINITE from the FP64 observables, CH_ETIMEOUT from a bounded
// host wait) without faulting, trapping or hanging a GPU.
#include <atomic>
#include <cerrno>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>

#include <cuda_runtime.h>

#include "ch.h"
#include "ch_internal.h"

namespace chk {
void record_error(const char* msg);  // ch_api.cu
}

namespace {

// Armed fault: its kind, the count of events before it fires (alloc), its argument (the
// member for nan, milliseconds for timeout).  One fault at a time, process-wide.
std::mutex g_mu;
int g_kind = chk::kFaultNone;
int64_t g_arg = 0;
std::once_flag g_env_once;

// "alloc[:N]", "nan[:M]", "timeout[:MS]"; empty or "none" disarms.  Returns false on a
// malformed spec.
bool parse(const char* spec, int* kind, int64_t* arg) {
  if (!spec || !*spec || std::strcmp(spec, "none") == 0) {
    *kind = chk::kFaultNone;
    *arg = 0;
    return true;
  }
  const char* colon = std::strchr(spec, ':');
  const std::string name = colon ? std::string(spec, colon - spec) : std::string(spec);
  int64_t value = -1;
  if (colon) {
    char* end = nullptr;
    errno = 0;
    const long long v = std::strtoll(colon + 1, &end, 10);
    if (errno || !end || *end || end == colon + 1 || v < 0) return false;
    value = v;
  }
  if (name == "alloc") {
    *kind = chk::kFaultAlloc;
    *arg = value < 0 ? 1 : value;
    return *arg >= 1;
  }
  if (name == "nan") {
    *kind = chk::kFaultNan;
    *arg = value < 0 ? 0 : value;
    return true;
  }
  if (name == "timeout") {
    *kind = chk::kFaultTimeout;
    *arg = value < 0 ? 2000 : value;
    return true;
  }
  return false;
}

void arm_from_env() {
  std::call_once(g_env_once, [] {
    const char* env = std::getenv("CH_FAULT");
    int kind;
    int64_t arg;
    if (env && parse(env, &kind, &arg)) {
      g_kind = kind;
      g_arg = arg;
    }
  });
}

}  // namespace

namespace chk {

cudaError_t dev_malloc(void** p, size_t bytes) {
  {
    std::lock_guard<std::mutex> lk(g_mu);
    arm_from_env();
    if (g_kind == kFaultAlloc && --g_arg == 0) {
      g_kind = kFaultNone;  // fires once
      *p = nullptr;
      return cudaErrorMemoryAllocation;
    }
  }
  return cudaMalloc(p, bytes);
}

int take_fault(int kind, int64_t* arg) {
  std::lock_guard<std::mutex> lk(g_mu);
  arm_from_env();
  if (g_kind != kind) return 0;
  if (arg) *arg = g_arg;
  g_kind = kFaultNone;  // fires once
  return 1;
}

cudaError_t inject_nan(void* C, int precision, const MemberParams* mp, int m, cudaStream_t st) {
  int64_t member = 0;
  if (!take_fault(kFaultNan, &member)) return cudaSuccess;
  if (member < 0 || member >= m) member = 0;
  const int64_t at = mp[member].offset;  // the member's first grid point
  if (precision == CH_FP64) {
    static const double nan64 = std::nan("");
    return cudaMemcpyAsync(static_cast<double*>(C) + at, &nan64, sizeof nan64, cudaMemcpyHostToDevice, st);
  }
  static const float nan32 = std::nanf("");
  return cudaMemcpyAsync(static_cast<float*>(C) + at, &nan32, sizeof nan32, cudaMemcpyHostToDevice, st);
}

void stall_if_armed() {
  int64_t ms = 0;
  if (take_fault(kFaultTimeout, &ms)) std::this_thread::sleep_for(std::chrono::milliseconds(ms));
}

}  // namespace chk

extern "C" int ch_set_fault(const char* spec) {
  int kind;
  int64_t arg;
  if (!parse(spec, &kind, &arg)) {
    chk::record_error("ch_set_fault: expected alloc[:N] (N >= 1), nan[:member], timeout[:ms] or none");
    return CH_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  arm_from_env();  // the environment applies once, before the first explicit setting
  g_kind = kind;
  g_arg = arg;
  return CH_OK;
}
