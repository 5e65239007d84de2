// me_noalloc.cu -- me_compute_noalloc: the me_compute computation with no device
// allocation anywhere on its path.
//
// me_compute keeps a per-stream workspace that it grows with cudaMallocAsync.  Some
// callers cannot allow that: a host framework that owns all device memory through its
// own pool and forbids direct driver allocations, or a caller running under a hard
// memory cap or a latency budget, where an allocation may fail or stall.  For them the
// scratch the kernels need (running helicity sums for the selection, the global slot
// buffer of the large processes, the per-event momentum table, colour weights) lives
// in one fixed device array declared in this file.  It is created when the library's
// device code is loaded on a GPU and stays there until the process exits.
#include <cuda.h>  // CUcontext and the driver call signatures (resolved at run time)
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/me.h"
#include "me_internal.h"
#include "me_kernels.cuh"

using namespace meb300;
using namespace meb300::detail;

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;  // 32 MiB, the stated maximum

// The fixed scratch.  In host code this name is a host-side stand-in, not a device
// address: the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
// per device: the device address of the scratch and the id of the CUDA context it
// belongs to.  A device reset (or a primary context torn down and made again) gives the
// device a new context with a new id, and the address is then looked up again.
void* g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};

// the unique id of the current CUDA context (0 if there is none or it cannot be read);
// the two driver calls are resolved through the runtime, so the library does not link
// the driver library itself
unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool resolved = false;
  if (!resolved) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
    cudaGetLastError();
    resolved = true;
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// Device address of the scratch on the current device, looked up once per device and
// context (the argument checks before this have made the device's context current).
int scratch_address(me_handle* h, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(h, e, "me_compute_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(h, ME_ERR_ARG, "me_compute_noalloc: device index out of range");
  std::lock_guard<std::mutex> g(g_mu);
  const unsigned long long ctx = current_context_id();
  if (!g_scratch_addr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return cuda_fail(h, e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                       "me_compute_noalloc: cudaGetSymbolAddress of the fixed scratch");
    }
    g_scratch_addr[dev] = p;
    g_scratch_ctx[dev] = current_context_id();
  }
  *out = g_scratch_addr[dev];
  return ME_OK;
}

// The largest batch whose scratch fits the fixed array (0 if not even one event does).
// The plan's scratch never shrinks as the batch grows (the main pass grows with
// min(events, resident threads), the rescue list with the events), so a bisection over
// the planner, host arithmetic only, finds it.
int64_t largest_batch(const me_handle* h, bool want_hel, bool want_col) {
  auto fits = [&](int64_t n) { return plan_call(h, n, n, want_hel, want_col).total <= kScratchBytes; };
  if (!fits(1)) return 0;
  int64_t lo = 1, hi = INT32_MAX;  // fits(lo); the answer is in [lo, hi]
  if (fits(hi)) return hi;
  while (hi - lo > 1) {
    const int64_t mid = lo + (hi - lo) / 2;
    (fits(mid) ? lo : hi) = mid;
  }
  return lo;
}

}  // namespace

extern "C" int me_compute_noalloc(me_handle* h, int64_t nevt, const double* momenta, const double* alphas,
                                  const double* rnd_hel, const double* rnd_col, double* me, int32_t* sel_hel,
                                  int32_t* sel_col, void* cuda_stream) {
  if (!h) return fail(nullptr, ME_ERR_ARG, "me_compute_noalloc: null handle");
  if (nevt < 0) return fail(h, ME_ERR_ARG, "me_compute_noalloc: nevt < 0");
  if (nevt == 0) return ME_OK;
  if (nevt > INT32_MAX) return fail(h, ME_ERR_ARG, "me_compute_noalloc: more than 2^31 - 1 events in one call");
  if (!momenta || !me) return fail(h, ME_ERR_ARG, "me_compute_noalloc: momenta and me are required");
  if (reinterpret_cast<uintptr_t>(momenta) % 16)
    return fail(h, ME_ERR_ARG, "me_compute_noalloc: momenta must be 16-byte aligned");
  if ((sel_hel && !rnd_hel) || (sel_col && !rnd_col))
    return fail(h, ME_ERR_ARG, "me_compute_noalloc: a selection output needs its random numbers");
  const void* ptrs[] = {momenta, me, alphas, rnd_hel, rnd_col, sel_hel, sel_col};
  for (const void* p : ptrs)
    if (p && !is_device_ptr(p)) return fail(h, ME_ERR_ARG, "me_compute_noalloc: arrays must be device memory");
  if (h->err_host && *h->err_host) {
    *h->err_host = 0;
    return fail(h, ME_ERR_TIMEOUT, "me_compute_noalloc: a device-side wait of an earlier call on this handle "
                                   "timed out; its events were set to NaN");
  }
  const int ngood = int(h->good.size());
  const bool want_hel = sel_hel && rnd_hel;
  const bool want_col = sel_col && rnd_col;
  // one persistent main launch (plus the FP64 rescue pass of the FP32 and mixed modes):
  // its scratch, one row per resident thread, must fit the fixed array
  const CallPlan cp = plan_call(h, nevt, nevt, want_hel, want_col);
  if (cp.total > kScratchBytes) {
    char msg[320];
    std::snprintf(msg, sizeof msg,
                  "me_compute_noalloc: %lld events need %zu bytes of scratch, more than the fixed %zu bytes; "
                  "at most %lld events of this process, mode and choice of selection outputs fit in one call",
                  static_cast<long long>(nevt), cp.total, kScratchBytes,
                  static_cast<long long>(largest_batch(h, want_hel, want_col)));
    return fail(h, ME_ERR_ARG, msg);
  }
  void* scratch = nullptr;
  int rc = scratch_address(h, &scratch);
  if (rc) return rc;
  // Nothing in the scratch has to start at zero: the kernels write every running sum,
  // colour weight, slot and momentum-table entry of an event before they read it, and
  // the rescue counter is cleared on the stream at the start of every call.
  MeLaunch a{};
  fill_common(h, a);
  a.err = h->err_dev;
  a.mom = momenta;
  a.alphas = alphas;
  a.rnd_hel = rnd_hel;
  a.rnd_col = rnd_col;
  a.me = me;
  a.sel_hel = want_hel ? sel_hel : nullptr;
  a.sel_col = want_col ? sel_col : nullptr;
  a.ngood = ngood;
  for (int i = 0; i < ngood; ++i) a.good[i] = uint8_t(h->good[i]);
  cudaError_t e = run_call(h, cp, a, nevt, scratch, static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return cuda_fail(h, e, "me_compute_noalloc launch");
  return ME_OK;
}
