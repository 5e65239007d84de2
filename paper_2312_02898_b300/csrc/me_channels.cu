// me_channels.cu -- me_compute_channels: one batch of events that belong to different
// channels (subprocesses) of a hadronic process, each event evaluated by its channel's
// handle, as an event generator for p p -> t t~ needs (g g -> t t~ and the
// quark-initiated q q~ -> t t~ in either beam order, routed per event).
//
// On the stream: the counts per channel are cleared, one kernel partitions the event
// indices by channel into per-channel lists (one atomic per warp and channel; the order
// inside a list does not matter, every event is evaluated on its own), and each channel's main
// kernel then walks its list in indexed mode -- the mode the FP64 rescue pass uses --
// reading that channel's count on the device, so the host never waits for the
// partition.  Results land at the events' own positions.  An FP32 channel runs its FP64
// rescue pass over its flagged events as in me_compute.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>

#include "../../include/me.h"
#include "me_internal.h"
#include "me_kernels.cuh"

using namespace meb300;
using namespace meb300::detail;

namespace {

constexpr int kMaxChannels = 32;  // the counts take the first 256 bytes of the partition buffer (64 ints)

// One atomic per warp and channel: the lanes of a warp that hold the same channel
// (__match_any_sync) take consecutive list positions from one atomicAdd by their lowest
// lane, instead of every event contending for the same few counters.
__global__ void __launch_bounds__(256) partition_channels(int64_t nevt, const int32_t* __restrict__ channel, int nchan,
                                                          int* __restrict__ counts, int* __restrict__ lists,
                                                          double* __restrict__ me, int32_t* __restrict__ sel_hel,
                                                          int32_t* __restrict__ sel_col) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  const unsigned lane = threadIdx.x & 31u;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < nevt; e += stride) {
    const int c = channel[e];
    const bool valid = c >= 0 && c < nchan;
    const unsigned active = __activemask();
    const unsigned peers = __match_any_sync(active, valid ? c : -1);
    if (valid) {
      const int leader = __ffs(peers) - 1;
      int base = 0;
      if (int(lane) == leader) base = atomicAdd(counts + c, __popc(peers));
      base = __shfl_sync(peers, base, leader);
      const int pos = base + __popc(peers & ((1u << lane) - 1u));
      lists[int64_t(c) * nevt + pos] = int(e);
    } else {  // no such channel: the event gets NaN and selections 0
      me[e] = __longlong_as_double(0x7ff8000000000000ll);
      if (sel_hel) sel_hel[e] = 0;
      if (sel_col) sel_col[e] = 0;
    }
  }
}

}  // namespace

extern "C" int me_compute_channels(me_handle* const* hs, int nchan, int64_t nevt, const int32_t* channel,
                                   const double* momenta, const double* alphas, const double* rnd_hel,
                                   const double* rnd_col, double* me, int32_t* sel_hel, int32_t* sel_col,
                                   void* cuda_stream) {
  if (!hs || nchan < 1 || nchan > kMaxChannels)
    return fail(nullptr, ME_ERR_ARG, "me_compute_channels: 1 to 32 handles are required");
  for (int c = 0; c < nchan; ++c)
    if (!hs[c]) return fail(nullptr, ME_ERR_ARG, "me_compute_channels: null handle");
  me_handle* h0 = hs[0];
  if (nevt < 0) return fail(h0, ME_ERR_ARG, "me_compute_channels: nevt < 0");
  if (nevt == 0) return ME_OK;
  if (nevt > (int64_t(1) << 30)) return fail(h0, ME_ERR_ARG, "me_compute_channels: more than 2^30 events in one call");
  if (!channel || !momenta || !me) return fail(h0, ME_ERR_ARG, "me_compute_channels: channel, momenta and me are required");
  if (reinterpret_cast<uintptr_t>(momenta) % 16)
    return fail(h0, ME_ERR_ARG, "me_compute_channels: momenta must be 16-byte aligned");
  if ((sel_hel && !rnd_hel) || (sel_col && !rnd_col))
    return fail(h0, ME_ERR_ARG, "me_compute_channels: a selection output needs its random numbers");
  const void* ptrs[] = {channel, momenta, me, alphas, rnd_hel, rnd_col, sel_hel, sel_col};
  for (const void* p : ptrs)
    if (p && !is_device_ptr(p)) return fail(h0, ME_ERR_ARG, "me_compute_channels: arrays must be device memory");
  for (int c = 0; c < nchan; ++c) {
    me_handle* h = hs[c];
    if (h->ops->npar != h0->ops->npar)
      return fail(h0, ME_ERR_ARG, "me_compute_channels: every channel must have the same number of particles");
    const int prec = h->par.precision;
    if ((prec != ME_PREC_FP64 && prec != ME_PREC_FP32) || h->ops->needs(prec, h->config).ept != 1)
      return fail(h0, ME_ERR_MODE, "me_compute_channels: channels run in FP64 or FP32 with one event per thread");
    if (h->err_host && *h->err_host) {
      *h->err_host = 0;
      return fail(h0, ME_ERR_TIMEOUT, "me_compute_channels: a device-side wait of an earlier call on a channel "
                                      "handle timed out");
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // partition buffers: per-channel counts, then per-channel index lists of nevt entries
  const size_t off_lists = 256;
  const size_t bytes = off_lists + size_t(nchan) * size_t(nevt) * sizeof(int);
  void* part = nullptr;
  int rc = get_workspace(h0, (reinterpret_cast<uintptr_t>(s) << 2) | 2, s, bytes, &part);
  if (rc) return rc;
  int* counts = static_cast<int*>(part);
  int* lists = reinterpret_cast<int*>(static_cast<char*>(part) + off_lists);
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int) * nchan, s);
  if (e != cudaSuccess) return cuda_fail(h0, e, "me_compute_channels: clear counts");
  const int64_t blocks = std::min<int64_t>((nevt + 255) / 256, int64_t(h0->nsm) * 8);
  partition_channels<<<unsigned(blocks), 256, 0, s>>>(nevt, channel, nchan, counts, lists, me, sel_hel, sel_col);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h0, e, "me_compute_channels: partition launch");
  const bool want_hel = sel_hel && rnd_hel;
  const bool want_col = sel_col && rnd_col;
  for (int c = 0; c < nchan; ++c) {
    me_handle* h = hs[c];
    // sized for the whole batch: the channel's count is known only on the device
    const CallPlan cp = plan_call(h, nevt, nevt, want_hel, want_col);
    void* wsp = nullptr;
    if (cp.total) {
      rc = get_workspace(h, reinterpret_cast<uintptr_t>(s) << 1, s, cp.total, &wsp);
      if (rc) return rc;
    }
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
    a.ngood = int(h->good.size());
    for (int i = 0; i < a.ngood; ++i) a.good[i] = uint8_t(h->good[i]);
    a.index = lists + int64_t(c) * nevt;
    a.index_count = counts + c;
    a.index_cap = int(nevt);
    e = run_call(h, cp, a, nevt, wsp, s);
    if (e != cudaSuccess) return cuda_fail(h0, e, "me_compute_channels launch");
  }
  return ME_OK;
}
