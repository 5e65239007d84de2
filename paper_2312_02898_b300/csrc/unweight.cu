// unweight.cu -- GPU-assisted batch unweighting (Section 3, Table 2).
//
// madevent turns weighted events into unweighted ones by hit-or-miss against the
// largest weight.  With a multi-event interface the largest weight of a whole batch is
// known before any decision, so no event has to be kept provisionally.  The full event
// weight is the matrix element times the host's Jacobian and PDF factor, formed on the
// device where the matrix elements already are; the batch maximum is a parallel
// reduction; each event is kept when its weight exceeds r times that maximum.
//
// Two passes over HBM-resident arrays (both bound by memory bandwidth, a few bytes per
// event against the megaflops of the matrix element):
//   1. w_i = me_i * wgt_i; the maximum over valid weights (finite and >= 0) by a warp
//      and block reduction and one 64-bit atomicMax per block on the bit pattern (for
//      non-negative IEEE doubles the bit patterns order like the values);
//   2. accept_i = valid_i && w_i > r_i * w_max; the count by a block reduction and one
//      atomicAdd per block.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/me.h"
#include "me_internal.h"

using namespace meb300;
using namespace meb300::detail;

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 148 * 8;

__device__ __forceinline__ bool valid_weight(double w) { return isfinite(w) && w >= 0.0; }

__global__ void __launch_bounds__(kThreads) unweight_max(int64_t n, const double* __restrict__ me,
                                                         const double* __restrict__ wgt, double* __restrict__ w,
                                                         unsigned long long* wmax_bits) {
  double m = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * kThreads + threadIdx.x; i < n; i += int64_t(gridDim.x) * kThreads) {
    const double wi = me[i] * wgt[i];
    if (w) w[i] = wi;
    if (valid_weight(wi)) m = fmax(m, wi);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double s_m[kThreads / 32];
  if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < kThreads / 32 ? s_m[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0 && m > 0.0) atomicMax(wmax_bits, static_cast<unsigned long long>(__double_as_longlong(m)));
  }
}

__global__ void __launch_bounds__(kThreads) unweight_accept(int64_t n, const double* __restrict__ me,
                                                            const double* __restrict__ wgt,
                                                            const double* __restrict__ rnd,
                                                            const unsigned long long* wmax_bits,
                                                            uint8_t* __restrict__ accept,
                                                            unsigned long long* n_accept) {
  const double wmax = __longlong_as_double(static_cast<long long>(*wmax_bits));
  unsigned c = 0;
  for (int64_t i = int64_t(blockIdx.x) * kThreads + threadIdx.x; i < n; i += int64_t(gridDim.x) * kThreads) {
    const double wi = me[i] * wgt[i];  // the same product as pass 1, recomputed rather than re-read
    const bool a = valid_weight(wi) && wi > rnd[i] * wmax;
    if (accept) accept[i] = a ? 1 : 0;
    c += a ? 1u : 0u;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  __shared__ unsigned s_c[kThreads / 32];
  if ((threadIdx.x & 31) == 0) s_c[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x < 32) {
    c = threadIdx.x < kThreads / 32 ? s_c[threadIdx.x] : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (threadIdx.x == 0 && n_accept && c) atomicAdd(n_accept, static_cast<unsigned long long>(c));
  }
}

}  // namespace

extern "C" int me_unweight(me_handle* h, int64_t nevt, const double* me, const double* wgt, const double* rnd,
                           double* w, uint8_t* accept, double* w_max, int64_t* n_accept, void* cuda_stream) {
  if (!h) return fail(nullptr, ME_ERR_ARG, "me_unweight: null handle");
  if (nevt < 0) return fail(h, ME_ERR_ARG, "me_unweight: nevt < 0");
  if (nevt == 0) return ME_OK;
  if (!me || !wgt || !w_max) return fail(h, ME_ERR_ARG, "me_unweight: me, wgt and w_max are required");
  if ((accept || n_accept) && !rnd) return fail(h, ME_ERR_ARG, "me_unweight: accept/n_accept need rnd");
  if (reinterpret_cast<uintptr_t>(w_max) % 8 || reinterpret_cast<uintptr_t>(n_accept) % 8)
    return fail(h, ME_ERR_ARG, "me_unweight: w_max and n_accept must be 8-byte aligned");
  const void* ptrs[] = {me, wgt, rnd, w, accept, w_max, n_accept};
  for (const void* p : ptrs)
    if (p && !is_device_ptr(p)) return fail(h, ME_ERR_ARG, "me_unweight: arrays must be device memory");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  auto* bits = reinterpret_cast<unsigned long long*>(w_max);
  auto* cnt = reinterpret_cast<unsigned long long*>(n_accept);
  const int64_t want = (nevt + kThreads - 1) / kThreads;
  const int blocks = int(want < kMaxBlocks ? want : kMaxBlocks);
  cudaError_t e = cudaMemsetAsync(bits, 0, sizeof(double), s);  // +0.0
  if (e == cudaSuccess && cnt) e = cudaMemsetAsync(cnt, 0, sizeof(int64_t), s);
  if (e != cudaSuccess) return cuda_fail(h, e, "me_unweight: clearing the outputs");
  unweight_max<<<blocks, kThreads, 0, s>>>(nevt, me, wgt, w, bits);
  if (accept || cnt) unweight_accept<<<blocks, kThreads, 0, s>>>(nevt, me, wgt, rnd, bits, accept, cnt);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "me_unweight launch");
  return ME_OK;
}

// me_compute and me_unweight in one call, with the weight and the batch maximum formed in
// the matrix-element kernel's epilogue (the selection step of the kernel), so the only
// extra work is the accept/reject pass, which needs the finished maximum.
extern "C" int me_compute_unweight(me_handle* h, int64_t nevt, const double* momenta, const double* alphas,
                                   const double* rnd_hel, const double* rnd_col, const double* wgt, const double* rnd,
                                   double* me, int32_t* sel_hel, int32_t* sel_col, double* w, uint8_t* accept,
                                   double* w_max, int64_t* n_accept, void* cuda_stream) {
  if (!h) return fail(nullptr, ME_ERR_ARG, "me_compute_unweight: null handle");
  if (nevt < 0) return fail(h, ME_ERR_ARG, "me_compute_unweight: nevt < 0");
  if (nevt == 0) return ME_OK;
  if (nevt > INT32_MAX) return fail(h, ME_ERR_ARG, "me_compute_unweight: more than 2^31 - 1 events in one call");
  if (!momenta || !me || !wgt || !w_max)
    return fail(h, ME_ERR_ARG, "me_compute_unweight: momenta, me, wgt and w_max are required");
  if (reinterpret_cast<uintptr_t>(momenta) % 16)
    return fail(h, ME_ERR_ARG, "me_compute_unweight: momenta must be 16-byte aligned");
  if ((sel_hel && !rnd_hel) || (sel_col && !rnd_col))
    return fail(h, ME_ERR_ARG, "me_compute_unweight: a selection output needs its random numbers");
  if ((accept || n_accept) && !rnd) return fail(h, ME_ERR_ARG, "me_compute_unweight: accept/n_accept need rnd");
  if (reinterpret_cast<uintptr_t>(w_max) % 8 || reinterpret_cast<uintptr_t>(n_accept) % 8)
    return fail(h, ME_ERR_ARG, "me_compute_unweight: w_max and n_accept must be 8-byte aligned");
  const void* ptrs[] = {momenta, me, alphas, rnd_hel, rnd_col, sel_hel, sel_col, wgt, rnd, w, accept, w_max, n_accept};
  for (const void* p : ptrs)
    if (p && !is_device_ptr(p)) return fail(h, ME_ERR_ARG, "me_compute_unweight: arrays must be device memory");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  auto* bits = reinterpret_cast<unsigned long long*>(w_max);
  auto* cnt = reinterpret_cast<unsigned long long*>(n_accept);
  cudaError_t e = cudaMemsetAsync(bits, 0, sizeof(double), s);  // +0.0
  if (e == cudaSuccess && cnt) e = cudaMemsetAsync(cnt, 0, sizeof(int64_t), s);
  if (e != cudaSuccess) return cuda_fail(h, e, "me_compute_unweight: clearing the outputs");
  int rc = compute_device(h, nevt, momenta, alphas, rnd_hel, rnd_col, me, sel_hel, sel_col, s, wgt, w, bits);
  if (rc) return rc;
  if (accept || cnt) {
    const int64_t want = (nevt + kThreads - 1) / kThreads;
    const int blocks = int(want < kMaxBlocks ? want : kMaxBlocks);
    unweight_accept<<<blocks, kThreads, 0, s>>>(nevt, me, wgt, rnd, bits, accept, cnt);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "me_compute_unweight: accept launch");
  }
  return ME_OK;
}
