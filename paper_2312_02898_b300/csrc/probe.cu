// probe.cu -- FMA-throughput probe for the ALU roofline (see include/me_probe.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>

#include "../../include/me_probe.h"

namespace {

// 8 independent accumulators per thread, each an FMA chain; the result is stored so
// that the compiler keeps the work.
template <class T>
__global__ void __launch_bounds__(256) fma_loop(T* out, int iters, T a, T b) {
  T x0 = T(threadIdx.x), x1 = x0 + T(1), x2 = x0 + T(2), x3 = x0 + T(3);
  T x4 = x0 + T(4), x5 = x0 + T(5), x6 = x0 + T(6), x7 = x0 + T(7);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

// The same with packed FP32 pairs: fma.rn.f32x2 does two FP32 FMAs per instruction
// (sm_100 family); one 64-bit register holds a pair.
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
  return (static_cast<unsigned long long>(__float_as_uint(hi)) << 32) | __float_as_uint(lo);
}
__global__ void __launch_bounds__(256) fma_loop_x2(float* out, int iters, float a, float b) {
  const unsigned long long A = pack2(a, a), B = pack2(b, b);
  const float t = float(threadIdx.x);
  unsigned long long x0 = pack2(t, t + 8), x1 = pack2(t + 1, t + 9), x2 = pack2(t + 2, t + 10),
                     x3 = pack2(t + 3, t + 11), x4 = pack2(t + 4, t + 12), x5 = pack2(t + 5, t + 13),
                     x6 = pack2(t + 6, t + 14), x7 = pack2(t + 7, t + 15);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      x0 = fma2(x0, A, B); x1 = fma2(x1, A, B); x2 = fma2(x2, A, B); x3 = fma2(x3, A, B);
      x4 = fma2(x4, A, B); x5 = fma2(x5, A, B); x6 = fma2(x6, A, B); x7 = fma2(x7, A, B);
    }
  }
  const unsigned long long s[8] = {x0, x1, x2, x3, x4, x5, x6, x7};
  float acc = 0.f;
  for (int k = 0; k < 8; ++k) acc += __uint_as_float(unsigned(s[k])) + __uint_as_float(unsigned(s[k] >> 32));
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

template <class T, bool PACKED = false>
int probe(double seconds, double* fps) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -4;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -4;
  const int blocks = nsm * 8, threads = 256;
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * blocks * threads) != cudaSuccess) return -4;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int iters = 64;
  double best = 0;
  float ms = 0;
  // warm up and scale the loop to the requested duration
  for (int round = 0; round < 12; ++round) {
    cudaEventRecord(e0);
    if constexpr (PACKED)
      fma_loop_x2<<<blocks, threads>>>(reinterpret_cast<float*>(out), iters, 0.999999f, 1e-7f);
    else
      fma_loop<T><<<blocks, threads>>>(out, iters, T(0.999999), T(1e-7));
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flops = (PACKED ? 4.0 : 2.0) * 8 * 16 * double(iters) * blocks * threads;
    if (ms > 0) best = std::max(best, flops / (ms * 1e-3));
    if (ms < seconds * 1e3 / 4 && iters < (1 << 28)) iters *= 2;
  }
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return -4;
  *fps = best;
  return 0;
}

}  // namespace

extern "C" int me_probe_alu_peak(int prec, double seconds, double* flops_per_s) {
  if (!flops_per_s || prec < 0 || prec > 2) return -1;
  seconds = std::min(5.0, std::max(0.05, seconds));
  if (prec == 0) return probe<double>(seconds, flops_per_s);
  if (prec == 1) return probe<float>(seconds, flops_per_s);
  return probe<float, true>(seconds, flops_per_s);
}
