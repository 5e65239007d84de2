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

template <class T>
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
    fma_loop<T><<<blocks, threads>>>(out, iters, T(0.999999), T(1e-7));
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flops = 2.0 * 8 * 16 * double(iters) * blocks * threads;
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
  if (!flops_per_s || (prec != 0 && prec != 1)) return -1;
  seconds = std::min(5.0, std::max(0.05, seconds));
  return prec == 0 ? probe<double>(seconds, flops_per_s) : probe<float>(seconds, flops_per_s);
}
