// rambo.cu -- synthetic inputs generated on the device: counter-based uniforms and RAMBO
// phase-space points, for the standalone multi-event testbed (Section 2, Fig. 1b) in
// which a batch of test events is generated and its matrix elements computed without a
// host round trip.
//
// Uniforms: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), every number a function
// of (seed, event index, stream, draw index):
//   key = (seed mod 2^32, seed div 2^32); counter = (event mod 2^32, event div 2^32,
//   draw div 2, stream); draw j takes output words (x0, x1) for even j, (x2, x3) for odd;
//   u = (((hi << 32 | lo) >> 12) + 1/2) 2^-52, strictly inside (0, 1).
// These are integer operations and one exact conversion, so the numbers are identical to
// any other implementation of the same definition.
//
// RAMBO (Kleiss, Stirling, Ellis, Comput. Phys. Commun. 40 (1986) 359): n isotropic
// massless vectors with energies from q0 e^{-q0}, a conformal boost to the rest frame of
// their sum and a scale to sqrt(s); massive final states by rescaling every three-momentum
// by xi, found by Newton's method on sum_i sqrt(m_i^2 + xi^2 E_i^2) = sqrt(s).
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/me.h"
#include "me_internal.h"

using namespace meb300;
using namespace meb300::detail;

namespace {

constexpr int kMaxFinal = 8;
constexpr int kThreads = 128;
constexpr int kNewtonSteps = 50;

struct RamboArgs {
  int64_t nevt;
  uint64_t seed, first;
  double sqrt_s;
  int nfinal;
  double mass[kMaxFinal];
  double* mom;  // [nevt][nfinal + 2][4]
};

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t p0 = uint64_t(0xD2511F53u) * c[0];
    const uint64_t p1 = uint64_t(0xCD9E8D57u) * c[2];
    const uint32_t n0 = uint32_t(p1 >> 32) ^ c[1] ^ k0;
    const uint32_t n2 = uint32_t(p0 >> 32) ^ c[3] ^ k1;
    c[1] = uint32_t(p1);
    c[3] = uint32_t(p0);
    c[0] = n0;
    c[2] = n2;
  }
}

// draws 2*call and 2*call + 1 of (seed, event, stream)
__device__ __forceinline__ void uniform_pair(uint64_t seed, uint64_t event, uint32_t stream, uint32_t call, double& u0,
                                             double& u1) {
  uint32_t c[4] = {uint32_t(event), uint32_t(event >> 32), call, stream};
  philox4x32_10(c, uint32_t(seed), uint32_t(seed >> 32));
  const uint64_t b0 = ((uint64_t(c[0]) << 32) | c[1]) >> 12;
  const uint64_t b1 = ((uint64_t(c[2]) << 32) | c[3]) >> 12;
  u0 = (double(b0) + 0.5) * 0x1p-52;
  u1 = (double(b1) + 0.5) * 0x1p-52;
}

__global__ void __launch_bounds__(kThreads) uniforms_kernel(int64_t n, uint64_t seed, uint64_t first, uint32_t stream,
                                                            double offset, double scale, double* out) {
  for (int64_t i = int64_t(blockIdx.x) * kThreads + threadIdx.x; i < n; i += int64_t(gridDim.x) * kThreads) {
    double u0, u1;
    uniform_pair(seed, first + uint64_t(i), stream, 0, u0, u1);
    out[i] = __dadd_rn(offset, __dmul_rn(scale, u0));  // rounded twice, as written: no FMA contraction
  }
}

__global__ void __launch_bounds__(kThreads) rambo_kernel(const RamboArgs a) {
  const int n = a.nfinal;
  for (int64_t i = int64_t(blockIdx.x) * kThreads + threadIdx.x; i < a.nevt; i += int64_t(gridDim.x) * kThreads) {
    const uint64_t ev = a.first + uint64_t(i);
    double q[kMaxFinal][4];
    for (int k = 0; k < n; ++k) {
      double u[4];
      uniform_pair(a.seed, ev, 0, uint32_t(2 * k), u[0], u[1]);
      uniform_pair(a.seed, ev, 0, uint32_t(2 * k + 1), u[2], u[3]);
      const double c = 2.0 * u[0] - 1.0;
      const double phi = 2.0 * 3.14159265358979323846 * u[1];
      const double q0 = -log(u[2] * u[3]);
      const double st = sqrt(1.0 - c * c);
      q[k][0] = q0;
      q[k][1] = q0 * st * cos(phi);
      q[k][2] = q0 * st * sin(phi);
      q[k][3] = q0 * c;
    }
    double Q[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k = 0; k < n; ++k)
      for (int m = 0; m < 4; ++m) Q[m] += q[k][m];
    const double M = sqrt(Q[0] * Q[0] - Q[1] * Q[1] - Q[2] * Q[2] - Q[3] * Q[3]);
    const double b[3] = {-Q[1] / M, -Q[2] / M, -Q[3] / M};
    const double gam = Q[0] / M, aa = 1.0 / (1.0 + gam), x = a.sqrt_s / M;
    double p[kMaxFinal][4];
    for (int k = 0; k < n; ++k) {
      const double bq = b[0] * q[k][1] + b[1] * q[k][2] + b[2] * q[k][3];
      p[k][0] = x * (gam * q[k][0] + bq);
      for (int m = 1; m < 4; ++m) p[k][m] = x * (q[k][m] + b[m - 1] * q[k][0] + aa * bq * b[m - 1]);
    }
    // The boost multiplies the rounding of the massless vectors by up to its gamma
    // factor, so the residual of the three-momentum sum is taken out in equal parts, each
    // vector is put on the light cone (E = |p|), the rescaling xi solves
    // sum_i sqrt(m_i^2 + xi^2 |p_i|^2) = sqrt(s) (massless final states too), and each
    // final energy comes from its final three-momentum: momentum conservation and every
    // mass shell hold to rounding.
    for (int m = 1; m < 4; ++m) {
      double r = 0.0;
      for (int k = 0; k < n; ++k) r += p[k][m];
      for (int k = 0; k < n; ++k) p[k][m] -= r / n;
    }
    for (int k = 0; k < n; ++k) p[k][0] = sqrt(p[k][1] * p[k][1] + p[k][2] * p[k][2] + p[k][3] * p[k][3]);
    double msum = 0.0;
    for (int k = 0; k < n; ++k) msum += a.mass[k];
    const double r0 = 1.0 - (msum / a.sqrt_s) * (msum / a.sqrt_s);
    double xi = sqrt(r0 > 0.0 ? r0 : 0.0);
    bool ok = false;
    for (int it = 0; it < kNewtonSteps; ++it) {
      double rsum = 0.0, fp = 0.0;
      for (int k = 0; k < n; ++k) {
        const double e = xi * p[k][0];
        const double r = sqrt(a.mass[k] * a.mass[k] + e * e);
        rsum += r;
        fp += xi * p[k][0] * p[k][0] / r;
      }
      const double f = rsum - a.sqrt_s;
      if (fabs(f) <= 1e-15 * a.sqrt_s) {
        ok = true;
        break;
      }
      xi -= f / fp;
    }
    for (int k = 0; k < n; ++k) {
      for (int m = 1; m < 4; ++m) p[k][m] *= xi;
      p[k][0] = sqrt(a.mass[k] * a.mass[k] + (p[k][1] * p[k][1] + p[k][2] * p[k][2] + p[k][3] * p[k][3]));
    }
    double* out = a.mom + i * (n + 2) * 4;
    const double half = 0.5 * a.sqrt_s, nan = __longlong_as_double(0x7ff8000000000000ll);
    out[0] = half; out[1] = 0.0; out[2] = 0.0; out[3] = half;
    out[4] = half; out[5] = 0.0; out[6] = 0.0; out[7] = -half;
    for (int k = 0; k < n; ++k)
      for (int m = 0; m < 4; ++m) out[8 + 4 * k + m] = ok ? p[k][m] : nan;
  }
}

int grid_for(int64_t n) {
  const int64_t want = (n + kThreads - 1) / kThreads;
  return int(want < 148 * 16 ? want : 148 * 16);
}

}  // namespace

extern "C" int me_rambo(me_handle* h, int64_t nevt, uint64_t seed, uint64_t first_event, double sqrt_s,
                        double* momenta, void* cuda_stream) {
  if (!h) return fail(nullptr, ME_ERR_ARG, "me_rambo: null handle");
  if (nevt < 0) return fail(h, ME_ERR_ARG, "me_rambo: nevt < 0");
  if (nevt == 0) return ME_OK;
  if (!momenta || !is_device_ptr(momenta)) return fail(h, ME_ERR_ARG, "me_rambo: momenta must be device memory");
  RamboArgs a{};
  a.nevt = nevt;
  a.seed = seed;
  a.first = first_event;
  a.sqrt_s = sqrt_s;
  const std::vector<double> m = final_masses(h->ops, h->par.mt);
  a.nfinal = int(m.size());
  double msum = 0.0;
  for (int k = 0; k < a.nfinal && k < kMaxFinal; ++k) {
    a.mass[k] = m[k];
    msum += m[k];
  }
  if (!(sqrt_s > msum)) return fail(h, ME_ERR_ARG, "me_rambo: sqrt_s must exceed the sum of the final masses");
  a.mom = momenta;
  rambo_kernel<<<grid_for(nevt), kThreads, 0, static_cast<cudaStream_t>(cuda_stream)>>>(a);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ME_OK : cuda_fail(h, e, "me_rambo launch");
}

extern "C" int me_uniforms(int64_t nevt, uint64_t seed, uint64_t first_event, int stream_id, double offset,
                           double scale, double* out, void* cuda_stream) {
  if (nevt < 0 || stream_id < 0) return fail(nullptr, ME_ERR_ARG, "me_uniforms: nevt < 0 or stream_id < 0");
  if (nevt == 0) return ME_OK;
  if (!out || !is_device_ptr(out)) return fail(nullptr, ME_ERR_ARG, "me_uniforms: out must be device memory");
  uniforms_kernel<<<grid_for(nevt), kThreads, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
      nevt, seed, first_event, uint32_t(stream_id), offset, scale, out);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ME_OK : cuda_fail(nullptr, e, "me_uniforms launch");
}
