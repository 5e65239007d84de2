// me_lib.cu -- the C ABI declared in include/me.h.
//
// Host side of the multi-event interface (paper Section 3, Fig. 1c): a handle per
// process keeps the derived couplings, the helicities kept by the filter and one
// device workspace per CUDA stream; me_compute checks its arguments and launches the
// process kernel on the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/me.h"
#include "me_internal.h"
#include "me_kernels.cuh"

// Each process lives in its own translation unit; a build may leave one out (weak
// references resolve to null and the process is then reported as unknown).
namespace meb300 {
extern const ProcessOps ops_eemumu __attribute__((weak));
extern const ProcessOps ops_ggtt __attribute__((weak));
extern const ProcessOps ops_ggttg __attribute__((weak));
extern const ProcessOps ops_ggttgg __attribute__((weak));
extern const ProcessOps ops_ggttggg __attribute__((weak));
extern const ProcessOps ops_qqtt __attribute__((weak));
extern const ProcessOps ops_qxqtt __attribute__((weak));
extern const ProcessOps ops_qqttg __attribute__((weak));
extern const ProcessOps ops_qxqttg __attribute__((weak));
extern const ProcessOps ops_qgttq __attribute__((weak));
extern const ProcessOps ops_gqttq __attribute__((weak));
extern const ProcessOps ops_qxgttqx __attribute__((weak));
extern const ProcessOps ops_gqxttqx __attribute__((weak));
extern const ProcessOps ops_qqttgg __attribute__((weak));
extern const ProcessOps ops_qxqttgg __attribute__((weak));
extern const ProcessOps ops_qgttqg __attribute__((weak));
extern const ProcessOps ops_gqttqg __attribute__((weak));
extern const ProcessOps ops_qxgttqxg __attribute__((weak));
extern const ProcessOps ops_gqxttqxg __attribute__((weak));
extern const ProcessOps ops_ggttqqx __attribute__((weak));
extern const ProcessOps ops_uuxttddx __attribute__((weak));
extern const ProcessOps ops_uxuttddx __attribute__((weak));
extern const ProcessOps ops_udttud __attribute__((weak));
extern const ProcessOps ops_udxttudx __attribute__((weak));
extern const ProcessOps ops_uxdxttuxdx __attribute__((weak));
extern const ProcessOps ops_uuttuu __attribute__((weak));
extern const ProcessOps ops_uxuxttuxux __attribute__((weak));
extern const ProcessOps ops_uuxttuux __attribute__((weak));
extern const ProcessOps ops_uxuttuux __attribute__((weak));
}
using namespace meb300;

namespace {

const ProcessOps* const kProcs[] = {&ops_eemumu, &ops_ggtt,   &ops_ggttg,  &ops_ggttgg,  &ops_ggttggg,
                                    &ops_qqtt,   &ops_qxqtt,  &ops_qqttg,  &ops_qxqttg,  &ops_qgttq,
                                    &ops_gqttq,  &ops_qxgttqx, &ops_gqxttqx, &ops_qqttgg, &ops_qxqttgg,
                                    &ops_qgttqg, &ops_gqttqg, &ops_qxgttqxg, &ops_gqxttqxg, &ops_ggttqqx,
                                    &ops_uuxttddx, &ops_uxuttddx, &ops_udttud, &ops_udxttudx, &ops_uxdxttuxdx,
                                    &ops_uuttuu, &ops_uxuxttuxux, &ops_uuxttuux, &ops_uxuttuux};

thread_local std::string g_init_error;


// events per launch: the rescue list holds 32-bit event indices
constexpr int64_t kMaxChunk = int64_t(1) << 30;

}  // namespace

namespace meb300 {
namespace detail {

int fail(me_handle* h, int code, const std::string& msg) {
  if (h) {
    std::lock_guard<std::mutex> g(h->mu);
    h->err = msg;
  } else {
    g_init_error = msg;
  }
  return code;
}

int cuda_fail(me_handle* h, cudaError_t e, const char* where) {
  const int code = (e == cudaErrorMemoryAllocation) ? ME_ERR_NOMEM : ME_ERR_CUDA;
  return fail(h, code, std::string(where) + ": " + cudaGetErrorString(e));
}

// splitmix64 (Steele, Lea, Flood 2014) for the library's own filter sample
struct SplitMix {
  uint64_t s;
  double uniform() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double(z >> 12) + 0.5) * (1.0 / 4503599627370496.0);
  }
};

// RAMBO (Kleiss, Stirling, Ellis 1986): flat n-body phase space at sqrt(s), massless
// vectors rescaled to the final-state masses.  Writes [nevt][2+n][4].
void rambo_sample(int nevt, double sqrt_s, const std::vector<double>& masses, uint64_t seed, double* out) {
  const int n = int(masses.size());
  SplitMix rng{seed};
  std::vector<double> q(4 * n), p(4 * n);
  const int npar = n + 2;
  double msum = 0;
  for (double m : masses) msum += m;
  for (int e = 0; e < nevt; ++e) {
    double Q[4] = {0, 0, 0, 0};
    for (int i = 0; i < n; ++i) {
      const double c = 2 * rng.uniform() - 1, phi = 2 * M_PI * rng.uniform();
      const double q0 = -std::log(rng.uniform() * rng.uniform());
      const double st = std::sqrt(1 - c * c);
      q[4 * i] = q0;
      q[4 * i + 1] = q0 * st * std::cos(phi);
      q[4 * i + 2] = q0 * st * std::sin(phi);
      q[4 * i + 3] = q0 * c;
      for (int m = 0; m < 4; ++m) Q[m] += q[4 * i + m];
    }
    const double M = std::sqrt(Q[0] * Q[0] - Q[1] * Q[1] - Q[2] * Q[2] - Q[3] * Q[3]);
    const double b[3] = {-Q[1] / M, -Q[2] / M, -Q[3] / M};
    const double gam = Q[0] / M, a = 1 / (1 + gam), x = sqrt_s / M;
    for (int i = 0; i < n; ++i) {
      const double* qi = &q[4 * i];
      const double bq = b[0] * qi[1] + b[1] * qi[2] + b[2] * qi[3];
      p[4 * i] = x * (gam * qi[0] + bq);
      for (int k = 0; k < 3; ++k) p[4 * i + 1 + k] = x * (qi[1 + k] + b[k] * qi[0] + a * bq * b[k]);
    }
    double xi = 1.0;
    if (msum > 0) {
      xi = std::sqrt(1 - (msum / sqrt_s) * (msum / sqrt_s));
      for (int it = 0; it < 50; ++it) {
        double f = -sqrt_s, fp = 0;
        for (int i = 0; i < n; ++i) {
          const double r = std::sqrt(masses[i] * masses[i] + xi * xi * p[4 * i] * p[4 * i]);
          f += r;
          fp += xi * p[4 * i] * p[4 * i] / r;
        }
        if (std::fabs(f) <= 1e-15 * sqrt_s) break;
        xi -= f / fp;
      }
    }
    double* o = out + size_t(e) * npar * 4;
    o[0] = o[3] = sqrt_s / 2;
    o[1] = o[2] = 0;
    o[4] = sqrt_s / 2;
    o[5] = o[6] = 0;
    o[7] = -sqrt_s / 2;
    for (int i = 0; i < n; ++i) {
      double* pi = o + 4 * (i + 2);
      pi[0] = std::sqrt(masses[i] * masses[i] + xi * xi * p[4 * i] * p[4 * i]);
      for (int k = 1; k < 4; ++k) pi[k] = xi * p[4 * i + k];
    }
  }
}

std::vector<double> final_masses(const ProcessOps* ops, double mt) {
  if (ops == &ops_eemumu) return {0.0, 0.0};
  std::vector<double> m = {mt, mt};
  for (int i = 4; i < ops->npar; ++i) m.push_back(0.0);
  return m;
}

void fill_common(const me_handle* h, MeLaunch& a) {
  a.mma_wait_limit = h->wait_limit < 0 ? kMmaWaitDefault : uint32_t(std::min<int64_t>(h->wait_limit, UINT32_MAX));
  a.alphas_default = h->par.alphas_default;
  a.mt = h->par.mt;
  a.wt = h->par.wt;
  a.zwt = h->par.zero_width_tchan;
  for (int i = 0; i < 4; ++i) a.zc[i] = h->zc[i];
  a.coup = h->coup;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// stream-ordered workspace of at least 'bytes' under key
int get_workspace(me_handle* h, uintptr_t key, cudaStream_t s, size_t bytes, void** out) {
  std::lock_guard<std::mutex> g(h->mu);
  Workspace& w = h->ws[key];
  if (w.bytes < bytes) {
    if (w.ptr) cudaFreeAsync(w.ptr, s);
    w.ptr = nullptr;
    w.bytes = 0;
    const size_t want = bytes + bytes / 4;
    cudaError_t e = cudaMallocAsync(&w.ptr, want, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      w.ptr = nullptr;
      h->err = std::string("workspace allocation: ") + cudaGetErrorString(e);
      return e == cudaErrorMemoryAllocation ? ME_ERR_NOMEM : ME_ERR_CUDA;
    }
    w.bytes = want;
  }
  *out = w.ptr;
  return ME_OK;
}


Carve carve(const ProcessOps* ops, const LaunchNeeds& nd, int ngood, int64_t rows, bool want_hel, bool want_col) {
  Carve c;
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  // running helicity sums and colour weights: one value per event of each row
  if (want_hel) c.cum = up(size_t(ngood) * rows * nd.ept * sizeof(double));
  if (want_col && nd.colw_global) c.colw = up(size_t(ops->ncol) * rows * nd.ept * sizeof(double));
  c.slots = up(nd.slot_bytes_per_event * rows);  // rows cover whole blocks
  c.ktab = up(nd.ktab_bytes_per_event * rows);
  c.den = up(nd.den_bytes_per_event * rows);
  c.jt = up(nd.j_bytes_per_event * rows);
  return c;
}

// Blocks of the persistent grid for nevt events: no more than are resident at once.
int persistent_grid(const me_handle* h, const LaunchNeeds& nd, int64_t nevt) {
  const int64_t per_tile = int64_t(nd.block) * nd.ept;
  const int64_t tiles = (std::max<int64_t>(nevt, 1) + per_tile - 1) / per_tile;
  int64_t resident = int64_t(h->nsm) * nd.blocks_per_sm;
  if (h->max_blocks > 0) resident = std::min<int64_t>(resident, h->max_blocks);
  return int(std::max<int64_t>(1, std::min(tiles, resident)));
}

// Launch 'a' over nevt events in chunks, each on at most 'grid' blocks of 'block'
// threads with 'hsplit' threads per event, with workspace 'wsp' carved per 'cv'.
cudaError_t launch_chunks(const ProcessOps* ops, int prec, int config, MeLaunch a, int64_t nevt, int64_t chunk,
                          int grid, int block, int hsplit, const Carve& cv, void* wsp, cudaStream_t s, int ept) {
  char* w = static_cast<char*>(wsp);
  double* cum = cv.cum ? reinterpret_cast<double*>(w) : a.cum;
  double* colw = cv.colw ? reinterpret_cast<double*>(w + cv.cum) : nullptr;
  void* slots = cv.slots ? static_cast<void*>(w + cv.cum + cv.colw) : nullptr;
  void* ktab = cv.ktab ? static_cast<void*>(w + cv.cum + cv.colw + cv.slots) : nullptr;
  void* dtile = cv.den ? static_cast<void*>(w + cv.cum + cv.colw + cv.slots + cv.ktab) : nullptr;
  void* jtile = cv.jt ? static_cast<void*>(w + cv.cum + cv.colw + cv.slots + cv.ktab + cv.den) : nullptr;
  const int npar = ops->npar;
  for (int64_t off = 0; off < nevt; off += chunk) {
    MeLaunch b = a;
    b.nevt = std::min(chunk, nevt - off);
    b.mom = a.mom + off * npar * 4;
    if (a.alphas) b.alphas = a.alphas + off;
    if (a.rnd_hel) b.rnd_hel = a.rnd_hel + off;
    if (a.rnd_col) b.rnd_col = a.rnd_col + off;
    b.me = a.me + off;
    if (a.sel_hel) b.sel_hel = a.sel_hel + off;
    if (a.sel_col) b.sel_col = a.sel_col + off;
    b.cum = cum;
    b.colw = colw;
    b.slots = slots;
    b.ktab = ktab;
    b.dtile = dtile;
    b.jtile = jtile;
    b.ibase = off;
    b.hsplit = hsplit;
    const int64_t per_block = int64_t(block) * ept;
    b.grid_blocks = int(std::min<int64_t>(grid, (b.nevt * hsplit + per_block - 1) / per_block));
    cudaError_t e = ops->launch(prec, config, b, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int64_t chunk_for(const LaunchNeeds&, int64_t nevt) { return std::min<int64_t>(nevt, kMaxChunk); }

static size_t up256(size_t b) { return (b + 255) / 256 * 256; }

CallPlan plan_call(const me_handle* h, int64_t nevt, int64_t chunk, bool want_hel, bool want_col) {
  const ProcessOps* ops = h->ops;
  CallPlan cp;
  cp.prec = h->par.precision;
  cp.config = h->config;
  cp.chunk = chunk;
  const int ngood = int(h->good.size());
  const LaunchNeeds nd = ops->needs(cp.prec, cp.config);
  // One thread per event, so that results do not depend on the batch they come in;
  // except for a process with a single colour flow, which has no colour weights to
  // combine.  There a group of threads per event gives the same bits (its first lane
  // sums the helicities in order), and a batch that would leave most resident threads
  // idle is spread over up to ngood threads per event.
  cp.hsplit = 1;
  if (ops->ncol == 1) {
    const int64_t resident = int64_t(h->nsm) * nd.blocks_per_sm * nd.block;
    while (cp.hsplit < 32 && 2 * cp.hsplit <= ngood && 2 * cp.hsplit * chunk <= resident) cp.hsplit *= 2;
  }
  cp.grid = persistent_grid(h, nd, chunk * cp.hsplit);
  cp.block = nd.block;
  cp.ept = nd.ept;
  // the split's first lane reads the group's per-helicity values back from cum
  cp.main = carve(ops, nd, ngood, int64_t(cp.grid) * nd.block, want_hel || cp.hsplit > 1, want_col);
  size_t off = cp.main.total();
  cp.rescue = (cp.prec == ME_PREC_FP32 || cp.prec == ME_PREC_MIXED) && h->par.rescue_kappa > 0;
  if (cp.rescue) {
    const LaunchNeeds n64 = ops->needs(ME_PREC_FP64, 0);
    // one entry per event (4 bytes each): every flagged event is re-evaluated, however
    // many a batch holds (a batch from a phase-space channel mapped onto a collinear
    // region may flag most of its events)
    const int64_t cap = nevt;
    cp.rescue_cap = int(cap);
    // few events, each far slower in FP64: every event is spread over a group of up to
    // 32 threads, which sum its helicities in the same order as one thread would
    cp.rescue_hsplit = 1;
    while (cp.rescue_hsplit < 32 && 2 * cp.rescue_hsplit <= ngood) cp.rescue_hsplit *= 2;
    // the grid walks the list tile by tile, so any size is correct: it is sized for the
    // usual flagged fraction (well under 1%), not for the capacity; a batch that flags
    // more takes proportionally longer in that pass, never loses an event
    const int64_t expect = std::min<int64_t>(cap, std::max<int64_t>(64, nevt / 100));
    cp.rescue_grid = persistent_grid(h, n64, expect * cp.rescue_hsplit);
    const size_t rows = size_t(cp.rescue_grid) * n64.block;
    cp.off_count = off; off += 256;
    cp.off_list = off; off += up256(size_t(cap) * sizeof(int));
    cp.off_cum = off; off += up256(size_t(ngood) * rows * sizeof(double));  // the split needs it
    cp.off_colw = off; if (want_col && n64.colw_global) off += up256(size_t(ops->ncol) * rows * sizeof(double));
    cp.off_slots = off; off += up256(n64.slot_bytes_per_event * rows);
    cp.off_ktab = off; off += up256(n64.ktab_bytes_per_event * rows);
    cp.off_den = off; off += up256(n64.den_bytes_per_event * rows);
    cp.off_j = off; off += up256(n64.j_bytes_per_event * rows);
  }
  cp.total = off;
  return cp;
}

cudaError_t run_call(const me_handle* h, const CallPlan& cp, const MeLaunch& a0, int64_t nevt, void* wsp,
                     cudaStream_t s) {
  const ProcessOps* ops = h->ops;
  char* w = static_cast<char*>(wsp);
  MeLaunch a = a0;
  if (cp.rescue) {
    cudaError_t e = cudaMemsetAsync(w + cp.off_count, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    a.rescue_kappa = h->par.rescue_kappa;
    a.rescue_count = reinterpret_cast<int*>(w + cp.off_count);
    a.rescue_list = reinterpret_cast<int*>(w + cp.off_list);
    a.rescue_cap = cp.rescue_cap;
  }
  cudaError_t e = launch_chunks(ops, cp.prec, cp.config, a, nevt, cp.chunk, cp.grid, cp.block, cp.hsplit, cp.main, wsp,
                                s, cp.ept);
  if (e != cudaSuccess || !cp.rescue) return e;
  // FP64 pass over the flagged events, in place: same inputs and outputs
  MeLaunch b = a0;
  const bool want_col = a0.sel_col != nullptr;
  b.nevt = nevt;
  b.cum = reinterpret_cast<double*>(w + cp.off_cum);
  b.colw = (want_col && ops->needs(ME_PREC_FP64, 0).colw_global) ? reinterpret_cast<double*>(w + cp.off_colw) : nullptr;
  b.slots = w + cp.off_slots;
  b.ktab = w + cp.off_ktab;
  b.dtile = w + cp.off_den;
  b.jtile = w + cp.off_j;
  b.index = reinterpret_cast<const int*>(w + cp.off_list);
  b.index_count = reinterpret_cast<const int*>(w + cp.off_count);
  b.index_cap = cp.rescue_cap;
  b.grid_blocks = cp.rescue_grid;
  b.hsplit = cp.rescue_hsplit;
  return ops->launch(ME_PREC_FP64, 0, b, s);
}

}  // namespace detail
}  // namespace meb300
using namespace meb300::detail;

extern "C" {

void me_default_params(me_sm_params* p) {
  if (!p) return;
  p->mZ = 91.188;
  p->wZ = 2.4414;
  p->mt = 173.0;
  p->wt = 1.4915;
  p->aEWM1 = 132.5;
  p->Gf = 1.16639e-5;
  p->alphas_default = 0.118;
  p->precision = ME_PREC_FP64;
  p->zero_width_tchan = 0;
  p->rescue_kappa = 2000.0;
}

int me_init(const char* process, const me_sm_params* p, me_handle** out) {
  if (out) *out = nullptr;
  if (!process || !p || !out) return fail(nullptr, ME_ERR_ARG, "me_init: null argument");
  const ProcessOps* ops = nullptr;
  for (const ProcessOps* o : kProcs)
    if (o && std::strcmp(o->name, process) == 0) ops = o;
  if (!ops) return fail(nullptr, ME_ERR_ARG, std::string("me_init: unknown process '") + process + "'");
  if (!(p->mZ > 0 && p->wZ >= 0 && p->mt > 0 && p->wt >= 0 && p->aEWM1 > 0 && p->Gf > 0 && p->alphas_default > 0 &&
        p->rescue_kappa >= 0))
    return fail(nullptr, ME_ERR_ARG, "me_init: parameters must be positive (widths non-negative)");
  if (p->precision < 0 || p->precision > 3) return fail(nullptr, ME_ERR_ARG, "me_init: unknown precision mode");
  if (p->precision == ME_PREC_MIXED && !ops->has_mixed)
    return fail(nullptr, ME_ERR_MODE, "me_init: mixed precision is not available for this process");
  if (ops->nconfig[p->precision] <= 0)
    return fail(nullptr, ME_ERR_MODE, "me_init: this precision mode is not built for this process");
  const double alpha = 1.0 / p->aEWM1;
  const double mz2 = p->mZ * p->mZ;
  const double disc = mz2 * mz2 / 4.0 - M_PI * alpha * mz2 / (std::sqrt(2.0) * p->Gf);
  if (!(disc > 0)) return fail(nullptr, ME_ERR_ARG, "me_init: (alpha, G_F, mZ) admit no W mass");

  me_handle* h = new me_handle();
  h->ops = ops;
  h->par = *p;
  {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        nsm > 0)
      h->nsm = nsm;
    cudaGetLastError();
  }
  if (cudaHostAlloc(reinterpret_cast<void**>(&h->err_host), sizeof(int), cudaHostAllocMapped) == cudaSuccess) {
    *h->err_host = 0;
    if (cudaHostGetDevicePointer(reinterpret_cast<void**>(&h->err_dev), h->err_host, 0) != cudaSuccess) h->err_dev = nullptr;
  } else {
    cudaGetLastError();
    h->err_host = nullptr;
  }
  if (const char* env = std::getenv("ME_B300_CONFIG")) {
    const int c = std::atoi(env);
    if (c >= 0 && c < ops->nconfig[p->precision]) h->config = c;
  }
  if (const char* env = std::getenv("ME_B300_MAX_BLOCKS")) h->max_blocks = std::max(0, std::atoi(env));
  const double ee = std::sqrt(4.0 * M_PI * alpha);
  const double mw2 = mz2 / 2.0 + std::sqrt(disc);
  const double sw2 = 1.0 - mw2 / mz2, sw = std::sqrt(sw2), cw = std::sqrt(1.0 - sw2);
  h->zc[0] = (-0.5 + sw2) / (sw * cw);  // charged lepton, left-handed: (T3 - Q sw^2)/(sw cw)
  h->zc[1] = sw2 / (sw * cw);           // right-handed: -Q sw^2/(sw cw)
  h->zc[2] = p->mZ;
  h->zc[3] = p->wZ;
  h->coup = ee * ee * ee * ee;

  // helicity filter on 1024 fixed RAMBO events, every helicity, FP64
  const int nf = 1024;
  std::vector<double> mom(size_t(nf) * ops->npar * 4);
  rambo_sample(nf, 1500.0, final_masses(ops, p->mt), 12345, mom.data());
  const LaunchNeeds nd = ops->needs(ME_PREC_FP64, 0);
  const int fgrid = (nf + nd.block - 1) / nd.block;  // one event per thread: rows == events
  Carve cv = carve(ops, nd, 0, int64_t(fgrid) * nd.block, false, false);
  double *d_mom = nullptr, *d_me = nullptr, *d_cum = nullptr;
  void* d_ws = nullptr;
  cudaError_t e = cudaMalloc(&d_mom, mom.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_me, nf * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_cum, size_t(ops->ncomb) * nf * sizeof(double));
  if (e == cudaSuccess && cv.total()) e = cudaMalloc(&d_ws, cv.total());
  if (e == cudaSuccess) e = cudaMemcpy(d_mom, mom.data(), mom.size() * sizeof(double), cudaMemcpyHostToDevice);
  std::vector<double> cum(size_t(ops->ncomb) * nf);
  if (e == cudaSuccess) {
    MeLaunch a{};
    fill_common(h, a);
    a.mom = d_mom;
    a.me = d_me;
    a.ngood = ops->ncomb;
    a.cum_mode = 1;
    for (int i = 0; i < ops->ncomb; ++i) a.good[i] = uint8_t(i);
    a.cum = d_cum;  // [ncomb][rows] with rows == nf: one tile per block, one event per thread
    if (int64_t(fgrid) * nd.block != nf) e = cudaErrorInvalidConfiguration;
    if (e == cudaSuccess) e = launch_chunks(ops, ME_PREC_FP64, 0, a, nf, nf, fgrid, nd.block, 1, cv, d_ws, 0, 1);
    if (e == cudaSuccess) e = cudaMemcpy(cum.data(), d_cum, cum.size() * sizeof(double), cudaMemcpyDeviceToHost);
  }
  cudaFree(d_mom);
  cudaFree(d_me);
  cudaFree(d_cum);
  cudaFree(d_ws);
  if (e != cudaSuccess) {
    int rc = cuda_fail(nullptr, e, "me_init helicity filter");
    delete h;
    return rc;
  }
  for (int hh = 0; hh < ops->ncomb; ++hh) {
    bool nz = false;
    for (int ev = 0; ev < nf && !nz; ++ev) nz = cum[size_t(hh) * nf + ev] != 0.0;
    if (nz) h->good.push_back(hh);
  }
  *out = h;
  return ME_OK;
}

}  // extern "C"

namespace meb300 {
namespace detail {
int compute_device(me_handle* h, int64_t nevt, const double* momenta, const double* alphas, const double* rnd_hel,
                   const double* rnd_col, double* me, int32_t* sel_hel, int32_t* sel_col, cudaStream_t s,
                   const double* wgt, double* w, unsigned long long* wmax_bits) {
  if (h->err_host && *h->err_host) {
    *h->err_host = 0;
    return fail(h, ME_ERR_TIMEOUT, "me_compute: a device-side wait of an earlier call on this handle timed out; "
                                   "its events were set to NaN");
  }
  const ProcessOps* ops = h->ops;
  const int ngood = int(h->good.size());
  const bool want_hel = sel_hel && rnd_hel;
  const bool want_col = sel_col && rnd_col;
  const LaunchNeeds nd = ops->needs(h->par.precision, h->config);
  if (wgt && nd.ept != 1)
    return fail(h, ME_ERR_MODE, "fused unweighting: the selected launch configuration carries two events per thread");
  const CallPlan cp = plan_call(h, nevt, chunk_for(nd, nevt), want_hel, want_col);
  void* wsp = nullptr;
  if (cp.total) {
    int rc = get_workspace(h, reinterpret_cast<uintptr_t>(s) << 1, s, cp.total, &wsp);
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
  a.ngood = ngood;
  for (int i = 0; i < ngood; ++i) a.good[i] = uint8_t(h->good[i]);
  a.wgt = wgt;
  a.w = w;
  a.wmax_bits = wmax_bits;
  cudaError_t e = run_call(h, cp, a, nevt, wsp, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "me_compute launch");
  return ME_OK;
}
}  // namespace detail
}  // namespace meb300

extern "C" {

int me_reserve(me_handle* h, int64_t nevt, void* cuda_stream) {
  if (!h) return fail(nullptr, ME_ERR_ARG, "me_reserve: null handle");
  if (nevt < 0) return fail(h, ME_ERR_ARG, "me_reserve: nevt < 0");
  if (nevt == 0) return ME_OK;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const LaunchNeeds nd = h->ops->needs(h->par.precision, h->config);
  const CallPlan cp = plan_call(h, nevt, chunk_for(nd, nevt), true, true);
  void* wsp = nullptr;
  return cp.total ? get_workspace(h, reinterpret_cast<uintptr_t>(s) << 1, s, cp.total, &wsp) : ME_OK;
}

int me_compute(me_handle* h, int64_t nevt, const double* momenta, const double* alphas, const double* rnd_hel,
               const double* rnd_col, double* me, int32_t* sel_hel, int32_t* sel_col, void* cuda_stream) {
  if (!h) return fail(nullptr, ME_ERR_ARG, "me_compute: null handle");
  if (nevt < 0) return fail(h, ME_ERR_ARG, "me_compute: nevt < 0");
  if (nevt == 0) return ME_OK;
  if (nevt > INT32_MAX) return fail(h, ME_ERR_ARG, "me_compute: more than 2^31 - 1 events in one call");
  if (!momenta || !me) return fail(h, ME_ERR_ARG, "me_compute: momenta and me are required");
  if (reinterpret_cast<uintptr_t>(momenta) % 16) return fail(h, ME_ERR_ARG, "me_compute: momenta must be 16-byte aligned");
  if ((sel_hel && !rnd_hel) || (sel_col && !rnd_col))
    return fail(h, ME_ERR_ARG, "me_compute: a selection output needs its random numbers");
  const void* ptrs[] = {momenta, me, alphas, rnd_hel, rnd_col, sel_hel, sel_col};
  for (const void* p : ptrs)
    if (p && !is_device_ptr(p)) return fail(h, ME_ERR_ARG, "me_compute: arrays must be device memory");
  return compute_device(h, nevt, momenta, alphas, rnd_hel, rnd_col, me, sel_hel, sel_col,
                        static_cast<cudaStream_t>(cuda_stream), nullptr, nullptr, nullptr);
}

int me_compute_host(me_handle* h, int64_t nevt, const double* momenta, const double* alphas,
                    const double* rnd_hel, const double* rnd_col, double* me, int32_t* sel_hel, int32_t* sel_col,
                    void* cuda_stream) {
  if (!h) return fail(nullptr, ME_ERR_ARG, "me_compute_host: null handle");
  if (nevt < 0) return fail(h, ME_ERR_ARG, "me_compute_host: nevt < 0");
  if (nevt == 0) return ME_OK;
  if (nevt > INT32_MAX) return fail(h, ME_ERR_ARG, "me_compute_host: more than 2^31 - 1 events in one call");
  if (!momenta || !me) return fail(h, ME_ERR_ARG, "me_compute_host: momenta and me are required");
  if ((sel_hel && !rnd_hel) || (sel_col && !rnd_col))
    return fail(h, ME_ERR_ARG, "me_compute_host: a selection output needs its random numbers");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const size_t nm = size_t(nevt) * h->ops->npar * 4;
  // device staging: momenta | alphas | rnd_hel | rnd_col | me | sel_hel | sel_col
  const size_t bytes = nm * 8 + 4 * size_t(nevt) * 8 + 2 * size_t(nevt) * 4 + 64;
  void* stage = nullptr;
  int rc = get_workspace(h, (reinterpret_cast<uintptr_t>(s) << 1) | 1, s, bytes, &stage);
  if (rc) return rc;
  char* c = static_cast<char*>(stage);
  double* d_mom = reinterpret_cast<double*>(c); c += nm * 8;
  double* d_as = reinterpret_cast<double*>(c); c += size_t(nevt) * 8;
  double* d_rh = reinterpret_cast<double*>(c); c += size_t(nevt) * 8;
  double* d_rc = reinterpret_cast<double*>(c); c += size_t(nevt) * 8;
  double* d_me = reinterpret_cast<double*>(c); c += size_t(nevt) * 8;
  int32_t* d_sh = reinterpret_cast<int32_t*>(c); c += size_t(nevt) * 4;
  int32_t* d_sc = reinterpret_cast<int32_t*>(c);
  cudaError_t e = cudaMemcpyAsync(d_mom, momenta, nm * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && alphas) e = cudaMemcpyAsync(d_as, alphas, nevt * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && rnd_hel) e = cudaMemcpyAsync(d_rh, rnd_hel, nevt * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && rnd_col) e = cudaMemcpyAsync(d_rc, rnd_col, nevt * 8, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "me_compute_host H2D");
  rc = compute_device(h, nevt, d_mom, alphas ? d_as : nullptr, rnd_hel ? d_rh : nullptr, rnd_col ? d_rc : nullptr,
                      d_me, sel_hel ? d_sh : nullptr, sel_col ? d_sc : nullptr, s, nullptr, nullptr, nullptr);
  if (rc) return rc;
  e = cudaMemcpyAsync(me, d_me, nevt * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && sel_hel) e = cudaMemcpyAsync(sel_hel, d_sh, nevt * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && sel_col) e = cudaMemcpyAsync(sel_col, d_sc, nevt * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(h, e, "me_compute_host D2H");
  if (h->err_host && *h->err_host) {
    *h->err_host = 0;
    return fail(h, ME_ERR_TIMEOUT, "me_compute_host: a device-side wait timed out; its events were set to NaN");
  }
  return ME_OK;
}

int me_info(const me_handle* h, int* npar, int* ncomb, int* ngood, int* ncol, int* ndiag) {
  if (!h) return ME_ERR_ARG;
  if (npar) *npar = h->ops->npar;
  if (ncomb) *ncomb = h->ops->ncomb;
  if (ngood) *ngood = int(h->good.size());
  if (ncol) *ncol = h->ops->ncol;
  if (ndiag) *ndiag = h->ops->ndiag;
  return ME_OK;
}

int me_good_helicities(const me_handle* h, int32_t* list) {
  if (!h || !list) return ME_ERR_ARG;
  for (size_t i = 0; i < h->good.size(); ++i) list[i] = h->good[i];
  return ME_OK;
}

int me_flops(const me_handle* h, int64_t* fa, int64_t* fc) {
  if (!h) return ME_ERR_ARG;
  if (fa) *fa = h->ops->flops_amp;
  if (fc) *fc = h->ops->flops_col;
  return ME_OK;
}

int me_plan(const me_handle* h, int64_t nevt, int64_t* launches, int64_t* workspace_bytes) {
  if (!h || nevt < 0) return ME_ERR_ARG;
  const LaunchNeeds nd = h->ops->needs(h->par.precision, h->config);
  const int64_t chunk = std::max<int64_t>(1, chunk_for(nd, nevt));
  const CallPlan cp = plan_call(h, std::max<int64_t>(nevt, 1), chunk, true, true);
  if (launches) *launches = nevt ? (nevt + chunk - 1) / chunk + (cp.rescue ? 1 : 0) : 0;
  if (workspace_bytes) *workspace_bytes = int64_t(cp.total);
  return ME_OK;
}

int me_launch_shape(const me_handle* h, int64_t nevt, int* grid, int* block, int* blocks_per_sm, int* nsm) {
  if (!h || nevt < 0) return ME_ERR_ARG;
  const LaunchNeeds nd = h->ops->needs(h->par.precision, h->config);
  if (grid) {
    const int64_t n = std::max<int64_t>(nevt, 1);
    *grid = plan_call(h, n, chunk_for(nd, n), true, true).grid;
  }
  if (block) *block = nd.block;
  if (blocks_per_sm) *blocks_per_sm = nd.blocks_per_sm;
  if (nsm) *nsm = h->nsm;
  return ME_OK;
}

int me_sync_status(me_handle* h, void* cuda_stream) {
  if (!h) return fail(nullptr, ME_ERR_ARG, "me_sync_status: null handle");
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return cuda_fail(h, e, "me_sync_status");
  if (h->err_host && *h->err_host) {
    *h->err_host = 0;
    return fail(h, ME_ERR_TIMEOUT, "me_sync_status: a device-side wait of a call on this handle timed out; "
                                   "the main-pass results of that call were set to NaN");
  }
  return ME_OK;
}

int me_set_wait_limit(me_handle* h, int64_t polls) {
  if (!h) return fail(nullptr, ME_ERR_ARG, "me_set_wait_limit: null handle");
  h->wait_limit = polls < 0 ? -1 : polls;
  return ME_OK;
}

int me_set_config(me_handle* h, int config) {
  if (!h) return ME_ERR_ARG;
  const int n = h->ops->nconfig[h->par.precision];
  if (config < 0) return n;
  if (config >= n) return fail(h, ME_ERR_ARG, "me_set_config: unknown configuration");
  h->config = config;
  return ME_OK;
}

const char* me_last_error(const me_handle* h) {
  if (!h) return g_init_error.c_str();
  return h->err.c_str();
}

void me_free(me_handle* h) {
  if (!h) return;
  cudaDeviceSynchronize();
  for (auto& kv : h->ws)
    if (kv.second.ptr) cudaFree(kv.second.ptr);
  if (h->err_host) cudaFreeHost(h->err_host);
  delete h;
}

}  // extern "C"
