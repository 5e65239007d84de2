// me_internal.h -- declarations shared by the translation units of libme_b300.so
// (the handle and the launch helpers); not part of the public C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/me.h"
#include "me_kernels.cuh"

struct Workspace {
  void* ptr = nullptr;
  size_t bytes = 0;
};

struct me_handle {
  const meb300::ProcessOps* ops = nullptr;
  me_sm_params par{};
  int config = 0;
  double zc[4] = {0, 0, 0, 0};
  double coup = 0;
  std::vector<int> good;
  std::mutex mu;
  std::unordered_map<uintptr_t, Workspace> ws;  // keyed by stream (and purpose)
  std::string err;
  int* err_host = nullptr;  // mapped pinned word the kernels raise on a timed-out wait
  int* err_dev = nullptr;
  int nsm = 1;              // streaming multiprocessors of the handle's device
  int max_blocks = 0;       // cap on the persistent grid (0: as many as are resident)
  int64_t wait_limit = -1;  // polls of the mixed kernel's MMA-completion wait (-1: default)
};

namespace meb300 {
namespace detail {

// Bytes of workspace of one persistent launch (one row per resident thread), and its
// carve-up.
struct Carve {
  size_t cum = 0, colw = 0, slots = 0, ktab = 0, den = 0, jt = 0;
  size_t total() const { return cum + colw + slots + ktab + den + jt; }
};

// A me_compute call: the main pass (one persistent launch per chunk of at most 2^30
// events), the rescue list of ill-conditioned events (FP32 and mixed modes) and the
// helicity-split FP64 pass over that list, and where each lives in the call's workspace.
struct CallPlan {
  int prec = 0, config = 0;
  int64_t chunk = 0;
  int grid = 0, block = 0;  // persistent grid of the main pass
  int hsplit = 1;           // threads per event of the main pass (helicity split)
  int ept = 1;              // events per thread of the main pass (2: packed FP32 kernel)
  Carve main;
  bool rescue = false;
  int rescue_cap = 0, rescue_grid = 0, rescue_hsplit = 1;
  size_t off_count = 0, off_list = 0, off_cum = 0, off_colw = 0, off_slots = 0, off_ktab = 0, off_den = 0,
         off_j = 0;
  size_t total = 0;
};

int fail(me_handle* h, int code, const std::string& msg);
int cuda_fail(me_handle* h, cudaError_t e, const char* where);
void fill_common(const me_handle* h, MeLaunch& a);
bool is_device_ptr(const void* p);
// stream-ordered workspace of the handle under key, grown to at least bytes
int get_workspace(me_handle* h, uintptr_t key, cudaStream_t s, size_t bytes, void** out);
Carve carve(const ProcessOps* ops, const LaunchNeeds& nd, int ngood, int64_t rows, bool want_hel, bool want_col);
int persistent_grid(const me_handle* h, const LaunchNeeds& nd, int64_t nevt);
std::vector<double> final_masses(const ProcessOps* ops, double mt);
cudaError_t launch_chunks(const ProcessOps* ops, int prec, int config, MeLaunch a, int64_t nevt, int64_t chunk,
                          int grid, int block, int hsplit,
                          const Carve& cv, void* wsp, cudaStream_t s, int ept);
CallPlan plan_call(const me_handle* h, int64_t nevt, int64_t chunk, bool want_hel, bool want_col);
cudaError_t run_call(const me_handle* h, const CallPlan& cp, const MeLaunch& a, int64_t nevt, void* wsp, cudaStream_t s);
// the body of me_compute for checked device arguments; with wgt, the fused unweighting
// outputs w (may be null) and the batch maximum's bit pattern (cleared by the caller)
int compute_device(me_handle* h, int64_t nevt, const double* momenta, const double* alphas, const double* rnd_hel,
                   const double* rnd_col, double* me, int32_t* sel_hel, int32_t* sel_col, cudaStream_t s,
                   const double* wgt, double* w, unsigned long long* wmax_bits);

}  // namespace detail
}  // namespace meb300
