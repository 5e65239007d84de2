// me_kernels.cuh -- the event-parallel matrix-element kernel: one event per thread (or,
// for the FP64 rescue pass, one event per group of up to 32 threads that split its
// helicities), on a persistent grid that walks the batch tile by tile.
//
// Per event:
//   1. load the FP64 momenta (array of structures, 16-byte vector loads);
//   2. evaluate every propagator denominator once, in FP64 (the only place where a
//      near-resonant top propagator can cancel), and keep 1/D in the working precision;
//   3. for each helicity kept by the filter: external wavefunctions, off-shell currents
//      and diagram terms accumulate the colour-flow amplitudes J (generated straight-line
//      code), then |M_h|^2 = g_s^(2n) sum_ij CF_ij Re(J_i^* J_j) / COL_DEN, accumulated
//      in FP64 over helicities;
//   4. me = total / IDEN and the helicity / colour selection from rnd_hel / rnd_col.
//
// Where each per-thread array lives is a per-process, per-precision choice (a Layout):
// registers for small processes; shared memory laid out [index][thread] so that a
// warp touches consecutive words; or a global tile per block laid out [index][thread]
// so that a warp's accesses coalesce.  The generated code keeps at most a fixed number of
// currents in registers (the variant's budget) and the rest in a slot buffer.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "helas.cuh"

namespace meb300 {

constexpr int MAX_COMB = 128;
// polls of a bounded spin on an mbarrier before the kernel gives up (error flag, NaN)
constexpr uint32_t kMmaWaitDefault = 1u << 22;

struct MeLaunch {
  int64_t nevt;
  const double* mom;
  const double* alphas;
  double alphas_default;
  const double* rnd_hel;
  const double* rnd_col;
  double* me;
  int32_t* sel_hel;
  int32_t* sel_col;
  double mt, wt;
  int zwt;
  double zc[4];      // e+e- -> mu+mu-: Z couplings gL, gR (units of e), mZ, wZ
  double coup;       // e+e- -> mu+mu-: e^4
  int ngood;
  int cum_mode;      // 0: cum holds running sums; 1: cum holds each |M_h|^2 (filter pass)
  uint8_t good[MAX_COMB];
  // Workspace.  The grid is persistent (at most the blocks that are resident at once);
  // each thread walks the batch and owns one workspace row, row = blockIdx.x * BLOCK +
  // threadIdx.x of gridDim.x * BLOCK rows, so the workspace scales with the resident
  // threads, not with the batch.
  double* cum;       // [ngood][rows]
  double* colw;      // [ncol][rows] (when the colour weights live in global memory)
  void* slots;       // [block][nslot][BLOCK][4] complex (slot buffer in global memory)
  void* ktab;        // [block][nkvec][BLOCK][4] real (momentum table in global memory)
  void* dtile;       // [block][nden_g][BLOCK] real, then [block][nden_t][BLOCK] complex (denominators in global memory)
  void* jtile;       // [block][ncol][BLOCK] complex (colour-flow amplitudes in global memory)
  // fused batch unweighting (me_compute_unweight): w = me * wgt per event and the batch
  // maximum of the valid weights, formed in the epilogue (null when not requested)
  const double* wgt;
  double* w;
  unsigned long long* wmax_bits;  // the maximum as the bit pattern of a non-negative double
  int* err;          // set to 1 when a bounded device-side wait runs out (mapped host memory)
  uint32_t mma_wait_limit;  // polls of the mixed kernel's wait for its MMAs (0: give up at once)
  // precision rescue (FP32 and mixed passes): events whose conditioning kappa exceeds
  // rescue_kappa are appended, as ibase + local index, to rescue_list (capacity
  // rescue_cap, counter rescue_count) for a later FP64 pass
  double rescue_kappa;
  int* rescue_count;
  int* rescue_list;
  int rescue_cap;
  int64_t ibase;
  // indexed mode (the FP64 rescue pass): process events index[0 .. min(*index_count,
  // index_cap)) instead of 0 .. nevt
  const int* index;
  const int* index_count;
  int index_cap;
  int grid_blocks;   // blocks of the launch (persistent grid)
  // helicity split: a group of hsplit consecutive threads (a power of two up to 32)
  // shares one event, each lane taking a contiguous slice of the helicities; the group
  // combines the lanes' sums with warp shuffles in a fixed order.  1 = one thread per
  // event.  Used where events are few (the FP64 rescue pass, small batches), so that the
  // latency of one event is spread over many threads.
  int hsplit;
};

// Fused unweighting, epilogue part: the event weight w = me * wgt and this thread's
// running maximum of the valid weights (finite and >= 0).  An event that the FP32 and
// mixed main passes flag for the FP64 rescue is left to the rescue pass, so that its
// reduced-precision value never enters the maximum.
__device__ __forceinline__ void fuse_weight(const MeLaunch& a, int64_t ievt, double me, bool flagged, double& wmax) {
  if (!a.wgt || flagged) return;
  const double wi = me * a.wgt[ievt];
  if (a.w) a.w[ievt] = wi;
  if (isfinite(wi) && wi >= 0.0) wmax = fmax(wmax, wi);
}
// The block maximum of the threads' running maxima and one 64-bit atomicMax per block on
// its bit pattern (non-negative IEEE doubles order like their bit patterns).  Every
// thread of the block calls it, once, after its tile loop.
static __device__ __noinline__ void flush_wmax(const MeLaunch& a, double wmax) {
  if (!a.wmax_bits) return;  // the same for the whole block
  __shared__ double s_m[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wmax = fmax(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
  const int warp = threadIdx.x >> 5, nwarp = (blockDim.x + 31) >> 5;
  if ((threadIdx.x & 31) == 0) s_m[warp] = wmax;
  __syncthreads();
  if (threadIdx.x < 32) {
    wmax = threadIdx.x < nwarp ? s_m[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wmax = fmax(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
    if (threadIdx.x == 0 && wmax > 0.0)
      atomicMax(a.wmax_bits, static_cast<unsigned long long>(__double_as_longlong(wmax)));
  }
}

// view of an array laid out [index][S]
template <class T, int S>
struct Strided {
  T* b;
  HD T& operator[](int i) const { return b[i * S]; }
};

// Launch configuration of one (process, precision):
//   V        jamps variant (register budget) of the generated code
//   BLOCK    threads per block
//   DEN_MODE denominators: 0 registers, 1 shared memory, 2 global tile per block
//   J_MODE   colour-flow amplitudes: 0 registers, 1 shared memory, 2 global tile per block
//   W_MODE   colour weights: 0 registers, 1 shared memory, 2 global workspace
//   S_MODE   slot buffer: 0 none, 1 shared memory, 2 global workspace
//   K_MODE   momentum table: 1 shared memory, 2 global workspace
//   SYNC     0: no block barriers in the helicity body; k > 0: a barrier every 8k schedule
//            steps (currents and diagram closings) and between diagram groups
//   MINB     blocks per SM the compiler must fit (caps the registers per thread)
template <int V_, int BLOCK_, int DEN_MODE, int J_MODE, int W_MODE, int S_MODE, int K_MODE, int SYNC = 0,
          int MINB = 1>
struct Layout {
  static constexpr int V = V_, BLOCK = BLOCK_, minb = MINB;
  static constexpr int den_mode = DEN_MODE, j_mode = J_MODE;
  // "view": an array laid out [index][BLOCK] (shared or global) rather than registers
  static constexpr bool den_view = DEN_MODE != 0, j_view = J_MODE != 0;
  static constexpr bool den_smem = DEN_MODE == 1, j_smem = J_MODE == 1;
  static constexpr int sync = SYNC;
  static constexpr int w_mode = W_MODE, s_mode = S_MODE, k_mode = K_MODE;
};

// Dynamic shared memory above which a kernel opts in to more than the default 48 KB per
// block.  The limit counts the kernel's static shared memory too (a few hundred bytes
// here), so the opt-in starts well below 48 KB.
constexpr size_t kSmemOptIn = 40 * 1024;

template <class P, class R, class L>
constexpr size_t me_smem_bytes() {
  size_t b = 0;
  if (L::den_smem) b += size_t(P::NDEN_G) * L::BLOCK * sizeof(R) + size_t(P::NDEN_T) * L::BLOCK * sizeof(cx<R>);
  if (L::j_smem) b += size_t(P::NCOL) * L::BLOCK * sizeof(cx<R>);
  if (L::w_mode == 1) b += size_t(P::NCOL) * L::BLOCK * sizeof(R);
  if (L::s_mode == 1) b += size_t(P::template nslot<L::V>()) * L::BLOCK * 4 * sizeof(cx<R>);
  if (L::k_mode == 1) b += size_t(P::NKVEC) * L::BLOCK * 4 * sizeof(R);
  return b;
}

template <class P, class L, class R, class DG, class DT, class JA>
__device__ __forceinline__ void call_jamps(int h, const MeLaunch& a, const DG& dg, const DT& dt, JA& J, cx<R>* ws,
                                           const R* kt) {
  if constexpr (P::QCD) {
    P::template jamps<L::V, L::BLOCK * 4, R, L::sync>(h, R(a.mt), dg, dt, J, ws, kt);
  } else {
    const R zc[2] = {R(a.zc[0]), R(a.zc[1])};
    P::template jamps<L::V, L::BLOCK * 4, R, L::sync>(h, zc, dg, dt, J, ws, kt);
  }
}

// Colour sum of flows held in shared memory, out of line so that its register use
// (every J is read by many rows) does not add to that of the amplitude code.
template <class P, class R, int BLOCK>
__device__ __noinline__ R colour_sum_strided(cx<R>* s_J_t) {
  Strided<cx<R>, BLOCK> J{s_J_t};
  return P::template colour_sum<R>(J);
}

// One helicity of one event for the large processes: currents, diagram closings,
// colour sum and colour weights.  Kept out of line so that the helicity-independent
// loads (denominators, momentum table) cannot be hoisted out of the helicity loop into
// registers that would stay live across it; everything per helicity lives here.
template <class P, class R, class L, bool COLOUR = true>
__device__ __noinline__ R one_helicity(int h, R mt, R* s_dg_t, cx<R>* s_dt_t, cx<R>* s_J_t, R* s_w_t, double* colw_t,
                                       int64_t colw_stride, cx<R>* ws, const R* kt, bool want_w) {
  constexpr int BLOCK = L::BLOCK;
  Strided<R, BLOCK> dg{s_dg_t};
  Strided<cx<R>, BLOCK> dt{s_dt_t};
  R cs;
  auto weights = [&](const cx<R> z, int c) {
    const R m2 = z.r * z.r + z.i * z.i;
    if constexpr (L::w_mode == 1) s_w_t[c * BLOCK] += m2;
    else if constexpr (L::w_mode == 2) colw_t[c * colw_stride] += double(m2);
  };
  if constexpr (L::j_view) {
    Strided<cx<R>, BLOCK> J{s_J_t};
    for (int c = 0; c < P::NCOL; ++c) J[c] = mk<R>(R(0), R(0));
    P::template jamps<L::V, BLOCK * 4, R, L::sync>(h, mt, dg, dt, J, ws, kt);
    cs = COLOUR ? colour_sum_strided<P, R, BLOCK>(s_J_t) : R(0);
    if (want_w)
      for (int c = 0; c < P::NCOL; ++c) weights(J[c], c);
  } else {
    cx<R> J[P::NCOL];
#pragma unroll
    for (int c = 0; c < P::NCOL; ++c) J[c] = mk<R>(R(0), R(0));
    P::template jamps<L::V, BLOCK * 4, R, L::sync>(h, mt, dg, dt, J, ws, kt);
    cs = P::template colour_sum<R>(J);
    if (want_w) {
#pragma unroll
      for (int c = 0; c < P::NCOL; ++c) weights(J[c], c);
    }
  }
  return cs;
}

// this block's tiles of the global denominator and colour-flow-amplitude workspaces
template <class P, class R, int BLOCK>
__device__ __forceinline__ R* den_tile_g(const MeLaunch& a) {
  const size_t per_block = size_t(P::NDEN_G) * BLOCK * sizeof(R) + size_t(P::NDEN_T) * BLOCK * sizeof(cx<R>);
  return reinterpret_cast<R*>(static_cast<char*>(a.dtile) + size_t(blockIdx.x) * per_block);
}
template <class P, class R, int BLOCK>
__device__ __forceinline__ cx<R>* den_tile_t(const MeLaunch& a) {
  return reinterpret_cast<cx<R>*>(den_tile_g<P, R, BLOCK>(a) + size_t(P::NDEN_G) * BLOCK);
}
template <class P, class R, int BLOCK>
__device__ __forceinline__ cx<R>* j_tile(const MeLaunch& a) {
  return static_cast<cx<R>*>(a.jtile) + size_t(blockIdx.x) * P::NCOL * BLOCK;
}

template <class P, class R, class L>
__global__ void __launch_bounds__(L::BLOCK, L::minb) me_kernel(const MeLaunch a) {
  constexpr int BLOCK = L::BLOCK;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x;
  const int64_t count = a.index ? int64_t(*a.index_count < a.index_cap ? *a.index_count : a.index_cap) : a.nevt;
  const int G = a.hsplit > 1 ? a.hsplit : 1;  // threads per event
  const int64_t nunit = count * G;
  const int64_t ntile = (nunit + BLOCK - 1) / BLOCK;
  const int lane = tid & (G - 1);
  const int64_t wrow = int64_t(blockIdx.x) * BLOCK + tid;  // this thread's workspace row
  const int64_t wstride = int64_t(gridDim.x) * BLOCK;
  // The persistent grid walks the batch one tile of BLOCK events at a time.  The tile
  // loop is uniform over the block: a thread past the end of the batch mirrors its last
  // event and writes nothing, so every thread reaches every block barrier.
  // A group of G threads never straddles the end of the batch (nunit is a multiple of G
  // and BLOCK of 32), so the shuffles below always see whole groups.
  double wmax_t = 0.0;  // fused unweighting: this thread's largest valid weight
  for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
  const int64_t unit = tile * BLOCK + tid;
  const bool active = unit < nunit;
  const int64_t ipos = active ? unit / G : count - 1;
  const int64_t ievt = a.index ? int64_t(a.index[ipos]) : ipos;

  // 1. momenta
  double pd[P::NPAR][4];
  {
    const double2* src = reinterpret_cast<const double2*>(a.mom + ievt * (P::NPAR * 4));
#pragma unroll
    for (int i = 0; i < P::NPAR; ++i) {
      const double2 v0 = __ldg(src + 2 * i), v1 = __ldg(src + 2 * i + 1);
      pd[i][0] = v0.x; pd[i][1] = v0.y; pd[i][2] = v1.x; pd[i][3] = v1.y;
    }
  }

  // shared-memory carve-up
  unsigned char* sp = smem_raw;
  R* s_dg = nullptr;
  cx<R>* s_dt = nullptr;
  cx<R>* s_J = nullptr;
  R* s_w = nullptr;
  cx<R>* s_slots = nullptr;
  R* s_kt = nullptr;
  if constexpr (L::den_smem) {
    s_dg = reinterpret_cast<R*>(sp); sp += size_t(P::NDEN_G) * BLOCK * sizeof(R);
    s_dt = reinterpret_cast<cx<R>*>(sp); sp += size_t(P::NDEN_T) * BLOCK * sizeof(cx<R>);
  } else if constexpr (L::den_mode == 2) {
    s_dg = den_tile_g<P, R, BLOCK>(a);
    s_dt = den_tile_t<P, R, BLOCK>(a);
  }
  if constexpr (L::j_smem) { s_J = reinterpret_cast<cx<R>*>(sp); sp += size_t(P::NCOL) * BLOCK * sizeof(cx<R>); }
  else if constexpr (L::j_mode == 2) s_J = j_tile<P, R, BLOCK>(a);
  if constexpr (L::w_mode == 1) { s_w = reinterpret_cast<R*>(sp); sp += size_t(P::NCOL) * BLOCK * sizeof(R); }
  constexpr int NS = P::template nslot<L::V>();
  static_assert(NS == 0 || L::s_mode != 0, "this jamps variant needs a slot buffer");
  static_assert(!P::template grouped<L::V>() || (L::den_view && L::j_view),
                "diagram-group variants take views of the denominators and J");
  if constexpr (L::s_mode == 1) { s_slots = reinterpret_cast<cx<R>*>(sp); sp += size_t(NS) * BLOCK * 4 * sizeof(cx<R>); }
  if constexpr (L::k_mode == 1) { s_kt = reinterpret_cast<R*>(sp); }

  // Slot buffer and momentum table: entry s of this thread at base + s * (BLOCK * 4),
  // 4 consecutive values.  Both shared and global placements use one tile per block,
  // so the stride is a compile-time constant and every access is base + immediate.
  cx<R>* ws = nullptr;
  if constexpr (L::s_mode == 1) ws = s_slots + tid * 4;
  else if constexpr (L::s_mode == 2) ws = static_cast<cx<R>*>(a.slots) + (size_t(blockIdx.x) * NS * BLOCK + tid) * 4;
  R* kt;
  if constexpr (L::k_mode == 1) kt = s_kt + tid * 4;
  else kt = static_cast<R*>(a.ktab) + (size_t(blockIdx.x) * P::NKVEC * BLOCK + tid) * 4;

  // 2. denominators and momentum table, FP64 once per event
  R r_dg[L::den_view ? 1 : P::NDEN_G];
  cx<R> r_dt[L::den_view ? 1 : P::NDEN_T];
  Strided<R, BLOCK> v_dg{s_dg + tid};
  Strided<cx<R>, BLOCK> v_dt{s_dt + tid};
  double gfac, kappa;
  if constexpr (P::QCD) {
    if constexpr (L::den_view) kappa = P::template precompute<BLOCK * 4, R>(pd, a.mt, a.wt, a.zwt, v_dg, v_dt, kt);
    else kappa = P::template precompute<BLOCK * 4, R>(pd, a.mt, a.wt, a.zwt, r_dg, r_dt, kt);
    const double as = a.alphas ? a.alphas[ievt] : a.alphas_default;
    const double g2 = 4.0 * 3.14159265358979323846 * as;
    double gp = 1.0;
#pragma unroll
    for (int k = 0; k < P::NGLUON; ++k) gp *= g2;
    gfac = gp / double(P::COL_DEN);
  } else {
    if constexpr (L::den_view) kappa = P::template precompute<BLOCK * 4, R>(pd, a.zc[2], a.zc[3], 0, v_dg, v_dt, kt);
    else kappa = P::template precompute<BLOCK * 4, R>(pd, a.zc[2], a.zc[3], 0, r_dg, r_dt, kt);
    gfac = a.coup / double(P::COL_DEN);
  }
  const bool flagged = a.rescue_list && kappa > a.rescue_kappa;
  if (active && lane == 0 && flagged) {
    const int slot = atomicAdd(a.rescue_count, 1);
    if (slot < a.rescue_cap) a.rescue_list[slot] = int(a.ibase + ievt);
  }

  // colour weights
  const bool want_w = a.sel_col != nullptr && P::NCOL > 1;
  R r_w[L::w_mode == 0 ? P::NCOL : 1];
  Strided<R, BLOCK> v_w{s_w + tid};
  if (want_w) {
    if constexpr (L::w_mode == 0) {
#pragma unroll
      for (int c = 0; c < P::NCOL; ++c) r_w[c] = R(0);
    } else if constexpr (L::w_mode == 1) {
      for (int c = 0; c < P::NCOL; ++c) v_w[c] = R(0);
    } else {
      for (int c = 0; c < P::NCOL; ++c) a.colw[c * wstride + wrow] = 0.0;
    }
  }

  // 3. helicity loop: helicities [h0, h0 + hper) of the good list (all of them when
  // G == 1); the trip count is the same for every thread, so block barriers stay
  // uniform, and a slot past the end of the list computes a copy and discards it
  double total = 0.0;
  const int hper = (a.ngood + G - 1) / G;
  const int h0 = lane * hper;
#pragma unroll 1
  for (int k = 0; k < hper; ++k) {
    const int ih = h0 + k;
    const bool valid = ih < a.ngood;
    const int h = a.good[valid ? ih : a.ngood - 1];
    // keep the block's warps on the same stretch of the (very long, straight-line)
    // helicity body, so that instruction fetches are shared instead of thrashing
    if constexpr (L::sync > 0) __syncthreads();
    R cs;
    if constexpr (P::QCD && L::den_view && L::w_mode != 0) {
      cs = one_helicity<P, R, L>(h, R(a.mt), s_dg + tid, s_dt + tid, L::j_view ? s_J + tid : nullptr,
                                 L::w_mode == 1 ? s_w + tid : nullptr, a.colw ? a.colw + wrow : nullptr, wstride,
                                 ws, kt, want_w && valid);
    } else if constexpr (L::j_view) {
      Strided<cx<R>, BLOCK> J{s_J + tid};
      for (int c = 0; c < P::NCOL; ++c) J[c] = mk<R>(R(0), R(0));
      if constexpr (L::den_view) call_jamps<P, L>(h, a, v_dg, v_dt, J, ws, kt);
      else call_jamps<P, L>(h, a, r_dg, r_dt, J, ws, kt);
      cs = P::template colour_sum<R>(J);
      if (want_w) {
        for (int c = 0; c < P::NCOL; ++c) {
          const cx<R> z = J[c];
          const R m2 = valid ? z.r * z.r + z.i * z.i : R(0);
          if constexpr (L::w_mode == 0) r_w[c] += m2;
          else if constexpr (L::w_mode == 1) v_w[c] += m2;
          else a.colw[c * wstride + wrow] += double(m2);
        }
      }
    } else {
      cx<R> J[P::NCOL];
#pragma unroll
      for (int c = 0; c < P::NCOL; ++c) J[c] = mk<R>(R(0), R(0));
      if constexpr (L::den_view) call_jamps<P, L>(h, a, v_dg, v_dt, J, ws, kt);
      else call_jamps<P, L>(h, a, r_dg, r_dt, J, ws, kt);
      cs = P::template colour_sum<R>(J);
      if (want_w) {
#pragma unroll
        for (int c = 0; c < P::NCOL; ++c) {
          const R m2 = valid ? J[c].r * J[c].r + J[c].i * J[c].i : R(0);
          if constexpr (L::w_mode == 0) r_w[c] += m2;
          else if constexpr (L::w_mode == 1) v_w[c] += m2;
          else a.colw[c * wstride + wrow] += double(m2);
        }
      }
    }
    const double mh = valid ? double(cs) * gfac : 0.0;
    total += mh;
    // split groups keep each |M_h|^2 for the group's first lane to sum in order
    if (a.cum && valid) a.cum[ih * wstride + wrow] = (a.cum_mode || G > 1) ? mh : total;
  }

  // 4. outputs
  int sel_split = 0;
  if (G > 1) {
    // The group's first lane sums the |M_h|^2 of all lanes in helicity order, exactly as
    // one thread would, so the result and the helicity selection do not depend on the
    // split.  The colour weights are summed over the lanes by a butterfly (the same bits
    // in every lane), a reassociation of the one-thread sum.
    const unsigned full = 0xffffffffu;
    __syncwarp();
    if (lane == 0) {
      double run = 0.0, prev = 0.0;
      const double target = a.sel_hel ? a.rnd_hel[ievt] : 0.0;  // scaled below
      for (int ih = 0; ih < a.ngood; ++ih) run += a.cum[ih * wstride + wrow + ih / hper];
      total = run;
      if (a.sel_hel && total > 0.0) {
        const double t = target * total;
        int found = -1, lastnz = -1;
        run = 0.0;
        for (int ih = 0; ih < a.ngood; ++ih) {
          run += a.cum[ih * wstride + wrow + ih / hper];
          if (run > prev) lastnz = ih;
          if (run > t) { found = ih; break; }
          prev = run;
        }
        const int pick = found >= 0 ? found : lastnz;
        sel_split = pick >= 0 ? a.good[pick] : 0;
      }
    }
    if (want_w) {
      for (int c = 0; c < P::NCOL; ++c) {
        double w;
        if constexpr (L::w_mode == 0) w = double(r_w[c]);
        else if constexpr (L::w_mode == 1) w = double(v_w[c]);
        else w = a.colw[c * wstride + wrow];
        for (int o = G >> 1; o > 0; o >>= 1) w += __shfl_xor_sync(full, w, o, G);
        if constexpr (L::w_mode == 0) r_w[c] = R(w);
        else if constexpr (L::w_mode == 1) v_w[c] = R(w);
        else a.colw[c * wstride + wrow] = w;
      }
    }
  }
  if (!active || lane != 0) continue;
  a.me[ievt] = total / double(P::IDEN);
  fuse_weight(a, ievt, total / double(P::IDEN), flagged, wmax_t);
  if (G > 1 && a.sel_hel) {
    a.sel_hel[ievt] = sel_split;
  } else if (a.sel_hel && a.cum && !a.cum_mode) {
    int sel = 0;
    if (total > 0.0) {
      const double target = a.rnd_hel[ievt] * total;
      int found = -1, lastnz = -1;
      double prev = 0.0;
      for (int ih = 0; ih < a.ngood; ++ih) {
        const double c = a.cum[ih * wstride + wrow];
        if (c > prev) lastnz = ih;
        if (c > target) { found = ih; break; }
        prev = c;
      }
      const int pick = found >= 0 ? found : lastnz;
      sel = pick >= 0 ? a.good[pick] : 0;
    }
    a.sel_hel[ievt] = sel;
  }
  if (a.sel_col) {
    int sel = 0;
    if (want_w) {
      double wt_tot = 0.0;
      for (int c = 0; c < P::NCOL; ++c) {
        if constexpr (L::w_mode == 0) wt_tot += double(r_w[c]);
        else if constexpr (L::w_mode == 1) wt_tot += double(v_w[c]);
        else wt_tot += a.colw[c * wstride + wrow];
      }
      if (wt_tot > 0.0) {
        const double target = a.rnd_col[ievt] * wt_tot;
        double run = 0.0;
        int found = -1, lastnz = -1;
        for (int c = 0; c < P::NCOL; ++c) {
          double w;
          if constexpr (L::w_mode == 0) w = double(r_w[c]);
          else if constexpr (L::w_mode == 1) w = double(v_w[c]);
          else w = a.colw[c * wstride + wrow];
          run += w;
          if (w > 0.0) lastnz = c;
          if (run > target) { found = c; break; }
        }
        sel = found >= 0 ? found : (lastnz >= 0 ? lastnz : 0);
      }
    }
    a.sel_col[ievt] = sel;
  }
  }  // tile loop
  flush_wmax(a, wmax_t);
}

// ---------------------------------------------------------------------------
// per-process launch table
// ---------------------------------------------------------------------------
// Workspace a launch needs beyond the caller's arrays, in bytes per event.
struct LaunchNeeds {
  size_t slot_bytes_per_event;  // global slot buffer, per workspace row
  size_t ktab_bytes_per_event;  // global momentum table, per workspace row
  size_t den_bytes_per_event;   // global denominators, per workspace row
  size_t j_bytes_per_event;     // global colour-flow amplitudes, per workspace row
  bool colw_global;             // colour weights in a global [ncol][rows] array
  int block;                    // threads per block (global tiles cover whole blocks)
  int blocks_per_sm;            // resident blocks per SM (occupancy of the kernel)
  int ept = 1;                  // events per thread (2: the packed FP32 kernel); the byte
                                // counts above are per thread (workspace row)
};

struct ProcessOps {
  const char* name;
  int npar, ncomb, ncol, ndiag, namp, iden;
  long flops_amp, flops_col;
  bool has_mixed;
  int nconfig[4];  // launch configurations available per precision (index 0 is the default;
                   // 0 configurations: the precision is not built for this process)
  LaunchNeeds (*needs)(int prec, int config);
  cudaError_t (*launch)(int prec, int config, const MeLaunch& a, cudaStream_t s);
};

// Resident blocks per SM of a kernel with 'threads' threads and 'smem' bytes of dynamic
// shared memory, at least 1: the tightest of the register file (registers are granted
// per warp in units of 256), shared memory (plus the per-block reservation), threads
// and blocks per SM.  The kernel's shared-memory carveout is set to what that many
// blocks need, so the hardware can place them all.
template <class K>
int resident_blocks(K k, int threads, size_t smem) {
  int dev = 0, regs_sm = 0, smem_sm = 0, smem_res = 0, thr_sm = 0, blk_sm = 0;
  cudaFuncAttributes fa{};
  if (cudaGetDevice(&dev) != cudaSuccess || cudaFuncGetAttributes(&fa, k) != cudaSuccess ||
      cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_res, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&blk_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  const int warps = (threads + 31) / 32;
  const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;
  int b = blk_sm;
  if (regs_warp > 0) b = std::min(b, regs_sm / (warps * regs_warp));
  const size_t per_block = smem + fa.sharedSizeBytes + size_t(smem_res);
  if (per_block > 0) b = std::min<int>(b, int(size_t(smem_sm) / per_block));
  b = std::min(b, thr_sm / threads);
  b = std::max(b, 1);
  if (smem > kSmemOptIn) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  const int pct = int((size_t(b) * per_block * 100 + size_t(smem_sm) - 1) / size_t(smem_sm));
  cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, std::min(100, pct));
  cudaGetLastError();
  return b;
}

// workspace sizes of a layout (everything but the occupancy)
template <class P, class R, class L>
LaunchNeeds sizes_of() {
  LaunchNeeds n;
  n.slot_bytes_per_event = L::s_mode == 2 ? size_t(P::template nslot<L::V>()) * 4 * sizeof(cx<R>) : 0;
  n.ktab_bytes_per_event = L::k_mode == 2 ? size_t(P::NKVEC) * 4 * sizeof(R) : 0;
  n.den_bytes_per_event = L::den_mode == 2 ? size_t(P::NDEN_G) * sizeof(R) + size_t(P::NDEN_T) * sizeof(cx<R>) : 0;
  n.j_bytes_per_event = L::j_mode == 2 ? size_t(P::NCOL) * sizeof(cx<R>) : 0;
  n.colw_global = L::w_mode == 2;
  n.block = L::BLOCK;
  n.blocks_per_sm = 1;
  return n;
}

template <class P, class R, class L>
LaunchNeeds needs_of() {
  static const int bps = resident_blocks(me_kernel<P, R, L>, L::BLOCK, me_smem_bytes<P, R, L>());
  LaunchNeeds n = sizes_of<P, R, L>();
  n.blocks_per_sm = bps;
  return n;
}

template <class P, class R, class L>
cudaError_t launch_me(const MeLaunch& a, cudaStream_t s) {
  constexpr size_t smem = me_smem_bytes<P, R, L>();
  static_assert(smem <= 227 * 1024, "shared-memory footprint of this layout exceeds 227 KB");
  auto k = me_kernel<P, R, L>;
  if (smem > kSmemOptIn) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
  }
  if (a.grid_blocks <= 0) return cudaErrorInvalidConfiguration;  // the caller sizes the persistent grid
  k<<<dim3(unsigned(a.grid_blocks)), dim3(L::BLOCK), smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace meb300
