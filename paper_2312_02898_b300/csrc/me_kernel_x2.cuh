// me_kernel_x2.cuh -- the FP32 matrix-element kernel with two events per thread on
// packed FP32 pairs (fx2.cuh).
//
// The same computation as me_kernel<P, float, L> (momenta, FP64 denominators and
// momentum table, per helicity the generated currents, diagram closings and colour sum,
// FP64 helicity sum, selections), but each thread carries two events, one per lane of
// every packed value, so each fetched instruction of the long straight-line helicity body
// does the arithmetic of two events.  Per-event work outside the helicity loop (momenta,
// FP64 invariants and denominators, conditioning, coupling, selections) runs lane by lane
// with the scalar code.  The FP64 rescue pass of the FP32 mode is unchanged.
//
// Thread t of tile k of a launch holds events 2 (k BLOCK + t) and 2 (k BLOCK + t) + 1 of
// the batch.  A lane past the end of the batch mirrors the last event and writes nothing.
#pragma once

#include "fx2.cuh"
#include "me_kernels.cuh"

namespace meb300 {

// one lane of packed storage, viewed as scalar storage by the generated precompute()
// (which writes each event's denominators and momentum table with R = float)
struct LaneKt {  // momentum table: fx2 entries, consecutive indices
  float* b;
  HD float& operator[](int i) const { return b[2 * i]; }
};
template <int BLOCK>
struct LaneDg {  // real denominators: fx2 entries laid out [index][BLOCK]
  float* b;
  HD float& operator[](int i) const { return b[2 * i * BLOCK]; }
};
struct LaneCxRef {  // one lane of a c2 = {float2 r, float2 i}: floats r0 r1 i0 i1
  float* p;
  HD void operator=(cx<float> z) const { p[0] = z.r; p[2] = z.i; }
};
template <int BLOCK>
struct LaneDt {  // complex denominators: c2 entries laid out [index][BLOCK]
  float* b;
  HD LaneCxRef operator[](int i) const { return LaneCxRef{b + 4 * i * BLOCK}; }
};
// the same views of register arrays, lane LN a compile-time constant
template <int LN>
struct LaneRegG {
  fx2* b;
  HD float& operator[](int i) const { return LN ? b[i].v.y : b[i].v.x; }
};
template <int LN>
struct LaneRegCxRef {
  c2* p;
  HD void operator=(cx<float> z) const {
    if (LN) { p->r.v.y = z.r; p->i.v.y = z.i; }
    else { p->r.v.x = z.r; p->i.v.x = z.i; }
  }
};
template <int LN>
struct LaneRegT {
  c2* b;
  HD LaneRegCxRef<LN> operator[](int i) const { return LaneRegCxRef<LN>{b + i}; }
};

template <class P, class L>
constexpr size_t me_x2_smem_bytes() { return me_smem_bytes<P, fx2, L>(); }

// One helicity of one event pair: currents, closings, colour sum, colour weights.  Out of
// line for the reason given at one_helicity (nothing per event may be hoisted into
// registers that stay live across the helicity loop).
template <class P, class L>
__device__ __noinline__ fx2 one_helicity_x2(int h, fx2 mt, fx2* s_dg_t, c2* s_dt_t, c2* s_J_t, fx2* s_w_t,
                                            double2* colw_t, int64_t colw_stride, c2* ws, const fx2* kt,
                                            bool want_w) {
  constexpr int BLOCK = L::BLOCK;
  Strided<fx2, BLOCK> dg{s_dg_t};
  Strided<c2, BLOCK> dt{s_dt_t};
  fx2 cs;
  auto weights = [&](const c2 z, int c) {
    const fx2 m2 = fmadd(z.r, z.r, z.i * z.i);
    if constexpr (L::w_mode == 1) s_w_t[c * BLOCK] = s_w_t[c * BLOCK] + m2;
    else if constexpr (L::w_mode == 2) {
      double2& w = colw_t[c * colw_stride];
      w.x += double(lane(m2, 0));
      w.y += double(lane(m2, 1));
    }
  };
  if constexpr (L::j_view) {
    Strided<c2, BLOCK> J{s_J_t};
    for (int c = 0; c < P::NCOL; ++c) J[c] = mk<fx2>(fx2(0.0f), fx2(0.0f));
    P::template jamps<L::V, BLOCK * 4, fx2, L::sync>(h, mt, dg, dt, J, ws, kt);
    cs = P::template colour_sum<fx2>(J);
    if (want_w)
      for (int c = 0; c < P::NCOL; ++c) weights(J[c], c);
  } else {
    c2 J[P::NCOL];
#pragma unroll
    for (int c = 0; c < P::NCOL; ++c) J[c] = mk<fx2>(fx2(0.0f), fx2(0.0f));
    P::template jamps<L::V, BLOCK * 4, fx2, L::sync>(h, mt, dg, dt, J, ws, kt);
    cs = P::template colour_sum<fx2>(J);
    if (want_w) {
#pragma unroll
      for (int c = 0; c < P::NCOL; ++c) weights(J[c], c);
    }
  }
  return cs;
}

template <class P, class L>
__global__ void __launch_bounds__(L::BLOCK, L::minb) me_kernel_x2(const MeLaunch a) {
  static_assert(P::QCD, "the packed kernel serves the QCD processes");
  static_assert(L::den_view == (L::w_mode != 0),
                "denominators and colour weights both in registers, or both in views");
  constexpr int BLOCK = L::BLOCK;
  extern __shared__ __align__(16) unsigned char smem_x2[];
  const int tid = threadIdx.x;
  const int64_t nevt = a.nevt;
  const int64_t npair = (nevt + 1) / 2;
  const int64_t ntile = (npair + BLOCK - 1) / BLOCK;
  const int64_t wrow = int64_t(blockIdx.x) * BLOCK + tid;  // this thread's workspace row
  const int64_t wstride = int64_t(gridDim.x) * BLOCK;

  // shared-memory carve-up (as me_kernel, with packed entries)
  unsigned char* sp = smem_x2;
  fx2* s_dg = nullptr;
  c2* s_dt = nullptr;
  if constexpr (L::den_smem) {
    s_dg = reinterpret_cast<fx2*>(sp); sp += size_t(P::NDEN_G) * BLOCK * sizeof(fx2);
    s_dt = reinterpret_cast<c2*>(sp); sp += size_t(P::NDEN_T) * BLOCK * sizeof(c2);
  } else if constexpr (L::den_mode == 2) {
    s_dg = den_tile_g<P, fx2, BLOCK>(a);
    s_dt = den_tile_t<P, fx2, BLOCK>(a);
  }
  c2* s_J = nullptr;
  if constexpr (L::j_smem) { s_J = reinterpret_cast<c2*>(sp); sp += size_t(P::NCOL) * BLOCK * sizeof(c2); }
  else if constexpr (L::j_mode == 2) s_J = j_tile<P, fx2, BLOCK>(a);
  fx2* s_w = nullptr;
  if constexpr (L::w_mode == 1) { s_w = reinterpret_cast<fx2*>(sp); sp += size_t(P::NCOL) * BLOCK * sizeof(fx2); }
  constexpr int NS = P::template nslot<L::V>();
  static_assert(NS == 0 || L::s_mode != 0, "this jamps variant needs a slot buffer");
  c2* s_slots = nullptr;
  fx2* s_kt = nullptr;
  if constexpr (L::s_mode == 1) { s_slots = reinterpret_cast<c2*>(sp); sp += size_t(NS) * BLOCK * 4 * sizeof(c2); }
  if constexpr (L::k_mode == 1) s_kt = reinterpret_cast<fx2*>(sp);
  c2* ws = nullptr;
  if constexpr (L::s_mode == 1) ws = s_slots + tid * 4;
  else if constexpr (L::s_mode == 2) ws = static_cast<c2*>(a.slots) + (size_t(blockIdx.x) * NS * BLOCK + tid) * 4;
  fx2* kt;
  if constexpr (L::k_mode == 1) kt = s_kt + tid * 4;
  else kt = static_cast<fx2*>(a.ktab) + (size_t(blockIdx.x) * P::NKVEC * BLOCK + tid) * 4;
  double2* cum2 = reinterpret_cast<double2*>(a.cum);
  double2* colw2 = reinterpret_cast<double2*>(a.colw);
  const bool want_w = a.sel_col != nullptr && P::NCOL > 1;
  // register placement (small processes): denominators and colour weights per thread
  fx2 r_dg[L::den_view ? 1 : P::NDEN_G];
  c2 r_dt[L::den_view ? 1 : P::NDEN_T];
  fx2 r_w[L::w_mode == 0 ? P::NCOL : 1];

  for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int64_t pair = tile * BLOCK + tid;
    int64_t ev[2];
    bool act[2];
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      const int64_t e = 2 * pair + l;
      act[l] = e < nevt;
      ev[l] = act[l] ? e : nevt - 1;
    }

    // per event: FP64 momenta, denominators and momentum table (lane by lane), the
    // conditioning for the rescue pass and the coupling factor
    double gfac[2];
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      double pd[P::NPAR][4];
      const double2* src = reinterpret_cast<const double2*>(a.mom + ev[l] * (P::NPAR * 4));
#pragma unroll
      for (int i = 0; i < P::NPAR; ++i) {
        const double2 v0 = __ldg(src + 2 * i), v1 = __ldg(src + 2 * i + 1);
        pd[i][0] = v0.x; pd[i][1] = v0.y; pd[i][2] = v1.x; pd[i][3] = v1.y;
      }
      LaneKt ktl{reinterpret_cast<float*>(kt) + l};
      double kappa;
      if constexpr (L::den_view) {
        LaneDg<BLOCK> dgl{reinterpret_cast<float*>(s_dg + tid) + l};
        LaneDt<BLOCK> dtl{reinterpret_cast<float*>(s_dt + tid) + l};
        kappa = P::template precompute<BLOCK * 4, float>(pd, a.mt, a.wt, a.zwt, dgl, dtl, ktl);
      } else if (l == 0) {
        LaneRegG<0> dgl{r_dg};
        LaneRegT<0> dtl{r_dt};
        kappa = P::template precompute<BLOCK * 4, float>(pd, a.mt, a.wt, a.zwt, dgl, dtl, ktl);
      } else {
        LaneRegG<1> dgl{r_dg};
        LaneRegT<1> dtl{r_dt};
        kappa = P::template precompute<BLOCK * 4, float>(pd, a.mt, a.wt, a.zwt, dgl, dtl, ktl);
      }
      if (act[l] && a.rescue_list && kappa > a.rescue_kappa) {
        const int slot = atomicAdd(a.rescue_count, 1);
        if (slot < a.rescue_cap) a.rescue_list[slot] = int(a.ibase + ev[l]);
      }
      const double as = a.alphas ? a.alphas[ev[l]] : a.alphas_default;
      const double g2 = 4.0 * 3.14159265358979323846 * as;
      double gp = 1.0;
#pragma unroll
      for (int k = 0; k < P::NGLUON; ++k) gp *= g2;
      gfac[l] = gp / double(P::COL_DEN);
    }

    // colour weights
    if (want_w) {
      if constexpr (L::w_mode == 0) {
#pragma unroll
        for (int c = 0; c < P::NCOL; ++c) r_w[c] = fx2(0.0f);
      } else {
        for (int c = 0; c < P::NCOL; ++c) {
          if constexpr (L::w_mode == 1) s_w[(c * BLOCK) + tid] = fx2(0.0f);
          else colw2[c * wstride + wrow] = make_double2(0.0, 0.0);
        }
      }
    }

    // helicity loop: the same helicity for both lanes
    double total[2] = {0.0, 0.0};
    const fx2 mt2(float(a.mt));
#pragma unroll 1
    for (int ih = 0; ih < a.ngood; ++ih) {
      const int h = a.good[ih];
      if constexpr (L::sync > 0) __syncthreads();
      fx2 cs;
      if constexpr (L::den_view) {
        cs = one_helicity_x2<P, L>(h, mt2, s_dg + tid, s_dt + tid, L::j_view ? s_J + tid : nullptr,
                                   L::w_mode == 1 ? s_w + tid : nullptr, colw2 ? colw2 + wrow : nullptr, wstride,
                                   ws, kt, want_w);
      } else {
        // small processes: everything per helicity in registers, inline
        static_assert(!L::j_view, "register denominators go with register colour-flow amplitudes");
        c2 J[P::NCOL];
#pragma unroll
        for (int c = 0; c < P::NCOL; ++c) J[c] = mk<fx2>(fx2(0.0f), fx2(0.0f));
        P::template jamps<L::V, BLOCK * 4, fx2, L::sync>(h, mt2, r_dg, r_dt, J, ws, kt);
        cs = P::template colour_sum<fx2>(J);
        if (want_w) {
#pragma unroll
          for (int c = 0; c < P::NCOL; ++c) r_w[c] = r_w[c] + fmadd(J[c].r, J[c].r, J[c].i * J[c].i);
        }
      }
      total[0] += double(lane(cs, 0)) * gfac[0];
      total[1] += double(lane(cs, 1)) * gfac[1];
      if (a.cum) cum2[ih * wstride + wrow] = make_double2(total[0], total[1]);
    }

    // outputs, lane by lane
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      if (!act[l]) continue;
      const int64_t ievt = ev[l];
      a.me[ievt] = total[l] / double(P::IDEN);
      if (a.sel_hel && a.cum) {
        int sel = 0;
        if (total[l] > 0.0) {
          const double target = a.rnd_hel[ievt] * total[l];
          int found = -1, lastnz = -1;
          double prev = 0.0;
          for (int ih = 0; ih < a.ngood; ++ih) {
            const double2 c2v = cum2[ih * wstride + wrow];
            const double c = l ? c2v.y : c2v.x;
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
          auto weight = [&](int c) -> double {
            if constexpr (L::w_mode == 0) return double(lane(r_w[c], l));
            else if constexpr (L::w_mode == 1) return double(lane(s_w[c * BLOCK + tid], l));
            else {
              const double2 w = colw2[c * wstride + wrow];
              return l ? w.y : w.x;
            }
          };
          double wt_tot = 0.0;
          for (int c = 0; c < P::NCOL; ++c) wt_tot += weight(c);
          if (wt_tot > 0.0) {
            const double target = a.rnd_col[ievt] * wt_tot;
            double run = 0.0;
            int found = -1, lastnz = -1;
            for (int c = 0; c < P::NCOL; ++c) {
              const double w = weight(c);
              run += w;
              if (w > 0.0) lastnz = c;
              if (run > target) { found = c; break; }
            }
            sel = found >= 0 ? found : (lastnz >= 0 ? lastnz : 0);
          }
        }
        a.sel_col[ievt] = sel;
      }
    }
  }  // tile loop
}

template <class P, class L>
LaunchNeeds needs_x2_of() {
  static const int bps = resident_blocks(me_kernel_x2<P, L>, L::BLOCK, me_x2_smem_bytes<P, L>());
  LaunchNeeds n = sizes_of<P, fx2, L>();
  n.blocks_per_sm = bps;
  n.ept = 2;
  return n;
}

template <class P, class L>
cudaError_t launch_x2(const MeLaunch& a, cudaStream_t s) {
  constexpr size_t smem = me_x2_smem_bytes<P, L>();
  static_assert(smem <= 227 * 1024, "shared-memory footprint of this layout exceeds 227 KB");
  auto k = me_kernel_x2<P, L>;
  if (smem > kSmemOptIn) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
  }
  if (a.grid_blocks <= 0) return cudaErrorInvalidConfiguration;  // the caller sizes the persistent grid
  k<<<dim3(unsigned(a.grid_blocks)), dim3(L::BLOCK), smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace meb300
