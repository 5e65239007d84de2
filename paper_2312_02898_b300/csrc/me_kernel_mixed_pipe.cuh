// me_kernel_mixed_pipe.cuh -- the mixed-precision kernel with its tensor-core colour
// sum overlapped with the amplitude work of the next helicity (software pipelining).
//
// Same computation as me_kernel_mixed (FP32 amplitudes, colour sum D = A C on the tensor
// cores with split 16-bit operands and FP32 accumulation in TMEM, FP64 inputs,
// denominators and helicity sum), for colour bases whose real and imaginary A tiles fit
// shared memory together (one MMA round per helicity).  Per 128-event tile, helicity k:
//
//   1. the colour-flow amplitudes J_k of every thread's event, in registers;
//   2. wait for the MMAs of helicity k-1 (issued at the end of the previous step, so they
//      ran while step 1 was computing), read D_{k-1} from TMEM and form
//      |M_{k-1}|^2 = sum_c Re(J_{k-1,c}^* D_{k-1,c}) with J_{k-1} from the FP32 J store;
//   3. write J_k to the FP32 J store and its split 16-bit terms to the A tiles;
//   4. one block barrier; one elected thread issues the MMAs of helicity k and commits
//      them to the mbarrier.
//
// After the last helicity one more wait finishes it.  One barrier per helicity instead of
// two, no thread idles while the tensor cores work, and J accumulates in registers
// rather than in shared memory.  The helicity sum is still taken in helicity order, so
// the result equals the unpipelined kernel's up to the FP32 rounding of the same terms.
//
// Every wait is bounded (MeLaunch::mma_wait_limit polls).  A wait that runs out fails the
// block (a block-wide vote): its events become NaN, the error flag is raised, and before
// the TMEM columns are freed the block waits, with the default limit, for the MMAs it had
// issued.
#pragma once

#include "me_kernel_mixed.cuh"

namespace meb300 {

template <class P, int NTERM, bool F16>
struct PipeShape {
  using S = MixedShape<P, NTERM, F16>;
  static_assert(!S::TWO_ROUNDS, "the pipelined kernel needs both A tiles of a helicity in shared memory");
  static constexpr size_t JBYTES = size_t(P::NCOL) * 128 * sizeof(cx<float>);  // FP32 J store
  static constexpr size_t TC_BYTES = S::TC_BYTES + JBYTES;
};

template <class P, class L, int NTERM, bool F16>
constexpr size_t me_mixed_pipe_smem_bytes() {
  return PipeShape<P, NTERM, F16>::TC_BYTES + me_smem_bytes<P, float, L>();
}

// Steps 1-3 of one helicity (see the file comment).  Returns the colour sum of the
// previous helicity (0 when there is none); ok is false when the wait for the previous
// helicity's MMAs ran out (nothing of this helicity is stored then).  unscale holds the
// previous row's power-of-two unscaling on entry (FP16 operands) and this row's on exit.
template <class P, class L, int NTERM, bool F16>
__device__ __noinline__ float mixed_pipe_helicity(int h, float mt, float* s_dg_t, cx<float>* s_dt_t, float* s_w_t,
                                                  double* colw_t, int64_t colw_stride, cx<float>* ws,
                                                  const float* kt, bool want_w, cx<float>* sJ_t,
                                                  unsigned char* s_A, int tid, uint32_t lane_base, uint64_t* mbar,
                                                  bool have_prev, uint32_t parity, uint32_t limit, float& unscale,
                                                  bool& ok) {
  using R = float;
  using S = MixedShape<P, NTERM, F16>;
  constexpr int BLOCK = 128;
  Strided<R, BLOCK> dg{s_dg_t};
  Strided<cx<R>, BLOCK> dt{s_dt_t};
  // 1. amplitudes and colour weights
  cx<R> J[P::NCOL];
#pragma unroll
  for (int c = 0; c < P::NCOL; ++c) J[c] = mk<R>(R(0), R(0));
  P::template jamps<L::V, BLOCK * 4, R, L::sync>(h, mt, dg, dt, J, ws, kt);
  if (want_w) {
#pragma unroll
    for (int c = 0; c < P::NCOL; ++c) {
      const R m2 = J[c].r * J[c].r + J[c].i * J[c].i;
      if constexpr (L::w_mode == 1) s_w_t[c * BLOCK] += m2;
      else colw_t[c * colw_stride] += double(m2);
    }
  }
  // 2. the previous helicity
  float cs = 0.0f;
  ok = true;
  if (have_prev) {
    ok = tc::mbar_wait_bounded(mbar, parity, limit);
    if (ok) {
      tc::fence_after_sync();
#pragma unroll 1
      for (int c0 = 0; c0 < S::NP; c0 += 16) {
        float dre[16], dim[16];
        tc::tmem_ld16(lane_base + c0, dre);
        tc::tmem_ld16(lane_base + S::NP + c0, dim);
        tc::tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = c0 + j;
          if (c < S::NC) {
            const cx<R> z = sJ_t[c * BLOCK];
            cs += z.r * (dre[j] * unscale) + z.i * (dim[j] * unscale);
          }
        }
      }
    }
  }
  if (!ok) return 0.0f;
  // 3. this helicity's J: the FP32 store and the split operand rows
  float scale = 1.0f;
  unscale = 1.0f;
  if constexpr (F16) {
    float amax = 0.0f;
#pragma unroll
    for (int c = 0; c < S::NC; ++c) amax = fmaxf(amax, fmaxf(fabsf(J[c].r), fabsf(J[c].i)));
    if (amax > 0.0f && isfinite(amax)) {
      const int e = max(-120, min(120, 14 - ilogbf(amax)));
      scale = ldexpf(1.0f, e);
      unscale = ldexpf(1.0f, -e);
    }
  }
#pragma unroll
  for (int c = 0; c < P::NCOL; ++c) sJ_t[c * BLOCK] = J[c];
#pragma unroll
  for (int kc = 0; kc < S::KP / 8; ++kc) {
#pragma unroll
    for (int part = 0; part < 2; ++part) {
      float x[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = kc * 8 + j;
        x[j] = c < S::NC ? (part ? J[c].i : J[c].r) * scale : 0.0f;
      }
#pragma unroll
      for (int t = 0; t < NTERM; ++t) {
        __align__(16) uint16_t b[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) b[j] = split_term<F16>(x[j]);
        *reinterpret_cast<uint4*>(s_A + (t * 2 + part) * S::TILE + tc::kmajor_offset(tid, kc * 8, S::KP)) =
            *reinterpret_cast<const uint4*>(b);
      }
    }
  }
  return cs;
}

template <class P, class L, int NTERM, bool F16>
__global__ void __launch_bounds__(128) me_kernel_mixed_pipe(const MeLaunch a) {
  using R = float;
  using S = MixedShape<P, NTERM, F16>;
  using PS = PipeShape<P, NTERM, F16>;
  constexpr int BLOCK = 128;
  static_assert(L::BLOCK == 128, "one block is the 128-row tile of the MMA");
  static_assert(L::den_view && L::j_mode == 0 && L::w_mode != 0,
                "pipelined kernel: views of the denominators and weights, J in registers");
  static_assert(F16 ? P::CF_FP16_EXACT : P::CF_BF16_EXACT, "the colour matrix must be exact in the operand type");
  extern __shared__ __align__(16) unsigned char smem_pipe[];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t nevt = a.nevt;
  const int64_t ntile = (nevt + BLOCK - 1) / BLOCK;
  const int64_t wrow = int64_t(blockIdx.x) * BLOCK + tid;
  const int64_t wstride = int64_t(gridDim.x) * BLOCK;

  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem_pipe);
  uint64_t* s_mbar = reinterpret_cast<uint64_t*>(smem_pipe + 16);
  unsigned char* s_B = smem_pipe + S::HEAD;
  unsigned char* s_A = s_B + S::BBYTES;
  cx<R>* s_Jst = reinterpret_cast<cx<R>*>(s_A + size_t(S::NTILE) * S::TILE);
  unsigned char* sp = smem_pipe + PS::TC_BYTES;

  // --- tensor-core set-up: barrier, TMEM columns, the colour matrix as operand B
  if (tid == 0) tc::mbar_init(s_mbar, 1);
  if (warp == 0) {
    tc::tmem_alloc(s_tmem, S::TCOLS);
    tc::tmem_relinquish();
  }
  for (int idx = tid; idx < S::NP * S::KP; idx += BLOCK) {
    const int n = idx / S::KP, k = idx % S::KP;
    float v = (n < S::NC && k < S::NC) ? float(P::cf_device(n * S::NC + k)) : 0.0f;
    *reinterpret_cast<uint16_t*>(s_B + tc::kmajor_offset(n, k, S::KP)) = split_term<F16>(v);  // exact
  }
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *s_tmem;
  const uint32_t lane_base = tbase + (uint32_t(32 * warp) << 16);
  uint32_t nwait = 0;  // completed waits = index of the next commit to wait for
  bool failed = false;

  // --- per-thread working storage, carved once for all tiles
  R* s_dg;
  cx<R>* s_dt;
  if constexpr (L::den_smem) {
    s_dg = reinterpret_cast<R*>(sp); sp += size_t(P::NDEN_G) * BLOCK * sizeof(R);
    s_dt = reinterpret_cast<cx<R>*>(sp); sp += size_t(P::NDEN_T) * BLOCK * sizeof(cx<R>);
  } else {
    s_dg = den_tile_g<P, R, BLOCK>(a);
    s_dt = den_tile_t<P, R, BLOCK>(a);
  }
  R* s_w = nullptr;
  if constexpr (L::w_mode == 1) { s_w = reinterpret_cast<R*>(sp); sp += size_t(P::NCOL) * BLOCK * sizeof(R); }
  constexpr int NS = P::template nslot<L::V>();
  cx<R>* s_slots = nullptr;
  R* s_kt = nullptr;
  if constexpr (L::s_mode == 1) { s_slots = reinterpret_cast<cx<R>*>(sp); sp += size_t(NS) * BLOCK * 4 * sizeof(cx<R>); }
  if constexpr (L::k_mode == 1) s_kt = reinterpret_cast<R*>(sp);
  cx<R>* ws = nullptr;
  if constexpr (L::s_mode == 1) ws = s_slots + tid * 4;
  else if constexpr (L::s_mode == 2) ws = static_cast<cx<R>*>(a.slots) + (size_t(blockIdx.x) * NS * BLOCK + tid) * 4;
  R* kt;
  if constexpr (L::k_mode == 1) kt = s_kt + tid * 4;
  else kt = static_cast<R*>(a.ktab) + (size_t(blockIdx.x) * P::NKVEC * BLOCK + tid) * 4;
  Strided<R, BLOCK> v_dg{s_dg + tid};
  Strided<cx<R>, BLOCK> v_dt{s_dt + tid};
  R* const w_t = L::w_mode == 1 ? s_w + tid : nullptr;
  auto weight = [&](int c) -> double {
    if constexpr (L::w_mode == 1) return double(w_t[c * BLOCK]);
    else return a.colw[c * wstride + wrow];
  };

  double wmax_t = 0.0;  // fused unweighting: this thread's largest valid weight
  for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int64_t ievt_raw = tile * BLOCK + tid;
    const bool active = ievt_raw < nevt;
    const int64_t ievt = active ? ievt_raw : nevt - 1;
    if (failed) {
      // a wait of this block ran out: the rest of its tiles get NaN without any work
      if (active) {
        a.me[ievt] = __longlong_as_double(0x7ff8000000000000ll);
        if (a.sel_hel) a.sel_hel[ievt] = 0;
        if (a.sel_col) a.sel_col[ievt] = 0;
      }
      continue;
    }

    // --- per-event set-up, as in me_kernel
    double pd[P::NPAR][4];
    {
      const double2* src = reinterpret_cast<const double2*>(a.mom + ievt * (P::NPAR * 4));
#pragma unroll
      for (int i = 0; i < P::NPAR; ++i) {
        const double2 v0 = __ldg(src + 2 * i), v1 = __ldg(src + 2 * i + 1);
        pd[i][0] = v0.x; pd[i][1] = v0.y; pd[i][2] = v1.x; pd[i][3] = v1.y;
      }
    }
    const double kappa = P::template precompute<BLOCK * 4, R>(pd, a.mt, a.wt, a.zwt, v_dg, v_dt, kt);
    const bool flagged = a.rescue_list && kappa > a.rescue_kappa;
    if (active && flagged) {
      const int slot = atomicAdd(a.rescue_count, 1);
      if (slot < a.rescue_cap) a.rescue_list[slot] = int(a.ibase + ievt);
    }
    const double as = a.alphas ? a.alphas[ievt] : a.alphas_default;
    const double g2 = 4.0 * 3.14159265358979323846 * as;
    double gp = 1.0;
#pragma unroll
    for (int k = 0; k < P::NGLUON; ++k) gp *= g2;
    const double gfac = gp / double(P::COL_DEN);
    const bool want_w = a.sel_col != nullptr && P::NCOL > 1;
    if (want_w) {
      for (int c = 0; c < P::NCOL; ++c) {
        if constexpr (L::w_mode == 1) w_t[c * BLOCK] = R(0);
        else a.colw[c * wstride + wrow] = 0.0;
      }
    }

    // --- helicity loop, one step behind on the colour sum; the last pass only finishes
    double total = 0.0;
    float unscale = 1.0f;
    for (int ih = 0; ih <= a.ngood; ++ih) {
      bool ok = true;
      float cs;
      if (ih < a.ngood) {
        cs = mixed_pipe_helicity<P, L, NTERM, F16>(a.good[ih], R(a.mt), s_dg + tid, s_dt + tid, w_t,
                                                   a.colw ? a.colw + wrow : nullptr, wstride, ws, kt, want_w,
                                                   s_Jst + tid, s_A, tid, lane_base, s_mbar, ih > 0, nwait & 1u,
                                                   a.mma_wait_limit, unscale, ok);
      } else {
        cs = 0.0f;
        ok = tc::mbar_wait_bounded(s_mbar, nwait & 1u, a.mma_wait_limit);
        if (ok) {
          tc::fence_after_sync();
#pragma unroll 1
          for (int c0 = 0; c0 < S::NP; c0 += 16) {
            float dre[16], dim[16];
            tc::tmem_ld16(lane_base + c0, dre);
            tc::tmem_ld16(lane_base + S::NP + c0, dim);
            tc::tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int c = c0 + j;
              if (c < S::NC) {
                const cx<R> z = s_Jst[c * BLOCK + tid];
                cs += z.r * (dre[j] * unscale) + z.i * (dim[j] * unscale);
              }
            }
          }
        }
      }
      tc::fence_proxy_async_smem();
      tc::fence_before_sync();
      if (__syncthreads_or(!ok)) {  // the same value in every thread of the block
        failed = true;
        break;
      }
      if (ih > 0) {
        ++nwait;
        const double mh = double(cs) * gfac;
        total += mh;
        if (a.cum) a.cum[(ih - 1) * wstride + wrow] = total;
      }
      if (ih < a.ngood && tid == 0) {
        tc::fence_after_sync();
        for (int part = 0; part < 2; ++part)
          for (int t = 0; t < NTERM; ++t)
            for (int ks = 0; ks < S::KP / 16; ++ks) {
              const uint64_t ad = tc::smem_desc(tc::smem_u32(s_A + (t * 2 + part) * S::TILE) + ks * 256, 128, S::KP * 16);
              const uint64_t bd = tc::smem_desc(tc::smem_u32(s_B) + ks * 256, 128, S::KP * 16);
              tc::mma_f16kind(tbase + part * S::NP, ad, bd, S::IDESC, (t > 0 || ks > 0) ? 1u : 0u);
            }
        tc::mma_commit(s_mbar);
      }
    }

    if (!active) continue;
    a.me[ievt] = failed ? __longlong_as_double(0x7ff8000000000000ll) : total / double(P::IDEN);
    if (!failed) fuse_weight(a, ievt, total / double(P::IDEN), flagged, wmax_t);
    if (a.sel_hel && a.cum) {
      int sel = 0;
      if (total > 0.0 && !failed) {
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
      if (want_w && !failed) {
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
  }  // tile loop

  flush_wmax(a, wmax_t);

  // --- teardown: the commit whose wait ran out may still be in flight; wait for it with
  // the default limit before the columns are freed
  if (failed) {
    if (tid == 0 && a.err) atomicOr(a.err, 1);
    tc::mbar_wait_bounded(s_mbar, nwait & 1u, kMmaWaitDefault);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tbase, S::TCOLS);
  }
}

template <class P, class L, int NTERM, bool F16>
LaunchNeeds needs_mixed_pipe_of() {
  static const int bps =
      resident_blocks(me_kernel_mixed_pipe<P, L, NTERM, F16>, 128, me_mixed_pipe_smem_bytes<P, L, NTERM, F16>());
  LaunchNeeds n = sizes_of<P, float, L>();
  n.blocks_per_sm = bps;
  return n;
}

template <class P, class L, int NTERM, bool F16>
cudaError_t launch_mixed_pipe(const MeLaunch& a, cudaStream_t s) {
  constexpr size_t smem = me_mixed_pipe_smem_bytes<P, L, NTERM, F16>();
  static_assert(smem <= 227 * 1024, "shared-memory footprint of the pipelined mixed kernel exceeds 227 KB");
  auto k = me_kernel_mixed_pipe<P, L, NTERM, F16>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  if (a.grid_blocks <= 0) return cudaErrorInvalidConfiguration;  // the caller sizes the persistent grid
  k<<<dim3(unsigned(a.grid_blocks)), dim3(128), smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace meb300
