// me_kernel_mixed.cuh -- the mixed-precision matrix-element kernel: FP32 amplitudes
// (generated code, one event per thread, as in me_kernel), colour sum on the tensor
// cores (colour_mma.cuh), FP64 inputs, denominators and helicity sum.
//
// One block tile = 128 events = the M = 128 rows of one tcgen05 MMA.  The grid is
// persistent: each block sets up its tensor-core state once and walks the batch tile by
// tile.  Every thread of the block takes part in every barrier (threads past the end
// of the batch mirror the last event and write nothing).
//
// Operand type: BF16 when the integer colour matrix is exact in BF16 (8-bit
// significand), else FP16 (11 bits).  FP16 has a narrow exponent range, so each event's
// row of J is first scaled by a power of two that brings its largest component near
// 2^14; the row of D = (sJ) C is scaled back exactly.  A large colour basis writes and
// multiplies the real and imaginary parts in two rounds through one set of A tiles, so
// that the tiles fit beside the colour matrix in shared memory.
#pragma once

#include <cuda_fp16.h>

#include "colour_mma.cuh"
#include "me_kernels.cuh"

namespace meb300 {


template <class P, int NTERM, bool F16>
struct MixedShape {
  static constexpr int NC = P::NCOL;
  static constexpr int KP = (NC + 15) / 16 * 16;  // flows padded to the MMA K step
  static constexpr int NP = KP;                   // C is square
  static_assert(NP <= 256, "MMA N is at most 256");
  static constexpr uint32_t TILE = 128u * KP * 2;  // one 16-bit A tile
  static constexpr bool TWO_ROUNDS = 2u * NTERM * TILE > 64u * 1024u;
  static constexpr int NTILE = TWO_ROUNDS ? NTERM : 2 * NTERM;  // A tiles in shared memory
  static constexpr uint32_t BBYTES = (uint32_t(NP) * KP * 2 + 1023u) / 1024u * 1024u;
  static constexpr uint32_t TCOLS = (2 * NP <= 32) ? 32 : (2 * NP <= 64) ? 64 : (2 * NP <= 128) ? 128 : (2 * NP <= 256) ? 256 : 512;
  static constexpr uint32_t IDESC = tc::idesc_f16kind(128, NP, F16);
  static constexpr size_t HEAD = 1024;  // TMEM address, mbarrier
  static constexpr size_t TC_BYTES = HEAD + BBYTES + size_t(NTILE) * TILE;
};

template <class P, class L, int NTERM, bool F16>
constexpr size_t me_mixed_smem_bytes() {
  return MixedShape<P, NTERM, F16>::TC_BYTES + me_smem_bytes<P, float, L>();
}

// one 16-bit term of x (rounded to nearest), leaving the remainder in x
template <bool F16>
__device__ __forceinline__ uint16_t split_term(float& x) {
  if constexpr (F16) {
    const __half h = __float2half_rn(x);
    x -= __half2float(h);
    return __half_as_ushort(h);
  } else {
    const __nv_bfloat16 b = __float2bfloat16_rn(x);
    x -= __bfloat162float(b);
    return __bfloat16_as_ushort(b);
  }
}

template <class P, class L, int NTERM, bool F16>
__global__ void __launch_bounds__(128) me_kernel_mixed(const MeLaunch a) {
  using R = float;
  using S = MixedShape<P, NTERM, F16>;
  constexpr int BLOCK = 128;
  static_assert(L::BLOCK == 128, "one block is the 128-row tile of the MMA");
  static_assert(L::den_view && L::j_view && L::w_mode != 0,
                "mixed kernel takes views of the denominators, J and the colour weights");
  static_assert(F16 ? P::CF_FP16_EXACT : P::CF_BF16_EXACT, "the colour matrix must be exact in the operand type");
  extern __shared__ __align__(16) unsigned char smem_mixed[];  // 16 B suffices for the descriptors
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t nevt = a.nevt;
  const int64_t ntile = (nevt + BLOCK - 1) / BLOCK;
  const int64_t wrow = int64_t(blockIdx.x) * BLOCK + tid;  // this thread's workspace row
  const int64_t wstride = int64_t(gridDim.x) * BLOCK;

  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem_mixed);
  uint64_t* s_mbar = reinterpret_cast<uint64_t*>(smem_mixed + 16);
  unsigned char* s_B = smem_mixed + S::HEAD;
  unsigned char* s_A = s_B + S::BBYTES;
  unsigned char* sp = smem_mixed + S::TC_BYTES;

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
  uint32_t phase = 0;
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
  cx<R>* s_J;
  if constexpr (L::j_smem) { s_J = reinterpret_cast<cx<R>*>(sp); sp += size_t(P::NCOL) * BLOCK * sizeof(cx<R>); }
  else s_J = j_tile<P, R, BLOCK>(a);
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
  Strided<cx<R>, BLOCK> J{s_J + tid};
  R* const w_t = L::w_mode == 1 ? s_w + tid : nullptr;  // this thread's shared colour weights
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
    // (the value of 'failed' is the same in every thread of the block)
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

  // --- helicity loop
  double total = 0.0;
  for (int ih = 0; ih < a.ngood; ++ih) {
    const int h = a.good[ih];
    one_helicity<P, R, L, false>(h, R(a.mt), s_dg + tid, s_dt + tid, s_J + tid, w_t,
                                 a.colw ? a.colw + wrow : nullptr, wstride, ws, kt, want_w);
    // FP16 operands: scale this row by 2^e so that its largest component is near 2^14
    float scale = 1.0f, unscale = 1.0f;
    if constexpr (F16) {
      float amax = 0.0f;
      for (int c = 0; c < S::NC; ++c) {
        const cx<R> z = J[c];
        amax = fmaxf(amax, fmaxf(fabsf(z.r), fabsf(z.i)));
      }
      if (amax > 0.0f && isfinite(amax)) {
        const int e = max(-120, min(120, 14 - ilogbf(amax)));
        scale = ldexpf(1.0f, e);
        unscale = ldexpf(1.0f, -e);
      }
    }
    // the real and imaginary parts in one round, or one after the other through the
    // same A tiles when both do not fit
    constexpr int NROUND = S::TWO_ROUNDS ? 2 : 1;
    constexpr int NPART = S::TWO_ROUNDS ? 1 : 2;
    bool block_failed = false;
    for (int round = 0; round < NROUND; ++round) {
      // split this event's row of A (J times the scale) into NTERM 16-bit terms
#pragma unroll 1
      for (int kc = 0; kc < S::KP / 8; ++kc) {
#pragma unroll
        for (int pp = 0; pp < NPART; ++pp) {
          const int part = S::TWO_ROUNDS ? round : pp;
          float x[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int c = kc * 8 + j;
            x[j] = 0.0f;
            if (c < S::NC) {
              const cx<R> z = J[c];
              x[j] = (part ? z.i : z.r) * scale;
            }
          }
#pragma unroll
          for (int t = 0; t < NTERM; ++t) {
            __align__(16) uint16_t b[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) b[j] = split_term<F16>(x[j]);
            const int slot = S::TWO_ROUNDS ? t : t * 2 + part;
            *reinterpret_cast<uint4*>(s_A + slot * S::TILE + tc::kmajor_offset(tid, kc * 8, S::KP)) =
                *reinterpret_cast<const uint4*>(b);
          }
        }
      }
      tc::fence_proxy_async_smem();
      tc::fence_before_sync();
      __syncthreads();
      if (tid == 0) {
        tc::fence_after_sync();
        for (int pp = 0; pp < NPART; ++pp) {
          const int part = S::TWO_ROUNDS ? round : pp;
          for (int t = 0; t < NTERM; ++t) {
            const int slot = S::TWO_ROUNDS ? t : t * 2 + part;
            for (int ks = 0; ks < S::KP / 16; ++ks) {
              const uint64_t ad = tc::smem_desc(tc::smem_u32(s_A + slot * S::TILE) + ks * 256, 128, S::KP * 16);
              const uint64_t bd = tc::smem_desc(tc::smem_u32(s_B) + ks * 256, 128, S::KP * 16);
              tc::mma_f16kind(tbase + part * S::NP, ad, bd, S::IDESC, (t > 0 || ks > 0) ? 1u : 0u);
            }
          }
        }
        tc::mma_commit(s_mbar);
      }
      // completion also means the MMAs have read the A tiles: the next round may reuse them
      const bool ok = tc::mbar_wait_bounded(s_mbar, phase, a.mma_wait_limit);
      phase ^= 1u;
      block_failed = __syncthreads_or(!ok);  // the same value in every thread of the block
      if (block_failed) break;
    }
    if (block_failed) {
      failed = true;
      break;
    }
    tc::fence_after_sync();
    // colour sum: sum_c Re(J_c) D_re[c] + Im(J_c) D_im[c], sixteen columns at a time
    const uint32_t lane_base = tbase + (uint32_t(32 * warp) << 16);
    float cs = 0.0f;
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
          const cx<R> z = J[c];
          cs += z.r * (dre[j] * unscale) + z.i * (dim[j] * unscale);
        }
      }
    }
    const double mh = double(cs) * gfac;
    total += mh;
    if (a.cum) a.cum[ih * wstride + wrow] = a.cum_mode ? mh : total;
  }

  if (!active) continue;
  a.me[ievt] = failed ? __longlong_as_double(0x7ff8000000000000ll) : total / double(P::IDEN);
  if (!failed) fuse_weight(a, ievt, total / double(P::IDEN), flagged, wmax_t);
  if (a.sel_hel && a.cum && !a.cum_mode) {
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

  // --- teardown: no MMA may still be in flight when the columns are freed, so the
  // wait for the commit that the failed wait gave up on gets the full default limit
  if (failed) {
    if (tid == 0 && a.err) atomicOr(a.err, 1);
    tc::mbar_wait_bounded(s_mbar, phase ^ 1u, kMmaWaitDefault);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tbase, S::TCOLS);
  }
}

template <class P, class L, int NTERM, bool F16>
LaunchNeeds needs_mixed_of() {
  static const int bps =
      resident_blocks(me_kernel_mixed<P, L, NTERM, F16>, 128, me_mixed_smem_bytes<P, L, NTERM, F16>());
  LaunchNeeds n = sizes_of<P, float, L>();
  n.blocks_per_sm = bps;
  return n;
}

template <class P, class L, int NTERM, bool F16>
cudaError_t launch_mixed(const MeLaunch& a, cudaStream_t s) {
  constexpr size_t smem = me_mixed_smem_bytes<P, L, NTERM, F16>();
  static_assert(smem <= 227 * 1024, "shared-memory footprint of the mixed kernel exceeds 227 KB");
  auto k = me_kernel_mixed<P, L, NTERM, F16>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  if (a.grid_blocks <= 0) return cudaErrorInvalidConfiguration;  // the caller sizes the persistent grid
  k<<<dim3(unsigned(a.grid_blocks)), dim3(128), smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace meb300
