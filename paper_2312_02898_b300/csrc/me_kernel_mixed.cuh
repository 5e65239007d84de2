// me_kernel_mixed.cuh -- the mixed-precision matrix-element kernel: FP32 amplitudes
// (generated code, one event per thread, as in me_kernel), colour sum on the tensor
// cores (colour_mma.cuh), FP64 inputs, denominators and helicity sum.
//
// One block tile = 128 events = the M = 128 rows of one tcgen05 MMA.  The grid is
// persistent: each block sets up its tensor-core state once and walks the batch tile by
// tile.  Every thread of the block takes part in every barrier (threads past the end
// of the batch mirror the last event and write nothing).
#pragma once

#include "colour_mma.cuh"
#include "me_kernels.cuh"

namespace meb300 {

constexpr uint32_t kMmaWaitLimit = 1u << 22;  // bounded spin on the MMA-completion barrier

template <class P, int NTERM>
struct MixedShape {
  static constexpr int NC = P::NCOL;
  static constexpr int KP = (NC + 15) / 16 * 16;  // flows padded to the MMA K step
  static constexpr int NP = KP;                   // C is square
  static constexpr uint32_t TILE = 128u * KP * 2;  // one BF16 A tile
  static constexpr uint32_t BBYTES = (uint32_t(NP) * KP * 2 + 1023u) / 1024u * 1024u;
  static constexpr uint32_t TCOLS = (2 * NP <= 32) ? 32 : (2 * NP <= 64) ? 64 : (2 * NP <= 128) ? 128 : (2 * NP <= 256) ? 256 : 512;
  static constexpr uint32_t IDESC = tc::idesc_bf16(128, NP);
  static constexpr size_t HEAD = 1024;  // TMEM address, mbarrier
  static constexpr size_t TC_BYTES = HEAD + BBYTES + size_t(2) * NTERM * TILE;
};

template <class P, class L, int NTERM>
constexpr size_t me_mixed_smem_bytes() {
  return MixedShape<P, NTERM>::TC_BYTES + me_smem_bytes<P, float, L>();
}

template <class P, class L, int NTERM>
__global__ void __launch_bounds__(128) me_kernel_mixed(const MeLaunch a) {
  using R = float;
  using S = MixedShape<P, NTERM>;
  constexpr int BLOCK = 128;
  static_assert(L::BLOCK == 128, "one block is the 128-row tile of the MMA");
  static_assert(L::den_smem && L::j_smem && L::w_mode == 1, "mixed kernel expects J and weights in shared memory");
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
    const float v = (n < S::NC && k < S::NC) ? float(P::cf_device(n * S::NC + k)) : 0.0f;
    *reinterpret_cast<__nv_bfloat16*>(s_B + tc::kmajor_offset(n, k, S::KP)) = __float2bfloat16_rn(v);
  }
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *s_tmem;
  uint32_t phase = 0;
  bool failed = false;

  // --- per-thread working storage, carved once for all tiles
  R* s_dg = reinterpret_cast<R*>(sp); sp += size_t(P::NDEN_G) * BLOCK * sizeof(R);
  cx<R>* s_dt = reinterpret_cast<cx<R>*>(sp); sp += size_t(P::NDEN_T) * BLOCK * sizeof(cx<R>);
  cx<R>* s_J = reinterpret_cast<cx<R>*>(sp); sp += size_t(P::NCOL) * BLOCK * sizeof(cx<R>);
  R* s_w = reinterpret_cast<R*>(sp); sp += size_t(P::NCOL) * BLOCK * sizeof(R);
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

  for (int64_t tile = blockIdx.x; tile < ntile && !failed; tile += gridDim.x) {
  const int64_t ievt_raw = tile * BLOCK + tid;
  const bool active = ievt_raw < nevt;
  const int64_t ievt = active ? ievt_raw : nevt - 1;

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
  if (active && a.rescue_list && kappa > a.rescue_kappa) {
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
  Strided<R, BLOCK> v_w{s_w + tid};
  Strided<cx<R>, BLOCK> J{s_J + tid};
  if (want_w)
    for (int c = 0; c < P::NCOL; ++c) v_w[c] = R(0);

  // --- helicity loop
  double total = 0.0;
  for (int ih = 0; ih < a.ngood; ++ih) {
    const int h = a.good[ih];
    one_helicity<P, R, L, false>(h, R(a.mt), s_dg + tid, s_dt + tid, s_J + tid, s_w + tid, nullptr, 0, ws, kt, want_w);
    // split this event's row of A into NTERM BF16 terms (real and imaginary parts)
#pragma unroll
    for (int kc = 0; kc < S::KP / 8; ++kc) {
#pragma unroll
      for (int part = 0; part < 2; ++part) {
        float x[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int c = kc * 8 + j;
          x[j] = 0.0f;
          if (c < S::NC) {
            const cx<R> z = J[c];
            x[j] = part ? z.i : z.r;
          }
        }
#pragma unroll
        for (int t = 0; t < NTERM; ++t) {
          __align__(16) __nv_bfloat16 b[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            b[j] = __float2bfloat16_rn(x[j]);
            x[j] -= __bfloat162float(b[j]);
          }
          *reinterpret_cast<uint4*>(s_A + (t * 2 + part) * S::TILE + tc::kmajor_offset(tid, kc * 8, S::KP)) =
              *reinterpret_cast<const uint4*>(b);
        }
      }
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int part = 0; part < 2; ++part)
#pragma unroll
        for (int t = 0; t < NTERM; ++t)
#pragma unroll
          for (int ks = 0; ks < S::KP / 16; ++ks) {
            const uint64_t ad = tc::smem_desc(tc::smem_u32(s_A + (t * 2 + part) * S::TILE) + ks * 256, 128, S::KP * 16);
            const uint64_t bd = tc::smem_desc(tc::smem_u32(s_B) + ks * 256, 128, S::KP * 16);
            tc::mma_bf16(tbase + part * S::NP, ad, bd, S::IDESC, (t > 0 || ks > 0) ? 1u : 0u);
          }
      tc::mma_commit(s_mbar);
    }
    const bool ok = tc::mbar_wait_bounded(s_mbar, phase, kMmaWaitLimit);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    tc::fence_after_sync();
    float dre[S::NP], dim[S::NP];
    const uint32_t lane_base = tbase + (uint32_t(32 * warp) << 16);
#pragma unroll
    for (int c0 = 0; c0 < S::NP; c0 += 16) {
      tc::tmem_ld16(lane_base + c0, dre + c0);
      tc::tmem_ld16(lane_base + S::NP + c0, dim + c0);
    }
    tc::tmem_wait_ld();
    float cs = 0.0f;
#pragma unroll
    for (int c = 0; c < S::NC; ++c) {
      const cx<R> z = J[c];
      cs += z.r * dre[c] + z.i * dim[c];
    }
    const double mh = double(cs) * gfac;
    total += mh;
    if (a.cum) a.cum[ih * wstride + wrow] = a.cum_mode ? mh : total;
  }

  if (!active) continue;
  a.me[ievt] = failed ? __longlong_as_double(0x7ff8000000000000ll) : total / double(P::IDEN);
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
      for (int c = 0; c < P::NCOL; ++c) wt_tot += double(v_w[c]);
      if (wt_tot > 0.0) {
        const double target = a.rnd_col[ievt] * wt_tot;
        double run = 0.0;
        int found = -1, lastnz = -1;
        for (int c = 0; c < P::NCOL; ++c) {
          const double w = double(v_w[c]);
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

  // --- teardown: no MMA may still be in flight when the columns are freed
  if (failed) {
    if (tid == 0 && a.err) atomicOr(a.err, 1);
    tc::mbar_wait_bounded(s_mbar, phase ^ 1u, kMmaWaitLimit);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tbase, S::TCOLS);
  }
}

template <class P, class L, int NTERM>
LaunchNeeds needs_mixed_of() {
  static const int bps = resident_blocks(me_kernel_mixed<P, L, NTERM>, 128, me_mixed_smem_bytes<P, L, NTERM>());
  LaunchNeeds n = sizes_of<P, float, L>();
  n.blocks_per_sm = bps;
  return n;
}

template <class P, class L, int NTERM>
cudaError_t launch_mixed(const MeLaunch& a, cudaStream_t s) {
  constexpr size_t smem = me_mixed_smem_bytes<P, L, NTERM>();
  static_assert(smem <= 227 * 1024, "shared-memory footprint of the mixed kernel exceeds 227 KB");
  auto k = me_kernel_mixed<P, L, NTERM>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  if (a.grid_blocks <= 0) return cudaErrorInvalidConfiguration;  // the caller sizes the persistent grid
  k<<<dim3(unsigned(a.grid_blocks)), dim3(128), smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace meb300
