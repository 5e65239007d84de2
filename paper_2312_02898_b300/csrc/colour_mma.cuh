// colour_mma.cuh -- colour sum J^dagger C J on the tensor cores (tcgen05, sm_100+ family).
//
// For one helicity, a block of 128 events forms the 128 x K matrices A_re, A_im of
// colour-flow amplitudes (one event per row, K = number of flows padded to a multiple
// of 16).  The colour matrix C (integer numerators, symmetric, exact in the 16-bit
// operand type) is resident in shared memory as the N x K operand B.
//   D_re = A_re C,  D_im = A_im C          (tcgen05.mma, FP32 accumulation in TMEM)
//   |M_h|^2 * COL_DEN = sum_j (Re J_j D_re[j] + Im J_j D_im[j])   (per thread, FP32 J)
// A is split into NTERM 16-bit terms, A = a_1 + a_2 (+ a_3), each the rounding of what
// the previous terms leave, so the product carries ~8*NTERM (BF16) or ~11*NTERM (FP16)
// significant bits of J; every term accumulates into the same TMEM columns.
//
// Operands use the no-swizzle K-major shared-memory layout: 8-row x 16-byte core
// matrices, adjacent along K every 128 bytes (leading byte offset) and along M/N every
// K*16/8 bytes (stride byte offset).  One elected thread issues the MMAs and commits
// them to an mbarrier that every thread waits on with a bounded spin; a wait that runs
// out sets an error flag, the event results become NaN, and the block still frees its
// TMEM before it exits.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace meb300 {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 64-bit shared-memory matrix descriptor (no swizzle, K-major)
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= uint64_t((saddr & 0x3FFFFu) >> 4);
  d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
  d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
  d |= uint64_t(1) << 46;  // descriptor version field (fixed 0b001)
  return d;                // base offset 0, relative LBO, no swizzle
}

// instruction descriptor of kind::f16 with an FP32 accumulator, both operands K-major:
// A and B both FP16 (f16 = true) or both BF16
__host__ __device__ constexpr uint32_t idesc_f16kind(int M, int N, bool f16) {
  return (1u << 4)                                   // D format FP32
         | (f16 ? 0u : ((1u << 7) | (1u << 10)))     // A, B format: 0 FP16, 1 BF16
         | (uint32_t(N >> 3) << 17)                  // N / 8
         | (uint32_t(M >> 4) << 24);                 // M / 16
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// D (TMEM) = A B (+ D when accumulate), operand types as the instruction descriptor says
__device__ __forceinline__ void mma_f16kind(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
               : "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(mbar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: false when the limit ran out
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* mbar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_try_wait(mbar, parity)) return true;
  return false;
}

// 32 lanes x 32 bits, 16 consecutive columns per thread
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// byte offset of element (row, k) in a no-swizzle K-major tile with KP columns
__host__ __device__ constexpr uint32_t kmajor_offset(int row, int k, int KP) {
  return uint32_t(((row >> 3) * (KP >> 3) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

}  // namespace tc
}  // namespace meb300
