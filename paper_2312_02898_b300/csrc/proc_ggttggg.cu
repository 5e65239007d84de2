// Kernel instantiations and launch table for the process in generated/proc_ggttggg.cuh.
// Layout<jamps variant (register budget), threads per block, denominators and J and
// colour weights (each 0 registers, 1 shared memory, 2 global tile), slot buffer (0 none,
// 1 shared, 2 global), momentum table (1 shared, 2 global), block barriers in the
// helicity body (default none)>.
// The first layout of each precision is the default; the others are alternatives for
// tuning sweeps (me_set_config / ME_B300_CONFIG).
#include "generated/proc_ggttggg.cuh"
#include "me_kernel_mixed.cuh"
#include "me_kernels.cuh"

namespace meb300 {
namespace {
using P = proc_ggttggg;
template <int PREC, int C> struct Cfg;
// Every per-thread array in global tiles leaves shared memory free, so registers alone
// bound the blocks per SM: four 64-thread blocks in FP64, two 128-thread blocks in FP32.
// Each layout sums the amplitudes whose colour vectors agree up to a phase in registers
// (jamps variant 3: eight pending colour sums, variant 4: sixteen) before they are added
// into J, which removes 43% (eight) or 49% (sixteen) of the adds into J in global memory.
// Measured at 131072 events with diagram groups of 160 steps: FP64 2.23e4 ME/s with
// sixteen, 2.19e4 with eight, 1.97e4 with none (variant 0); FP32 1.49e5, 1.46e5 and
// 1.26e5; mixed 1.44e5, 1.40e5 and 1.13e5.  Larger groups merge more closings and pass
// fewer values through the slot buffer: groups of 320 steps with sixteen pending sums
// (jamps variant 5, the alternative layout of each precision) FP64 2.28e4, FP32 1.54e5,
// mixed 1.52e5; groups of 480 with twenty-four (variant 6, the default of each precision)
// FP64 2.33e4, FP32 1.58e5, mixed 1.59e5.  Larger groups lengthen this unit's build.
// Measured alternatives (not compiled, to keep the build of this large translation unit
// short): shared-memory denominators and J (176 KB, one block per SM) were 1.6-1.7x
// slower; block barriers between diagram groups add 13% in FP64 and nothing in FP32; a
// register budget of 20 currents instead of 12 changed nothing; FP32 with J in shared
// memory and small blocks (64- or 32-thread blocks, six or seven warps per SM) ran at
// 1.15e5 and 1.38e5 ME/s against 1.40e5 with J in global tiles.
template <> struct Cfg<0, 0> { using R = double; using L = Layout<6, 64, 2, 2, 2, 2, 2, 3>; };
template <> struct Cfg<0, 1> { using R = double; using L = Layout<5, 64, 2, 2, 2, 2, 2, 3>; };
template <> struct Cfg<1, 0> { using R = float; using L = Layout<6, 128, 2, 2, 2, 2, 2>; };
template <> struct Cfg<1, 1> { using R = float; using L = Layout<5, 128, 2, 2, 2, 2, 2>; };

// mixed precision: every per-thread array in global tiles, so that the FP16 operand
// tiles (120 flows padded to 128) and the colour matrix fit in shared memory beside two
// blocks per SM; two FP16 terms (the colour matrix is exact in FP16, not in BF16)
template <int C> struct MixedCfg;
template <> struct MixedCfg<0> { using L = Layout<6, 128, 2, 2, 2, 2, 2>; static constexpr int NTERM = 2; static constexpr bool F16 = true; };
template <> struct MixedCfg<1> { using L = Layout<5, 128, 2, 2, 2, 2, 2>; static constexpr int NTERM = 2; static constexpr bool F16 = true; };

LaunchNeeds needs(int prec, int config) {
  switch (prec * 8 + config) {
    case 0: return needs_of<P, Cfg<0, 0>::R, Cfg<0, 0>::L>();
    case 1: return needs_of<P, Cfg<0, 1>::R, Cfg<0, 1>::L>();
    case 8: return needs_of<P, Cfg<1, 0>::R, Cfg<1, 0>::L>();
    case 9: return needs_of<P, Cfg<1, 1>::R, Cfg<1, 1>::L>();
    case 16: return needs_mixed_of<P, MixedCfg<0>::L, MixedCfg<0>::NTERM, MixedCfg<0>::F16>();
    case 17: return needs_mixed_of<P, MixedCfg<1>::L, MixedCfg<1>::NTERM, MixedCfg<1>::F16>();
    default: return LaunchNeeds{0, 0, 0, 0, false, 128, 1};
  }
}

cudaError_t launch(int prec, int config, const MeLaunch& a, cudaStream_t s) {
  switch (prec * 8 + config) {
    case 0: return launch_me<P, Cfg<0, 0>::R, Cfg<0, 0>::L>(a, s);
    case 1: return launch_me<P, Cfg<0, 1>::R, Cfg<0, 1>::L>(a, s);
    case 8: return launch_me<P, Cfg<1, 0>::R, Cfg<1, 0>::L>(a, s);
    case 9: return launch_me<P, Cfg<1, 1>::R, Cfg<1, 1>::L>(a, s);
    case 16: return launch_mixed<P, MixedCfg<0>::L, MixedCfg<0>::NTERM, MixedCfg<0>::F16>(a, s);
    case 17: return launch_mixed<P, MixedCfg<1>::L, MixedCfg<1>::NTERM, MixedCfg<1>::F16>(a, s);
    default: return cudaErrorNotSupported;
  }
}
}  // namespace

extern const ProcessOps ops_ggttggg = {P::NAME, P::NPAR, P::NCOMB, P::NCOL, P::NDIAG, P::NAMP, P::IDEN,
                                   P::FLOPS_AMP, P::FLOPS_COL, /*has_mixed=*/true, {2, 2, 2, 0},
                                   needs, launch};
}  // namespace meb300
