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
// Measured alternatives (not compiled, to keep the build of this large translation unit
// short): shared-memory denominators and J (176 KB, one block per SM) were 1.6-1.7x
// slower; block barriers between diagram groups add 13% in FP64 and nothing in FP32; a
// register budget of 20 currents instead of 12 changed nothing.
template <> struct Cfg<0, 0> { using R = double; using L = Layout<0, 64, 2, 2, 2, 2, 2, 3>; };
// FP32 with J in shared memory and small blocks (960 bytes per thread: 64-thread blocks,
// six warps per SM, or 32-thread blocks, seven warps per SM) ran at 1.15e5 and 1.38e5
// ME/s against 1.40e5 with J in global tiles: the J accumulations are not the limit.
template <> struct Cfg<1, 0> { using R = float; using L = Layout<0, 128, 2, 2, 2, 2, 2>; };

// mixed precision: every per-thread array in global tiles, so that the FP16 operand
// tiles (120 flows padded to 128) and the colour matrix fit in shared memory beside two
// blocks per SM; two FP16 terms (the colour matrix is exact in FP16, not in BF16)
template <int C> struct MixedCfg;
template <> struct MixedCfg<0> { using L = Layout<0, 128, 2, 2, 2, 2, 2>; static constexpr int NTERM = 2; static constexpr bool F16 = true; };

LaunchNeeds needs(int prec, int config) {
  switch (prec * 8 + config) {
    case 0: return needs_of<P, Cfg<0, 0>::R, Cfg<0, 0>::L>();
    case 8: return needs_of<P, Cfg<1, 0>::R, Cfg<1, 0>::L>();
    case 16: return needs_mixed_of<P, MixedCfg<0>::L, MixedCfg<0>::NTERM, MixedCfg<0>::F16>();
    default: return LaunchNeeds{0, 0, 0, 0, false, 128, 1};
  }
}

cudaError_t launch(int prec, int config, const MeLaunch& a, cudaStream_t s) {
  switch (prec * 8 + config) {
    case 0: return launch_me<P, Cfg<0, 0>::R, Cfg<0, 0>::L>(a, s);
    case 8: return launch_me<P, Cfg<1, 0>::R, Cfg<1, 0>::L>(a, s);
    case 16: return launch_mixed<P, MixedCfg<0>::L, MixedCfg<0>::NTERM, MixedCfg<0>::F16>(a, s);
    default: return cudaErrorNotSupported;
  }
}
}  // namespace

extern const ProcessOps ops_ggttggg = {P::NAME, P::NPAR, P::NCOMB, P::NCOL, P::NDIAG, P::NAMP, P::IDEN,
                                   P::FLOPS_AMP, P::FLOPS_COL, /*has_mixed=*/true, {1, 1, 1, 0},
                                   needs, launch};
}  // namespace meb300
