// Kernel instantiations and launch table for the process in generated/proc_ggttgg.cuh.
// Layout<jamps variant (register budget), threads per block, denominators and J and
// colour weights (each 0 registers, 1 shared memory, 2 global tile), slot buffer (0 none,
// 1 shared, 2 global), momentum table (1 shared, 2 global), block barriers in the
// helicity body (default none)>.
// The first layout of each precision is the default; the others are alternatives for
// tuning sweeps (me_set_config / ME_B300_CONFIG).
#include "generated/proc_ggttgg.cuh"
#include "me_kernel_mixed.cuh"
#include "me_kernel_mixed_pipe.cuh"
#include "me_kernel_x2.cuh"
#include "me_kernels.cuh"

namespace meb300 {
namespace {
using P = proc_ggttgg;
template <int PREC, int C> struct Cfg;
// FP64 default: jamps variant 9 (variant 3, a register budget of 6 currents, with twelve
// pending colour sums: amplitudes whose colour vectors agree up to a phase summed in
// registers before they are added into J).  Measured at 655360 events: 5.43e5 ME/s
// against 5.20e5 without (Cfg<0, 6>), 5.35e5 and 5.40e5 with four or eight
template <> struct Cfg<0, 0> { using R = double; using L = Layout<9, 64, 1, 1, 1, 2, 2, 3>; };
template <> struct Cfg<0, 1> { using R = double; using L = Layout<3, 64, 1, 1, 1, 2, 2>; };
template <> struct Cfg<0, 2> { using R = double; using L = Layout<4, 64, 1, 1, 1, 2, 2>; };
template <> struct Cfg<0, 3> { using R = double; using L = Layout<5, 64, 1, 1, 1, 2, 2>; };
// jamps variants 6 and 8: variant 3 with four or eight pending colour sums
template <> struct Cfg<0, 4> { using R = double; using L = Layout<6, 64, 1, 1, 1, 2, 2, 3>; };
template <> struct Cfg<0, 5> { using R = double; using L = Layout<8, 64, 1, 1, 1, 2, 2, 3>; };
template <> struct Cfg<0, 6> { using R = double; using L = Layout<3, 64, 1, 1, 1, 2, 2, 3>; };
// FP32 default: jamps variant 10 (variant 1, a register budget of 20 currents, with twelve
// pending colour sums); 1.093e7 ME/s at 655360 events against 1.052e7 without (Cfg<1, 14>)
// and 1.084e7 with four (variant 7, Cfg<1, 13>)
template <> struct Cfg<1, 0> { using R = float; using L = Layout<10, 64, 1, 0, 1, 1, 2, 3>; };
template <> struct Cfg<1, 1> { using R = float; using L = Layout<1, 128, 1, 0, 1, 1, 2, 3>; };
template <> struct Cfg<1, 2> { using R = float; using L = Layout<1, 64, 1, 0, 1, 1, 2>; };
template <> struct Cfg<1, 3> { using R = float; using L = Layout<0, 128, 1, 0, 1, 0, 2>; };
template <> struct Cfg<1, 4> { using R = float; using L = Layout<1, 128, 1, 0, 1, 2, 2>; };
template <> struct Cfg<1, 5> { using R = float; using L = Layout<2, 128, 1, 0, 1, 2, 2>; };
// one 256-thread block per SM (255 registers): every resident warp of an SM in one block,
// held to the same stretch of the helicity body by its barriers (every 8 or 24 steps)
template <> struct Cfg<1, 6> { using R = float; using L = Layout<1, 256, 1, 0, 1, 1, 2, 1>; };
template <> struct Cfg<1, 7> { using R = float; using L = Layout<1, 256, 1, 0, 1, 1, 2, 3>; };
// more resident warps (12 or 16 per SM) at 168 or 128 registers: small register budgets
// (6 or 3 currents), colour weights and the slot buffer in global memory
template <> struct Cfg<1, 8> { using R = float; using L = Layout<3, 64, 1, 1, 2, 2, 2, 3, 8>; };
template <> struct Cfg<1, 9> { using R = float; using L = Layout<4, 64, 1, 0, 2, 2, 2, 3, 8>; };
template <> struct Cfg<1, 10> { using R = float; using L = Layout<3, 64, 1, 1, 2, 2, 2, 3, 6>; };
template <> struct Cfg<1, 11> { using R = float; using L = Layout<2, 64, 1, 0, 2, 2, 2, 3, 6>; };
template <> struct Cfg<1, 13> { using R = float; using L = Layout<7, 64, 1, 0, 1, 1, 2, 3>; };
template <> struct Cfg<1, 14> { using R = float; using L = Layout<1, 64, 1, 0, 1, 1, 2, 3>; };

// FP32 on packed pairs, two events per thread (me_kernel_x2): register budget of 6
// currents, J in shared memory, slot buffer in global memory.  Correct, but slower than
// the scalar kernel here: it halves the FMA-pipe instructions, yet its larger per-thread
// state moves to memory and its instruction-fetch stall per issue doubles.
template <int C> struct X2Cfg;
template <> struct X2Cfg<0> { using L = Layout<3, 64, 1, 1, 1, 2, 2, 3>; };

// mixed precision.  Default: the pipelined kernel with four pending colour sums (jamps
// variant 7: 1.002e7 ME/s at 655360 events, against 9.75e6 without (PipeCfg<2>) and 9.97e6
// with twelve; before the pending sums the pipelined kernel ran at 9.0e6 ME/s at 2^20
// events, against 8.4e6 for the first layout of the unpipelined kernel below).  The unpipelined
// kernel (me_kernel_mixed) follows: amplitude layout (views of J and the weights, 128
// threads), the number of 16-bit terms of the split colour-flow amplitudes (2 = the hi +
// lo split), and the operand type (the colour matrix of this process is exact in BF16)
template <int C> struct MixedCfg;
template <> struct MixedCfg<0> { using L = Layout<1, 128, 1, 1, 1, 2, 2>; static constexpr int NTERM = 2; static constexpr bool F16 = false; };
template <> struct MixedCfg<1> { using L = Layout<1, 128, 1, 1, 1, 2, 2, 3>; static constexpr int NTERM = 3; static constexpr bool F16 = false; };
template <> struct MixedCfg<2> { using L = Layout<1, 128, 1, 1, 1, 2, 2>; static constexpr int NTERM = 3; static constexpr bool F16 = false; };
template <> struct MixedCfg<3> { using L = Layout<2, 128, 1, 1, 1, 2, 2>; static constexpr int NTERM = 3; static constexpr bool F16 = false; };
// pipelined mixed kernel (me_kernel_mixed_pipe): J in registers, the colour sum of one
// helicity on the tensor cores while the next helicity's amplitudes are computed; slot
// buffer in global memory so that two blocks fit an SM; with and without barriers
template <int C> struct PipeCfg;
template <> struct PipeCfg<0> { using L = Layout<7, 128, 1, 0, 1, 2, 2, 3>; static constexpr int NTERM = 2; static constexpr bool F16 = false; };
template <> struct PipeCfg<1> { using L = Layout<1, 128, 1, 0, 1, 2, 2>; static constexpr int NTERM = 2; static constexpr bool F16 = false; };
template <> struct PipeCfg<2> { using L = Layout<1, 128, 1, 0, 1, 2, 2, 3>; static constexpr int NTERM = 2; static constexpr bool F16 = false; };
template <> struct PipeCfg<3> { using L = Layout<10, 128, 1, 0, 1, 2, 2, 3>; static constexpr int NTERM = 2; static constexpr bool F16 = false; };

LaunchNeeds needs(int prec, int config) {
  switch (prec * 16 + config) {
    case 0: return needs_of<P, Cfg<0, 0>::R, Cfg<0, 0>::L>();
    case 1: return needs_of<P, Cfg<0, 1>::R, Cfg<0, 1>::L>();
    case 2: return needs_of<P, Cfg<0, 2>::R, Cfg<0, 2>::L>();
    case 3: return needs_of<P, Cfg<0, 3>::R, Cfg<0, 3>::L>();
    case 4: return needs_of<P, Cfg<0, 4>::R, Cfg<0, 4>::L>();
    case 5: return needs_of<P, Cfg<0, 5>::R, Cfg<0, 5>::L>();
    case 6: return needs_of<P, Cfg<0, 6>::R, Cfg<0, 6>::L>();
    case 16: return needs_of<P, Cfg<1, 0>::R, Cfg<1, 0>::L>();
    case 17: return needs_of<P, Cfg<1, 1>::R, Cfg<1, 1>::L>();
    case 18: return needs_of<P, Cfg<1, 2>::R, Cfg<1, 2>::L>();
    case 19: return needs_of<P, Cfg<1, 3>::R, Cfg<1, 3>::L>();
    case 20: return needs_of<P, Cfg<1, 4>::R, Cfg<1, 4>::L>();
    case 21: return needs_of<P, Cfg<1, 5>::R, Cfg<1, 5>::L>();
    case 22: return needs_of<P, Cfg<1, 6>::R, Cfg<1, 6>::L>();
    case 23: return needs_of<P, Cfg<1, 7>::R, Cfg<1, 7>::L>();
    case 24: return needs_of<P, Cfg<1, 8>::R, Cfg<1, 8>::L>();
    case 25: return needs_of<P, Cfg<1, 9>::R, Cfg<1, 9>::L>();
    case 26: return needs_of<P, Cfg<1, 10>::R, Cfg<1, 10>::L>();
    case 27: return needs_of<P, Cfg<1, 11>::R, Cfg<1, 11>::L>();
    case 28: return needs_x2_of<P, X2Cfg<0>::L>();
    case 29: return needs_of<P, Cfg<1, 13>::R, Cfg<1, 13>::L>();
    case 30: return needs_of<P, Cfg<1, 14>::R, Cfg<1, 14>::L>();
    case 32: return needs_mixed_pipe_of<P, PipeCfg<0>::L, PipeCfg<0>::NTERM, PipeCfg<0>::F16>();
    case 33: return needs_mixed_pipe_of<P, PipeCfg<1>::L, PipeCfg<1>::NTERM, PipeCfg<1>::F16>();
    case 34: return needs_mixed_of<P, MixedCfg<0>::L, MixedCfg<0>::NTERM, MixedCfg<0>::F16>();
    case 35: return needs_mixed_of<P, MixedCfg<1>::L, MixedCfg<1>::NTERM, MixedCfg<1>::F16>();
    case 36: return needs_mixed_of<P, MixedCfg<2>::L, MixedCfg<2>::NTERM, MixedCfg<2>::F16>();
    case 37: return needs_mixed_of<P, MixedCfg<3>::L, MixedCfg<3>::NTERM, MixedCfg<3>::F16>();
    case 38: return needs_mixed_pipe_of<P, PipeCfg<2>::L, PipeCfg<2>::NTERM, PipeCfg<2>::F16>();
    case 39: return needs_mixed_pipe_of<P, PipeCfg<3>::L, PipeCfg<3>::NTERM, PipeCfg<3>::F16>();
    default: return LaunchNeeds{0, 0, 0, 0, false, 128, 1};
  }
}

cudaError_t launch(int prec, int config, const MeLaunch& a, cudaStream_t s) {
  switch (prec * 16 + config) {
    case 0: return launch_me<P, Cfg<0, 0>::R, Cfg<0, 0>::L>(a, s);
    case 1: return launch_me<P, Cfg<0, 1>::R, Cfg<0, 1>::L>(a, s);
    case 2: return launch_me<P, Cfg<0, 2>::R, Cfg<0, 2>::L>(a, s);
    case 3: return launch_me<P, Cfg<0, 3>::R, Cfg<0, 3>::L>(a, s);
    case 4: return launch_me<P, Cfg<0, 4>::R, Cfg<0, 4>::L>(a, s);
    case 5: return launch_me<P, Cfg<0, 5>::R, Cfg<0, 5>::L>(a, s);
    case 6: return launch_me<P, Cfg<0, 6>::R, Cfg<0, 6>::L>(a, s);
    case 16: return launch_me<P, Cfg<1, 0>::R, Cfg<1, 0>::L>(a, s);
    case 17: return launch_me<P, Cfg<1, 1>::R, Cfg<1, 1>::L>(a, s);
    case 18: return launch_me<P, Cfg<1, 2>::R, Cfg<1, 2>::L>(a, s);
    case 19: return launch_me<P, Cfg<1, 3>::R, Cfg<1, 3>::L>(a, s);
    case 20: return launch_me<P, Cfg<1, 4>::R, Cfg<1, 4>::L>(a, s);
    case 21: return launch_me<P, Cfg<1, 5>::R, Cfg<1, 5>::L>(a, s);
    case 22: return launch_me<P, Cfg<1, 6>::R, Cfg<1, 6>::L>(a, s);
    case 23: return launch_me<P, Cfg<1, 7>::R, Cfg<1, 7>::L>(a, s);
    case 24: return launch_me<P, Cfg<1, 8>::R, Cfg<1, 8>::L>(a, s);
    case 25: return launch_me<P, Cfg<1, 9>::R, Cfg<1, 9>::L>(a, s);
    case 26: return launch_me<P, Cfg<1, 10>::R, Cfg<1, 10>::L>(a, s);
    case 27: return launch_me<P, Cfg<1, 11>::R, Cfg<1, 11>::L>(a, s);
    case 28: return launch_x2<P, X2Cfg<0>::L>(a, s);
    case 29: return launch_me<P, Cfg<1, 13>::R, Cfg<1, 13>::L>(a, s);
    case 30: return launch_me<P, Cfg<1, 14>::R, Cfg<1, 14>::L>(a, s);
    case 32: return launch_mixed_pipe<P, PipeCfg<0>::L, PipeCfg<0>::NTERM, PipeCfg<0>::F16>(a, s);
    case 33: return launch_mixed_pipe<P, PipeCfg<1>::L, PipeCfg<1>::NTERM, PipeCfg<1>::F16>(a, s);
    case 34: return launch_mixed<P, MixedCfg<0>::L, MixedCfg<0>::NTERM, MixedCfg<0>::F16>(a, s);
    case 35: return launch_mixed<P, MixedCfg<1>::L, MixedCfg<1>::NTERM, MixedCfg<1>::F16>(a, s);
    case 36: return launch_mixed<P, MixedCfg<2>::L, MixedCfg<2>::NTERM, MixedCfg<2>::F16>(a, s);
    case 37: return launch_mixed<P, MixedCfg<3>::L, MixedCfg<3>::NTERM, MixedCfg<3>::F16>(a, s);
    case 38: return launch_mixed_pipe<P, PipeCfg<2>::L, PipeCfg<2>::NTERM, PipeCfg<2>::F16>(a, s);
    case 39: return launch_mixed_pipe<P, PipeCfg<3>::L, PipeCfg<3>::NTERM, PipeCfg<3>::F16>(a, s);
    default: return cudaErrorNotSupported;
  }
}
}  // namespace

extern const ProcessOps ops_ggttgg = {P::NAME, P::NPAR, P::NCOMB, P::NCOL, P::NDIAG, P::NAMP, P::IDEN,
                                   P::FLOPS_AMP, P::FLOPS_COL, /*has_mixed=*/true, {7, 15, 8, 0},
                                   needs, launch};
}  // namespace meb300
