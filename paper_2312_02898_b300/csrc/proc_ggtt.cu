// Kernel instantiations and launch table for the process in generated/proc_ggtt.cuh.
// Layout<jamps variant (register budget), threads per block, denominators and J and
// colour weights (each 0 registers, 1 shared memory, 2 global tile), slot buffer (0 none,
// 1 shared, 2 global), momentum table (1 shared, 2 global), block barriers in the
// helicity body (default none)>.
// The first layout of each precision is the default; the others are alternatives for
// tuning sweeps (me_set_config / ME_B300_CONFIG).
#include "generated/proc_ggtt.cuh"
#include "dfloat.cuh"
#include "me_kernel_x2.cuh"
#include "me_kernels.cuh"

namespace meb300 {
namespace {
using P = proc_ggtt;
template <int PREC, int C> struct Cfg;
template <> struct Cfg<0, 0> { using R = double; using L = Layout<0, 128, 0, 0, 0, 0, 1>; };
// FP32: registers capped at 96 by asking for 5 blocks per SM (20 warps), without
// spills; the uncapped layout (151 registers, 12 warps) and a cap at 128 follow
template <> struct Cfg<1, 0> { using R = float; using L = Layout<0, 128, 0, 0, 0, 0, 1, 0, 5>; };
template <> struct Cfg<1, 1> { using R = float; using L = Layout<0, 128, 0, 0, 0, 0, 1>; };
template <> struct Cfg<1, 2> { using R = float; using L = Layout<0, 128, 0, 0, 0, 0, 1, 0, 4>; };

// FP32 on packed pairs, two events per thread (me_kernel_x2), everything in registers:
// correct, a little slower than the scalar kernel here (measured)
// FP64-emulating double-float amplitudes: the FP64 default layout (same 8-byte storage)
template <> struct Cfg<3, 0> { using R = dfloat; using L = Layout<0, 128, 0, 0, 0, 0, 1>; };

template <int C> struct X2Cfg;
template <> struct X2Cfg<0> { using L = Layout<0, 128, 0, 0, 0, 0, 1, 0, 3>; };

LaunchNeeds needs(int prec, int config) {
  switch (prec * 8 + config) {
    case 0: return needs_of<P, Cfg<0, 0>::R, Cfg<0, 0>::L>();
    case 8: return needs_of<P, Cfg<1, 0>::R, Cfg<1, 0>::L>();
    case 9: return needs_of<P, Cfg<1, 1>::R, Cfg<1, 1>::L>();
    case 10: return needs_of<P, Cfg<1, 2>::R, Cfg<1, 2>::L>();
    case 11: return needs_x2_of<P, X2Cfg<0>::L>();
    case 24: return needs_of<P, Cfg<3, 0>::R, Cfg<3, 0>::L>();
    default: return LaunchNeeds{0, 0, 0, 0, false, 128, 1};
  }
}

cudaError_t launch(int prec, int config, const MeLaunch& a, cudaStream_t s) {
  switch (prec * 8 + config) {
    case 0: return launch_me<P, Cfg<0, 0>::R, Cfg<0, 0>::L>(a, s);
    case 8: return launch_me<P, Cfg<1, 0>::R, Cfg<1, 0>::L>(a, s);
    case 9: return launch_me<P, Cfg<1, 1>::R, Cfg<1, 1>::L>(a, s);
    case 10: return launch_me<P, Cfg<1, 2>::R, Cfg<1, 2>::L>(a, s);
    case 11: return launch_x2<P, X2Cfg<0>::L>(a, s);
    case 24: return launch_me<P, Cfg<3, 0>::R, Cfg<3, 0>::L>(a, s);
    default: return cudaErrorNotSupported;
  }
}
}  // namespace

extern const ProcessOps ops_ggtt = {P::NAME, P::NPAR, P::NCOMB, P::NCOL, P::NDIAG, P::NAMP, P::IDEN,
                                   P::FLOPS_AMP, P::FLOPS_COL, /*has_mixed=*/false, {1, 4, 0, 1},
                                   needs, launch};
}  // namespace meb300
