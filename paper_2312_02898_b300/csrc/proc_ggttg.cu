// Kernel instantiations and launch table for the process in generated/proc_ggttg.cuh.
// Layout<jamps variant (register budget), threads per block, denominators and J and
// colour weights (each 0 registers, 1 shared memory, 2 global tile), slot buffer (0 none,
// 1 shared, 2 global), momentum table (1 shared, 2 global), block barriers in the
// helicity body (default none)>.
// The first layout of each precision is the default; the others are alternatives for
// tuning sweeps (me_set_config / ME_B300_CONFIG).
#include "generated/proc_ggttg.cuh"
#include "dfloat.cuh"
#include "me_kernel_x2.cuh"
#include "me_kernels.cuh"

namespace meb300 {
namespace {
using P = proc_ggttg;
template <int PREC, int C> struct Cfg;
template <> struct Cfg<0, 0> { using R = double; using L = Layout<1, 128, false, false, 0, 1, 1, 3>; };
template <> struct Cfg<0, 1> { using R = double; using L = Layout<1, 128, false, false, 0, 1, 1>; };
// FP32: registers capped at 168 by asking for 3 blocks per SM (12 warps), without
// spills; then the uncapped layout (254 registers, 8 warps), the same without block
// barriers, and a cap at 128
template <> struct Cfg<1, 0> { using R = float; using L = Layout<0, 128, 0, 0, 0, 0, 1, 3, 3>; };
template <> struct Cfg<1, 1> { using R = float; using L = Layout<0, 128, false, false, 0, 0, 1, 3>; };
template <> struct Cfg<1, 2> { using R = float; using L = Layout<0, 128, false, false, 0, 0, 1>; };
template <> struct Cfg<1, 3> { using R = float; using L = Layout<0, 128, 0, 0, 0, 0, 1, 3, 4>; };

// FP32 on packed pairs, two events per thread (me_kernel_x2), everything in registers:
// correct, a little slower than the scalar kernel here (measured)
// FP64-emulating double-float amplitudes: the FP64 default layout (same 8-byte storage)
template <> struct Cfg<3, 0> { using R = dfloat; using L = Layout<1, 128, false, false, 0, 1, 1, 3>; };

template <int C> struct X2Cfg;
template <> struct X2Cfg<0> { using L = Layout<0, 128, 0, 0, 0, 0, 1, 3>; };

LaunchNeeds needs(int prec, int config) {
  switch (prec * 8 + config) {
    case 0: return needs_of<P, Cfg<0, 0>::R, Cfg<0, 0>::L>();
    case 1: return needs_of<P, Cfg<0, 1>::R, Cfg<0, 1>::L>();
    case 8: return needs_of<P, Cfg<1, 0>::R, Cfg<1, 0>::L>();
    case 9: return needs_of<P, Cfg<1, 1>::R, Cfg<1, 1>::L>();
    case 10: return needs_of<P, Cfg<1, 2>::R, Cfg<1, 2>::L>();
    case 11: return needs_of<P, Cfg<1, 3>::R, Cfg<1, 3>::L>();
    case 12: return needs_x2_of<P, X2Cfg<0>::L>();
    case 24: return needs_of<P, Cfg<3, 0>::R, Cfg<3, 0>::L>();
    default: return LaunchNeeds{0, 0, 0, 0, false, 128, 1};
  }
}

cudaError_t launch(int prec, int config, const MeLaunch& a, cudaStream_t s) {
  switch (prec * 8 + config) {
    case 0: return launch_me<P, Cfg<0, 0>::R, Cfg<0, 0>::L>(a, s);
    case 1: return launch_me<P, Cfg<0, 1>::R, Cfg<0, 1>::L>(a, s);
    case 8: return launch_me<P, Cfg<1, 0>::R, Cfg<1, 0>::L>(a, s);
    case 9: return launch_me<P, Cfg<1, 1>::R, Cfg<1, 1>::L>(a, s);
    case 10: return launch_me<P, Cfg<1, 2>::R, Cfg<1, 2>::L>(a, s);
    case 11: return launch_me<P, Cfg<1, 3>::R, Cfg<1, 3>::L>(a, s);
    case 12: return launch_x2<P, X2Cfg<0>::L>(a, s);
    case 24: return launch_me<P, Cfg<3, 0>::R, Cfg<3, 0>::L>(a, s);
    default: return cudaErrorNotSupported;
  }
}
}  // namespace

extern const ProcessOps ops_ggttg = {P::NAME, P::NPAR, P::NCOMB, P::NCOL, P::NDIAG, P::NAMP, P::IDEN,
                                   P::FLOPS_AMP, P::FLOPS_COL, /*has_mixed=*/false, {2, 5, 0, 1},
                                   needs, launch};
}  // namespace meb300
