// Kernel instantiations and launch table for the process in generated/proc_udxttudx.cuh
// (u d~ > t t~ u d~, a four-quark channel of p p -> t t~ + 2 jets with two light
// flavours): one event per thread, in FP64 and FP32.
#include "generated/proc_udxttudx.cuh"
#include "me_kernels.cuh"

namespace meb300 {
namespace {
using P = proc_udxttudx;
template <int PREC, int C> struct Cfg;
// The first layout of each precision is the default, the others alternatives for sweeps
// (me_set_config).  Measured on u d > t t~ u d at 262144 events: FP64 with the
// denominators, J and colour weights in shared memory 1.89e7 ME/s, everything in
// registers 1.86e7; FP32 capped at 168 registers 4.0e8, at 128 3.4e8, uncapped 3.7e8
template <> struct Cfg<0, 0> { using R = double; using L = Layout<0, 128, 1, 1, 1, 0, 1>; };
template <> struct Cfg<0, 1> { using R = double; using L = Layout<0, 128, 0, 0, 0, 0, 1>; };
template <> struct Cfg<1, 0> { using R = float; using L = Layout<0, 128, 0, 0, 0, 0, 1, 0, 3>; };
template <> struct Cfg<1, 1> { using R = float; using L = Layout<0, 128, 0, 0, 0, 0, 1, 0, 4>; };
template <> struct Cfg<1, 2> { using R = float; using L = Layout<0, 128, 0, 0, 0, 0, 1>; };

LaunchNeeds needs(int prec, int config) {
  switch (prec * 8 + config) {
    case 0: return needs_of<P, Cfg<0, 0>::R, Cfg<0, 0>::L>();
    case 1: return needs_of<P, Cfg<0, 1>::R, Cfg<0, 1>::L>();
    case 8: return needs_of<P, Cfg<1, 0>::R, Cfg<1, 0>::L>();
    case 9: return needs_of<P, Cfg<1, 1>::R, Cfg<1, 1>::L>();
    case 10: return needs_of<P, Cfg<1, 2>::R, Cfg<1, 2>::L>();
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
    default: return cudaErrorNotSupported;
  }
}
}  // namespace

extern const ProcessOps ops_udxttudx = {P::NAME, P::NPAR, P::NCOMB, P::NCOL, P::NDIAG, P::NAMP, P::IDEN,
                                   P::FLOPS_AMP, P::FLOPS_COL, /*has_mixed=*/false, {2, 3, 0, 0},
                                   needs, launch};
}  // namespace meb300
