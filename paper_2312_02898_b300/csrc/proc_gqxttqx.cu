// Kernel instantiations and launch table for the process in generated/proc_gqxttqx.cuh
// (g u~ > t t~ u~, a one-jet quark channel of p p -> t t~ + jet): everything in registers, one
// event per thread, in FP64, FP32 and double-float.
#include "generated/proc_gqxttqx.cuh"
#include "dfloat.cuh"
#include "me_kernels.cuh"

namespace meb300 {
namespace {
using P = proc_gqxttqx;
template <int PREC, int C> struct Cfg;
// FP64: the layouts tried (64 or 128 threads; denominators, J and colour weights in
// registers or shared memory) all ran within 1% (2.7e7 ME/s); FP32: registers capped at
// 128 (four 128-thread blocks per SM) ran 25% faster than the uncapped 211 registers
template <> struct Cfg<0, 0> { using R = double; using L = Layout<0, 128, 0, 0, 0, 0, 1>; };
template <> struct Cfg<0, 1> { using R = double; using L = Layout<0, 128, 1, 1, 1, 0, 1>; };
template <> struct Cfg<1, 0> { using R = float; using L = Layout<0, 128, 0, 0, 0, 0, 1, 0, 4>; };
template <> struct Cfg<1, 1> { using R = float; using L = Layout<0, 128, 0, 0, 0, 0, 1, 0, 3>; };
template <> struct Cfg<1, 2> { using R = float; using L = Layout<0, 128, 0, 0, 0, 0, 1>; };
// FP64-emulating double-float amplitudes: the FP64 default layout
template <> struct Cfg<3, 0> { using R = dfloat; using L = Layout<0, 128, 0, 0, 0, 0, 1>; };

LaunchNeeds needs(int prec, int config) {
  switch (prec * 8 + config) {
    case 0: return needs_of<P, Cfg<0, 0>::R, Cfg<0, 0>::L>();
    case 1: return needs_of<P, Cfg<0, 1>::R, Cfg<0, 1>::L>();
    case 8: return needs_of<P, Cfg<1, 0>::R, Cfg<1, 0>::L>();
    case 9: return needs_of<P, Cfg<1, 1>::R, Cfg<1, 1>::L>();
    case 10: return needs_of<P, Cfg<1, 2>::R, Cfg<1, 2>::L>();
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
    case 24: return launch_me<P, Cfg<3, 0>::R, Cfg<3, 0>::L>(a, s);
    default: return cudaErrorNotSupported;
  }
}
}  // namespace

extern const ProcessOps ops_gqxttqx = {P::NAME, P::NPAR, P::NCOMB, P::NCOL, P::NDIAG, P::NAMP, P::IDEN,
                                   P::FLOPS_AMP, P::FLOPS_COL, /*has_mixed=*/false, {2, 3, 0, 1},
                                   needs, launch};
}  // namespace meb300
