// Host evaluation of one generated process header (compiled for the host by nvcc; no
// GPU): reads nevt events [nevt][NPAR][4] FP64 from standard input and prints, per event,
// g_s^(2 NGLUON) sum over all helicities of colour_sum(J_h) / (COL_DEN IDEN) -- the
// matrix element the kernels accumulate -- from the header's own precompute, jamps and
// colour_sum in FP64.  PROC_HEADER and PROC are given on the command line, and VARIANT
// (default 0) picks the jamps variant (its slot buffer is a host array).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include PROC_HEADER

using namespace meb300;
using P = PROC;
#ifndef VARIANT
#define VARIANT 0
#endif

int main(int argc, char** argv) {
  if (argc < 5) return 2;
  const int n = atoi(argv[1]);
  const double wt = atof(argv[2]), as = atof(argv[4]), mt = 173.0;
  const int zwt = atoi(argv[3]);
  std::vector<double> mom(size_t(n) * P::NPAR * 4);
  std::vector<cx<double>> ws(4 * size_t(P::NSLOT[VARIANT] > 0 ? P::NSLOT[VARIANT] : 1));
  if (fread(mom.data(), sizeof(double), mom.size(), stdin) != mom.size()) return 3;
  for (int e = 0; e < n; ++e) {
    const double(*p)[4] = reinterpret_cast<const double(*)[4]>(mom.data() + size_t(e) * P::NPAR * 4);
    double dg[P::NDEN_G];
    cx<double> dt[P::NDEN_T];
    double kt[P::NKVEC * 4];
    P::precompute<4, double>(p, mt, wt, zwt, dg, dt, kt);
    double s = 0;
    for (int h = 0; h < P::NCOMB; ++h) {
      cx<double> J[P::NCOL];
      for (int i = 0; i < P::NCOL; ++i) J[i] = mk<double>(0, 0);
      P::jamps<VARIANT, 4, double>(h, mt, dg, dt, J, ws.data(), kt);
      s += P::colour_sum<double>(J);
    }
    double gp = 1, g2 = 4.0 * M_PI * as;
    for (int k = 0; k < P::NGLUON; ++k) gp *= g2;
    printf("%.17g\n", s * gp / P::COL_DEN / P::IDEN);
  }
  return 0;
}
