// Host-only check of the double-float arithmetic (csrc/dfloat.cuh) against exact
// quadruple-precision results (__float128), on random operands over a wide range of
// magnitudes and signs, including near-cancelling sums:
//   * TwoSum and TwoProd are exact (hi + lo equals the exact sum or product);
//   * addition and subtraction within 3u^2 and multiplication within 5u^2 relative
//     (u = 2^-24), the bounds of Joldes, Muller and Popescu (2017);
//   * division and square root (one Newton correction) within 32u^2.
// Prints the largest relative error of each operation; exit status 1 on any violation.
#include <cmath>
#include <cstdio>
#include <random>

#include "dfloat.cuh"

using namespace meb300;
typedef __float128 quad;

static quad q(dfloat x) { return quad(x.hi) + quad(x.lo); }
static double rel(quad got, quad want) {
  if (want == 0) return got == 0 ? 0.0 : 1.0;
  quad d = (got - want) / want;
  return double(d < 0 ? -d : d);
}

int main() {
  std::mt19937_64 rng(11);
  std::uniform_real_distribution<double> mant(-1.0, 1.0);
  std::uniform_int_distribution<int> ex(-30, 30);
  auto draw = [&]() { return std::ldexp(mant(rng), ex(rng)); };
  const double u2 = std::ldexp(1.0, -48);
  double worst[5] = {0, 0, 0, 0, 0};
  const char* names[5] = {"add", "sub", "mul", "div", "sqrt"};
  const double bound[5] = {3 * u2, 3 * u2, 5 * u2, 32 * u2, 32 * u2};
  int bad_exact = 0;
  for (int t = 0; t < 200000; ++t) {
    const dfloat x(draw()), y(t % 4 == 0 ? -double(dfloat(draw())) : draw());
    dfloat yc = y;
    if (t % 8 == 1) yc = -x + dfloat(std::ldexp(draw(), -20));  // near cancellation
    const float a = x.hi, b = yc.hi;
    const dfloat s = two_sum(a, b), p = two_prod(a, b);
    if (q(s) != quad(a) + quad(b) || q(p) != quad(a) * quad(b)) ++bad_exact;
    const double r[5] = {rel(q(x + yc), q(x) + q(yc)), rel(q(x - yc), q(x) - q(yc)), rel(q(x * yc), q(x) * q(yc)),
                         rel(q(x / yc), q(x) / q(yc)), 0.0};
    const dfloat ax = x.hi < 0 ? -x : x;
    const quad sq = quad(std::sqrt(double(q(ax))));  // start, then two Newton steps in quad
    quad sqe = (sq + q(ax) / sq) / 2;
    sqe = (sqe + q(ax) / sqe) / 2;
    const double rs = rel(q(sqrt(ax)), sqe);
    for (int k = 0; k < 4; ++k) worst[k] = std::fmax(worst[k], r[k]);
    worst[4] = std::fmax(worst[4], rs);
  }
  int fail = bad_exact != 0;
  for (int k = 0; k < 5; ++k) {
    std::printf("%-5s largest relative error %.3e (bound %.3e)\n", names[k], worst[k], bound[k]);
    if (!(worst[k] <= bound[k])) fail = 1;
  }
  std::printf("inexact TwoSum/TwoProd results: %d\n", bad_exact);
  return fail;
}
