// dfloat.cuh -- double-float arithmetic (a value is hi + lo, two FP32 numbers) for the
// FP64-emulating amplitude mode.
//
// B300 issues FP32 FMAs at about 60 times its FP64 rate.  A double-float operation takes
// a handful of FP32 instructions and keeps about 48 significant bits (the FP32 exponent
// range), so the amplitude code of the smaller processes -- whose FP32 kernels are not
// bound by instruction fetch -- runs faster on it than in native FP64, with errors far
// below the reduced-precision modes.  The algorithms are the published error-free
// transformations, named at each use:
//   * TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s + e = a + b exactly;
//   * FastTwoSum (Dekker 1971): the same when |a| >= |b|;
//   * TwoProd with an FMA: p + e = a b exactly;
//   * double-word addition and multiplication of Joldes, Muller and Popescu (ACM TOMS
//     44 (2017) 1, "Tight and rigorous error bounds for basic building blocks of
//     double-word arithmetic"): AccurateDWPlusDW (relative error <= 3u^2) and
//     DWTimesDW2 (<= 5u^2), u = 2^-24;
//   * division and square root by one Newton correction of the FP32 result.
// Every FP32 step uses the __f*_rn intrinsics, which the compiler never contracts or
// reassociates, so the error-free transformations stay exact.
#pragma once

#include <cuda_runtime.h>

#include "helas.cuh"

namespace meb300 {

#if defined(__CUDA_ARCH__)
#define MEB_FADD(a, b) __fadd_rn(a, b)
#define MEB_FSUB(a, b) __fsub_rn(a, b)
#define MEB_FMUL(a, b) __fmul_rn(a, b)
#define MEB_FFMA(a, b, c) __fmaf_rn(a, b, c)
#define MEB_FDIV(a, b) __fdiv_rn(a, b)
#define MEB_FSQRT(a) __fsqrt_rn(a)
#else
#define MEB_FADD(a, b) ((a) + (b))
#define MEB_FSUB(a, b) ((a) - (b))
#define MEB_FMUL(a, b) ((a) * (b))
#define MEB_FFMA(a, b, c) std::fma(a, b, c)
#define MEB_FDIV(a, b) ((a) / (b))
#define MEB_FSQRT(a) std::sqrt(a)
#endif

struct dfloat {
  float hi, lo;
  dfloat() = default;
  HD dfloat(double x) {
    hi = float(x);
    lo = float(x - double(hi));
  }
  HD explicit operator double() const { return double(hi) + double(lo); }
};

HD dfloat df_make(float hi, float lo) {
  dfloat r;
  r.hi = hi;
  r.lo = lo;
  return r;
}
// Knuth's TwoSum
HD dfloat two_sum(float a, float b) {
  const float s = MEB_FADD(a, b);
  const float bb = MEB_FSUB(s, a);
  const float e = MEB_FADD(MEB_FSUB(a, MEB_FSUB(s, bb)), MEB_FSUB(b, bb));
  return df_make(s, e);
}
// Dekker's FastTwoSum (|a| >= |b|)
HD dfloat fast_two_sum(float a, float b) {
  const float s = MEB_FADD(a, b);
  return df_make(s, MEB_FSUB(b, MEB_FSUB(s, a)));
}
// TwoProd with an FMA
HD dfloat two_prod(float a, float b) {
  const float p = MEB_FMUL(a, b);
  return df_make(p, MEB_FFMA(a, b, -p));
}

// AccurateDWPlusDW (Joldes, Muller, Popescu 2017, Algorithm 6)
HD dfloat operator+(dfloat x, dfloat y) {
  const dfloat s = two_sum(x.hi, y.hi);
  const dfloat t = two_sum(x.lo, y.lo);
  const dfloat v = fast_two_sum(s.hi, MEB_FADD(s.lo, t.hi));
  return fast_two_sum(v.hi, MEB_FADD(t.lo, v.lo));
}
HD dfloat operator-(dfloat x) { return df_make(-x.hi, -x.lo); }
HD dfloat operator-(dfloat x, dfloat y) { return x + (-y); }
// DWTimesDW2 (Joldes, Muller, Popescu 2017, Algorithm 11)
HD dfloat operator*(dfloat x, dfloat y) {
  const dfloat c = two_prod(x.hi, y.hi);
  const float tl = MEB_FMUL(x.hi, y.lo);
  const float cl2 = MEB_FFMA(x.lo, y.hi, tl);
  return fast_two_sum(c.hi, MEB_FADD(c.lo, cl2));
}
// x / y: q1 = xh / yh, then one correction from the double-float residual x - q1 y
HD dfloat operator/(dfloat x, dfloat y) {
  const float q1 = MEB_FDIV(x.hi, y.hi);
  const dfloat r = x - y * dfloat(double(q1));
  const float q2 = MEB_FDIV(r.hi, y.hi);
  return fast_two_sum(q1, q2);
}
HD void operator+=(dfloat& a, dfloat b) { a = a + b; }
HD void operator-=(dfloat& a, dfloat b) { a = a - b; }
HD bool operator==(dfloat a, dfloat b) { return a.hi == b.hi && a.lo == b.lo; }
HD bool operator>(dfloat a, dfloat b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
HD bool operator>=(dfloat a, dfloat b) { return a > b || a == b; }
// sqrt: s = sqrt(xh), then s + (x - s^2) / (2 s) with the residual in double-float
HD dfloat sqrt(dfloat x) {
  if (!(x.hi > 0.0f)) return df_make(MEB_FSQRT(x.hi), 0.0f);
  const float s = MEB_FSQRT(x.hi);
  const dfloat r = x - two_prod(s, s);
  return fast_two_sum(s, MEB_FDIV(r.hi, MEB_FADD(s, s)));
}

}  // namespace meb300
