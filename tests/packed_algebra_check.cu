// Host-only check that every packed FP32 routine (csrc/fx2.cuh) equals the scalar
// routine of csrc/helas.cuh lane by lane: lane 0 on one set of random inputs, lane 1 on
// another.  Compiled by nvcc for the host (the packed routines then run their lane-by-lane
// host bodies), so it pins the algebra of each routine -- the signs, indices and operand
// order of its fused form -- on the CPU; the device instructions are pinned by the GPU
// parity tests.  Prints the largest relative difference; exit status 1 above 1e-5.
#include <cmath>
#include <cstdio>
#include <random>

#include "fx2.cuh"

using namespace meb300;

static std::mt19937_64 rng(7);
static float uni() { return std::uniform_real_distribution<float>(-1.0f, 1.0f)(rng); }
static double worst = 0.0;
static const char* worst_name = "";

static void cmp(const char* name, float packed_lane, float scalar, float scale) {
  const double d = std::fabs(double(packed_lane) - double(scalar)) / std::max(1e-30, double(scale));
  if (d > worst) { worst = d; worst_name = name; }
}
static float mag(const cx<float>* v, int n) {
  float s = 0;
  for (int i = 0; i < n; ++i) s = std::max(s, std::max(std::fabs(v[i].r), std::fabs(v[i].i)));
  return s;
}
static void cmpv(const char* name, const c2* p, const cx<float>* s0, const cx<float>* s1, int n) {
  const float m0 = mag(s0, n), m1 = mag(s1, n);
  for (int i = 0; i < n; ++i) {
    cmp(name, p[i].r.v.x, s0[i].r, m0); cmp(name, p[i].i.v.x, s0[i].i, m0);
    cmp(name, p[i].r.v.y, s1[i].r, m1); cmp(name, p[i].i.v.y, s1[i].i, m1);
  }
}
struct Vecs {  // one complex 4-vector and one real 4-vector per lane, and the packed forms
  cx<float> c0[4], c1[4];
  float k0[4], k1[4];
  c2 c[4];
  fx2 k[4];
  void fill(bool timelike = false) {
    for (int m = 0; m < 4; ++m) {
      c0[m] = mk<float>(uni(), uni()); c1[m] = mk<float>(uni(), uni());
      k0[m] = uni(); k1[m] = uni();
    }
    if (timelike) { k0[0] = 2.0f + std::fabs(k0[0]); k1[0] = 2.0f + std::fabs(k1[0]); }
    for (int m = 0; m < 4; ++m) { c[m] = pack(c0[m], c1[m]); k[m] = pack(k0[m], k1[m]); }
  }
};

int main() {
  for (int trial = 0; trial < 200; ++trial) {
    Vecs X, Y, Z, P;
    X.fill(); Y.fill(); Z.fill(); P.fill(true);
    const float s0 = uni(), s1 = uni(), m0 = 0.5f + std::fabs(uni()), m1 = m0;
    const fx2 s = pack(s0, s1), m = pack(m0, m1);
    const cx<float> d0 = mk<float>(uni(), uni()), d1 = mk<float>(uni(), uni());
    const c2 d = pack(d0, d1);
    c2 out[4];
    cx<float> o0[4], o1[4];
    {  // Minkowski products
      c2 r = mdot<fx2>(X.c, Y.c);
      cx<float> r0 = mdot<float>(X.c0, Y.c0), r1 = mdot<float>(X.c1, Y.c1);
      cmpv("mdot(cx,cx)", &r, &r0, &r1, 1);
      r = mdot<fx2>(X.k, Y.c); r0 = mdot<float>(X.k0, Y.c0); r1 = mdot<float>(X.k1, Y.c1);
      cmpv("mdot(re,cx)", &r, &r0, &r1, 1);
    }
    g3_current<fx2>(X.c, X.k, Y.c, Y.k, s, out);
    g3_current<float>(X.c0, X.k0, Y.c0, Y.k0, s0, o0); g3_current<float>(X.c1, X.k1, Y.c1, Y.k1, s1, o1);
    cmpv("g3_current", out, o0, o1, 4);
    g4_current<1, fx2>(X.c, Y.c, Z.c, s, out);
    g4_current<1, float>(X.c0, Y.c0, Z.c0, s0, o0); g4_current<1, float>(X.c1, Y.c1, Z.c1, s1, o1);
    cmpv("g4_current<1>", out, o0, o1, 4);
    g4_current<2, fx2>(X.c, Y.c, Z.c, s, out);
    g4_current<2, float>(X.c0, Y.c0, Z.c0, s0, o0); g4_current<2, float>(X.c1, Y.c1, Z.c1, s1, o1);
    cmpv("g4_current<2>", out, o0, o1, 4);
    g4_current<3, fx2>(X.c, Y.c, Z.c, s, out);
    g4_current<3, float>(X.c0, Y.c0, Z.c0, s0, o0); g4_current<3, float>(X.c1, Y.c1, Z.c1, s1, o1);
    cmpv("g4_current<3>", out, o0, o1, 4);
    {
      c2 r = close_dot<fx2>(P.c, X.c);
      cx<float> r0 = close_dot<float>(P.c0, X.c0), r1 = close_dot<float>(P.c1, X.c1);
      cmpv("close_dot", &r, &r0, &r1, 1);
      r = close_v3<fx2>(P.c, X.c, X.k, Y.c, Y.k, s);
      r0 = close_v3<float>(P.c0, X.c0, X.k0, Y.c0, Y.k0, s0); r1 = close_v3<float>(P.c1, X.c1, X.k1, Y.c1, Y.k1, s1);
      cmpv("close_v3", &r, &r0, &r1, 1);
      r = close_v4<1, fx2>(P.c, X.c, Y.c, Z.c, s);
      r0 = close_v4<1, float>(P.c0, X.c0, Y.c0, Z.c0, s0); r1 = close_v4<1, float>(P.c1, X.c1, Y.c1, Z.c1, s1);
      cmpv("close_v4<1>", &r, &r0, &r1, 1);
      r = close_v4<2, fx2>(P.c, X.c, Y.c, Z.c, s);
      r0 = close_v4<2, float>(P.c0, X.c0, Y.c0, Z.c0, s0); r1 = close_v4<2, float>(P.c1, X.c1, Y.c1, Z.c1, s1);
      cmpv("close_v4<2>", &r, &r0, &r1, 1);
      r = close_v4<3, fx2>(P.c, X.c, Y.c, Z.c, s);
      r0 = close_v4<3, float>(P.c0, X.c0, Y.c0, Z.c0, s0); r1 = close_v4<3, float>(P.c1, X.c1, Y.c1, Z.c1, s1);
      cmpv("close_v4<3>", &r, &r0, &r1, 1);
    }
    bra_step<fx2>(X.c, Y.c, P.k, m, d, out);
    bra_step<float>(X.c0, Y.c0, P.k0, m0, d0, o0); bra_step<float>(X.c1, Y.c1, P.k1, m1, d1, o1);
    cmpv("bra_step", out, o0, o1, 4);
    ket_step<fx2>(Y.c, X.c, P.k, m, d, out);
    ket_step<float>(Y.c0, X.c0, P.k0, m0, d0, o0); ket_step<float>(Y.c1, X.c1, P.k1, m1, d1, o1);
    cmpv("ket_step", out, o0, o1, 4);
    pair_current<fx2>(X.c, Y.c, out);
    pair_current<float>(X.c0, Y.c0, o0); pair_current<float>(X.c1, Y.c1, o1);
    cmpv("pair_current", out, o0, o1, 4);
    for (int lam = -1; lam <= 1; lam += 2) {
      for (int outgoing = 0; outgoing < 2; ++outgoing) {
        ext_eps<fx2>(P.k, lam, outgoing, out);
        ext_eps<float>(P.k0, lam, outgoing, o0); ext_eps<float>(P.k1, lam, outgoing, o1);
        cmpv("ext_eps", out, o0, o1, 4);
      }
      ext_u<fx2>(P.k, m, lam, out); ext_u<float>(P.k0, m0, lam, o0); ext_u<float>(P.k1, m1, lam, o1);
      cmpv("ext_u", out, o0, o1, 4);
      ext_v<fx2>(P.k, m, lam, out); ext_v<float>(P.k0, m0, lam, o0); ext_v<float>(P.k1, m1, lam, o1);
      cmpv("ext_v", out, o0, o1, 4);
      ext_ubar<fx2>(P.k, m, lam, out); ext_ubar<float>(P.k0, m0, lam, o0); ext_ubar<float>(P.k1, m1, lam, o1);
      cmpv("ext_ubar", out, o0, o1, 4);
      ext_vbar<fx2>(P.k, m, lam, out); ext_vbar<float>(P.k0, m0, lam, o0); ext_vbar<float>(P.k1, m1, lam, o1);
      cmpv("ext_vbar", out, o0, o1, 4);
    }
    {  // colour-flow accumulation
      c2 J = d;
      cx<float> J0 = d0, J1 = d1;
      acc_pi<fx2>(J, X.c[0]); acc_pi<float>(J0, X.c0[0]); acc_pi<float>(J1, X.c1[0]);
      acc_mi<fx2>(J, Y.c[1]); acc_mi<float>(J0, Y.c0[1]); acc_mi<float>(J1, Y.c1[1]);
      cmpv("acc_pi/acc_mi", &J, &J0, &J1, 1);
    }
  }
  std::printf("largest relative difference %.3e (%s)\n", worst, worst_name);
  return worst > 1e-5 ? 1 : 0;
}
