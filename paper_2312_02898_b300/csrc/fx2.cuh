// fx2.cuh -- packed FP32 pairs (two events per thread) for the FP32 amplitude kernels.
//
// Straight-line amplitude code of the large processes is longer than the instruction
// caches, and on B300 such code is bound by instruction fetch: a 288 KB stream of FP32
// FMAs issues at about a third of the FMA peak with 8 warps per SM.  The packed FP32
// instructions of sm_100+ (FFMA2 / FADD2 / FMUL2: two independent lanes per instruction)
// do twice the arithmetic per fetched instruction.  fx2 holds the same quantity of two
// different events, one per lane, so every routine below is the scalar routine of
// helas.cuh applied to two events at once, lane by lane, with the same rounding as
// scalar FP32 arithmetic (each packed FMA rounds once per lane).
//
// The packed instructions have no negated-operand form, so every signed sum of products
// is written as a chain of fused multiply-adds over its positive terms and one over its
// negative terms, joined by a single subtraction, or uses negated copies prepared once;
// a scalar FFMA negates its operands for free, a packed one would otherwise pay an
// instruction per sign.
//
// The host-side bodies (scalar lane-by-lane arithmetic) only let the host pass of nvcc
// compile the __host__ __device__ templates of helas.cuh for fx2; nothing calls them on
// the host.
#pragma once

#include <cuda_runtime.h>

#include "helas.cuh"

namespace meb300 {

struct fx2 {
  float2 v;
  fx2() = default;
  HD explicit fx2(float s) : v(make_float2(s, s)) {}
  HD fx2(float2 x) : v(x) {}
};

HD fx2 operator+(fx2 a, fx2 b) {
#if defined(__CUDA_ARCH__)
  return fx2(__fadd2_rn(a.v, b.v));
#else
  return fx2(make_float2(a.v.x + b.v.x, a.v.y + b.v.y));
#endif
}
HD fx2 operator*(fx2 a, fx2 b) {
#if defined(__CUDA_ARCH__)
  return fx2(__fmul2_rn(a.v, b.v));
#else
  return fx2(make_float2(a.v.x * b.v.x, a.v.y * b.v.y));
#endif
}
HD fx2 fmadd(fx2 a, fx2 b, fx2 c) {
#if defined(__CUDA_ARCH__)
  return fx2(__ffma2_rn(a.v, b.v, c.v));
#else
  return fx2(make_float2(fmaf(a.v.x, b.v.x, c.v.x), fmaf(a.v.y, b.v.y, c.v.y)));
#endif
}
// a - b as b * (-1) + a: one packed FMA, exact product, one rounding (= subtraction)
HD fx2 operator-(fx2 a, fx2 b) { return fmadd(b, fx2(-1.0f), a); }
HD fx2 operator-(fx2 a) { return a * fx2(-1.0f); }
HD void operator+=(fx2& a, fx2 b) { a = a + b; }
HD void operator-=(fx2& a, fx2 b) { a = a - b; }
HD fx2 operator/(fx2 a, fx2 b) { return fx2(make_float2(a.v.x / b.v.x, a.v.y / b.v.y)); }

using c2 = cx<fx2>;

// lanes of packed values
HD float lane(fx2 a, int l) { return l ? a.v.y : a.v.x; }
HD cx<float> lane(c2 a, int l) { return mk<float>(lane(a.r, l), lane(a.i, l)); }
HD fx2 pack(float a, float b) { return fx2(make_float2(a, b)); }
HD c2 pack(cx<float> a, cx<float> b) { return mk<fx2>(pack(a.r, b.r), pack(a.i, b.i)); }

// J += i a and J -= i a
template <> HD void acc_pi<fx2>(c2& J, c2 a) { J.r = J.r - a.i; J.i = J.i + a.r; }
template <> HD void acc_mi<fx2>(c2& J, c2 a) { J.r = J.r + a.i; J.i = J.i - a.r; }

// ---------------------------------------------------------------------------
// Minkowski products
// ---------------------------------------------------------------------------
// a.b = a0 b0 - a1 b1 - a2 b2 - a3 b3 for complex 4-vectors
HD c2 mdot_x2(const c2* a, const c2* b) {
  const fx2 pr = fmadd(a[3].i, b[3].i, fmadd(a[2].i, b[2].i, fmadd(a[1].i, b[1].i, a[0].r * b[0].r)));
  const fx2 nr = fmadd(a[3].r, b[3].r, fmadd(a[2].r, b[2].r, fmadd(a[1].r, b[1].r, a[0].i * b[0].i)));
  const fx2 pi = fmadd(a[0].i, b[0].r, a[0].r * b[0].i);
  const fx2 ni = fmadd(a[3].i, b[3].r, fmadd(a[3].r, b[3].i, fmadd(a[2].i, b[2].r,
                 fmadd(a[2].r, b[2].i, fmadd(a[1].i, b[1].r, a[1].r * b[1].i)))));
  return mk<fx2>(pr - nr, pi - ni);
}
// k.a for a real k
HD c2 mdot_x2(const fx2* k, const c2* a) {
  const fx2 nr = fmadd(k[3], a[3].r, fmadd(k[2], a[2].r, k[1] * a[1].r));
  const fx2 ni = fmadd(k[3], a[3].i, fmadd(k[2], a[2].i, k[1] * a[1].i));
  return mk<fx2>(fmadd(k[0], a[0].r, -nr), fmadd(k[0], a[0].i, -ni));
}
template <> HD c2 mdot<fx2>(const c2* a, const c2* b) { return mdot_x2(a, b); }
template <> HD c2 mdot<fx2>(const fx2* k, const c2* a) { return mdot_x2(k, a); }

// ---------------------------------------------------------------------------
// vertices
// ---------------------------------------------------------------------------
// s V3(X, Y): V3 = (X.Y)(kx - ky) + Y (kx + 2ky).X - X (2kx + ky).Y
HD void v3_x2(const c2* X, const fx2* kx, const c2* Y, const fx2* ky, fx2 s, c2* out) {
  const fx2 two(2.0f);
  fx2 d[4], a[4], b[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    d[m] = kx[m] - ky[m];
    a[m] = fmadd(two, ky[m], kx[m]);
    b[m] = fmadd(two, kx[m], ky[m]);
  }
  const c2 xy = mdot_x2(X, Y), ax = mdot_x2(a, X), by = mdot_x2(b, Y);
  const fx2 ns = -s;
  const fx2 xyr = s * xy.r, xyi = s * xy.i;
  const fx2 axr = s * ax.r, axi = s * ax.i, naxi = ns * ax.i;
  const fx2 byi = s * by.i, nbyr = ns * by.r, nbyi = ns * by.i;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    out[m].r = fmadd(X[m].i, byi, fmadd(X[m].r, nbyr, fmadd(Y[m].i, naxi, fmadd(Y[m].r, axr, d[m] * xyr))));
    out[m].i = fmadd(X[m].i, nbyr, fmadd(X[m].r, nbyi, fmadd(Y[m].i, axr, fmadd(Y[m].r, axi, d[m] * xyi))));
  }
}

template <> HD void g3_current<fx2>(const c2* X, const fx2* kx, const c2* Y, const fx2* ky, fx2 invK2, c2* out) {
  v3_x2(X, kx, Y, ky, invK2, out);
}

// s V4_S(X, Y, Z) = A U + B W with (S=1) A = s X.Z, U = Y, B = -s Y.Z, W = X;
// (S=2) A = s X.Y, U = Z, B = -s Y.Z, W = X; (S=3) A = s X.Y, U = Z, B = -s X.Z, W = Y
HD void lin2_x2(fx2 s, c2 pa, const c2* U, c2 pb, const c2* W, c2* out) {
  const fx2 ns = -s;
  const fx2 ar = s * pa.r, ai = s * pa.i, nai = ns * pa.i;
  const fx2 br = ns * pb.r, bi = ns * pb.i, nbi = s * pb.i;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    out[m].r = fmadd(W[m].i, nbi, fmadd(W[m].r, br, fmadd(U[m].i, nai, U[m].r * ar)));
    out[m].i = fmadd(W[m].i, br, fmadd(W[m].r, bi, fmadd(U[m].i, ar, U[m].r * ai)));
  }
}
template <int S>
HD void g4_x2(const c2* X, const c2* Y, const c2* Z, fx2 s, c2* out) {
  if (S == 1) lin2_x2(s, mdot_x2(X, Z), Y, mdot_x2(Y, Z), X, out);
  else if (S == 2) lin2_x2(s, mdot_x2(X, Y), Z, mdot_x2(Y, Z), X, out);
  else lin2_x2(s, mdot_x2(X, Y), Z, mdot_x2(X, Z), Y, out);
}
template <> HD void g4_current<1, fx2>(const c2* X, const c2* Y, const c2* Z, fx2 s, c2* out) { g4_x2<1>(X, Y, Z, s, out); }
template <> HD void g4_current<2, fx2>(const c2* X, const c2* Y, const c2* Z, fx2 s, c2* out) { g4_x2<2>(X, Y, Z, s, out); }
template <> HD void g4_current<3, fx2>(const c2* X, const c2* Y, const c2* Z, fx2 s, c2* out) { g4_x2<3>(X, Y, Z, s, out); }

// complex a b - c d, and s (a b - c d)
HD c2 cdiff_x2(c2 a, c2 b, c2 c, c2 d) {
  const fx2 pr = fmadd(c.i, d.i, a.r * b.r), nr = fmadd(c.r, d.r, a.i * b.i);
  const fx2 pi = fmadd(a.i, b.r, a.r * b.i), ni = fmadd(c.i, d.r, c.r * d.i);
  return mk<fx2>(pr - nr, pi - ni);
}

template <> HD c2 close_dot<fx2>(const c2* PJ, const c2* G) { return mdot_x2(PJ, G); }

template <> HD c2 close_v3<fx2>(const c2* PJ, const c2* X, const fx2* kx, const c2* Y, const fx2* ky, fx2 invK2) {
  c2 v[4];
  v3_x2(X, kx, Y, ky, invK2, v);
  return mdot_x2(PJ, v);
}

template <int S>
HD c2 close_v4_x2(const c2* PJ, const c2* X, const c2* Y, const c2* Z, fx2 s) {
  c2 r;
  if (S == 1) r = cdiff_x2(mdot_x2(X, Z), mdot_x2(Y, PJ), mdot_x2(Y, Z), mdot_x2(X, PJ));
  else if (S == 2) r = cdiff_x2(mdot_x2(X, Y), mdot_x2(Z, PJ), mdot_x2(Y, Z), mdot_x2(X, PJ));
  else r = cdiff_x2(mdot_x2(X, Y), mdot_x2(Z, PJ), mdot_x2(X, Z), mdot_x2(Y, PJ));
  return mk<fx2>(s * r.r, s * r.i);
}
template <> HD c2 close_v4<1, fx2>(const c2* PJ, const c2* X, const c2* Y, const c2* Z, fx2 s) { return close_v4_x2<1>(PJ, X, Y, Z, s); }
template <> HD c2 close_v4<2, fx2>(const c2* PJ, const c2* X, const c2* Y, const c2* Z, fx2 s) { return close_v4_x2<2>(PJ, X, Y, Z, s); }
template <> HD c2 close_v4<3, fx2>(const c2* PJ, const c2* X, const c2* Y, const c2* Z, fx2 s) { return close_v4_x2<3>(PJ, X, Y, Z, s); }

// ---------------------------------------------------------------------------
// quark line
// ---------------------------------------------------------------------------
// G0 +- G3 and G1 +- i G2 of a complex 4-vector
struct slash_x2 {
  c2 p03, m03, p12, m12;
};
HD slash_x2 slash_parts(const c2* G) {
  slash_x2 s;
  s.p03 = mk<fx2>(G[0].r + G[3].r, G[0].i + G[3].i);
  s.m03 = mk<fx2>(G[0].r - G[3].r, G[0].i - G[3].i);
  s.p12 = mk<fx2>(G[1].r - G[2].i, G[1].i + G[2].r);
  s.m12 = mk<fx2>(G[1].r + G[2].i, G[1].i - G[2].r);
  return s;
}
// complex a b + c d, and a b - c d
HD c2 csum_x2(c2 a, c2 b, c2 c, c2 d) {
  const fx2 pr = fmadd(c.r, d.r, a.r * b.r), nr = fmadd(c.i, d.i, a.i * b.i);
  const fx2 im = fmadd(c.i, d.r, fmadd(c.r, d.i, fmadd(a.i, b.r, a.r * b.i)));
  return mk<fx2>(pr - nr, im);
}

// (a | b) gamma.G = (b G.sigmabar | a G.sigma)
HD void bra_gslash_x2(const c2* f, const c2* G, c2* o) {
  const slash_x2 s = slash_parts(G);
  o[0] = csum_x2(f[2], s.p03, f[3], s.p12);
  o[1] = csum_x2(f[2], s.m12, f[3], s.m03);
  o[2] = cdiff_x2(f[0], s.m03, f[1], s.p12);
  o[3] = cdiff_x2(f[1], s.p03, f[0], s.m12);
}
// gamma.G (l ; r) = (G.sigma r ; G.sigmabar l)
HD void gslash_ket_x2(const c2* G, const c2* f, c2* o) {
  const slash_x2 s = slash_parts(G);
  o[0] = cdiff_x2(s.m03, f[2], s.m12, f[3]);
  o[1] = cdiff_x2(s.p03, f[3], s.p12, f[2]);
  o[2] = csum_x2(s.p03, f[0], s.m12, f[1]);
  o[3] = csum_x2(s.p12, f[0], s.m03, f[1]);
}

// (c | d) (qslash + m) = (m c + d q.sigmabar | c q.sigma + m d), q real:
//   o0 = m c0 + p03 c2 + (q1 + i q2) c3      o1 = m c1 + (q1 - i q2) c2 + m03 c3
//   o2 = m03 c0 - (q1 + i q2) c1 + m c2      o3 = p03 c1 - (q1 - i q2) c0 + m c3
// with p03 = q0 + q3, m03 = q0 - q3; every term is one fused multiply-add, the negative
// ones through nq1 = -q1, nq2 = -q2
HD void bra_prop_x2(const c2* c, const fx2* q, fx2 m, c2* o) {
  const fx2 p03 = q[0] + q[3], m03 = q[0] - q[3];
  const fx2 q1 = q[1], q2 = q[2], nq1 = -q1, nq2 = -q2;
  o[0].r = fmadd(c[3].i, nq2, fmadd(c[3].r, q1, fmadd(c[2].r, p03, m * c[0].r)));
  o[0].i = fmadd(c[3].r, q2, fmadd(c[3].i, q1, fmadd(c[2].i, p03, m * c[0].i)));
  o[1].r = fmadd(c[3].r, m03, fmadd(c[2].i, q2, fmadd(c[2].r, q1, m * c[1].r)));
  o[1].i = fmadd(c[3].i, m03, fmadd(c[2].r, nq2, fmadd(c[2].i, q1, m * c[1].i)));
  o[2].r = fmadd(c[1].i, q2, fmadd(c[1].r, nq1, fmadd(c[0].r, m03, m * c[2].r)));
  o[2].i = fmadd(c[1].r, nq2, fmadd(c[1].i, nq1, fmadd(c[0].i, m03, m * c[2].i)));
  o[3].r = fmadd(c[0].i, nq2, fmadd(c[0].r, nq1, fmadd(c[1].r, p03, m * c[3].r)));
  o[3].i = fmadd(c[0].r, q2, fmadd(c[0].i, nq1, fmadd(c[1].i, p03, m * c[3].i)));
}
// (qslash + m) (l ; r) = (m l + q.sigma r ; q.sigmabar l + m r), q real:
//   o0 = m c0 + m03 c2 - (q1 - i q2) c3      o1 = m c1 + p03 c3 - (q1 + i q2) c2
//   o2 = p03 c0 + (q1 - i q2) c1 + m c2      o3 = (q1 + i q2) c0 + m03 c1 + m c3
HD void prop_ket_x2(const fx2* q, fx2 m, const c2* c, c2* o) {
  const fx2 p03 = q[0] + q[3], m03 = q[0] - q[3];
  const fx2 q1 = q[1], q2 = q[2], nq1 = -q1, nq2 = -q2;
  o[0].r = fmadd(c[3].i, nq2, fmadd(c[3].r, nq1, fmadd(c[2].r, m03, m * c[0].r)));
  o[0].i = fmadd(c[3].r, q2, fmadd(c[3].i, nq1, fmadd(c[2].i, m03, m * c[0].i)));
  o[1].r = fmadd(c[2].i, q2, fmadd(c[2].r, nq1, fmadd(c[3].r, p03, m * c[1].r)));
  o[1].i = fmadd(c[2].r, nq2, fmadd(c[2].i, nq1, fmadd(c[3].i, p03, m * c[1].i)));
  o[2].r = fmadd(c[1].i, q2, fmadd(c[1].r, q1, fmadd(c[0].r, p03, m * c[2].r)));
  o[2].i = fmadd(c[1].r, nq2, fmadd(c[1].i, q1, fmadd(c[0].i, p03, m * c[2].i)));
  o[3].r = fmadd(c[0].i, nq2, fmadd(c[0].r, q1, fmadd(c[1].r, m03, m * c[3].r)));
  o[3].i = fmadd(c[0].r, q2, fmadd(c[0].i, q1, fmadd(c[1].i, m03, m * c[3].i)));
}
// u z for a complex constant z given as (zr, zi, -zi)
HD c2 cscale_x2(c2 u, fx2 zr, fx2 zi, fx2 nzi) {
  return mk<fx2>(fmadd(u.i, nzi, u.r * zr), fmadd(u.i, zr, u.r * zi));
}

template <> HD void bra_step<fx2>(const c2* F, const c2* G, const fx2* q, fx2 m, c2 invD, c2* out) {
  c2 t[4], u[4];
  bra_gslash_x2(F, G, t);
  bra_prop_x2(t, q, m, u);
  const fx2 nzi = -invD.i;
#pragma unroll
  for (int j = 0; j < 4; ++j) out[j] = cscale_x2(u[j], invD.r, invD.i, nzi);
}

template <> HD void ket_step<fx2>(const c2* G, const c2* F, const fx2* q, fx2 m, c2 invD, c2* out) {
  c2 t[4], u[4];
  gslash_ket_x2(G, F, t);
  prop_ket_x2(q, m, t, u);
  const fx2 nzi = -invD.i;
#pragma unroll
  for (int j = 0; j < 4; ++j) out[j] = cscale_x2(u[j], invD.r, invD.i, nzi);
}

// j^mu = B gamma^mu K = a sigma^mu r + b sigmabar^mu l, B = (a|b), K = (l;r)
template <> HD void pair_current<fx2>(const c2* B, const c2* K, c2* j) {
  // the eight bilinears, each the product of a row and a column component
  auto cm = [](c2 a, c2 b) {
    return mk<fx2>(a.r * b.r - a.i * b.i, fmadd(a.i, b.r, a.r * b.i));
  };
  const c2 a1r1 = cm(B[0], K[2]), a2r2 = cm(B[1], K[3]), a1r2 = cm(B[0], K[3]), a2r1 = cm(B[1], K[2]);
  const c2 b1l1 = cm(B[2], K[0]), b2l2 = cm(B[3], K[1]), b1l2 = cm(B[2], K[1]), b2l1 = cm(B[3], K[0]);
  j[0] = mk<fx2>((a1r1.r + a2r2.r) + (b1l1.r + b2l2.r), (a1r1.i + a2r2.i) + (b1l1.i + b2l2.i));
  j[1] = mk<fx2>((a1r2.r + a2r1.r) - (b1l2.r + b2l1.r), (a1r2.i + a2r1.i) - (b1l2.i + b2l1.i));
  // i ((a2r1 - a1r2) - (b2l1 - b1l2))
  j[2] = mk<fx2>((a1r2.i - a2r1.i) + (b2l1.i - b1l2.i), (a2r1.r - a1r2.r) - (b2l1.r - b1l2.r));
  j[3] = mk<fx2>((a1r1.r - a2r2.r) - (b1l1.r - b2l2.r), (a1r1.i - a2r2.i) - (b1l1.i - b2l2.i));
}

// ---------------------------------------------------------------------------
// external wavefunctions: lane by lane with the scalar routines (a few per helicity)
// ---------------------------------------------------------------------------
HD void unpack4(const fx2* p, float* p0, float* p1) {
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    p0[m] = lane(p[m], 0);
    p1[m] = lane(p[m], 1);
  }
}
HD void pack4(const cx<float>* w0, const cx<float>* w1, c2* w) {
#pragma unroll
  for (int m = 0; m < 4; ++m) w[m] = pack(w0[m], w1[m]);
}
template <> HD void ext_eps<fx2>(const fx2* k, int lam, bool outgoing, c2* w) {
  float k0[4], k1[4];
  cx<float> w0[4], w1[4];
  unpack4(k, k0, k1);
  ext_eps<float>(k0, lam, outgoing, w0);
  ext_eps<float>(k1, lam, outgoing, w1);
  pack4(w0, w1, w);
}
#define MEB_EXT_X2(NAME)                                                   \
  template <> HD void NAME<fx2>(const fx2* p, fx2 m, int lam, c2* w) {     \
    float p0[4], p1[4];                                                    \
    cx<float> w0[4], w1[4];                                                \
    unpack4(p, p0, p1);                                                    \
    NAME<float>(p0, lane(m, 0), lam, w0);                                  \
    NAME<float>(p1, lane(m, 1), lam, w1);                                  \
    pack4(w0, w1, w);                                                      \
  }
MEB_EXT_X2(ext_u)
MEB_EXT_X2(ext_v)
MEB_EXT_X2(ext_ubar)
MEB_EXT_X2(ext_vbar)
#undef MEB_EXT_X2

}  // namespace meb300
