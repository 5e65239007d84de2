// helas.cuh -- HELAS-style helicity wavefunctions and vertex currents for the
// event-parallel matrix-element kernels (one event per thread).
//
// Conventions (the physics of the HELAS library, Murayama/Watanabe/Hagiwara KEK 91-11,
// re-derived here in the chiral representation):
//   * gamma^mu = [[0, sigma^mu], [sigmabar^mu, 0]], sigma = (1, s), sigmabar = (1, -s);
//     a Dirac spinor is (psi_L ; psi_R), P_L keeps the upper two components;
//   * a "bra" wavefunction is a row spinor already multiplied by gamma^0 (ubar, vbar);
//     a "ket" is a column spinor (u, v); a vector wavefunction holds contravariant
//     components W^mu;
//   * momenta are "incoming": incoming particles carry +p, outgoing ones -p; a fermion
//     current carries the momentum that flows along the fermion arrow.
//
// Every routine computes a *raw* value: no coupling constant and no factor of i; the
// generator folds g_s (one power per external gluon) and the phases of vertices and
// propagators into the colour-flow coefficients, so the device code multiplies by no
// constants.  Propagator denominators arrive precomputed in FP64 (once per event,
// outside the helicity loop) and converted to the working precision R.
#pragma once

#include <cmath>
#include <cstdint>

#if defined(__CUDACC__)
#define HD __host__ __device__ __forceinline__
#define NOINL __host__ __device__ __noinline__
#else
#define HD inline
#define NOINL __attribute__((noinline))
#endif
// block barrier of the generated code's optional sync points (nothing on the host)
#if defined(__CUDA_ARCH__)
#define MEB_BLOCK_SYNC() __syncthreads()
#else
#define MEB_BLOCK_SYNC() ((void)0)
#endif

namespace meb300 {

template <class R>
struct alignas(2 * sizeof(R)) cx {
  R r, i;
};

template <class R> HD cx<R> mk(R r, R i) { cx<R> z; z.r = r; z.i = i; return z; }
template <class R> HD cx<R> operator+(cx<R> a, cx<R> b) { return mk<R>(a.r + b.r, a.i + b.i); }
template <class R> HD cx<R> operator-(cx<R> a, cx<R> b) { return mk<R>(a.r - b.r, a.i - b.i); }
template <class R> HD cx<R> operator-(cx<R> a) { return mk<R>(-a.r, -a.i); }
template <class R> HD cx<R> operator*(cx<R> a, cx<R> b) { return mk<R>(a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r); }
template <class R> HD cx<R> operator*(R s, cx<R> a) { return mk<R>(s * a.r, s * a.i); }
template <class R> HD cx<R> conjg(cx<R> a) { return mk<R>(a.r, -a.i); }
template <class R> HD cx<R> times_i(cx<R> a) { return mk<R>(-a.i, a.r); }
template <class R> HD void operator+=(cx<R>& a, cx<R> b) { a.r += b.r; a.i += b.i; }
template <class R> HD void operator-=(cx<R>& a, cx<R> b) { a.r -= b.r; a.i -= b.i; }

// J += i a  and  J -= i a  (the colour-flow accumulation of the generated code)
template <class R> HD void acc_pi(cx<R>& J, cx<R> a) { J.r -= a.i; J.i += a.r; }
template <class R> HD void acc_mi(cx<R>& J, cx<R> a) { J.r += a.i; J.i -= a.r; }
// a * b + c for real types (contracted into one FMA for float and double)
template <class R> HD R fmadd(R a, R b, R c) { return a * b + c; }

template <class R> HD void copy4(cx<R>* dst, const cx<R>* src) {
#pragma unroll
  for (int m = 0; m < 4; ++m) dst[m] = src[m];
}

// Sums of complex products as chains of real multiply-adds.  Written with the cx
// operators, every complex product is rounded on its own and then added (two
// multiplies, two multiply-adds and two adds for c + a b); as one chain each real part
// of c + a b takes two multiply-adds, so a sum of n complex products costs 4n - 2
// instructions instead of 6n - 2.  Negated operands are free in an FMA.
template <class R> HD cx<R> cmul(cx<R> a, cx<R> b) { return mk<R>(fmadd(a.r, b.r, -(a.i * b.i)), fmadd(a.r, b.i, a.i * b.r)); }
// c + a b
template <class R> HD cx<R> cfma(cx<R> a, cx<R> b, cx<R> c) {
  return mk<R>(fmadd(a.r, b.r, fmadd(-a.i, b.i, c.r)), fmadd(a.r, b.i, fmadd(a.i, b.r, c.i)));
}
// c - a b
template <class R> HD cx<R> cfms(cx<R> a, cx<R> b, cx<R> c) {
  return mk<R>(fmadd(-a.r, b.r, fmadd(a.i, b.i, c.r)), fmadd(-a.r, b.i, fmadd(-a.i, b.r, c.i)));
}
// c + s a and c - s a for real s
template <class R> HD cx<R> rfma(R s, cx<R> a, cx<R> c) { return mk<R>(fmadd(s, a.r, c.r), fmadd(s, a.i, c.i)); }
template <class R> HD cx<R> rfms(R s, cx<R> a, cx<R> c) { return mk<R>(fmadd(-s, a.r, c.r), fmadd(-s, a.i, c.i)); }

// Minkowski product of two complex 4-vectors (bilinear, no conjugation)
template <class R> HD cx<R> mdot(const cx<R>* a, const cx<R>* b) {
  return cfms(a[3], b[3], cfms(a[2], b[2], cfms(a[1], b[1], cmul(a[0], b[0]))));
}
// Minkowski product of a real and a complex 4-vector
template <class R> HD cx<R> mdot(const R* k, const cx<R>* a) {
  return mk<R>(k[0] * a[0].r - k[1] * a[1].r - k[2] * a[2].r - k[3] * a[3].r,
               k[0] * a[0].i - k[1] * a[1].i - k[2] * a[2].i - k[3] * a[3].i);
}

// ---------------------------------------------------------------------------
// Double-double arithmetic (Dekker 1971; Knuth TAOCP vol. 2, 4.2.2) for propagator
// invariants: the Minkowski square of a nearly light-like sum of momenta cancels most
// of its digits in plain FP64, so the sum and the square are formed without rounding
// error (error-free sums, FMA-exact products) and rounded once at the end.
// ---------------------------------------------------------------------------
struct dd {
  double hi, lo;
};
HD dd dd_two_sum(double a, double b) {
  const double s = a + b, bb = s - a;
  return dd{s, (a - (s - bb)) + (b - bb)};
}
HD dd dd_renorm(double hi, double lo) {
  const double s = hi + lo;
  return dd{s, lo - (s - hi)};
}
HD dd dd_add(dd x, dd y) {
  const dd s = dd_two_sum(x.hi, y.hi);
  return dd_renorm(s.hi, s.lo + (x.lo + y.lo));
}
HD dd dd_add(dd x, double y) {
  const dd s = dd_two_sum(x.hi, y);
  return dd_renorm(s.hi, s.lo + x.lo);
}
HD dd dd_sq(dd x) {
  const double p = x.hi * x.hi;
  const double e = fma(x.hi, x.hi, -p);
  return dd_renorm(p, e + 2.0 * x.hi * x.lo);
}
HD dd dd_neg(dd x) { return dd{-x.hi, -x.lo}; }
// q^2 - m^2 for q given as four double-double components
HD double dd_invariant(const dd* q, double m) {
  dd s = dd_sq(q[0]);
  s = dd_add(s, dd_neg(dd_sq(q[1])));
  s = dd_add(s, dd_neg(dd_sq(q[2])));
  s = dd_add(s, dd_neg(dd_sq(q[3])));
  s = dd_add(s, -m * m);
  return s.hi + s.lo;
}
// The same calls in plain FP64, for the FP32 and mixed modes.  There the invariants
// only need to be far more accurate than the FP32 amplitudes: the rounding error of a
// plain FP64 invariant is about 1e-16 times the event's conditioning number, and events
// conditioned worse than the rescue threshold are evaluated again in FP64 (with the
// error-free forms).  The error-free forms take about ten FP64 operations each, and
// B300 issues FP64 at 1/64 of its FP32 rate, so in those modes they would outweigh the
// amplitudes of the smaller processes.
struct dd_plain {
  double hi, lo;  // lo stays 0; the same initialiser as dd
};
HD dd_plain dd_add(dd_plain x, double y) { return dd_plain{x.hi + y, 0.0}; }
HD double dd_invariant(const dd_plain* q, double m) {
  return q[0].hi * q[0].hi - q[1].hi * q[1].hi - q[2].hi * q[2].hi - q[3].hi * q[3].hi - m * m;
}
// invariant arithmetic for amplitudes of type R: error-free for FP64, plain otherwise
template <class R> struct dd_select { using type = dd; };
template <> struct dd_select<float> { using type = dd_plain; };
template <class R> using dd_for = typename dd_select<R>::type;

// ---------------------------------------------------------------------------
// external wavefunctions
// ---------------------------------------------------------------------------
// Two-component helicity eigenvector chi_lam of sigma.p_hat.  Phase convention:
// chi_+ = (cos th/2, e^{i ph} sin th/2), chi_- = (-e^{-i ph} sin th/2, cos th/2), in
// the forward hemisphere; in the backward hemisphere both are multiplied by e^{-i ph}
// (resp. e^{+i ph}) so that no component is computed as a small difference.
template <class R>
HD void helicity_chi(const R* p, int lam, cx<R>* chi) {
  const R px = p[1], py = p[2], pz = p[3];
  const R ap = sqrt(px * px + py * py + pz * pz);
  if (pz >= R(0)) {
    const R s = ap + pz;
    const R nrm = R(1) / sqrt(R(2) * ap * s);
    if (lam > 0) { chi[0] = mk<R>(s * nrm, R(0)); chi[1] = mk<R>(px * nrm, py * nrm); }
    else         { chi[0] = mk<R>(-px * nrm, py * nrm); chi[1] = mk<R>(s * nrm, R(0)); }
  } else {
    const R d = ap - pz;
    const R nrm = R(1) / sqrt(R(2) * ap * d);
    if (lam > 0) { chi[0] = mk<R>(px * nrm, -py * nrm); chi[1] = mk<R>(d * nrm, R(0)); }
    else         { chi[0] = mk<R>(-d * nrm, R(0));      chi[1] = mk<R>(px * nrm, py * nrm); }
  }
}

// sqrt(E + |p|) and sqrt(E - |p|) = m / sqrt(E + |p|), free of cancellation
template <class R>
HD void omegas(const R* p, R m, R& wp, R& wm) {
  const R ap = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
  wp = sqrt(p[0] + ap);
  wm = (m == R(0)) ? R(0) : m / wp;
}

// u(p, lam) = (sqrt(E - lam|p|) chi_lam ; sqrt(E + lam|p|) chi_lam)   [ket]
template <class R>
HD void ext_u(const R* p, R m, int lam, cx<R>* w) {
  cx<R> chi[2];
  R wp, wm;
  helicity_chi(p, lam, chi);
  omegas(p, m, wp, wm);
  const R lo = lam > 0 ? wm : wp, hi = lam > 0 ? wp : wm;
  w[0] = lo * chi[0]; w[1] = lo * chi[1]; w[2] = hi * chi[0]; w[3] = hi * chi[1];
}

// v(p, lam) for an antiparticle of helicity lam:
// (sqrt(E + lam|p|) chi_{-lam} ; -sqrt(E - lam|p|) chi_{-lam})   [ket]
template <class R>
HD void ext_v(const R* p, R m, int lam, cx<R>* w) {
  cx<R> chi[2];
  R wp, wm;
  helicity_chi(p, -lam, chi);
  omegas(p, m, wp, wm);
  const R up = lam > 0 ? wp : wm, dn = lam > 0 ? wm : wp;
  w[0] = up * chi[0]; w[1] = up * chi[1]; w[2] = (-dn) * chi[0]; w[3] = (-dn) * chi[1];
}

// bar(psi) = psi^dagger gamma^0: swap the chiral halves and conjugate
template <class R>
HD void dirac_bar(const cx<R>* s, cx<R>* b) {
  b[0] = conjg(s[2]); b[1] = conjg(s[3]); b[2] = conjg(s[0]); b[3] = conjg(s[1]);
}

template <class R> HD void ext_ubar(const R* p, R m, int lam, cx<R>* w) { cx<R> t[4]; ext_u(p, m, lam, t); dirac_bar(t, w); }
template <class R> HD void ext_vbar(const R* p, R m, int lam, cx<R>* w) { cx<R> t[4]; ext_v(p, m, lam, t); dirac_bar(t, w); }

// Helicity polarisation vector eps(k, lam) = (-lam e1 - i e2)/sqrt2,
// e1 = (0, cos th cos ph, cos th sin ph, -sin th), e2 = (0, -sin ph, cos ph, 0);
// an outgoing gluon takes the complex conjugate.
template <class R>
HD void ext_eps(const R* k, int lam, bool outgoing, cx<R>* w) {
  const R px = k[1], py = k[2], pz = k[3];
  const R pt2 = px * px + py * py;
  const R ap = sqrt(pt2 + pz * pz);
  const R rt2 = R(0.70710678118654752440);
  R e1[3], e2[3];
  if (pt2 > R(0)) {
    const R pt = sqrt(pt2);
    const R ct = pz / ap, st = pt / ap, cp = px / pt, sp = py / pt;
    e1[0] = ct * cp; e1[1] = ct * sp; e1[2] = -st;
    e2[0] = -sp; e2[1] = cp; e2[2] = R(0);
  } else {
    e1[0] = pz >= R(0) ? R(1) : R(-1); e1[1] = R(0); e1[2] = R(0);
    e2[0] = R(0); e2[1] = R(1); e2[2] = R(0);
  }
  const R sgn = outgoing ? R(1) : R(-1);  // imaginary part flips for eps*
  w[0] = mk<R>(R(0), R(0));
  for (int j = 0; j < 3; ++j) w[j + 1] = mk<R>(-R(lam) * rt2 * e1[j], sgn * rt2 * e2[j]);
}

// ---------------------------------------------------------------------------
// vertices (raw: no couplings, no factors of i)
// ---------------------------------------------------------------------------
// three-gluon vertex contracted with two currents X (momentum kx) and Y (ky):
//   V3^rho = (X.Y)(kx - ky)^rho + Y^rho (kx + 2 ky).X - X^rho (2 kx + ky).Y
// (all momenta incoming; the third leg carries q = -(kx + ky)).
// (s scales the three scalar products, so that V3 / K^2 costs no extra pass)
template <class R>
HD void v3_scaled(const cx<R>* X, const R* kx, const cx<R>* Y, const R* ky, R s, cx<R>* out) {
  R a[4], b[4], d[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    d[m] = kx[m] - ky[m];
    a[m] = fmadd(R(2), ky[m], kx[m]);
    b[m] = fmadd(R(2), kx[m], ky[m]);
  }
  const cx<R> xy = s * mdot(X, Y), ax = s * mdot(a, X), by = s * mdot(b, Y);
#pragma unroll
  for (int m = 0; m < 4; ++m) out[m] = cfms(X[m], by, cfma(Y[m], ax, d[m] * xy));
}
template <class R>
HD void v3_raw(const cx<R>* X, const R* kx, const cx<R>* Y, const R* ky, cx<R>* out) {
  v3_scaled(X, kx, Y, ky, R(1), out);
}

// off-shell gluon from a three-gluon vertex: V3 / K^2   (phase i)
template <class R>
HD void g3_current(const cx<R>* X, const R* kx, const cx<R>* Y, const R* ky, R invK2, cx<R>* out) {
  v3_scaled(X, kx, Y, ky, invK2, out);
}

// Lorentz structure s of the four-gluon vertex contracted with X, Y, Z (legs a, b, c):
//   s=1 (f^abe f^cde): (X.Z) Y - (Y.Z) X
//   s=2 (f^ace f^bde): (X.Y) Z - (Y.Z) X
//   s=3 (f^ade f^bce): (X.Y) Z - (X.Z) Y
// (s scales the two scalar products, as in v3_scaled)
template <int S, class R>
HD void v4_scaled(const cx<R>* X, const cx<R>* Y, const cx<R>* Z, R s, cx<R>* out) {
  // out = u U - w W with (u, U, w, W) by structure
  const cx<R>* U = S == 1 ? Y : Z;
  const cx<R>* W = S == 3 ? Y : X;
  const cx<R> u = s * (S == 1 ? mdot(X, Z) : mdot(X, Y));
  const cx<R> w = s * (S == 3 ? mdot(X, Z) : mdot(Y, Z));
#pragma unroll
  for (int m = 0; m < 4; ++m) out[m] = cfms(w, W[m], cmul(u, U[m]));
}
template <int S, class R>
HD void v4_raw(const cx<R>* X, const cx<R>* Y, const cx<R>* Z, cx<R>* out) {
  v4_scaled<S>(X, Y, Z, R(1), out);
}

// off-shell gluon from a four-gluon structure: V4_s / K^2   (phase -1)
template <int S, class R>
HD void g4_current(const cx<R>* X, const cx<R>* Y, const cx<R>* Z, R invK2, cx<R>* out) {
  v4_scaled<S>(X, Y, Z, invK2, out);
}

// row spinor (a | b) times gamma.G, G contravariant:
//   (a|b) [[0, G.sigma], [G.sigmabar, 0]] = (b (G.sigmabar) | a (G.sigma))
template <class R>
HD void bra_gslash(const cx<R>* f, const cx<R>* G, cx<R>* o) {
  const cx<R> p03 = G[0] + G[3], m03 = G[0] - G[3];
  const cx<R> p12 = G[1] + times_i(G[2]), m12 = G[1] - times_i(G[2]);  // G1 +- i G2
  // G.sigmabar = [[G0+G3, G1-iG2], [G1+iG2, G0-G3]], G.sigma = [[G0-G3, -(G1-iG2)], [-(G1+iG2), G0+G3]]
  o[0] = cfma(f[2], p03, cmul(f[3], p12));
  o[1] = cfma(f[2], m12, cmul(f[3], m03));
  o[2] = cfms(f[1], p12, cmul(f[0], m03));
  o[3] = cfms(f[0], m12, cmul(f[1], p03));
}

// gamma.G times column spinor (l ; r) = (G.sigma r ; G.sigmabar l)
template <class R>
HD void gslash_ket(const cx<R>* G, const cx<R>* f, cx<R>* o) {
  const cx<R> p03 = G[0] + G[3], m03 = G[0] - G[3];
  const cx<R> p12 = G[1] + times_i(G[2]), m12 = G[1] - times_i(G[2]);
  o[0] = cfms(m12, f[3], cmul(m03, f[2]));
  o[1] = cfms(p12, f[2], cmul(p03, f[3]));
  o[2] = cfma(m12, f[1], cmul(p03, f[0]));
  o[3] = cfma(m03, f[1], cmul(p12, f[0]));
}

// row spinor times (qslash + m), q real
template <class R>
HD void bra_prop(const cx<R>* c, const R* q, R m, cx<R>* o) {
  // (c|d) [[m, q.sigma], [q.sigmabar, m]] = (m c + d q.sigmabar | c q.sigma + m d)
  // with q1 +- i q2 written out: c (q1 + i q2) = (c.r q1 - c.i q2, c.i q1 + c.r q2)
  const R p03 = q[0] + q[3], m03 = q[0] - q[3], q1 = q[1], q2 = q[2];
  o[0] = mk<R>(fmadd(m, c[0].r, fmadd(p03, c[2].r, fmadd(c[3].r, q1, -(c[3].i * q2)))),
               fmadd(m, c[0].i, fmadd(p03, c[2].i, fmadd(c[3].i, q1, c[3].r * q2))));
  o[1] = mk<R>(fmadd(m, c[1].r, fmadd(m03, c[3].r, fmadd(c[2].r, q1, c[2].i * q2))),
               fmadd(m, c[1].i, fmadd(m03, c[3].i, fmadd(c[2].i, q1, -(c[2].r * q2)))));
  o[2] = mk<R>(fmadd(m, c[2].r, fmadd(m03, c[0].r, fmadd(-c[1].r, q1, c[1].i * q2))),
               fmadd(m, c[2].i, fmadd(m03, c[0].i, fmadd(-c[1].i, q1, -(c[1].r * q2)))));
  o[3] = mk<R>(fmadd(m, c[3].r, fmadd(p03, c[1].r, fmadd(-c[0].r, q1, -(c[0].i * q2)))),
               fmadd(m, c[3].i, fmadd(p03, c[1].i, fmadd(-c[0].i, q1, c[0].r * q2))));
}

// (qslash + m) times column spinor, q real
template <class R>
HD void prop_ket(const R* q, R m, const cx<R>* c, cx<R>* o) {
  // [[m, q.sigma], [q.sigmabar, m]] (l ; r) = (m l + q.sigma r ; q.sigmabar l + m r)
  const R p03 = q[0] + q[3], m03 = q[0] - q[3], q1 = q[1], q2 = q[2];
  // -(q1 - i q2) c3 = (-q1 c3.r - q2 c3.i, -q1 c3.i + q2 c3.r)
  o[0] = mk<R>(fmadd(m, c[0].r, fmadd(m03, c[2].r, fmadd(-q1, c[3].r, -(q2 * c[3].i)))),
               fmadd(m, c[0].i, fmadd(m03, c[2].i, fmadd(-q1, c[3].i, q2 * c[3].r))));
  // -(q1 + i q2) c2 = (-q1 c2.r + q2 c2.i, -q1 c2.i - q2 c2.r)
  o[1] = mk<R>(fmadd(m, c[1].r, fmadd(p03, c[3].r, fmadd(-q1, c[2].r, q2 * c[2].i))),
               fmadd(m, c[1].i, fmadd(p03, c[3].i, fmadd(-q1, c[2].i, -(q2 * c[2].r)))));
  // (q1 - i q2) c1 = (q1 c1.r + q2 c1.i, q1 c1.i - q2 c1.r)
  o[2] = mk<R>(fmadd(m, c[2].r, fmadd(p03, c[0].r, fmadd(q1, c[1].r, q2 * c[1].i))),
               fmadd(m, c[2].i, fmadd(p03, c[0].i, fmadd(q1, c[1].i, -(q2 * c[1].r)))));
  // (q1 + i q2) c0 = (q1 c0.r - q2 c0.i, q1 c0.i + q2 c0.r)
  o[3] = mk<R>(fmadd(m, c[3].r, fmadd(m03, c[1].r, fmadd(q1, c[0].r, -(q2 * c[0].i)))),
               fmadd(m, c[3].i, fmadd(m03, c[1].i, fmadd(q1, c[0].i, q2 * c[0].r))));
}

// bra chain step: F (gamma.G) (qslash + m) / D       (phase +1)
template <class R>
HD void bra_step(const cx<R>* F, const cx<R>* G, const R* q, R m, cx<R> invD, cx<R>* out) {
  cx<R> t[4], u[4];
  bra_gslash(F, G, t);
  bra_prop(t, q, m, u);
#pragma unroll
  for (int j = 0; j < 4; ++j) out[j] = u[j] * invD;
}

// ket chain step: (qslash + m) (gamma.G) F / D       (phase +1)
template <class R>
HD void ket_step(const cx<R>* G, const cx<R>* F, const R* q, R m, cx<R> invD, cx<R>* out) {
  cx<R> t[4], u[4];
  gslash_ket(G, F, t);
  prop_ket(q, m, t, u);
#pragma unroll
  for (int j = 0; j < 4; ++j) out[j] = u[j] * invD;
}

// fermion-pair vector current j^mu = B gamma^mu K = a sigma^mu r + b sigmabar^mu l,
// B = (a|b), K = (l;r)
template <class R>
HD void pair_current(const cx<R>* B, const cx<R>* K, cx<R>* j) {
  // j0 = s + t, j3 = s - t with s = a1r1 + b2l2, t = a2r2 + b1l1 (each one chain)
  const cx<R> s = cfma(B[3], K[1], cmul(B[0], K[2])), t = cfma(B[2], K[0], cmul(B[1], K[3]));
  j[0] = s + t;
  j[3] = s - t;
  const cx<R> a1r2 = cmul(B[0], K[3]), a2r1 = cmul(B[1], K[2]), b1l2 = cmul(B[2], K[1]), b2l1 = cmul(B[3], K[0]);
  j[1] = (a1r2 + a2r1) - (b1l2 + b2l1);
  j[2] = times_i((a2r1 - a1r2) - (b2l1 - b1l2));
}

// chiral couplings: j^mu = B gamma^mu (cL P_L + cR P_R) K = cR a sigma^mu r + cL b sigmabar^mu l
template <class R>
HD void pair_current_lr(const cx<R>* B, const cx<R>* K, R cL, R cR, cx<R>* j) {
  const cx<R> a1r1 = B[0] * K[2], a2r2 = B[1] * K[3], a1r2 = B[0] * K[3], a2r1 = B[1] * K[2];
  const cx<R> b1l1 = B[2] * K[0], b2l2 = B[3] * K[1], b1l2 = B[2] * K[1], b2l1 = B[3] * K[0];
  j[0] = cR * (a1r1 + a2r2) + cL * (b1l1 + b2l2);
  j[1] = cR * (a1r2 + a2r1) - cL * (b1l2 + b2l1);
  j[2] = times_i(cR * (a2r1 - a1r2) - cL * (b2l1 - b1l2));
  j[3] = cR * (a1r1 - a2r2) - cL * (b1l1 - b2l2);
}

// closing kinds: PJ . G,  PJ . V3(X, Y) / K^2,  PJ . V4_s(X, Y, Z) / K^2
// (the in-place forms evaluate the block's root vertex and the gluon propagator that
// joins it to the quark line without storing the block current)
template <class R>
HD cx<R> close_dot(const cx<R>* PJ, const cx<R>* G) { return mdot(PJ, G); }

template <class R>
HD cx<R> close_v3(const cx<R>* PJ, const cx<R>* X, const R* kx, const cx<R>* Y, const R* ky, R invK2) {
  cx<R> v[4];
  v3_raw(X, kx, Y, ky, v);
  return invK2 * mdot(PJ, v);
}

template <int S, class R>
HD cx<R> close_v4(const cx<R>* PJ, const cx<R>* X, const cx<R>* Y, const cx<R>* Z, R invK2) {
  if (S == 1) return invK2 * cfms(mdot(Y, Z), mdot(X, PJ), cmul(mdot(X, Z), mdot(Y, PJ)));
  if (S == 2) return invK2 * cfms(mdot(Y, Z), mdot(X, PJ), cmul(mdot(X, Y), mdot(Z, PJ)));
  return invK2 * cfms(mdot(X, Z), mdot(Y, PJ), cmul(mdot(X, Y), mdot(Z, PJ)));
}

}  // namespace meb300
