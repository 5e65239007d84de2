/*
 * me_oracle.c -- plain, slow, FP64 CPU oracle for tree-level matrix elements |M|^2.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link or call this file:
 * only the tests, the smoke check and the CPU-baseline leg of the benchmark use it.
 * It shares no code, header, table or generator with the CUDA path.
 *
 * What it computes (the quantity the paper offloads, Section 2, Eq.-free text of
 * the abstract and Section 3: "matrix elements" for a batch of events):
 *
 *     me(p) = (1/IDEN) * sum_{all helicities h} sum_{all colours} |M(p, h, colours)|^2
 *
 * with IDEN = (initial spin states) x (initial colour states) x (identical final
 * gluons)!.  The paper gives no formulas; the physics follows published textbook
 * methods, each named where it is used:
 *
 *   * helicity spinors / polarisation vectors: the helicity basis of the HELAS
 *     library (Murayama, Watanabe, Hagiwara, KEK Report 91-11), written here in the
 *     chiral (Weyl) representation of Peskin & Schroeder (eqs. 3.25, 3.50-3.62);
 *   * Feynman rules in Feynman gauge (Peskin & Schroeder Fig. 16.7 with g -> -g);
 *   * colour decomposition of q qbar + n gluons into colour-ordered amplitudes
 *     (Mangano & Parke, Phys. Rep. 200 (1991) 301), evaluated here with the
 *     Berends-Giele recursion (Nucl. Phys. B306 (1988) 759);
 *   * colour matrix C_{st} = Tr(T^s (T^t)^dagger), evaluated exactly in rationals by
 *     the Fierz identity sum_a T^a_ij T^a_kl = (d_il d_kj - d_ij d_kl / N)/2.
 *
 * For e+ e- -> mu+ mu- the two s-channel diagrams (photon, Z) are written out with
 * explicit 4x4 gamma matrices.  For q qbar -> t tbar (a light quark of either beam; the
 * quark-initiated channel of p p -> t tbar) the one s-channel gluon diagram is written
 * out with explicit colour indices and explicit Gell-Mann matrices T^a = lambda^a / 2:
 * |M|^2 is summed over all 81 colour assignments, and the colour-flow amplitudes are the
 * coefficients of the amplitude on the two flow tensors (a 2 x 2 Gram system).  Its
 * one-jet crossings (q qbar -> t tbar g, q g -> t tbar q, qbar g -> t tbar qbar) are the
 * five Feynman diagrams of one light-quark line, the top line and one gluon, summed the
 * same way over all 648 colour assignments and projected onto four flow tensors.  The
 * two-jet channels with one light line (q qbar -> t tbar g g and crossings) are their 36
 * Feynman diagrams (38 terms), summed over all 5184 colour assignments and projected
 * onto 13 flow tensors.  The four-quark channels with two light flavours are the 7
 * diagrams of three fermion lines joined by gluons, summed over all 729 colour
 * assignments and projected onto the six colour-routing tensors; with one light flavour
 * the second pairing of the light quarks (their column ends exchanged) is added with the
 * sign -1 of exchanging identical fermions.
 *
 * Conventions shared with the product only through their published definitions:
 *   * momenta [nevt][npar][4] = (E, px, py, pz); particle order of the process string;
 *   * helicity index h in [0, 2^npar): particle i has helicity +1 if bit
 *     (npar-1-i) of h is set, else -1 (physical helicity of that particle);
 *   * colour-flow index: the lexicographic rank of the gluon permutation s in the
 *     string (T^{a_s1} ... T^{a_sn})_{i_t j_tbar}, gluons named by particle index;
 *   * selection: first index whose running sum exceeds r * total (strict);
 *     helicity weights |M_h|^2, colour weights w_i = sum_h |A_{h,i}|^2.
 *
 * Compile with -ffp-contract=off so that no FMA contraction changes the rounding.
 */
#define _USE_MATH_DEFINES
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cx;

#define NPROC 29
#define MAXPAR 7
#define MAXG 5
#define MAXCOL 120

typedef struct {
  double mZ, wZ, mt, wt, aEWM1, Gf, alphas;
  int zero_width_tchan;
} oracle_params;

/* roles of external particles */
enum { R_EBAR_IN, R_E_IN, R_MUBAR_OUT, R_MU_OUT, R_G_IN, R_G_OUT, R_T_OUT, R_TBAR_OUT, R_Q_IN, R_QB_IN,
       R_Q_OUT, R_QB_OUT, R_D_IN, R_DB_IN, R_D_OUT, R_DB_OUT };

/* kind: 0 e+ e- -> mu+ mu-; 1 g g -> t tbar + gluons (Berends-Giele); 2 q qbar -> t tbar
 * (explicit colour); 3 q qbar -> t tbar g and its crossings with one light quark line, a
 * top line and one gluon (explicit colour, five Feynman diagrams); 4 the same with two
 * gluons (explicit colour, 36 Feynman diagrams); 5 two light quark lines of different
 * flavours and the top line (explicit colour, 7 Feynman diagrams); 6 the same with one
 * light flavour (both pairings of the light quarks, 14 diagrams) */
typedef struct {
  const char* name;
  int npar;
  int ngluon;
  int iden;
  int role[MAXPAR];
  int kind;
  int ncol;
} proc_def;

static const proc_def PROCS[NPROC] = {
    {"e+ e- > mu+ mu-", 4, 0, 4, {R_EBAR_IN, R_E_IN, R_MUBAR_OUT, R_MU_OUT}, 0, 1},
    {"g g > t t~", 4, 2, 256, {R_G_IN, R_G_IN, R_T_OUT, R_TBAR_OUT}, 1, 2},
    {"g g > t t~ g", 5, 3, 256, {R_G_IN, R_G_IN, R_T_OUT, R_TBAR_OUT, R_G_OUT}, 1, 6},
    {"g g > t t~ g g", 6, 4, 512, {R_G_IN, R_G_IN, R_T_OUT, R_TBAR_OUT, R_G_OUT, R_G_OUT}, 1, 24},
    {"g g > t t~ g g g", 7, 5, 1536,
     {R_G_IN, R_G_IN, R_T_OUT, R_TBAR_OUT, R_G_OUT, R_G_OUT, R_G_OUT}, 1, 120},
    /* IDEN = 4 initial spin states x 9 initial colour states */
    {"u u~ > t t~", 4, 0, 36, {R_Q_IN, R_QB_IN, R_T_OUT, R_TBAR_OUT}, 2, 2},
    {"u~ u > t t~", 4, 0, 36, {R_QB_IN, R_Q_IN, R_T_OUT, R_TBAR_OUT}, 2, 2},
    /* one extra jet: IDEN = 4 x 9 (q qbar) or 4 x 3 x 8 (q g) initial states */
    {"u u~ > t t~ g", 5, 0, 36, {R_Q_IN, R_QB_IN, R_T_OUT, R_TBAR_OUT, R_G_OUT}, 3, 4},
    {"u~ u > t t~ g", 5, 0, 36, {R_QB_IN, R_Q_IN, R_T_OUT, R_TBAR_OUT, R_G_OUT}, 3, 4},
    {"u g > t t~ u", 5, 0, 96, {R_Q_IN, R_G_IN, R_T_OUT, R_TBAR_OUT, R_Q_OUT}, 3, 4},
    {"g u > t t~ u", 5, 0, 96, {R_G_IN, R_Q_IN, R_T_OUT, R_TBAR_OUT, R_Q_OUT}, 3, 4},
    {"u~ g > t t~ u~", 5, 0, 96, {R_QB_IN, R_G_IN, R_T_OUT, R_TBAR_OUT, R_QB_OUT}, 3, 4},
    {"g u~ > t t~ u~", 5, 0, 96, {R_G_IN, R_QB_IN, R_T_OUT, R_TBAR_OUT, R_QB_OUT}, 3, 4},
    /* two extra partons: IDEN = 4 x 9 x 2! (two final gluons), 4 x 3 x 8 (q g), 4 x 64 (g g) */
    {"u u~ > t t~ g g", 6, 0, 72, {R_Q_IN, R_QB_IN, R_T_OUT, R_TBAR_OUT, R_G_OUT, R_G_OUT}, 4, 13},
    {"u~ u > t t~ g g", 6, 0, 72, {R_QB_IN, R_Q_IN, R_T_OUT, R_TBAR_OUT, R_G_OUT, R_G_OUT}, 4, 13},
    {"u g > t t~ u g", 6, 0, 96, {R_Q_IN, R_G_IN, R_T_OUT, R_TBAR_OUT, R_Q_OUT, R_G_OUT}, 4, 13},
    {"g u > t t~ u g", 6, 0, 96, {R_G_IN, R_Q_IN, R_T_OUT, R_TBAR_OUT, R_Q_OUT, R_G_OUT}, 4, 13},
    {"u~ g > t t~ u~ g", 6, 0, 96, {R_QB_IN, R_G_IN, R_T_OUT, R_TBAR_OUT, R_QB_OUT, R_G_OUT}, 4, 13},
    {"g u~ > t t~ u~ g", 6, 0, 96, {R_G_IN, R_QB_IN, R_T_OUT, R_TBAR_OUT, R_QB_OUT, R_G_OUT}, 4, 13},
    {"g g > t t~ u u~", 6, 0, 256, {R_G_IN, R_G_IN, R_T_OUT, R_TBAR_OUT, R_Q_OUT, R_QB_OUT}, 4, 13},
    /* four quarks of two different light flavours: IDEN = 4 x 9 */
    {"u u~ > t t~ d d~", 6, 0, 36, {R_Q_IN, R_QB_IN, R_T_OUT, R_TBAR_OUT, R_D_OUT, R_DB_OUT}, 5, 6},
    {"u~ u > t t~ d d~", 6, 0, 36, {R_QB_IN, R_Q_IN, R_T_OUT, R_TBAR_OUT, R_D_OUT, R_DB_OUT}, 5, 6},
    {"u d > t t~ u d", 6, 0, 36, {R_Q_IN, R_D_IN, R_T_OUT, R_TBAR_OUT, R_Q_OUT, R_D_OUT}, 5, 6},
    {"u d~ > t t~ u d~", 6, 0, 36, {R_Q_IN, R_DB_IN, R_T_OUT, R_TBAR_OUT, R_Q_OUT, R_DB_OUT}, 5, 6},
    {"u~ d~ > t t~ u~ d~", 6, 0, 36, {R_QB_IN, R_DB_IN, R_T_OUT, R_TBAR_OUT, R_QB_OUT, R_DB_OUT}, 5, 6},
    /* four quarks of one light flavour: IDEN = 4 x 9 (x 2! for two identical final quarks) */
    {"u u > t t~ u u", 6, 0, 72, {R_Q_IN, R_Q_IN, R_T_OUT, R_TBAR_OUT, R_Q_OUT, R_Q_OUT}, 6, 6},
    {"u~ u~ > t t~ u~ u~", 6, 0, 72, {R_QB_IN, R_QB_IN, R_T_OUT, R_TBAR_OUT, R_QB_OUT, R_QB_OUT}, 6, 6},
    {"u u~ > t t~ u u~", 6, 0, 36, {R_Q_IN, R_QB_IN, R_T_OUT, R_TBAR_OUT, R_Q_OUT, R_QB_OUT}, 6, 6},
    {"u~ u > t t~ u u~", 6, 0, 36, {R_QB_IN, R_Q_IN, R_T_OUT, R_TBAR_OUT, R_Q_OUT, R_QB_OUT}, 6, 6},
};

static int factorial(int n) { return n <= 1 ? 1 : n * factorial(n - 1); }

int oracle_nproc(void) { return NPROC; }

int oracle_process_id(const char* name) {
  for (int i = 0; i < NPROC; ++i)
    if (strcmp(name, PROCS[i].name) == 0) return i;
  return -1;
}

int oracle_info(int proc, int* npar, int* ncomb, int* ncol, int* iden) {
  if (proc < 0 || proc >= NPROC) return -1;
  *npar = PROCS[proc].npar;
  *ncomb = 1 << PROCS[proc].npar;
  *ncol = PROCS[proc].ncol;
  *iden = PROCS[proc].iden;
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Exact rationals for the colour algebra                                     */
/* ------------------------------------------------------------------------- */
typedef struct { int64_t n, d; } rat;

static int64_t gcd64(int64_t a, int64_t b) {
  if (a < 0) a = -a;
  if (b < 0) b = -b;
  while (b) { int64_t t = a % b; a = b; b = t; }
  return a;
}
static rat rnorm(rat r) {
  if (r.n == 0) { r.d = 1; return r; }
  int64_t g = gcd64(r.n, r.d);
  r.n /= g; r.d /= g;
  if (r.d < 0) { r.n = -r.n; r.d = -r.d; }
  return r;
}
static rat radd(rat a, rat b) { rat r = {a.n * b.d + b.n * a.d, a.d * b.d}; return rnorm(r); }
static rat rmul(rat a, rat b) { rat r = {a.n * b.n, a.d * b.d}; return rnorm(r); }

#define NC 3
#define MAXWORDS 8
#define MAXLEN (2 * MAXG)

/* A product of traces Tr(w_0) Tr(w_1) ...; each word lists adjoint labels, and
 * every label occurs exactly twice in the whole product (summed over). */
typedef struct {
  int nw;
  int len[MAXWORDS];
  int a[MAXWORDS][MAXLEN];
} tprod;

static rat trace_value(const tprod* t) {
  /* a trace of a single generator vanishes */
  for (int w = 0; w < t->nw; ++w)
    if (t->len[w] == 1) { rat z = {0, 1}; return z; }
  int w0 = -1;
  for (int w = 0; w < t->nw; ++w)
    if (t->len[w] > 0) { w0 = w; break; }
  if (w0 < 0) { /* every trace is Tr(1) = N */
    rat r = {1, 1};
    for (int w = 0; w < t->nw; ++w) { rat n = {NC, 1}; r = rmul(r, n); }
    return r;
  }
  int lab = t->a[w0][0];
  /* partner occurrence */
  int pw = -1, pi = -1;
  for (int i = 1; i < t->len[w0]; ++i)
    if (t->a[w0][i] == lab) { pw = w0; pi = i; break; }
  if (pw < 0) {
    for (int w = w0 + 1; w < t->nw && pw < 0; ++w)
      for (int i = 0; i < t->len[w]; ++i)
        if (t->a[w][i] == lab) { pw = w; pi = i; break; }
  }
  rat half = {1, 2}, mhalfn = {-1, 2 * NC};
  tprod t1, t2;
  if (pw == w0) {
    /* Tr(T^a B T^a C) = 1/2 [Tr(C) Tr(B) - Tr(B C)/N], A empty since a is first */
    int lenB = pi - 1, lenC = t->len[w0] - pi - 1;
    const int* B = &t->a[w0][1];
    const int* Cc = &t->a[w0][pi + 1];
    t1 = *t;
    t1.len[w0] = lenC;
    memcpy(t1.a[w0], Cc, sizeof(int) * lenC);
    t1.len[t1.nw] = lenB;
    memcpy(t1.a[t1.nw], B, sizeof(int) * lenB);
    t1.nw += 1;
    t2 = *t;
    t2.len[w0] = lenB + lenC;
    memcpy(t2.a[w0], B, sizeof(int) * lenB);
    memcpy(t2.a[w0] + lenB, Cc, sizeof(int) * lenC);
  } else {
    /* Tr(T^a X) Tr(T^a Y) = 1/2 [Tr(X Y) - Tr(X) Tr(Y)/N], with X = rest of w0 and
     * Y = rest of pw read cyclically after the label */
    int X[MAXLEN], Y[MAXLEN], lx = t->len[w0] - 1, ly = t->len[pw] - 1;
    memcpy(X, &t->a[w0][1], sizeof(int) * lx);
    for (int k = 0; k < ly; ++k) Y[k] = t->a[pw][(pi + 1 + k) % t->len[pw]];
    /* term 1: merge into w0, delete pw */
    t1 = *t;
    t1.len[w0] = lx + ly;
    memcpy(t1.a[w0], X, sizeof(int) * lx);
    memcpy(t1.a[w0] + lx, Y, sizeof(int) * ly);
    for (int w = pw; w + 1 < t1.nw; ++w) {
      t1.len[w] = t1.len[w + 1];
      memcpy(t1.a[w], t1.a[w + 1], sizeof(int) * MAXLEN);
    }
    t1.nw -= 1;
    t2 = *t;
    t2.len[w0] = lx;
    memcpy(t2.a[w0], X, sizeof(int) * lx);
    t2.len[pw] = ly;
    memcpy(t2.a[pw], Y, sizeof(int) * ly);
  }
  return radd(rmul(half, trace_value(&t1)), rmul(mhalfn, trace_value(&t2)));
}

/* permutation of {0..n-1} with lexicographic rank r */
static void perm_unrank(int n, int r, int* out) {
  int pool[MAXG];
  for (int i = 0; i < n; ++i) pool[i] = i;
  for (int i = 0; i < n; ++i) {
    int f = factorial(n - 1 - i);
    int k = r / f;
    r %= f;
    out[i] = pool[k];
    for (int j = k; j < n - 1 - i; ++j) pool[j] = pool[j + 1];
  }
}

/* C_{st} = Tr(T^{s_1}...T^{s_n} T^{t_n}...T^{t_1}) as num[ncol*ncol] / den[ncol*ncol]. */
static double qq_flow_tensor(int n, int i, int j, int k, int l);

static void qg_colour_init(void);
static void qg_gram(cx G[4][4]);
static void q4_colour_init(void);
static void q4_gram(cx* G);
static void q5_colour_init(void);
static void q5_gram(cx* G);

int oracle_colour_matrix_exact(int proc, int64_t* num, int64_t* den) {
  if (proc < 0 || proc >= NPROC) return -1;
  if (PROCS[proc].kind == 5 || PROCS[proc].kind == 6) {
    /* C_nm = number of colour assignments on which flows n and m are both 1 */
    cx G[36];
    q5_colour_init();
    q5_gram(G);
    for (int i = 0; i < 36; ++i) {
      num[i] = (int64_t)llround(creal(G[i]));
      den[i] = 1;
    }
    return 0;
  }
  if (PROCS[proc].kind == 4) {
    /* C_nm = sum over all colour assignments of conj(c_n) c_m, explicit Gell-Mann sums;
     * the entries are multiples of 1/3 */
    cx G[13 * 13];
    q4_colour_init();
    q4_gram(G);
    for (int i = 0; i < 13 * 13; ++i) {
      double r = round(creal(G[i]) * 3.0);
      if (fabs(creal(G[i]) * 3.0 - r) > 1e-8 || fabs(cimag(G[i])) > 1e-8) return -1;
      int64_t nn = (int64_t)r, dd = 3;
      if (nn % 3 == 0) { nn /= 3; dd = 1; }
      num[i] = nn;
      den[i] = dd;
    }
    return 0;
  }
  if (PROCS[proc].kind == 3) {
    /* C_nm = sum over all colour assignments of conj(c_n) c_m, with explicit Gell-Mann
     * matrices; the sums are integers (traces of pairs of generators) */
    cx G[4][4];
    qg_colour_init();
    qg_gram(G);
    for (int n = 0; n < 4; ++n)
      for (int m = 0; m < 4; ++m) {
        double r = round(creal(G[n][m]));
        if (fabs(creal(G[n][m]) - r) > 1e-9 || fabs(cimag(G[n][m])) > 1e-9) return -1;
        num[n * 4 + m] = (int64_t)r;
        den[n * 4 + m] = 1;
      }
    return 0;
  }
  if (PROCS[proc].kind == 2) {
    /* C_nm = sum over all colour indices of c_n c_m (the flow tensors are real, 0 or 1) */
    for (int n = 0; n < 2; ++n)
      for (int m = 0; m < 2; ++m) {
        int64_t c = 0;
        for (int i = 0; i < NC; ++i)
          for (int j = 0; j < NC; ++j)
            for (int k = 0; k < NC; ++k)
              for (int l = 0; l < NC; ++l) c += (int64_t)(qq_flow_tensor(n, i, j, k, l) * qq_flow_tensor(m, i, j, k, l));
        num[n * 2 + m] = c;
        den[n * 2 + m] = 1;
      }
    return 0;
  }
  int n = PROCS[proc].ngluon;
  if (n == 0) { num[0] = 1; den[0] = 1; return 0; }
  int ncol = factorial(n);
  for (int s = 0; s < ncol; ++s) {
    int ps[MAXG];
    perm_unrank(n, s, ps);
    for (int t = 0; t < ncol; ++t) {
      int pt[MAXG];
      perm_unrank(n, t, pt);
      tprod tp;
      memset(&tp, 0, sizeof tp);
      tp.nw = 1;
      tp.len[0] = 2 * n;
      for (int i = 0; i < n; ++i) {
        tp.a[0][i] = ps[i];
        tp.a[0][2 * n - 1 - i] = pt[i];
      }
      rat v = trace_value(&tp);
      num[s * ncol + t] = v.n;
      den[s * ncol + t] = v.d;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Dirac algebra (chiral representation)                                     */
/* ------------------------------------------------------------------------- */
static cx GAM[4][4][4]; /* GAM[mu][row][col] = gamma^mu */
static int gam_ready = 0;

static void gamma_init(void) {
  if (gam_ready) return;
  memset(GAM, 0, sizeof GAM);
  /* gamma^mu = [[0, sigma^mu], [sigmabar^mu, 0]], sigma = (1, s1, s2, s3),
   * sigmabar = (1, -s1, -s2, -s3) */
  cx pauli[4][2][2] = {{{1, 0}, {0, 1}},
                       {{0, 1}, {1, 0}},
                       {{0, -I}, {I, 0}},
                       {{1, 0}, {0, -1}}};
  for (int mu = 0; mu < 4; ++mu)
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        GAM[mu][i][2 + j] = pauli[mu][i][j];
        GAM[mu][2 + i][j] = (mu == 0 ? 1.0 : -1.0) * pauli[mu][i][j];
      }
  gam_ready = 1;
}

static cx mdot_c(const cx* a, const cx* b) { return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3]; }
static double mdot_r(const double* a, const double* b) { return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3]; }

/* slash(a) = gamma^mu a_mu = gamma^0 a^0 - gamma^k a^k */
static void slash(const cx* a, cx M[4][4]) {
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j)
      M[i][j] = GAM[0][i][j] * a[0] - GAM[1][i][j] * a[1] - GAM[2][i][j] * a[2] - GAM[3][i][j] * a[3];
}

/* row vector times matrix */
static void bra_mat(const cx* b, cx M[4][4], cx* out) {
  for (int j = 0; j < 4; ++j) {
    cx s = 0;
    for (int i = 0; i < 4; ++i) s += b[i] * M[i][j];
    out[j] = s;
  }
}
static cx bra_ket(const cx* b, const cx* k) { return b[0] * k[0] + b[1] * k[1] + b[2] * k[2] + b[3] * k[3]; }

/* Two-component helicity eigenvectors of sigma.p_hat with eigenvalue lam. */
static void xi_hel(const double* p, int lam, cx* xi) {
  double px = p[1], py = p[2], pz = p[3];
  double ap = sqrt(px * px + py * py + pz * pz);
  if (ap == 0.0) {
    xi[0] = lam > 0 ? 1 : 0;
    xi[1] = lam > 0 ? 0 : 1;
    return;
  }
  if (pz >= 0) {
    double nrm = 1.0 / sqrt(2.0 * ap * (ap + pz));
    if (lam > 0) { xi[0] = (ap + pz) * nrm; xi[1] = (px + I * py) * nrm; }
    else { xi[0] = (-px + I * py) * nrm; xi[1] = (ap + pz) * nrm; }
  } else {
    double nrm = 1.0 / sqrt(2.0 * ap * (ap - pz));
    if (lam > 0) { xi[0] = (px - I * py) * nrm; xi[1] = (ap - pz) * nrm; }
    else { xi[0] = (pz - ap) * nrm; xi[1] = (px + I * py) * nrm; }
  }
}

/* sqrt(E - lam|p|) and sqrt(E + lam|p|) without cancellation */
static void omega(const double* p, double m, int lam, double* wminus, double* wplus) {
  double ap = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
  double E = p[0];
  double big = sqrt(E + ap);
  double small = (m == 0.0) ? 0.0 : m / big; /* sqrt(E-|p|) = m / sqrt(E+|p|) */
  if (lam > 0) { *wminus = small; *wplus = big; }
  else { *wminus = big; *wplus = small; }
}

/* u(p, lam) = (sqrt(p.sigma) xi, sqrt(p.sigmabar) xi) with xi the helicity state */
static void spinor_u(const double* p, double m, int lam, cx* u) {
  cx xi[2];
  double wm, wp;
  xi_hel(p, lam, xi);
  omega(p, m, lam, &wm, &wp);
  u[0] = wm * xi[0]; u[1] = wm * xi[1];
  u[2] = wp * xi[0]; u[3] = wp * xi[1];
}

/* v(p, lam) for an antiparticle of physical helicity lam:
 * (sqrt(p.sigma) eta, -sqrt(p.sigmabar) eta), eta = xi_{-lam} */
static void spinor_v(const double* p, double m, int lam, cx* v) {
  cx eta[2];
  double wm, wp; /* sqrt(E - (-lam)|p|), sqrt(E + (-lam)|p|) */
  xi_hel(p, -lam, eta);
  omega(p, m, -lam, &wm, &wp);
  v[0] = wm * eta[0]; v[1] = wm * eta[1];
  v[2] = -wp * eta[0]; v[3] = -wp * eta[1];
}

/* psibar = psi^dagger gamma^0 */
static void dirac_bar(const cx* s, cx* b) {
  b[0] = conj(s[2]); b[1] = conj(s[3]); b[2] = conj(s[0]); b[3] = conj(s[1]);
}

/* helicity polarisation vector eps^mu(k, lam) = (-lam e1 - i e2)/sqrt(2) with
 * e1 = (0, cos th cos ph, cos th sin ph, -sin th), e2 = (0, -sin ph, cos ph, 0) */
static void polvec(const double* k, int lam, cx* e) {
  double px = k[1], py = k[2], pz = k[3];
  double ap = sqrt(px * px + py * py + pz * pz);
  double pt = sqrt(px * px + py * py);
  double e1[4], e2[4];
  if (pt > 0.0) {
    double ct = pz / ap, st = pt / ap, cp = px / pt, sp = py / pt;
    e1[0] = 0; e1[1] = ct * cp; e1[2] = ct * sp; e1[3] = -st;
    e2[0] = 0; e2[1] = -sp; e2[2] = cp; e2[3] = 0;
  } else {
    double ct = pz >= 0 ? 1.0 : -1.0;
    e1[0] = 0; e1[1] = ct; e1[2] = 0; e1[3] = 0;
    e2[0] = 0; e2[1] = 0; e2[2] = 1; e2[3] = 0;
  }
  for (int mu = 0; mu < 4; ++mu) e[mu] = (-lam * e1[mu] - I * e2[mu]) / sqrt(2.0);
}

/* ------------------------------------------------------------------------- */
/* Standard-model parameters                                                  */
/* ------------------------------------------------------------------------- */
typedef struct {
  double ee;           /* electric charge e = sqrt(4 pi alpha) */
  double sw2, sw, cw, mW;
  double gZ_L, gZ_R;   /* Z couplings of charged leptons in units of e */
} sm_derived;

static void sm_derive(const oracle_params* p, sm_derived* d) {
  double alpha = 1.0 / p->aEWM1;
  d->ee = sqrt(4.0 * M_PI * alpha);
  /* W mass from (alpha, G_F, m_Z): m_W^2 = mZ^2/2 + sqrt(mZ^4/4 - pi alpha mZ^2/(sqrt2 G_F)) */
  double mz2 = p->mZ * p->mZ;
  d->mW = sqrt(mz2 / 2.0 + sqrt(mz2 * mz2 / 4.0 - M_PI * alpha * mz2 / (sqrt(2.0) * p->Gf)));
  d->sw2 = 1.0 - d->mW * d->mW / mz2;
  d->sw = sqrt(d->sw2);
  d->cw = sqrt(1.0 - d->sw2);
  /* g = (T3 - Q sw^2)/(sw cw) for the left-handed, -Q sw^2/(sw cw) for the right-handed */
  double T3 = -0.5, Q = -1.0;
  d->gZ_L = (T3 - Q * d->sw2) / (d->sw * d->cw);
  d->gZ_R = (-Q * d->sw2) / (d->sw * d->cw);
}

int oracle_sm_derived(const oracle_params* p, double* out5) {
  sm_derived d;
  sm_derive(p, &d);
  out5[0] = d.ee; out5[1] = d.sw2; out5[2] = d.mW; out5[3] = d.gZ_L; out5[4] = d.gZ_R;
  return 0;
}

/* ------------------------------------------------------------------------- */
/* e+ e- -> mu+ mu- : photon and Z in the s channel                           */
/* ------------------------------------------------------------------------- */
/* current b gamma^mu (cL P_L + cR P_R) k, with P_L = diag(1,1,0,0) here */
static void vector_current(const cx* b, const cx* k, cx cL, cx cR, cx* j) {
  cx kc[4] = {cL * k[0], cL * k[1], cR * k[2], cR * k[3]};
  for (int mu = 0; mu < 4; ++mu) {
    cx s = 0;
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 4; ++c) s += b[r] * GAM[mu][r][c] * kc[c];
    j[mu] = s;
  }
}

static cx amp_eemumu(const double* mom, const int* lam, const oracle_params* par, const sm_derived* sm) {
  const double *p1 = mom, *p2 = mom + 4, *p3 = mom + 8, *p4 = mom + 12;
  cx v1[4], b1[4], u2[4], v3[4], u4[4], b4[4];
  spinor_v(p1, 0.0, lam[0], v1);  dirac_bar(v1, b1); /* incoming e+ : vbar */
  spinor_u(p2, 0.0, lam[1], u2);                       /* incoming e- : u    */
  spinor_v(p3, 0.0, lam[2], v3);                       /* outgoing mu+: v    */
  spinor_u(p4, 0.0, lam[3], u4);  dirac_bar(u4, b4);   /* outgoing mu-: ubar */
  double P[4] = {p1[0] + p2[0], p1[1] + p2[1], p1[2] + p2[2], p1[3] + p2[3]};
  double s = mdot_r(P, P);
  cx ee = sm->ee;
  cx total = 0;
  /* photon: vertex -i e Q gamma^mu, Q = -1 for e and mu; propagator -i g_{mu nu}/s */
  {
    cx je[4], jm[4];
    vector_current(b1, u2, -1.0, -1.0, je);
    vector_current(b4, v3, -1.0, -1.0, jm);
    total += (-I * ee) * (-I * ee) * (-I / s) * mdot_c(je, jm);
  }
  /* Z: vertex -i e gamma^mu (gL P_L + gR P_R); propagator -i g_{mu nu}/(s - mZ^2 + i mZ wZ)
   * (the k_mu k_nu part vanishes against the massless currents) */
  {
    cx je[4], jm[4];
    vector_current(b1, u2, sm->gZ_L, sm->gZ_R, je);
    vector_current(b4, v3, sm->gZ_L, sm->gZ_R, jm);
    cx den = s - par->mZ * par->mZ + I * par->mZ * par->wZ;
    total += (-I * ee) * (-I * ee) * (-I / den) * mdot_c(je, jm);
  }
  return total;
}

/* ------------------------------------------------------------------------- */
/* g g -> t t~ + n gluons : Berends-Giele colour-ordered recursion            */
/* ------------------------------------------------------------------------- */
/* colour-ordered three-gluon vertex contracted with two currents (legs in order
 * 1, 2; all momenta incoming, third momentum q = -(k1 + k2)):
 *   V^rho = (J1.J2)(k1-k2)^rho + J2^rho (k2-q).J1 + J1^rho (q-k1).J2
 * which is g^{mu nu}(k-p)^rho + g^{nu rho}(p-q)^mu + g^{rho mu}(q-k)^nu
 * contracted with J1_mu J2_nu. */
static void v3(const double* k1, const cx* J1, const double* k2, const cx* J2, cx* out) {
  double q[4], d12[4], a[4], b[4];
  for (int m = 0; m < 4; ++m) {
    q[m] = -(k1[m] + k2[m]);
    d12[m] = k1[m] - k2[m];
    a[m] = k2[m] - q[m];
    b[m] = q[m] - k1[m];
  }
  cx j12 = mdot_c(J1, J2);
  cx aj1 = a[0] * J1[0] - a[1] * J1[1] - a[2] * J1[2] - a[3] * J1[3];
  cx bj2 = b[0] * J2[0] - b[1] * J2[1] - b[2] * J2[2] - b[3] * J2[3];
  for (int m = 0; m < 4; ++m) out[m] = j12 * d12[m] + J2[m] * aj1 + J1[m] * bj2;
}

/* colour-ordered four-gluon vertex [2 g^{mu rho} g^{nu sigma} - g^{mu nu} g^{rho sigma}
 * - g^{mu sigma} g^{nu rho}] contracted with J1_mu J2_nu J3_rho */
static void v4(const cx* J1, const cx* J2, const cx* J3, cx* out) {
  cx d13 = mdot_c(J1, J3), d12 = mdot_c(J1, J2), d23 = mdot_c(J2, J3);
  for (int m = 0; m < 4; ++m) out[m] = 2.0 * d13 * J2[m] - d12 * J3[m] - d23 * J1[m];
}

/* Is the propagator whose momentum is the sum over 'mask' (bit i = particle i) in the
 * t channel, i.e. does it separate the two incoming particles (0 and 1)? */
static int is_tchannel(unsigned mask) {
  int a = (mask >> 0) & 1, b = (mask >> 1) & 1;
  return a != b;
}

typedef struct {
  cx eps[MAXG][4];   /* gluon polarisation (incoming: eps, outgoing: eps*) */
  double kin[MAXG][4];/* incoming momentum of each gluon */
  int pidx[MAXG];    /* particle index of each gluon */
  cx ubar_t[4];      /* outgoing top: ubar(p_t) */
  cx v_tb[4];        /* outgoing antitop: v(p_tbar) */
  double pt[4];      /* top momentum */
  int it;            /* particle index of the top */
} qcd_ext;

/* Propagator invariants in quadruple precision.  A propagator's momentum is a sum of
 * external momenta; when that sum is nearly light-like (a gluon almost collinear with a
 * beam or with another gluon) the plain FP64 square cancels most of its digits.  Each
 * invariant is therefore formed from the FP64 inputs in __float128 (113-bit
 * significand): the sums of a few doubles are exact there, each square rounds at
 * 2^-113 of the summed energy squared, so even an invariant 1e10 times smaller than
 * that keeps ~80 correct bits before its single rounding to FP64.  The invariants
 * depend only on the kinematics, so they are formed once per event, tabulated by the
 * set of external particles whose momenta they sum (bit i = particle i), and every
 * other operation of the oracle stays in FP64. */
#if !defined(__SIZEOF_FLOAT128__)
#error "the oracle's propagator invariants need the __float128 type (gcc on x86-64 or aarch64)"
#endif
typedef __float128 quad;
_Static_assert(sizeof(quad) == 16, "__float128 must be the IEEE binary128 format");

typedef struct {
  double gsq[1 << MAXPAR];  /* K^2, K = sum of the incoming momenta of the gluons in 'mask' */
  double tden[1 << MAXPAR]; /* q^2 - mt^2, q = p_t - K(gluons in 'mask'), the top-line propagator */
} invariants;

static quad msq_q(const quad* k) { return k[0] * k[0] - k[1] * k[1] - k[2] * k[2] - k[3] * k[3]; }

/* fills inv for every subset 'mask' of the gluons of process pd at momenta p
 * (incoming gluons carry +p, outgoing -p) */
static void event_invariants(const proc_def* pd, const double* p, double mt, invariants* inv) {
  int npar = pd->npar, it = -1;
  unsigned gl = 0;
  for (int i = 0; i < npar; ++i) {
    if (pd->role[i] == R_G_IN || pd->role[i] == R_G_OUT) gl |= 1u << i;
    if (pd->role[i] == R_T_OUT) it = i;
  }
  for (unsigned mask = 0; mask < (1u << npar); ++mask) {
    inv->gsq[mask] = 0.0;
    inv->tden[mask] = 0.0;
    if ((mask & ~gl) || it < 0) continue;
    quad K[4] = {0, 0, 0, 0};
    for (int i = 0; i < npar; ++i)
      if (mask >> i & 1)
        for (int m = 0; m < 4; ++m) K[m] += (pd->role[i] == R_G_IN) ? (quad)p[4 * i + m] : -(quad)p[4 * i + m];
    quad q[4];
    for (int m = 0; m < 4; ++m) q[m] = (quad)p[4 * it + m] - K[m];
    inv->gsq[mask] = (double)msq_q(K);
    inv->tden[mask] = (double)(msq_q(q) - (quad)mt * (quad)mt);
  }
}

/* colour-ordered amplitude A(sigma) for gluons in the order sigma (gluon slots) */
static cx amp_ordered(const qcd_ext* x, const invariants* inv, int n, const int* sigma, double gs, double mt,
                      double wt, int zwt) {
  cx J[MAXG][MAXG][4];
  double K[MAXG][MAXG][4];
  unsigned M[MAXG][MAXG];
  for (int len = 1; len <= n; ++len) {
    for (int i = 0; i + len - 1 < n; ++i) {
      int j = i + len - 1;
      if (len == 1) {
        for (int m = 0; m < 4; ++m) {
          J[i][i][m] = x->eps[sigma[i]][m];
          K[i][i][m] = x->kin[sigma[i]][m];
        }
        M[i][i] = 1u << x->pidx[sigma[i]];
        continue;
      }
      for (int m = 0; m < 4; ++m) K[i][j][m] = K[i][i][m] + K[i + 1][j][m];
      M[i][j] = M[i][i] | M[i + 1][j];
      cx cur[4] = {0, 0, 0, 0}, t[4];
      for (int k = i; k < j; ++k) {
        v3(K[i][k], J[i][k], K[k + 1][j], J[k + 1][j], t);
        for (int m = 0; m < 4; ++m) cur[m] += I * gs * t[m];
      }
      for (int k = i; k < j; ++k)
        for (int l = k + 1; l < j; ++l) {
          v4(J[i][k], J[k + 1][l], J[l + 1][j], t);
          for (int m = 0; m < 4; ++m) cur[m] += I * gs * gs * t[m];
        }
      double P2 = inv->gsq[M[i][j]];
      for (int m = 0; m < 4; ++m) J[i][j][m] = (-I / P2) * cur[m];
    }
  }
  /* quark line: ubar(t) [-i gs J(B1)-slash] S [-i gs J(B2)-slash] ... v(tbar) */
  cx U[MAXG][4];
  for (int m = 0; m < 4; ++m) U[0][m] = x->ubar_t[m];
  cx A = 0;
  for (int j = 1; j <= n; ++j) {
    cx acc[4] = {0, 0, 0, 0};
    for (int i = 0; i < j; ++i) {
      cx G[4][4], tmp[4], Jv[4];
      for (int m = 0; m < 4; ++m) Jv[m] = -I * gs * J[i][j - 1][m];
      slash(Jv, G);
      bra_mat(U[i], G, tmp);
      for (int m = 0; m < 4; ++m) acc[m] += tmp[m];
    }
    if (j == n) {
      A = bra_ket(acc, x->v_tb);
    } else {
      /* propagator i(q-slash + m)/(q^2 - m^2 + i m w) with q = p_t - K(first j gluons) */
      double q[4];
      for (int m = 0; m < 4; ++m) q[m] = x->pt[m] - K[0][j - 1][m];
      unsigned mask = M[0][j - 1] | (1u << x->it);
      double w = (zwt && is_tchannel(mask)) ? 0.0 : wt;
      cx den = inv->tden[M[0][j - 1]] + I * mt * w;
      cx qc[4] = {q[0], q[1], q[2], q[3]}, S[4][4];
      slash(qc, S);
      for (int r = 0; r < 4; ++r) S[r][r] += mt;
      cx tmp[4];
      bra_mat(acc, S, tmp);
      for (int m = 0; m < 4; ++m) U[j][m] = (I / den) * tmp[m];
    }
  }
  return A;
}

/* ------------------------------------------------------------------------- */
/* q qbar -> t tbar : one s-channel gluon, explicit colour                    */
/* ------------------------------------------------------------------------- */
static cx TGM[8][NC][NC]; /* T^a = lambda^a / 2 (Gell-Mann) */
static int tgm_ready = 0;

static void tgm_init(void) {
  if (tgm_ready) return;
  memset(TGM, 0, sizeof TGM);
  TGM[0][0][1] = TGM[0][1][0] = 0.5;
  TGM[1][0][1] = -0.5 * I; TGM[1][1][0] = 0.5 * I;
  TGM[2][0][0] = 0.5; TGM[2][1][1] = -0.5;
  TGM[3][0][2] = TGM[3][2][0] = 0.5;
  TGM[4][0][2] = -0.5 * I; TGM[4][2][0] = 0.5 * I;
  TGM[5][1][2] = TGM[5][2][1] = 0.5;
  TGM[6][1][2] = -0.5 * I; TGM[6][2][1] = 0.5 * I;
  TGM[7][0][0] = TGM[7][1][1] = 0.5 / sqrt(3.0); TGM[7][2][2] = -1.0 / sqrt(3.0);
  tgm_ready = 1;
}

/* flow tensors of q(i) qbar(j) -> t(k) tbar(l): c_0 = d_ki d_jl (the top takes the
 * quark's colour, the antitop the antiquark's), c_1 = d_ji d_kl */
static double qq_flow_tensor(int n, int i, int j, int k, int l) {
  return n == 0 ? (double)(k == i && j == l) : (double)(j == i && k == l);
}

/* colour-stripped amplitude A with M(i,j,k,l) = A sum_a T^a_{ji} T^a_{kl}:
 *   [vbar(p_qb) (-i gs gamma^mu T^a) u(p_q)] (-i g_{mu nu} / s) [ubar(p_t) (-i gs gamma^nu T^a) v(p_tb)] */
static cx amp_qqbar_tt(const double* mom, const int* lam, const proc_def* pd, double gs, double mt) {
  int iq = -1, iqb = -1, it = -1, itb = -1;
  for (int i = 0; i < pd->npar; ++i) {
    if (pd->role[i] == R_Q_IN) iq = i;
    if (pd->role[i] == R_QB_IN) iqb = i;
    if (pd->role[i] == R_T_OUT) it = i;
    if (pd->role[i] == R_TBAR_OUT) itb = i;
  }
  cx u[4], v[4], vb[4], ut[4], ubt[4], vt[4], lq[4], lt[4];
  spinor_u(mom + 4 * iq, 0.0, lam[iq], u);
  spinor_v(mom + 4 * iqb, 0.0, lam[iqb], v);
  dirac_bar(v, vb);
  spinor_u(mom + 4 * it, mt, lam[it], ut);
  dirac_bar(ut, ubt);
  spinor_v(mom + 4 * itb, mt, lam[itb], vt);
  vector_current(vb, u, 1.0, 1.0, lq);
  vector_current(ubt, vt, 1.0, 1.0, lt);
  double P[4];
  for (int m = 0; m < 4; ++m) P[m] = mom[4 * iq + m] + mom[4 * iqb + m];
  double s = mdot_r(P, P);
  return (-I * gs) * (-I * gs) * (-I / s) * mdot_c(lq, lt);
}

/* explicit colour sum of |M|^2 and the flow amplitudes J (M = sum_n J_n c_n): the
 * projections P_n = sum c_n M over all indices, then J = G^{-1} P with the Gram matrix
 * G_nm = sum c_n c_m */
static double qq_colour_sum(cx A, cx* J) {
  double m2 = 0;
  cx P[2] = {0, 0};
  double G[2][2] = {{0, 0}, {0, 0}};
  for (int i = 0; i < NC; ++i)
    for (int j = 0; j < NC; ++j)
      for (int k = 0; k < NC; ++k)
        for (int l = 0; l < NC; ++l) {
          cx col = 0;
          for (int a = 0; a < 8; ++a) col += TGM[a][j][i] * TGM[a][k][l];
          cx M = A * col;
          m2 += creal(M) * creal(M) + cimag(M) * cimag(M);
          for (int n = 0; n < 2; ++n) {
            P[n] += qq_flow_tensor(n, i, j, k, l) * M;
            for (int m = 0; m < 2; ++m) G[n][m] += qq_flow_tensor(n, i, j, k, l) * qq_flow_tensor(m, i, j, k, l);
          }
        }
  double det = G[0][0] * G[1][1] - G[0][1] * G[1][0];
  J[0] = (G[1][1] * P[0] - G[0][1] * P[1]) / det;
  J[1] = (G[0][0] * P[1] - G[1][0] * P[0]) / det;
  return m2;
}

/* ------------------------------------------------------------------------- */
/* q qbar -> t tbar g and its crossings: five Feynman diagrams, explicit colour */
/* ------------------------------------------------------------------------- */
/* The process has a light-quark line (its row end B_L -- vbar of an incoming antiquark
 * or ubar of an outgoing quark -- and its column end K_L -- u of an incoming quark or v
 * of an outgoing antiquark), the top line (ubar(p_t) ... v(p_tbar)) and one gluon of
 * colour a.  With the rules of the gg processes (quark-gluon vertex -i g_s gamma^mu T^a,
 * fermion propagator i(qslash + m)/(q^2 - m^2 + i m w) with q along the fermion arrow,
 * gluon propagator -i g_{mu nu}/K^2, three-gluon vertex -g_s f^{abc} V^{mu nu rho}(k1,
 * k2, k3) with all momenta incoming) the diagrams are, with L = B_L gamma K_L and
 * H = ubar gamma v:
 *   D1  gluon on the light line next to K_L:  i g^3 [B_L gamma^mu q1slash epsslash K_L]
 *       H_mu / (q1^2 s_H),       colour (T^b T^a)_{B_L K_L} T^b_{t tbar}
 *   D2  next to B_L:                          i g^3 [B_L epsslash q2slash gamma^mu K_L]
 *       H_mu / (q2^2 s_H),       colour (T^a T^b)_{B_L K_L} T^b_{t tbar}
 *   D3  on the top line next to the top:      i g^3 L_mu [ubar epsslash (q3slash + m)
 *       gamma^mu v] / (D3 s_L),  colour T^b_{B_L K_L} (T^a T^b)_{t tbar}
 *   D4  next to the antitop:                  i g^3 L_mu [ubar gamma^mu (q4slash + m)
 *       epsslash v] / (D4 s_L),  colour T^b_{B_L K_L} (T^b T^a)_{t tbar}
 *   D5  three-gluon vertex:  -g^3 V(L, k1; H, k2; eps, k3) / (s_L s_H),
 *       colour f^{b c a} T^b_{B_L K_L} T^c_{t tbar}
 * where P_i is the incoming momentum of particle i (+p incoming, -p outgoing),
 * q1 = P_{K_L} + P_g, q2 = -(P_{B_L} + P_g), q3 = -(P_t + P_g), q4 = P_tbar + P_g,
 * k1 = P_{B_L} + P_{K_L}, k2 = P_t + P_tbar, k3 = P_g, s_L = k1^2, s_H = k2^2 and
 * V = (L.H)(k1-k2).eps + (H.eps)(k2-k3).L + (eps.L)(k3-k1).H.  |M|^2 is summed over all
 * 3^4 x 8 colour assignments.  Colour flows (the basis of the selection weights):
 *   c_0 = T^a_{B_L tbar} d_{t K_L},  c_1 = T^a_{t K_L} d_{B_L tbar},
 *   c_2 = T^a_{B_L K_L} d_{t tbar},  c_3 = T^a_{t tbar} d_{B_L K_L}
 * (indices: B_L, K_L, t, tbar colours; row index first). */
#define Q3_NCOLIDX (NC * NC * NC * NC * 8)
static cx QG_DCOL[5][Q3_NCOLIDX]; /* colour factor of each diagram per assignment */
static cx QG_FLOW[4][Q3_NCOLIDX]; /* flow tensors per assignment */
static int qg_colour_ready = 0;

/* assignment index of (B_L, K_L, t, tbar, a) colours */
static int qg_cidx(int bl, int kl, int t, int tb, int a) { return (((bl * NC + kl) * NC + t) * NC + tb) * 8 + a; }

static void qg_colour_init(void) {
  if (qg_colour_ready) return;
  tgm_init();
  /* f^{abc} = -2 i Tr([T^a, T^b] T^c), from [T^a, T^b] = i f^{abc} T^c and Tr(T^a T^b) = d^{ab}/2 */
  static double F[8][8][8];
  for (int a = 0; a < 8; ++a)
    for (int b = 0; b < 8; ++b)
      for (int c = 0; c < 8; ++c) {
        cx tr = 0;
        for (int i = 0; i < NC; ++i)
          for (int j = 0; j < NC; ++j)
            for (int k = 0; k < NC; ++k)
              tr += (TGM[a][i][j] * TGM[b][j][k] - TGM[b][i][j] * TGM[a][j][k]) * TGM[c][k][i];
        F[a][b][c] = creal(-2.0 * I * tr);
      }
  for (int bl = 0; bl < NC; ++bl)
    for (int kl = 0; kl < NC; ++kl)
      for (int t = 0; t < NC; ++t)
        for (int tb = 0; tb < NC; ++tb)
          for (int a = 0; a < 8; ++a) {
            int x = qg_cidx(bl, kl, t, tb, a);
            cx c[5] = {0, 0, 0, 0, 0};
            for (int b = 0; b < 8; ++b) {
              cx ba = 0, ab = 0, hab = 0, hba = 0; /* (T^b T^a), (T^a T^b) on each line */
              for (int m = 0; m < NC; ++m) {
                ba += TGM[b][bl][m] * TGM[a][m][kl];
                ab += TGM[a][bl][m] * TGM[b][m][kl];
                hab += TGM[a][t][m] * TGM[b][m][tb];
                hba += TGM[b][t][m] * TGM[a][m][tb];
              }
              c[0] += ba * TGM[b][t][tb];
              c[1] += ab * TGM[b][t][tb];
              c[2] += TGM[b][bl][kl] * hab;
              c[3] += TGM[b][bl][kl] * hba;
              for (int cc = 0; cc < 8; ++cc) c[4] += F[b][cc][a] * TGM[b][bl][kl] * TGM[cc][t][tb];
            }
            for (int d = 0; d < 5; ++d) QG_DCOL[d][x] = c[d];
            QG_FLOW[0][x] = TGM[a][bl][tb] * (double)(t == kl);
            QG_FLOW[1][x] = TGM[a][t][kl] * (double)(bl == tb);
            QG_FLOW[2][x] = TGM[a][bl][kl] * (double)(t == tb);
            QG_FLOW[3][x] = TGM[a][t][tb] * (double)(bl == kl);
          }
  qg_colour_ready = 1;
}

/* Gram matrix of the flow tensors, G_nm = sum over assignments of conj(c_n) c_m */
static void qg_gram(cx G[4][4]) {
  for (int n = 0; n < 4; ++n)
    for (int m = 0; m < 4; ++m) {
      cx s = 0;
      for (int x = 0; x < Q3_NCOLIDX; ++x) s += conj(QG_FLOW[n][x]) * QG_FLOW[m][x];
      G[n][m] = s;
    }
}

typedef struct {
  int bl, kl, g, t, tb;    /* particle indices: light row end, light column end, gluon, top, antitop */
  double den[4];           /* q1^2, q2^2, q3^2 - mt^2, q4^2 - mt^2 */
  double sL, sH;           /* k1^2, k2^2 */
  int tch3, tch4;          /* the top propagators of D3, D4 separate the incoming particles */
} qg_kin;

/* incoming momentum of particle i, as quads */
static void qg_pin(const proc_def* pd, const double* mom, int i, quad* P) {
  int in = pd->role[i] == R_Q_IN || pd->role[i] == R_QB_IN || pd->role[i] == R_G_IN;
  for (int m = 0; m < 4; ++m) P[m] = in ? (quad)mom[4 * i + m] : -(quad)mom[4 * i + m];
}

/* roles and the propagator invariants of one event, formed in quadruple precision (as
 * for the gg processes: exact sums of the FP64 inputs, one rounding at the end) */
static void qg_kinematics(const proc_def* pd, const double* mom, double mt, qg_kin* k) {
  k->bl = k->kl = k->g = k->t = k->tb = 0;
  for (int i = 0; i < pd->npar; ++i) {
    int r = pd->role[i];
    if (r == R_QB_IN || r == R_Q_OUT) k->bl = i;
    if (r == R_Q_IN || r == R_QB_OUT) k->kl = i;
    if (r == R_G_IN || r == R_G_OUT) k->g = i;
    if (r == R_T_OUT) k->t = i;
    if (r == R_TBAR_OUT) k->tb = i;
  }
  quad Pbl[4], Pkl[4], Pg[4], Pt[4], Ptb[4], v[4];
  qg_pin(pd, mom, k->bl, Pbl);
  qg_pin(pd, mom, k->kl, Pkl);
  qg_pin(pd, mom, k->g, Pg);
  qg_pin(pd, mom, k->t, Pt);
  qg_pin(pd, mom, k->tb, Ptb);
  quad mt2 = (quad)mt * (quad)mt;
  for (int m = 0; m < 4; ++m) v[m] = Pkl[m] + Pg[m];
  k->den[0] = (double)msq_q(v);
  for (int m = 0; m < 4; ++m) v[m] = -(Pbl[m] + Pg[m]);
  k->den[1] = (double)msq_q(v);
  for (int m = 0; m < 4; ++m) v[m] = -(Pt[m] + Pg[m]);
  k->den[2] = (double)(msq_q(v) - mt2);
  for (int m = 0; m < 4; ++m) v[m] = Ptb[m] + Pg[m];
  k->den[3] = (double)(msq_q(v) - mt2);
  for (int m = 0; m < 4; ++m) v[m] = Pbl[m] + Pkl[m];
  k->sL = (double)msq_q(v);
  for (int m = 0; m < 4; ++m) v[m] = Pt[m] + Ptb[m];
  k->sH = (double)msq_q(v);
  k->tch3 = is_tchannel((1u << k->t) | (1u << k->g));
  k->tch4 = is_tchannel((1u << k->tb) | (1u << k->g));
}

/* the five diagrams' colour-stripped values A_d at one helicity */
static void qg_diagrams(const double* mom, const int* lam, const proc_def* pd, const qg_kin* k, double gs,
                        double mt, double wt, int zwt, int gauge_leg, cx* A) {
  cx BL[4], KL[4], BH[4], KH[4], eps[4], tmp[4];
  const double *pbl = mom + 4 * k->bl, *pkl = mom + 4 * k->kl, *pg = mom + 4 * k->g;
  if (pd->role[k->bl] == R_QB_IN) { spinor_v(pbl, 0.0, lam[k->bl], tmp); dirac_bar(tmp, BL); }
  else { spinor_u(pbl, 0.0, lam[k->bl], tmp); dirac_bar(tmp, BL); }
  if (pd->role[k->kl] == R_Q_IN) spinor_u(pkl, 0.0, lam[k->kl], KL);
  else spinor_v(pkl, 0.0, lam[k->kl], KL);
  spinor_u(mom + 4 * k->t, mt, lam[k->t], tmp);
  dirac_bar(tmp, BH);
  spinor_v(mom + 4 * k->tb, mt, lam[k->tb], KH);
  polvec(pg, lam[k->g], eps);
  if (pd->role[k->g] == R_G_OUT)
    for (int m = 0; m < 4; ++m) eps[m] = conj(eps[m]);
  if (k->g == gauge_leg)
    for (int m = 0; m < 4; ++m) eps[m] = pg[m] / pg[0];
  /* incoming momenta (FP64) */
  double P[MAXPAR][4];
  for (int i = 0; i < pd->npar; ++i) {
    int in = pd->role[i] == R_Q_IN || pd->role[i] == R_QB_IN || pd->role[i] == R_G_IN;
    for (int m = 0; m < 4; ++m) P[i][m] = in ? mom[4 * i + m] : -mom[4 * i + m];
  }
  double q1[4], q2[4], q3[4], q4[4], k1[4], k2[4], k3[4];
  for (int m = 0; m < 4; ++m) {
    q1[m] = P[k->kl][m] + P[k->g][m];
    q2[m] = -(P[k->bl][m] + P[k->g][m]);
    q3[m] = -(P[k->t][m] + P[k->g][m]);
    q4[m] = P[k->tb][m] + P[k->g][m];
    k1[m] = P[k->bl][m] + P[k->kl][m];
    k2[m] = P[k->t][m] + P[k->tb][m];
    k3[m] = P[k->g][m];
  }
  cx E[4][4], S[4][4], x[4], y[4];
  slash(eps, E);
  cx L[4], H[4], L1[4], L2[4], H3[4], H4[4];
  vector_current(BL, KL, 1.0, 1.0, L);
  vector_current(BH, KH, 1.0, 1.0, H);
  /* D1: B_L gamma^mu q1slash epsslash K_L */
  {
    cx qc[4] = {q1[0], q1[1], q1[2], q1[3]};
    slash(qc, S);
    for (int r = 0; r < 4; ++r) { x[r] = 0; for (int c = 0; c < 4; ++c) x[r] += E[r][c] * KL[c]; }
    for (int r = 0; r < 4; ++r) { y[r] = 0; for (int c = 0; c < 4; ++c) y[r] += S[r][c] * x[c]; }
    vector_current(BL, y, 1.0, 1.0, L1);
  }
  /* D2: B_L epsslash q2slash gamma^mu K_L */
  {
    cx qc[4] = {q2[0], q2[1], q2[2], q2[3]};
    slash(qc, S);
    bra_mat(BL, E, x);
    bra_mat(x, S, y);
    vector_current(y, KL, 1.0, 1.0, L2);
  }
  /* D3: ubar epsslash (q3slash + m) gamma^mu v */
  {
    cx qc[4] = {q3[0], q3[1], q3[2], q3[3]};
    slash(qc, S);
    for (int r = 0; r < 4; ++r) S[r][r] += mt;
    bra_mat(BH, E, x);
    bra_mat(x, S, y);
    vector_current(y, KH, 1.0, 1.0, H3);
  }
  /* D4: ubar gamma^mu (q4slash + m) epsslash v */
  {
    cx qc[4] = {q4[0], q4[1], q4[2], q4[3]};
    slash(qc, S);
    for (int r = 0; r < 4; ++r) S[r][r] += mt;
    for (int r = 0; r < 4; ++r) { x[r] = 0; for (int c = 0; c < 4; ++c) x[r] += E[r][c] * KH[c]; }
    for (int r = 0; r < 4; ++r) { y[r] = 0; for (int c = 0; c < 4; ++c) y[r] += S[r][c] * x[c]; }
    vector_current(BH, y, 1.0, 1.0, H4);
  }
  cx D3 = k->den[2] + I * mt * ((zwt && k->tch3) ? 0.0 : wt);
  cx D4 = k->den[3] + I * mt * ((zwt && k->tch4) ? 0.0 : wt);
  cx g3 = gs * gs * gs;
  A[0] = I * g3 * mdot_c(L1, H) / (k->den[0] * k->sH);
  A[1] = I * g3 * mdot_c(L2, H) / (k->den[1] * k->sH);
  A[2] = I * g3 * mdot_c(L, H3) / (D3 * k->sL);
  A[3] = I * g3 * mdot_c(L, H4) / (D4 * k->sL);
  double d12[4], d23[4], d31[4];
  for (int m = 0; m < 4; ++m) {
    d12[m] = k1[m] - k2[m];
    d23[m] = k2[m] - k3[m];
    d31[m] = k3[m] - k1[m];
  }
  cx ed12 = eps[0] * d12[0] - eps[1] * d12[1] - eps[2] * d12[2] - eps[3] * d12[3];
  cx ld23 = L[0] * d23[0] - L[1] * d23[1] - L[2] * d23[2] - L[3] * d23[3];
  cx hd31 = H[0] * d31[0] - H[1] * d31[1] - H[2] * d31[2] - H[3] * d31[3];
  cx V = mdot_c(L, H) * ed12 + mdot_c(H, eps) * ld23 + mdot_c(eps, L) * hd31;
  A[4] = -g3 * V / (k->sL * k->sH);
}

/* explicit colour sum of |M|^2 at one helicity and the flow amplitudes J (M = sum_n J_n
 * c_n, from the projections onto the flow tensors and their Gram matrix) */
static double qg_colour_sum(const cx* A, const cx Ginv[4][4], cx* J) {
  double m2 = 0;
  cx Pr[4] = {0, 0, 0, 0};
  for (int x = 0; x < Q3_NCOLIDX; ++x) {
    cx M = 0;
    for (int d = 0; d < 5; ++d) M += A[d] * QG_DCOL[d][x];
    m2 += creal(M) * creal(M) + cimag(M) * cimag(M);
    for (int n = 0; n < 4; ++n) Pr[n] += conj(QG_FLOW[n][x]) * M;
  }
  for (int n = 0; n < 4; ++n) {
    J[n] = 0;
    for (int m = 0; m < 4; ++m) J[n] += Ginv[n][m] * Pr[m];
  }
  return m2;
}

/* inverse of a 4 x 4 complex matrix by Gauss-Jordan elimination with partial pivoting */
static void inv4(const cx G[4][4], cx Ginv[4][4]) {
  cx a[4][8];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 8; ++j) a[i][j] = j < 4 ? G[i][j] : (cx)(j - 4 == i);
  for (int c = 0; c < 4; ++c) {
    int piv = c;
    for (int r = c + 1; r < 4; ++r) if (cabs(a[r][c]) > cabs(a[piv][c])) piv = r;
    for (int j = 0; j < 8; ++j) { cx t = a[c][j]; a[c][j] = a[piv][j]; a[piv][j] = t; }
    cx d = a[c][c];
    for (int j = 0; j < 8; ++j) a[c][j] /= d;
    for (int r = 0; r < 4; ++r)
      if (r != c) {
        cx f = a[r][c];
        for (int j = 0; j < 8; ++j) a[r][j] -= f * a[c][j];
      }
  }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) Ginv[i][j] = a[i][4 + j];
}

/* ------------------------------------------------------------------------- */
/* One light-quark line, the top line and two gluons (kind 4): q qbar -> t tbar g g and its
 * crossings, explicit colour                                                   */
/* ------------------------------------------------------------------------- */
/* The Feynman diagrams are built from three kinds of objects: gluon a and gluon b (a is
 * the one with the lower particle index) and the pair a b joined by a three-gluon vertex
 * into one off-shell gluon.  Each object hangs on the light line, on the top line or on
 * the gluon that joins the two lines (the connector); every order of the objects and of
 * the connector's end ("stub") along each line gives one diagram.  The connector is one
 * propagator (no object on it), a three-gluon vertex with one object, two three-gluon
 * vertices with a and b in either order, or the four-gluon vertex, whose three
 * colour-Lorentz structures are kept as three terms.  For two separate gluons this
 * gives 6 + 6 + 8 + 4 + 4 + 3 diagrams (both on the light line, both on the top line,
 * one on each, one on the connector and the other on either line, both on the
 * connector) and for the joined pair 2 + 2 + 1 (on either line or on the connector):
 * 36 diagrams, 38 terms.
 * Feynman rules as for the other QCD processes: quark-gluon vertex -i g gamma^mu T^x,
 * fermion propagator i(qslash + m)/(q^2 - m^2 + i m w) with q along the fermion arrow,
 * gluon propagator -i g_{mu nu}/K^2, three-gluon vertex -g f^{xyz} V^{mu nu rho}(k1, k2,
 * k3) (all momenta incoming), four-gluon vertex -i g^2 [f^{x y e} f^{z w e} (g^{mu rho}
 * g^{nu sigma} - g^{mu sigma} g^{nu rho}) + f^{x z e} f^{y w e} (g^{mu nu} g^{rho sigma} -
 * g^{mu sigma} g^{nu rho}) + f^{x w e} f^{y z e} (g^{mu nu} g^{rho sigma} - g^{mu rho}
 * g^{nu sigma})] for legs (x mu) (y nu) (z rho) (w sigma).
 * Colour flows (indices: light row end B, light column end K, top t, antitop y, gluons
 * a b; 13 independent tensors, the fourteenth string product being a combination of
 * these):
 *   0 (T^a T^b)_{B y} d_{t K}   1 (T^b T^a)_{B y} d_{t K}   2 T^a_{B y} T^b_{t K}
 *   3 T^b_{B y} T^a_{t K}       4 d_{B y} (T^a T^b)_{t K}   5 d_{B y} (T^b T^a)_{t K}
 *   6 (T^a T^b)_{B K} d_{t y}   7 (T^b T^a)_{B K} d_{t y}   8 T^a_{B K} T^b_{t y}
 *   9 T^b_{B K} T^a_{t y}       10 d_{B K} (T^a T^b)_{t y}  11 d_{B K} (T^b T^a)_{t y}
 *   12 d^{ab} d_{B y} d_{t K} */
#define Q4_NCI (NC * NC * NC * NC * 64)
#define Q4_NFLOW 13
#define Q4_MAXTERM 40
enum { Q4_A = 0, Q4_B = 1, Q4_AB = 2, Q4_STUB = 3 };

typedef struct {
  int nl, nh;  /* insertions on the light line (from its row end) and on the top line (from the top), stub included */
  int l[3], h[3];
  int conn;    /* 0 one propagator; 1, 2, 3 a three-gluon vertex with object a, b, ab;
                  4 a then b from the light side; 5 b then a; 6, 7, 8 four-gluon structure 1, 2, 3 */
} q4_term;

static q4_term Q4_TERMS[Q4_MAXTERM];
static int q4_nterm = 0;
static cx* Q4_DCOL = 0;            /* [term][Q4_NCI] */
static cx Q4_FLOW[Q4_NFLOW][Q4_NCI];
static double Q4_F[8][8][8];
static int q4_ready = 0;

/* colour assignment index of (B, K, t, y, a, b) */
static int q4_cidx(int B, int K, int t, int y, int a, int b) { return ((((B * NC + K) * NC + t) * NC + y) * 8 + a) * 8 + b; }

/* every order of the n items (n <= 3) */
static int q4_perms(const int* items, int n, int out[6][3]) {
  int np = 0;
  if (n == 1) { out[0][0] = items[0]; return 1; }
  for (int i = 0; i < n; ++i) {
    int rest[2], nr = 0;
    for (int j = 0; j < n; ++j) if (j != i) rest[nr++] = items[j];
    int sub[6][3];
    int ns = q4_perms(rest, n - 1, sub);
    for (int s = 0; s < ns; ++s) {
      out[np][0] = items[i];
      for (int j = 0; j < n - 1; ++j) out[np][j + 1] = sub[s][j];
      ++np;
    }
  }
  return np;
}

static void q4_enumerate(void) {
  q4_nterm = 0;
  for (int joined = 0; joined < 2; ++joined) {
    int nobj = joined ? 1 : 2;
    int obj[2] = {joined ? Q4_AB : Q4_A, Q4_B};
    for (int pa = 0; pa < 3; ++pa)
      for (int pb = 0; pb < (joined ? 1 : 3); ++pb) {
        int place[2] = {pa, pb};
        int li[3], hi[3], ci[2], nl = 0, nh = 0, nc = 0;
        for (int o = 0; o < nobj; ++o) {
          if (place[o] == 0) li[nl++] = obj[o];
          else if (place[o] == 1) hi[nh++] = obj[o];
          else ci[nc++] = obj[o];
        }
        li[nl++] = Q4_STUB;
        hi[nh++] = Q4_STUB;
        int conns[5], ncon = 0;
        if (nc == 0) conns[ncon++] = 0;
        else if (nc == 1) conns[ncon++] = 1 + ci[0];
        else { conns[0] = 4; conns[1] = 5; conns[2] = 6; conns[3] = 7; conns[4] = 8; ncon = 5; }
        int lp[6][3], hp[6][3];
        int nlp = q4_perms(li, nl, lp), nhp = q4_perms(hi, nh, hp);
        for (int x = 0; x < nlp; ++x)
          for (int y = 0; y < nhp; ++y)
            for (int c = 0; c < ncon; ++c) {
              q4_term* t = &Q4_TERMS[q4_nterm++];
              t->nl = nl;
              t->nh = nh;
              for (int j = 0; j < nl; ++j) t->l[j] = lp[x][j];
              for (int j = 0; j < nh; ++j) t->h[j] = hp[y][j];
              t->conn = conns[c];
            }
      }
  }
}

/* 3 x 3 colour matrix of one insertion: object a, b, the joined pair (colour e), the stub (colour c) */
static void q4_mat(int o, int a, int b, int c, int e, cx m[NC][NC]) {
  int x = o == Q4_A ? a : o == Q4_B ? b : o == Q4_AB ? e : c;
  for (int i = 0; i < NC; ++i)
    for (int j = 0; j < NC; ++j) m[i][j] = TGM[x][i][j];
}

static void q4_string(const int* items, int n, int a, int b, int c, int e, cx out[NC][NC]) {
  cx acc[NC][NC], m[NC][NC], t[NC][NC];
  q4_mat(items[0], a, b, c, e, acc);
  for (int k = 1; k < n; ++k) {
    q4_mat(items[k], a, b, c, e, m);
    for (int i = 0; i < NC; ++i)
      for (int j = 0; j < NC; ++j) {
        cx s = 0;
        for (int l = 0; l < NC; ++l) s += acc[i][l] * m[l][j];
        t[i][j] = s;
      }
    memcpy(acc, t, sizeof acc);
  }
  memcpy(out, acc, sizeof acc);
}

/* connector colour (with f^{abe} of a joined pair on either line); c1 the light stub,
 * c2 the top stub, e the internal gluon */
static double q4_conn_colour(const q4_term* t, int a, int b, int c1, int c2, int e) {
  int joined = 0;
  for (int j = 0; j < t->nl; ++j) joined |= t->l[j] == Q4_AB;
  for (int j = 0; j < t->nh; ++j) joined |= t->h[j] == Q4_AB;
  double f = joined ? Q4_F[a][b][e] : 1.0;
  switch (t->conn) {
    case 0: return joined ? f * (c1 == c2) : (double)(c1 == c2) * (e == 0);
    case 1: return Q4_F[c1][a][c2] * (e == 0);
    case 2: return Q4_F[c1][b][c2] * (e == 0);
    case 3: return Q4_F[c1][e][c2] * Q4_F[a][b][e];
    case 4: return Q4_F[c1][a][e] * Q4_F[e][b][c2];
    case 5: return Q4_F[c1][b][e] * Q4_F[e][a][c2];
    case 6: return Q4_F[c1][a][e] * Q4_F[b][c2][e];
    case 7: return Q4_F[c1][b][e] * Q4_F[a][c2][e];
    default: return Q4_F[c1][c2][e] * Q4_F[a][b][e];
  }
}

static void q4_colour_init(void) {
  if (q4_ready) return;
  tgm_init();
  for (int a = 0; a < 8; ++a)
    for (int b = 0; b < 8; ++b)
      for (int c = 0; c < 8; ++c) {
        cx tr = 0;
        for (int i = 0; i < NC; ++i)
          for (int j = 0; j < NC; ++j)
            for (int k = 0; k < NC; ++k)
              tr += (TGM[a][i][j] * TGM[b][j][k] - TGM[b][i][j] * TGM[a][j][k]) * TGM[c][k][i];
        Q4_F[a][b][c] = creal(-2.0 * I * tr);
      }
  q4_enumerate();
  Q4_DCOL = (cx*)calloc((size_t)q4_nterm * Q4_NCI, sizeof(cx));
  for (int d = 0; d < q4_nterm; ++d) {
    const q4_term* t = &Q4_TERMS[d];
    for (int a = 0; a < 8; ++a)
      for (int b = 0; b < 8; ++b)
        for (int c1 = 0; c1 < 8; ++c1)
          for (int c2 = 0; c2 < 8; ++c2)
            for (int e = 0; e < 8; ++e) {
              double w = q4_conn_colour(t, a, b, c1, c2, e);
              if (w == 0.0) continue;
              cx L[NC][NC], H[NC][NC];
              q4_string(t->l, t->nl, a, b, c1, e, L);
              q4_string(t->h, t->nh, a, b, c2, e, H);
              for (int B = 0; B < NC; ++B)
                for (int K = 0; K < NC; ++K)
                  for (int tt = 0; tt < NC; ++tt)
                    for (int y = 0; y < NC; ++y) Q4_DCOL[(size_t)d * Q4_NCI + q4_cidx(B, K, tt, y, a, b)] += w * L[B][K] * H[tt][y];
            }
  }
  for (int B = 0; B < NC; ++B)
    for (int K = 0; K < NC; ++K)
      for (int t = 0; t < NC; ++t)
        for (int y = 0; y < NC; ++y)
          for (int a = 0; a < 8; ++a)
            for (int b = 0; b < 8; ++b) {
              int x = q4_cidx(B, K, t, y, a, b);
              cx ab_By = 0, ba_By = 0, ab_tK = 0, ba_tK = 0, ab_BK = 0, ba_BK = 0, ab_ty = 0, ba_ty = 0;
              for (int m = 0; m < NC; ++m) {
                ab_By += TGM[a][B][m] * TGM[b][m][y];
                ba_By += TGM[b][B][m] * TGM[a][m][y];
                ab_tK += TGM[a][t][m] * TGM[b][m][K];
                ba_tK += TGM[b][t][m] * TGM[a][m][K];
                ab_BK += TGM[a][B][m] * TGM[b][m][K];
                ba_BK += TGM[b][B][m] * TGM[a][m][K];
                ab_ty += TGM[a][t][m] * TGM[b][m][y];
                ba_ty += TGM[b][t][m] * TGM[a][m][y];
              }
              double dtK = t == K, dBy = B == y, dBK = B == K, dty = t == y;
              Q4_FLOW[0][x] = ab_By * dtK;
              Q4_FLOW[1][x] = ba_By * dtK;
              Q4_FLOW[2][x] = TGM[a][B][y] * TGM[b][t][K];
              Q4_FLOW[3][x] = TGM[b][B][y] * TGM[a][t][K];
              Q4_FLOW[4][x] = dBy * ab_tK;
              Q4_FLOW[5][x] = dBy * ba_tK;
              Q4_FLOW[6][x] = ab_BK * dty;
              Q4_FLOW[7][x] = ba_BK * dty;
              Q4_FLOW[8][x] = TGM[a][B][K] * TGM[b][t][y];
              Q4_FLOW[9][x] = TGM[b][B][K] * TGM[a][t][y];
              Q4_FLOW[10][x] = dBK * ab_ty;
              Q4_FLOW[11][x] = dBK * ba_ty;
              Q4_FLOW[12][x] = (double)(a == b) * dBy * dtK;
            }
  q4_ready = 1;
}

/* inverse of an n x n complex matrix (n <= MAXFLOWINV) by Gauss-Jordan elimination with
 * partial pivoting */
#define MAXFLOWINV 16
static void invn(int n, const cx* G, cx* Ginv) {
  cx a[MAXFLOWINV][2 * MAXFLOWINV];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j) a[i][j] = j < n ? G[i * n + j] : (cx)(j - n == i);
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r) if (cabs(a[r][c]) > cabs(a[piv][c])) piv = r;
    for (int j = 0; j < 2 * n; ++j) { cx t = a[c][j]; a[c][j] = a[piv][j]; a[piv][j] = t; }
    cx dv = a[c][c];
    for (int j = 0; j < 2 * n; ++j) a[c][j] /= dv;
    for (int r = 0; r < n; ++r)
      if (r != c) {
        cx f = a[r][c];
        for (int j = 0; j < 2 * n; ++j) a[r][j] -= f * a[c][j];
      }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Ginv[i * n + j] = a[i][n + j];
}

static void q4_gram(cx* G) {
  for (int n = 0; n < Q4_NFLOW; ++n)
    for (int m = 0; m < Q4_NFLOW; ++m) {
      cx s = 0;
      for (int x = 0; x < Q4_NCI; ++x) s += conj(Q4_FLOW[n][x]) * Q4_FLOW[m][x];
      G[n * Q4_NFLOW + m] = s;
    }
}

typedef struct {
  int bl, kl, t, tb, ga, gb;       /* particle indices */
  double inv[1 << MAXPAR];         /* (sum over the mask of the incoming momenta)^2, formed in quad */
} q4_kin;

static int q4_in(int r) { return r == R_Q_IN || r == R_QB_IN || r == R_G_IN; }

static void q4_kinematics(const proc_def* pd, const double* mom, q4_kin* k) {
  int ng = 0;
  k->bl = k->kl = k->t = k->tb = k->ga = k->gb = 0;
  for (int i = 0; i < pd->npar; ++i) {
    int r = pd->role[i];
    if (r == R_QB_IN || r == R_Q_OUT) k->bl = i;
    if (r == R_Q_IN || r == R_QB_OUT) k->kl = i;
    if (r == R_T_OUT) k->t = i;
    if (r == R_TBAR_OUT) k->tb = i;
    if (r == R_G_IN || r == R_G_OUT) { if (ng++ == 0) k->ga = i; else k->gb = i; }
  }
  for (unsigned mask = 0; mask < (1u << pd->npar); ++mask) {
    quad K[4] = {0, 0, 0, 0};
    for (int i = 0; i < pd->npar; ++i)
      if (mask >> i & 1)
        for (int m = 0; m < 4; ++m) K[m] += q4_in(pd->role[i]) ? (quad)mom[4 * i + m] : -(quad)mom[4 * i + m];
    k->inv[mask] = (double)msq_q(K);
  }
}

/* the wavefunction, incoming momentum and particle mask of each object */
typedef struct {
  cx W[3][4];
  double P[3][4];
  unsigned mask[3];
} q4_objs;

/* fermion line B ... K with insertions ins[0..n-1] (from B), one of them the stub; the
 * line's vector current at the stub (including the stub's -i g) into L, and the mask of
 * the momentum it sends into the connector */
static unsigned q4_line(const cx* Bsp, const cx* Ksp, int ib, int ik, const int* ins, int n, const q4_objs* o,
                        const double (*Pin)[4], const q4_kin* k, double m, double wt, int zwt, double g, cx* L) {
  int s = 0;
  while (ins[s] != Q4_STUB) ++s;
  cx x[4], y[4], t[4], S[4][4], G[4][4];
  memcpy(x, Bsp, sizeof x);
  unsigned mB = 1u << ib;
  double qB[4] = {Pin[ib][0], Pin[ib][1], Pin[ib][2], Pin[ib][3]};
  for (int j = 0; j < s; ++j) {
    slash(o->W[ins[j]], G);
    bra_mat(x, G, t);
    for (int r = 0; r < 4; ++r) x[r] = -I * g * t[r];
    mB |= o->mask[ins[j]];
    for (int mu = 0; mu < 4; ++mu) qB[mu] += o->P[ins[j]][mu];
    /* propagator K-ward of vertex j: momentum along the arrow -(P_B + sum k) */
    cx qc[4] = {-qB[0], -qB[1], -qB[2], -qB[3]};
    slash(qc, S);
    for (int r = 0; r < 4; ++r) S[r][r] += m;
    double w = (m > 0.0 && !(zwt && is_tchannel(mB))) ? wt : 0.0;
    cx D = k->inv[mB] - m * m + I * m * w;
    bra_mat(x, S, t);
    for (int r = 0; r < 4; ++r) x[r] = I * t[r] / D;
  }
  memcpy(y, Ksp, sizeof y);
  unsigned mK = 1u << ik;
  double qK[4] = {Pin[ik][0], Pin[ik][1], Pin[ik][2], Pin[ik][3]};
  for (int j = n - 1; j > s; --j) {
    slash(o->W[ins[j]], G);
    for (int r = 0; r < 4; ++r) { t[r] = 0; for (int c = 0; c < 4; ++c) t[r] += G[r][c] * y[c]; }
    for (int r = 0; r < 4; ++r) y[r] = -I * g * t[r];
    mK |= o->mask[ins[j]];
    for (int mu = 0; mu < 4; ++mu) qK[mu] += o->P[ins[j]][mu];
    /* propagator B-ward of vertex j: momentum along the arrow P_K + sum k */
    cx qc[4] = {qK[0], qK[1], qK[2], qK[3]};
    slash(qc, S);
    for (int r = 0; r < 4; ++r) S[r][r] += m;
    double w = (m > 0.0 && !(zwt && is_tchannel(mK))) ? wt : 0.0;
    cx D = k->inv[mK] - m * m + I * m * w;
    for (int r = 0; r < 4; ++r) { t[r] = 0; for (int c = 0; c < 4; ++c) t[r] += S[r][c] * y[c]; }
    for (int r = 0; r < 4; ++r) y[r] = I * t[r] / D;
  }
  cx J[4];
  vector_current(x, y, 1.0, 1.0, J);
  for (int mu = 0; mu < 4; ++mu) L[mu] = -I * g * J[mu];
  return mB | mK;
}

/* the colour-stripped value of every term at one helicity */
static void q4_diagrams(const double* mom, const int* lam, const proc_def* pd, const q4_kin* k, double gs, double mt,
                        double wt, int zwt, int gauge_leg, cx* A) {
  double Pin[MAXPAR][4];
  for (int i = 0; i < pd->npar; ++i)
    for (int m = 0; m < 4; ++m) Pin[i][m] = q4_in(pd->role[i]) ? mom[4 * i + m] : -mom[4 * i + m];
  cx BL[4], KL[4], BH[4], KH[4], tmp[4];
  const double *pbl = mom + 4 * k->bl, *pkl = mom + 4 * k->kl;
  if (pd->role[k->bl] == R_QB_IN) spinor_v(pbl, 0.0, lam[k->bl], tmp);
  else spinor_u(pbl, 0.0, lam[k->bl], tmp);
  dirac_bar(tmp, BL);
  if (pd->role[k->kl] == R_Q_IN) spinor_u(pkl, 0.0, lam[k->kl], KL);
  else spinor_v(pkl, 0.0, lam[k->kl], KL);
  spinor_u(mom + 4 * k->t, mt, lam[k->t], tmp);
  dirac_bar(tmp, BH);
  spinor_v(mom + 4 * k->tb, mt, lam[k->tb], KH);
  q4_objs o;
  int gl[2] = {k->ga, k->gb};
  for (int x = 0; x < 2; ++x) {
    const double* pg = mom + 4 * gl[x];
    polvec(pg, lam[gl[x]], o.W[x]);
    if (pd->role[gl[x]] == R_G_OUT)
      for (int m = 0; m < 4; ++m) o.W[x][m] = conj(o.W[x][m]);
    if (gl[x] == gauge_leg)
      for (int m = 0; m < 4; ++m) o.W[x][m] = pg[m] / pg[0];
    for (int m = 0; m < 4; ++m) o.P[x][m] = Pin[gl[x]][m];
    o.mask[x] = 1u << gl[x];
  }
  /* the joined pair: vertex -g f^{abe} V(P_a, P_b, -(P_a + P_b)), propagator -i/s_ab */
  {
    cx v[4];
    v3(o.P[0], o.W[0], o.P[1], o.W[1], v);
    o.mask[2] = o.mask[0] | o.mask[1];
    double sab = k->inv[o.mask[2]];
    for (int m = 0; m < 4; ++m) {
      o.W[2][m] = (-gs) * (-I / sab) * v[m];
      o.P[2][m] = o.P[0][m] + o.P[1][m];
    }
  }
  for (int d = 0; d < q4_nterm; ++d) {
    const q4_term* t = &Q4_TERMS[d];
    cx L[4], H[4];
    unsigned mL = q4_line(BL, KL, k->bl, k->kl, t->l, t->nl, &o, (const double (*)[4])Pin, k, 0.0, 0.0, 0, gs, L);
    unsigned mH = q4_line(BH, KH, k->t, k->tb, t->h, t->nh, &o, (const double (*)[4])Pin, k, mt, wt, zwt, gs, H);
    /* momenta the lines send into the connector */
    double QL[4], QH[4];
    for (int m = 0; m < 4; ++m) {
      QL[m] = 0;
      QH[m] = 0;
      for (int i = 0; i < pd->npar; ++i) {
        if (mL >> i & 1) QL[m] += Pin[i][m];
        if (mH >> i & 1) QH[m] += Pin[i][m];
      }
    }
    cx pL = -I / k->inv[mL], pH = -I / k->inv[mH];
    cx v[4], val;
    switch (t->conn) {
      case 0:
        val = pL * mdot_c(L, H);
        break;
      case 1: case 2: case 3: {
        int x = t->conn - 1;
        v3(QL, L, o.P[x], o.W[x], v);
        val = (-gs) * pL * pH * mdot_c(v, H);
        break;
      }
      case 4: case 5: {
        int x1 = t->conn == 4 ? 0 : 1, x2 = 1 - x1;
        double Qe[4];
        for (int m = 0; m < 4; ++m) Qe[m] = QL[m] + o.P[x1][m];
        cx Je[4], w[4];
        v3(QL, L, o.P[x1], o.W[x1], w);
        cx pe = -I / k->inv[mL | o.mask[x1]];
        for (int m = 0; m < 4; ++m) Je[m] = (-gs) * pe * w[m];
        v3(Qe, Je, o.P[x2], o.W[x2], v);
        val = (-gs) * pL * pH * mdot_c(v, H);
        break;
      }
      default: {
        const cx *ea = o.W[0], *eb = o.W[1];
        cx lor;
        if (t->conn == 6) lor = mdot_c(L, eb) * mdot_c(ea, H) - mdot_c(L, H) * mdot_c(ea, eb);
        else if (t->conn == 7) lor = mdot_c(L, ea) * mdot_c(eb, H) - mdot_c(L, H) * mdot_c(ea, eb);
        else lor = mdot_c(L, ea) * mdot_c(eb, H) - mdot_c(L, eb) * mdot_c(ea, H);
        val = (-I * gs * gs) * pL * pH * lor;
      }
    }
    A[d] = val;
  }
}

/* explicit colour sum of |M|^2 at one helicity and the flow amplitudes */
static double q4_colour_sum(const cx* A, const cx* Ginv, cx* J) {
  double m2 = 0;
  cx Pr[Q4_NFLOW];
  for (int n = 0; n < Q4_NFLOW; ++n) Pr[n] = 0;
  for (int x = 0; x < Q4_NCI; ++x) {
    cx M = 0;
    for (int d = 0; d < q4_nterm; ++d) M += A[d] * Q4_DCOL[(size_t)d * Q4_NCI + x];
    if (M == 0) continue;
    m2 += creal(M) * creal(M) + cimag(M) * cimag(M);
    for (int n = 0; n < Q4_NFLOW; ++n) Pr[n] += conj(Q4_FLOW[n][x]) * M;
  }
  for (int n = 0; n < Q4_NFLOW; ++n) {
    J[n] = 0;
    for (int m = 0; m < Q4_NFLOW; ++m) J[n] += Ginv[n * Q4_NFLOW + m] * Pr[m];
  }
  return m2;
}

/* ------------------------------------------------------------------------- */
/* Three fermion lines (kind 5): the four-quark channels of p p -> t tbar + 2 jets with two
 * light quarks of different flavours (u and d), explicit colour                */
/* ------------------------------------------------------------------------- */
/* Lines: 0 the u line, 1 the d line, 2 the top line; each runs from its row end (an
 * incoming antiquark or outgoing quark: vbar or ubar) to its column end (an incoming
 * quark or outgoing antiquark: u or v).  The gluons form a tree joining the three lines:
 *   term 0: one three-gluon vertex joining a stub of every line;
 *   terms 1-6: line X carries the currents of the other two lines Y, Z (Y nearer X's row
 *   end), X = 0, 1, 2 and both orders.
 * Feynman rules as for the other QCD processes.  Colour flows over the row-end colours
 * (B0, B1, t) and column-end colours (K0, K1, y): the six products d_{B0 K_s0} d_{B1 K_s1}
 * d_{t K_s2} for the permutations s of (K0, K1, y) in lexicographic order. */
#define Q5_NCI (NC * NC * NC * NC * NC * NC)
#define Q5_NFLOW 6
#define Q5_NTERM 7
/* terms 7-13: the second pairing of one light flavour (column ends K0 and K1 exchanged) */
static cx Q5_DCOL[2 * Q5_NTERM][Q5_NCI];
static double Q5_FLOW[Q5_NFLOW][Q5_NCI];
static int q5_ready = 0;
static const int Q5_MID[Q5_NTERM][3] = {{-1, -1, -1}, {0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
static const int Q5_PERM[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

static void q5_colour_init(void) {
  if (q5_ready) return;
  q4_colour_init(); /* the structure constants */
  memset(Q5_DCOL, 0, sizeof Q5_DCOL);
  int B[3], K[3];
  for (int x = 0; x < Q5_NCI; ++x) {
    int r = x;
    K[2] = r % NC; r /= NC; B[2] = r % NC; r /= NC; K[1] = r % NC; r /= NC; B[1] = r % NC; r /= NC;
    K[0] = r % NC; r /= NC; B[0] = r;
    for (int f = 0; f < Q5_NFLOW; ++f)
      Q5_FLOW[f][x] = (B[0] == K[Q5_PERM[f][0]]) && (B[1] == K[Q5_PERM[f][1]]) && (B[2] == K[Q5_PERM[f][2]]);
    /* term 0: f^{c0 c1 c2} T^{c0}_{B0 K0} T^{c1}_{B1 K1} T^{c2}_{t y} */
    cx s = 0;
    for (int c0 = 0; c0 < 8; ++c0)
      for (int c1 = 0; c1 < 8; ++c1)
        for (int c2 = 0; c2 < 8; ++c2) {
          double f = Q4_F[c0][c1][c2];
          if (f != 0.0) s += f * TGM[c0][B[0]][K[0]] * TGM[c1][B[1]][K[1]] * TGM[c2][B[2]][K[2]];
        }
    Q5_DCOL[0][x] = s;
    /* terms 1-6: (T^{cY} T^{cZ})_{B_X K_X} T^{cY}_{B_Y K_Y} T^{cZ}_{B_Z K_Z} */
    for (int d = 1; d < Q5_NTERM; ++d) {
      int X = Q5_MID[d][0], Y = Q5_MID[d][1], Z = Q5_MID[d][2];
      cx v = 0;
      for (int cy = 0; cy < 8; ++cy)
        for (int cz = 0; cz < 8; ++cz) {
          cx m = 0;
          for (int l = 0; l < NC; ++l) m += TGM[cy][B[X]][l] * TGM[cz][l][K[X]];
          v += m * TGM[cy][B[Y]][K[Y]] * TGM[cz][B[Z]][K[Z]];
        }
      Q5_DCOL[d][x] = v;
    }
  }
  for (int x = 0; x < Q5_NCI; ++x) {
    int r = x, y = r % NC;
    r /= NC;
    int t = r % NC; r /= NC;
    int K1 = r % NC; r /= NC;
    int B1 = r % NC; r /= NC;
    int K0 = r % NC; r /= NC;
    int B0 = r;
    int xs = ((((B0 * NC + K1) * NC + B1) * NC + K0) * NC + t) * NC + y;
    for (int d = 0; d < Q5_NTERM; ++d) Q5_DCOL[Q5_NTERM + d][x] = Q5_DCOL[d][xs];
  }
  q5_ready = 1;
}

typedef struct {
  int B[3], K[3];                /* particle index of each line's row end and column end */
  double inv[1 << MAXPAR];
} q5_kin;

static int q5_row(int r) { return r == R_QB_IN || r == R_Q_OUT || r == R_DB_IN || r == R_D_OUT || r == R_T_OUT; }
static int q5_line_of(int r) {
  if (r == R_Q_IN || r == R_QB_IN || r == R_Q_OUT || r == R_QB_OUT) return 0;
  if (r == R_D_IN || r == R_DB_IN || r == R_D_OUT || r == R_DB_OUT) return 1;
  return 2;
}
static int q5_in(int r) { return r == R_Q_IN || r == R_QB_IN || r == R_D_IN || r == R_DB_IN; }

static void q5_kinematics(const proc_def* pd, const double* mom, q5_kin* k) {
  int nb = 0, nk = 0;
  for (int i = 0; i < pd->npar; ++i) {
    int r = pd->role[i], ln = q5_line_of(r);
    if (pd->kind == 6 && ln < 2) {
      /* one light flavour: row ends and column ends take slots 0, 1 in particle order */
      if (q5_row(r)) k->B[nb++] = i;
      else k->K[nk++] = i;
      continue;
    }
    if (q5_row(r)) k->B[ln] = i;
    else k->K[ln] = i;
  }
  for (unsigned mask = 0; mask < (1u << pd->npar); ++mask) {
    quad Q[4] = {0, 0, 0, 0};
    for (int i = 0; i < pd->npar; ++i)
      if (mask >> i & 1)
        for (int m = 0; m < 4; ++m) Q[m] += q5_in(pd->role[i]) ? (quad)mom[4 * i + m] : -(quad)mom[4 * i + m];
    k->inv[mask] = (double)msq_q(Q);
  }
}

/* external spinor of particle i: row (bar) spinor for a row end, column spinor else */
static void q5_spinor(const proc_def* pd, const double* mom, const int* lam, int i, double m, cx* w) {
  int r = pd->role[i];
  cx t[4];
  const double* p = mom + 4 * i;
  if (r == R_QB_IN || r == R_DB_IN) { spinor_v(p, m, lam[i], t); dirac_bar(t, w); }
  else if (r == R_Q_OUT || r == R_D_OUT || r == R_T_OUT) { spinor_u(p, m, lam[i], t); dirac_bar(t, w); }
  else if (r == R_Q_IN || r == R_D_IN) spinor_u(p, m, lam[i], w);
  else spinor_v(p, m, lam[i], w);
}

static void q5_diagrams(const double* mom, const int* lam, const proc_def* pd, const q5_kin* k, double gs, double mt,
                        double wt, int zwt, cx* A) {
  double Pin[MAXPAR][4];
  for (int i = 0; i < pd->npar; ++i)
    for (int m = 0; m < 4; ++m) Pin[i][m] = q5_in(pd->role[i]) ? mom[4 * i + m] : -mom[4 * i + m];
  cx Bs[3][4], Ks[3][4], J[3][4];
  double Q[3][4], ms[3] = {0.0, 0.0, mt};
  unsigned mk[3];
  for (int ln = 0; ln < 3; ++ln) {
    q5_spinor(pd, mom, lam, k->B[ln], ms[ln], Bs[ln]);
    q5_spinor(pd, mom, lam, k->K[ln], ms[ln], Ks[ln]);
    /* the line's current at a stub, -i g B gamma^mu K, and the momentum it sends out */
    vector_current(Bs[ln], Ks[ln], 1.0, 1.0, J[ln]);
    for (int m = 0; m < 4; ++m) {
      J[ln][m] *= -I * gs;
      Q[ln][m] = Pin[k->B[ln]][m] + Pin[k->K[ln]][m];
    }
    mk[ln] = (1u << k->B[ln]) | (1u << k->K[ln]);
  }
  /* term 0: three gluon propagators -i/Q^2 and the vertex -g f V(Q0, Q1, Q2) */
  {
    cx v[4];
    v3(Q[0], J[0], Q[1], J[1], v);
    cx p = (-I / k->inv[mk[0]]) * (-I / k->inv[mk[1]]) * (-I / k->inv[mk[2]]);
    A[0] = (-gs) * p * mdot_c(v, J[2]);
  }
  /* terms 1-6: line X with the currents of Y (row side) and Z, one fermion propagator */
  for (int d = 1; d < Q5_NTERM; ++d) {
    int X = Q5_MID[d][0], Y = Q5_MID[d][1], Z = Q5_MID[d][2];
    cx WY[4], WZ[4], G[4][4], S[4][4], x[4], t[4];
    for (int m = 0; m < 4; ++m) {
      WY[m] = (-I / k->inv[mk[Y]]) * J[Y][m];
      WZ[m] = (-I / k->inv[mk[Z]]) * J[Z][m];
    }
    /* B_X (-i g WYslash) i(qslash + m)/D (-i g WZslash) K_X, q = -(P_BX + Q_Y) */
    slash(WY, G);
    bra_mat(Bs[X], G, t);
    for (int r = 0; r < 4; ++r) x[r] = -I * gs * t[r];
    unsigned mB = (1u << k->B[X]) | mk[Y];
    cx qc[4];
    for (int m = 0; m < 4; ++m) qc[m] = -(Pin[k->B[X]][m] + Q[Y][m]);
    slash(qc, S);
    for (int r = 0; r < 4; ++r) S[r][r] += ms[X];
    double w = (X == 2 && !(zwt && is_tchannel(mB))) ? wt : 0.0;
    cx D = k->inv[mB] - ms[X] * ms[X] + I * ms[X] * w;
    bra_mat(x, S, t);
    for (int r = 0; r < 4; ++r) x[r] = I * t[r] / D;
    slash(WZ, G);
    bra_mat(x, G, t);
    A[d] = -I * gs * bra_ket(t, Ks[X]);
  }
}

static double q5_colour_sum(const cx* A, int nterm, const cx* Ginv, cx* Jf) {
  double m2 = 0;
  cx Pr[Q5_NFLOW];
  for (int n = 0; n < Q5_NFLOW; ++n) Pr[n] = 0;
  for (int x = 0; x < Q5_NCI; ++x) {
    cx M = 0;
    for (int d = 0; d < nterm; ++d) M += A[d] * Q5_DCOL[d][x];
    m2 += creal(M) * creal(M) + cimag(M) * cimag(M);
    for (int n = 0; n < Q5_NFLOW; ++n) Pr[n] += Q5_FLOW[n][x] * M;
  }
  for (int n = 0; n < Q5_NFLOW; ++n) {
    Jf[n] = 0;
    for (int m = 0; m < Q5_NFLOW; ++m) Jf[n] += Ginv[n * Q5_NFLOW + m] * Pr[m];
  }
  return m2;
}

static void q5_gram(cx* G) {
  for (int n = 0; n < Q5_NFLOW; ++n)
    for (int m = 0; m < Q5_NFLOW; ++m) {
      double s = 0;
      for (int x = 0; x < Q5_NCI; ++x) s += Q5_FLOW[n][x] * Q5_FLOW[m][x];
      G[n * Q5_NFLOW + m] = s;
    }
}

/* ------------------------------------------------------------------------- */
/* Driver                                                                     */
/* ------------------------------------------------------------------------- */
static int select_first_exceeding(const double* w, int n, double r) {
  double total = 0;
  for (int i = 0; i < n; ++i) total += w[i];
  if (!(total > 0)) return 0;
  double target = r * total, run = 0;
  for (int i = 0; i < n; ++i) {
    run += w[i];
    if (run > target) return i;
  }
  for (int i = n - 1; i >= 0; --i) if (w[i] > 0) return i;
  return 0;
}

/*
 * oracle_me: evaluate nevt events of process 'proc'.
 *   mom      [nevt][npar][4] FP64
 *   alphas   [nevt] or NULL (then par->alphas)
 *   rnd_hel, rnd_col [nevt] in (0,1) or NULL (then no selection is written)
 *   me       [nevt]                          (output, required)
 *   me_hel   [nevt][ncomb] or NULL           |M_h|^2 (before 1/IDEN)
 *   jamp     [nevt][ncomb][ncol][2] or NULL  colour-ordered amplitudes
 *   colw     [nevt][ncol] or NULL            w_i = sum_h |A_{h,i}|^2
 *   sel_hel, sel_col [nevt] or NULL
 *   gauge_leg: -1 normally; otherwise the particle index of one gluon whose
 *              polarisation is replaced by k/E (gauge check).
 * Returns 0, or -1 for a bad argument.
 */
int oracle_me(int proc, const oracle_params* par, int64_t nevt, const double* mom, const double* alphas,
              const double* rnd_hel, const double* rnd_col, double* me, double* me_hel, double* jamp,
              double* colw, int32_t* sel_hel, int32_t* sel_col, int gauge_leg) {
  if (proc < 0 || proc >= NPROC || nevt < 0 || !par || (nevt > 0 && (!mom || !me))) return -1;
  gamma_init();
  tgm_init();
  const proc_def* pd = &PROCS[proc];
  int npar = pd->npar, ncomb = 1 << npar, n = pd->ngluon;
  int ncol = pd->ncol;
  sm_derived sm;
  sm_derive(par, &sm);
  double* Cm = (double*)malloc(sizeof(double) * ncol * ncol);
  int64_t* cn = (int64_t*)malloc(sizeof(int64_t) * ncol * ncol);
  int64_t* cd = (int64_t*)malloc(sizeof(int64_t) * ncol * ncol);
  oracle_colour_matrix_exact(proc, cn, cd);
  for (int i = 0; i < ncol * ncol; ++i) Cm[i] = (double)cn[i] / (double)cd[i];
  free(cn);
  free(cd);
  int perms[MAXCOL][MAXG];
  for (int s = 0; s < ncol && n && pd->kind == 1; ++s) perm_unrank(n, s, perms[s]);
  cx Ginv[4][4];
  if (pd->kind == 3) {
    cx G[4][4];
    qg_colour_init();
    qg_gram(G);
    inv4(G, Ginv);
  }
  cx G5inv[Q5_NFLOW * Q5_NFLOW];
  if (pd->kind == 5 || pd->kind == 6) {
    cx G[Q5_NFLOW * Q5_NFLOW];
    q5_colour_init();
    q5_gram(G);
    invn(Q5_NFLOW, G, G5inv);
  }
  cx G4inv[Q4_NFLOW * Q4_NFLOW];
  if (pd->kind == 4) {
    cx G[Q4_NFLOW * Q4_NFLOW];
#pragma omp critical(q4_init)
    q4_colour_init();
    q4_gram(G);
    invn(Q4_NFLOW, G, G4inv);
  }

#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t e = 0; e < nevt; ++e) {
    const double* p = mom + e * npar * 4;
    double mh[1 << MAXPAR];
    double w[MAXCOL];
    for (int i = 0; i < ncol; ++i) w[i] = 0;
    double total = 0;
    double as = alphas ? alphas[e] : par->alphas;
    double gs = sqrt(4.0 * M_PI * as);
    invariants inv;
    qg_kin qk;
    q4_kin k4;
    q5_kin k5;
    if (pd->kind == 1) event_invariants(pd, p, par->mt, &inv);
    memset(&qk, 0, sizeof qk);
    if (pd->kind == 3) qg_kinematics(pd, p, par->mt, &qk);
    if (pd->kind == 4) q4_kinematics(pd, p, &k4);
    if (pd->kind == 5 || pd->kind == 6) q5_kinematics(pd, p, &k5);
    for (int h = 0; h < ncomb; ++h) {
      int lam[MAXPAR];
      for (int i = 0; i < npar; ++i) lam[i] = ((h >> (npar - 1 - i)) & 1) ? 1 : -1;
      cx A[MAXCOL];
      double m2 = 0;
      int explicit_colour = 0;
      if (pd->kind == 0) {
        A[0] = amp_eemumu(p, lam, par, &sm);
      } else if (pd->kind == 2) {
        m2 = qq_colour_sum(amp_qqbar_tt(p, lam, pd, gs, par->mt), A);
        explicit_colour = 1;
      } else if (pd->kind == 5 || pd->kind == 6) {
        cx D[2 * Q5_NTERM];
        q5_diagrams(p, lam, pd, &k5, gs, par->mt, par->wt, par->zero_width_tchan, D);
        int nterm = Q5_NTERM;
        if (pd->kind == 6) {
          /* the second pairing (column ends exchanged) enters with the relative sign -1 of
           * exchanging two identical fermions */
          q5_kin k2 = k5;
          k2.K[0] = k5.K[1];
          k2.K[1] = k5.K[0];
          q5_diagrams(p, lam, pd, &k2, gs, par->mt, par->wt, par->zero_width_tchan, D + Q5_NTERM);
          for (int d = 0; d < Q5_NTERM; ++d) D[Q5_NTERM + d] = -D[Q5_NTERM + d];
          nterm = 2 * Q5_NTERM;
        }
        m2 = q5_colour_sum(D, nterm, G5inv, A);
        explicit_colour = 1;
      } else if (pd->kind == 4) {
        cx D[Q4_MAXTERM];
        q4_diagrams(p, lam, pd, &k4, gs, par->mt, par->wt, par->zero_width_tchan, gauge_leg, D);
        m2 = q4_colour_sum(D, G4inv, A);
        explicit_colour = 1;
      } else if (pd->kind == 3) {
        cx D[5];
        qg_diagrams(p, lam, pd, &qk, gs, par->mt, par->wt, par->zero_width_tchan, gauge_leg, D);
        m2 = qg_colour_sum(D, Ginv, A);
        explicit_colour = 1;
      } else {
        qcd_ext x;
        int g = 0;
        for (int i = 0; i < npar; ++i) {
          const double* pi = p + 4 * i;
          int r = pd->role[i];
          if (r == R_G_IN || r == R_G_OUT) {
            cx e4[4];
            polvec(pi, lam[i], e4);
            for (int m = 0; m < 4; ++m) {
              x.eps[g][m] = (r == R_G_IN) ? e4[m] : conj(e4[m]);
              x.kin[g][m] = (r == R_G_IN) ? pi[m] : -pi[m];
            }
            if (i == gauge_leg)
              for (int m = 0; m < 4; ++m) x.eps[g][m] = pi[m] / pi[0];
            x.pidx[g] = i;
            ++g;
          } else if (r == R_T_OUT) {
            cx u[4];
            spinor_u(pi, par->mt, lam[i], u);
            dirac_bar(u, x.ubar_t);
            for (int m = 0; m < 4; ++m) x.pt[m] = pi[m];
            x.it = i;
          } else if (r == R_TBAR_OUT) {
            spinor_v(pi, par->mt, lam[i], x.v_tb);
          }
        }
        for (int s = 0; s < ncol; ++s)
          A[s] = amp_ordered(&x, &inv, n, perms[s], gs, par->mt, par->wt, par->zero_width_tchan);
      }
      if (!explicit_colour)
        for (int s = 0; s < ncol; ++s)
          for (int t = 0; t < ncol; ++t) m2 += Cm[s * ncol + t] * creal(conj(A[s]) * A[t]);
      mh[h] = m2;
      total += m2;
      for (int s = 0; s < ncol; ++s) w[s] += creal(A[s]) * creal(A[s]) + cimag(A[s]) * cimag(A[s]);
      if (jamp)
        for (int s = 0; s < ncol; ++s) {
          jamp[((e * ncomb + h) * ncol + s) * 2 + 0] = creal(A[s]);
          jamp[((e * ncomb + h) * ncol + s) * 2 + 1] = cimag(A[s]);
        }
    }
    me[e] = total / pd->iden;
    if (me_hel)
      for (int h = 0; h < ncomb; ++h) me_hel[e * ncomb + h] = mh[h];
    if (colw)
      for (int s = 0; s < ncol; ++s) colw[e * ncol + s] = w[s];
    if (sel_hel && rnd_hel) sel_hel[e] = select_first_exceeding(mh, ncomb, rnd_hel[e]);
    if (sel_col && rnd_col) sel_col[e] = select_first_exceeding(w, ncol, rnd_col[e]);
  }
  free(Cm);
  return 0;
}

/*
 * oracle_invariants: the propagator invariants the recursion of oracle_me uses, for
 * nevt events of a QCD process, indexed by particle mask (bit i = particle i):
 *   gsq  [nevt][2^npar]  K^2 of the gluons in the mask (incoming +p, outgoing -p)
 *   tden [nevt][2^npar]  q^2 - mt^2 with q = p_t - K(gluons in the mask)
 * Entries whose mask holds anything but gluons are 0.  Returns 0, or -1 for a bad
 * argument (e+ e- -> mu+ mu- has no such table).
 */
int oracle_invariants(int proc, const oracle_params* par, int64_t nevt, const double* mom, double* gsq,
                      double* tden) {
  if (proc <= 0 || proc >= NPROC || PROCS[proc].kind != 1 || nevt < 0 || !par || (nevt > 0 && (!mom || !gsq || !tden))) return -1;
  const proc_def* pd = &PROCS[proc];
  int ncomb = 1 << pd->npar;
  for (int64_t e = 0; e < nevt; ++e) {
    invariants inv;
    event_invariants(pd, mom + e * pd->npar * 4, par->mt, &inv);
    memcpy(gsq + e * ncomb, inv.gsq, sizeof(double) * ncomb);
    memcpy(tden + e * ncomb, inv.tden, sizeof(double) * ncomb);
  }
  return 0;
}
