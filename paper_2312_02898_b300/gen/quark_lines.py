"""Processes with one light-quark line, the top line and two gluons: q qbar -> t tbar g g
and its crossings (q g -> t tbar q g, qbar g -> t tbar qbar g, g g -> t tbar q qbar).

Build-time generator code.

Diagrams.  The objects are gluon a, gluon b (a has the lower particle index) and the pair
a b joined by a three-gluon vertex.  Each object sits on the light line, on the top line or
on the gluon joining the lines (the connector); the objects of a line and the connector's
end on it (the stub) come in every order.  The connector is a single propagator, a
three-gluon vertex carrying one object, two three-gluon vertices carrying a and b in either
order, or the four-gluon vertex (three colour-Lorentz structures, three terms): 36
diagrams, 38 terms.

Phases.  With the quark-gluon vertex -i g gamma T, fermion propagator i(qslash + m)/D,
gluon propagator -i/K^2, three-gluon vertex -g f V and four-gluon vertex -i g^2 (...), the
raw helas.cuh values pick up: +1 per fermion step (vertex and propagator), -i per stub
(pair current), i per joined pair, and from the connector -i (one propagator), +1 (one
three-gluon vertex), i (two three-gluon vertices or the four-gluon vertex).

Colour.  Every term's colour tensor over (B, K, t, y, a, b) -- light row end, light column
end, top, antitop, gluons -- is built from Gell-Mann matrices and solved for its
coefficients on the 13 flow tensors of flows() below.
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction

import numpy as np

from .colour import gell_mann_T

A, B_, AB, STUB = "a", "b", "ab", "S"


def terms():
    """[(light sequence from the row end, top sequence from the top, connector)]; the
    connector is 'prop', ('v3', obj), ('v3v3', first, second) or ('v4', s)"""
    out = []
    placements = [((A, pa), (B_, pb)) for pa in "LHC" for pb in "LHC"] + [((AB, p),) for p in "LHC"]
    for pl in placements:
        light = [o for o, p in pl if p == "L"] + [STUB]
        top = [o for o, p in pl if p == "H"] + [STUB]
        conn = [o for o, p in pl if p == "C"]
        if not conn:
            conns = ["prop"]
        elif len(conn) == 1:
            conns = [("v3", conn[0])]
        else:
            conns = [("v3v3", A, B_), ("v3v3", B_, A), ("v4", 1), ("v4", 2), ("v4", 3)]
        for lp in itertools.permutations(light):
            for hp in itertools.permutations(top):
                for c in conns:
                    out.append((tuple(lp), tuple(hp), c))
    return out


def _structure_constants(T):
    return np.real(-2j * (np.einsum("aij,bjk,cki->abc", T, T, T) - np.einsum("bij,ajk,cki->abc", T, T, T)))


def flows(T):
    d, d8, E = np.eye(3), np.eye(8), np.einsum
    return [E("aBm,bmy,tK->BKtyab", T, T, d), E("bBm,amy,tK->BKtyab", T, T, d),
            E("aBy,btK->BKtyab", T, T), E("bBy,atK->BKtyab", T, T),
            E("By,atm,bmK->BKtyab", d, T, T), E("By,btm,amK->BKtyab", d, T, T),
            E("aBm,bmK,ty->BKtyab", T, T, d), E("bBm,amK,ty->BKtyab", T, T, d),
            E("aBK,bty->BKtyab", T, T), E("bBK,aty->BKtyab", T, T),
            E("BK,atm,bmy->BKtyab", d, T, T), E("BK,btm,amy->BKtyab", d, T, T),
            E("ab,By,tK->BKtyab", d8, d, d)]


_LINE_CACHE = {}


def _line_colour(seq, T, f):
    """the line's colour string as a tensor [row, col, a, b, c(stub), e(joined pair)]"""
    if seq in _LINE_CACHE:
        return _LINE_CACHE[seq]
    m = np.zeros((3, 3, 8, 8, 8, 8), dtype=complex)
    for a, b, c, e in itertools.product(range(8), repeat=4):
        s = np.eye(3, dtype=complex)
        for o in seq:
            s = s @ T[{A: a, B_: b, AB: e, STUB: c}[o]]
        m[:, :, a, b, c, e] = s
    _LINE_CACHE[seq] = m
    return m


def term_colour(term, T, f):
    light, top, conn = term
    Lc, Hc = _line_colour(light, T, f), _line_colour(top, T, f)
    joined = AB in light or AB in top or conn == ("v3", AB)
    d8 = np.eye(8)
    # connector factor over (a, b, c1, c2, e)
    if conn == "prop":
        K = np.einsum("ab,cd,e->abcde", np.ones((8, 8)), d8, np.ones(8))
    elif conn[0] == "v3":
        x = conn[1]
        if x == A:
            K = np.einsum("cad,b,e->abcde", f, np.ones(8), np.ones(8))
        elif x == B_:
            K = np.einsum("cbd,a,e->abcde", f, np.ones(8), np.ones(8))
        else:
            K = np.einsum("ced,abe->abcde", f, f)
    elif conn[0] == "v3v3":
        K = np.einsum("cae,ebd->abcde", f, f) if conn[1] == A else np.einsum("cbe,ead->abcde", f, f)
    else:
        s = conn[1]
        K = {1: np.einsum("cae,bde->abcde", f, f), 2: np.einsum("cbe,ade->abcde", f, f),
             3: np.einsum("cde,abe->abcde", f, f)}[s]
    if joined and conn != ("v3", AB):  # (the v3 connector with the pair carries f^{abe} already)
        K = K * f[:, :, None, None, :]  # f^{abe} of the joined pair
    uses_e = joined or (conn != "prop" and conn[0] in ("v3v3", "v4"))
    if not uses_e:
        K = K[..., :1]
        Lc, Hc = Lc[..., :1], Hc[..., :1]
    # light stub colour c1, top stub colour c2; e shared
    return np.einsum("BKabce,tyabde,abcde->BKtyab", Lc, Hc, K)


def colour_coefficients():
    """(flow coefficients of every term, scaled to Gaussian integers, the scale, the Gram
    matrix of the flows as exact fractions)"""
    T = gell_mann_T()
    f = _structure_constants(T)
    Fm = np.stack([x.ravel() for x in flows(T)], axis=1)
    coef = []
    for t in terms():
        x = term_colour(t, T, f).ravel()
        c = np.linalg.lstsq(Fm, x, rcond=None)[0]
        if np.abs(Fm @ c - x).max() > 1e-10:
            raise RuntimeError(f"colour of term {t} is not in the span of the flows")
        coef.append(c)
    coef = np.array(coef)
    scale = None
    for s in (1, 2, 3, 4, 6, 12, 24, 36, 48, 72):
        cs = coef * s
        if np.abs(cs - np.round(cs.real) - 1j * np.round(cs.imag)).max() < 1e-9:
            scale = s
            break
    if scale is None:
        raise RuntimeError("flow coefficients are not multiples of 1/72")
    ci = np.round(coef.real * scale) + 1j * np.round(coef.imag * scale)
    G = Fm.conj().T @ Fm
    if np.abs(G.imag).max() > 1e-9:
        raise RuntimeError("flow Gram matrix is not real")
    Gf = [[Fraction(round(v * 9)) / 9 for v in row] for row in G.real]
    for i in range(13):
        for j in range(13):
            if abs(float(Gf[i][j]) - G.real[i, j]) > 1e-9:
                raise RuntimeError("flow Gram matrix is not a multiple of 1/9")
    return ci, scale, Gf


# ----------------------------------------------------------------------------
# code emission
# ----------------------------------------------------------------------------
# real-flop counts of the helas.cuh calls (as in emit.py)
_FL = {"ext": 40, "eps": 30, "g3": 170, "step": 160, "pj": 72, "dot": 30, "v3": 194, "v4": 136, "scale": 2, "add": 2}

CONN_PHASE = {"prop": -1j, "v3": 1, "v3v3": 1j, "v4": 1j}


def emit(em):
    """(header text, stats) for the process of Emitter em"""
    roles, npar, tag = em.roles, em.npar, em.tag
    ib = next(i for i, r in enumerate(roles) if r in ("qb_in", "q_out"))   # light row end
    ik = next(i for i, r in enumerate(roles) if r in ("q_in", "qb_out"))   # light column end
    ga, gb = (i for i, r in enumerate(roles) if r in ("g_in", "g_out"))
    it, itb = roles.index("t"), roles.index("tb")

    def parts(S, sign=1):
        """signed incoming momenta summing to sign * P(S), particle order"""
        out = []
        for i in sorted(S):
            s = 1 if roles[i].endswith("_in") else -1
            out.append(("+" if s * sign > 0 else "-", i))
        return tuple(out)

    # An invariant is formed from the particle set its momentum is routed from (a line's
    # end for a fermion propagator, each line's side for the gluon between the lines),
    # not from the complementary set: with inputs that conserve momentum only to
    # rounding the two sums differ by O(eps E^2), which near a pole is visible.
    def canon(S):
        return frozenset(S)

    kvec, dgs, dts = {}, {}, {}

    def kv(S, sign=1):
        key = parts(S, sign)
        if key not in kvec:
            kvec[key] = npar + len(kvec)
        return f"(kt + {kvec[key]} * S)"

    def dg(S):
        key = canon(S)
        if key not in dgs:
            dgs[key] = len(dgs)
        return f"dg[{dgs[key]}]"

    def dt(S, massive):
        key = (canon(S), massive)
        if key not in dts:
            dts[key] = len(dts)
        return f"dt[{dts[key]}]"

    objset = {A: frozenset([ga]), B_: frozenset([gb]), AB: frozenset([ga, gb])}
    objw = {A: f"x{ga}", B_: f"x{gb}", AB: "wab"}
    fl = {"n": 0}

    def flop(k, n=1):
        fl["n"] += _FL[k] * n

    body = [f"  int lam[{npar}];",
            f"  for (int i = 0; i < {npar}; ++i) lam[i] = ((h >> ({npar - 1} - i)) & 1) ? 1 : -1;",
            "  " + " ".join(f"cx<R> x{i}[4];" for i in range(npar))]
    for i, r in enumerate(roles):
        ktp = f"(kt + {i} * S)"
        if r == "q_in":
            body.append(f"  ext_u<R>({ktp}, R(0), lam[{i}], x{i});")
        elif r == "qb_in":
            body.append(f"  ext_vbar<R>({ktp}, R(0), lam[{i}], x{i});")
        elif r == "q_out":
            body.append(f"  ext_ubar<R>({ktp}, R(0), lam[{i}], x{i});")
        elif r == "qb_out":
            body.append(f"  ext_v<R>({ktp}, R(0), lam[{i}], x{i});")
        elif r in ("g_in", "g_out"):
            body.append(f"  ext_eps<R>({ktp}, lam[{i}], {'true' if r == 'g_out' else 'false'}, x{i});")
        elif r == "t":
            body.append(f"  ext_ubar<R>({ktp}, mt, lam[{i}], x{i});")
        else:
            body.append(f"  ext_v<R>({ktp}, mt, lam[{i}], x{i});")
        flop("eps" if r.startswith("g") else "ext")
    body.append(f"  cx<R> wab[4]; g3_current<R>(x{ga}, {kv(objset[A])}, x{gb}, {kv(objset[B_])}, "
                f"{dg(objset[AB])}, wab);  // the joined pair")
    flop("g3")

    coef, scale, gram = colour_coefficients()
    tl = terms()
    by_place = {}
    for d, (light, top, conn) in enumerate(tl):
        key = (tuple(sorted(o for o in light if o != STUB)), tuple(sorted(o for o in top if o != STUB)))
        by_place.setdefault(key, []).append(d)
    npairs = 0
    # every distinct fermion-chain prefix and line current is computed once (the same
    # values recur across placements), so the code and its flop count describe the work
    # that runs
    memo = {}
    cnt = {"v": 0}
    for key, ds in by_place.items():

        def newvar(prefix):
            cnt["v"] += 1
            return f"{prefix}{cnt['v']}"

        def chain(side, massive, row, col, seq):
            """vector current of a line with insertions seq (row end first), the stub inside"""
            mkey = (side, seq)
            if mkey in memo:
                return memo[mkey]
            s = seq.index(STUB)
            m = "mt" if massive else "R(0)"
            # row side: bra steps
            x, Sx = f"x{row}", frozenset([row])
            for j in range(s):
                pre = (side, "B", seq[:j + 1])
                Sx = Sx | objset[seq[j]]
                if pre in memo:
                    x = memo[pre]
                    continue
                v = newvar("b")
                body.append(f"    cx<R> {v}[4]; bra_step<R>({x}, {objw[seq[j]]}, {kv(Sx, -1)}, {m}, {dt(Sx, massive)}, {v});")
                flop("step")
                memo[pre] = v
                x = v
            y, Sy = f"x{col}", frozenset([col])
            for j in range(len(seq) - 1, s, -1):
                pre = (side, "K", seq[j:])
                Sy = Sy | objset[seq[j]]
                if pre in memo:
                    y = memo[pre]
                    continue
                v = newvar("k")
                body.append(f"    cx<R> {v}[4]; ket_step<R>({objw[seq[j]]}, {y}, {kv(Sy)}, {m}, {dt(Sy, massive)}, {v});")
                flop("step")
                memo[pre] = v
                y = v
            v = newvar("L" if side == "L" else "H")
            body.append(f"    cx<R> {v}[4]; pair_current<R>({x}, {y}, {v});")
            flop("pj")
            S = frozenset([row, col]).union(*[objset[o] for o in seq if o != STUB])
            memo[mkey] = (v, S)
            return memo[mkey]

        for d in ds:
            light, top, conn = tl[d]
            L, SL = chain("L", False, ib, ik, light)
            H, SH = chain("H", True, it, itb, top)
            if conn == "prop":
                expr = f"{dg(SL)} * mdot({L}, {H})"
                flop("dot")
                flop("scale")
                ph = CONN_PHASE["prop"]
            elif conn[0] == "v3":
                x = conn[1]
                expr = f"{dg(SH)} * close_v3<R>({H}, {L}, {kv(SL)}, {objw[x]}, {kv(objset[x])}, {dg(SL)})"
                flop("v3")
                flop("scale")
                ph = CONN_PHASE["v3"]
            elif conn[0] == "v3v3":
                x1, x2 = conn[1], conn[2]
                Se = SL | objset[x1]
                je = newvar("e")
                body.append(f"    cx<R> {je}[4]; g3_current<R>({L}, {kv(SL)}, {objw[x1]}, {kv(objset[x1])}, {dg(Se)}, {je});")
                flop("g3")
                expr = f"{dg(SL)} * close_v3<R>({H}, {je}, {kv(Se)}, {objw[x2]}, {kv(objset[x2])}, {dg(SH)})"
                flop("v3")
                flop("scale")
                ph = CONN_PHASE["v3v3"]
            else:
                expr = f"{dg(SL)} * close_v4<{conn[1]}, R>({H}, {L}, {objw[A]}, {objw[B_]}, {dg(SH)})"
                flop("v4")
                flop("scale")
                ph = CONN_PHASE["v4"]
            joined = AB in light or AB in top or conn == ("v3", AB)
            ph = ph * (-1j) * (-1j) * (1j if joined else 1)
            ops, mags = [], set()
            for n in range(13):
                k = complex(coef[d][n]) * ph
                k = complex(round(k.real), round(k.imag))
                if k == 0:
                    continue
                mag = int(abs(k.real) + abs(k.imag))
                unit = k / mag
                src = "a" if mag == 1 else f"a{mag}"
                if mag != 1:
                    mags.add(mag)
                ops.append({1: f"J[{n}] += {src};", -1: f"J[{n}] -= {src};", 1j: f"acc_pi(J[{n}], {src});",
                            -1j: f"acc_mi(J[{n}], {src});"}[unit])
                flop("add")
                npairs += 1
            pre = "".join(f" const cx<R> a{m} = R({m}) * a;" for m in sorted(mags))
            flop("scale", len(mags))
            body.append(f"    {{ const cx<R> a = {expr};{pre} {' '.join(ops)} }}")
    return body, dict(kvec=kvec, dgs=dgs, dts=dts, flops=fl["n"], pairs=npairs, scale=scale, gram=gram,
                      parts=parts, ncol=13, ndiag=36, namp=38)


def header(em):
    """the generated proc_<tag>.cuh text and its stats (one light-quark line and two
    gluons, or two light-quark lines of different flavours)"""
    from .emit import _lit
    three = sum(1 for r in em.roles if r.split("_")[0] in ("q", "qb", "d", "db")) == 4
    body, st = emit3(em) if three else emit(em)
    ncol, ndiag, namp = st["ncol"], st["ndiag"], st["namp"]
    roles, npar, tag = em.roles, em.npar, em.tag
    parts = st["parts"]
    # IDEN: initial spins x initial colours x (identical final gluons)!
    ncolour = 1
    for r in roles:
        if r.endswith("_in"):
            ncolour *= 8 if r == "g_in" else 3
    iden = 4 * ncolour
    for r in set(roles):
        if r.endswith("_out"):
            iden *= math.factorial(sum(1 for x in roles if x == r))
    # colour matrix: flows carried times scale, so |M|^2 = J'^+ G J' / scale^2
    scale = st["scale"]
    G = st["gram"]
    den = scale * scale
    lcm = 1
    for row in G:
        for g in row:
            lcm = lcm * g.denominator // math.gcd(lcm, g.denominator)
    cf = [[int(g * lcm) for g in row] for row in G]
    cden = den * lcm
    gg = 0
    for row in cf:
        for v in row:
            gg = math.gcd(gg, v)
    gg = math.gcd(gg, cden)
    cf = [[v // gg for v in row] for row in cf]
    cden //= gg

    den_lines = ["  using DD = dd_for<R>;", "  DD q[4];",
                 "  double kappa = 0.0;  // conditioning: max over light-quark and gluon invariants of (sum E)^2 / |K^2|"]

    def dd_sum(pp):
        out = []
        for mu in range(4):
            s0, i0 = pp[0]
            e = f"DD{{{'-' if s0 == '-' else ''}p[{i0}][{mu}], 0.0}}"
            for sgn, i in pp[1:]:
                e = f"dd_add({e}, {'-' if sgn == '-' else ''}p[{i}][{mu}])"
            out.append(f"  q[{mu}] = {e};")
        return out

    for S, idx in sorted(st["dgs"].items(), key=lambda t: t[1]):
        pp = parts(S)
        es = " + ".join(f"p[{i}][0]" for _, i in pp)
        den_lines += dd_sum(pp)
        den_lines.append(f"  {{ const double k2 = dd_invariant(q, 0.0), es = {es};")
        den_lines.append(f"    dg[{idx}] = R(1.0 / k2); kappa = fmax(kappa, es * es / fabs(k2)); }}")
    for (S, massive), idx in sorted(st["dts"].items(), key=lambda t: t[1]):
        pp = parts(S)
        den_lines += dd_sum(pp)
        if massive:
            mask = sum(1 << i for i in S)
            tchan = (mask & 1) != ((mask >> 1) & 1)
            den_lines.append(f"  {{ const double w = {'(zwt ? 0.0 : wt)' if tchan else 'wt'};")
            den_lines.append("    const double re = dd_invariant(q, mt);")
            den_lines.append("    const double im = mt * w, inv = 1.0 / (re * re + im * im);")
            den_lines.append(f"    dt[{idx}] = mk<R>(R(re * inv), R(-im * inv)); }}")
        else:
            es = " + ".join(f"p[{i}][0]" for _, i in pp)
            den_lines.append(f"  {{ const double k2 = dd_invariant(q, 0.0), es = {es};")
            den_lines.append(f"    dt[{idx}] = mk<R>(R(1.0 / k2), R(0)); kappa = fmax(kappa, es * es / fabs(k2)); }}")
    den_lines.append("  // momentum table: external momenta, then the vectors the vertices use")
    den_lines.append(f"  for (int i = 0; i < {npar}; ++i)")
    den_lines.append("    for (int m = 0; m < 4; ++m) kt[i * S + m] = R(p[i][m]);")
    for key, idx in sorted(st["kvec"].items(), key=lambda t: t[1]):
        for mu in range(4):
            den_lines.append(f"  kt[{idx} * S + {mu}] = R({em._sum_expr(list(key), mu)});")
    nk = npar + len(st["kvec"])

    cs, csflops = [], 0

    def fused(tt):
        e = f"{tt[-1][0]} * {tt[-1][1]}"
        for a_, b_ in reversed(tt[:-1]):
            e = f"fmadd({a_}, {b_}, {e})"
        return e

    for i in range(ncol):
        tr, ti = [], []
        for j in range(i, ncol):
            c = cf[i][j] * (1 if j == i else 2)
            if c == 0:
                continue
            tr.append((_lit(c), f"J[{j}].r"))
            ti.append((_lit(c), f"J[{j}].i"))
            csflops += 4
        cs.append(f"  {{ const R tr = {fused(tr)}; const R ti = {fused(ti)};")
        cs.append(f"    s = fmadd(J[{i}].r, tr, fmadd(J[{i}].i, ti, s)); }}")
        csflops += 4
    out = [f"// Generated by paper_2312_02898_b300/gen/quark_lines.py for '{em.process}'. Do not edit.",
           "#pragma once", '#include "../helas.cuh"', "namespace meb300 {", f"struct proc_{tag} {{",
           f'static constexpr const char* NAME = "{em.process}";',
           "// NGLUON counts the powers of g_s^2 in |M|^2 (four QCD vertices)",
           f"static constexpr int NPAR = {npar}, NCOMB = {1 << npar}, NCOL = {ncol}, NDIAG = {ndiag}, NAMP = {namp}, NNODE = 0, "
           f"IDEN = {iden}, NGLUON = 4;",
           f"static constexpr int NDEN_G = {len(st['dgs'])}, NDEN_T = {len(st['dts'])}, COL_DEN = {cden}, "
           f"NCOLPAIR = {st['pairs']}, MAX_LIVE = 8, NKVEC = {nk};",
           f"static constexpr long FLOPS_AMP = {st['flops']}, FLOPS_COL = {csflops};",
           "static constexpr bool QCD = true;",
           "static constexpr bool CF_BF16_EXACT = false, CF_FP16_EXACT = false;  // (no tensor-core path)",
           "// dg: 1/K^2 of the gluon propagators; dt: 1/q^2 of the light-quark propagators and",
           "// 1/(q^2 - mt^2 + i mt wt) of the top propagators (by particle set)",
           "template <int S, class R, class DG, class DT, class KT>",
           "static HD double precompute(const double (*p)[4], double mt, double wt, int zwt, DG& dg, DT& dt, KT kt) {"]
    out += den_lines
    out += ["  return kappa;", "}",
            "static constexpr int NVARIANT = 1;",
            "static constexpr int NSLOT[1] = {0};",
            "template <int V> static HD constexpr int nslot() { return 0; }",
            "template <int V> static HD constexpr bool grouped() { return false; }",
            "static constexpr int BUDGET[1] = {-1};",
            "template <int V, int S, class R, int SYNC = 0, class DG, class DT, class JA>",
            "static HD void jamps(int h, R mt, const DG& dg, const DT& dt, JA& J, cx<R>*, const R* kt) {"]
    out += body
    out += ["}", "template <class R, class JA>", "static HD R colour_sum(JA& J) {", "  R s = R(0);"] + cs
    out += ["  return s;", "}", "};",
            f"constexpr int proc_{tag}_CF[{ncol * ncol}] = {{{', '.join(str(v) for row in cf for v in row)}}};",
            "}  // namespace meb300"]
    stats = dict(ndiag=ndiag, namp=namp, nnode=0, ncol=ncol, pairs=st["pairs"], flops_amp=st["flops"], flops_col=csflops,
                 nden_g=len(st["dgs"]), nden_t=len(st["dts"]), col_den=cden, max_live=8, iden=iden)
    return "\n".join(out) + "\n", stats


# ----------------------------------------------------------------------------
# two light-quark lines of different flavours and the top line
# ----------------------------------------------------------------------------
# terms: 0 the three-gluon vertex joining the three lines; then line X carrying the
# currents of Y (nearer X's row end) and Z, for (X, Y, Z) in this order
MIDDLE = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


def three_line_colour(swap=False):
    """(flow coefficients of the 7 terms scaled to Gaussian integers, the scale, the Gram
    matrix of the 6 flows).  Indices (B0, K0, B1, K1, t, y): row and column ends of the
    two light lines and the top line; flows d_{B0 K_s0} d_{B1 K_s1} d_{t K_s2} for the
    permutations s of (K0, K1, y) in lexicographic order.  With swap the light lines are
    (B0, K1) and (B1, K0): the second pairing of one light flavour."""
    T = gell_mann_T()
    f = _structure_constants(T)
    d = np.eye(3)
    perms = list(itertools.permutations(range(3)))
    flows3 = []
    for s in perms:
        x = np.zeros((3,) * 6)
        for B0, K0, B1, K1, t, y in itertools.product(range(3), repeat=6):
            K = (K0, K1, y)
            x[B0, K0, B1, K1, t, y] = d[B0, K[s[0]]] * d[B1, K[s[1]]] * d[t, K[s[2]]]
        flows3.append(x.ravel())
    Fm = np.array(flows3).T
    letters = ("BK", "CL", "ty")  # index letters of the rows/columns of lines 0, 1, 2
    tens = [np.einsum("abc,aBK,bCL,cty->BKCLty", f, T, T, T)]
    for X, Y, Z in MIDDLE:
        # gluon colours: g joins X and Y, h joins X and Z
        spec = {X: f"g{letters[X][0]}m,hm{letters[X][1]}", Y: f"g{letters[Y]}", Z: f"h{letters[Z]}"}
        tens.append(np.einsum(f"{spec[X]},{spec[Y]},{spec[Z]}->BKCLty", T, T, T, T))
    coef = []
    for x in tens:
        if swap:
            x = np.swapaxes(x, 1, 3)  # K0 <-> K1
        c = np.linalg.lstsq(Fm, x.ravel(), rcond=None)[0]
        if np.abs(Fm @ c - x.ravel()).max() > 1e-10:
            raise RuntimeError("colour of a three-line term is not in the span of the flows")
        coef.append(c)
    coef = np.array(coef)
    for scale in (1, 2, 3, 4, 6, 12, 24, 36):
        cs = coef * scale
        if np.abs(cs - np.round(cs.real) - 1j * np.round(cs.imag)).max() < 1e-9:
            break
    else:
        raise RuntimeError("three-line flow coefficients are not multiples of 1/36")
    ci = np.round(coef.real * scale) + 1j * np.round(coef.imag * scale)
    G = Fm.T @ Fm
    return ci, scale, [[Fraction(int(round(v))) for v in row] for row in G]


def emit3(em):
    """(jamps body, stats) for two light-quark lines and the top line.  With two flavours
    the lines are the u line and the d line; with one flavour the row ends (B0 < B1) and
    column ends (K0 < K1) of the light quarks pair up both ways, (B0 K0)(B1 K1) and
    (B0 K1)(B1 K0), the second pairing with the sign -1 of exchanging identical
    fermions."""
    roles, npar = em.roles, em.npar
    line_of = {"q": 0, "qb": 0, "d": 1, "db": 1, "t": 2, "tb": 2}
    row_roles = ("qb_in", "q_out", "db_in", "d_out", "t")
    same = not any(r.startswith("d") for r in roles)
    B, K = [None] * 3, [None] * 3
    rows, cols = [], []
    for i, r in enumerate(roles):
        ln = line_of[r.split("_")[0]]
        if same and ln < 2:
            (rows if r in row_roles else cols).append(i)
            continue
        if r in row_roles:
            B[ln] = i
        else:
            K[ln] = i
    if same:
        B[0], B[1] = rows
        K[0], K[1] = cols

    def parts(S, sign=1):
        out = []
        for i in sorted(S):
            s = 1 if roles[i].endswith("_in") else -1
            out.append(("+" if s * sign > 0 else "-", i))
        return tuple(out)

    kvec, dgs, dts = {}, {}, {}

    def kv(S, sign=1):
        key = parts(S, sign)
        if key not in kvec:
            kvec[key] = npar + len(kvec)
        return f"(kt + {kvec[key]} * S)"

    def dg(S):
        S = frozenset(S)
        if S not in dgs:
            dgs[S] = len(dgs)
        return f"dg[{dgs[S]}]"

    def dt(S, massive):
        key = (frozenset(S), massive)
        if key not in dts:
            dts[key] = len(dts)
        return f"dt[{dts[key]}]"

    fl = {"n": 0}

    def flop(k, n=1):
        fl["n"] += _FL[k] * n

    body = [f"  int lam[{npar}];",
            f"  for (int i = 0; i < {npar}; ++i) lam[i] = ((h >> ({npar - 1} - i)) & 1) ? 1 : -1;",
            "  " + " ".join(f"cx<R> x{i}[4];" for i in range(npar))]
    for i, r in enumerate(roles):
        ktp, m = f"(kt + {i} * S)", "mt" if r in ("t", "tb") else "R(0)"
        fn = {"q_in": "ext_u", "d_in": "ext_u", "qb_in": "ext_vbar", "db_in": "ext_vbar", "q_out": "ext_ubar",
              "d_out": "ext_ubar", "t": "ext_ubar", "qb_out": "ext_v", "db_out": "ext_v", "tb": "ext_v"}[r]
        body.append(f"  {fn}<R>({ktp}, {m}, lam[{i}], x{i});")
        flop("ext")
    body.append(f"  cx<R> J2[4]; pair_current<R>(x{B[2]}, x{K[2]}, J2);")
    flop("pj")
    amps = []
    coefs = []
    for pr in ((0, 1) if same else (0,)):
        Kp = [K[1], K[0], K[2]] if pr else list(K)
        sfx = "x" if pr else ""
        sign = -1 if pr else 1
        lines = [frozenset([B[l], Kp[l]]) for l in range(3)]
        J = [f"J0{sfx}", f"J1{sfx}", "J2"]
        for l in range(2):
            body.append(f"  cx<R> {J[l]}[4]; pair_current<R>(x{B[l]}, x{Kp[l]}, {J[l]});")
            flop("pj")
        coef, scale, gram = three_line_colour(swap=bool(pr))
        coefs += list(coef)
        # term 0: the three-gluon vertex; phases -i per line current (3), -i per gluon
        # propagator (3), -1 for the vertex -g f V: +1 overall
        amps.append((f"{dg(lines[1])} * {dg(lines[2])} * close_v3<R>({J[2]}, {J[0]}, {kv(lines[0])}, {J[1]}, "
                     f"{kv(lines[1])}, {dg(lines[0])})", sign))
        flop("v3")
        flop("scale", 2)
        for n, (X, Y, Z) in enumerate(MIDDLE):
            # line X: the current of Y enters nearer its row end, one fermion propagator, the
            # current of Z; phases -i (Y), -i (Z), +1 (step), -i (last vertex), -i -i (gluon
            # propagators): -i overall
            SX = frozenset([B[X]]) | lines[Y]
            m = "mt" if X == 2 else "R(0)"
            body.append(f"  cx<R> c{n}{sfx}[4]; bra_step<R>(x{B[X]}, {J[Y]}, {kv(SX, -1)}, {m}, {dt(SX, X == 2)}, "
                        f"c{n}{sfx});")
            body.append(f"  cx<R> v{n}{sfx}[4]; pair_current<R>(c{n}{sfx}, x{Kp[X]}, v{n}{sfx});")
            flop("step")
            flop("pj")
            amps.append((f"{dg(lines[Y])} * {dg(lines[Z])} * mdot(v{n}{sfx}, {J[Z]})", -1j * sign))
            flop("dot")
            flop("scale", 2)
    coef = coefs
    npairs = 0
    for d, (expr, ph) in enumerate(amps):
        ops, mags = [], set()
        for n in range(6):
            k = complex(coef[d][n]) * ph
            k = complex(round(k.real), round(k.imag))
            if k == 0:
                continue
            mag = int(abs(k.real) + abs(k.imag))
            unit = k / mag
            src = "a" if mag == 1 else f"a{mag}"
            if mag != 1:
                mags.add(mag)
            ops.append({1: f"J[{n}] += {src};", -1: f"J[{n}] -= {src};", 1j: f"acc_pi(J[{n}], {src});",
                        -1j: f"acc_mi(J[{n}], {src});"}[unit])
            flop("add")
            npairs += 1
        pre = "".join(f" const cx<R> a{m} = R({m}) * a;" for m in sorted(mags))
        flop("scale", len(mags))
        body.append(f"  {{ const cx<R> a = {expr};{pre} {' '.join(ops)} }}")
    nd = 14 if same else 7
    return body, dict(kvec=kvec, dgs=dgs, dts=dts, flops=fl["n"], pairs=npairs, scale=scale, gram=gram,
                      parts=parts, ncol=6, ndiag=nd, namp=nd)
