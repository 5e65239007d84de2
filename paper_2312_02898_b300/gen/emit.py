"""Emit the per-process device code (straight-line CUDA over the helas.cuh routines).

Build-time generator code.  For each process it writes ``proc_<tag>.cuh`` holding a
struct ``proc_<tag>`` with

  * constants: NPAR, NCOMB, NCOL, NDIAG (Feynman diagrams, four-gluon vertices counted
    once), NAMP (diagram terms: a four-gluon vertex gives three), NNODE (off-shell
    currents per helicity), IDEN, NGLUON, the number of gluon / top propagator
    denominators, the colour-matrix denominator and the flop counts of one helicity;
  * denominators<R>(): every distinct propagator denominator, evaluated in FP64 from
    the FP64 momenta once per event (1/K^2 for gluons, 1/(q^2 - m^2 + i m w) for tops)
    and stored in the working precision R;
  * jamps<R>(): for one helicity, the external wavefunctions, the off-shell currents
    and the diagram terms, each added to its colour flows with a coefficient in
    {+-1, +-i} (no multiplications);
  * colour_sum<R>(): sum_ij CF_ij Re(J_i^* J_j) using the symmetry of CF;

plus the integer colour matrix proc_<tag>_CF.
"""
from __future__ import annotations

import math
import os

from . import colour as colmod
from . import diagrams as dg
from . import schedule as sc

# Processes: particle roles in the order of the process string.
PROCESSES = {
    "e+ e- > mu+ mu-": dict(tag="eemumu", roles=("ebar_in", "e_in", "mubar_out", "mu_out")),
    "g g > t t~": dict(tag="ggtt", roles=("g_in", "g_in", "t", "tb")),
    "g g > t t~ g": dict(tag="ggttg", roles=("g_in", "g_in", "t", "tb", "g_out")),
    "g g > t t~ g g": dict(tag="ggttgg", roles=("g_in", "g_in", "t", "tb", "g_out", "g_out")),
    "g g > t t~ g g g": dict(tag="ggttggg", roles=("g_in", "g_in", "t", "tb", "g_out", "g_out", "g_out")),
    # the quark-initiated channel of p p -> t t~ (any light flavour; either beam order)
    "u u~ > t t~": dict(tag="qqtt", roles=("q_in", "qb_in", "t", "tb")),
    "u~ u > t t~": dict(tag="qxqtt", roles=("qb_in", "q_in", "t", "tb")),
    # the one-jet quark channels of p p -> t t~ + jet (with g g -> t t~ g)
    "u u~ > t t~ g": dict(tag="qqttg", roles=("q_in", "qb_in", "t", "tb", "g_out")),
    "u~ u > t t~ g": dict(tag="qxqttg", roles=("qb_in", "q_in", "t", "tb", "g_out")),
    "u g > t t~ u": dict(tag="qgttq", roles=("q_in", "g_in", "t", "tb", "q_out")),
    "g u > t t~ u": dict(tag="gqttq", roles=("g_in", "q_in", "t", "tb", "q_out")),
    "u~ g > t t~ u~": dict(tag="qxgttqx", roles=("qb_in", "g_in", "t", "tb", "qb_out")),
    "g u~ > t t~ u~": dict(tag="gqxttqx", roles=("g_in", "qb_in", "t", "tb", "qb_out")),
}
QUARK_JET_TAGS = ("qqttg", "qxqttg", "qgttq", "gqttq", "qxgttqx", "gqxttqx")
# the two-jet channels with one light-quark line (gen/quark_lines.py)
PROCESSES.update({
    "u u~ > t t~ g g": dict(tag="qqttgg", roles=("q_in", "qb_in", "t", "tb", "g_out", "g_out")),
    "u~ u > t t~ g g": dict(tag="qxqttgg", roles=("qb_in", "q_in", "t", "tb", "g_out", "g_out")),
    "u g > t t~ u g": dict(tag="qgttqg", roles=("q_in", "g_in", "t", "tb", "q_out", "g_out")),
    "g u > t t~ u g": dict(tag="gqttqg", roles=("g_in", "q_in", "t", "tb", "q_out", "g_out")),
    "u~ g > t t~ u~ g": dict(tag="qxgttqxg", roles=("qb_in", "g_in", "t", "tb", "qb_out", "g_out")),
    "g u~ > t t~ u~ g": dict(tag="gqxttqxg", roles=("g_in", "qb_in", "t", "tb", "qb_out", "g_out")),
    "g g > t t~ u u~": dict(tag="ggttqqx", roles=("g_in", "g_in", "t", "tb", "q_out", "qb_out")),
})
# the four-quark channels with two light flavours (gen/quark_lines.py, three lines)
PROCESSES.update({
    "u u~ > t t~ d d~": dict(tag="uuxttddx", roles=("q_in", "qb_in", "t", "tb", "d_out", "db_out")),
    "u~ u > t t~ d d~": dict(tag="uxuttddx", roles=("qb_in", "q_in", "t", "tb", "d_out", "db_out")),
    "u d > t t~ u d": dict(tag="udttud", roles=("q_in", "d_in", "t", "tb", "q_out", "d_out")),
    "u d~ > t t~ u d~": dict(tag="udxttudx", roles=("q_in", "db_in", "t", "tb", "q_out", "db_out")),
    "u~ d~ > t t~ u~ d~": dict(tag="uxdxttuxdx", roles=("qb_in", "db_in", "t", "tb", "qb_out", "db_out")),
    # one light flavour: both pairings of the light quarks
    "u u > t t~ u u": dict(tag="uuttuu", roles=("q_in", "q_in", "t", "tb", "q_out", "q_out")),
    "u~ u~ > t t~ u~ u~": dict(tag="uxuxttuxux", roles=("qb_in", "qb_in", "t", "tb", "qb_out", "qb_out")),
    "u u~ > t t~ u u~": dict(tag="uuxttuux", roles=("q_in", "qb_in", "t", "tb", "q_out", "qb_out")),
    "u~ u > t t~ u u~": dict(tag="uxuttuux", roles=("qb_in", "q_in", "t", "tb", "q_out", "qb_out")),
})
QUARK_JET2_TAGS = ("qqttgg", "qxqttgg", "qgttqg", "gqttqg", "qxgttqxg", "gqxttqxg", "ggttqqx",
                   "uuxttddx", "uxuttddx", "udttud", "udxttudx", "uxdxttuxdx", "uuttuu", "uxuxttuxux", "uuxttuux",
                   "uxuttuux")

# jamps variants per process: (register budget, diagram-group size[, pending colour
# accumulators]).  The budget is the number of currents kept in registers (None: all); a
# group size splits the emission sequence into out-of-line functions of that many steps
# (diagram groups), with every value that crosses a group boundary passed through the slot
# buffer.  With P pending accumulators, amplitudes whose colour vectors agree up to a
# factor 1, i, -1 or -i are summed in registers before they are added into J (see
# _pending_plan).
VARIANTS = {
    "ggtt": ((None, None),),
    "ggttg": ((None, None), (6, None)),
    "ggttgg": ((None, None), (20, None), (10, None), (6, None), (3, None), (10, 160), (6, None, 4), (20, None, 4),
               (6, None, 8), (6, None, 12), (20, None, 12)),
    "ggttggg": ((12, 160), (6, 160), (12, 160, 4), (12, 160, 8), (12, 160, 16), (12, 320, 16), (12, 480, 24)),
}

# real-flop counts of the helas.cuh routines (complex multiply 6, complex add 2,
# real x complex 2); counted from the formulas as written
FLOPS = {
    "ext_eps": 30, "ext_ubar": 40, "ext_v": 40, "ext_u": 40, "ext_vbar": 40,
    "g3": 24 + 30 + 14 + 14 + 4 * (4 + 6 + 6 + 4) + 8,      # 170
    "g4": 2 * 30 + 4 * (6 + 6 + 2) + 8,                     # 124
    "bra": 8 * 6 + 4 * 2 + 4 * (2 + 2 * 6 + 4) + 8 + 4 * 6,  # 160
    "ket": 8 * 6 + 4 * 2 + 4 * (2 + 2 * 6 + 4) + 8 + 4 * 6,  # 160
    "pj": 8 * 6 + 12 * 2,                                    # 72
    "dot": 4 * 6 + 3 * 2,                                    # 30
    "v3": 24 + 30 + 14 + 14 + 4 * (4 + 6 + 6 + 4) + 30 + 2,  # 194
    "v4": 4 * 30 + 2 * 6 + 2 + 2,                           # 136
    "add": 2,
}


_PHASES = (1, 1j, -1, -1j)


def colour_class(col):
    """(base, ph) with base the colour vector col scaled by ph so that its entry of
    lowest flow index is 1: amplitude a then adds sum_c base[c] * (a / ph) into J"""
    items = sorted(col.items())
    for ph in _PHASES:
        if abs(complex(items[0][1]) * ph - 1) < 1e-9:
            base = []
            for c, v in items:
                w = complex(v) * ph
                q = next((u for u in _PHASES if abs(w - u) < 1e-9), None)
                if q is None:
                    raise ValueError(f"unexpected colour coefficient {v}")
                base.append((c, q))
            return tuple(base), ph
    raise ValueError(f"unexpected colour coefficient {items[0][1]}")


def _pending_plan(keys, segs, npend):
    """Accumulation plan for the closings in emission order.  keys[j] is closing j's
    colour class, segs[j] the out-of-line function it is emitted in.  A class with a
    later member in the same function may take one of npend pending accumulators: its
    members are summed there and the sum is distributed over J once, after the last
    member or when the slot is taken by a class whose next member comes sooner (the
    pending class with the farthest next member is the one given up).  Returns, per
    closing, (action, slot, flushes): action 'direct' (add into J now), 'open', 'merge'
    or 'last' (merge, then distribute); flushes lists (slot, class) distributed before
    the closing."""
    nxt, last = [None] * len(keys), {}
    for j in reversed(range(len(keys))):
        k = (keys[j], segs[j])
        nxt[j] = last.get(k)
        last[k] = j
    pend, free, plan = {}, list(reversed(range(npend))), []
    for j, key in enumerate(keys):
        flushes = []
        if key in pend:
            slot = pend[key][0]
            if nxt[j] is None:
                del pend[key]
                free.append(slot)
                plan.append(("last", slot, flushes))
            else:
                pend[key][1] = nxt[j]
                plan.append(("merge", slot, flushes))
            continue
        if nxt[j] is None or npend == 0:
            plan.append(("direct", None, flushes))
            continue
        if not free:
            far = max(pend, key=lambda q: pend[q][1])
            if pend[far][1] > nxt[j]:
                flushes.append((pend[far][0], far))
                free.append(pend.pop(far)[0])
        if free:
            slot = free.pop()
            pend[key] = [slot, nxt[j]]
            plan.append(("open", slot, flushes))
        else:
            plan.append(("direct", None, flushes))
    assert not pend
    return plan


def _add_into(target, src, coef):
    """target += coef * src for coef in (1, i, -1, -i)"""
    if coef == 1:
        return f"{target} += {src};"
    if coef == -1:
        return f"{target} -= {src};"
    if coef == 1j:
        return f"acc_pi({target}, {src});"
    if coef == -1j:
        return f"acc_mi({target}, {src});"
    raise ValueError(f"unexpected colour coefficient {coef}")


def _exact(cf, bits):
    """every integer entry representable with a significand of 'bits' bits (the
    exponent range of FP16 reaches 65504, beyond every colour-matrix entry here)"""
    for x in (abs(int(v)) for v in cf.flatten()):
        if x and (x >> max(0, x.bit_length() - bits)) << max(0, x.bit_length() - bits) != x:
            return False
        if bits == 11 and x > 65504:
            return False
    return True


SYNC_STEP = 8  # schedule steps (currents and diagram closings) between optional barrier points


def _lit(x):
    return f"R({float(x)!r})"


def allocate_storage(seq, deps_of, externals, budget, boundaries=()):
    """Decide where each current lives: registers while at most ``budget`` values are
    register-resident, otherwise a slot of the per-thread slot buffer.  Belady's rule:
    when a new value needs a register and none is free, the resident value whose next
    use is furthest away moves to a slot (a copy at that point), unless the new value's
    own next use is further still, in which case it is written to a slot directly.

    Returns (plan, nslot): plan[k] = (evictions [(value, slot)], output location) for
    step k of seq, location ("R",) or ("S", slot); externals are defined before step 0.
    budget None keeps everything in registers.  At every step index in ``boundaries``
    all register-resident live values move to slots (a diagram-group boundary).
    """
    uses = {}
    for k, (t, x) in enumerate(seq):
        for d in deps_of(t, x):
            uses.setdefault(d, []).append(k)
    last = {v: u[-1] for v, u in uses.items()}
    ptr = {v: 0 for v in uses}

    def next_use(v, k):
        u = uses.get(v, [])
        i = ptr.get(v, 0)
        while i < len(u) and u[i] <= k:
            i += 1
        ptr[v] = i
        return u[i] if i < len(u) else float("inf")

    regs, slots_of = set(externals), {}
    free, nslot = [], 0
    plan = []

    def take_slot():
        nonlocal nslot
        if free:
            free.sort()
            return free.pop(0)
        nslot += 1
        return nslot - 1

    boundaries = set(boundaries)
    for k, (t, x) in enumerate(seq):
        ev, loc = [], ("R",)
        if k in boundaries:
            for v in sorted((v for v in regs if last.get(v, -1) >= k), key=repr):
                sl = take_slot()
                ev.append((v, sl))
                slots_of[v] = sl
            regs.clear()
        if t == "N" and budget is not None:
            live_regs = [v for v in regs if last.get(v, -1) >= k]
            if len(live_regs) >= budget:
                nu_new = next_use(x, k)
                far = max(live_regs, key=lambda v: next_use(v, k - 1))
                if next_use(far, k - 1) > nu_new:
                    sl = take_slot()
                    ev.append((far, sl))
                    regs.discard(far)
                    slots_of[far] = sl
                    regs.add(x)
                else:
                    sl = take_slot()
                    slots_of[x] = sl
                    loc = ("S", sl)
            else:
                regs.add(x)
        elif t == "N":
            regs.add(x)
        plan.append((ev, loc))
        # release values whose last use is this step
        for d in deps_of(t, x):
            if last.get(d) == k:
                regs.discard(d)
                if d in slots_of:
                    free.append(slots_of.pop(d))
        if t == "N" and x not in uses:
            regs.discard(x)
            if x in slots_of:
                free.append(slots_of.pop(x))
    return plan, nslot


class Emitter:
    def __init__(self, process: str):
        self.process = process
        self.spec = PROCESSES[process]
        self.roles = self.spec["roles"]
        self.tag = self.spec["tag"]
        self.npar = len(self.roles)
        self.gluons = tuple(i for i, r in enumerate(self.roles) if r in ("g_in", "g_out"))

    def mask_of_leaves(self, leaves):
        m = 0
        for i in leaves:
            m |= 1 << i
        return m

    def kin_terms(self, mask):
        """signed external momenta whose sum is the incoming momentum of 'mask'
        (incoming particles +p, outgoing -p)"""
        terms = []
        for i in range(self.npar):
            if mask >> i & 1:
                r = self.roles[i]
                terms.append(("+" if r.endswith("_in") else "-", i))
        return terms

    @staticmethod
    def _sum_expr(parts, mu, arr="p"):
        e = " ".join(f"{s} {arr}[{i}][{mu}]" for s, i in parts)
        return e[2:] if e.startswith("+ ") else e

    # ------------------------------------------------------------------ QCD
    def emit_qcd(self, budgets=((None, None),)):
        it = self.roles.index("t")
        itb = self.roles.index("tb")
        gl = self.gluons
        n = len(gl)
        sched = sc.build_qcd_schedule(gl, it, itb, restarts=8 if n >= 5 else 24)
        ndiag = len(dg.qcd_diagrams(gl, split4=False))
        ncol = math.factorial(n)
        cf, cden = colmod.colour_matrix(n)
        iden = 4 * 64 * math.factorial(sum(1 for r in self.roles if r == "g_out"))

        base_name = {("EXT", i): f"x{i}" for i in range(self.npar)}
        for k, node in enumerate(sched.nodes):
            base_name[node] = f"w{k}"
        name = dict(base_name)

        gmask_idx, tmask_idx = {}, {}

        def gmask_of_tree(tree):
            m = self.mask_of_leaves(dg.leaves(tree))
            if m not in gmask_idx:
                gmask_idx[m] = len(gmask_idx)
            return gmask_idx[m]

        def tmask(node):
            m = 1 << (it if node[0] == "BRA" else itb)
            for b in node[1]:
                m |= self.mask_of_leaves(dg.leaves(b))
            if m not in tmask_idx:
                tmask_idx[m] = len(tmask_idx)
            return m, tmask_idx[m]

        kvars = {}
        body = []

        def fermion_parts(mask):
            # momentum along the fermion arrow: top side q = p_t - K(gluons);
            # antitop side q = -p_tb + K(gluons)
            if mask >> it & 1:
                return [("+", it)] + [("-" if s == "+" else "+", i) for s, i in self.kin_terms(mask & ~(1 << it))]
            return [("-", itb)] + self.kin_terms(mask & ~(1 << itb))

        def kvar(mask, fermion=False):
            """index expression of a momentum vector in the per-event table kt (filled
            once per event by precompute(), outside the helicity loop)"""
            key = (mask, fermion)
            if key not in kvars:
                kvars[key] = self.npar + len(kvars)  # entries 0..npar-1: external momenta
            return f"(kt + {kvars[key]} * S)"

        fl = {"amp": 0}

        def flop(kind):
            fl["amp"] += FLOPS[kind]

        for i, r in enumerate(self.roles):
            if r in ("g_in", "g_out"):
                body.append(f"  cx<R> x{i}[4]; ext_eps<R>((kt + {i} * S), lam[{i}], {'true' if r == 'g_out' else 'false'}, x{i});")
                flop("ext_eps")
            elif r == "t":
                body.append(f"  cx<R> x{i}[4]; ext_ubar<R>((kt + {i} * S), mt, lam[{i}], x{i});")
                flop("ext_ubar")
            elif r == "tb":
                body.append(f"  cx<R> x{i}[4]; ext_v<R>((kt + {i} * S), mt, lam[{i}], x{i});")
                flop("ext_v")

        def gk(node):
            if node[0] == "EXT":
                return kvar(1 << node[1])
            return kvar(self.mask_of_leaves(dg.leaves(node[1])))

        pair_count = 0

        def emit_amp(a, act=None):
            nonlocal pair_count
            nm = [name[x] for x in a.inputs]
            if act is not None:
                for slot, base in act[2]:
                    body.append("  " + " ".join(_add_into(f"J[{c}]", f"pc{slot}", q) for c, q in base))
            if a.kind == "DOT":
                body.append(f"  {{ const cx<R> a = close_dot<R>({nm[0]}, {nm[1]});")
                flop("dot")
            else:
                blk = tuple(x[1] if x[0] == "G" else ("L", x[1]) for x in a.inputs[1:])
                ig = gmask_of_tree(("3",) + blk) if a.kind == "V3" else gmask_of_tree(("4", a.struct) + blk)
                if a.kind == "V3":
                    body.append(f"  {{ const cx<R> a = close_v3<R>({nm[0]}, {nm[1]}, {gk(a.inputs[1])}, "
                                f"{nm[2]}, {gk(a.inputs[2])}, dg[{ig}]);")
                    flop("v3")
                else:
                    body.append(f"  {{ const cx<R> a = close_v4<{a.struct}, R>({nm[0]}, {nm[1]}, {nm[2]}, "
                                f"{nm[3]}, dg[{ig}]);")
                    flop("v4")
            # the algorithmic count is the accumulation as written, J_c += colour_c * a,
            # whether or not the closing's amplitude is first summed in a pending slot
            for _ in a.colour:
                flop("add")
                pair_count += 1
            base, ph = colour_class(a.colour)
            kind = "direct" if act is None else act[0]
            if kind == "direct":
                ops = [_add_into(f"J[{c}]", "a", q / ph) for c, q in base]
            elif kind == "open":
                # pc = a / ph
                init = {1: "a", -1: "mk<R>(-a.r, -a.i)", 1j: "mk<R>(a.i, -a.r)", -1j: "mk<R>(-a.i, a.r)"}[ph]
                ops = [f"pc{act[1]} = {init};"]
            else:
                ops = [_add_into(f"pc{act[1]}", "a", 1 / ph)]
                if kind == "last":
                    ops += [_add_into(f"J[{c}]", f"pc{act[1]}", q) for c, q in base]
            body.append("    " + " ".join(ops) + " }")

        def emit_node(node, loc):
            if loc[0] == "S":
                v = f"(ws + {loc[1]} * S)"
                decl = " "
            else:
                v = base_name[node]
                decl = f"  cx<R> {v}[4];"
            name[node] = v
            kind = node[0]
            if kind == "G":
                t = node[1]
                kids = sc.deps(node, it, itb)
                ig = gmask_of_tree(t)
                if t[0] == "3":
                    body.append(f"{decl} g3_current<R>({name[kids[0]]}, {gk(kids[0])}, "
                                f"{name[kids[1]]}, {gk(kids[1])}, dg[{ig}], {v});")
                    flop("g3")
                else:
                    body.append(f"{decl} g4_current<{t[1]}, R>({name[kids[0]]}, {name[kids[1]]}, "
                                f"{name[kids[2]]}, dg[{ig}], {v});")
                    flop("g4")
            elif kind == "BRA":
                prev, g = sc.deps(node, it, itb)
                m, idx = tmask(node)
                body.append(f"{decl} bra_step<R>({name[prev]}, {name[g]}, {kvar(m, True)}, mt, dt[{idx}], {v});")
                flop("bra")
            elif kind == "KET":
                g, prev = sc.deps(node, it, itb)
                m, idx = tmask(node)
                body.append(f"{decl} ket_step<R>({name[g]}, {name[prev]}, {kvar(m, True)}, mt, dt[{idx}], {v});")
                flop("ket")
            elif kind == "PJ":
                b, k = sc.deps(node, it, itb)
                body.append(f"{decl} pair_current<R>({name[b]}, {name[k]}, {v});")
                flop("pj")

        def deps_of(t, x):
            return sc.deps(x, it, itb) if t == "N" else sched.amps[x].inputs

        externals = [("EXT", i) for i in range(self.npar)]
        ext_lines = list(body)
        variants = []
        for vi, vdef in enumerate(budgets):
            budget, group = vdef[0], vdef[1]
            npend = vdef[2] if len(vdef) > 2 else 0
            bounds = list(range(group, len(sched.seq), group)) if group else []
            amp_steps = [k for k, (t, _) in enumerate(sched.seq) if t == "A"]
            aplan = _pending_plan([colour_class(sched.amps[sched.seq[k][1]].colour)[0] for k in amp_steps],
                                  [sum(1 for b in bounds if b <= k) for k in amp_steps], npend)
            aplan = dict(zip(amp_steps, aplan))
            plan, nslot = allocate_storage(sched.seq, deps_of, externals, budget, bounds)
            body[:] = list(ext_lines)
            name.clear()
            name.update(base_name)
            fl["amp"] = sum(FLOPS["ext_eps"] if r.startswith("g") else FLOPS["ext_ubar"] for r in self.roles)
            pair_count = 0
            groups = []
            for k, ((t, x), (ev, loc)) in enumerate(zip(sched.seq, plan)):
                # evictions (at a group boundary: every live register value) are written by
                # the group that still holds the values, then the next group starts
                for u, sl in ev:
                    body.append(f"  copy4<R>((ws + {sl} * S), {name[u]});")
                    name[u] = f"(ws + {sl} * S)"
                if k in bounds:
                    groups.append(list(body))
                    body[:] = []
                elif k and k % SYNC_STEP == 0:
                    body.append(f"  if constexpr (SYNC > 0 && {k // SYNC_STEP} % SYNC == 0) MEB_BLOCK_SYNC();")
                if t == "N":
                    emit_node(x, loc)
                else:
                    emit_amp(sched.amps[x], aplan[k])
            groups.append(list(body))
            variants.append((budget, group, nslot, groups, npend))

        den = ["  using DD = dd_for<R>;", "  DD q[4];"]

        def dd_sum(parts):
            # exact sum of signed momenta, component by component
            out = []
            for mu in range(4):
                s0, i0 = parts[0]
                e = f"DD{{{'-' if s0 == '-' else ''}p[{i0}][{mu}], 0.0}}"
                for sgn, i in parts[1:]:
                    e = f"dd_add({e}, {'-' if sgn == '-' else ''}p[{i}][{mu}])"
                out.append(f"  q[{mu}] = {e};")
            return out

        den.append("  double kappa = 0.0;  // conditioning: max over gluon propagators of (sum E)^2 / |K^2|")
        for m, idx in sorted(gmask_idx.items(), key=lambda t: t[1]):
            den += dd_sum(self.kin_terms(m))
            esum = " + ".join(f"p[{i}][0]" for _, i in self.kin_terms(m))
            den.append(f"  {{ const double k2 = dd_invariant(q, 0.0), es = {esum};")
            den.append(f"    dg[{idx}] = R(1.0 / k2); kappa = fmax(kappa, es * es / fabs(k2)); }}")
        for m, idx in sorted(tmask_idx.items(), key=lambda t: t[1]):
            tchan = (m & 1) != ((m >> 1) & 1)  # separates the two incoming particles
            den += dd_sum(fermion_parts(m))
            den.append(f"  {{ const double w = {'(zwt ? 0.0 : wt)' if tchan else 'wt'};")
            den.append("    const double re = dd_invariant(q, mt);")
            den.append("    const double im = mt * w, inv = 1.0 / (re * re + im * im);")
            den.append(f"    dt[{idx}] = mk<R>(R(re * inv), R(-im * inv)); }}")
        den.append("  // momentum table: external momenta, then the vectors the vertices use")
        den.append(f"  for (int i = 0; i < {self.npar}; ++i)")
        den.append("    for (int m = 0; m < 4; ++m) kt[i * S + m] = R(p[i][m]);")
        for (mask, fermion), idx in sorted(kvars.items(), key=lambda t: t[1]):
            parts = fermion_parts(mask) if fermion else self.kin_terms(mask)
            for mu in range(4):
                den.append(f"  kt[{idx} * S + {mu}] = R({self._sum_expr(parts, mu)});")
        nk = self.npar + len(kvars)

        cs = []
        csflops = 0

        def fused(terms):
            # sum of products as a chain of fused multiply-adds: fmadd(a, b, fmadd(c, d, e * f))
            e = f"{terms[-1][0]} * {terms[-1][1]}"
            for a_, b_ in reversed(terms[:-1]):
                e = f"fmadd({a_}, {b_}, {e})"
            return e

        for i in range(ncol):
            tr, ti = [], []
            for j in range(i, ncol):
                c = int(cf[i, j]) * (1 if j == i else 2)
                if c == 0:
                    continue
                tr.append((_lit(c), f"J[{j}].r"))
                ti.append((_lit(c), f"J[{j}].i"))
                csflops += 4
            cs.append(f"  {{ const R tr = {fused(tr)}; const R ti = {fused(ti)};")
            cs.append(f"    s = fmadd(J[{i}].r, tr, fmadd(J[{i}].i, ti, s)); }}")
            csflops += 4

        ngden, ntden = max(1, len(gmask_idx)), max(1, len(tmask_idx))
        tag = self.tag
        out = [f"// Generated by paper_2312_02898_b300/gen/emit.py for '{self.process}'. Do not edit.",
               "#pragma once", '#include "../helas.cuh"', "namespace meb300 {",
               "#if defined(__CUDACC__)",
               f"// integer colour-matrix numerators for device code (tensor-core operand)",
               f"static __device__ __constant__ int proc_{tag}_CFD[{ncol * ncol}] = "
               f"{{{', '.join(str(int(x)) for x in cf.flatten())}}};",
               "#endif",
               f"struct proc_{tag} {{",
               f'static constexpr const char* NAME = "{self.process}";',
               f"static constexpr int NPAR = {self.npar}, NCOMB = {1 << self.npar}, NCOL = {ncol}, NDIAG = {ndiag};",
               f"static constexpr int NAMP = {len(sched.amps)}, NNODE = {len(sched.nodes)}, IDEN = {iden}, NGLUON = {n};",
               f"static constexpr int NDEN_G = {ngden}, NDEN_T = {ntden}, COL_DEN = {cden}, NCOLPAIR = {pair_count};",
               f"static constexpr long FLOPS_AMP = {fl['amp']}, FLOPS_COL = {csflops};  // per helicity, real flops",
               f"static constexpr int MAX_LIVE = {sc.max_live(sched, it, itb)};  // currents alive at once",
               f"static constexpr bool CF_BF16_EXACT = {'true' if _exact(cf, 8) else 'false'}, "
               f"CF_FP16_EXACT = {'true' if _exact(cf, 11) else 'false'};  // colour matrix exact in 16-bit",
               "static constexpr bool QCD = true;", "",
               f"static constexpr int NKVEC = {nk};  // momentum vectors in the per-event table",
               "template <int S, class R, class DG, class DT, class KT>",
               "static HD double precompute(const double (*p)[4], double mt, double wt, int zwt, DG& dg, DT& dt,"
               " KT kt) {"]
        out += den
        out.append("  return kappa;")
        out.append("}")
        out.append("// jamps variants: register budget (currents kept in registers, -1 = all), diagram-group")
        out.append("// size (0 = one function) and slots used in the per-thread slot buffer ws (slot s at")
        out.append("// ws + s * S; momentum-table entry k at kt + k * S; S = threads per block * 4)")
        out.append(f"static constexpr int NVARIANT = {len(variants)};")
        out.append("static constexpr int NSLOT[NVARIANT] = {" + ", ".join(str(v[2]) for v in variants) + "};")
        out.append("static constexpr int BUDGET[NVARIANT] = {" + ", ".join(str(-1 if v[0] is None else v[0]) for v in variants) + "};")
        out.append("static constexpr int GROUP[NVARIANT] = {" + ", ".join(str(v[1] or 0) for v in variants) + "};")
        chain_s, chain_g = "0", "false"
        for vi in reversed(range(len(variants))):
            chain_s = f"(V == {vi} ? {variants[vi][2]} : {chain_s})"
            chain_g = f"(V == {vi} ? {'true' if variants[vi][1] else 'false'} : {chain_g})"
        out.append(f"template <int V> static HD constexpr int nslot() {{ return {chain_s}; }}")
        out.append(f"template <int V> static HD constexpr bool grouped() {{ return {chain_g}; }}")
        lam = (f"  int lam[{self.npar}];\n  for (int i = 0; i < {self.npar}; ++i) "
               f"lam[i] = ((h >> ({self.npar - 1} - i)) & 1) ? 1 : -1;")
        for vi, (budget, group, nslot, groups, npend) in enumerate(variants):
            pdecl = [f"  cx<R> {', '.join(f'pc{i}' for i in range(npend))};  // pending colour sums"] if npend else []
            # SYNC > 0: a block barrier every SYNC * SYNC_STEP steps and between diagram
            # groups, which keeps the warps of a block on the same stretch of code (all
            # threads of the block must then call the function together)
            if not group:
                out += ["", "template <int S, class R, int SYNC = 0, class DG, class DT, class JA>",
                        f"static HD void jamps_v{vi}(int h, R mt, const DG& dg, const DT& dt, JA& J, cx<R>* ws,"
                        " const R* kt) {", lam] + pdecl
                out += groups[0]
                out.append("}")
            else:
                for gi, gbody in enumerate(groups):
                    out += ["", "template <int S, class R, int SYNC = 0, class DG, class DT, class JA>",
                            f"static NOINL void jamps_v{vi}_g{gi}(int h, R mt, DG dg, DT dt, JA J, cx<R>* ws, const R* kt) {{",
                            lam] + pdecl
                    out += gbody
                    out.append("}")
                out += ["", "template <int S, class R, int SYNC = 0, class DG, class DT, class JA>",
                        f"static HD void jamps_v{vi}(int h, R mt, const DG& dg, const DT& dt, JA& J, cx<R>* ws,"
                        " const R* kt) {"]
                for gi in range(len(groups)):
                    if gi:
                        out.append("  if constexpr (SYNC > 0) MEB_BLOCK_SYNC();")
                    out.append(f"  jamps_v{vi}_g{gi}<S, R, SYNC>(h, mt, dg, dt, J, ws, kt);")
                out.append("}")
        out += ["", "template <int V, int S, class R, int SYNC = 0, class DG, class DT, class JA>",
                "static HD void jamps(int h, R mt, const DG& dg, const DT& dt, JA& J, cx<R>* ws, const R* kt) {"]
        for vi in range(len(variants)):
            out.append(f"  {'if' if vi == 0 else 'else if'} constexpr (V == {vi}) jamps_v{vi}<S, R, SYNC>(h, mt, dg, dt, J, ws, kt);")
        out += ["}"]
        out += ["#if defined(__CUDACC__)",
                f"static __device__ int cf_device(int i) {{ return proc_{self.tag}_CFD[i]; }}",
                "#endif"]
        out += ["", "template <class R, class JA>", "static HD R colour_sum(JA& J) {", "  R s = R(0);"]
        out += cs
        out += ["  return s;", "}", "};",
                f"constexpr int proc_{tag}_CF[{ncol} * {ncol}] = {{{', '.join(str(int(x)) for x in cf.flatten())}}};",
                "}  // namespace meb300"]
        stats = dict(ndiag=ndiag, namp=len(sched.amps), nnode=len(sched.nodes), ncol=ncol, pairs=pair_count,
                     flops_amp=fl["amp"], flops_col=csflops, nden_g=ngden, nden_t=ntden, col_den=cden,
                     max_live=sc.max_live(sched, it, itb), schedule=sc.summary(sched),
                     variants=[(b, g, ns, npd) for b, g, ns, _, npd in variants])
        return "\n".join(out) + "\n", stats

    # ------------------------------------------------------------------ e+e- -> mu+mu-
    def emit_eemumu(self):
        fa = 4 * FLOPS["ext_u"] + 4 * FLOPS["pj"] + 2 * FLOPS["dot"] + 6 + 6 + 2
        out = [f"// Generated by paper_2312_02898_b300/gen/emit.py for '{self.process}'. Do not edit.",
               "#pragma once", '#include "../helas.cuh"', "namespace meb300 {", "struct proc_eemumu {",
               f'static constexpr const char* NAME = "{self.process}";',
               "static constexpr int NPAR = 4, NCOMB = 16, NCOL = 1, NDIAG = 2, NAMP = 2, NNODE = 2, IDEN = 4, NGLUON = 0;",
               "static constexpr int NDEN_G = 1, NDEN_T = 1, COL_DEN = 1, NCOLPAIR = 2, MAX_LIVE = 2, NKVEC = 4;",
               f"static constexpr long FLOPS_AMP = {fa}, FLOPS_COL = 4;",
               "static constexpr bool QCD = false;",
               "// Photon and Z in the s channel.  dg[0] = 1/s;  dt[0] = 1/(s - mZ^2 + i mZ wZ).",
               "template <int S, class R, class DG, class DT, class KT>",
               "static HD double precompute(const double (*p)[4], double mZ, double wZ, int, DG& dg, DT& dt, KT kt) {",
               "  for (int i = 0; i < 4; ++i)",
               "    for (int m = 0; m < 4; ++m) kt[i * S + m] = R(p[i][m]);",
               "  double q[4];",
               "  for (int m = 0; m < 4; ++m) q[m] = p[0][m] + p[1][m];",
               "  const double s = q[0] * q[0] - q[1] * q[1] - q[2] * q[2] - q[3] * q[3];",
               "  dg[0] = R(1.0 / s);",
               "  const double re = s - mZ * mZ, im = mZ * wZ, inv = 1.0 / (re * re + im * im);",
               "  dt[0] = mk<R>(R(re * inv), R(-im * inv));",
               "  return 0.0;",
               "}",
               "// J = i [ (j_e . j_mu)_photon / s + (j_e . j_mu)_Z / D_Z ] in units of e^2: the photon",
               "// couples with Q_e Q_mu = 1 overall, the Z with (gL, gR) = zc[0..1] on each current.",
               "static constexpr int NVARIANT = 1;",
               "static constexpr int NSLOT[1] = {0};",
               "template <int V> static HD constexpr int nslot() { return 0; }",
               "template <int V> static HD constexpr bool grouped() { return false; }",
               "static constexpr int BUDGET[1] = {-1};",
               "template <int V, int S, class R, int SYNC = 0, class DG, class DT, class JA>",
               "static HD void jamps(int h, const R* zc, const DG& dg, const DT& dt, JA& J, cx<R>*, const R* kt) {",
               "  int lam[4];",
               "  for (int i = 0; i < 4; ++i) lam[i] = ((h >> (3 - i)) & 1) ? 1 : -1;",
               "  cx<R> x0[4], x1[4], x2[4], x3[4];",
               "  ext_vbar<R>(kt, R(0), lam[0], x0);            // incoming e+",
               "  ext_u<R>(kt + S, R(0), lam[1], x1);          // incoming e-",
               "  ext_v<R>(kt + 2 * S, R(0), lam[2], x2);      // outgoing mu+",
               "  ext_ubar<R>(kt + 3 * S, R(0), lam[3], x3);   // outgoing mu-",
               "  cx<R> je[4], jm[4];",
               "  pair_current<R>(x0, x1, je); pair_current<R>(x3, x2, jm);",
               "  const cx<R> aa = dg[0] * mdot(je, jm);",
               "  pair_current_lr<R>(x0, x1, zc[0], zc[1], je); pair_current_lr<R>(x3, x2, zc[0], zc[1], jm);",
               "  const cx<R> az = mdot(je, jm) * dt[0];",
               "  J[0] += times_i(aa + az);",
               "}",
               "template <class R, class JA>",
               "static HD R colour_sum(JA& J) { return J[0].r * J[0].r + J[0].i * J[0].i; }",
               "};",
               "constexpr int proc_eemumu_CF[1] = {1};",
               "}  // namespace meb300"]
        stats = dict(ndiag=2, namp=2, nnode=2, ncol=1, pairs=2, flops_amp=fa, flops_col=4, nden_g=1, nden_t=1,
                     col_den=1, max_live=2)
        return "\n".join(out) + "\n", stats

    # ------------------------------------------------------------------ q q~ -> t t~
    def emit_qqtt(self):
        """q qbar -> t tbar through one s-channel gluon.  With the quark-gluon vertex
        -i g T^a gamma^mu and the gluon propagator -i g_{mu nu} / s the amplitude is
        i g^2 (L_q . L_t) / s times the colour factor sum_a T^a_{ji} T^a_{kl} =
        (c_0 - c_1 / 3) / 2, c_0 = d_ki d_jl and c_1 = d_ji d_kl (i, j: quark and antiquark
        colours; k, l: top and antitop).  The flows are carried scaled by 6, J = (3, -1) x
        i (L_q . L_t) / s, with the colour matrix sum c_n c_m = [[9, 3], [3, 9]] over 36."""
        iq, iqb = self.roles.index("q_in"), self.roles.index("qb_in")
        fa = 4 * FLOPS["ext_u"] + 2 * FLOPS["pj"] + FLOPS["dot"] + 2 + 2 + 2
        cf = [[9, 3], [3, 9]]
        cs = []
        csflops = 0
        for i in range(2):
            tr = [f"{_lit(cf[i][j] * (1 if j == i else 2))} * J[{j}].r" for j in range(i, 2)]
            ti = [f"{_lit(cf[i][j] * (1 if j == i else 2))} * J[{j}].i" for j in range(i, 2)]
            csflops += 4 * len(tr) + 4
            cs.append(f"  {{ const R tr = {' + '.join(tr)}; const R ti = {' + '.join(ti)};")
            cs.append(f"    s = fmadd(J[{i}].r, tr, fmadd(J[{i}].i, ti, s)); }}")
        tag = self.tag
        out = [f"// Generated by paper_2312_02898_b300/gen/emit.py for '{self.process}'. Do not edit.",
               "#pragma once", '#include "../helas.cuh"', "namespace meb300 {", f"struct proc_{tag} {{",
               f'static constexpr const char* NAME = "{self.process}";',
               "// NGLUON counts the powers of g_s^2 in |M|^2 (two quark-gluon vertices)",
               "static constexpr int NPAR = 4, NCOMB = 16, NCOL = 2, NDIAG = 1, NAMP = 1, NNODE = 2, IDEN = 36, NGLUON = 2;",
               "static constexpr int NDEN_G = 1, NDEN_T = 1, COL_DEN = 36, NCOLPAIR = 2, MAX_LIVE = 2, NKVEC = 4;",
               f"static constexpr long FLOPS_AMP = {fa}, FLOPS_COL = {csflops};",
               "static constexpr bool QCD = true;",
               "static constexpr bool CF_BF16_EXACT = true, CF_FP16_EXACT = true;",
               "// dg[0] = 1/s of the s-channel gluon; no top propagator (dt unused)",
               "template <int S, class R, class DG, class DT, class KT>",
               "static HD double precompute(const double (*p)[4], double, double, int, DG& dg, DT& dt, KT kt) {",
               "  for (int i = 0; i < 4; ++i)",
               "    for (int m = 0; m < 4; ++m) kt[i * S + m] = R(p[i][m]);",
               "  double q[4];",
               f"  for (int m = 0; m < 4; ++m) q[m] = p[{iq}][m] + p[{iqb}][m];",
               "  const double s = q[0] * q[0] - q[1] * q[1] - q[2] * q[2] - q[3] * q[3];",
               "  dg[0] = R(1.0 / s);",
               "  dt[0] = mk<R>(R(0), R(0));",
               "  return 0.0;",
               "}",
               "static constexpr int NVARIANT = 1;",
               "static constexpr int NSLOT[1] = {0};",
               "template <int V> static HD constexpr int nslot() { return 0; }",
               "template <int V> static HD constexpr bool grouped() { return false; }",
               "static constexpr int BUDGET[1] = {-1};",
               "template <int V, int S, class R, int SYNC = 0, class DG, class DT, class JA>",
               "static HD void jamps(int h, R mt, const DG& dg, const DT&, JA& J, cx<R>*, const R* kt) {",
               "  int lam[4];",
               "  for (int i = 0; i < 4; ++i) lam[i] = ((h >> (3 - i)) & 1) ? 1 : -1;",
               "  cx<R> xq[4], xqb[4], xt[4], xtb[4];",
               f"  ext_u<R>(kt + {iq} * S, R(0), lam[{iq}], xq);        // incoming quark",
               f"  ext_vbar<R>(kt + {iqb} * S, R(0), lam[{iqb}], xqb);  // incoming antiquark",
               "  ext_ubar<R>(kt + 2 * S, mt, lam[2], xt);         // outgoing top",
               "  ext_v<R>(kt + 3 * S, mt, lam[3], xtb);           // outgoing antitop",
               "  cx<R> lq[4], lt[4];",
               "  pair_current<R>(xqb, xq, lq);",
               "  pair_current<R>(xt, xtb, lt);",
               "  const cx<R> a = dg[0] * mdot(lq, lt);",
               "  acc_pi(J[0], R(3) * a);",
               "  acc_mi(J[1], a);",
               "}",
               "template <class R, class JA>",
               "static HD R colour_sum(JA& J) {", "  R s = R(0);"] + cs + ["  return s;", "}", "};",
               f"constexpr int proc_{tag}_CF[4] = {{9, 3, 3, 9}};",
               "}  // namespace meb300"]
        stats = dict(ndiag=1, namp=1, nnode=2, ncol=2, pairs=2, flops_amp=fa, flops_col=csflops, nden_g=1, nden_t=1,
                     col_den=36, max_live=2)
        return "\n".join(out) + "\n", stats

    # ------------------------------------------------------------------ q q~ -> t t~ g and crossings
    def emit_quark_jet(self):
        """One light-quark line, the top line and one gluon: q qbar -> t tbar g, q g ->
        t tbar q, qbar g -> t tbar qbar.  Five diagrams (raw values r_d, no couplings):
          D1  gluon on the light line next to its column end K:  (B g.. K current) . H / s_H
          D2  next to its row end B,  D3/D4  on the top line next to the top / antitop
              (light current . top-line current / s_L),
          D5  the three-gluon vertex, eps . V3(L, k1; H, k2) / (s_L s_H);
        with the quark-gluon vertex -i g_s gamma T^a, fermion propagators i(qslash + m)/D,
        gluon propagators -i g/K^2 and the three-gluon vertex -g_s f^{abc} V, the amplitude
        is g_s^3 (i (r1 c1 + ... + r4 c4) - r5 c5) with c_d the diagrams' colour tensors.
        Each c_d is a fixed combination of four flow tensors (gen/colour.py); the flows are
        carried scaled by 6, which makes every coefficient a Gaussian integer."""
        roles = self.roles
        ib = next(i for i, r in enumerate(roles) if r in ("qb_in", "q_out"))  # light row end
        ik = next(i for i, r in enumerate(roles) if r in ("q_in", "qb_out"))  # light column end
        ig = next(i for i, r in enumerate(roles) if r in ("g_in", "g_out"))
        it, itb = roles.index("t"), roles.index("tb")

        def P(i):
            return [("+" if roles[i].endswith("_in") else "-", i)]

        def neg(parts):
            return [("-" if s == "+" else "+", i) for s, i in parts]

        vecs = [("q1", P(ik) + P(ig)), ("q2", neg(P(ib) + P(ig))), ("q3", neg(P(it) + P(ig))),
                ("q4", P(itb) + P(ig)), ("k1", P(ib) + P(ik)), ("k2", P(it) + P(itb))]
        kix = {nm: self.npar + n for n, (nm, _) in enumerate(vecs)}
        coef, gram = colmod.quark_jet_colour()
        # gcd of the Gram matrix folded into the colour denominator (flows scaled by 6)
        g = 0
        for v in gram.flatten():
            g = math.gcd(g, int(v))
        cf = gram // g
        cden = 36 // math.gcd(36, g)
        cf = cf * (cden * g // 36) if (cden * g) % 36 == 0 else None
        assert cf is not None
        phases = [1j, 1j, 1j, 1j, -1]
        fa = 4 * FLOPS["ext_u"] + FLOPS["ext_eps"] + 6 * FLOPS["pj"] + 2 * FLOPS["ket"] + 2 * FLOPS["bra"]
        fa += 4 * FLOPS["dot"] + 5 * 2 + FLOPS["v3"]
        pairs = 0
        acc = []
        for d in range(5):
            ops = []
            for c in range(4):
                k = coef[d][c] * phases[d]
                k = complex(round(k.real), round(k.imag))
                if k == 0:
                    continue
                mag = int(abs(k.real) + abs(k.imag))
                unit = k / mag
                src = "a" if mag == 1 else f"a{mag}"
                if unit == 1:
                    ops.append(f"J[{c}] += {src};")
                elif unit == -1:
                    ops.append(f"J[{c}] -= {src};")
                elif unit == 1j:
                    ops.append(f"acc_pi(J[{c}], {src});")
                elif unit == -1j:
                    ops.append(f"acc_mi(J[{c}], {src});")
                else:
                    raise ValueError(k)
                pairs += 1
                fa += 2
            mags = sorted({int(abs(complex(coef[d][c] * phases[d]).real) + abs(complex(coef[d][c] * phases[d]).imag))
                           for c in range(4) if coef[d][c] != 0} - {1})
            pre = "".join(f" const cx<R> a{m} = R({m}) * a;" for m in mags)
            fa += 2 * len(mags)
            acc.append(pre + " " + " ".join(ops))

        def ext(i):
            r = roles[i]
            kt = f"(kt + {i} * S)"
            if r == "q_in":
                return f"ext_u<R>({kt}, R(0), lam[{i}], x{i});"
            if r == "qb_in":
                return f"ext_vbar<R>({kt}, R(0), lam[{i}], x{i});"
            if r == "q_out":
                return f"ext_ubar<R>({kt}, R(0), lam[{i}], x{i});"
            if r == "qb_out":
                return f"ext_v<R>({kt}, R(0), lam[{i}], x{i});"
            if r in ("g_in", "g_out"):
                return f"ext_eps<R>({kt}, lam[{i}], {'true' if r == 'g_out' else 'false'}, x{i});"
            if r == "t":
                return f"ext_ubar<R>({kt}, mt, lam[{i}], x{i});"
            return f"ext_v<R>({kt}, mt, lam[{i}], x{i});"

        K = lambda nm: f"(kt + {kix[nm]} * S)"
        body = [f"  int lam[{self.npar}];",
                f"  for (int i = 0; i < {self.npar}; ++i) lam[i] = ((h >> ({self.npar - 1} - i)) & 1) ? 1 : -1;",
                "  " + " ".join(f"cx<R> x{i}[4];" for i in range(self.npar))]
        body += ["  " + ext(i) for i in range(self.npar)]
        body += ["  cx<R> L[4], H[4], w[4], c[4];",
                 f"  pair_current<R>(x{ib}, x{ik}, L);",
                 f"  pair_current<R>(x{it}, x{itb}, H);",
                 f"  ket_step<R>(x{ig}, x{ik}, {K('q1')}, R(0), dt[0], w);  // D1",
                 f"  pair_current<R>(x{ib}, w, c);",
                 f"  {{ const cx<R> a = dg[1] * mdot(c, H);{acc[0]} }}",
                 f"  bra_step<R>(x{ib}, x{ig}, {K('q2')}, R(0), dt[1], w);  // D2",
                 f"  pair_current<R>(w, x{ik}, c);",
                 f"  {{ const cx<R> a = dg[1] * mdot(c, H);{acc[1]} }}",
                 f"  bra_step<R>(x{it}, x{ig}, {K('q3')}, mt, dt[2], w);  // D3",
                 f"  pair_current<R>(w, x{itb}, c);",
                 f"  {{ const cx<R> a = dg[0] * mdot(L, c);{acc[2]} }}",
                 f"  ket_step<R>(x{ig}, x{itb}, {K('q4')}, mt, dt[3], w);  // D4",
                 f"  pair_current<R>(x{it}, w, c);",
                 f"  {{ const cx<R> a = dg[0] * mdot(L, c);{acc[3]} }}",
                 f"  {{ const cx<R> a = dg[1] * close_v3<R>(x{ig}, L, {K('k1')}, H, {K('k2')}, dg[0]);{acc[4]} }}  // D5"]

        # denominators, in FP64 from the FP64 momenta (error-free sums and squares in the
        # FP64 mode), once per event
        den = ["  using DD = dd_for<R>;", "  DD q[4];",
               "  double kappa = 0.0;  // conditioning: max over light-line and gluon invariants of (sum E)^2 / |K^2|"]

        def dd_sum(parts):
            out = []
            for mu in range(4):
                s0, i0 = parts[0]
                e = f"DD{{{'-' if s0 == '-' else ''}p[{i0}][{mu}], 0.0}}"
                for sgn, i in parts[1:]:
                    e = f"dd_add({e}, {'-' if sgn == '-' else ''}p[{i}][{mu}])"
                out.append(f"  q[{mu}] = {e};")
            return out

        def esum(parts):
            return " + ".join(f"p[{i}][0]" for _, i in parts)

        vd = dict(vecs)
        for slot, nm in ((0, "q1"), (1, "q2")):
            den += dd_sum(vd[nm])
            den.append(f"  {{ const double k2 = dd_invariant(q, 0.0), es = {esum(vd[nm])};")
            den.append(f"    dt[{slot}] = mk<R>(R(1.0 / k2), R(0)); kappa = fmax(kappa, es * es / fabs(k2)); }}")
        for slot, nm, other in ((2, "q3", it), (3, "q4", itb)):
            mask = (1 << other) | (1 << ig)
            tchan = (mask & 1) != ((mask >> 1) & 1)
            den += dd_sum(vd[nm])
            den.append(f"  {{ const double w = {'(zwt ? 0.0 : wt)' if tchan else 'wt'};")
            den.append("    const double re = dd_invariant(q, mt);")
            den.append("    const double im = mt * w, inv = 1.0 / (re * re + im * im);")
            den.append(f"    dt[{slot}] = mk<R>(R(re * inv), R(-im * inv)); }}")
        for slot, nm in ((0, "k1"), (1, "k2")):
            den += dd_sum(vd[nm])
            den.append(f"  {{ const double k2 = dd_invariant(q, 0.0), es = {esum(vd[nm])};")
            den.append(f"    dg[{slot}] = R(1.0 / k2); kappa = fmax(kappa, es * es / fabs(k2)); }}")
        den.append("  // momentum table: external momenta, then the vectors the vertices use")
        den.append(f"  for (int i = 0; i < {self.npar}; ++i)")
        den.append("    for (int m = 0; m < 4; ++m) kt[i * S + m] = R(p[i][m]);")
        for nm, parts in vecs:
            for mu in range(4):
                den.append(f"  kt[{kix[nm]} * S + {mu}] = R({self._sum_expr(parts, mu)});")

        cs, csflops = [], 0
        for i in range(4):
            tr = [f"{_lit(int(cf[i][j]) * (1 if j == i else 2))} * J[{j}].r" for j in range(i, 4) if cf[i][j]]
            ti = [f"{_lit(int(cf[i][j]) * (1 if j == i else 2))} * J[{j}].i" for j in range(i, 4) if cf[i][j]]
            csflops += 4 * len(tr) + 4
            cs.append(f"  {{ const R tr = {' + '.join(tr)}; const R ti = {' + '.join(ti)};")
            cs.append(f"    s = fmadd(J[{i}].r, tr, fmadd(J[{i}].i, ti, s)); }}")
        iden = 4 * (9 if ig >= 2 else 24)
        tag = self.tag
        out = [f"// Generated by paper_2312_02898_b300/gen/emit.py for '{self.process}'. Do not edit.",
               "#pragma once", '#include "../helas.cuh"', "namespace meb300 {", f"struct proc_{tag} {{",
               f'static constexpr const char* NAME = "{self.process}";',
               "// NGLUON counts the powers of g_s^2 in |M|^2 (three QCD vertices)",
               f"static constexpr int NPAR = 5, NCOMB = 32, NCOL = 4, NDIAG = 5, NAMP = 5, NNODE = 6, IDEN = {iden}, NGLUON = 3;",
               f"static constexpr int NDEN_G = 2, NDEN_T = 4, COL_DEN = {cden}, NCOLPAIR = {pairs}, MAX_LIVE = 4, NKVEC = {self.npar + len(vecs)};",
               f"static constexpr long FLOPS_AMP = {fa}, FLOPS_COL = {csflops};",
               "static constexpr bool QCD = true;",
               "static constexpr bool CF_BF16_EXACT = true, CF_FP16_EXACT = true;",
               "// dg[0] = 1/s_L, dg[1] = 1/s_H (the gluons off the light and the top line);",
               "// dt[0], dt[1]: 1/q^2 of the light-quark propagators; dt[2], dt[3]: the top propagators",
               "template <int S, class R, class DG, class DT, class KT>",
               "static HD double precompute(const double (*p)[4], double mt, double wt, int zwt, DG& dg, DT& dt, KT kt) {"]
        out += den
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
                f"constexpr int proc_{tag}_CF[16] = {{{', '.join(str(int(x)) for x in cf.flatten())}}};",
                "}  // namespace meb300"]
        stats = dict(ndiag=5, namp=5, nnode=6, ncol=4, pairs=pairs, flops_amp=fa, flops_col=csflops, nden_g=2,
                     nden_t=4, col_den=cden, max_live=4)
        return "\n".join(out) + "\n", stats

    def emit(self):
        if self.tag in QUARK_JET2_TAGS:
            from . import quark_lines
            return quark_lines.header(self)
        if self.tag in QUARK_JET_TAGS:
            return self.emit_quark_jet()
        if self.tag == "eemumu":
            return self.emit_eemumu()
        if self.tag in ("qqtt", "qxqtt"):
            return self.emit_qqtt()
        return self.emit_qcd(budgets=VARIANTS.get(self.tag, ((None, None),)))


def generate_all(outdir: str, processes=None, verbose=False):
    """Write proc_<tag>.cuh for every process (only when the text changes)."""
    os.makedirs(outdir, exist_ok=True)
    stats = {}
    for proc in (processes or PROCESSES):
        text, st = Emitter(proc).emit()
        path = os.path.join(outdir, f"proc_{PROCESSES[proc]['tag']}.cuh")
        old = open(path).read() if os.path.exists(path) else None
        if old != text:
            with open(path, "w") as f:
                f.write(text)
        stats[proc] = st
        if verbose:
            print(proc, st)
    return stats
