"""Evaluation schedule: which off-shell currents to build, how each diagram is closed,
and in which order, so that currents are computed once and shared by many diagrams.

Build-time generator code.  Node kinds (each identified by a hashable key):

  ("EXT", i)          external wavefunction of particle i
  ("G", tree)         off-shell gluon current of a gluon tree (propagator included)
  ("BRA", blocks)     ubar(top) with blocks B1..Bj attached, ending in a top propagator
  ("KET", blocks)     v(antitop) with blocks Bj..Br attached, ending in a top propagator
  ("PJ", bra, ket)    the fermion-pair vector current j^mu = BRA gamma^mu KET (no
                      propagator): the quark line with one block position left open

Every diagram term (B1..Br) is closed at the quark-gluon vertex of one block k, either
    DOT:  amp = PJ(B1..B(k-1) | B(k+1)..Br) . G(Bk)            (a Minkowski dot product)
or, when Bk is composite, with Bk's root vertex evaluated in place,
    V3 :  amp = PJ . V3(G(X), G(Y)) / K^2,   V4: amp = PJ . V4_s(G(X), G(Y), G(Z)) / K^2,
which all equal the usual vertex evaluation.  The generator picks the closing per
diagram to minimise a flop-weighted count of distinct currents plus closings: greedy
starts from several diagram orders, each followed by passes of local search that move
one diagram at a time.

Constant factors: the strong coupling is set to 1 inside the schedule (every
amplitude of q qbar + n gluons carries exactly g_s^n) and the factors of i of vertices
and propagators are tracked symbolically as a power of i per node, so that the
device code multiplies by no constants.  With the Feynman rules
  q-qbar-g: -i g gamma^mu T^a;  ggg: -g f V3;  gggg: -i g^2 (three f f structures);
  gluon propagator -i g_{mu nu}/K^2;  top propagator i (qslash + m)/(q^2 - m^2 + i m w)
the phases are:  G(three-gluon) i,  G(four-gluon) -1,  BRA/KET +1,  closing vertex -i.
"""
from __future__ import annotations

import random
from dataclasses import dataclass, field

from . import diagrams as dg


def g_node(tree):
    return ("EXT", tree[1]) if tree[0] == "L" else ("G", tree)


def bra_node(blocks, it):
    return ("EXT", it) if not blocks else ("BRA", tuple(blocks))


def ket_node(blocks, itb):
    return ("EXT", itb) if not blocks else ("KET", tuple(blocks))


def deps(node, it, itb):
    """direct inputs of a node"""
    kind = node[0]
    if kind == "EXT":
        return ()
    if kind == "G":
        t = node[1]
        kids = t[1:] if t[0] == "3" else t[2:]
        return tuple(g_node(k) for k in kids)
    if kind == "BRA":
        b = node[1]
        return (bra_node(b[:-1], it), g_node(b[-1]))
    if kind == "KET":
        b = node[1]
        return (g_node(b[0]), ket_node(b[1:], itb))
    if kind == "PJ":
        return (bra_node(node[1], it), ket_node(node[2], itb))
    raise ValueError(node)


# power of i carried by each node kind (see module docstring)
NODE_PHASE = {"EXT": 0, "G3": 1, "G4": 2, "BRA": 0, "KET": 0, "PJ": 0}
CLOSE_PHASE = 3  # -i


def node_phase(node):
    if node[0] == "G":
        return NODE_PHASE["G3"] if node[1][0] == "3" else NODE_PHASE["G4"]
    return NODE_PHASE[node[0]]


@dataclass
class Amp:
    kind: str              # "DOT": PJ . G;  "V3": PJ . V3(X, Y);  "V4": PJ . V4_s(X, Y, Z)
    inputs: tuple          # (PJ node, gluon node)  or  (PJ node, X, Y[, Z])
    struct: int            # four-gluon structure for "V4"
    diagram: tuple         # the diagram term
    colour: dict           # {flow index: complex coefficient}, phases folded in


@dataclass
class Schedule:
    nodes: list = field(default_factory=list)   # emission order of the currents
    amps: list = field(default_factory=list)    # emission order of the closings
    seq: list = field(default_factory=list)     # interleaved ("N", node) / ("A", amp index)


def _closure(node, it, itb, acc):
    if node in acc or node[0] == "EXT":
        return
    for d in deps(node, it, itb):
        _closure(d, it, itb, acc)
    acc.add(node)


def _options(D, it, itb):
    """(kind, inputs, struct, extra phase power) for each way to close D"""
    out = []
    for k in range(len(D)):
        pj = ("PJ", tuple(D[:k]), tuple(D[k + 1:]))
        blk = D[k]
        out.append(("DOT", (pj, g_node(blk)), 0, 0))
        if blk[0] == "3":
            # the block's root vertex evaluated in place: its phase joins the amplitude
            out.append(("V3", (pj, g_node(blk[1]), g_node(blk[2])), 0, NODE_PHASE["G3"]))
        elif blk[0] == "4":
            out.append(("V4", (pj,) + tuple(g_node(x) for x in blk[2:]), blk[1], NODE_PHASE["G4"]))
    return out


def _total_phase(inputs, extra, it, itb):
    """power of i of an amplitude: closing vertex, an in-place vertex and every node
    it depends on (a tree diagram uses each node once)."""
    acc = set()
    for n in inputs:
        _closure(n, it, itb, acc)
    return (CLOSE_PHASE + extra + sum(node_phase(n) for n in acc)) % 4


# relative cost (real flops, order of magnitude) of each node kind and closing kind
NODE_COST = {"G": 140, "BRA": 150, "KET": 150, "PJ": 60}
AMP_COST = {"DOT": 30, "V3": 160, "V4": 110}


def _optimise(opts, order, passes):
    cnt = {}

    def cost(o):
        return AMP_COST[o[0]] + sum(NODE_COST[n[0]] for n in o[4] if cnt.get(n, 0) == 0)

    choice = [0] * len(opts)
    for d in order:
        ol = opts[d]
        j = min(range(len(ol)), key=lambda k: cost(ol[k]))
        choice[d] = j
        for n in ol[j][4]:
            cnt[n] = cnt.get(n, 0) + 1
    for _ in range(passes):
        moved = 0
        for d in order:
            ol = opts[d]
            for n in ol[choice[d]][4]:
                cnt[n] -= 1
            j = min(range(len(ol)), key=lambda k: (cost(ol[k]), k != choice[d]))
            moved += j != choice[d]
            choice[d] = j
            for n in ol[j][4]:
                cnt[n] = cnt.get(n, 0) + 1
        if not moved:
            break
    total = sum(AMP_COST[opts[d][choice[d]][0]] for d in range(len(opts)))
    total += sum(NODE_COST[n[0]] for n, c in cnt.items() if c > 0)
    return total, choice


def emission_order(amps, it, itb, alpha=1.0):
    """Order the closings to keep few currents alive at once: repeatedly take the
    closing that needs the fewest currents not yet built, minus the number of built
    currents it is the last remaining user of.  Each closing's missing currents are
    emitted (inputs first) just before it."""
    need = []
    for a in amps:
        acc = set()
        for n in a.inputs:
            _closure(n, it, itb, acc)
        need.append(frozenset(acc))
    users = {}
    for i, nd in enumerate(need):
        for n in nd:
            users.setdefault(n, set()).add(i)
    done, emitted = set(), set()
    remaining = set(range(len(amps)))
    seq = []
    seen = set()

    def visit(n):
        if n in seen or n[0] == "EXT":
            return
        seen.add(n)
        for d in deps(n, it, itb):
            visit(d)
        seq.append(("N", n))

    while remaining:
        best = None
        for i in sorted(remaining):
            new = len(need[i] - emitted)
            kill = sum(1 for n in need[i] if n in emitted and users[n] - done <= {i})
            score = new - alpha * kill
            if best is None or score < best[0]:
                best = (score, i)
        i = best[1]
        for n in amps[i].inputs:
            visit(n)
        seq.append(("A", i))
        done.add(i)
        remaining.discard(i)
        emitted |= need[i]
    return seq


def build_qcd_schedule(gluons, it, itb, passes=12, restarts=24, seed=1):
    terms = dg.qcd_diagrams(gluons, split4=True)
    flows = dg.flow_index(gluons)
    opts = []
    for D in terms:
        ol = []
        for kind, inputs, s, extra in _options(D, it, itb):
            acc = set()
            for n in inputs:
                _closure(n, it, itb, acc)
            ol.append((kind, inputs, s, extra, frozenset(acc)))
        opts.append(ol)
    rng = random.Random(seed)
    best = None
    orders = [list(range(len(terms))), list(reversed(range(len(terms)))),
              sorted(range(len(terms)), key=lambda d: -len(terms[d]))]
    for r in range(restarts):
        if r < len(orders):
            order = orders[r]
        else:
            order = list(range(len(terms)))
            rng.shuffle(order)
        res = _optimise(opts, order, passes)
        if best is None or res[0] < best[0]:
            best = res
    _, choice = best
    amps = []
    for D, ol, j in zip(terms, opts, choice):
        kind, inputs, s, extra, _ = ol[j]
        ph = 1j ** _total_phase(inputs, extra, it, itb)
        col = {flows[k]: v * ph for k, v in dg.colour_expansion(D).items()}
        amps.append(Amp(kind, inputs, s, D, col))
    seq = emission_order(amps, it, itb)
    sched = Schedule()
    sched.seq = seq
    sched.nodes = [x for t, x in seq if t == "N"]
    sched.amps = amps
    return sched


def max_live(sched, it, itb):
    """largest number of simultaneously alive non-external currents in sched.seq"""
    last = {}
    for k, (t, x) in enumerate(sched.seq):
        ins = deps(x, it, itb) if t == "N" else sched.amps[x].inputs
        for d in ins:
            last[d] = k
    ev = []
    for k, (t, x) in enumerate(sched.seq):
        if t == "N":
            ev.append((k, 1))
            ev.append((last.get(x, k) + 0.5, -1))
    ev.sort()
    cur = mx = 0
    for _, d in ev:
        cur += d
        mx = max(mx, cur)
    return mx


def summary(s: Schedule):
    kinds, akinds = {}, {}
    for n in s.nodes:
        kinds[n[0]] = kinds.get(n[0], 0) + 1
    for a in s.amps:
        akinds[a.kind] = akinds.get(a.kind, 0) + 1
    cost = sum(NODE_COST[n[0]] for n in s.nodes) + sum(AMP_COST[a.kind] for a in s.amps)
    return {"nodes": kinds, "amps": akinds, "colour_pairs": sum(len(a.colour) for a in s.amps),
            "est_flops": cost}
