"""The pending colour sums of the generated gluon-process code (gen/emit.py): amplitudes
whose colour vectors agree up to a factor 1, i, -1 or -i are summed in registers before
they are added into the colour-flow amplitudes J.

The emitted accumulation statements of a jamps variant are read back and executed on
symbols (each closing's amplitude a_k a symbol; the pending sums and J linear
combinations of them): at the end of the helicity body every J_c must be exactly
sum_k colour_k[c] a_k with the colour coefficients of the schedule, whatever the number of
pending sums and wherever the diagram groups split the body.  The GPU parity tests run
the same code against the oracle."""
import re

import pytest

from paper_2312_02898_b300.gen import emit
from paper_2312_02898_b300.gen import schedule as sc

OP = re.compile(r"(J\[\d+\]|pc\d+) (\+=|-=) (a|pc\d+);|acc_(pi|mi)\((J\[\d+\]|pc\d+), (a|pc\d+)\);|"
                r"(pc\d+) = (a|mk<R>\([^;]*\));")
INIT = {"a": 1, "mk<R>(-a.r, -a.i)": -1, "mk<R>(a.i, -a.r)": -1j, "mk<R>(-a.i, a.r)": 1j}


def run_symbolic(lines):
    """execute the accumulation statements of one jamps variant; returns (J, number of
    closings, number of scalar adds into J and into the pending sums)"""
    val, k, adds = {}, -1, 0

    def get(name):
        return val.setdefault(name, {})

    def add(dst, src, coef):
        d = get(dst)
        for j, c in (({k: 1} if src == "a" else get(src))).items():
            d[j] = d.get(j, 0) + coef * c

    for line in lines:
        if "const cx<R> a = close_" in line:
            k += 1
        for m in OP.finditer(line):
            if m.group(1):
                add(m.group(1), m.group(3), 1 if m.group(2) == "+=" else -1)
                adds += 2
            elif m.group(4):
                add(m.group(5), m.group(6), 1j if m.group(4) == "pi" else -1j)
                adds += 2
            else:
                val[m.group(7)] = {k: INIT[m.group(8)]}
    return {n: v for n, v in val.items() if n.startswith("J")}, k + 1, adds


@pytest.fixture(scope="module")
def ggttgg():
    em = emit.Emitter("g g > t t~ g g")
    variants = ((6, None), (6, None, 4), (20, None, 12), (10, 160, 4), (10, 40, 12))
    text, _ = em.emit_qcd(budgets=variants)
    it, itb = em.roles.index("t"), em.roles.index("tb")
    sched = sc.build_qcd_schedule(em.gluons, it, itb, restarts=24)
    colours = [sched.amps[x].colour for t, x in sched.seq if t == "A"]
    return text, variants, colours


def variant_lines(text, vi):
    """the statements of jamps variant vi: its function, or its diagram groups in order
    followed by the wrapper that calls them (which accumulates nothing)"""
    out, on = [], False
    head = re.compile(rf"static (HD|NOINL) void jamps_v{vi}(_g\d+)?\(")
    for line in text.splitlines():
        if head.match(line):
            on = True
        elif on and line.startswith("}"):
            on = False
        elif on:
            out.append(line)
    return out


@pytest.mark.parametrize("vi", range(5))
def test_every_flow_gets_each_amplitude_once(ggttgg, vi):
    text, variants, colours = ggttgg
    J, nclosing, adds = run_symbolic(variant_lines(text, vi))
    assert nclosing == len(colours) == 159
    want = {}
    for k, col in enumerate(colours):
        for c, v in col.items():
            want.setdefault(f"J[{c}]", {})[k] = complex(v)
    assert set(J) == set(want)
    for name, terms in want.items():
        got = {j: c for j, c in J[name].items() if c != 0}
        assert got.keys() == terms.keys(), name
        for j, c in terms.items():
            assert got[j] == c, (name, j, got[j], c)
    direct = 2 * sum(len(c) for c in colours)
    npend = variants[vi][2] if len(variants[vi]) > 2 else 0
    if npend == 0:
        assert adds == direct == 1344
    else:
        # summing amplitudes of one colour class first takes fewer adds
        assert adds < direct


def test_pending_plan_respects_groups_and_capacity():
    """the plan never keeps more than npend classes pending, never carries a sum across
    a group boundary, and flushes every class it opens"""
    keys = ["A", "B", "A", "C", "B", "A", "C", "D", "A", "D"]
    segs = [0, 0, 0, 0, 0, 1, 1, 1, 1, 1]
    for npend in (0, 1, 2, 3):
        plan = emit._pending_plan(keys, segs, npend)
        live = {}
        for j, (act, slot, flushes) in enumerate(plan):
            for s, key in flushes:
                assert live.pop(s) == (key, segs[j])
            if act == "open":
                assert slot not in live and len(live) < npend
                live[slot] = (keys[j], segs[j])
            elif act in ("merge", "last"):
                assert live[slot] == (keys[j], segs[j])
                if act == "last":
                    del live[slot]
            else:
                assert slot is None
            assert len(live) <= npend
            if j + 1 < len(keys) and segs[j + 1] != segs[j]:
                assert not live
        assert not live
