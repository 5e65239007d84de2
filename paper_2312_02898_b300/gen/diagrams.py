"""Tree-level Feynman diagrams of q qbar + n gluons and their colour-flow expansion.

Build-time generator code (runs on the host when the CUDA sources are generated).

A diagram of g g -> t t~ + gluons has one quark line running from the outgoing top
(bra end, ubar) to the outgoing antitop (ket end, v).  Gluon subtrees ("blocks") hang
off that line in a definite order; each block is a rooted tree of three- and
four-gluon vertices whose leaves are external gluons.  Enumerating every ordered
sequence of blocks that partitions the gluons, with every tree shape for each block,
gives every diagram exactly once (2 -> 3, 3 -> 16, 4 -> 123, 5 -> 1240 diagrams).

Colour: with Tr(T^a T^b) = delta/2 and [T^a, T^b] = i f^{abc} T^c, a three-gluon
vertex f^{x y c} whose leg c points toward the quark line contributes
sum_c f^{xyc} T^c = -i [T^x, T^y]; the three colour structures of the four-gluon
vertex contribute -[[T^x,T^y],T^z], -[[T^x,T^z],T^y] and -[[T^y,T^z],T^x].  Expanding
every diagram this way writes its colour factor as a sum of strings
(T^{a_s1} ... T^{a_sn})_{i_t j_tbar} with coefficients in {+-1, +-i}: the colour-flow
basis, indexed by the lexicographic rank of the permutation s of the gluon particle
indices.
"""
from __future__ import annotations

import itertools
from functools import lru_cache

# A tree is a nested tuple:
#   ("L", i)              external gluon with particle index i
#   ("3", X, Y)           three-gluon vertex, legs in the order (X, Y, root)
#   ("4", s, X, Y, Z)     one colour/Lorentz structure s in {1,2,3} of the
#                         four-gluon vertex, legs (X, Y, Z, root)


def leaves(t) -> tuple:
    if t[0] == "L":
        return (t[1],)
    kids = t[1:] if t[0] == "3" else t[2:]
    return tuple(sorted(sum((leaves(k) for k in kids), ())))


def _key(t):
    return (leaves(t), repr(t))


def unordered_partitions(items, nparts):
    """Partitions of a sorted tuple into nparts unordered non-empty blocks."""
    items = tuple(items)
    if nparts == 1:
        yield (items,)
        return
    first, rest = items[0], items[1:]
    for r in range(len(rest) + 1):
        for comb in itertools.combinations(rest, r):
            block = (first,) + comb
            remaining = tuple(x for x in rest if x not in comb)
            if len(remaining) < nparts - 1:
                continue
            for tail in unordered_partitions(remaining, nparts - 1):
                yield (block,) + tail


@lru_cache(maxsize=None)
def trees(subset: tuple, split4: bool) -> tuple:
    """All rooted gluon trees with leaf set ``subset`` (sorted tuple).

    With split4, a four-gluon vertex appears as its three structures (three trees);
    without, as one tree ("4", 0, ...) so that diagrams are counted once.
    """
    if len(subset) == 1:
        return (("L", subset[0]),)
    out = []
    for a, b in unordered_partitions(subset, 2):
        for x in trees(a, split4):
            for y in trees(b, split4):
                out.append(("3",) + tuple(sorted((x, y), key=_key)))
    for a, b, c in unordered_partitions(subset, 3):
        for x in trees(a, split4):
            for y in trees(b, split4):
                for z in trees(c, split4):
                    kids = tuple(sorted((x, y, z), key=_key))
                    for s in ((1, 2, 3) if split4 else (0,)):
                        out.append(("4", s) + kids)
    return tuple(out)


def ordered_set_partitions(items):
    """Ordered sequences of disjoint non-empty blocks covering items."""
    items = tuple(items)
    if not items:
        yield ()
        return
    for r in range(1, len(items) + 1):
        for first in itertools.combinations(items, r):
            rest = tuple(x for x in items if x not in first)
            for tail in ordered_set_partitions(rest):
                yield (first,) + tail


def qcd_diagrams(gluons, split4: bool):
    """Every diagram (or diagram term, with split4) as a tuple of block trees ordered
    from the top (bra) end of the quark line to the antitop (ket) end."""
    out = []
    for seq in ordered_set_partitions(tuple(sorted(gluons))):
        for combo in itertools.product(*(trees(b, split4) for b in seq)):
            out.append(combo)
    return out


# ----------------------------------------------------------------------------
# colour expansion
# ----------------------------------------------------------------------------
def _cat(e1, e2):
    out = {}
    for s1, c1 in e1.items():
        for s2, c2 in e2.items():
            k = s1 + s2
            out[k] = out.get(k, 0) + c1 * c2
    return out


def _add(e1, e2, f=1):
    out = dict(e1)
    for k, v in e2.items():
        out[k] = out.get(k, 0) + f * v
    return {k: v for k, v in out.items() if v != 0}


def _comm(e1, e2):
    return _add(_cat(e1, e2), _cat(e2, e1), -1)


@lru_cache(maxsize=None)
def _colour_tree(t):
    if t[0] == "L":
        return (((t[1],), 1),)
    if t[0] == "3":
        x, y = (dict(_colour_tree(k)) for k in t[1:])
        e = {k: -1j * v for k, v in _comm(x, y).items()}
    else:
        s = t[1]
        x, y, z = (dict(_colour_tree(k)) for k in t[2:])
        if s == 1:
            e = _comm(_comm(x, y), z)
        elif s == 2:
            e = _comm(_comm(x, z), y)
        elif s == 3:
            e = _comm(_comm(y, z), x)
        else:
            raise ValueError("colour of an unsplit four-gluon vertex")
        e = {k: -v for k, v in e.items()}
    return tuple(sorted(e.items()))


def colour_expansion(diagram):
    """{gluon-order tuple: coefficient} for a diagram term (blocks from the top end)."""
    e = {(): 1}
    for blk in diagram:
        e = _cat(e, dict(_colour_tree(blk)))
    return {k: v for k, v in e.items() if v != 0}


def flow_index(gluons):
    """map gluon-order tuple -> lexicographic rank among permutations of the gluons."""
    return {p: i for i, p in enumerate(itertools.permutations(sorted(gluons)))}
