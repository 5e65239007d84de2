"""Explicit-colour brute force for g g -> t t~ + n gluons (a pin for the oracle).

Independent of the oracle in every choice that does not change the physical answer:
Dirac (not chiral) representation, spin states along z (not helicity), linear (not
circular) gluon polarisations, and full colour: gluon currents carry an explicit
adjoint index, the f^{abc} structure constants and the Gell-Mann matrices T^a = l^a/2
are written out, and the recursion runs over unordered subsets of gluons with the
plain Feynman rules, so no colour decomposition or colour matrix is involved.

Feynman rules (Feynman gauge; Peskin & Schroeder Fig. 16.7 with g -> -g):
  quark-gluon  -i g gamma^mu T^a
  3-gluon      -g f^{abc} [g^{mu nu}(k-p)^rho + g^{nu rho}(p-q)^mu + g^{rho mu}(q-k)^nu]
  4-gluon      -i g^2 [f^{abe}f^{cde}(g^{mu rho}g^{nu sigma} - g^{mu sigma}g^{nu rho})
                      + f^{ace}f^{bde}(g^{mu nu}g^{rho sigma} - g^{mu sigma}g^{nu rho})
                      + f^{ade}f^{bce}(g^{mu nu}g^{rho sigma} - g^{mu rho}g^{nu sigma})]
  propagators  -i g_{mu nu} delta^{ab}/k^2,  i(qslash + m)/(q^2 - m^2 + i m w)

The top width w is either the same in every top propagator, or (zero_width_tchan)
zero in each propagator whose momentum is in the t channel: written as a signed sum of
external momenta, it carries exactly one of the two incoming momenta, so it separates
the two beams.

Returns the spin- and colour-summed |M|^2 (not averaged).  Slow; small n only.
"""
import itertools

import numpy as np

METRIC = np.diag([1.0, -1.0, -1.0, -1.0])


def gell_mann():
    l = np.zeros((8, 3, 3), dtype=complex)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1], l[1][1, 0] = -1j, 1j
    l[2][0, 0], l[2][1, 1] = 1, -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2], l[4][2, 0] = -1j, 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2], l[6][2, 1] = -1j, 1j
    l[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    return l / 2


T = gell_mann()
# f^{abc} = -2 i Tr([T^a, T^b] T^c)
F = np.real(-2j * (np.einsum("aij,bjk,cki->abc", T, T, T) - np.einsum("bij,ajk,cki->abc", T, T, T)))

SIG = [np.eye(2), np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]])]
GAM = np.zeros((4, 4, 4), dtype=complex)
GAM[0] = np.diag([1, 1, -1, -1])
for k in (1, 2, 3):
    GAM[k][:2, 2:] = SIG[k]
    GAM[k][2:, :2] = -SIG[k]


def mdot(a, b):
    return a[..., 0] * b[..., 0] - a[..., 1] * b[..., 1] - a[..., 2] * b[..., 2] - a[..., 3] * b[..., 3]


def slash(a):
    """gamma^mu a_mu for a[..., 4] -> [..., 4, 4]."""
    al = a * np.array([1, -1, -1, -1])
    return np.einsum("...m,mij->...ij", al, GAM)


def dirac_spinors(p, m):
    """u(p,s), v(p,s) for s in the z basis; Dirac representation, normalised ubar u = 2m."""
    E = p[0]
    sp = SIG[1] * p[1] + SIG[2] * p[2] + SIG[3] * p[3]
    us, vs = [], []
    for chi in (np.array([1, 0]), np.array([0, 1])):
        us.append(np.sqrt(E + m) * np.concatenate([chi, sp @ chi / (E + m)]))
        vs.append(np.sqrt(E + m) * np.concatenate([sp @ chi / (E + m), chi]))
    return us, vs


def bar(s):
    return s.conj() @ GAM[0]


def linear_pols(k):
    """two real polarisation vectors orthogonal to k (and to the time axis)."""
    n = k[1:] / np.linalg.norm(k[1:])
    ref = np.array([1.0, 0, 0]) if abs(n[0]) < 0.9 else np.array([0, 1.0, 0])
    e1 = np.cross(n, ref)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(n, e1)
    return [np.concatenate([[0.0], e1]), np.concatenate([[0.0], e2])]


def v3_full(k1, J1, k2, J2, g):
    """-g f^{a b c} V^{mu nu rho}(k1, k2, q) J1^a_mu J2^b_nu for colour-carrying currents
    J[..., a, mu]; returns [..., c, rho]."""
    q = -(k1 + k2)
    a = k2 - q
    b = q - k1
    d12 = k1 - k2
    j12 = np.einsum("...am,...bm,m->...ab", J1, J2, np.diag(METRIC))
    aj1 = np.einsum("...am,m->...a", J1, a * np.diag(METRIC))
    bj2 = np.einsum("...bm,m->...b", J2, b * np.diag(METRIC))
    out = (np.einsum("abc,...ab,r->...cr", F, j12, d12)
           + np.einsum("abc,...a,...br->...cr", F, aj1, J2)
           + np.einsum("abc,...ar,...b->...cr", F, J1, bj2))
    return -g * out


def v4_full(J1, J2, J3, g):
    """full four-gluon vertex contracted with three colour-carrying currents."""
    gm = np.diag(METRIC)
    d12 = np.einsum("...am,...bm,m->...ab", J1, J2, gm)
    d13 = np.einsum("...am,...cm,m->...ac", J1, J3, gm)
    d23 = np.einsum("...bm,...cm,m->...bc", J2, J3, gm)
    ff1 = np.einsum("abe,cde->abcd", F, F)
    ff2 = np.einsum("ace,bde->abcd", F, F)
    ff3 = np.einsum("ade,bce->abcd", F, F)
    out = (np.einsum("abcd,...ac,...bs->...ds", ff1, d13, J2) - np.einsum("abcd,...bc,...as->...ds", ff1, d23, J1)
           + np.einsum("abcd,...ab,...cs->...ds", ff2, d12, J3) - np.einsum("abcd,...bc,...as->...ds", ff2, d23, J1)
           + np.einsum("abcd,...ab,...cs->...ds", ff3, d12, J3) - np.einsum("abcd,...ac,...bs->...ds", ff3, d13, J2))
    return -1j * g * g * out


def set_partitions(items, nparts):
    """unordered partitions of a tuple into nparts non-empty blocks."""
    items = list(items)
    if nparts == 1:
        yield (tuple(items),)
        return
    first, rest = items[0], items[1:]
    # the block holding 'first'
    for r in range(0, len(rest) + 1):
        for comb in itertools.combinations(rest, r):
            block = (first,) + comb
            remaining = [x for x in rest if x not in comb]
            if len(remaining) < nparts - 1:
                continue
            for tail in set_partitions(remaining, nparts - 1):
                yield (block,) + tail


def summed_me2(mom, mt, gs, roles, wt=0.0, zero_width_tchan=False):
    """sum over spins, polarisations and colours of |M|^2 for g g -> t t~ + gluons.

    roles: list of 'gin', 'gout', 't', 'tb' in particle order; wt: top width; with
    zero_width_tchan, no width in t-channel top propagators (see the module docstring).
    """
    gl = [i for i, r in enumerate(roles) if r in ("gin", "gout")]
    it = roles.index("t")
    itb = roles.index("tb")
    n = len(gl)
    kin = {i: (mom[i] if roles[i] == "gin" else -mom[i]) for i in gl}
    pols = {i: linear_pols(mom[i]) for i in gl}
    us, _ = dirac_spinors(mom[it], mt)
    _, vs = dirac_spinors(mom[itb], mt)
    ncfg = 8 ** n
    # colour assignment index A -> colour of gluon slot j
    acol = np.array(list(itertools.product(range(8), repeat=n)))  # [ncfg, n]
    total = 0.0
    for pol_choice in itertools.product(range(2), repeat=n):
        J = {}
        K = {}
        for j, i in enumerate(gl):
            e = pols[i][pol_choice[j]].astype(complex)
            cur = np.zeros((ncfg, 8, 4), dtype=complex)
            cur[np.arange(ncfg), acol[:, j], :] = e
            J[(i,)] = cur
            K[(i,)] = kin[i]
        for size in range(2, n + 1):
            for S in itertools.combinations(gl, size):
                Ks = sum(kin[i] for i in S)
                K[S] = Ks
                acc = np.zeros((ncfg, 8, 4), dtype=complex)
                for S1, S2 in set_partitions(S, 2):
                    acc += v3_full(K[S1], J[S1], K[S2], J[S2], gs)
                for S1, S2, S3 in set_partitions(S, 3):
                    acc += v4_full(J[S1], J[S2], J[S3], gs)
                J[S] = (-1j / mdot(Ks, Ks)) * acc
        # quark line over ordered sequences of disjoint subsets, from the top end
        allg = tuple(gl)
        # Gamma(B)[A, colour row, colour col, spin, spin] = -i g gamma.J_B^c T^c
        Gam = {}
        for S in J:
            sl = slash(J[S])  # [A, c, 4, 4]
            Gam[S] = -1j * gs * np.einsum("Acij,ckl->Aklij", sl, T)
        for ut in us:
            ub = bar(ut)
            for vt in vs:
                U = {(): np.broadcast_to(np.einsum("kl,s->kls", np.eye(3), ub), (ncfg, 3, 3, 4)).copy()}
                order = sorted((S for S in itertools.chain.from_iterable(
                    itertools.combinations(allg, r) for r in range(1, n + 1))), key=len)
                amp = np.zeros((ncfg, 3, 3), dtype=complex)
                for R in order:
                    acc = np.zeros((ncfg, 3, 3, 4), dtype=complex)
                    for r in range(1, len(R) + 1):
                        for B in itertools.combinations(R, r):
                            rest = tuple(x for x in R if x not in B)
                            if rest not in U:
                                continue
                            acc += np.einsum("Aiks,Aklst->Ailt", U[rest], Gam[tuple(sorted(B))])
                    if R == allg:
                        amp = np.einsum("Ailt,t->Ail", acc, vt)
                    else:
                        # q = p_t - sum of the incoming momenta of the gluons R on the top
                        # side; as a sum of external momenta it holds p_in for each
                        # incoming gluon in R
                        q = mom[it] - K[R]
                        n_beams = sum(1 for i in R if roles[i] == "gin")
                        w = 0.0 if (zero_width_tchan and n_beams == 1) else wt
                        prop = (1j * (slash(q.astype(complex)) + mt * np.eye(4))
                                / (mdot(q, q) - mt * mt + 1j * mt * w))
                        U[R] = np.einsum("Ailt,tu->Ailu", acc, prop)
                total += float(np.sum(np.abs(amp) ** 2))
    return total
