"""Nearly collinear test events (shared by the CPU pins of the oracle's invariants and
the GPU parity tests).

Events whose gluon propagator is nearly on shell, at sqrt(s):
* g g > t t~ g g: the two final gluons are a small angle theta apart, so the
  s-channel invariant is (k1 + k2)^2 ~ E1 E2 theta^2;
* g g > t t~ g: the final gluon is theta from the first beam, so the t-channel
  invariant is (p1 - k)^2 ~ -E1 E theta^2.
The gluons are massless, E (1, n), and the top pair balances them.  The invariant is
then 1e4 to 1e6 times smaller than the square of the summed energies.
"""
import numpy as np

GGTTG = "g g > t t~ g"
GGTTGG = "g g > t t~ g g"

# the nearly light-like propagator momentum of the events below, as signed particles
COLLINEAR_TERMS = {GGTTG: ((1, 0), (-1, 4)), GGTTGG: ((1, 4), (1, 5))}


def top_pair(P, mt, rng):
    """t and t~ on the mass shell, back to back in the rest frame of P, boosted to the lab"""
    M = np.sqrt(P[0] ** 2 - P[1:] @ P[1:])
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    q = np.sqrt(M * M / 4 - mt * mt) * u
    out = []
    for qv in (q, -q):
        en = (P[0] * M / 2 + P[1:] @ qv) / M
        out.append(np.concatenate([[en], qv + P[1:] * (M / 2 + en) / (P[0] + M)]))
    return out


def collinear_events(process, n, seed, theta=(3e-3, 1e-2), sqrt_s=1500.0, mt=173.0):
    """n events of process (g g > t t~ g or g g > t t~ g g) with one nearly on-shell
    gluon propagator (see the module docstring), [n][npar][4]"""
    rng = np.random.default_rng(seed)
    npar = 6 if process == GGTTGG else 5
    mom = np.zeros((n, npar, 4))
    h = sqrt_s / 2
    p1, p2 = np.array([h, 0, 0, h]), np.array([h, 0, 0, -h])
    for e in range(n):
        th = rng.uniform(*theta)
        if process == GGTTGG:
            nv = rng.normal(size=3)
            nv /= np.linalg.norm(nv)
            m = np.cross(nv, rng.normal(size=3))
            m /= np.linalg.norm(m)
            n2 = np.cos(th) * nv + np.sin(th) * m
            e1, e2 = rng.uniform(100.0, 300.0, size=2)
            gl = [np.concatenate([[e1], e1 * nv]), np.concatenate([[e2], e2 * n2])]
        else:
            en, phi = rng.uniform(100.0, 300.0), rng.uniform(0, 2 * np.pi)
            gl = [en * np.array([1.0, np.sin(th) * np.cos(phi), np.sin(th) * np.sin(phi), np.cos(th)])]
        tops = top_pair(p1 + p2 - sum(gl), mt, rng)
        mom[e] = [p1, p2] + tops + gl
    return mom
