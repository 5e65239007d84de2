"""Seeded synthetic inputs: a counter-based RNG and the RAMBO flat phase-space generator.

This module is the one input source shared by the CPU oracle's tests, the GPU parity
tests and ``bench.py``.  It holds none of the matrix-element arithmetic: it only makes
the batches of momenta and random numbers that the multi-event interface consumes
(the standalone testbed of the paper's Section 2 / Fig. 1b generates its test batches
with RAMBO in exactly this role).

Random numbers
--------------
Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11).  Every uniform is a pure function of (seed, event index, stream,
draw index), so an event's inputs do not depend on how a workload is split into
batches or requests.

* key     = (seed mod 2^32, seed div 2^32)
* counter = (event mod 2^32, event div 2^32, draw // 2, stream)
* draw j uses output words (x0, x1) when j is even and (x2, x3) when j is odd;
  u = (((hi << 32 | lo) >> 12) + 0.5) * 2^-52, which lies strictly inside (0, 1).

Streams: 0 = RAMBO momenta (4 draws per final-state particle), 1 = alpha_s,
2 = helicity-selection number, 3 = colour-selection number.

RAMBO
-----
Kleiss, Stirling, Ellis, Comput. Phys. Commun. 40 (1986) 359: isotropic massless
vectors with energies drawn from q0 e^{-q0}, a conformal boost to the centre of mass
and a scale to sqrt(s); massive final states are reached by rescaling all
three-momenta by one factor xi, found by Newton iteration on
sum_i sqrt(m_i^2 + xi^2 E_i^2) = sqrt(s).
"""
from __future__ import annotations

import numpy as np

_MASK32 = np.uint64(0xFFFFFFFF)
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)

STREAM_MOMENTA = 0
STREAM_ALPHAS = 1
STREAM_RND_HEL = 2
STREAM_RND_COL = 3


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox rounds on uint64 arrays holding 32-bit values (SC'11 definition)."""
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & _MASK32 for x in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK32
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK32
    for r in range(10):
        if r > 0:
            k0 = (k0 + _W0) & _MASK32
            k1 = (k1 + _W1) & _MASK32
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def uniforms(seed: int, events: np.ndarray, stream: int, ndraw: int) -> np.ndarray:
    """Uniforms in (0,1), shape [len(events), ndraw], keyed by (seed, event, stream, draw)."""
    ev = np.asarray(events, dtype=np.uint64)
    out = np.empty((ev.shape[0], ndraw), dtype=np.float64)
    k0 = np.uint64(seed & 0xFFFFFFFF)
    k1 = np.uint64((seed >> 32) & 0xFFFFFFFF)
    e_lo = ev & _MASK32
    e_hi = ev >> np.uint64(32)
    for call in range((ndraw + 1) // 2):
        x0, x1, x2, x3 = philox4x32_10(e_lo, e_hi, np.uint64(call), np.uint64(stream), k0, k1)
        for half, (hi, lo) in enumerate(((x0, x1), (x2, x3))):
            j = 2 * call + half
            if j >= ndraw:
                break
            bits = ((hi << np.uint64(32)) | lo) >> np.uint64(12)
            out[:, j] = (bits.astype(np.float64) + 0.5) * 2.0 ** -52
    return out


def rambo(sqrt_s: float, masses_final, seed: int, nevt: int, first_event: int = 0,
          max_newton: int = 50) -> np.ndarray:
    """RAMBO momenta [nevt][2 + n_final][4] (E, px, py, pz), FP64.

    Particles 0 and 1 are the incoming beams along +z and -z with sqrt(s)/2 each;
    the final-state particles follow in the order of ``masses_final``.
    """
    masses = np.asarray(masses_final, dtype=np.float64)
    n = masses.shape[0]
    ev = np.arange(first_event, first_event + nevt, dtype=np.uint64)
    u = uniforms(seed, ev, STREAM_MOMENTA, 4 * n)
    q = np.empty((nevt, n, 4))
    for i in range(n):
        c = 2.0 * u[:, 4 * i] - 1.0
        phi = 2.0 * np.pi * u[:, 4 * i + 1]
        q0 = -np.log(u[:, 4 * i + 2] * u[:, 4 * i + 3])
        st = np.sqrt(1.0 - c * c)
        q[:, i, 0] = q0
        q[:, i, 1] = q0 * st * np.cos(phi)
        q[:, i, 2] = q0 * st * np.sin(phi)
        q[:, i, 3] = q0 * c
    Q = q.sum(axis=1)
    M = np.sqrt(Q[:, 0] ** 2 - Q[:, 1] ** 2 - Q[:, 2] ** 2 - Q[:, 3] ** 2)
    b = -Q[:, 1:] / M[:, None]
    gam = Q[:, 0] / M
    a = 1.0 / (1.0 + gam)
    x = sqrt_s / M
    p = np.empty_like(q)
    bq = np.einsum("ek,eik->ei", b, q[:, :, 1:])
    p[:, :, 0] = x[:, None] * (gam[:, None] * q[:, :, 0] + bq)
    p[:, :, 1:] = x[:, None, None] * (q[:, :, 1:] + b[:, None, :] * q[:, :, 0:1]
                                      + a[:, None, None] * bq[:, :, None] * b[:, None, :])
    # The boost multiplies the rounding of the massless vectors by up to its gamma factor,
    # which could leave a particle off its mass shell, the three-momenta not summing to
    # zero or the energies off sqrt(s) by 1e-11 relative -- enough to separate two exact
    # FP64 evaluations of a matrix element (which may route a propagator's momentum from
    # either side) by 1e-12.  So the residual of the three-momentum sum is taken out in
    # equal parts, each vector is put on the light cone (E = |p|), the rescaling xi solves
    # sum_i sqrt(m_i^2 + xi^2 |p_i|^2) = sqrt(s) for massless and massive final states
    # alike, and each final energy comes from its final three-momentum: momentum
    # conservation and every mass shell hold to rounding.
    resid = p[:, :, 1:].sum(axis=1)
    p[:, :, 1:] -= resid[:, None, :] / n
    E = np.sqrt(p[:, :, 1] * p[:, :, 1] + p[:, :, 2] * p[:, :, 2] + p[:, :, 3] * p[:, :, 3])
    xi = np.full(nevt, np.sqrt(max(0.0, 1.0 - (masses.sum() / sqrt_s) ** 2)))
    done = np.zeros(nevt, dtype=bool)
    for _ in range(max_newton):
        r = np.sqrt(masses[None, :] ** 2 + (xi[:, None] * E) ** 2)
        f = r.sum(axis=1) - sqrt_s
        done |= np.abs(f) <= 1e-15 * sqrt_s
        if done.all():
            break
        fp = (xi[:, None] * E * E / r).sum(axis=1)
        xi = np.where(done, xi, xi - f / fp)
    if not done.all():
        raise RuntimeError("RAMBO mass rescaling did not converge")
    p[:, :, 1:] *= xi[:, None, None]
    p3 = p[:, :, 1:]
    p[:, :, 0] = np.sqrt(masses[None, :] ** 2 + (p3[..., 0] * p3[..., 0] + p3[..., 1] * p3[..., 1]
                                                 + p3[..., 2] * p3[..., 2]))
    out = np.empty((nevt, n + 2, 4))
    half = 0.5 * sqrt_s
    out[:, 0] = (half, 0.0, 0.0, half)
    out[:, 1] = (half, 0.0, 0.0, -half)
    out[:, 2:] = p
    return out


# ---------------------------------------------------------------------------
# Process catalogue for input generation only (masses of the final state).
# ---------------------------------------------------------------------------
PROCESS_FINAL_MASSES = {
    "e+ e- > mu+ mu-": lambda mt: (0.0, 0.0),
    "g g > t t~": lambda mt: (mt, mt),
    "g g > t t~ g": lambda mt: (mt, mt, 0.0),
    "g g > t t~ g g": lambda mt: (mt, mt, 0.0, 0.0),
    "g g > t t~ g g g": lambda mt: (mt, mt, 0.0, 0.0, 0.0),
    "u u~ > t t~": lambda mt: (mt, mt),
    "u~ u > t t~": lambda mt: (mt, mt),
    "u u~ > t t~ g": lambda mt: (mt, mt, 0.0),
    "u~ u > t t~ g": lambda mt: (mt, mt, 0.0),
    "u g > t t~ u": lambda mt: (mt, mt, 0.0),
    "g u > t t~ u": lambda mt: (mt, mt, 0.0),
    "u~ g > t t~ u~": lambda mt: (mt, mt, 0.0),
    "g u~ > t t~ u~": lambda mt: (mt, mt, 0.0),
    "u u~ > t t~ g g": lambda mt: (mt, mt, 0.0, 0.0),
    "u~ u > t t~ g g": lambda mt: (mt, mt, 0.0, 0.0),
    "u g > t t~ u g": lambda mt: (mt, mt, 0.0, 0.0),
    "g u > t t~ u g": lambda mt: (mt, mt, 0.0, 0.0),
    "u~ g > t t~ u~ g": lambda mt: (mt, mt, 0.0, 0.0),
    "g u~ > t t~ u~ g": lambda mt: (mt, mt, 0.0, 0.0),
    "g g > t t~ u u~": lambda mt: (mt, mt, 0.0, 0.0),
    "u u~ > t t~ d d~": lambda mt: (mt, mt, 0.0, 0.0),
    "u~ u > t t~ d d~": lambda mt: (mt, mt, 0.0, 0.0),
    "u d > t t~ u d": lambda mt: (mt, mt, 0.0, 0.0),
    "u d~ > t t~ u d~": lambda mt: (mt, mt, 0.0, 0.0),
    "u~ d~ > t t~ u~ d~": lambda mt: (mt, mt, 0.0, 0.0),
    "u u > t t~ u u": lambda mt: (mt, mt, 0.0, 0.0),
    "u~ u~ > t t~ u~ u~": lambda mt: (mt, mt, 0.0, 0.0),
    "u u~ > t t~ u u~": lambda mt: (mt, mt, 0.0, 0.0),
    "u~ u > t t~ u u~": lambda mt: (mt, mt, 0.0, 0.0),
}


def make_batch(process: str, nevt: int, seed: int = 0, first_event: int = 0,
               sqrt_s: float = 1500.0, mt: float = 173.0, alphas=None):
    """One synthetic batch: momenta, alphas, rnd_hel, rnd_col (all FP64 numpy arrays).

    ``alphas`` is either a float (fixed coupling for every event), ``"uniform"`` for
    alpha_s = 0.10 + 0.03 u drawn per event from stream 1, or None (no array).
    """
    masses = PROCESS_FINAL_MASSES[process](mt)
    mom = rambo(sqrt_s, masses, seed, nevt, first_event)
    ev = np.arange(first_event, first_event + nevt, dtype=np.uint64)
    if alphas is None:
        a = None
    elif isinstance(alphas, str):
        if alphas != "uniform":
            raise ValueError(alphas)
        a = 0.10 + 0.03 * uniforms(seed, ev, STREAM_ALPHAS, 1)[:, 0]
    else:
        a = np.full(nevt, float(alphas))
    rh = uniforms(seed, ev, STREAM_RND_HEL, 1)[:, 0]
    rc = uniforms(seed, ev, STREAM_RND_COL, 1)[:, 0]
    return mom, a, rh, rc
