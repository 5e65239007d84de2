"""Pins for the seeded input generator (Philox4x32-10 and RAMBO)."""
import os

import numpy as np
import pytest

from paper_2312_02898_b300 import phasespace as ps

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def test_philox_known_answers():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = ps.philox4x32_10(*v[:6])
        assert [int(o) for o in out] == v[6:]


def test_uniforms_open_interval_and_batch_independent():
    ev = np.arange(0, 4096, dtype=np.uint64)
    u = ps.uniforms(7, ev, 0, 5)
    assert u.min() > 0.0 and u.max() < 1.0
    # the same event drawn inside another batch gives the same numbers
    u2 = ps.uniforms(7, ev[100:200], 0, 5)
    assert np.array_equal(u[100:200], u2)
    # streams and seeds decorrelate
    assert not np.array_equal(u, ps.uniforms(8, ev, 0, 5))
    assert not np.array_equal(u, ps.uniforms(7, ev, 1, 5))
    assert abs(u.mean() - 0.5) < 0.01


@pytest.mark.parametrize("process", list(ps.PROCESS_FINAL_MASSES))
def test_rambo_conservation_and_mass_shell(process):
    mom, _, _, _ = ps.make_batch(process, 2000, seed=3)
    sqrt_s = 1500.0
    tot_in = mom[:, 0] + mom[:, 1]
    tot_out = mom[:, 2:].sum(axis=1)
    assert np.abs(tot_in - tot_out).max() <= 1e-12 * sqrt_s
    masses = np.array(ps.PROCESS_FINAL_MASSES[process](173.0))
    m2 = mom[:, 2:, 0] ** 2 - (mom[:, 2:, 1:] ** 2).sum(-1)
    # relative to E^2: the conformal boost amplifies component rounding by its gamma
    assert (np.abs(m2 - masses ** 2) / mom[:, 2:, 0] ** 2).max() <= 1e-11
    assert (mom[:, 2:, 0] > 0).all()


def test_rambo_two_body_isotropic():
    # flat two-body phase space: cos(theta) of the first final particle is uniform
    mom, _, _, _ = ps.make_batch("g g > t t~", 200000, seed=11)
    c = mom[:, 2, 3] / np.linalg.norm(mom[:, 2, 1:], axis=1)
    hist, _ = np.histogram(c, bins=10, range=(-1, 1))
    assert np.all(np.abs(hist / hist.mean() - 1) < 0.03)
    # fixed top energy sqrt(s)/2 for equal masses (rare nearly collinear RAMBO seeds
    # have a large conformal boost, which costs a few digits)
    assert np.allclose(mom[:, 2, 0], 750.0, rtol=1e-9, atol=0)
    assert np.median(np.abs(mom[:, 2, 0] / 750.0 - 1)) < 1e-14


def test_make_batch_alphas_streams():
    _, a, rh, rc = ps.make_batch("g g > t t~ g g", 1000, seed=0, alphas="uniform")
    assert a.min() >= 0.10 and a.max() <= 0.13
    assert not np.array_equal(rh, rc)
    _, a2, _, _ = ps.make_batch("g g > t t~ g g", 1000, seed=0, alphas=0.118)
    assert np.all(a2 == 0.118)


@pytest.mark.parametrize("process", ["g g > t t~", "g g > t t~ g g", "e+ e- > mu+ mu-"])
def test_rambo_particles_on_shell_to_rounding(process):
    """Every final particle is on its mass shell to the rounding of its own components,
    and the final momenta add up to (sqrt(s), 0, 0, 0) to rounding, also on the rare
    events whose RAMBO boost amplifies the rounding of the massless vectors."""
    mom, _, _, _ = ps.make_batch(process, 20000, seed=51)
    masses = np.array(ps.PROCESS_FINAL_MASSES[process](173.0))
    p = mom[:, 2:]
    m2 = p[..., 0] ** 2 - np.sum(p[..., 1:] ** 2, axis=-1)
    assert np.max(np.abs(m2 - masses ** 2) / p[..., 0] ** 2) <= 4e-16
    assert np.max(np.abs(p[..., 0].sum(axis=1) - 1500.0)) <= 4e-15 * 1500.0
    assert np.max(np.abs(p[..., 1:].sum(axis=1))) <= 4e-15 * 1500.0
