"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle, event by
event, on identical seeded RAMBO inputs.

Bars: FP64 mode max relative error <= 1e-12 on every event; FP32 mode <= 1e-5 (max and
median printed); selected helicity and colour identical except where r * total lies
within a relative 1e-10 (FP64) of a running-sum boundary.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2312_02898_b300 import phasespace as ps
from tests.collinear import COLLINEAR_TERMS, collinear_events

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

PROCS = ["e+ e- > mu+ mu-", "g g > t t~", "g g > t t~ g", "g g > t t~ g g", "g g > t t~ g g g"]
# ME_B300_TEST_PROCS="0,1,2,3" restricts a development run to some processes
_SEL = os.environ.get("ME_B300_TEST_PROCS")
ACTIVE = [PROCS[int(i)] for i in _SEL.split(",")] if _SEL else PROCS
# several thread blocks plus a ragged tail, small enough for the oracle in seconds
NEV = {PROCS[0]: 1000, PROCS[1]: 1000, PROCS[2]: 700, PROCS[3]: 300, PROCS[4]: 77}
FP32_BOUND = 1e-5


def mk(process, precision="fp64", **kw):
    from paper_2312_02898_b300.binding import MatrixElement
    return MatrixElement(process, precision=precision, **kw)


def to_dev(*arrs):
    return [None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def boundary_ok(sel_gpu, sel_ref, weights, r, rel):
    """selection equal, or r*total within rel*total of a running-sum boundary"""
    for e in np.nonzero(sel_gpu != sel_ref)[0]:
        c = np.cumsum(weights[e])
        if np.min(np.abs(c - r[e] * c[-1])) > rel * c[-1]:
            return False, e
    return True, None


_ref_cache = {}


def reference(process, nevt, seed=0, alphas="uniform"):
    key = (process, nevt, seed, alphas)
    if key not in _ref_cache:
        mom, a, rh, rc = ps.make_batch(process, nevt, seed=seed, alphas=alphas)
        ref = oracle.me(process, mom, alphas=a, rnd_hel=rh, rnd_col=rc, want_hel=True, want_colw=True)
        _ref_cache[key] = (mom, a, rh, rc, ref)
    return _ref_cache[key]


def run_gpu(m, mom, a, rh, rc):
    me, sh, sc = m.compute(*to_dev(mom, a, rh, rc))
    torch.cuda.synchronize()
    return me.cpu().numpy(), sh.cpu().numpy(), sc.cpu().numpy()


@pytest.mark.parametrize("process", ACTIVE)
def test_fp64_parity(process):
    mom, a, rh, rc, ref = reference(process, NEV[process])
    m = mk(process, "fp64")
    for config in range(m.nconfig):
        m.set_config(config)
        me, sh, sc = run_gpu(m, mom, a, rh, rc)
        rel = np.abs(me / ref["me"] - 1)
        assert rel.max() <= 1e-12, (config, rel.max(), np.argmax(rel))
        ok, e = boundary_ok(sh, ref["sel_hel"], ref["me_hel"], rh, 1e-10)
        assert ok, ("sel_hel", config, e)
        ok, e = boundary_ok(sc, ref["sel_col"], ref["colw"], rc, 1e-10)
        assert ok, ("sel_col", config, e)


@pytest.mark.parametrize("process", ACTIVE)
def test_fp32_parity(process):
    mom, a, rh, rc, ref = reference(process, NEV[process])
    m = mk(process, "fp32")
    for config in range(m.nconfig):
        m.set_config(config)
        me, sh, sc = run_gpu(m, mom, a, rh, rc)
        rel = np.abs(me / ref["me"] - 1)
        print(f"{process} fp32 config {config}: max rel {rel.max():.3e} median {np.median(rel):.3e}")
        assert rel.max() <= FP32_BOUND
        assert np.mean(sh == ref["sel_hel"]) > 0.99
        assert np.mean(sc == ref["sel_col"]) > 0.99


MIXED = [p for p in ACTIVE if p in (PROCS[3], PROCS[4])]
MIXED_BOUND = 1e-5


@pytest.mark.parametrize("process", MIXED)
def test_mixed_parity(process):
    """FP32 amplitudes + tensor-core colour sum (split BF16 operands, FP32 accumulation):
    every event within the stated 1e-5 of the FP64 oracle; max and median printed."""
    mom, a, rh, rc, ref = reference(process, NEV[process])
    m = mk(process, "mixed")
    for config in range(m.nconfig):
        m.set_config(config)
        me, sh, sc = run_gpu(m, mom, a, rh, rc)
        rel = np.abs(me / ref["me"] - 1)
        print(f"{process} mixed config {config}: max rel {rel.max():.3e} median {np.median(rel):.3e}")
        assert np.isfinite(me).all()
        assert rel.max() <= MIXED_BOUND, (config, rel.max())
        assert np.mean(sh == ref["sel_hel"]) > 0.99
        assert np.mean(sc == ref["sel_col"]) > 0.99


@pytest.mark.parametrize("process", [p for p in ACTIVE if p != PROCS[0]])
def test_rescue_pass_reproduces_fp64(process):
    """With a conditioning threshold below every event's, the FP32 call flags all events.
    Its FP64 rescue pass spreads each event's helicities over a group of threads, whose
    first lane sums them in helicity order: the matrix elements and the helicity
    selection are bit-identical to the FP64 handle's.  The colour weights are summed over
    the lanes in another order, so the colour selection may differ only where r * total
    lies at a running-sum boundary."""
    n = 600 if process != PROCS[4] else 100
    mom, a, rh, rc = ps.make_batch(process, n, seed=19, alphas="uniform")
    r64 = run_gpu(mk(process, "fp64"), mom, a, rh, rc)
    r32 = run_gpu(mk(process, "fp32", rescue_kappa=1e-300), mom, a, rh, rc)
    assert np.array_equal(r64[0], r32[0])
    assert np.array_equal(r64[1], r32[1])
    ref = oracle.me(process, mom, alphas=a, want_colw=True)
    ok, e = boundary_ok(r32[2], r64[2], ref["colw"], rc, 1e-10)
    assert ok, e


@pytest.mark.parametrize("process", [p for p in ACTIVE if p in (PROCS[2], PROCS[3])])
def test_nearly_collinear_gluons(process):
    """On events whose gluon propagator invariant cancels four to six digits, a plain FP64
    invariant is off by more than 1e-12.  The FP64 mode still stays within 1e-12 of the
    oracle, because it forms the invariants in double-double.  The FP32 (and mixed) modes
    flag every such event for their FP64 rescue pass, and so return the FP64 mode's bits."""
    from fractions import Fraction
    n = 64
    mom = collinear_events(process, n, seed=31)
    np.testing.assert_allclose(mom[:, 2:].sum(axis=1), mom[:, :2].sum(axis=1), rtol=0, atol=1e-9)
    rng = np.random.default_rng(32)
    rh, rc = rng.random(n), rng.random(n)
    # the inputs are as ill-conditioned as intended: the plain FP64 invariant against its
    # exact value (rational arithmetic on the same doubles)
    terms = COLLINEAR_TERMS[process]
    k = sum(sg * mom[:, i] for sg, i in terms)
    plain = k[:, 0] ** 2 - k[:, 1] ** 2 - k[:, 2] ** 2 - k[:, 3] ** 2
    exact = []
    for e in range(n):
        c = [sum(sg * Fraction(mom[e, i, mu]) for sg, i in terms) for mu in range(4)]
        exact.append(float(c[0] ** 2 - c[1] ** 2 - c[2] ** 2 - c[3] ** 2))
    exact = np.array(exact)
    assert np.median(np.abs(plain / exact - 1)) > 1e-12
    kappa = sum(mom[:, i, 0] for _, i in terms) ** 2 / np.abs(exact)
    assert kappa.min() > 2000.0  # above the default rescue threshold
    ref = oracle.me(process, mom, rnd_hel=rh, rnd_col=rc)
    r64 = run_gpu(mk(process, "fp64"), mom, None, rh, rc)
    rel = np.abs(r64[0] / ref["me"] - 1)
    print(f"{process} collinear: kappa {kappa.min():.2e}..{kappa.max():.2e}, FP64 max rel {rel.max():.3e}")
    assert rel.max() <= 1e-12
    for prec in ("fp32", "mixed") if process == PROCS[3] else ("fp32",):
        r = run_gpu(mk(process, prec), mom, None, rh, rc)
        assert np.array_equal(r[0], r64[0]), prec
        assert np.array_equal(r[1], r64[1]), prec


@pytest.mark.parametrize("process", [p for p in ACTIVE if p in (PROCS[2], PROCS[3])])
def test_rescue_removes_the_fp32_error_tail(process):
    """Without the rescue the FP32 error tail comes from nearly collinear gluons; with
    it (default threshold) every event stays within the FP32 bound."""
    mom, a, rh, rc = ps.make_batch(process, 3000, seed=23, alphas="uniform")
    ref = oracle.me(process, mom, alphas=a)["me"]
    plain = run_gpu(mk(process, "fp32", rescue_kappa=0.0), mom, a, rh, rc)[0]
    resc = run_gpu(mk(process, "fp32"), mom, a, rh, rc)[0]
    e_plain = np.abs(plain / ref - 1)
    e_resc = np.abs(resc / ref - 1)
    print(f"{process}: fp32 max rel without rescue {e_plain.max():.3e}, with {e_resc.max():.3e}; "
          f"events changed {np.mean(plain != resc):.4f}")
    assert e_resc.max() <= FP32_BOUND
    assert e_resc.max() <= e_plain.max()


@pytest.mark.parametrize("process", MIXED)
def test_mixed_matches_fp32_amplitudes(process):
    """The tensor-core colour sum (BF16 terms for gg -> ttbar gg, FP16 terms with a
    per-event power-of-two scale for gg -> ttbar ggg) agrees with the FP32 CUDA-core
    colour sum of the same FP32 amplitudes far below the FP32 rounding level of the
    amplitudes themselves."""
    mom, a, rh, rc = ps.make_batch(process, 1000 if process == PROCS[3] else 300, seed=17, alphas="uniform")
    m32 = mk(process, "fp32")
    m32.set_config(0)
    mx = mk(process, "mixed")
    r32 = run_gpu(m32, mom, a, rh, rc)[0]
    rmx = run_gpu(mx, mom, a, rh, rc)[0]
    assert np.max(np.abs(rmx / r32 - 1)) < 2e-6


@pytest.mark.parametrize("process", ACTIVE)
def test_helicity_filter_keeps_every_contributing_helicity(process):
    m = mk(process)
    good = set(m.good_helicities())
    mom, a, _, _ = ps.make_batch(process, 20, seed=99)
    ref = oracle.me(process, mom, want_hel=True)
    contributing = set(np.nonzero((ref["me_hel"] != 0).any(axis=0))[0].tolist())
    assert contributing <= good
    if process == PROCS[0]:
        assert m.ngood == 4
    assert m.ncomb == 2 ** m.npar


def test_info_matches_process_tables():
    expect = {PROCS[0]: (4, 16, 1, 2), PROCS[1]: (4, 16, 2, 3), PROCS[2]: (5, 32, 6, 16),
              PROCS[3]: (6, 64, 24, 123), PROCS[4]: (7, 128, 120, 1240)}
    for p, (npar, ncomb, ncol, ndiag) in expect.items():
        if p not in ACTIVE:
            continue
        m = mk(p)
        assert (m.npar, m.ncomb, m.ncol, m.ndiag) == (npar, ncomb, ncol, ndiag)


def test_edge_cases_and_errors():
    from paper_2312_02898_b300.binding import MEError
    p = PROCS[1]
    m = mk(p)
    # nevt = 0 is a no-op
    me, _, _ = m.compute(torch.empty((0, 4, 4), dtype=torch.float64, device="cuda"))
    assert me.numel() == 0
    # one event, no alphas (the default is used), no selection
    mom, a, rh, rc = ps.make_batch(p, 1, seed=3)
    me, sh, sc = m.compute(to_dev(mom)[0])
    torch.cuda.synchronize()
    ref = oracle.me(p, mom)
    assert abs(me.item() / ref["me"][0] - 1) < 1e-12 and sh is None and sc is None
    # non-finite momenta poison only their own event
    mom, a, rh, rc = ps.make_batch(p, 300, seed=4)
    mom[17, 2, 1] = np.nan
    me, sh, sc = run_gpu(m, mom, a, rh, rc)
    assert np.isnan(me[17]) and np.isfinite(np.delete(me, 17)).all()
    # host memory is rejected with a status code
    host = torch.from_numpy(mom)
    dev_me = torch.empty(300, dtype=torch.float64, device="cuda")
    rc_ = m.lib.me_compute(m.handle, 300, host.data_ptr(), None, None, None, dev_me.data_ptr(), None, None, None)
    assert rc_ == -1 and b"device memory" in m.lib.me_last_error(m.handle)
    assert m.lib.me_compute(m.handle, -1, None, None, None, None, None, None, None, None) == -1
    d = to_dev(mom)[0]
    rc_ = m.lib.me_compute(m.handle, 10, d.data_ptr() + 8, None, None, None, dev_me.data_ptr(), None, None, None)
    assert rc_ == -1 and b"aligned" in m.lib.me_last_error(m.handle)
    assert m.lib.me_set_config(m.handle, 99) == -1
    # a process without a tensor-core path reports ME_ERR_MODE for mixed precision
    with pytest.raises(MEError) as ei:
        mk(PROCS[1], "mixed")
    assert ei.value.code == -2


def test_host_entry_point_matches_device():
    p = PROCS[2]
    m = mk(p)
    mom, a, rh, rc = ps.make_batch(p, 500, seed=5, alphas="uniform")
    me_d, sh_d, sc_d = m.compute(*to_dev(mom, a, rh, rc))
    pin = [torch.from_numpy(x).pin_memory() for x in (mom, a, rh, rc)]
    me_h, sh_h, sc_h = m.compute_host(*pin)
    assert torch.equal(me_d.cpu(), me_h) and torch.equal(sh_d.cpu(), sh_h) and torch.equal(sc_d.cpu(), sc_h)


def test_concurrent_streams_match_sequential():
    p = PROCS[3]
    m = mk(p, "fp32")
    b1 = to_dev(*ps.make_batch(p, 3000, seed=6, alphas="uniform"))
    b2 = to_dev(*ps.make_batch(p, 2000, seed=7, alphas="uniform"))
    seq1 = [x.clone() for x in m.compute(*b1)]
    seq2 = [x.clone() for x in m.compute(*b2)]
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    r1 = m.compute(*b1, stream=s1)
    r2 = m.compute(*b2, stream=s2)
    torch.cuda.synchronize()
    for x, y in zip(seq1 + seq2, list(r1) + list(r2)):
        assert torch.equal(x, y)


def test_batch_split_invariance():
    # an event's result does not depend on the batch it is evaluated in
    p = PROCS[3]
    m = mk(p, "fp64")
    mom, a, rh, rc = ps.make_batch(p, 2000, seed=8, alphas="uniform")
    whole = run_gpu(m, mom, a, rh, rc)
    part = run_gpu(m, mom[700:1300], a[700:1300], rh[700:1300], rc[700:1300])
    for x, y in zip(whole, part):
        assert np.array_equal(x[700:1300], y)


@pytest.mark.skipif(PROCS[0] not in ACTIVE, reason="process not selected")
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_split_helicities_give_the_same_bits(precision):
    """e+ e- > mu+ mu- has one colour flow, so a small batch spreads each event's
    helicities over a group of threads while a large batch keeps one thread per event.
    Either way an event's matrix element and helicity selection have the same bits."""
    p = PROCS[0]
    m = mk(p, precision)
    _, block, bps, nsm = m.launch_shape(1)
    big = 2 * block * bps * nsm  # beyond the resident threads: one thread per event
    mom, _, rh, rc = ps.make_batch(p, big, seed=12)
    whole = run_gpu(m, mom, None, rh, rc)
    for lo, hi in ((0, 1), (100, 131), (5000, 5777), (big - 1000, big)):
        part = run_gpu(m, mom[lo:hi], None, rh[lo:hi], rc[lo:hi])
        for x, y in zip(whole, part):
            assert np.array_equal(x[lo:hi], y), (lo, hi)


FULL = [(PROCS[0], 16384, "fp64", None), (PROCS[1], 524288, "fp64", 0.118), (PROCS[2], 524288, "fp32", 0.118),
        (PROCS[3], 1048576, "fp64", "uniform"), (PROCS[3], 1048576, "fp32", "uniform"),
        (PROCS[3], 1048576, "mixed", "uniform"),
        (PROCS[4], 262144, "fp32", 0.118), (PROCS[4], 262144, "mixed", 0.118)]


@pytest.mark.parametrize("process,nevt,precision,alphas", [f for f in FULL if f[0] in ACTIVE])
def test_full_size_sampled(process, nevt, precision, alphas):
    """Workload-size batches in the benchmark's launch configuration: properties on every
    event and the oracle on a random sample of events."""
    mom, a, rh, rc = ps.make_batch(process, nevt, seed=0, alphas=alphas)
    m = mk(process, precision)
    me, sh, sc = run_gpu(m, mom, a, rh, rc)
    assert np.isfinite(me).all() and (me > 0).all()
    assert set(np.unique(sh).tolist()) <= set(m.good_helicities())
    assert sc.min() >= 0 and sc.max() < m.ncol
    rng = np.random.default_rng(1)
    idx = np.sort(rng.choice(nevt, size=24 if process == PROCS[4] else 64, replace=False))
    idx = np.unique(np.concatenate([idx, [0, nevt - 1]]))
    ref = oracle.me(process, mom[idx], alphas=None if a is None else a[idx], rnd_hel=rh[idx], rnd_col=rc[idx])
    rel = np.abs(me[idx] / ref["me"] - 1)
    assert rel.max() <= {"fp64": 1e-12, "fp32": FP32_BOUND, "mixed": MIXED_BOUND}[precision]
    assert np.mean(sh[idx] == ref["sel_hel"]) >= 0.95


@pytest.mark.parametrize("process", ACTIVE)
def test_persistent_grid_walks_many_tiles_per_block(process, monkeypatch):
    """A grid of 3 blocks walks the whole batch tile by tile, with a ragged last tile
    whose idle threads still take part in every block barrier: every configuration of
    every precision gives the oracle's results."""
    monkeypatch.setenv("ME_B300_MAX_BLOCKS", "3")
    mom, a, rh, rc, ref = reference(process, NEV[process])
    for prec in ("fp64", "fp32", "mixed"):
        if prec == "mixed" and process not in MIXED:
            continue
        m = mk(process, prec)
        bound = 1e-12 if prec == "fp64" else FP32_BOUND
        for config in range(m.nconfig):
            m.set_config(config)
            me, sh, sc = run_gpu(m, mom, a, rh, rc)
            rel = np.abs(me / ref["me"] - 1)
            assert rel.max() <= bound, (prec, config, rel.max())
            if prec == "fp64":
                assert boundary_ok(sh, ref["sel_hel"], ref["me_hel"], rh, 1e-10)[0]
                assert boundary_ok(sc, ref["sel_col"], ref["colw"], rc, 1e-10)[0]
        m.close()


@pytest.mark.skipif(PROCS[2] not in ACTIVE, reason="process not selected")
def test_rescue_is_lossless_when_every_event_is_flagged():
    """With a threshold below every event's conditioning, every one of 40000 events is
    flagged (far more than the max(1024, nevt/16) = 2500 entries the list once held):
    each is re-evaluated in FP64, so the FP32 handle returns the FP64 handle's matrix
    elements and helicity selections bit for bit, and colour selections equal up to
    running-sum boundaries (the rescue pass sums colour weights over helicity lanes)."""
    p = PROCS[2]
    n = 40000
    mom, a, rh, rc = ps.make_batch(p, n, seed=41, alphas="uniform")
    r64 = run_gpu(mk(p, "fp64"), mom, a, rh, rc)
    r32 = run_gpu(mk(p, "fp32", rescue_kappa=1e-300), mom, a, rh, rc)
    assert np.array_equal(r64[0], r32[0])
    assert np.array_equal(r64[1], r32[1])
    diff = np.nonzero(r64[2] != r32[2])[0]
    if diff.size:
        ref = oracle.me(p, mom[diff], alphas=a[diff], want_colw=True)
        ok, e = boundary_ok(r32[2][diff], r64[2][diff], ref["colw"], rc[diff], 1e-10)
        assert ok, e


@pytest.mark.skipif(PROCS[3] not in ACTIVE, reason="process not selected")
def test_rescue_is_lossless_in_the_mixed_mode():
    p = PROCS[3]
    n = 3000
    mom, a, rh, rc = ps.make_batch(p, n, seed=42, alphas="uniform")
    r64 = run_gpu(mk(p, "fp64"), mom, a, rh, rc)
    rmx = run_gpu(mk(p, "mixed", rescue_kappa=1e-300), mom, a, rh, rc)
    assert np.array_equal(r64[0], rmx[0])
    assert np.array_equal(r64[1], rmx[1])


@pytest.mark.skipif(PROCS[3] not in ACTIVE, reason="process not selected")
def test_mixed_wait_timeout_is_reported_and_the_handle_recovers():
    """The mixed kernel's bounded wait for its MMAs, driven to give up at once through
    the testing hook (no fault is involved: the wait simply makes zero polls): every event
    of the call becomes NaN with selections 0, the kernel keeps its tensor memory until
    the issued MMAs complete, the host sees ME_ERR_TIMEOUT (from me_sync_status, or from
    the next me_compute, which then does not compute), and a later call with the default
    limit returns the oracle's values on the same handle."""
    from paper_2312_02898_b300.binding import ME_ERR_TIMEOUT, MEError
    p = PROCS[3]
    m = mk(p, "mixed", rescue_kappa=0.0)
    mom, a, rh, rc = ps.make_batch(p, 1000, seed=43, alphas="uniform")
    dev = to_dev(mom, a, rh, rc)
    m.set_wait_limit(0)
    me, sh, sc = m.compute(*dev)
    with pytest.raises(MEError) as ei:
        m.sync_status()
    assert ei.value.code == ME_ERR_TIMEOUT
    assert torch.isnan(me).all() and (sh == 0).all() and (sc == 0).all()
    m.sync_status()  # reporting cleared the flag
    # the same failure reported by the next compute call, which does not run
    m.compute(*dev)
    torch.cuda.synchronize()
    with pytest.raises(MEError) as ei:
        m.compute(*dev)
    assert ei.value.code == ME_ERR_TIMEOUT
    m.set_wait_limit(-1)
    me, sh, sc = run_gpu(m, mom, a, rh, rc)
    m.sync_status()
    ref = oracle.me(p, mom, alphas=a)["me"]
    assert np.abs(me / ref - 1).max() <= MIXED_BOUND


@pytest.mark.skipif(PROCS[1] not in ACTIVE, reason="process not selected")
def test_binding_rejects_tensors_the_abi_would_misread():
    m = mk(PROCS[1])
    mom, a, rh, rc = to_dev(*ps.make_batch(PROCS[1], 64, seed=9, alphas="uniform"))
    strided = torch.empty((64, 4, 8), dtype=torch.float64, device="cuda")[:, :, :4]
    strided.copy_(mom)
    cases = [dict(momenta=mom.float()), dict(momenta=strided), dict(momenta=mom[:, :3]),
             dict(alphas=a[:63]), dict(alphas=a.float()), dict(rnd_hel=rh.cpu()), dict(rnd_col=rc[::2])]
    for bad in cases:
        args = dict(momenta=mom, alphas=a, rnd_hel=rh, rnd_col=rc)
        args.update(bad)
        with pytest.raises(ValueError):
            m.compute(**args)
    out = (torch.empty(64, dtype=torch.float64, device="cuda"), torch.empty(64, dtype=torch.int64, device="cuda"),
           torch.empty(64, dtype=torch.int32, device="cuda"))
    with pytest.raises(ValueError):
        m.compute(mom, a, rh, rc, out=out)


DFLOAT = [p for p in ACTIVE if p in (PROCS[1], PROCS[2])]
DFLOAT_BOUND = 1e-10


@pytest.mark.parametrize("process", DFLOAT)
def test_dfloat_parity(process):
    """FP64-emulating double-float amplitudes (about 48 significant bits on the FP32
    pipe), with FP64 inputs, error-free invariants and FP64 helicity sum: every event
    within the stated bound of the FP64 oracle (max and median printed), and the
    selections equal except at running-sum boundaries."""
    mom, a, rh, rc, ref = reference(process, NEV[process])
    m = mk(process, "dfloat")
    me, sh, sc = run_gpu(m, mom, a, rh, rc)
    rel = np.abs(me / ref["me"] - 1)
    print(f"{process} dfloat: max rel {rel.max():.3e} median {np.median(rel):.3e}")
    assert rel.max() <= DFLOAT_BOUND
    ok, e = boundary_ok(sh, ref["sel_hel"], ref["me_hel"], rh, 1e-8)
    assert ok, ("sel_hel", e)
    ok, e = boundary_ok(sc, ref["sel_col"], ref["colw"], rc, 1e-8)
    assert ok, ("sel_col", e)


@pytest.mark.skipif(PROCS[2] not in ACTIVE, reason="process not selected")
def test_dfloat_on_nearly_collinear_gluons():
    """The double-float mode forms its invariants error-free like the FP64 mode, so
    nearly collinear gluons stay within its bound without any rescue pass."""
    mom = collinear_events(PROCS[2], 64, seed=31)
    ref = oracle.me(PROCS[2], mom)["me"]
    me = mk(PROCS[2], "dfloat").compute(to_dev(mom)[0])[0].cpu().numpy()
    rel = np.abs(me / ref - 1)
    print(f"collinear dfloat: max rel {rel.max():.3e}")
    assert rel.max() <= DFLOAT_BOUND


def test_dfloat_is_not_built_for_the_large_processes():
    from paper_2312_02898_b300.binding import MEError
    with pytest.raises(MEError) as ei:
        mk(PROCS[3], "dfloat")
    assert ei.value.code == -2
