"""Per-event subprocess dispatch (me_compute_channels) for p p -> t t~: one batch whose
events belong to g g -> t t~, u u~ -> t t~ or u~ u -> t t~ (the 2 -> 2 momenta of RAMBO
serve all three channels: massless beams, massive tops).  Every event's results must be
those of me_compute with its channel's handle, bit for bit, and within the mode's bound
of the FP64 oracle of its channel."""
import numpy as np
import pytest

import oracle
from paper_2312_02898_b300 import phasespace as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CHANNELS = ("g g > t t~", "u u~ > t t~", "u~ u > t t~")


def dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in arrs]


@pytest.mark.parametrize("precision,bound", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_channels_match_single_channel_calls_and_the_oracle(precision, bound):
    from paper_2312_02898_b300.binding import MatrixElement, compute_channels
    n = 5003
    mom, a, rh, rc = ps.make_batch(CHANNELS[0], n, seed=51, alphas="uniform")
    ch = np.random.default_rng(52).choice(3, size=n, p=[0.8, 0.1, 0.1]).astype(np.int32)
    hs = [MatrixElement(p, precision=precision) for p in CHANNELS]
    d = dev(mom, a, rh, rc)
    me, sh, sc = compute_channels(hs, dev(ch)[0], *d)
    torch.cuda.synchronize()
    me, sh, sc = me.cpu().numpy(), sh.cpu().numpy(), sc.cpu().numpy()
    for c, p in enumerate(CHANNELS):
        sel = ch == c
        r = [x.cpu().numpy() for x in hs[c].compute(*d)]
        assert np.array_equal(me[sel], r[0][sel]) and np.array_equal(sh[sel], r[1][sel])
        assert np.array_equal(sc[sel], r[2][sel])
        ref = oracle.me(p, mom[sel], alphas=a[sel])["me"]
        rel = np.abs(me[sel] / ref - 1)
        print(f"{p} {precision}: {sel.sum()} events, max rel {rel.max():.3e}")
        assert rel.max() <= bound


def test_invalid_channel_and_mismatched_handles():
    from paper_2312_02898_b300.binding import MatrixElement, MEError, compute_channels
    n = 300
    mom, a, rh, rc = ps.make_batch(CHANNELS[0], n, seed=53, alphas="uniform")
    ch = np.zeros(n, dtype=np.int32)
    ch[7] = 5
    ch[9] = -1
    hs = [MatrixElement(p) for p in CHANNELS[:2]]
    me, sh, sc = compute_channels(hs, dev(ch)[0], *dev(mom, a, rh, rc))
    torch.cuda.synchronize()
    me = me.cpu().numpy()
    assert np.isnan(me[7]) and np.isnan(me[9]) and np.isfinite(np.delete(me, [7, 9])).all()
    with pytest.raises(MEError) as ei:
        compute_channels([hs[0], MatrixElement("g g > t t~ g")], dev(ch)[0], *dev(mom, a, rh, rc))
    assert ei.value.code == -1
    with pytest.raises(MEError) as ei:
        compute_channels([hs[0], MatrixElement("g g > t t~", precision="dfloat")], dev(ch)[0], *dev(mom, a, rh, rc))
    assert ei.value.code == -2
