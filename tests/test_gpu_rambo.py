"""Device-side input generation against the host generator: the counter-based uniforms
are the same numbers bit for bit (integer arithmetic and one exact conversion); the
RAMBO momenta agree to rounding (the device and host transcendental functions may
differ in the last bit), and so do the matrix elements computed from them."""
import numpy as np
import pytest

from paper_2312_02898_b300 import phasespace as ps

pytestmark = pytest.mark.gpu

PROCS = ["e+ e- > mu+ mu-", "g g > t t~", "g g > t t~ g", "g g > t t~ g g", "g g > t t~ g g g"]


@pytest.mark.parametrize("seed,first,stream", [(0, 0, 1), (7, 12345, 2), (2 ** 40 + 3, 2 ** 33 + 5, 3),
                                                (123456789, 0, 0)])
def test_uniforms_are_bit_identical(seed, first, stream):
    from paper_2312_02898_b300.binding import device_uniforms
    n = 10007
    ev = np.arange(first, first + n, dtype=np.uint64)
    host = ps.uniforms(seed, ev, stream, 1)[:, 0]
    dev = device_uniforms(n, seed, first, stream).cpu().numpy()
    assert np.array_equal(host, dev)
    a_host = 0.10 + 0.03 * host
    a_dev = device_uniforms(n, seed, first, stream, 0.10, 0.03).cpu().numpy()
    assert np.array_equal(a_host, a_dev)


@pytest.mark.parametrize("process", PROCS)
def test_rambo_momenta_match_the_host_generator(process):
    import torch
    from paper_2312_02898_b300.binding import MatrixElement
    m = MatrixElement(process, precision="fp64")
    n, seed, first = 4099, 31, 1000
    dev = m.rambo(n, seed=seed, first_event=first).cpu().numpy()
    host = ps.rambo(1500.0, ps.PROCESS_FINAL_MASSES[process](m.params.mt), seed, n, first)
    assert np.all(np.isfinite(dev))
    assert np.max(np.abs(dev - host)) <= 1e-12 * 1500.0
    # exact kinematics on the device output: momentum conservation and on-shell masses
    tot_in = dev[:, 0] + dev[:, 1]
    tot_out = dev[:, 2:].sum(axis=1)
    assert np.max(np.abs(tot_in - tot_out)) <= 1e-12 * 1500.0
    # E^2 - p^2 cancels for light particles, and the conformal boost amplifies rounding
    # by its gamma factor, so the mass shell holds to ~1e-12 of E^2 (the host generator's
    # own output is no closer)
    masses = np.array([0.0, 0.0] + list(ps.PROCESS_FINAL_MASSES[process](m.params.mt)))
    m2 = dev[..., 0] ** 2 - (dev[..., 1:] ** 2).sum(axis=-1)
    assert np.max(np.abs(m2 - masses ** 2) / (dev[..., 0] ** 2)) <= 1e-10
    # the two batches differ in the last bits of the momenta, which a matrix element
    # amplifies by its conditioning (nearly collinear gluons): equal to ~1e-15 typically
    me_dev = m.compute(torch.from_numpy(dev).cuda())[0].cpu().numpy()
    me_host = m.compute(torch.from_numpy(host).cuda())[0].cpu().numpy()
    rel = np.abs(me_dev / me_host - 1)
    assert np.median(rel) <= 1e-14 and rel.max() <= 1e-10


def test_rambo_edge_cases():
    import ctypes
    import torch
    from paper_2312_02898_b300.binding import MatrixElement
    m = MatrixElement("g g > t t~", precision="fp64")
    out = torch.full((1, 4, 4), -1.0, dtype=torch.float64, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert m.lib.me_rambo(m.handle, 0, 0, 0, 1500.0, ctypes.c_void_p(out.data_ptr()), s) == 0
    torch.cuda.synchronize()
    assert out.eq(-1.0).all()                                 # nevt == 0 writes nothing
    assert m.lib.me_rambo(m.handle, 1, 0, 0, 300.0, ctypes.c_void_p(out.data_ptr()), s) == -1  # below 2 mt
    host = np.zeros((1, 4, 4))
    assert m.lib.me_rambo(m.handle, 1, 0, 0, 1500.0, ctypes.c_void_p(host.ctypes.data), s) == -1
    assert m.lib.me_uniforms(-1, 0, 0, 1, 0.0, 1.0, None, s) == -1
    assert m.lib.me_uniforms(1, 0, 0, 1, 0.0, 1.0, ctypes.c_void_p(host.ctypes.data), s) == -1
