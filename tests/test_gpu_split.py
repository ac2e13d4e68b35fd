"""Lattices divided along t between device memory and host memory
(qcd_lattice_create_split).  The kernels are the ones of a device-resident
lattice, so the bar is equality: every link bit-identical to the same chain on
a device-resident lattice after sweeps, phases, reunitarizations and
measurements, and the measurements equal.  One all-host FP64 case is also held
to the oracle (every link within 1e-9 after one sweep, the bar of the
device-resident FP64 parity tests)."""
import numpy as np
import pytest

import oracle
from workloads import COLD, FP32_COMPRESSED, FP64_PLAIN, HOT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1310_7087_gb300 import build
    build.build()
    import paper_1310_7087_gb300 as q
    return q


def make_split(q, *args, **kw):
    try:
        return q.Lattice(*args, **kw)
    except q.QcdError as e:
        if e.code == q.QCD_ERR_NOT_SUPPORTED:
            pytest.skip("device cannot map host-NUMA memory: " + str(e))
        raise


# (group, precision, Ns, Nt, beta, flux, flux8, field mode, nt_device)
# 32^3 x 16 FP32 SU(3): one t-slice of a link array is 256 KB, so 8 t-slices
# are one 2 MB granule and the lattice splits at t = 8.  The small lattices
# have arrays of one granule: nt_device = 0 puts every link in host memory.
CASES = [
    (3, FP32_COMPRESSED, 32, 16, 6.0, 1, 0, 0, 8),
    (3, FP32_COMPRESSED, 8, 4, 5.7, 1, 1, 0, 0),
    (3, FP64_PLAIN, 8, 4, 5.7, 2, 0, 1, 0),
    (2, FP32_COMPRESSED, 16, 8, 2.3, 1, 0, 0, 0),
    (2, FP64_PLAIN, 8, 4, 2.3, 0, 0, 0, 0),
]
IDS = ["su%d_%s_%dx%d_n%d_n8%d_%s_ntdev%d" % (c[0], "f64" if c[1] == FP64_PLAIN else "f32", c[2], c[3], c[5],
                                               c[6], "links" if c[7] == 0 else "frozen", c[8]) for c in CASES]


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_split_equals_device_resident(q, case):
    group, prec, ns, nt, beta, flux, flux8, mode, ntd = case
    kw = dict(precision=prec, start=HOT, seed=11, field_mode=mode, flux8=flux8)
    a = q.Lattice(group, ns, nt, beta, flux, **kw)
    b = make_split(q, group, ns, nt, beta, flux, nt_device=ntd, **kw)
    dev_b, host_b, nt_dev = q.qcd_get_residency(b.h)
    assert host_b > 0
    assert nt_dev == ntd
    assert q.qcd_get_residency(a.h)[1:] == (0, nt)
    for lat in (a, b):
        q.qcd_set_block(lat.h, 128)  # same launch shape: the block-wise sums match too
    assert np.array_equal(a.get_links(), b.get_links())
    for lat in (a, b):
        lat.sweep(1, 2, 11)
        lat.phase(0, 1, 3, 11)
        lat.reunitarize()
    m = [q.qcd_working_sweep(lat.h, 1, 4, 11) for lat in (a, b)]
    assert np.array_equal(a.get_links(), b.get_links())
    assert m[0] == m[1]
    assert a.measure() == b.measure()
    assert a.sweep_counter == b.sweep_counter == 2
    a.close()
    b.close()


def test_split_links_round_trip_and_copy(q):
    """set_links / get_links and the raw copies reach both parts."""
    ns, nt = 32, 16
    a = q.Lattice(3, ns, nt, 6.0, 1, FP32_COMPRESSED, HOT, 5)
    b = make_split(q, 3, ns, nt, 6.0, 1, FP32_COMPRESSED, COLD, 5, nt_device=4)
    assert q.qcd_get_residency(b.h)[2] == 8  # 4 t-slices rounded up to one granule
    b.set_links(a.get_links())
    assert np.array_equal(a.get_links(), b.get_links())
    for lat in (a, b):
        q.qcd_working_sweep(lat.h, 1, 1, 5)
    ref = a.get_links()
    assert np.array_equal(ref, b.get_links())
    raw = np.empty(q.qcd_link_bytes(b.h), np.uint8)
    q.qcd_copy_links_out(b.h, raw.ctypes.data, raw.size)
    c = make_split(q, 3, ns, nt, 6.0, 1, FP32_COMPRESSED, COLD, 5, nt_device=4)
    q.qcd_copy_links_in(c.h, raw.ctypes.data, raw.size)
    assert np.array_equal(ref, c.get_links())
    for lat in (a, b, c):
        lat.close()


def test_split_fp64_all_host_matches_oracle(q):
    oracle.build()
    ns, nt, beta = 4, 4, 5.7
    b = make_split(q, 3, ns, nt, beta, 1, FP64_PLAIN, HOT, 7, nt_device=0)
    o = oracle.OracleLattice(3, ns, nt, beta, 1, 10, 0)
    o.set_links(b.get_links())
    b.sweep(1, 1, 7)
    o.sweep(1, 1, 7)
    assert np.abs(b.get_links() - o.get_links()).max() < 1e-9
    g, r = np.concatenate(b.measure()), np.concatenate(o.measure())
    assert np.abs(g - r).max() < 1e-12
    b.close()
    o.close()


def test_split_bad_arguments(q):
    for ntd in (-1, 5):
        with pytest.raises(q.QcdError) as e:
            q.Lattice(3, 4, 4, 5.7, 0, FP32_COMPRESSED, HOT, 1, nt_device=ntd)
        assert e.value.code == q.QCD_ERR_INVALID_ARG
