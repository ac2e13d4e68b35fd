"""The allocation-free measurement entry point (qcd_measure_noalloc).

It exists for callers that cannot let the library allocate device memory,
for instance code inside a host framework that owns all device memory through
its own pool.  It must give what qcd_measure gives on the same links, call
after call, although every call reuses one shared scratch array.  This file is
named so that pytest collects it last.
"""
import numpy as np
import pytest

from workloads import FP32_COMPRESSED, FP64_PLAIN, HOT

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


def device_links(q, lat):
    """A device copy of the lattice's link storage, in memory the caller
    (here: PyTorch) allocated."""
    import torch
    n = lat.link_bytes
    host = torch.empty(n, dtype=torch.uint8)
    q.qcd_copy_links_out(lat.h, host.data_ptr(), n)
    return host.cuda()


# measurement tolerances of the other GPU tests: FP64 storage 1e-12, FP32 1e-6
CASES = [(3, FP32_COMPRESSED, 8, 4, 6.0, 1), (3, FP64_PLAIN, 6, 4, 5.7, 0),
         (2, FP32_COMPRESSED, 6, 2, 2.3, 2), (2, FP64_PLAIN, 4, 4, 2.3, 3)]


@pytest.mark.parametrize("case", CASES, ids=["su%d_p%d_%dx%d_n%d" % (c[0], c[1], c[2], c[3], c[5]) for c in CASES])
def test_noalloc_matches_measure_on_two_calls(q, case):
    group, precision, Ns, Nt, beta, flux = case
    lat = q.Lattice(group, Ns, Nt, beta, flux, precision, HOT, 5)
    lat.sweep(1, 1, 5)
    ref_p, ref_l = lat.measure()
    dev = device_links(q, lat)
    tol = 1e-12 if precision == FP64_PLAIN else 1e-6
    for _ in range(2):
        p, l = q.qcd_measure_noalloc(dev.data_ptr(), lat.link_bytes, group, precision, Ns, Nt, flux)
        np.testing.assert_allclose(p, ref_p, rtol=0, atol=tol)
        np.testing.assert_allclose(l, ref_l, rtol=0, atol=tol)
    lat.close()


def test_noalloc_back_to_back_lattices(q):
    """A large lattice, then a small one, then the large one again: what the
    shared array kept from the previous call must not leak into the next."""
    big = q.Lattice(3, 16, 8, 6.0, 2, FP32_COMPRESSED, HOT, 9)
    small = q.Lattice(2, 4, 2, 2.3, 1, FP64_PLAIN, HOT, 9)
    big.sweep(1, 1, 9)
    small.sweep(1, 1, 9)
    refs = [big.measure(), small.measure()]
    devs = [device_links(q, big), device_links(q, small)]
    args = [(3, FP32_COMPRESSED, 16, 8, 2), (2, FP64_PLAIN, 4, 2, 1)]
    for k in (0, 1, 0, 1):
        p, l = q.qcd_measure_noalloc(devs[k].data_ptr(), devs[k].numel(), *args[k])
        tol = 1e-6 if args[k][1] == FP32_COMPRESSED else 1e-12
        np.testing.assert_allclose(p, refs[k][0], rtol=0, atol=tol)
        np.testing.assert_allclose(l, refs[k][1], rtol=0, atol=tol)
    big.close()
    small.close()


def test_noalloc_split_and_lambda8_storage(q):
    """Storage of a lattice divided between device and host memory (link
    arrays padded to the mapping granule, not to 64 vectors), and of a lattice
    with a lambda8 background: the call reads the padding off the size it is
    given and builds the full diagonal background."""
    import torch
    lats = []
    try:
        lats.append((q.Lattice(3, 8, 4, 6.0, 1, FP32_COMPRESSED, HOT, 4, nt_device=2), 1, 0))
    except q.QcdError as e:  # a device that cannot map host memory
        assert e.code == q.QCD_ERR_NOT_SUPPORTED
    lats.append((q.Lattice(3, 6, 4, 5.8, 1, FP32_COMPRESSED, HOT, 4, flux8=2), 1, 2))
    lats.append((q.Lattice(3, 6, 4, 5.8, 2, FP64_PLAIN, HOT, 4, flux8=1), 2, 1))
    for lat, n, n8 in lats:
        lat.sweep(1, 1, 4)
        ref_p, ref_l = lat.measure()
        dev = device_links(q, lat)
        tol = 1e-12 if lat.precision == FP64_PLAIN else 1e-6
        for _ in range(2):
            p, l = q.qcd_measure_noalloc(dev.data_ptr(), lat.link_bytes, 3, lat.precision, lat.Ns, lat.Nt, n, n8)
            np.testing.assert_allclose(p, ref_p, rtol=0, atol=tol)
            np.testing.assert_allclose(l, ref_l, rtol=0, atol=tol)
        lat.close()


def test_noalloc_rejects_lattices_beyond_its_scratch(q):
    import torch
    buf = torch.zeros(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(q.QcdError) as e:
        q.qcd_measure_noalloc(buf.data_ptr(), 24 * 16 * 96 ** 3 * 8, 3, FP32_COMPRESSED, 96, 16, 0)
    assert e.value.code == q.QCD_ERR_INVALID_ARG
    assert "bytes of measurement scratch" in str(e.value)


def test_noalloc_rejects_a_size_that_is_not_link_storage(q):
    import torch
    lat = q.Lattice(3, 4, 4, 6.0, 0, FP32_COMPRESSED, HOT, 1)
    dev = device_links(q, lat)
    for nbytes in (lat.link_bytes - 16, lat.link_bytes // 2, 0):
        with pytest.raises(q.QcdError) as e:
            q.qcd_measure_noalloc(dev.data_ptr(), nbytes, 3, FP32_COMPRESSED, 4, 4, 0)
        assert e.value.code == q.QCD_ERR_INVALID_ARG
    lat.close()
