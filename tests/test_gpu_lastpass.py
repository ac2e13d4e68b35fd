"""Link-by-link parity of the kernels of a sweep's last overrelaxation pass.

In a sweep the reunitarization (sec. 5) is carried by the last
overrelaxation pass: its kernels reunitarize each link right after updating
it, and in a working sweep the plane-summing phases of that pass (odd parity,
mu = 1, 2, 3) also sum the plaquettes of the planes (mu, nu < mu).  Each of
the eight phases runs here on its own through qcd_phase, from the state the
GPU left, against the oracle's overrelaxation of the same phase followed by
the reunitarization of that phase's links:
  FP64 storage  every link within 1e-9;
  FP32 storage  the FP32Tally bar of the other kernel-by-kernel tests (links
                outside the phase bit-identical, >= 99.99 % of the updated
                links within 1e-5, none beyond 1e-4).
After the pass, qcd_measure_fused_finish gives the working sweep's
measurement and the mean plaquette of the planes each plane-summing phase
summed; both are held to the oracle's measurement of the final configuration
(1e-6 FP32, 1e-12 FP64).
"""
import numpy as np
import pytest

import oracle
from test_gpu_parity import FP32Tally, check_links, phase_mask
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
    oracle.build()
    return q


# (group, precision, Ns, Nt, beta, flux, flux8, field_mode)
CASES = [
    (3, FP32_COMPRESSED, 6, 4, 5.7, 0, 0, 0),   # field level 0, ragged Vh = 432
    (3, FP32_COMPRESSED, 8, 4, 6.0, 1, 0, 0),   # lambda3 field (the benchmark's level)
    (3, FP32_COMPRESSED, 6, 6, 5.9, 1, 1, 0),   # lambda3 + lambda8: general diagonal
    (3, FP32_COMPRESSED, 6, 4, 5.9, 2, 0, 1),   # frozen-boundary mode (reunitarize only)
    (3, FP32_COMPRESSED, 16, 4, 5.7, 0, 0, 0),  # C2-sized: 65536 links per pass
    (2, FP32_COMPRESSED, 6, 4, 2.3, 0, 0, 0),
    (2, FP32_COMPRESSED, 8, 4, 2.4, 2, 0, 0),
    (2, FP32_COMPRESSED, 6, 4, 2.3, 1, 0, 1),
    (2, FP64_PLAIN, 6, 4, 2.3, 3, 0, 0),
    (3, FP64_PLAIN, 6, 2, 6.0, 1, 0, 0),        # FP64 SU(3): no fused measurement
    (3, FP64_PLAIN, 4, 4, 5.7, 1, 1, 0),
]
IDS = ["su%d_%s_%dx%d_n%d_n8_%d_%s" % (g, "f64" if p == FP64_PLAIN else "f32", ns, nt, n, n8,
                                        "frozen" if m else "links")
       for g, p, ns, nt, b, n, n8, m in CASES]


def fused(q, group, precision, mode):
    return mode == q.QCD_FIELD_LINKS and not (group == 3 and precision == FP64_PLAIN)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_last_pass_link_by_link(q, case):
    group, precision, Ns, Nt, beta, flux, flux8, mode = case
    seed = 7
    lat = q.Lattice(group, Ns, Nt, beta, flux, precision, HOT, seed, field_mode=mode, flux8=flux8)
    orc = oracle.OracleLattice(group, Ns, Nt, beta, flux, 10, 0, mode, flux8)
    n_or = 4 if group == 3 else 1
    lat.sweep(1, n_or, seed)  # a state inside the chain; launch shape chosen as in a normal run
    with_meas = fused(q, group, precision, mode)
    tally = FP32Tally()
    for parity in (0, 1):
        for mu in range(4):
            kind = (q.QCD_OVERRELAX_MEASURE if with_meas and parity == 1 and mu >= 1
                    else q.QCD_OVERRELAX_REUNIT)
            orc.set_links(lat.get_links())
            orc.sweep_counter = lat.sweep_counter
            lat.phase(kind, parity, mu, seed)
            orc.phase(oracle.OVERRELAX, parity, mu, seed)
            orc.reunitarize_phase(parity, mu)
            got, ref = lat.get_links(), orc.get_links()
            if precision == FP64_PLAIN:
                check_links(got, ref, precision, (kind, parity, mu))
            else:
                tally.add(got, ref, phase_mask(Ns, Nt, parity, mu), (kind, parity, mu))
    tally.check()
    # every link was reunitarized by the pass
    U = lat.get_links().reshape(-1, group, group)
    unit = np.abs(np.einsum("nki,nkj->nij", U.conj(), U) - np.eye(group)).max()
    assert unit < (1e-14 if precision == FP64_PLAIN else 5e-7), unit
    if with_meas:
        got = q.qcd_measure_fused_finish(lat.h)
        orc.set_links(lat.get_links())
        (op, ol), pl = orc.measure(), orc.measure_planes()
        ref = list(op) + list(ol) + [pl[0], (pl[1] + pl[2]) / 2, (pl[3] + pl[4] + pl[5]) / 3]
        tol = 1e-12 if precision == FP64_PLAIN else 1e-6
        assert np.abs(np.array(got) - np.array(ref)).max() <= tol, (got, ref)
    else:
        with pytest.raises(q.QcdError) as e:
            q.qcd_measure_fused_finish(lat.h)
        assert e.value.code == q.QCD_ERR_NOT_SUPPORTED
    lat.close()


def test_last_pass_by_phases_equals_working_sweep(q):
    """The eight last-pass phases launched one by one after an HB + 3 OR sweep
    part give the links and the measurement of qcd_working_sweep (HB + 4 OR)
    bit for bit: the kernels tested above are the ones the sweep runs."""
    Ns, Nt, beta, flux, seed = 8, 4, 6.0, 1, 5
    a = q.Lattice(3, Ns, Nt, beta, flux, FP32_COMPRESSED, HOT, seed)
    b = q.Lattice(3, Ns, Nt, beta, flux, FP32_COMPRESSED, HOT, seed)
    for lat in (a, b):  # one launch shape, so the block partials are summed alike
        q.qcd_set_block(lat.h, 128)
    want = q.qcd_working_sweep(a.h, 1, 4, seed)
    for kind, passes in ((q.QCD_HEATBATH, 1), (q.QCD_OVERRELAX, 3)):
        for _ in range(passes):
            for parity in (0, 1):
                for mu in range(4):
                    b.phase(kind, parity, mu, seed)
    for parity in (0, 1):
        for mu in range(4):
            kind = q.QCD_OVERRELAX_MEASURE if parity == 1 and mu >= 1 else q.QCD_OVERRELAX_REUNIT
            b.phase(kind, parity, mu, seed)
    got = q.qcd_measure_fused_finish(b.h)
    assert np.array_equal(a.get_links(), b.get_links())
    assert got[:5] == want
    a.close()
    b.close()


def test_measure_phase_argument_checks(q):
    lat = q.Lattice(3, 4, 4, 6.0, 0, FP64_PLAIN, HOT, 1)
    with pytest.raises(q.QcdError) as e:
        lat.phase(q.QCD_OVERRELAX_MEASURE, 1, 2, 1)
    assert e.value.code == q.QCD_ERR_NOT_SUPPORTED
    lat.close()
    lat = q.Lattice(3, 4, 4, 6.0, 0, FP32_COMPRESSED, HOT, 1)
    for parity, mu in ((0, 1), (1, 0)):
        with pytest.raises(q.QcdError) as e:
            lat.phase(q.QCD_OVERRELAX_MEASURE, parity, mu, 1)
        assert e.value.code == q.QCD_ERR_INVALID_ARG
    with pytest.raises(q.QcdError) as e:
        lat.phase(4, 0, 0, 1)
    assert e.value.code == q.QCD_ERR_INVALID_ARG
    lat.close()
