"""Parity of the lambda8 background component (SU(3)) with the FP64 oracle:
B_y(x) = diag(e^{i(p3 + p8)}, e^{i(-p3 + p8)}, e^{-2 i p8}) on effective links
and on the frozen boundary.  Same bars as the lambda3-only field: FP64 every
link within 1e-9 after a sweep, FP32 kernel by kernel (pooled), measurements
within 1e-12 (FP64) / 1e-6 (FP32)."""
import numpy as np
import pytest

import oracle
from test_gpu_parity import FP32Tally, check_links, link_err, phase_mask
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
    oracle.build()
    return q


# (precision, Ns, Nt, beta, flux, flux8, field mode)
CASES = [
    (FP64_PLAIN, 4, 4, 5.7, 1, 1, 0),
    (FP32_COMPRESSED, 4, 4, 5.7, 1, 2, 0),
    (FP32_COMPRESSED, 6, 4, 6.0, 0, 1, 0),
    (FP64_PLAIN, 6, 2, 6.0, 2, -1, 1),
    (FP32_COMPRESSED, 4, 4, 5.7, 1, 1, 1),
]
IDS = ["%s_%dx%d_n%d_n8%d_%s" % ("f64" if c[0] == FP64_PLAIN else "f32", c[1], c[2], c[4], c[5],
                                  "links" if c[6] == 0 else "frozen") for c in CASES]


def pair(q, case, start=HOT, seed=7):
    p, ns, nt, beta, n, n8, mode = case
    lat = q.Lattice(3, ns, nt, beta, n, p, start, seed, field_mode=mode, flux8=n8)
    orc = oracle.OracleLattice(3, ns, nt, beta, n, 10, 0, mode, n8)
    return lat, orc


@pytest.mark.parametrize("precision", [FP64_PLAIN, FP32_COMPRESSED])
def test_cold_start_closed_form(q, precision):
    from test_oracle_lattice import flux_closed_form
    for Ns, n, n8 in [(4, 0, 1), (6, 1, 1), (8, 2, -1)]:
        lat = q.Lattice(3, Ns, 2, 6.0, n, precision, COLD, 1, flux8=n8)
        plaq, poly = lat.measure()
        tol = 1e-12 if precision == FP64_PLAIN else 1e-6
        np.testing.assert_allclose(plaq, flux_closed_form(3, Ns, n, n8), atol=tol)
        np.testing.assert_allclose(lat.measure_bare(), [1.0, 1.0, 1.0], atol=tol)
        lat.close()


def test_lambda8_rejected_for_su2(q):
    with pytest.raises(q.QcdError) as e:
        q.Lattice(2, 4, 2, 2.0, 1, FP64_PLAIN, COLD, 1, flux8=1)
    assert e.value.code == q.QCD_ERR_INVALID_ARG


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_start_and_measurements(q, case):
    lat, orc = pair(q, case)
    orc.set_links(lat.get_links())
    lat.sweep(1, 1, 3)
    orc.set_links(lat.get_links())
    (gp, gl), (op, ol) = lat.measure(), orc.measure()
    tol = 1e-12 if case[0] == FP64_PLAIN else 1e-6
    assert np.abs(np.array(gp) - op).max() <= tol
    assert np.abs(np.array(gl) - ol).max() <= tol
    assert np.abs(np.array(lat.measure_bare()) - orc.measure_bare()).max() <= tol
    lat.close()


@pytest.mark.parametrize("case", [c for c in CASES if c[0] == FP64_PLAIN],
                         ids=[i for c, i in zip(CASES, IDS) if c[0] == FP64_PLAIN])
def test_fp64_sweep(q, case):
    lat, orc = pair(q, case)
    orc.set_links(lat.get_links())
    lat.sweep(1, 2, 7)
    orc.sweep(1, 2, 7)
    check_links(lat.get_links(), orc.get_links(), FP64_PLAIN, "lambda8 sweep")
    lat.close()


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_kernel_by_kernel(q, case):
    lat, orc = pair(q, case)
    schedule = [(q.QCD_HEATBATH, p, mu) for p in (0, 1) for mu in range(4)]
    schedule += [(q.QCD_OVERRELAX, p, mu) for _ in range(2) for p in (0, 1) for mu in range(4)]
    schedule += [("reunitarize", 0, 0)]
    tally = FP32Tally()
    for kind, parity, mu in schedule:
        orc.set_links(lat.get_links())
        orc.sweep_counter = lat.sweep_counter
        if kind == "reunitarize":
            lat.reunitarize()
            orc.reunitarize()
            mask = np.ones(lat.V * 4, dtype=bool)
        else:
            lat.phase(kind, parity, mu, 7)
            orc.phase(kind, parity, mu, 7)
            mask = phase_mask(case[1], case[2], parity, mu)
        if case[0] == FP64_PLAIN:
            check_links(lat.get_links(), orc.get_links(), FP64_PLAIN, (kind, parity, mu))
        else:
            tally.add(lat.get_links(), orc.get_links(), mask, (kind, parity, mu))
    tally.check()
    lat.close()


def test_checkpoint_keeps_lambda8(q, tmp_path):
    path = str(tmp_path / "l8.qcd")
    a = q.Lattice(3, 4, 4, 5.7, 1, FP32_COMPRESSED, HOT, 5, flux8=2)
    a.sweep(1, 1, 5)
    a.save(path)
    b = q.Lattice.load(path, FP32_COMPRESSED)
    assert b.flux8 == 2
    a.sweep(1, 1, 5)
    b.sweep(1, 1, 5)
    assert np.array_equal(a.get_links(), b.get_links())
    assert a.measure() == b.measure()
    a.close()
    b.close()
