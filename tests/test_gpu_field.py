"""Parity of the frozen-boundary field mode (QCD_FIELD_FROZEN) with the FP64
oracle in the same mode: the spatial links of the t = 0 slice hold the
background field B and are never updated or reunitarized, every other link
carries no phase.  Same bars as the effective-link mode: FP64 storage every
link within 1e-9 after whole sweeps, FP32 storage kernel by kernel (pooled
over the schedule)."""
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


# (group, precision, Ns, Nt, beta, flux): ragged tail (6^3 x 4: Vh = 432), the
# 2^4 lattice where every slice is next to t = 0, several flux quanta.
CASES = [
    (2, FP64_PLAIN, 4, 4, 2.3, 1),
    (2, FP32_COMPRESSED, 6, 4, 2.3, 2),
    (2, FP64_PLAIN, 2, 2, 2.0, 1),
    (3, FP64_PLAIN, 4, 4, 5.7, 1),
    (3, FP32_COMPRESSED, 6, 2, 6.0, 3),
    (3, FP64_PLAIN, 6, 4, 6.0, 2),
]
IDS = ["su%d_%s_%dx%d_n%d" % (g, "f64" if p == FP64_PLAIN else "f32", ns, nt, f)
       for g, p, ns, nt, b, f in CASES]


def pair(q, case, start=HOT, seed=7):
    g, p, ns, nt, beta, flux = case
    lat = q.Lattice(g, ns, nt, beta, flux, p, start, seed, field_mode=q.QCD_FIELD_FROZEN)
    orc = oracle.OracleLattice(g, ns, nt, beta, flux, 10, 0, oracle.FIELD_FROZEN)
    return lat, orc


def frozen_part(U, Ns):
    return U[: Ns ** 3, :3]


@pytest.mark.parametrize("case", CASES, ids=IDS)
@pytest.mark.parametrize("start", [COLD, HOT])
def test_start_matches_oracle(q, case, start):
    lat, orc = pair(q, case, start)
    if start == HOT:
        orc.hot_start(7)
    tol = 1e-13 if case[1] == FP64_PLAIN else 2e-7
    assert link_err(lat.get_links(), orc.get_links()).max() < tol
    assert q.qcd_get_field_mode(lat.h) == q.QCD_FIELD_FROZEN
    (gp, gl), (op, ol) = lat.measure(), orc.measure()
    mtol = 1e-12 if case[1] == FP64_PLAIN else 1e-6
    assert np.abs(np.array(gp) - op).max() <= mtol
    assert np.abs(np.array(gl) - ol).max() <= mtol
    lat.close()


@pytest.mark.parametrize("case", [c for c in CASES if c[1] == FP64_PLAIN],
                         ids=[i for c, i in zip(CASES, IDS) if c[1] == FP64_PLAIN])
def test_sweeps_match_oracle(q, case):
    """Graph-launched sweeps from a shared hot start, FP64 storage: SU(2) two
    sweeps of HB + 1 OR, SU(3) one sweep of HB + 2 OR.  The chain amplifies
    rounding-order differences: a 2e-16 relative perturbation of the start
    ends one SU(3) HB + 4 OR sweep of the oracle up to 1.9e-9 away from the
    unperturbed run (two sweeps: 5e-5), HB + 2 OR stays below 1e-11."""
    lat, orc = pair(q, case)
    orc.set_links(lat.get_links())
    n_hb, n_or = (1, 2) if case[0] == 3 else (2, 1)
    lat.sweep(n_hb, n_or, 7)
    orc.sweep(n_hb, n_or, 7)
    check_links(lat.get_links(), orc.get_links(), FP64_PLAIN, "frozen sweep")
    (gp, gl), (op, ol) = lat.measure(), orc.measure()
    assert np.abs(np.array(gp) - op).max() <= 1e-9
    assert np.abs(np.array(gl) - ol).max() <= 1e-9
    lat.close()


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_kernel_by_kernel(q, case):
    """Every phase kernel and the reunitarization from the state the previous
    GPU kernel left; the frozen links stay bit-identical throughout."""
    lat, orc = pair(q, case)
    Ns = case[2]
    frozen0 = frozen_part(lat.get_links(), Ns).copy()
    n_or = 4 if case[0] == 3 else 1
    schedule = [(q.QCD_HEATBATH, p, mu) for p in (0, 1) for mu in range(4)]
    schedule += [(q.QCD_OVERRELAX, p, mu) for _ in range(n_or) for p in (0, 1) for mu in range(4)]
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
            mask = phase_mask(case[2], case[3], parity, mu)
        got = lat.get_links()
        if case[1] == FP64_PLAIN:
            check_links(got, orc.get_links(), case[1], (kind, parity, mu))
        else:
            tally.add(got, orc.get_links(), mask, (kind, parity, mu))
        assert np.array_equal(frozen_part(got, Ns), frozen0), (kind, parity, mu)
    tally.check()
    lat.close()


@pytest.mark.parametrize("group", [2, 3])
def test_beta_zero_matches_oracle(q, group):
    """beta = 0 (every dynamical link drawn from Haar measure, the frozen slice
    kept) from a cold start: links equal the oracle's."""
    case = (group, FP64_PLAIN, 4, 2, 0.0, 2)
    lat, orc = pair(q, case, start=COLD)
    lat.sweep(1, 0, 5)
    orc.sweep(1, 0, 5)
    check_links(lat.get_links(), orc.get_links(), FP64_PLAIN, "beta=0")
    lat.close()


@pytest.mark.parametrize("precision", [FP64_PLAIN, FP32_COMPRESSED])
def test_checkpoint_keeps_field_mode(q, tmp_path, precision):
    path = str(tmp_path / "frozen.qcd")
    a = q.Lattice(3, 4, 4, 5.7, 2, precision, HOT, 5, field_mode=q.QCD_FIELD_FROZEN)
    a.sweep(1, 1, 5)
    a.save(path)
    b = q.Lattice.load(path, precision)
    assert b.field_mode == q.QCD_FIELD_FROZEN
    a.sweep(1, 1, 5)
    b.sweep(1, 1, 5)
    assert np.array_equal(a.get_links(), b.get_links())
    a.close()
    b.close()


def test_unknown_field_mode_is_an_error(q):
    with pytest.raises(q.QcdError) as e:
        q.Lattice(2, 4, 2, 2.0, 1, FP64_PLAIN, COLD, 1, field_mode=2)
    assert e.value.code == q.QCD_ERR_INVALID_ARG
