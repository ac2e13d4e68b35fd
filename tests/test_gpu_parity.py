"""Parity of the CUDA sweep (through the C ABI) with the FP64 CPU oracle.

Bars:
  FP64 plain storage      every link within 1e-9 after one sweep (rounding
                          order only, amplified by the chaotic chain),
                          measurements within 1e-12;
  FP32 compressed storage at least 99.99% of links within 1e-5 (max abs over
                          the link's reals) after every kernel of the sweep
                          schedule from a shared state, and after one short
                          sweep (SU(2) HB + 1 OR, SU(3) HB, SU(3) 16^3 x 4
                          HB + 1 OR); links that diverge on an accept/reject
                          branch are counted; plaquette of one configuration
                          |dP| <= 1e-6.
The chain amplifies any perturbation: with FP32 rounding of the stored links as
the only difference, the oracle itself ends one SU(3) 16^3 x 4 HB + 4 OR sweep
with every link beyond 1e-5 of its pure FP64 run (tests/test_oracle_fp32_sweep.py).
The FP32 path is therefore held to the link bar kernel by kernel, on
heat-bath sweeps and against the oracle's own divergence on whole sweeps
(tests/test_gpu_fp32_sweep.py), and to the FP64 chain statistically
(tests/test_gpu_ensemble.py).
"""
import numpy as np
import pytest

import oracle
from workloads import FP32_COMPRESSED, FP64_PLAIN, HOT, COLD

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


def link_err(a, b):
    V = a.shape[0]
    return np.abs(a - b).reshape(V * 4, -1).max(axis=1)


def check_links(a, b, precision, what=""):
    err = link_err(a, b)
    if precision == FP64_PLAIN:
        assert err.max() < 1e-9, (what, err.max())
    else:
        frac = (err <= 1e-5).mean()
        assert frac >= 0.9999, (what, frac, int((err > 1e-5).sum()), err.max())
    return err


def phase_mask(Ns, Nt, parity, mu):
    """Links a checkerboard phase (parity, mu) updates, in the canonical order
    [t][z][y][x][mu]."""
    t, z, y, x = np.meshgrid(*(np.arange(n) for n in (Nt, Ns, Ns, Ns)), indexing="ij")
    on = ((x + y + z + t) & 1).reshape(-1) == parity
    m = np.zeros((on.size, 4), dtype=bool)
    m[on, mu] = True
    return m.reshape(-1)


class FP32Tally:
    """FP32 bar pooled over the kernels of one schedule: links outside a phase
    bit-identical, at least 99.99 % of updated links within 1e-5 of the oracle
    (one such link is always allowed: a 4^3 x 4 schedule has only 6144
    updates), none beyond 1e-4.  An overrelaxation reflection divides by the
    norm of the subgroup block, so the rare links where that norm is small
    amplify FP32 rounding past 1e-5 (about one update in 10^5, in any FP32
    evaluation order)."""

    def __init__(self):
        self.n = self.bad = 0
        self.worst = 0.0

    def add(self, got, ref, mask, what):
        err = link_err(got, ref)
        assert err[~mask].max(initial=0.0) == 0.0, (what, "link outside the phase changed")
        e = err[mask]
        self.n += e.size
        self.bad += int((e > 1e-5).sum())
        self.worst = max(self.worst, float(e.max(initial=0.0)))
        assert self.worst < 1e-4, (what, self.worst)

    def check(self):
        assert self.bad <= max(1.0, 1e-4 * self.n), (self.bad, self.n, self.worst)


# (group, precision, Ns, Nt, beta, flux): several tiles, ragged tails (Vh = 432,
# 216), the degenerate 2^4 lattice, field on and off.
CASES = [
    (2, FP64_PLAIN, 4, 4, 2.3, 0),
    (2, FP32_COMPRESSED, 4, 4, 2.3, 0),
    (2, FP64_PLAIN, 6, 4, 2.3, 2),
    (2, FP32_COMPRESSED, 6, 4, 2.3, 2),
    (2, FP64_PLAIN, 2, 2, 2.0, 1),
    (3, FP64_PLAIN, 4, 4, 5.7, 0),
    (3, FP32_COMPRESSED, 4, 4, 5.7, 0),
    (3, FP64_PLAIN, 6, 2, 6.0, 1),
    (3, FP32_COMPRESSED, 6, 2, 6.0, 1),
    (3, FP32_COMPRESSED, 8, 6, 6.0, 4),
    (3, FP64_PLAIN, 2, 2, 5.0, 1),
]
IDS = ["su%d_%s_%dx%d_b%g_n%d" % (g, "f64" if p == FP64_PLAIN else "f32", ns, nt, b, f)
       for g, p, ns, nt, b, f in CASES]


def pair(q, case, start=HOT, seed=7, nhit=10):
    g, p, ns, nt, beta, flux = case
    lat = q.Lattice(g, ns, nt, beta, flux, p, start, seed, nhit=nhit)
    orc = oracle.OracleLattice(g, ns, nt, beta, flux, nhit, 0)
    return lat, orc


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_hot_start_matches_oracle(q, case):
    lat, orc = pair(q, case)
    orc.hot_start(7)
    tol = 1e-13 if case[1] == FP64_PLAIN else 2e-7
    assert link_err(lat.get_links(), orc.get_links()).max() < tol
    lat.close()


WHOLE_SWEEP = [c for c in CASES if c[1] == FP64_PLAIN or c[0] == 2]


@pytest.mark.parametrize("case", WHOLE_SWEEP, ids=[IDS[CASES.index(c)] for c in WHOLE_SWEEP])
def test_one_sweep_from_shared_start(q, case):
    """One whole graph-launched sweep from a shared start: HB + 4 OR (SU(3))
    or HB + 1 OR (SU(2)) with FP64 storage; an SU(2) heat-bath pass with FP32
    storage.  The chain amplifies FP32 rounding past 1e-5 within an OR pass
    (and, for SU(3), through small subgroup norms within a heat-bath pass), so
    FP32 SU(3) and every FP32 OR kernel are held to the bar kernel by kernel
    (test_sweep_schedule_kernel_by_kernel)."""
    lat, orc = pair(q, case)
    orc.set_links(lat.get_links())
    n_or = (4 if case[0] == 3 else 1) if case[1] == FP64_PLAIN else 0
    lat.sweep(1, n_or, 7)
    orc.sweep(1, n_or, 7)
    check_links(lat.get_links(), orc.get_links(), case[1], "sweep")
    assert lat.sweep_counter == 1 == orc.sweep_counter
    lat.close()


def run_kernel_by_kernel(q, case, seed=7):
    """Every kernel of one HB + n_or OR sweep (n_or = 4 for SU(3)) and the
    reunitarization, each from the state the previous GPU kernel left, against
    the oracle started from that same state."""
    lat, orc = pair(q, case, seed=seed)
    lat.sweep(1, 1, seed)  # launch shape chosen as in a normal run
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
            lat.phase(kind, parity, mu, seed)
            orc.phase(kind, parity, mu, seed)
            mask = phase_mask(case[2], case[3], parity, mu)
        if case[1] == FP64_PLAIN:
            check_links(lat.get_links(), orc.get_links(), case[1], (kind, parity, mu))
        else:
            tally.add(lat.get_links(), orc.get_links(), mask, (kind, parity, mu))
    tally.check()
    lat.close()


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_sweep_schedule_kernel_by_kernel(q, case):
    run_kernel_by_kernel(q, case)


def test_su3_16x4_fp32_kernel_by_kernel(q):
    """SU(3) 16^3 x 4, beta 5.7, hot start seed 7, FP32-compressed links: the
    whole HB + 4 OR + reunitarization schedule, 65536 links per check."""
    run_kernel_by_kernel(q, (3, FP32_COMPRESSED, 16, 4, 5.7, 0))


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_measurements_on_one_configuration(q, case):
    lat, orc = pair(q, case)
    lat.sweep(2, 1, 11)
    orc.set_links(lat.get_links())
    (gp, gl), (op, ol) = lat.measure(), orc.measure()
    tol = 1e-12 if case[1] == FP64_PLAIN else 1e-6
    assert np.abs(np.array(gp) - op).max() <= tol, (gp, op)
    assert np.abs(np.array(gl) - ol).max() <= tol, (gl, ol)
    assert np.abs(np.array(lat.measure_bare()) - orc.measure_bare()).max() <= tol
    lat.close()


@pytest.mark.parametrize("case", [CASES[2], CASES[3], CASES[7], CASES[8]], ids=[IDS[2], IDS[3], IDS[7], IDS[8]])
def test_every_single_phase(q, case):
    lat, orc = pair(q, case)
    lat.sweep(1, 1, 3)
    tally = FP32Tally()
    for kind in (q.QCD_HEATBATH, q.QCD_OVERRELAX):
        for parity in (0, 1):
            for mu in range(4):
                orc.set_links(lat.get_links())
                orc.sweep_counter = lat.sweep_counter
                lat.phase(kind, parity, mu, 21)
                orc.phase(kind, parity, mu, 21)
                if case[1] == FP64_PLAIN:
                    check_links(lat.get_links(), orc.get_links(), case[1], (kind, parity, mu))
                else:
                    tally.add(lat.get_links(), orc.get_links(), phase_mask(case[2], case[3], parity, mu),
                              (kind, parity, mu))
    tally.check()
    lat.close()


@pytest.mark.parametrize("group", [2, 3])
@pytest.mark.parametrize("precision", [FP64_PLAIN, FP32_COMPRESSED])
def test_cold_start_and_flux_closed_form(q, group, precision):
    from test_oracle_lattice import flux_closed_form
    for Ns, n in [(4, 1), (6, 2), (8, 3)]:
        lat = q.Lattice(group, Ns, 2, 6.0, n, precision, COLD, 1)
        plaq, poly = lat.measure()
        tol = 1e-12 if precision == FP64_PLAIN else 1e-6
        np.testing.assert_allclose(plaq, flux_closed_form(group, Ns, n), atol=tol)
        np.testing.assert_allclose(poly, [1.0, 0.0], atol=tol)
        np.testing.assert_allclose(lat.measure_bare(), [1.0, 1.0, 1.0], atol=tol)
        lat.close()


@pytest.mark.parametrize("group", [2, 3])
def test_beta_zero_haar_branch(q, group):
    case = (group, FP64_PLAIN, 4, 2, 0.0, 1)
    lat, orc = pair(q, case, start=COLD)
    lat.sweep(1, 0, 5)
    orc.sweep(1, 0, 5)
    check_links(lat.get_links(), orc.get_links(), FP64_PLAIN, "beta=0")
    lat.close()


@pytest.mark.parametrize("group", [2, 3])
def test_nhit_exhaustion_count(q, group):
    case = (group, FP64_PLAIN, 4, 4, 0.05, 0)
    lat, orc = pair(q, case, nhit=1)
    orc.set_links(lat.get_links())
    lat.sweep(1, 0, 9)
    orc.sweep(1, 0, 9)
    assert orc.exhausted > 0
    assert lat.exhausted == orc.exhausted
    check_links(lat.get_links(), orc.get_links(), FP64_PLAIN, "nhit=1")
    lat.close()


@pytest.mark.parametrize("precision", [FP64_PLAIN, FP32_COMPRESSED])
def test_set_get_round_trip(q, precision):
    lat = q.Lattice(3, 4, 2, 5.0, 0, precision, HOT, 3)
    orc = oracle.OracleLattice(3, 4, 2, 5.0, 0, 10, 0)
    orc.hot_start(99)
    ref = orc.get_links()
    lat.set_links(ref)
    tol = 0.0 if precision == FP64_PLAIN else 6e-7
    assert link_err(lat.get_links(), ref).max() <= tol
    lat.close()


def test_bad_arguments_are_errors(q):
    for args in [(4, 4, 4, 1.0), (2, 3, 4, 1.0), (2, 4, 5, 1.0), (3, 0, 4, 1.0), (3, 4, 4, -1.0)]:
        with pytest.raises(q.QcdError) as e:
            q.Lattice(*args)
        assert e.value.code == q.QCD_ERR_INVALID_ARG
    lat = q.Lattice(2, 4, 2, 1.0)
    with pytest.raises(q.QcdError):
        q.qcd_phase(lat.h, 5, 0, 0, 1)
    with pytest.raises(q.QcdError):
        q.qcd_set_nhit(lat.h, 0)
    with pytest.raises(q.QcdError):
        q.qcd_sweep(lat.h, -1, 0, 1)
    lat.close()


def binned(x, b=20):
    x = np.asarray(x)
    n = len(x) // b
    m = x[: n * b].reshape(n, b).mean(1)
    return m.mean(), m.std(ddof=1) / np.sqrt(n)


@pytest.mark.parametrize("precision", [FP64_PLAIN, FP32_COMPRESSED])
def test_ensemble_su2_4x4(q, precision):
    """SU(2) 4^3 x 4, beta 2.3, cold start, 1 HB + 1 OR: 10^3 sweeps on the GPU
    and an independent oracle chain agree within 3 sigma in <P> and <L>."""
    lat = q.Lattice(2, 4, 4, 2.3, 0, precision, COLD, 1)
    orc = oracle.OracleLattice(2, 4, 4, 2.3, 0, 10, 0)
    g_p, g_l, o_p, o_l = [], [], [], []
    for i in range(1100):
        lat.sweep(1, 1, 1)
        orc.sweep(1, 1, 2)
        if i >= 100:
            (p, l), (op, ol) = lat.measure(), orc.measure()
            g_p.append(p[0]); g_l.append(l[0]); o_p.append(op[0]); o_l.append(ol[0])
    for a, b in ((g_p, o_p), (g_l, o_l)):
        (ma, ea), (mb, eb) = binned(a), binned(b)
        assert abs(ma - mb) < 3 * np.hypot(ea, eb) + 1e-12, (ma, ea, mb, eb)
    lat.close()


@pytest.mark.parametrize("group", [2, 3])
@pytest.mark.parametrize("precision", [FP64_PLAIN, FP32_COMPRESSED])
def test_reunitarization_of_perturbed_links(q, group, precision):
    """Links pushed 1e-3 off the group: the GPU's reunitarization matches the
    oracle's FP64 Gram-Schmidt of the same stored values to rounding (FP32
    storage: about one unit in the last place) and restores unitarity."""
    lat = q.Lattice(group, 4, 4, 2.0, 0, precision, HOT, 13)
    U = lat.get_links()
    rng = np.random.default_rng(1)
    P = U + 1e-3 * (rng.normal(size=U.shape) + 1j * rng.normal(size=U.shape))
    lat.set_links(P)
    stored = lat.get_links()  # what the storage keeps (FP32 rows, SU(2) projection)
    orc = oracle.OracleLattice(group, 4, 4, 2.0, 0, 10, 0)
    orc.set_links(stored)
    lat.reunitarize()
    orc.reunitarize()
    got, ref = lat.get_links(), orc.get_links()
    tol = 1e-14 if precision == FP64_PLAIN else 2.5e-7
    assert link_err(got, ref).max() < tol
    M = got.reshape(-1, group, group)
    unit = np.abs(np.einsum("nki,nkj->nij", M.conj(), M) - np.eye(group)).max()
    assert unit < (1e-14 if precision == FP64_PLAIN else 5e-7)
    lat.close()


def test_measure_async_equals_measure(q):
    import torch
    lat = q.Lattice(3, 6, 4, 5.9, 1, FP32_COMPRESSED, HOT, 3)
    lat.sweep(1, 1, 3)
    out = torch.zeros(5, dtype=torch.float64, pin_memory=True)
    q.qcd_measure_async(lat.h, out.data_ptr())
    torch.cuda.synchronize()
    (p, l) = lat.measure()
    assert out.tolist() == list(p) + list(l)
    lat.close()


@pytest.mark.parametrize("group,precision,flux,flux8,mode", [
    (3, FP32_COMPRESSED, 1, 0, 0), (3, FP32_COMPRESSED, 0, 0, 0), (3, FP32_COMPRESSED, 1, 1, 0),
    (3, FP32_COMPRESSED, 1, 0, 1), (3, FP64_PLAIN, 1, 0, 0), (2, FP32_COMPRESSED, 1, 0, 0)])
def test_working_sweep_equals_sweep_then_measure(q, group, precision, flux, flux8, mode):
    """qcd_working_sweep (measurement fused into the last overrelaxation pass
    where available) gives the links of qcd_sweep and the measurement of
    qcd_measure on them."""
    Ns, Nt, beta = 6, 4, (5.8 if group == 3 else 2.3)
    a = q.Lattice(group, Ns, Nt, beta, flux, precision, HOT, 5, field_mode=mode, flux8=flux8)
    b = q.Lattice(group, Ns, Nt, beta, flux, precision, HOT, 5, field_mode=mode, flux8=flux8)
    for n_hb, n_or in ((1, 4), (2, 1), (1, 0)):
        got = q.qcd_working_sweep(a.h, n_hb, n_or, 5)
        b.sweep(n_hb, n_or, 5)
        assert np.array_equal(a.get_links(), b.get_links())
        (p, l) = b.measure()
        tol = 1e-12 if precision == FP64_PLAIN else 1e-6
        assert np.abs(np.array(got) - np.array(list(p) + list(l))).max() <= tol, (got, p, l)
    a.close()
    b.close()


@pytest.mark.parametrize("Ns,Nt", [(4, 2), (6, 6), (4, 8), (8, 16), (6, 10)])
def test_fused_polyakov_any_nt(q, Ns, Nt):
    """The fused Polyakov loop (its own kernel, products by rows 0-1 with row 2
    rebuilt) gives the measurement of qcd_measure at every time extent,
    including the partly unrolled t-loop's remainders."""
    a = q.Lattice(3, Ns, Nt, 5.8, 1, FP32_COMPRESSED, HOT, 5)
    b = q.Lattice(3, Ns, Nt, 5.8, 1, FP32_COMPRESSED, HOT, 5)
    got = q.qcd_working_sweep(a.h, 1, 2, 5)
    b.sweep(1, 2, 5)
    (p, l) = b.measure()
    assert np.abs(np.array(got) - np.array(list(p) + list(l))).max() <= 1e-6, (got, p, l)
    a.close()
    b.close()


def test_working_sweep_matches_oracle_measure(q):
    """Fused measurement on a 16^3 x 4 FP32 lattice against the oracle's
    measurement of the same configuration."""
    lat = q.Lattice(3, 16, 4, 5.9, 1, FP32_COMPRESSED, HOT, 9)
    got = q.qcd_working_sweep(lat.h, 1, 2, 9)
    orc = oracle.OracleLattice(3, 16, 4, 5.9, 1, 10, 0)
    orc.set_links(lat.get_links())
    (op, ol) = orc.measure()
    assert np.abs(np.array(got) - np.array(list(op) + list(ol))).max() <= 1e-6, (got, op, ol)
    lat.close()


def test_live_profile_counts_every_kernel(q):
    """Live profile over sweeps and working sweeps: launches per category as
    the sweep schedule has them, positive times, sum within the wall time."""
    import torch
    lat = q.Lattice(3, 8, 4, 5.9, 1, FP32_COMPRESSED, HOT, 3)
    lat.sweep(1, 4, 3)
    q.qcd_set_profiling(lat.h, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    lat.sweep(3, 4, 3)
    for _ in range(2):
        q.qcd_working_sweep(lat.h, 1, 4, 3)
    e1.record()
    torch.cuda.synchronize()
    ms, n = q.qcd_get_profile(lat.h)
    q.qcd_set_profiling(lat.h, False)
    assert list(n) == [5 * 8, 5 * 24, 5 * 9, 2 * 2], n
    assert all(m > 0 for m in ms)
    assert sum(ms) <= e0.elapsed_time(e1) * 1.001
    lat.close()
