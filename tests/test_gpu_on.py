"""Parity of the CUDA O(N) model sweep (multi-hit Metropolis) with the FP64
oracle, through the C ABI.

Bars: FP64 storage every component within 1e-12 after whole sweeps and the
accepted-hit counts equal; FP32 storage phase by phase from a shared state,
at least 99.9 % of the updated sites within 1e-5 (a site whose Metropolis
decision falls the other way in FP32 than in FP64 -- u within rounding of
exp(-dS) -- follows another path from that hit on; such sites are counted,
at most 0.1 % + 1), measurements of one configuration within 1e-6.  A
statistical check against the free-field propagator ties the FP32 chain to
the closed form without the oracle."""
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
    oracle.build()
    return q


# (N, precision, Ns, Nt, kappa, lambda, delta, nhit): several blocks and a
# ragged tail (6^3 x 4: Vh = 432), the 2^4 lattice, N = 1..4.
CASES = [
    (4, FP64_PLAIN, 4, 4, 0.3, 1.0, 0.8, 100),
    (4, FP32_COMPRESSED, 4, 4, 0.3, 1.0, 0.8, 100),
    (4, FP32_COMPRESSED, 6, 4, 0.3, 1.0, 0.8, 100),
    (4, FP64_PLAIN, 6, 4, 0.25, 0.5, 1.0, 20),
    (1, FP64_PLAIN, 4, 2, 0.2, 0.8, 1.5, 30),
    (2, FP32_COMPRESSED, 4, 2, 0.2, 0.8, 1.2, 30),
    (3, FP64_PLAIN, 2, 2, 0.3, 1.0, 1.0, 50),
]
IDS = ["o%d_%s_%dx%d_k%g_l%g" % (c[0], "f64" if c[1] == FP64_PLAIN else "f32", c[2], c[3], c[4], c[5])
       for c in CASES]


def pair(q, case, start=HOT, seed=5):
    N, p, ns, nt, kappa, lam, delta, nhit = case
    m = q.ONModel(N, ns, nt, kappa, lam, delta, p, start, seed, nhit=nhit)
    o = oracle.OracleON(N, ns, nt, kappa, lam, delta, nhit)
    if start == HOT:
        o.hot_start(seed)
    return m, o


def parity_of_sites(Ns, Nt):
    s = np.arange(Ns ** 3 * Nt)
    return (s % Ns + (s // Ns) % Ns + (s // Ns ** 2) % Ns + s // Ns ** 3) & 1


@pytest.mark.parametrize("case", CASES, ids=IDS)
@pytest.mark.parametrize("start", [COLD, HOT])
def test_start_matches_oracle(q, case, start):
    m, o = pair(q, case, start)
    tol = 0.0 if case[1] == FP64_PLAIN else 1e-7
    assert np.abs(m.get_field() - o.get_field()).max() <= tol
    g, r = np.array(m.measure()), np.array(o.measure())
    assert np.abs(g - r).max() <= (1e-12 if case[1] == FP64_PLAIN else 1e-6)
    m.close()


@pytest.mark.parametrize("case", [c for c in CASES if c[1] == FP64_PLAIN],
                         ids=[i for c, i in zip(CASES, IDS) if c[1] == FP64_PLAIN])
def test_fp64_sweeps_match_oracle(q, case):
    m, o = pair(q, case)
    m.sweep(3, 5)
    o.sweep(3, 5)
    assert np.abs(m.get_field() - o.get_field()).max() < 1e-12
    assert m.accepted == o.accepted
    assert m.sweep_counter == o.sweep_counter == 3
    g, r = np.array(m.measure()), np.array(o.measure())
    assert np.abs(g - r).max() < 1e-12
    m.close()


@pytest.mark.parametrize("case", [c for c in CASES if c[1] == FP32_COMPRESSED],
                         ids=[i for c, i in zip(CASES, IDS) if c[1] == FP32_COMPRESSED])
def test_fp32_phase_by_phase(q, case):
    m, o = pair(q, case)
    par = parity_of_sites(case[2], case[3])
    n = bad = 0
    for k in range(6):
        parity = k & 1
        before = m.get_field()
        o.set_field(before)
        o.sweep_counter = m.sweep_counter
        m.phase(parity, 5)
        o.phase(parity, 5)
        got, ref = m.get_field(), o.get_field()
        err = np.abs(got - ref).max(axis=1)
        assert np.all(got[par != parity] == before[par != parity])  # other parity untouched
        e = err[par == parity]
        n += e.size
        bad += int((e > 1e-5).sum())
        if parity == 1:
            m.sweep_counter = m.sweep_counter + 1
    assert bad <= 1e-3 * n + 1, (bad, n)
    o.set_field(m.get_field())
    g, r = np.array(m.measure()), np.array(o.measure())
    assert np.abs(g - r).max() <= 1e-6
    m.close()


def test_sweep_is_two_phases_and_an_advance(q):
    case = (4, FP64_PLAIN, 4, 2, 0.3, 1.0, 0.8, 10)
    a, _ = pair(q, case)
    b, _ = pair(q, case)
    a.sweep(2, 9)
    for _ in range(2):
        b.phase(0, 9)
        b.phase(1, 9)
        b.sweep_counter = b.sweep_counter + 1
    assert np.array_equal(a.get_field(), b.get_field())
    assert a.accepted == b.accepted
    a.close()
    b.close()


def test_free_field_on_gpu(q):
    """lambda = 0, FP32: <phi.phi> and the link term against the lattice
    propagator (no oracle involved)."""
    from test_oracle_on import binned, free_field
    N, Ns, Nt, kappa = 4, 8, 8, 0.1
    m = q.ONModel(N, Ns, Nt, kappa, 0.0, 1.6, FP32_COMPRESSED, HOT, 3, nhit=10)
    m.sweep(50, 3)
    pp, hop = [], []
    for _ in range(1500):
        m.sweep(1, 3)
        v = m.measure()
        pp.append(v[0])
        hop.append(v[1])
    want_pp, want_hop = free_field(N, Ns, Nt, kappa)
    (a, ea), (b, eb) = binned(pp), binned(hop)
    assert abs(a - want_pp) < 4 * ea, (a, ea, want_pp)
    assert abs(b - want_hop) < 4 * eb, (b, eb, want_hop)
    m.close()


def test_full_size_sampled_sites(q):
    """O(4) 32^4, kappa 0.3, lambda 1, delta 0.8, NHIT 100, FP32, the bench's
    launch shape: 2000 sites of one phase recomputed one by one by the
    oracle from the same pre-phase field."""
    N, Ns, Nt = 4, 32, 32
    m = q.ONModel(N, Ns, Nt, 0.3, 1.0, 0.8, FP32_COMPRESSED, HOT, 7)
    m.sweep(1, 7)
    before = m.get_field()
    o = oracle.OracleON(N, Ns, Nt, 0.3, 1.0, 0.8, 100)
    o.set_field(before)
    o.sweep_counter = m.sweep_counter
    m.phase(1, 7)
    after = m.get_field()
    par = parity_of_sites(Ns, Nt)
    rng = np.random.default_rng(0)
    sites = rng.choice(np.nonzero(par == 1)[0], size=2000, replace=False)
    bad = 0
    for s in sites:
        ref, _ = o.site_update(int(s), 7)
        bad += int(np.abs(ref - after[s]).max() > 1e-5)
    assert bad <= 3, bad
    assert np.all(after[par == 0] == before[par == 0])
    m.close()
    o.close()


def test_bad_arguments(q):
    for args in [(0, 4, 4, 0.1, 1.0, 1.0), (5, 4, 4, 0.1, 1.0, 1.0), (4, 3, 4, 0.1, 1.0, 1.0),
                 (4, 4, 4, 0.1, 1.0, 0.0)]:
        with pytest.raises(q.QcdError) as e:
            q.ONModel(*args)
        assert e.value.code == q.QCD_ERR_INVALID_ARG
    m = q.ONModel(4, 4, 2, 0.1, 1.0, 1.0)
    with pytest.raises(q.QcdError):
        q.qcd_on_set_nhit(m.h, 0)
    with pytest.raises(q.QcdError):
        q.qcd_on_phase(m.h, 2, 1)
    m.close()
