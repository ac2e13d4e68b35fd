"""Pins for the O(N) model oracle (multi-hit Metropolis on the lattice phi^4
action), none of which re-types the oracle's formulas:
  - the local action difference equals the total action difference of a
    one-site change, the total action computed independently in numpy;
  - lambda = 0 is the free field: <phi.phi> and the link term follow from the
    lattice propagator 1 / (2 - 4 kappa sum_mu cos p_mu);
  - kappa = 0 decouples the sites: <phi.phi> is a ratio of one-dimensional
    integrals;
  - one site with its neighbours held fixed samples exp(-s(phi)), s the local
    action: moments against two-dimensional quadrature;
  - start, counters and thread-count independence."""
import numpy as np
import pytest

scipy_integrate = pytest.importorskip("scipy.integrate")


def binned(x, b=20):
    x = np.asarray(x, dtype=float)
    n = len(x) // b
    m = x[: n * b].reshape(n, b).mean(1)
    return m.mean(), m.std(ddof=1) / np.sqrt(n)


def np_action(phi, Ns, Nt, kappa, lam):
    """S = sum_x [-2 kappa sum_mu phi_x.phi_{x+mu} + phi_x^2 + lam (phi_x^2 - 1)^2]
    on a field of shape (V, N) in the order [t][z][y][x]."""
    N = phi.shape[1]
    f = phi.reshape(Nt, Ns, Ns, Ns, N)
    pp = (f * f).sum(-1)
    hop = 0.0
    for axis in range(4):  # axes of f: t, z, y, x
        hop += (f * np.roll(f, -1, axis=axis)).sum()
    return -2.0 * kappa * hop + pp.sum() + lam * ((pp - 1.0) ** 2).sum()


@pytest.mark.parametrize("N", [1, 2, 4])
def test_local_action_difference_is_total_difference(oracle_mod, N):
    Ns, Nt, kappa, lam = 4, 2, 0.23, 0.7
    L = oracle_mod.OracleON(N, Ns, Nt, kappa, lam, 1.0, 10)
    L.hot_start(5)
    phi = L.get_field()
    assert abs(L.action() - np_action(phi, Ns, Nt, kappa, lam)) < 1e-11
    rng = np.random.default_rng(1)
    for s in rng.integers(0, L.V, size=12):
        new = rng.normal(size=N)
        d_local = L.local_action(int(s), new) - L.local_action(int(s), phi[s])
        phi2 = phi.copy()
        phi2[s] = new
        d_total = np_action(phi2, Ns, Nt, kappa, lam) - np_action(phi, Ns, Nt, kappa, lam)
        assert abs(d_local - d_total) < 1e-11, (s, d_local, d_total)


def free_field(N, Ns, Nt, kappa):
    """<phi.phi> and (1/4V) sum <phi_x.phi_{x+mu}> of the Gaussian model
    S = sum_x [phi_x^2 - 2 kappa sum_mu phi_x.phi_{x+mu}]: with
    M(p) = 2 - 4 kappa sum_mu cos p_mu, <phi^a_x phi^b_y> = delta^ab (1/V)
    sum_p e^{ip(x-y)} / M(p)."""
    ps = [2 * np.pi * np.arange(Ns) / Ns] * 3 + [2 * np.pi * np.arange(Nt) / Nt]
    P = np.meshgrid(*ps, indexing="ij")
    c = sum(np.cos(p) for p in P)
    M = 2.0 - 4.0 * kappa * c
    V = Ns ** 3 * Nt
    return N * (1.0 / M).sum() / V, N * ((c / 4.0) / M).sum() / V


def test_free_field_propagator(oracle_mod):
    N, Ns, Nt, kappa = 4, 4, 4, 0.1
    L = oracle_mod.OracleON(N, Ns, Nt, kappa, 0.0, 1.6, 8)
    L.hot_start(11)
    L.sweep(50, 11)
    pp, hop = [], []
    for _ in range(1500):
        L.sweep(1, 11)
        m = L.measure()
        pp.append(m[0])
        hop.append(m[1])
    want_pp, want_hop = free_field(N, Ns, Nt, kappa)
    (a, ea), (b, eb) = binned(pp), binned(hop)
    assert abs(a - want_pp) < 4 * ea, (a, ea, want_pp)
    assert abs(b - want_hop) < 4 * eb, (b, eb, want_hop)
    assert abs(want_hop) > 10 * eb  # the coupling is visible


@pytest.mark.parametrize("N,lam", [(1, 0.5), (4, 1.0)])
def test_decoupled_sites(oracle_mod, N, lam):
    """kappa = 0: each site is drawn from r^(N-1) exp(-r^2 - lam (r^2-1)^2) dr."""
    Ns, Nt = 4, 2
    L = oracle_mod.OracleON(N, Ns, Nt, 0.0, lam, 1.2, 20)
    L.hot_start(2)
    L.sweep(10, 2)
    vals = []
    for _ in range(800):
        L.sweep(1, 2)
        vals.append(L.measure()[0])
    w = lambda r, k: r ** k * np.exp(-r * r - lam * (r * r - 1.0) ** 2)
    num = scipy_integrate.quad(lambda r: w(r, N + 1), 0, 6)[0]
    den = scipy_integrate.quad(lambda r: w(r, N - 1), 0, 6)[0]
    want = num / den
    m, e = binned(vals)
    assert abs(m - want) < 4 * e, (m, e, want)


def test_one_site_samples_local_weight(oracle_mod):
    """Neighbours fixed, the site's own chain (one visit = 100 hits) samples
    exp(-s(phi)), s = -2 kappa phi.F + phi^2 + lam (phi^2 - 1)^2.  With
    a = phi.F/|F| and b = |phi - a F/|F||, the N = 4 measure is b^2 da db."""
    N, Ns, Nt, kappa, lam = 4, 4, 2, 0.3, 1.0
    L = oracle_mod.OracleON(N, Ns, Nt, kappa, lam, 0.8, 100)
    L.hot_start(9)
    phi = L.get_field()
    s = 37
    Fvec = np.zeros(N)
    x, y, z, t = s % Ns, (s // Ns) % Ns, (s // Ns ** 2) % Ns, s // Ns ** 3
    for axis, ext in ((0, Ns), (1, Ns), (2, Ns), (3, Nt)):
        for d in (-1, 1):
            c = [x, y, z, t]
            c[axis] = (c[axis] + d) % ext
            Fvec += phi[c[0] + Ns * (c[1] + Ns * (c[2] + Ns * c[3]))]
    F = np.linalg.norm(Fvec)
    u = Fvec / F
    a_s, r2_s = [], []
    cur = phi[s].copy()
    for k in range(20000):
        L.sweep_counter = k
        f = L.get_field() if k == 0 else f
        f[s] = cur
        L.set_field(f)
        cur, _ = L.site_update(s, 17)
        a_s.append(cur @ u)
        r2_s.append(cur @ cur)

    def weight(a, b):
        return b * b * np.exp(2 * kappa * a * F - (a * a + b * b) - lam * (a * a + b * b - 1.0) ** 2)

    Z = scipy_integrate.dblquad(lambda b, a: weight(a, b), -5, 5, 0, 5)[0]
    want_a = scipy_integrate.dblquad(lambda b, a: a * weight(a, b), -5, 5, 0, 5)[0] / Z
    want_r2 = scipy_integrate.dblquad(lambda b, a: (a * a + b * b) * weight(a, b), -5, 5, 0, 5)[0] / Z
    (ma, ea), (mr, er) = binned(a_s, 50), binned(r2_s, 50)
    assert abs(ma - want_a) < 4 * ea, (ma, ea, want_a)
    assert abs(mr - want_r2) < 4 * er, (mr, er, want_r2)


def test_hot_start_and_counters(oracle_mod):
    L = oracle_mod.OracleON(3, 4, 2, 0.2, 0.5, 1.0, 5)
    np.testing.assert_array_equal(L.get_field(), np.tile([1.0, 0.0, 0.0], (L.V, 1)))
    L.hot_start(4)
    f = L.get_field()
    assert np.all(np.abs(f) < 1.0)
    assert abs(f.mean()) < 0.1 and abs(f.var() - 1.0 / 3.0) < 0.05
    assert L.sweep_counter == 0
    L.phase(0, 4)
    assert L.sweep_counter == 0
    L.sweep(3, 4)
    assert L.sweep_counter == 3
    assert 0 < L.accepted <= (L.V // 2 + 3 * L.V) * 5


def test_tiny_step_accepts_almost_everything(oracle_mod):
    L = oracle_mod.OracleON(4, 4, 2, 0.3, 1.0, 1e-4, 10)
    L.hot_start(1)
    L.sweep(2, 1)
    assert L.accepted / (2 * L.V * 10) > 0.99


def test_phase_is_independent_of_thread_count(oracle_mod):
    a = oracle_mod.OracleON(4, 6, 4, 0.3, 1.0, 0.8, 20)
    b = oracle_mod.OracleON(4, 6, 4, 0.3, 1.0, 0.8, 20)
    a.hot_start(3)
    b.hot_start(3)
    n0 = oracle_mod.get_threads()
    try:
        oracle_mod.set_threads(1)
        a.sweep(2, 3)
        oracle_mod.set_threads(max(2, n0))
        b.sweep(2, 3)
    finally:
        oracle_mod.set_threads(n0)
    np.testing.assert_array_equal(a.get_field(), b.get_field())
    assert a.accepted == b.accepted
