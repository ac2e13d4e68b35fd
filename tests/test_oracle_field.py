"""Pins for the frozen-boundary field mode of the oracle: the background field
is imposed through the spatial links of the t = 0 slice, which are fixed to B
and never updated; all other links carry no phase."""
import numpy as np
import pytest

import lattice_np as ln


def make(oracle_mod, N, Ns, Nt, beta, flux, hot_seed=None):
    L = oracle_mod.OracleLattice(N, Ns, Nt, beta, flux, 10, 0, oracle_mod.FIELD_FROZEN)
    if hot_seed is not None:
        L.hot_start(hot_seed)
    return L


def frozen_config(N, Ns, Nt, flux, U=None):
    """Links with the t = 0 spatial links set to B (numpy, independent)."""
    V = Ns ** 3 * Nt
    if U is None:
        U = np.broadcast_to(np.eye(N, dtype=complex), (V, 4, N, N)).copy()
    for s in range(Ns ** 3):
        for mu in range(3):
            U[s, mu] = ln.background(N, Ns, Nt, flux, s, mu)
    return U


@pytest.mark.parametrize("N", [2, 3])
@pytest.mark.parametrize("Ns,Nt,n", [(4, 2, 1), (4, 4, 3), (6, 2, 2)])
def test_cold_start_matches_brute_force(oracle_mod, N, Ns, Nt, n):
    L = make(oracle_mod, N, Ns, Nt, 2.0, n)
    U = L.get_links()
    np.testing.assert_array_equal(U, frozen_config(N, Ns, Nt, n))
    plaq, poly = L.measure()
    np.testing.assert_allclose(plaq, ln.plaquettes(U, Ns, Nt), atol=1e-13)
    # the temporal plaquettes at t = 0 and t = Nt-1 see the frozen y-links
    assert plaq[2] < 1.0 - 1e-3
    np.testing.assert_allclose(L.measure_bare(), plaq, atol=0)


@pytest.mark.parametrize("N", [2, 3])
def test_frozen_links_never_change(oracle_mod, N):
    Ns, Nt, n = 4, 4, 2
    L = make(oracle_mod, N, Ns, Nt, 2.3 if N == 2 else 5.7, n, hot_seed=3)
    U0 = L.get_links()
    np.testing.assert_array_equal(U0[: Ns ** 3, :3], frozen_config(N, Ns, Nt, n)[: Ns ** 3, :3])
    L.sweep(3, 2, 3)
    U1 = L.get_links()
    np.testing.assert_array_equal(U1[: Ns ** 3, :3], U0[: Ns ** 3, :3])
    moved = np.abs(U1 - U0).reshape(L.V, 4, -1).max(-1)
    moved[: Ns ** 3, :3] = 1.0
    assert (moved > 1e-6).all()  # every other link was updated


@pytest.mark.parametrize("N", [2, 3])
def test_overrelaxation_conserves_action_with_frozen_slice(oracle_mod, N):
    L = make(oracle_mod, N, 4, 4, 2.0 if N == 2 else 5.7, 3, hot_seed=8)
    L.sweep(1, 0, 1)
    for p in range(2):
        for mu in range(4):
            before = L.measure()[0][0]
            L.phase(oracle_mod.OVERRELAX, p, mu, 0)
            assert abs(L.measure()[0][0] - before) < 1e-13


@pytest.mark.parametrize("N", [2, 3])
def test_staple_next_to_frozen_slice(oracle_mod, N):
    Ns, Nt, n = 4, 4, 1
    L = make(oracle_mod, N, Ns, Nt, 1.0, n, hot_seed=11)
    U = L.get_links()  # effective links are the links themselves here
    for c in ([1, 2, 3, 1], [0, 0, 1, 0], [3, 1, 0, 3]):
        s = ln.index(Ns, c)
        for mu in range(4):
            np.testing.assert_allclose(L.staple(s, mu), ln.staple_from_plaquettes(U, Ns, Nt, s, mu), atol=1e-12)


@pytest.mark.parametrize("N", [2, 3])
def test_beta_zero_leaves_only_frozen_plaquettes(oracle_mod, N):
    """beta = 0: every dynamical link becomes Haar, so only the spatial
    plaquettes of the frozen slice (all four links fixed) keep a mean:
    <P_s> = (2 + <xy>) / (3 Nt) with <xy> the closed-form flux value, P_t -> 0."""
    from test_oracle_lattice import flux_closed_form
    Ns, Nt, n = 4, 4, 3
    L = make(oracle_mod, N, Ns, Nt, 0.0, n)
    ps, pt = [], []
    for _ in range(20):
        L.sweep(1, 0, 7)
        p, _ = L.measure()
        ps.append(p[1])
        pt.append(p[2])
    xy = 3.0 * flux_closed_form(N, Ns, n)[1] - 2.0  # mean xy value of the slice
    expect = (2.0 + xy) / (3.0 * Nt)
    sigma = np.sqrt(1.0 / N ** 2 / (3 * L.V) / len(ps))
    assert abs(np.mean(ps) - expect) < 6 * sigma, (np.mean(ps), expect)
    assert abs(np.mean(pt)) < 6 * sigma
    assert abs(expect - 1.0 / Nt) > 10 * sigma or n == 0  # the field is visible
