"""Pins for the lambda8 component of the background field (SU(3)): on y-links
B = diag(e^{i(p3 + p8)}, e^{i(-p3 + p8)}, e^{-2 i p8}), p = 2 pi n x / Ns^2,
in both field modes.  Checked against closed forms, brute-force numpy
plaquettes and the staple-as-derivative identity, not against the oracle's
own formulas."""
import numpy as np
import pytest

import lattice_np as ln
from test_oracle_lattice import flux_closed_form


def test_lambda8_rejected_for_su2(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.OracleLattice(2, 4, 4, 2.0, 1, 10, 0, oracle_mod.FIELD_LINKS, 1)


@pytest.mark.parametrize("Ns,n,n8", [(4, 0, 1), (4, 1, 1), (6, 2, -1), (8, 1, 3)])
def test_cold_start_closed_form(oracle_mod, Ns, n, n8):
    L = oracle_mod.OracleLattice(3, Ns, 2, 6.0, n, 10, 0, oracle_mod.FIELD_LINKS, n8)
    plaq, poly = L.measure()
    np.testing.assert_allclose(plaq, flux_closed_form(3, Ns, n, n8), rtol=0, atol=1e-12)
    assert poly == [1.0, 0.0]
    # lambda8 alone moves the plaquette away from the lambda3-only value
    if n8:
        assert abs(plaq[1] - flux_closed_form(3, Ns, n)[1]) > 1e-4


def test_closed_form_helper_is_brute_force():
    """The closed form itself against numpy plaquettes of B on a cold lattice."""
    for Ns, n, n8 in [(4, 1, 1), (6, 2, -1)]:
        V = Ns ** 3 * 2
        U = np.broadcast_to(np.eye(3, dtype=complex), (V, 4, 3, 3)).copy()
        Ut = ln.effective(U, Ns, 2, n, n8)
        ps = ln.plaquettes(Ut, Ns, 2)
        want = flux_closed_form(3, Ns, n, n8)
        assert abs(ps[0] - want[0]) < 1e-12 and abs(ps[1] - want[1]) < 1e-12


def test_measure_and_staple_brute_force(oracle_mod):
    Ns, Nt, n, n8 = 4, 2, 1, 2
    L = oracle_mod.OracleLattice(3, Ns, Nt, 5.7, n, 10, 0, oracle_mod.FIELD_LINKS, n8)
    L.hot_start(3)
    L.sweep(1, 1, 9)
    U = L.get_links()
    Ut = ln.effective(U, Ns, Nt, n, n8)
    plaq, _ = L.measure()
    np.testing.assert_allclose(plaq, ln.plaquettes(Ut, Ns, Nt), atol=1e-13)
    for s in (0, 5, 21):
        for mu in range(4):
            np.testing.assert_allclose(L.staple(s, mu), ln.staple_from_plaquettes(Ut, Ns, Nt, s, mu), atol=1e-12)


def test_lambda8_is_a_change_of_variables(oracle_mod):
    """As for lambda3: the field-(n, n8) run from U0 = W0 B^+ tracks the
    field-free run from W0 in effective links."""
    Ns, Nt, n, n8, beta = 4, 4, 1, 2, 5.7
    A = oracle_mod.OracleLattice(3, Ns, Nt, beta, 0, 10, 0)
    A.hot_start(17)
    W0 = A.get_links()
    B = oracle_mod.OracleLattice(3, Ns, Nt, beta, n, 10, 0, oracle_mod.FIELD_LINKS, n8)
    U0 = W0.copy()
    for s in range(A.V):
        U0[s, 1] = W0[s, 1] @ ln.background(3, Ns, Nt, n, s, 1, n8).conj().T
    B.set_links(U0)
    A.sweep(2, 2, 55)
    B.sweep(2, 2, 55)
    assert np.abs(A.get_links() - ln.effective(B.get_links(), Ns, Nt, n, n8)).max() < 1e-8


def test_frozen_mode_with_lambda8(oracle_mod):
    """Frozen boundary: the t = 0 spatial links hold the (lambda3 + lambda8)
    B at start and after sweeps; cold-start plaquettes from numpy."""
    Ns, Nt, n, n8 = 4, 4, 1, 1
    L = oracle_mod.OracleLattice(3, Ns, Nt, 5.7, n, 10, 0, oracle_mod.FIELD_FROZEN, n8)
    U = L.get_links()
    for s in range(Ns ** 3):
        for mu in range(3):
            np.testing.assert_array_equal(U[s, mu], ln.background(3, Ns, Nt, n, s, mu, n8))
    np.testing.assert_allclose(L.measure()[0], ln.plaquettes(U, Ns, Nt), atol=1e-13)
    L.hot_start(5)
    L.sweep(2, 1, 5)
    U2 = L.get_links()
    for s in range(Ns ** 3):
        np.testing.assert_array_equal(U2[s, 1], ln.background(3, Ns, Nt, n, s, 1, n8))
