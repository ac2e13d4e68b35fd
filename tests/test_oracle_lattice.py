"""Pins for the oracle's lattice routines: measurements, staple, updates,
reunitarization and the background field, each tied to a closed form, an
invariant or a brute-force numpy computation."""
import numpy as np
import pytest

import lattice_np as ln
from test_oracle_sampling import chi2_pvalue, kp_bin_probs


def make(oracle_mod, N, Ns, Nt, beta, flux=0, nhit=10, hot_seed=None, lid=0):
    L = oracle_mod.OracleLattice(N, Ns, Nt, beta, flux, nhit, lid)
    if hot_seed is not None:
        L.hot_start(hot_seed)
    return L


@pytest.mark.parametrize("N", [2, 3])
def test_create_rejects_bad_arguments(oracle_mod, N):
    for args in [(N, 3, 4, 1.0), (N, 4, 3, 1.0), (N, 0, 4, 1.0), (4, 4, 4, 1.0), (N, 4, 4, -1.0)]:
        with pytest.raises(ValueError):
            oracle_mod.OracleLattice(*args)


@pytest.mark.parametrize("N", [2, 3])
def test_cold_start_closed_form(oracle_mod, N):
    L = make(oracle_mod, N, 4, 2, 2.0)
    plaq, poly = L.measure()
    assert plaq == [1.0, 1.0, 1.0]
    assert poly == [1.0, 0.0]
    assert L.measure_bare() == [1.0, 1.0, 1.0]


def flux_closed_form(N, Ns, n, n8=0):
    """Cold start, effective links = B: only xy-plaquettes see the field.  The
    diagonal entry k of B_y carries the phase 2 pi h_k x / Ns^2 with
    h = n (1, -1, 0) + n8 (1, 1, -2); an xy-plaquette is (1/N) sum_k cos of its
    phase difference, 2 pi h_k / Ns^2 inside and -2 pi h_k (Ns-1)/Ns^2 across
    the periodic x boundary."""
    h = n * np.array([1.0, -1.0, 0.0][:N]) + (n8 * np.array([1.0, 1.0, -2.0]) if N == 3 else 0.0)
    f = lambda d: np.cos(d * h).mean()
    inner = 2 * np.pi / Ns ** 2
    edge = -2 * np.pi * (Ns - 1) / Ns ** 2
    xy = ((Ns - 1) * f(inner) + f(edge)) / Ns
    ps = (xy + 2.0) / 3.0
    return (3 * ps + 3.0) / 6.0, ps, 1.0


@pytest.mark.parametrize("N", [2, 3])
@pytest.mark.parametrize("Ns,n", [(4, 1), (4, 3), (6, 2), (8, 1)])
def test_flux_closed_form(oracle_mod, N, Ns, n):
    L = make(oracle_mod, N, Ns, 2, 6.0, flux=n)
    plaq, poly = L.measure()
    np.testing.assert_allclose(plaq, flux_closed_form(N, Ns, n), rtol=0, atol=1e-12)
    assert poly == [1.0, 0.0]
    assert L.measure_bare() == [1.0, 1.0, 1.0]


@pytest.mark.parametrize("N,Ns,Nt,flux", [(2, 4, 2, 1), (3, 2, 4, 1), (3, 4, 2, 3)])
def test_measure_matches_brute_force(oracle_mod, N, Ns, Nt, flux):
    L = make(oracle_mod, N, Ns, Nt, 2.0, flux=flux, hot_seed=3)
    L.sweep(1, 1, 9)
    U = L.get_links()
    Ut = ln.effective(U, Ns, Nt, flux)
    plaq, poly = L.measure()
    np.testing.assert_allclose(plaq, ln.plaquettes(Ut, Ns, Nt), atol=1e-13)
    np.testing.assert_allclose(L.measure_bare(), ln.plaquettes(U, Ns, Nt), atol=1e-13)
    pl = ln.polyakov(Ut, Ns, Nt)
    np.testing.assert_allclose(poly, [pl.real, pl.imag], atol=1e-13)


@pytest.mark.parametrize("N,Ns,Nt,flux", [(2, 4, 4, 2), (3, 4, 2, 1), (3, 2, 2, 1), (2, 2, 2, 0)])
def test_staple_is_plaquette_derivative(oracle_mod, N, Ns, Nt, flux):
    L = make(oracle_mod, N, Ns, Nt, 1.0, flux=flux, hot_seed=11)
    Ut = ln.effective(L.get_links(), Ns, Nt, flux)
    rng = np.random.default_rng(0)
    for s in rng.integers(0, L.V, size=6):
        for mu in range(4):
            A = L.staple(int(s), mu)
            np.testing.assert_allclose(A, ln.staple_from_plaquettes(Ut, Ns, Nt, int(s), mu), atol=1e-12)


@pytest.mark.parametrize("N,flux", [(2, 0), (2, 1), (3, 0), (3, 2)])
def test_staple_sum_rule(oracle_mod, N, flux):
    # every plaquette holds 4 links: sum_{x,mu} Re Tr(Ut A) = 4 * N * 6V * P
    Ns, Nt = 4, 4
    L = make(oracle_mod, N, Ns, Nt, 1.0, flux=flux, hot_seed=5)
    L.sweep(1, 0, 2)
    total = sum(L.link_action(s, mu) for s in range(L.V) for mu in range(4))
    P = L.measure()[0][0]
    assert abs(total - 24 * N * L.V * P) < 1e-9


@pytest.mark.parametrize("N,flux", [(2, 0), (2, 3), (3, 0), (3, 1)])
def test_overrelaxation_conserves_action(oracle_mod, N, flux):
    L = make(oracle_mod, N, 4, 4, 2.0 if N == 2 else 5.7, flux=flux, hot_seed=8)
    L.sweep(1, 0, 1)  # away from the hot start, then no reunitarization below
    for p in range(2):
        for mu in range(4):
            before = L.measure()[0][0]
            L.phase(oracle_mod.OVERRELAX, p, mu, 0)
            assert abs(L.measure()[0][0] - before) < 1e-13
    # link level: Re Tr(Ut A) is unchanged and the link moved
    U = L.get_links()
    for s, mu in [(0, 0), (5, 1), (17, 2), (40, 3)]:
        new, _ = L.link_update(oracle_mod.OVERRELAX, s, mu, 0)
        B = ln.background(N, 4, 4, flux, s, mu)
        A = L.staple(s, mu)
        assert abs(np.trace(new @ B @ A).real - L.link_action(s, mu)) < 1e-12
        assert np.abs(new - U[s, mu]).max() > 1e-6


def test_su2_heatbath_conditional_distribution(oracle_mod):
    """Repeated heat-bath draws of one y-link under a fixed staple follow
    sqrt(1-a0^2) exp(beta k a0) with a0 = Re Tr(Ut_new A) / (2k), and the
    remaining direction of Ut_new V is isotropic."""
    Ns, Nt, flux, beta = 4, 4, 1, 0.7
    L = make(oracle_mod, 2, Ns, Nt, beta, flux=flux, hot_seed=21)
    s, mu = ln.index(Ns, [3, 1, 2, 1]), 1
    A = L.staple(s, mu)
    k = np.sqrt(np.linalg.det(A).real)
    V = A / k
    B = ln.background(2, Ns, Nt, flux, s, mu)
    n = 40000
    a0 = np.empty(n)
    vec = np.empty((n, 3))
    for i in range(n):
        L.sweep_counter = i
        new, ex = L.link_update(oracle_mod.HEATBATH, s, mu, 99)
        assert ex == 0
        X = new @ B @ V
        a0[i] = np.trace(X).real / 2
        vec[i] = [X[0, 1].imag, X[0, 1].real, X[0, 0].imag]
    edges = np.linspace(-1, 1, 41)
    counts, _ = np.histogram(a0, bins=edges)
    assert chi2_pvalue(counts.astype(float), kp_bin_probs(beta * k, edges)) > 1e-3
    assert np.all(np.abs(vec.mean(0)) < 5 * np.sqrt(1 / 3 / n))


@pytest.mark.parametrize("N", [2, 3])
def test_heatbath_at_huge_beta_maximises_link_action(oracle_mod, N):
    # beta -> infinity: each (subgroup) draw tends to the maximiser R = V^+,
    # so the link action cannot go down (SU(2): reaches its maximum 2k).
    L = make(oracle_mod, N, 4, 2, 1e5, flux=2, hot_seed=4)
    for s, mu in [(1, 0), (6, 1), (9, 3), (30, 2)]:
        A = L.staple(s, mu)
        before = L.link_action(s, mu)
        new, _ = L.link_update(oracle_mod.HEATBATH, s, mu, 1)
        B = ln.background(N, 4, 2, 2, s, mu)
        after = np.trace(new @ B @ A).real
        assert after > before
        if N == 2:
            k = np.sqrt(np.linalg.det(A).real)
            assert abs(after - 2 * k) < 1e-3 * k


@pytest.mark.parametrize("N,flux", [(2, 0), (2, 1), (3, 0), (3, 2)])
def test_links_stay_in_group(oracle_mod, N, flux):
    L = make(oracle_mod, N, 4, 4, 2.3 if N == 2 else 5.7, flux=flux, hot_seed=6)
    e1, e2 = ln.unitarity_error(L.get_links())
    assert e1 < 1e-13 and e2 < 1e-13
    L.sweep(3, 4, 6)
    e1, e2 = ln.unitarity_error(L.get_links())
    assert e1 < 1e-12 and e2 < 1e-12


@pytest.mark.parametrize("N", [2, 3])
def test_reunitarization(oracle_mod, N):
    L = make(oracle_mod, N, 2, 2, 1.0, hot_seed=1)
    U = L.get_links()
    rng = np.random.default_rng(3)
    P = U + 1e-3 * (rng.normal(size=U.shape) + 1j * rng.normal(size=U.shape))
    if N == 2:  # keep the perturbation inside real multiples of SU(2)
        q0 = 0.5 * (P[..., 0, 0] + P[..., 1, 1]).real
        q3 = 0.5 * (P[..., 0, 0] - P[..., 1, 1]).imag
        q1 = 0.5 * (P[..., 0, 1] + P[..., 1, 0]).imag
        q2 = 0.5 * (P[..., 0, 1] - P[..., 1, 0]).real
        P = np.empty_like(U)
        P[..., 0, 0] = q0 + 1j * q3
        P[..., 0, 1] = q2 + 1j * q1
        P[..., 1, 0] = -q2 + 1j * q1
        P[..., 1, 1] = q0 - 1j * q3
    L.set_links(P)
    L.reunitarize()
    R = L.get_links()
    e1, e2 = ln.unitarity_error(R)
    assert e1 < 1e-14 and e2 < 1e-14
    if N == 2:
        nrm = np.sqrt(np.abs(P[..., 0, 0]) ** 2 + np.abs(P[..., 0, 1]) ** 2)
        np.testing.assert_allclose(R, P / nrm[..., None, None], atol=1e-15)
    else:
        # row 1 keeps its direction; row 2 stays in span(row1, row2)
        r1 = P[..., 0, :] / np.linalg.norm(P[..., 0, :], axis=-1, keepdims=True)
        np.testing.assert_allclose(R[..., 0, :], r1, atol=1e-15)
        for s in range(R.shape[0]):
            for mu in range(4):
                Mt = np.stack([P[s, mu, 0], P[s, mu, 1]], axis=1)
                c, *_ = np.linalg.lstsq(Mt, R[s, mu, 1], rcond=None)
                assert np.abs(Mt @ c - R[s, mu, 1]).max() < 1e-14


@pytest.mark.parametrize("N", [2, 3])
def test_background_field_is_a_change_of_variables(oracle_mod, N):
    """Effective links absorb a fixed per-link phase: starting the field-n run
    from U0 = W0 B^+ and the field-free run from W0, with one seed, the
    field-n effective links equal the field-free links after any number of
    sweeps."""
    Ns, Nt, n, beta = 4, 4, 3, 2.3 if N == 2 else 5.7
    A = make(oracle_mod, N, Ns, Nt, beta, flux=0, hot_seed=17)
    W0 = A.get_links()
    Bl = make(oracle_mod, N, Ns, Nt, beta, flux=n)
    U0 = W0.copy()
    for s in range(A.V):
        U0[s, 1] = W0[s, 1] @ ln.background(N, Ns, Nt, n, s, 1).conj().T
    Bl.set_links(U0)
    # The two chains differ only by rounding (W B^+ B != W in floating point),
    # and the chain is chaotic: the difference grows by a bounded factor per
    # sweep.  Measured on this case (sweeps of HB + 2 OR): the largest
    # difference after sweeps 1..4 is 4e-14, 1.6e-12, 1.6e-11, 1.9e-10 for
    # SU(2) (x10..40 per sweep) and 3.5e-12, 2.3e-10, 1.2e-8, 3.4e-7 for SU(3)
    # (x28..66).  The bound below allows 1e-11 after one sweep and a factor 200
    # per further sweep; a real inconsistency (a phase on the wrong side, a
    # dropped B) is O(1) after the first sweep.
    dev = []
    for k in range(4):
        A.sweep(1, 2, 55)
        Bl.sweep(1, 2, 55)
        W = A.get_links()
        Wt = ln.effective(Bl.get_links(), Ns, Nt, n)
        dev.append(np.abs(W - Wt).max())
        assert dev[-1] < 1e-11 * 200.0 ** k, dev
    assert all(b < 200.0 * max(a, 1e-15) for a, b in zip(dev, dev[1:])), dev
    pa, la = A.measure()
    pb, lb = Bl.measure()
    np.testing.assert_allclose(pa, pb, atol=10 * dev[-1])
    np.testing.assert_allclose(la, lb, atol=10 * dev[-1])
    assert abs(Bl.measure_bare()[1] - pb[1]) > 1e-3  # the bare links see the field


@pytest.mark.parametrize("N", [2, 3])
def test_beta_zero_gives_haar_links(oracle_mod, N):
    Ns, Nt = 4, 4
    L = make(oracle_mod, N, Ns, Nt, 0.0)
    vals, polys = [], []
    for i in range(8):
        L.sweep(1, 0, 123)
        p, l = L.measure()
        vals.append(p[0])
        polys.append(l[0])
    U = L.get_links().reshape(-1, N, N)
    tr = np.trace(U, axis1=1, axis2=2)
    n = len(tr)
    sigma_plaq = np.sqrt(1.0 / N ** 2 / (6 * L.V))  # Var(Re Tr U_P / N) <= 1/N^2
    assert abs(np.mean(vals)) < 5 * sigma_plaq / np.sqrt(len(vals))
    assert abs(np.mean(polys)) < 5 * np.sqrt(1.0 / Ns ** 3 / len(polys))
    assert abs((np.abs(tr) ** 2).mean() - 1.0) < 5 * np.sqrt(2.0 / n)


def test_nhit_exhaustion_keeps_link(oracle_mod):
    L = make(oracle_mod, 2, 4, 2, 0.05, nhit=1, hot_seed=2)
    U = L.get_links()
    kept = moved = 0
    for s in range(L.V):
        new, ex = L.link_update(oracle_mod.HEATBATH, s, 0, 3)
        if ex:
            kept += 1
            assert np.array_equal(new, U[s, 0])
        else:
            moved += 1
            assert np.abs(new - U[s, 0]).max() > 0
    assert kept > 0 and moved > 0
    L.sweep(1, 0, 3)
    assert L.exhausted > 0


def test_results_do_not_depend_on_thread_count(oracle_mod):
    out = []
    for threads in (1, 3):
        oracle_mod.set_threads(threads)
        L = make(oracle_mod, 3, 4, 4, 5.7, flux=1, hot_seed=9)
        L.sweep(2, 2, 10)
        out.append(L.get_links())
    oracle_mod.set_threads(0)
    assert np.array_equal(out[0], out[1])


def test_sweep_counter_and_seed(oracle_mod):
    A = make(oracle_mod, 2, 4, 2, 2.3, hot_seed=1)
    B = make(oracle_mod, 2, 4, 2, 2.3, hot_seed=1)
    A.sweep(2, 1, 7)
    B.sweep(1, 1, 7)
    B.sweep(1, 1, 7)
    assert A.sweep_counter == 2 and B.sweep_counter == 2
    assert np.array_equal(A.get_links(), B.get_links())
    C = make(oracle_mod, 2, 4, 2, 2.3, hot_seed=1)
    C.sweep(2, 1, 8)
    assert not np.array_equal(A.get_links(), C.get_links())
    D = make(oracle_mod, 2, 4, 2, 2.3, hot_seed=1, lid=1)
    D.sweep(2, 1, 7)
    assert not np.array_equal(A.get_links(), D.get_links())


def perturbed(U, rng, N):
    """Links pushed about 1e-3 off the group (for SU(2): real multiples of
    SU(2) matrices, the form the SU(2) projection keeps)."""
    P = U + 1e-3 * (rng.normal(size=U.shape) + 1j * rng.normal(size=U.shape))
    if N == 2:
        q0 = 0.5 * (P[..., 0, 0] + P[..., 1, 1]).real
        q3 = 0.5 * (P[..., 0, 0] - P[..., 1, 1]).imag
        q1 = 0.5 * (P[..., 0, 1] + P[..., 1, 0]).imag
        q2 = 0.5 * (P[..., 0, 1] - P[..., 1, 0]).real
        P = np.empty_like(U)
        P[..., 0, 0] = q0 + 1j * q3
        P[..., 0, 1] = q2 + 1j * q1
        P[..., 1, 0] = -q2 + 1j * q1
        P[..., 1, 1] = q0 - 1j * q3
    return P


def check_gram_schmidt(P, R):
    """R is the Gram-Schmidt reunitarization of P, by the properties that fix
    it: unitary with det 1, its first row a positive multiple of P's first
    row, its second row in span(P's rows 1, 2) with a positive real overlap
    with P's second row (for SU(2), R = P / |first row|)."""
    N = P.shape[-1]
    M = R.reshape(-1, N, N)
    assert np.abs(np.einsum("nki,nkj->nij", M.conj(), M) - np.eye(N)).max() < 1e-14
    assert np.abs(np.linalg.det(M) - 1.0).max() < 1e-14
    Pm = P.reshape(-1, N, N)
    if N == 2:
        nrm = np.linalg.norm(Pm[:, 0, :], axis=-1)
        np.testing.assert_allclose(M, Pm / nrm[:, None, None], rtol=0, atol=1e-15)
        return
    r1 = Pm[:, 0, :] / np.linalg.norm(Pm[:, 0, :], axis=-1, keepdims=True)
    np.testing.assert_allclose(M[:, 0, :], r1, rtol=0, atol=1e-15)
    for k in range(M.shape[0]):
        basis = np.stack([Pm[k, 0], Pm[k, 1]], axis=1)
        c, *_ = np.linalg.lstsq(basis, M[k, 1], rcond=None)
        assert np.abs(basis @ c - M[k, 1]).max() < 1e-14
        ov = np.vdot(Pm[k, 1], M[k, 1])
        assert abs(ov.imag) < 1e-14 and ov.real > 0


@pytest.mark.parametrize("N", [2, 3])
def test_reunitarize_matrix_is_gram_schmidt(oracle_mod, N):
    L = make(oracle_mod, N, 2, 2, 1.0, hot_seed=4)
    P = perturbed(L.get_links()[:6], np.random.default_rng(8), N)
    R = np.stack([[oracle_mod.reunitarize_matrix(P[s, mu]) for mu in range(4)] for s in range(P.shape[0])])
    check_gram_schmidt(P, R)


@pytest.mark.parametrize("N", [2, 3])
@pytest.mark.parametrize("mode", [0, 1])
def test_reunitarize_phase_touches_only_its_links(oracle_mod, N, mode):
    """Reunitarization of the links of one checkerboard phase, as a sweep's
    last overrelaxation pass applies it link by link: those links become the
    Gram-Schmidt projections of their values, every other link (and a frozen
    link of the phase) keeps its bits."""
    Ns, Nt = 4, 2
    L = oracle_mod.OracleLattice(N, Ns, Nt, 2.0, 1, 10, 0, mode)
    L.hot_start(3)
    P = perturbed(L.get_links(), np.random.default_rng(9), N)
    L.set_links(P)
    parity, mu = 1, 2
    L.reunitarize_phase(parity, mu)
    R = L.get_links()
    c = ln.coords(Ns, Nt, np.arange(L.V))
    on = ((c[0] + c[1] + c[2] + c[3]) % 2 == parity)
    frozen = (c[3] == 0) if mode == 1 else np.zeros(L.V, bool)
    sel = on & ~frozen
    check_gram_schmidt(P[sel, mu], R[sel, mu])
    keep = np.ones((L.V, 4), bool)
    keep[sel, mu] = False
    assert np.array_equal(R[keep], P[keep])


@pytest.mark.parametrize("N,Ns,Nt,flux,flux8", [(2, 4, 2, 1, 0), (3, 2, 4, 1, 0), (3, 4, 2, 3, 1)])
def test_measure_planes_matches_brute_force(oracle_mod, N, Ns, Nt, flux, flux8):
    L = oracle_mod.OracleLattice(N, Ns, Nt, 2.0, flux, 10, 0, 0, flux8)
    L.hot_start(12)
    L.sweep(1, 1, 12)
    Ut = ln.effective(L.get_links(), Ns, Nt, flux, flux8)
    planes = [(0, 1), (0, 2), (1, 2), (0, 3), (1, 3), (2, 3)]
    ref = [np.mean([ln.plaquette_value(Ut, Ns, Nt, s, m, n) for s in range(L.V)]) for m, n in planes]
    np.testing.assert_allclose(L.measure_planes(), ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("N", [2, 3])
def test_measure_planes_cold_start_closed_form(oracle_mod, N):
    """Cold start with a field: only the (x, y) plane sees it, with the value
    of the flux closed form; every other plane is 1."""
    Ns, n = 6, 2
    L = make(oracle_mod, N, Ns, 2, 6.0, flux=n)
    xy = 3 * flux_closed_form(N, Ns, n)[1] - 2.0
    np.testing.assert_allclose(L.measure_planes(), [xy, 1, 1, 1, 1, 1], rtol=0, atol=1e-14)


def su3_class_moments(b, n=192):
    """<t> and <t^2>, t = (1/3) Re Tr U, under exp(b Re Tr U) on SU(3), by the
    Weyl integration formula over the eigenphases (th1, th2, -th1-th2)."""
    th = 2 * np.pi * np.arange(n) / n
    t1, t2 = np.meshgrid(th, th, indexing="ij")
    t3 = -t1 - t2
    tr = (np.exp(1j * t1) + np.exp(1j * t2) + np.exp(1j * t3)).real
    vdm = (np.abs(np.exp(1j * t1) - np.exp(1j * t2)) ** 2
           * np.abs(np.exp(1j * t1) - np.exp(1j * t3)) ** 2
           * np.abs(np.exp(1j * t2) - np.exp(1j * t3)) ** 2)
    w = vdm * np.exp(b * tr)
    t = tr / 3
    return float((w * t).sum() / w.sum()), float((w * t * t).sum() / w.sum())


@pytest.mark.parametrize("beta", [0.4, 1.0])
def test_su3_heatbath_conditional_distribution(oracle_mod, beta):
    """Cabibbo-Marinari heat-bath of one link under a fixed staple A = 6 (all
    other links the unit matrix): applied over and over, its link must follow
    exp((beta/3) Re Tr(U A)) = exp(2 beta Re Tr U), a class function, so the
    first two moments of (1/3) Re Tr U are Weyl integrals.  A wrong subgroup
    coupling (alpha = 2 beta k / 3), embedding or rotation order moves them."""
    Ns, Nt = 4, 2
    L = make(oracle_mod, 3, Ns, Nt, beta, nhit=1000)
    s, mu = ln.index(Ns, [1, 2, 3, 1]), 2
    np.testing.assert_allclose(L.staple(s, mu), 6 * np.eye(3), atol=1e-14)
    U = L.get_links()
    n_therm, n = 200, 12000
    t = np.empty(n)
    for i in range(n_therm + n):
        L.sweep_counter = i
        new, ex = L.link_update(oracle_mod.HEATBATH, s, mu, 31)
        assert ex == 0
        U[s, mu] = new
        L.set_links(U)
        if i >= n_therm:
            t[i - n_therm] = np.trace(new).real / 3
    m1, m2 = su3_class_moments(2 * beta)
    for x, ref in ((t, m1), (t * t, m2)):
        nb = 60
        b = x[: len(x) // nb * nb].reshape(nb, -1).mean(1)
        err = b.std(ddof=1) / np.sqrt(nb)
        assert abs(b.mean() - ref) < 4 * err, (b.mean(), ref, err)
