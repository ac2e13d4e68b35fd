"""The flux scan of the SU(3) 32^3 x 8 workload: beta = 6.0, background field
along lambda3 with flux quantum n in {0, 1, 2, 4}, hot start, 500 working
sweeps of 1 heat-bath + 4 overrelaxation passes, FP32-compressed links,
P, P_s, P_t and the Polyakov loop after every sweep.

In the effective-link mode the field is a change of variables (the action and
every update use U B with B a fixed unitary per link, and Haar measure does not
see a fixed right factor), so:
  (i)  a run at flux n started from W0 B^+ is the n = 0 run started from W0:
       with FP64 storage its effective links equal the n = 0 links after one
       sweep to rounding (1e-8; every overrelaxation pass multiplies rounding
       differences, a second sweep already takes them to 1e-5 at this size);
  (ii) the effective-link <P>, <P_s>, <P_t>, <Re L> and <|L|> do not depend on
       n: every n agrees with n = 0 within 3 sigma.  beta = 6.0 lies just
       below the Nt = 8 deconfinement transition, where the Polyakov loop
       drifts slowly between the Z3 sectors, so the scan runs 2000 sweeps
       (100 of thermalization) rather than the workload's 500 and takes its
       errors from the integrated autocorrelation time (automatic window):
       500 sweeps with errors from bins of 20 sweeps put <Re L> of n = 0 and
       n = 1 4.4 "sigma" apart, an artefact of the underestimated error;
  (iii) the bare-link spatial plaquette does see the field: on every
       configuration of the n = 0 chain it equals the effective one exactly,
       and for n >= 1 their difference, averaged over the chain, is nonzero
       by more than 5 sigma (and grows with n).
"""
import numpy as np
import pytest

import workloads
from workloads import FP64_PLAIN, HOT

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


def background_y(Ns, Nt, n):
    """diag(B_y(x)) for every site, lambda3 direction: phases (+phi, -phi, 0),
    phi = 2 pi n x / Ns^2."""
    x = np.arange(Ns ** 3 * Nt) % Ns
    phi = 2 * np.pi * n * x / Ns ** 2
    return np.stack([np.exp(1j * phi), np.exp(-1j * phi), np.ones_like(phi, dtype=complex)], axis=-1)


def test_change_of_variables_on_the_gpu(q):
    w = workloads.SU3_32x8[0]
    a = q.Lattice(3, w.Ns, w.Nt, w.beta, 0, FP64_PLAIN, HOT, w.seed)
    W0 = a.get_links()
    for n in (1, 4):
        b = q.Lattice(3, w.Ns, w.Nt, w.beta, n, FP64_PLAIN, HOT, w.seed)
        U0 = W0.copy()
        U0[:, 1] = W0[:, 1] * np.conj(background_y(w.Ns, w.Nt, n))[:, None, :]  # W0 B^+
        b.set_links(U0)
        a.set_links(W0)
        a.sweep_counter = 0
        a.sweep(1, 4, w.seed)
        b.sweep(1, 4, w.seed)
        Wa = a.get_links()
        Ut = b.get_links()
        Ut[:, 1] = Ut[:, 1] * background_y(w.Ns, w.Nt, n)[:, None, :]  # U B
        dev = np.abs(Wa - Ut).max()
        print("n = %d: largest effective-link difference after one sweep %.3g" % (n, dev))
        assert dev < 1e-8
        (pa, la), (pb, lb) = a.measure(), b.measure()
        np.testing.assert_allclose(pb, pa, rtol=0, atol=1e-10)
        np.testing.assert_allclose(lb, la, rtol=0, atol=1e-10)
        b.close()
    a.close()


@pytest.fixture(scope="module")
def scan(q):
    from paper_1310_7087_gb300 import analysis
    w = workloads.SU3_32x8[0]
    return analysis.flux_scan(q, [v.flux for v in workloads.SU3_32x8], w.Ns, w.Nt, w.beta, 2000,
                              n_or=w.n_or, seed=w.seed, n_therm=100, bare_every=5)


@pytest.mark.parametrize("name", ["P", "P_s", "P_t", "Re L", "|L|"])
def test_effective_observables_do_not_depend_on_flux(scan, name):
    m0, e0, t0 = scan[0][name]
    for n in (1, 2, 4):
        m, e, t = scan[n][name]
        z = abs(m - m0) / np.hypot(e, e0)
        print("%s: n = %d %.6f +- %.6f (tau %.1f), n = 0 %.6f +- %.6f (tau %.1f): %.2f sigma"
              % (name, n, m, e, t, m0, e0, t0, z))
        assert z < 3.0, (name, n, m, e, m0, e0)


def test_bare_spatial_plaquette_sees_the_field(scan):
    assert scan[0]["P_s bare - P_s"][:2] == (0.0, 0.0)  # n = 0: no field, bare = effective
    shift = []
    for n in (1, 2, 4):
        m, e, _ = scan[n]["P_s bare - P_s"]
        mb, eb, _ = scan[n]["P_s bare"]
        print("bare P_s - P_s: n = %d %.3g +- %.2g (%.1f sigma); bare P_s %.6f +- %.6f"
              % (n, m, e, abs(m) / e, mb, eb))
        assert abs(m) > 5.0 * e, (n, m, e)
        shift.append(abs(m))
    assert shift[0] < shift[1] < shift[2], shift
