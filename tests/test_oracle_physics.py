"""Ensemble pins for the oracle's Markov chain: strong-coupling and
weak-coupling limits of the average plaquette, computed independently of the
oracle (Bessel functions, the SU(3) Weyl integral, equipartition)."""
import numpy as np
import pytest
from scipy.special import iv


def binned_mean(x, bin_size=20):
    x = np.asarray(x)
    nb = len(x) // bin_size
    b = x[: nb * bin_size].reshape(nb, bin_size).mean(1)
    return b.mean(), b.std(ddof=1) / np.sqrt(nb)


def su2_strong_coupling(beta):
    """Single-plaquette <(1/2) Tr U> under exp((beta/2) Re Tr U) on SU(2)."""
    return iv(2, beta) / iv(1, beta)


def su3_single_plaquette(beta, n=256):
    """<(1/3) Re Tr U> under exp((beta/3) Re Tr U) on SU(3), by the Weyl
    integration formula over eigenphases (th1, th2, -th1-th2); the periodic
    trapezoid rule converges exponentially."""
    th = 2 * np.pi * np.arange(n) / n
    t1, t2 = np.meshgrid(th, th, indexing="ij")
    t3 = -t1 - t2
    tr = np.exp(1j * t1) + np.exp(1j * t2) + np.exp(1j * t3)
    vdm = (np.abs(np.exp(1j * t1) - np.exp(1j * t2)) ** 2
           * np.abs(np.exp(1j * t1) - np.exp(1j * t3)) ** 2
           * np.abs(np.exp(1j * t2) - np.exp(1j * t3)) ** 2)
    w = vdm * np.exp(beta / 3 * tr.real)
    return float((w * tr.real / 3).sum() / w.sum())


def run_chain(oracle_mod, N, Ns, Nt, beta, n_or, therm, meas, seed):
    L = oracle_mod.OracleLattice(N, Ns, Nt, beta, 0, 10, 0)
    L.hot_start(seed)
    L.sweep(therm, n_or, seed)
    vals = []
    for _ in range(meas):
        L.sweep(1, n_or, seed)
        vals.append(L.measure()[0][0])
    return vals


def test_weyl_integral_small_beta():
    # leading order of the character expansion: beta / 18
    assert abs(su3_single_plaquette(1e-3) - 1e-3 / 18) < 1e-8


@pytest.mark.parametrize("beta", [0.5])
def test_su2_strong_coupling(oracle_mod, beta):
    vals = run_chain(oracle_mod, 2, 4, 4, beta, 1, 20, 2000, 2024)
    m, e = binned_mean(vals)
    u = su2_strong_coupling(beta)
    assert abs(m - u) < 4 * e + 10 * u ** 5, (m, e, u)


@pytest.mark.parametrize("beta", [1.0])
def test_su3_strong_coupling(oracle_mod, beta):
    vals = run_chain(oracle_mod, 3, 4, 4, beta, 1, 20, 1000, 2025)
    m, e = binned_mean(vals)
    u = su3_single_plaquette(beta)
    assert abs(m - u) < 4 * e + 10 * u ** 5, (m, e, u)


@pytest.mark.parametrize("N,beta", [(2, 50.0), (3, 100.0)])
def test_weak_coupling_equipartition(oracle_mod, N, beta):
    # 3V(N^2-1) physical quadratic modes, each <beta * ...> = 1/2:
    # 1 - <P> -> (N^2 - 1) / (4 beta)
    L = oracle_mod.OracleLattice(N, 4, 4, beta, 0, 10, 0)
    L.sweep(30, 1, 77)
    vals = []
    for _ in range(200 if N == 2 else 60):
        L.sweep(1, 1, 77)
        vals.append(1.0 - L.measure()[0][0])
    m, e = binned_mean(vals, 10)
    target = (N * N - 1) / (4 * beta)
    assert abs(m / target - 1.0) < 0.05, (m, target)
