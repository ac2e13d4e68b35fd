"""Pins for the oracle's random group elements: the Kennedy-Pendleton sampler
against its target density, direction isotropy, and Haar moments of the SU(2)
and SU(3) generators."""
import numpy as np
import pytest
from scipy import integrate, stats
from scipy.special import gamma as gamma_fn


def kp_bin_probs(alpha, edges):
    """Bin probabilities of sqrt(1-a^2) exp(alpha a) on [-1, 1] (scaled by
    exp(-alpha) to avoid overflow)."""
    f = lambda a: np.sqrt(max(0.0, 1.0 - a * a)) * np.exp(alpha * (a - 1.0))
    p = np.array([integrate.quad(f, lo, hi, epsabs=0, epsrel=1e-10)[0]
                  for lo, hi in zip(edges[:-1], edges[1:])])
    return p / p.sum()


def chi2_pvalue(counts, probs, min_expected=5.0):
    n = counts.sum()
    exp = probs * n
    # merge sparse bins from the left into their neighbour
    obs_m, exp_m, co, ce = [], [], 0.0, 0.0
    for o, e in zip(counts, exp):
        co += o
        ce += e
        if ce >= min_expected:
            obs_m.append(co)
            exp_m.append(ce)
            co, ce = 0.0, 0.0
    if ce > 0:
        obs_m[-1] += co
        exp_m[-1] += ce
    obs_m, exp_m = np.array(obs_m), np.array(exp_m)
    chi2 = ((obs_m - exp_m) ** 2 / exp_m).sum()
    return stats.chi2.sf(chi2, len(obs_m) - 1)


@pytest.mark.parametrize("alpha", [0.5, 1.0, 2.3, 5.0, 20.0])
def test_kp_density_chi_square(oracle_mod, alpha):
    n = 1_000_000
    a0, tries = oracle_mod.kp_samples(alpha, 1_000_000, seed=12345 + int(alpha * 10), n=n)
    assert (tries > 0).all()
    assert a0.min() >= -1.0 and a0.max() < 1.0
    edges = np.linspace(-1.0, 1.0, 51)
    counts, _ = np.histogram(a0, bins=edges)
    p = chi2_pvalue(counts.astype(float), kp_bin_probs(alpha, edges))
    assert p > 1e-3, p


def kp_acceptance(alpha):
    """Acceptance of one Kennedy-Pendleton try: delta ~ Gamma(3/2, 1/alpha)
    accepted with probability sqrt(1 - delta/2) on [0, 2]."""
    g = lambda d: alpha ** 1.5 * np.sqrt(d) * np.exp(-alpha * d) / gamma_fn(1.5)
    return integrate.quad(lambda d: g(d) * np.sqrt(1.0 - d / 2.0), 0.0, 2.0)[0]


@pytest.mark.parametrize("alpha", [0.5, 2.3, 8.0])
def test_kp_single_try_acceptance(oracle_mod, alpha):
    n = 400_000
    _, tries = oracle_mod.kp_samples(alpha, 1, seed=777, n=n)
    acc = (tries == 1).mean()
    p = kp_acceptance(alpha)
    assert abs(acc - p) < 5 * np.sqrt(p * (1 - p) / n), (acc, p)


def test_kp_tries_geometric(oracle_mod):
    alpha, n = 1.0, 300_000
    _, tries = oracle_mod.kp_samples(alpha, 1000, seed=99, n=n)
    p = kp_acceptance(alpha)
    assert abs(tries.mean() - 1.0 / p) < 5 * np.sqrt((1 - p) / p ** 2 / n)


def test_su2_direction_isotropy(oracle_mod):
    x = oracle_mod.su2_samples(2.3, 1_000_000, seed=4242, n=400_000)
    assert np.allclose((x ** 2).sum(1), 1.0, atol=1e-12)
    a = x[:, 1:]
    n = len(x)
    assert np.all(np.abs(a.mean(0)) < 5 * np.sqrt(1 / 3 / n))
    target = (1.0 - (x[:, 0] ** 2).mean()) / 3.0
    second = (a ** 2).mean(0)
    assert np.all(np.abs(second - target) < 5 * np.sqrt(2 * target ** 2 / n) + 1e-4)
    cross = np.array([(a[:, i] * a[:, j]).mean() for i, j in ((0, 1), (0, 2), (1, 2))])
    assert np.all(np.abs(cross) < 5 * target / np.sqrt(n) * 2)
    # the a0 marginal is the Kennedy-Pendleton target
    edges = np.linspace(-1.0, 1.0, 41)
    counts, _ = np.histogram(x[:, 0], bins=edges)
    assert chi2_pvalue(counts.astype(float), kp_bin_probs(2.3, edges)) > 1e-3


def test_su2_alpha_zero_is_haar(oracle_mod):
    # alpha = 0 -> uniform on S^3: E x_i^2 = 1/4, E x_i^4 = 1/8
    x = oracle_mod.su2_samples(0.0, 10, seed=5, n=400_000)
    n = len(x)
    assert np.allclose((x ** 2).sum(1), 1.0, atol=1e-12)
    assert np.all(np.abs((x ** 2).mean(0) - 0.25) < 5 * np.sqrt(0.0625 / n) * 1.5)
    assert np.all(np.abs((x ** 4).mean(0) - 0.125) < 0.003)
    # marginal of x0: (2/pi) sqrt(1 - x0^2)
    edges = np.linspace(-1.0, 1.0, 41)
    counts, _ = np.histogram(x[:, 0], bins=edges)
    assert chi2_pvalue(counts.astype(float), kp_bin_probs(0.0, edges)) > 1e-3


@pytest.mark.parametrize("N", [2, 3])
def test_haar_generator(oracle_mod, N):
    n = 200_000
    U = oracle_mod.haar_samples(N, seed=31337, n=n)
    eye = np.eye(N)
    err = np.abs(np.einsum("nki,nkj->nij", U.conj(), U) - eye).max()
    assert err < 1e-12
    assert np.abs(np.linalg.det(U) - 1.0).max() < 1e-12
    tr = np.trace(U, axis1=1, axis2=2)
    sig = lambda m: 5 * np.sqrt(m / n)
    assert abs(tr.mean()) < sig(1.0)
    assert abs((np.abs(tr) ** 2).mean() - 1.0) < sig(2.0)
    assert abs((np.abs(tr) ** 4).mean() - 2.0) < sig(20.0)
    third = (tr ** 3).mean()
    # SU(3): one singlet in 3 x 3 x 3 -> E (Tr U)^3 = 1; SU(2): odd moment 0
    expect = 1.0 if N == 3 else 0.0
    assert abs(third - expect) < sig(8.0), third
