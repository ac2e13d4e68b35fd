"""Host-side run statistics (paper_1310_7087_gb300.analysis): the integrated
autocorrelation time and the error of a correlated mean, against the closed
forms of a first-order autoregressive series x_i = a x_{i-1} + e_i, whose
autocorrelation is rho(k) = a^k, so tau = (1 + a) / (2 (1 - a)) and the
variance of the mean of n terms tends to 2 tau var / n."""
import numpy as np
import pytest

from paper_1310_7087_gb300 import analysis


def ar1(a, n, seed):
    rng = np.random.default_rng(seed)
    e = rng.normal(size=n)
    x = np.empty(n)
    x[0] = e[0] / np.sqrt(1 - a * a)
    for i in range(1, n):
        x[i] = a * x[i - 1] + e[i]
    return x


@pytest.mark.parametrize("a", [0.0, 0.5, 0.9])
def test_tau_int_matches_the_ar1_closed_form(a):
    x = ar1(a, 100000, 3)
    tau = (1 + a) / (2 * (1 - a))
    assert abs(analysis.tau_int(x) - tau) < 0.1 * tau


def test_error_of_a_correlated_mean_covers_the_scatter_of_means():
    a, n = 0.9, 2000
    means, errs = [], []
    for seed in range(200):
        m, e, _ = analysis.mean_error(ar1(a, n, seed))
        means.append(m)
        errs.append(e)
    # the scatter of the 200 means is what the error claims, to ~15 %
    assert 0.8 < np.std(means) / np.mean(errs) < 1.25
    # plain binning with bins shorter than tau would claim a smaller error
    _, eb = analysis.binned(ar1(a, n, 0), 2)
    assert eb < 0.6 * np.mean(errs)


def test_binned_mean():
    x = np.repeat([1.0, 3.0], 10)
    assert analysis.binned(x, 10) == (2.0, 1.0)
    with pytest.raises(ValueError):
        analysis.binned(x, 15)
