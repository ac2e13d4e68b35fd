"""Run statistics and the background-field flux scan, on top of the C ABI.

The paper's data-analysis block (sec. 3.1) turns the measurements of a run
into averages with errors; its physics runs scan the flux of the external
chromomagnetic field (abstract, sec. 1).  This module is host-side
bookkeeping only: every sweep and every measurement runs in the library's
kernels, and numpy only averages the numbers they return.
"""
from __future__ import annotations

import time

import numpy as np


def binned(x, bin_size: int):
    """Mean of a Monte Carlo series and its error from the scatter of the
    means of consecutive bins of ``bin_size`` measurements (bins longer than
    the autocorrelation time make the bin means independent)."""
    x = np.asarray(x, dtype=np.float64)
    n = len(x) // bin_size
    if n < 2:
        raise ValueError("need at least two bins")
    m = x[: n * bin_size].reshape(n, bin_size).mean(axis=1)
    return float(m.mean()), float(m.std(ddof=1) / np.sqrt(n))


def tau_int(x, c: float = 6.0) -> float:
    """Integrated autocorrelation time of a Monte Carlo series, in units of
    its spacing, with the automatic window of Madras and Sokal (J. Stat. Phys.
    50 (1988) 109): tau(W) = 1/2 + sum_{k=1..W} rho(k), W the smallest window
    with W >= c tau(W)."""
    x = np.asarray(x, dtype=np.float64)
    n = len(x)
    d = x - x.mean()
    var = float(d @ d) / n
    if n < 4 or var == 0.0:
        return 0.5
    f = np.fft.rfft(d, 2 * n)
    acov = np.fft.irfft(f * np.conj(f))[:n] / np.arange(n, 0, -1)
    rho = acov / acov[0]
    tau = 0.5
    for w in range(1, n // 2):
        tau += rho[w]
        if w >= c * tau:
            break
    return float(max(tau, 0.5))


def mean_error(x, c: float = 6.0):
    """(mean, error, tau): the error of the mean of a correlated series,
    sqrt(2 tau var / n) with tau from tau_int."""
    x = np.asarray(x, dtype=np.float64)
    tau = tau_int(x, c)
    return float(x.mean()), float(np.sqrt(2.0 * tau * x.var() / len(x))), tau


def flux_scan(q, fluxes, Ns, Nt, beta, n_sweeps, n_or=4, seed=1, n_therm=100, field_mode=0,
              bare_every=1, stream=None):
    """One SU(3) FP32 chain per flux quantum n: ``n_sweeps`` working sweeps
    (1 heat-bath + n_or overrelaxation passes + reunitarization +
    measurement) from a hot start, the first ``n_therm`` discarded.

    Returns {n: stats}, stats holding (mean, error, tau) of P, P_s, P_t,
    Re L and |L| (errors from the integrated autocorrelation time, which near
    a deconfinement transition is long for the Polyakov loop) on the links
    the action uses (in the effective-link mode U B, a change
    of variables of the n = 0 theory), of the bare-link P_s (U alone, measured
    every ``bare_every`` sweeps) and of its difference from P_s on the same
    configuration (the field's imprint, free of most of the configuration
    noise), the per-sweep series, and the working-sweep rate in link updates
    per second (wall clock, measurements included)."""
    out = {}
    lu = (1 + n_or) * 4 * Ns ** 3 * Nt
    for n in fluxes:
        lat = q.Lattice(3, Ns, Nt, beta, n, q.QCD_FP32_COMPRESSED, q.QCD_HOT, seed, stream,
                        field_mode=field_mode)
        series = np.zeros((n_sweeps, 5))
        bare, diff = [], []
        t0 = time.perf_counter()
        for i in range(n_sweeps):
            series[i] = q.qcd_working_sweep(lat.h, 1, n_or, seed)
            if i >= n_therm and (i - n_therm) % bare_every == 0:
                bare.append(q.qcd_measure_bare(lat.h)[1])
                diff.append(bare[-1] - q.qcd_measure(lat.h)[0][1])  # same kernel, effective links
        wall = time.perf_counter() - t0
        lat.close()
        meas = series[n_therm:]
        stats = {name: mean_error(col) for name, col in
                 (("P", meas[:, 0]), ("P_s", meas[:, 1]), ("P_t", meas[:, 2]), ("Re L", meas[:, 3]),
                  ("|L|", np.hypot(meas[:, 3], meas[:, 4])))}
        stats["P_s bare"] = mean_error(bare)
        stats["P_s bare - P_s"] = mean_error(diff)
        stats["series"] = series
        stats["lu_per_s_wall"] = lu * n_sweeps / wall
        out[n] = stats
    return out
