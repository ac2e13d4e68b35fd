"""The FP32 reading of the one-sweep link bar, pinned on the oracle alone.

The bar: after one sweep from the same start at least 99.99 % of the links
agree with the FP64 oracle within 1e-5.  With FP32-compressed storage the
start itself is the FP64 start rounded to the storage (rows 1-2 of each
SU(3) link to FP32, row 3 rebuilt), and the sweep of the SU(3) 16^3 x 4,
beta = 5.7 workload (hot start, seed 7; one heat-bath pass and four
overrelaxation passes) amplifies that rounding: each overrelaxation pass
multiplies a perturbation by about ten, because every phase reflects links
about staples that the earlier phases of the pass have just changed.  The
oracle run twice, once from the FP64 start and once from its FP32 rounding,
with no other difference and exact FP64 arithmetic in both, ends the sweep
with every link beyond 1e-5 (median 2.4e-3).  So no FP32 implementation can
meet the link bar on this sweep; the FP32 GPU path is held instead to
  - the bar kernel by kernel (each kernel from the state the GPU left),
  - the bar on a heat-bath-only sweep, where the oracle's own divergence
    stays below 1e-5,
  - the oracle's own divergence on the full sweep, within a stated factor
    (tests/test_gpu_fp32_sweep.py),
  - the total plaquette after the full sweep within 1e-6 of the FP64 run:
    overrelaxation conserves the action exactly, so the chains' plaquettes
    stay together (6e-11 apart here) while P_s and P_t move apart (2e-5).
These tests measure all of that on the oracle.
"""
import numpy as np
import pytest

import lattice_np as ln

NS, NT, BETA, SEED = 16, 4, 5.7, 7


def link_err(a, b):
    return np.abs(a - b).reshape(a.shape[0] * 4, -1).max(axis=1)


@pytest.fixture(scope="module")
def runs(oracle_mod):
    """For n_or = 0, 1, 4: the oracle's sweep (1 HB + n_or OR +
    reunitarization) from the FP64 hot start and from its FP32 rounding."""
    A = oracle_mod.OracleLattice(3, NS, NT, BETA, 0, 10, 0)
    A.hot_start(SEED)
    S64 = A.get_links()
    S32 = ln.round_to_fp32_storage(S64)
    B = oracle_mod.OracleLattice(3, NS, NT, BETA, 0, 10, 0)
    out = {}
    for n_or in (0, 1, 4):
        A.set_links(S64)
        A.sweep_counter = 0
        B.set_links(S32)
        B.sweep_counter = 0
        A.sweep(1, n_or, SEED)
        B.sweep(1, n_or, SEED)
        out[n_or] = (A.get_links(), B.get_links(), A.measure(), B.measure())
    A.close()
    B.close()
    return S64, S32, out


def test_start_rounding_is_fp32_sized(runs):
    S64, S32, _ = runs
    e = link_err(S32, S64)
    assert 1e-9 < e.max() < 2e-7


def test_heatbath_sweep_keeps_the_link_bar(runs):
    """One heat-bath pass: the rounding of the start stays below 1e-5 on at
    least 99.99 % of the links (here: all, largest 7.7e-6, median 1e-7)."""
    _, _, out = runs
    R64, R32, _, _ = out[0]
    e = link_err(R32, R64)
    assert (e <= 1e-5).mean() >= 0.9999, ((e > 1e-5).sum(), e.max())
    assert np.median(e) < 1e-6


def test_overrelaxation_amplifies_the_start_rounding(runs):
    """Every overrelaxation pass multiplies the deviation: after HB + 1 OR
    about 1 % of the links are beyond 1e-5 (median 1e-6); after the
    workload's HB + 4 OR all of them are (median 2.4e-3)."""
    _, _, out = runs
    med = {}
    for n_or in (0, 1, 4):
        R64, R32, _, _ = out[n_or]
        e = link_err(R32, R64)
        med[n_or] = np.median(e)
        if n_or == 1:
            assert 1e-3 < (e > 1e-5).mean() < 0.1, (e > 1e-5).mean()
        if n_or == 4:
            assert (e > 1e-5).mean() > 0.5, (e > 1e-5).mean()
            assert med[4] > 1e-4, med[4]
    assert med[0] < med[1] < med[4], med
    assert med[4] / med[1] > 100.0, med  # three more passes, about x10 each


def test_total_plaquette_stays_within_the_metric_bar(runs):
    """Overrelaxation conserves the action, so after the full sweep the total
    plaquette of the two chains differs only by the heat-bath pass's
    deviation (measured 6e-11), far inside |dP| <= 1e-6, while the spatial and
    temporal parts drift apart by the energy the reflections moved between
    planes (measured 1.9e-5)."""
    _, _, out = runs
    (p64, l64), (p32, l32) = out[4][2], out[4][3]
    assert abs(p32[0] - p64[0]) < 1e-9, (p32, p64)
    assert abs(p32[1] - p64[1]) > 1e-6, (p32, p64)
