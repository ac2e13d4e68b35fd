"""Pins for the oracle's random numbers: Philox-4x32-10 known answers and the
word -> uniform map."""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            words = [int(w, 16) for w in line.split()]
            rows.append((words[0:4], words[4:6], words[6:10]))
    return rows


def test_kat_file_has_vectors():
    assert len(_kat_rows()) == 3


@pytest.mark.parametrize("row", _kat_rows())
def test_philox_known_answers(oracle_mod, row):
    ctr, key, expect = row
    assert oracle_mod.philox4x32_10(ctr, key) == expect


def test_philox_counter_sensitivity(oracle_mod):
    base = oracle_mod.philox4x32_10([1, 2, 3, 4], [5, 6])
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        assert oracle_mod.philox4x32_10(c, [5, 6]) != base
    assert oracle_mod.philox4x32_10([1, 2, 3, 4], [5, 7]) != base


def test_uniform_grid(oracle_mod):
    # ((w >> 9) + 1/2) 2^-23: open interval, 2^23 midpoints, FP32-exact.
    assert oracle_mod.uniform(0) == 0.5 * 2.0 ** -23
    assert oracle_mod.uniform(0x1FF) == 0.5 * 2.0 ** -23
    assert oracle_mod.uniform(0xFFFFFFFF) == 1.0 - 0.5 * 2.0 ** -23
    assert oracle_mod.uniform(1 << 31) == 0.5 + 0.5 * 2.0 ** -23
    rng = np.random.default_rng(0)
    for w in rng.integers(0, 2 ** 32, size=2000, dtype=np.uint64):
        u = oracle_mod.uniform(int(w))
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u
        assert u == ((int(w) >> 9) + 0.5) / 2 ** 23


def test_uniform_moments(oracle_mod):
    rng = np.random.default_rng(1)
    ws = rng.integers(0, 2 ** 32, size=200000, dtype=np.uint64)
    us = np.array([oracle_mod.uniform(int(w)) for w in ws[:20000]])
    assert abs(us.mean() - 0.5) < 5 * np.sqrt(1 / 12 / len(us))
