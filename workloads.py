"""Seeded synthetic workloads for the SU(N) gauge sweep.

This module holds only workload descriptions and the seeded draw of the
batched parameter scan.  It contains none of the method's arithmetic and is
shared by the tests, the smoke check and the benchmark on both sides (CUDA
library and CPU oracle).

A Monte Carlo chain generates its own configurations, so the "inputs" are the
run parameters: gauge group, lattice extents (Ns^3 x Nt, finite temperature
means Nt < Ns), coupling beta, flux quantum n of the background field, start
(cold = unit links, hot = Haar links from the seed) and the sweep content.  The
shapes follow the paper's finite-temperature setting (sec. 4: the time extent is
the short one) and its benchmark lattices (sec. 5, Table 1: L^4 with L = 8..48).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

COLD, HOT = 0, 1
FP64_PLAIN, FP32_COMPRESSED = 0, 1


@dataclass(frozen=True)
class Workload:
    name: str
    group: int
    Ns: int
    Nt: int
    beta: float
    flux: int = 0
    start: int = HOT
    seed: int = 1
    n_hb: int = 1
    n_or: int = 1
    sweeps: int = 1
    nhit: int = 10

    @property
    def volume(self) -> int:
        return self.Ns ** 3 * self.Nt

    @property
    def links(self) -> int:
        return 4 * self.volume


# SU(2) 4^3 x 4, beta 2.3, no field, cold start, 100 x (1 HB + 1 OR), FP64.
SU2_4x4 = Workload("su2_4^3x4_b2.3", 2, 4, 4, 2.3, 0, COLD, 1, 1, 1, 100)
# SU(3) 16^3 x 4, beta 5.7, hot start seed 7, 1 HB (3 subgroups) + 4 OR.
SU3_16x4 = Workload("su3_16^3x4_b5.7", 3, 16, 4, 5.7, 0, HOT, 7, 1, 4, 1)
# SU(3) 32^3 x 8, beta 6.0, flux n in {0,1,2,4}, 500 x (HB + 4 OR).
SU3_32x8 = tuple(Workload("su3_32^3x8_b6.0_n%d" % n, 3, 32, 8, 6.0, n, HOT, 3, 1, 4, 500)
                 for n in (0, 1, 2, 4))
# SU(3) 64^3 x 16 (4.2M sites), beta 6.2, flux n = 1, 100 x (HB + 4 OR).
SU3_64x16 = Workload("su3_64^3x16_b6.2_n1", 3, 64, 16, 6.2, 1, HOT, 5, 1, 4, 100)


@dataclass(frozen=True)
class ONWorkload:
    """O(N) model run: lattice L^4, phi^4 couplings, Metropolis step delta,
    NHIT hits per site visit."""
    name: str
    N: int
    L: int
    kappa: float
    lam: float
    delta: float
    nhit: int = 100
    seed: int = 7

    @property
    def volume(self) -> int:
        return self.L ** 4


# O(4) on 32^4 with NHIT = 100 (the paper's Table 1 O(4) setting and lattice);
# kappa near the O(4) transition of the lambda = 1 model, delta for ~1/3 of
# the hits accepted.
O4_32 = ONWorkload("o4_32^4_k0.3_l1_nhit100", 4, 32, 0.3, 1.0, 0.8, 100, 7)


@dataclass
class BatchScan:
    """Batched parameter scan: independent SU(2) lattices of uneven sizes."""
    Ns: list = field(default_factory=list)
    Nt: list = field(default_factory=list)
    beta: list = field(default_factory=list)
    flux: list = field(default_factory=list)
    sweeps: int = 200
    n_or: int = 1
    seed: int = 11

    @property
    def n(self) -> int:
        return len(self.Ns)

    @property
    def volumes(self):
        return [ns ** 3 * nt for ns, nt in zip(self.Ns, self.Nt)]


def batch_scan(n_lattices: int = 64, seed: int = 11, sweeps: int = 200,
               n_or: int = 1) -> BatchScan:
    """Draw the scan: for each lattice, in this order, Ns from {8,12,16,24},
    Nt from {4,6,8}, beta uniform in [2.2, 2.5], flux n from {0,1,2,3}."""
    rng = np.random.default_rng(seed)
    b = BatchScan(sweeps=sweeps, n_or=n_or, seed=seed)
    for _ in range(n_lattices):
        b.Ns.append(int(rng.choice([8, 12, 16, 24])))
        b.Nt.append(int(rng.choice([4, 6, 8])))
        b.beta.append(float(rng.uniform(2.2, 2.5)))
        b.flux.append(int(rng.integers(0, 4)))
    return b


def small_batch(seed: int = 5, n_lattices: int = 5) -> BatchScan:
    """A few tiny uneven SU(2) lattices for parity tests of the batched path."""
    rng = np.random.default_rng(seed)
    b = BatchScan(sweeps=2, n_or=1, seed=seed)
    for _ in range(n_lattices):
        b.Ns.append(int(rng.choice([2, 4, 6])))
        b.Nt.append(int(rng.choice([2, 4])))
        b.beta.append(float(rng.uniform(2.2, 2.5)))
        b.flux.append(int(rng.integers(0, 4)))
    return b
