"""Ensemble parity of the SU(3) chain: 10^3 sweeps on the GPU against an
independent oracle chain (another seed), FP64 and FP32 storage.

SU(3) 8^3 x 4, hot start, sweeps of 1 heat-bath + 4 overrelaxation passes +
reunitarization (the sweep of the 16^3 x 4 workload), 100 sweeps of
thermalization, then 1000 measured sweeps.  Two couplings on either side of
the Nt = 4 deconfinement transition (beta_c about 5.69), where the Polyakov
loop decorrelates in a few sweeps (the oracle's integrated autocorrelation
times at 8^3 x 4: plaquette 1.5-4, Polyakov loop 0.6-2.6 sweeps; at
beta = 5.7 itself the Polyakov loop's is about 100, too long for 10^3
sweeps):
  beta = 5.5 (confined)    <P>, <Re L> and <|L|> within 3 sigma;
  beta = 5.9 (deconfined)  <P> and <|L|> within 3 sigma (Re L depends on
                           which of the three Z3 sectors a chain settled in,
                           |L| does not).
sigma combines both chains' errors from bins of 50 sweeps.
"""
import numpy as np
import pytest

import oracle
from workloads import FP32_COMPRESSED, FP64_PLAIN, HOT

pytestmark = pytest.mark.gpu

NS, NT, N_THERM, N_MEAS, BIN = 8, 4, 100, 1000, 50


@pytest.fixture(scope="module")
def q():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1310_7087_gb300 import build
    build.build()
    import paper_1310_7087_gb300 as q
    oracle.build()
    return q


def series(obj, measure, seed):
    p, rl, al = [], [], []
    for i in range(N_THERM + N_MEAS):
        obj.sweep(1, 4, seed)
        if i >= N_THERM:
            (pl, l) = measure()
            p.append(pl[0])
            rl.append(l[0])
            al.append(np.hypot(l[0], l[1]))
    return np.array(p), np.array(rl), np.array(al)


def binned(x):
    n = len(x) // BIN
    m = x[: n * BIN].reshape(n, BIN).mean(1)
    return m.mean(), m.std(ddof=1) / np.sqrt(n)


_oracle_cache = {}


def oracle_series(beta):
    if beta not in _oracle_cache:
        orc = oracle.OracleLattice(3, NS, NT, beta, 0, 10, 0)
        orc.hot_start(4)
        _oracle_cache[beta] = series(orc, orc.measure, 4)
        orc.close()
    return _oracle_cache[beta]


@pytest.mark.parametrize("beta,observables", [(5.5, ("P", "Re L", "|L|")), (5.9, ("P", "|L|"))])
@pytest.mark.parametrize("precision", [FP64_PLAIN, FP32_COMPRESSED])
def test_ensemble_su3_8x4(q, precision, beta, observables):
    lat = q.Lattice(3, NS, NT, beta, 0, precision, HOT, 3)
    gpu = series(lat, lat.measure, 3)
    lat.close()
    ref = oracle_series(beta)
    names = ("P", "Re L", "|L|")
    for name in observables:
        k = names.index(name)
        (ma, ea), (mb, eb) = binned(gpu[k]), binned(ref[k])
        z = abs(ma - mb) / np.hypot(ea, eb)
        print("beta %.2f %s: GPU %.5f +- %.5f, oracle %.5f +- %.5f (%.2f sigma)" % (beta, name, ma, ea, mb, eb, z))
        assert z < 3.0, (name, ma, ea, mb, eb)
