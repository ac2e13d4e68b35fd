"""The batched scan (one persistent launch for many uneven SU(2) lattices)
against the oracle and against the single-lattice path."""
import numpy as np
import pytest

import oracle
import workloads
from workloads import COLD, FP32_COMPRESSED, FP64_PLAIN, HOT

pytestmark = pytest.mark.gpu


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


def link_err(a, b):
    return np.abs(a - b).reshape(a.shape[0] * 4, -1).max(axis=1)


SMALL = workloads.small_batch()  # five tiny lattices, Ns in {2,4,6}, Nt in {2,4}, flux 0..3


def oracles_for(batch_desc, i, nhit=10):
    return oracle.OracleLattice(2, batch_desc.Ns[i], batch_desc.Nt[i], batch_desc.beta[i],
                                batch_desc.flux[i], nhit, i)


@pytest.mark.parametrize("precision", [FP64_PLAIN, FP32_COMPRESSED])
def test_batch_hot_start_uses_per_lattice_keys(q, precision):
    d = SMALL
    b = q.Batch(d.Ns, d.Nt, d.beta, d.flux, precision, HOT, 17)
    for i in range(b.n):
        o = oracles_for(d, i)
        o.hot_start(17)
        tol = 1e-14 if precision == FP64_PLAIN else 2e-7
        assert link_err(b.get_links(i), o.get_links()).max() < tol
    b.close()


@pytest.mark.parametrize("precision", [FP64_PLAIN, FP32_COMPRESSED])
def test_batch_sweep_matches_oracle(q, precision):
    d = SMALL
    b = q.Batch(d.Ns, d.Nt, d.beta, d.flux, precision, HOT, 5)
    orcs = []
    for i in range(b.n):
        o = oracles_for(d, i)
        o.set_links(b.get_links(i))
        orcs.append(o)
    # FP32: one heat-bath-only sweep, since the chain amplifies FP32 rounding
    # (the overrelaxation code is the same template, checked with FP64 here)
    n_sweeps, n_or = (2, 1) if precision == FP64_PLAIN else (1, 0)
    meas = b.sweep(n_sweeps, n_or, 5)
    assert b.sweep_counter == n_sweeps
    tol = 1e-12 if precision == FP64_PLAIN else 1e-6
    for i, o in enumerate(orcs):
        for s in range(n_sweeps):
            o.sweep(1, n_or, 5)
            p, l = o.measure()
            np.testing.assert_allclose(meas[i, s, :3], p, atol=tol)
            np.testing.assert_allclose(meas[i, s, 3:], l, atol=tol)
        err = link_err(b.get_links(i), o.get_links())
        if precision == FP64_PLAIN:
            assert err.max() < 1e-9, (i, err.max())
        else:
            assert (err <= 1e-5).mean() >= 0.9999, (i, err.max())
    b.close()


def test_batch_lattice_zero_equals_single_lattice_path(q):
    """Lattice 0 of a batch has the single-lattice Philox key; with FP64
    storage both paths run the same per-site code and agree to rounding
    (the compiler may contract multiply-adds differently in the two kernels)."""
    d = SMALL
    b = q.Batch(d.Ns, d.Nt, d.beta, d.flux, FP64_PLAIN, HOT, 9)
    lat = q.Lattice(2, d.Ns[0], d.Nt[0], d.beta[0], d.flux[0], FP64_PLAIN, HOT, 9)
    assert np.array_equal(b.get_links(0), lat.get_links())
    meas = b.sweep(3, 1, 9)
    for s in range(3):
        lat.sweep(1, 1, 9)
        p, l = lat.measure()
        np.testing.assert_allclose(meas[0, s, :3], p, atol=1e-12)
    assert link_err(b.get_links(0), lat.get_links()).max() < 1e-12
    lat.close()
    b.close()


def test_batch_results_do_not_depend_on_launch_shape(q):
    d = SMALL
    out = []
    for threads in (64, 128, 512):
        b = q.Batch(d.Ns, d.Nt, d.beta, d.flux, FP64_PLAIN, HOT, 3)
        q.qcd_batch_set_block(b.h, threads)
        assert q.qcd_batch_get_shape(b.h)[0] == threads
        m = b.sweep(2, 1, 3)
        out.append((m, [b.get_links(i) for i in range(b.n)]))
        b.close()
    for k in (1, 2):
        np.testing.assert_allclose(out[0][0], out[k][0], atol=1e-13)
        for a, c in zip(out[0][1], out[k][1]):
            assert np.array_equal(a, c)


@pytest.mark.parametrize("precision", [FP64_PLAIN, FP32_COMPRESSED])
def test_batch_waves_give_the_one_wave_results(q, precision):
    """Waves of consecutive lattices (here forced small: at most one or two
    lattices each) sweep every lattice as one launch does: links bit-identical,
    measurements equal to rounding, and the barrier-timeout path still works."""
    d = SMALL
    out = []
    for budget in (0, 1, 40000):
        b = q.Batch(d.Ns, d.Nt, d.beta, d.flux, precision, HOT, 3)
        q.qcd_batch_set_wave_bytes(b.h, budget)
        m = b.sweep(3, 1, 3)
        waves, got = q.qcd_batch_get_waves(b.h)
        assert got == budget and (waves == 1 if budget == 0 else waves > 1), (budget, waves)
        if budget == 1:
            assert waves == d.n  # one lattice per wave
        out.append((m, [b.get_links(i) for i in range(b.n)]))
        b.close()
    for k in (1, 2):
        np.testing.assert_allclose(out[0][0], out[k][0], atol=1e-13 if precision == FP64_PLAIN else 1e-6)
        for a, c in zip(out[0][1], out[k][1]):
            assert np.array_equal(a, c)


def test_batch_wave_timeout(q):
    d = SMALL
    b = q.Batch(d.Ns, d.Nt, d.beta, d.flux, FP32_COMPRESSED, HOT, 2)
    q.qcd_batch_set_wave_bytes(b.h, 1)
    b.sweep(1, 1, 2)
    q.qcd_batch_set_wait(b.h, 0.2)
    q.qcd_batch_inject_stall(b.h, d.n - 1)  # a lattice of the last wave
    with pytest.raises(q.QcdError) as e:
        b.sweep(1, 1, 2)
    assert e.value.code == q.QCD_ERR_TIMEOUT
    q.qcd_batch_inject_stall(b.h, -1)
    assert np.isfinite(b.sweep(1, 1, 2)).all()
    b.close()


def test_batch_barrier_timeout_is_reported_and_recoverable(q):
    """A barrier that waits for an arrival that never comes runs out after
    the bounded wait; the call returns QCD_ERR_TIMEOUT and the next sweep on
    the same context works."""
    d = SMALL
    b = q.Batch(d.Ns, d.Nt, d.beta, d.flux, FP32_COMPRESSED, HOT, 2)
    b.sweep(1, 1, 2)  # choose the launch shape first
    q.qcd_batch_set_wait(b.h, 0.2)
    q.qcd_batch_inject_stall(b.h, 0)
    with pytest.raises(q.QcdError) as e:
        b.sweep(1, 1, 2)
    assert e.value.code == q.QCD_ERR_TIMEOUT
    q.qcd_batch_inject_stall(b.h, -1)
    ref = q.Batch(d.Ns, d.Nt, d.beta, d.flux, FP32_COMPRESSED, COLD, 2)
    m = ref.sweep(1, 1, 2)
    assert np.isfinite(m).all()
    m2 = b.sweep(1, 1, 2)
    assert np.isfinite(m2).all()
    ref.close()
    b.close()


def test_batch_lattice_size_limit(q):
    """FP32 batches index a lattice's links in 32-bit arithmetic: a lattice of
    2^29 sites is refused before anything is allocated (128^3 x 256), FP64
    keeps the 2^31 limit."""
    with pytest.raises(q.QcdError) as e:
        q.qcd_batch_create(2, [4, 128], [4, 256], [2.3, 2.3], [0, 0], FP32_COMPRESSED)
    assert e.value.code == q.QCD_ERR_INVALID_ARG
    with pytest.raises(q.QcdError) as e:
        q.qcd_batch_create(2, [4, 256], [4, 128], [2.3, 2.3], [0, 0], FP64_PLAIN)
    assert e.value.code == q.QCD_ERR_INVALID_ARG


def test_batch_bad_arguments(q):
    with pytest.raises(q.QcdError) as e:
        q.qcd_batch_create(3, [4], [4], [1.0], [0])
    assert e.value.code == q.QCD_ERR_NOT_SUPPORTED
    with pytest.raises(q.QcdError) as e:
        q.qcd_batch_create(2, [4, 5], [4, 4], [1.0, 1.0], [0, 0])
    assert e.value.code == q.QCD_ERR_INVALID_ARG


def test_batch_scan_64_lattices(q):
    """The 64-lattice scan (Ns in {8,12,16,24}, Nt in {4,6,8}, seed 11): a few
    sweeps, then for five lattices one more sweep against the oracle from the
    same state (the three smallest, the smallest whose Nt and the smallest
    whose Ns is not a power of two: their threads walk several sites per
    phase, with carries through every coordinate); every lattice's plaquette
    in a physical range."""
    d = workloads.batch_scan()
    b = q.Batch(d.Ns, d.Nt, d.beta, d.flux, FP32_COMPRESSED, HOT, d.seed)
    m = b.sweep(5, 1, d.seed)
    assert m.shape == (64, 5, 5)
    assert np.isfinite(m).all()
    assert (m[:, -1, 0] > 0.45).all() and (m[:, -1, 0] < 0.75).all()
    by_size = sorted(range(64), key=lambda i: d.volumes[i])
    pow2 = lambda n: n & (n - 1) == 0
    odd_t = next(i for i in by_size if not pow2(d.Nt[i]))
    odd_s = next(i for i in by_size if not pow2(d.Ns[i]))
    small = by_size[:3] + [odd_t, odd_s]
    orcs = {}
    for i in small:
        o = oracles_for(d, i)
        o.set_links(b.get_links(i))
        o.sweep_counter = b.sweep_counter
        orcs[i] = o
    m = b.sweep(1, 1, d.seed)
    for i, o in orcs.items():
        o.sweep(1, 1, d.seed)
        err = link_err(b.get_links(i), o.get_links())
        assert (err <= 1e-5).mean() >= 0.9999, (i, err.max())
        p, l = o.measure()
        np.testing.assert_allclose(m[i, 0, :3], p, atol=1e-6)
    b.close()
