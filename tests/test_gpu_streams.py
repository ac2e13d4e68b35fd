"""Independent lattices on their own CUDA streams: working sweeps of several
lattices queued side by side (no host wait between them, as a parameter scan
queues its chains) give, lattice by lattice, the links and the measurements
of the same lattice swept alone, bit for bit.  Each lattice owns its
scratch, sweep counter and captured sweep graphs; nothing is shared between
streams."""
import numpy as np
import pytest

from workloads import FP32_COMPRESSED, FP64_PLAIN, HOT

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


# (group, precision, Ns, Nt, beta, fluxes): one lattice per flux quantum
CASES = [(3, FP32_COMPRESSED, 8, 4, 6.0, (0, 1, 2, 4)),
         (3, FP32_COMPRESSED, 6, 4, 5.7, (1, 3)),     # extents not powers of two
         (2, FP32_COMPRESSED, 8, 4, 2.3, (0, 1, 2)),
         (3, FP64_PLAIN, 4, 4, 5.7, (0, 2))]


@pytest.mark.parametrize("group,precision,Ns,Nt,beta,fluxes", CASES)
def test_side_by_side_chains_equal_lone_chains(q, group, precision, Ns, Nt, beta, fluxes):
    import torch
    seed, n_or, sweeps = 13, 2, 6
    # alone, one lattice at a time on the current stream, blocking calls; one
    # launch shape everywhere, so the block partials of the fused measurement
    # are summed alike
    alone = []
    for n in fluxes:
        lat = q.Lattice(group, Ns, Nt, beta, n, precision, HOT, seed)
        q.qcd_set_block(lat.h, 128)
        meas = [q.qcd_working_sweep(lat.h, 1, n_or, seed) for _ in range(sweeps)]
        alone.append((lat.get_links(), meas))
        lat.close()
    # side by side: one stream per lattice, every sweep queued before any wait
    streams = [torch.cuda.Stream() for _ in fluxes]
    lats = [q.Lattice(group, Ns, Nt, beta, n, precision, HOT, seed, s) for n, s in zip(fluxes, streams)]
    for lat in lats:
        q.qcd_set_block(lat.h, 128)
    buf = torch.zeros((len(lats), sweeps, 5), dtype=torch.float64, pin_memory=True)
    for i in range(sweeps):
        for k, lat in enumerate(lats):
            q.qcd_working_sweep(lat.h, 1, n_or, seed, buf[k, i].data_ptr(), wait=False)
    torch.cuda.synchronize()
    for k, lat in enumerate(lats):
        links, meas = alone[k]
        assert np.array_equal(lat.get_links(), links), (fluxes[k], "links differ")
        assert np.array_equal(buf[k].numpy(), np.array(meas)), (fluxes[k], buf[k], meas)
        lat.close()
