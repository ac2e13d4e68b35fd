"""The multi-rank host logic, run as two gloo ranks on the CPU: every rank
computes the same partition of the 64-lattice scan, the parts are disjoint and
cover every lattice with balanced volume, and the timing reductions return
the slowest rank's time and the total."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world_size, port, out):
    import torch.distributed as dist

    import workloads
    from paper_1310_7087_gb300 import dist as qd
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world_size), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world_size)
    assert qd.world() == (world_size, rank, rank)
    scan = workloads.batch_scan()
    mine = qd.shard(scan.volumes, world_size, rank)
    gathered = [None] * world_size
    dist.all_gather_object(gathered, mine)
    slowest = qd.max_over_ranks(1.0 + rank)
    total = qd.sum_over_ranks(float(sum(scan.volumes[i] for i in mine)))
    out[rank] = (gathered, slowest, total, qd.replica_seed(5, rank))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world_size", [2])
def test_gloo_sharding_and_reductions(world_size):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import workloads
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, world_size, port, out)) for r in range(world_size)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    scan = workloads.batch_scan()
    parts = out[0][0]
    assert all(out[r][0] == parts for r in range(world_size))  # same partition everywhere
    flat = sorted(i for part in parts for i in part)
    assert flat == list(range(64))  # disjoint and complete
    loads = [sum(scan.volumes[i] for i in part) for part in parts]
    assert max(loads) - min(loads) <= max(scan.volumes)
    assert all(out[r][1] == float(world_size) for r in range(world_size))  # slowest rank's time
    assert all(out[r][2] == float(sum(scan.volumes)) for r in range(world_size))
    assert len({out[r][3] for r in range(world_size)}) == world_size  # distinct replica seeds


def test_shard_is_deterministic_and_balanced():
    from paper_1310_7087_gb300 import dist as qd
    w = [5, 1, 1, 1, 1, 1]
    parts = [qd.shard(w, 2, r) for r in range(2)]
    assert sorted(parts[0] + parts[1]) == list(range(6))
    assert parts[0] == [0] and parts[1] == [1, 2, 3, 4, 5]
    assert qd.shard(w, 1, 0) == list(range(6))
    with pytest.raises(ValueError):
        qd.shard(w, 2, 2)
