"""The N > 1 benchmark path on CPU: independent replicas, world size 2 over gloo.  The
whole-job value sums the particle-steps of every rank and divides by the slowest rank's
time (a barrier brackets the timed region; no collective touches the data path)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import sys
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [120.0, 150.0][rank]             # rank 1 is the slower replica
    units = [1.0e9, 2.0e9][rank]
    dist.barrier()
    out = bench.aggregate(ms, units, dist, "cpu")
    dist.barrier()
    q.put((rank, out))
    dist.destroy_process_group()


def test_replica_aggregation_over_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        assert res[r]["ms_max"] == 150.0
        assert res[r]["units"] == 3.0e9
        assert abs(res[r]["value"] - 3.0e9 / 0.150) < 1e-3


def test_single_process_aggregation_is_identity():
    import bench
    out = bench.aggregate(100.0, 5e9)
    assert out == {"ms_max": 100.0, "units": 5e9, "value": 5e10}
