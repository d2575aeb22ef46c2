"""Multi-GPU runs are replicas: the whole-job figures of bench.py are the slowest rank's time and
the sum of the ranks' work, with one configuration broadcast from rank 0.  Checked here with two
gloo processes on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=2)
    import bench
    t, units = bench.replica_reduce(1.0 + rank, 10.0 * (rank + 1))
    skin = bench.replica_choice(0.02 if rank == 0 else 0.1)
    out.put((rank, t, units, skin))
    dist.destroy_process_group()


def test_replica_figures_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, units, skin in res:
        assert t == 2.0            # the slowest rank's time
        assert units == 30.0       # the work of both ranks
        assert skin == 0.02        # rank 0's configuration everywhere


def test_single_process_is_identity():
    import bench
    assert bench.replica_reduce(3.0, 7.0) == (3.0, 7.0)
    assert bench.replica_choice(0.5) == 0.5
