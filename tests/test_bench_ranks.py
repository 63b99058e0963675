"""The replica reduction of bench.py over two gloo ranks on the CPU: value is
the sum of the ranks' units over the slowest rank's time."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=2)
    ws, rk, local = bench.dist_setup()
    assert (ws, rk, local) == (2, rank, rank)
    ms = [100.0, 140.0][rank]
    units = [1.0e9, 1.5e9][rank]
    res = bench.reduce_over_ranks(dist, ms, units, [3.0, 2.5][rank], [4.0e9, 5.0e9][rank], "cpu")
    out.put((rank, res))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_reduction_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        t_max, total, t_host, all_units = got[r]
        assert t_max == 140.0 and total == 2.5e9 and t_host == 3.0 and all_units == 9.0e9
    # whole-job value as bench.py forms it
    assert total / (t_max / 1e3) == pytest.approx(2.5e9 / 0.14)
