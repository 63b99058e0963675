"""Realisation sharding of a disorder ensemble (host logic, CPU).

Two and three gloo ranks each evolve their block of realisations (here with the
oracle as the slice runner, so the test needs no GPU) and one all-reduce forms
the disorder-averaged autocorrelation; every rank must hold the same mean as a
single process that runs all realisations itself.
"""
import os
import socket

import numpy as np
import pytest

from paper_2603_07341_gb300 import sharding
from paper_2603_07341_gb300 import workloads as W

R_TEST, NSTEPS = 5, 6


def test_shard_range_covers_every_realisation_once():
    for R in (0, 1, 2, 5, 7, 256):
        for world in (1, 2, 3, 4, 8):
            blocks = [sharding.shard_range(R, world, k) for k in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == R
            assert all(a[1] == b[0] for a, b in zip(blocks, blocks[1:]))
            sizes = [hi - lo for lo, hi in blocks]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        sharding.shard_range(4, 2, 2)


def _cfg():
    return dict(W.WORKLOADS["disorder12"], n_sites=4, dims=(4, 1, 1), cap=2, m_init=3, theta=1e-4)


def oracle_slice_runner(cfg):
    """run_slice with the oracle: one instance per realisation."""
    from oracle.oracle import Oracle

    def run(lo, hi):
        out = np.zeros((NSTEPS + 1, hi - lo), dtype=np.complex128)
        for i, r in enumerate(range(lo, hi)):
            o = Oracle(**W.model_kwargs(cfg, eps=W.realisation_eps(cfg, r)))
            o.set_state(*W.start_state(cfg))
            st = o.stats()
            out[0, i] = st["C_re"] + 1j * st["C_im"]
            for k in range(NSTEPS):
                o.step(cfg["dt"], cfg["theta"])
                st = o.stats()
                out[k + 1, i] = st["C_re"] + 1j * st["C_im"]
        return out

    return run


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    C, (lo, hi), C_loc = sharding.run_sharded_ensemble(R_TEST, NSTEPS, oracle_slice_runner(_cfg()))
    out.put((rank, C, lo, hi))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_mean_equals_single_process(world):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict((g[0], g[1:]) for g in (q.get(timeout=300) for _ in range(world)))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = oracle_slice_runner(_cfg())(0, R_TEST).mean(axis=1)
    blocks = sorted((lo, hi) for _, lo, hi in got.values())
    assert blocks[0][0] == 0 and blocks[-1][1] == R_TEST
    for k in range(world):
        C = got[k][0]
        assert np.max(np.abs(C - ref)) <= 1e-14
    assert abs(ref[0] - 1.0) < 1e-14 and np.max(np.abs(np.diff(ref))) > 1e-3   # a non-trivial signal


def test_single_process_driver_without_a_process_group():
    C, (lo, hi), _ = sharding.run_sharded_ensemble(2, NSTEPS, oracle_slice_runner(_cfg()))
    assert (lo, hi) == (0, 2) and C.shape == (NSTEPS + 1,)
