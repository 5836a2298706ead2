"""Time-sharded estimation of one long stream, merged across ranks (CPU, gloo, 2 ranks).

Each rank estimates its own segment with the oracle (as a GPU rank would with libcyc),
the ranks merge with one all-reduce, and the result must equal the oracle on the whole
stream.  This exercises the partition plan and the reduction with a real process group.
"""
import os
import socket

import numpy as np
import pytest

import oracle
import synth
from paper_2405_16911_gb300 import shard


def test_time_shards_partition():
    for T, M, world in [(1000, 7, 2), (1000, 0, 3), (10, 20, 2), (257, 3, 8), (5, 4, 4)]:
        sh = shard.time_shards(T, M, world)
        assert len(sh) == world
        n = 0
        for s0, s1, a, cnt in sh:
            assert a == n and cnt >= 0
            if cnt:
                assert s0 == a and s1 == a + cnt + M and s1 <= T
            n += cnt
        assert n == max(0, T - M)


def test_merge_is_n_weighted():
    R1, R2 = np.array([1 + 1j, 2.0]), np.array([3.0, 4 - 1j])
    R, n = shard.merge([(R1, 10), (R2, 30), (None, 0)])
    assert n == 40 and np.allclose(R, (10 * R1 + 30 * R2) / 40)
    assert shard.merge([]) == (None, 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        T, lags = 3001, np.array([0, 3, 11, 5])
        M = 11
        alphas = np.array([0.0, 0.125, -0.31, 0.4])
        x = synth.white(T, seed=77).astype(np.complex64)
        s0, s1, a, cnt = shard.time_shards(T, M, world)[rank]
        R, n = oracle.estimate(x[s0:s1], lags, alphas, n0=a)
        Rm, nm = shard.allreduce_merge(R, n)
        q.put((rank, Rm, nm))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_gloo_two_ranks_merge_equals_whole_stream(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    T, lags, M = 3001, np.array([0, 3, 11, 5]), 11
    x = synth.white(T, seed=77).astype(np.complex64)
    Ro, no = oracle.estimate(x, lags, np.array([0.0, 0.125, -0.31, 0.4]))
    for rank, Rm, nm in got:
        assert nm == no
        assert np.allclose(Rm, Ro, atol=1e-12), rank
