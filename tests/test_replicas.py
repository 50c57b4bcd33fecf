"""The replica path of bench.py (one rank per GPU, independent systems) on
CPU: two gloo ranks reduce their step times and charge counts the way the
benchmark does (max time, summed charges)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2101_07088_b300 import replicas  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, rate = replicas.job_rate(10.0 + rank, 100 * (rank + 1), dist)
        out[rank] = (ms, rate, replicas.replica_seed(2, rank))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_benchmark():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        ms, rate, seed = res[r]
        assert ms == 11.0                      # the slowest rank's step time
        assert abs(rate - 300 / 0.011) < 1e-6 * rate   # every rank's charges
    assert res[0][2] == 2 and res[1][2] != res[0][2]   # rank 0 keeps the seed; the other differs


def test_one_process():
    ms, rate = replicas.job_rate(20.0, 1000)
    assert ms == 20.0 and abs(rate - 50000.0) < 1e-9
