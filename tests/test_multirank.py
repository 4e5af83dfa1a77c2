"""Multi-rank host logic of bench.py on CPU ranks (gloo, world size 2): each
rank draws its own cosmologies (weak scaling, no data exchange), the job time
is the slowest rank's, and the whole-job rate counts every rank's units."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    from paper_2602_15104_gb300 import workload as W
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = bench.rank_params(W.BATCH64, 4, rank)
        t = bench.max_over_ranks([10.0 * (rank + 1), 3.0 - rank], dist, "cpu")
        gathered = [None] * world
        dist.all_gather_object(gathered, p.tolist())
        out[rank] = (t, gathered, bench.whole_job_rate(4, world, t[0]))
    finally:
        dist.destroy_process_group()


def test_two_cpu_ranks_weak_scaling_and_max_timing():
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as m:  # no fork of a threaded process
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, start_method="spawn")
        res = dict(out)
    for rank in range(world):
        t, gathered, rate = res[rank]
        assert t == [20.0, 3.0]  # element-wise max over ranks
        assert rate == pytest.approx(4 * 2 / 20e-3)
        a, b = np.array(gathered[0]), np.array(gathered[1])
        assert a.shape == b.shape == (4, 6)
        assert not np.allclose(a, b)  # independent batches per rank


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([1.5, 2.5], None, "cpu") == [1.5, 2.5]
    assert bench.whole_job_rate(64, 1, 1000.0) == pytest.approx(64.0)
