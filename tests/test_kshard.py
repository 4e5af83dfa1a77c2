"""k-range sharding of the C_l quadrature (the exchange step of the k-shard
form of the path): CPU ranks over gloo, world sizes 2 and 3.  Each rank
projects and k-integrates only its shard of the k nodes with the oracle, the
partial C_l are sum-reduced, and the result must equal the single-pass
oracle C_l up to the order of summation (~1e-14 relative)."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2602_15104_gb300.shard import k_shard  # noqa: E402

N_K, N_TAU, LMAX = 23, 400, 120


def _inputs():
    from paper_2602_15104_gb300 import workload as W
    p = W.BATCH64.params()[5]
    k = W.log_k_nodes(N_K, 1e-3, 0.1)
    S = W.synthetic_sources(N_K, N_TAU, 7)
    return p, k, S


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import oracle as O
    from paper_2602_15104_gb300.shard import k_shard, reduce_partial_cl
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p, k, S = _inputs()
        lo, hi = k_shard(N_K, rank, world)
        s = O.scalars(p)
        lna, tau, w = O.nodes(p, N_TAU)
        D = O.project(tau, w, s["tau0"], k[lo:hi], S[lo:hi], LMAX, nthreads=1)
        C = torch.tensor(O.cl(k[lo:hi], D, LMAX, s["A_s"], p[3]))
        reduce_partial_cl(C, dist)
        out[rank] = C.numpy().copy()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_partial_cl_sum_equals_single_pass(world):
    import oracle as O
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:  # no fork of a threaded process
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, start_method="spawn")
        res = dict(out)
    p, k, S = _inputs()
    s = O.scalars(p)
    lna, tau, w = O.nodes(p, N_TAU)
    ref = O.cl(k, O.project(tau, w, s["tau0"], k, S, LMAX, nthreads=1), LMAX, s["A_s"], p[3])
    for rank in range(world):
        np.testing.assert_array_equal(res[rank], res[0])  # every rank holds the same sum
    scale = np.abs(ref).max(axis=1, keepdims=True)
    assert np.all(np.abs(res[0] - ref) <= 1e-14 * scale)
    tt = np.abs(res[0][0] - ref[0]) / np.abs(ref[0])
    assert tt.max() < 1e-13


def test_shards_cover_every_interval_once():
    for n in (2, 3, 10, 400):
        for world in range(1, min(n - 1, 9) + 1):
            shards = [k_shard(n, r, world) for r in range(world)]
            assert shards[0][0] == 0 and shards[-1][1] == n
            for (lo, hi), (lo2, hi2) in zip(shards, shards[1:]):
                assert lo2 == hi - 1  # one shared boundary node
            assert all(hi - lo >= 2 for lo, hi in shards)
    with pytest.raises(ValueError):
        k_shard(3, 0, 3)
