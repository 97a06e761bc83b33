"""The N > 1 path of bench.py on CPU: two gloo ranks, each with its own problem and its own
time; the whole-job rate divides all ranks' eigenpairs by the slowest rank's time, and
each rank's (independent) problem is solved without any collective on the data path.
The eigenpairs here come from the CPU oracle (no GPU in this test)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    import oracle
    from paper_1405_7537_gb300 import workloads as W
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    # each rank: its own problem (seed + rank), as bench.py does
    d, z, rho = W.hard(64, bench.SEED + rank)
    r = oracle.eig_all(d, z, rho)
    total_ms = [120.0, 300.0][rank]
    value, max_ms = bench.aggregate(total_ms, d.size, 3, world, dist, "cpu")
    out[rank] = (value, max_ms, float(np.sum(r["lam"])))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    v0, m0, s0 = out[0]
    v1, m1, s1 = out[1]
    assert m0 == m1 == 300.0
    assert v0 == v1 == pytest.approx(2 * 64 * 3 / 0.3)
    assert s0 != s1          # the ranks solved different problems
