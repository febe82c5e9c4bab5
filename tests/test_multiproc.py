"""The multi-rank path of bench.py on CPU: two gloo ranks, each with its own
key set (seed 1 + rank), a barrier, the slowest rank's time taken by every
rank, and the whole-job throughput of independent per-rank hypergraphs."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    from paper_1312_0526_gb300 import inputs
    w, r, lr = bench.dist_setup()
    keys = inputs.keys(2000, bench.KEY_SEED + r)
    m = oracle.num_vertices(2000, bench.GAMMA_MILLI, bench.R)
    res = oracle.peel_rounds(oracle.hash_edges(keys, m, 3, bench.HASH_SEED), m)
    dist.barrier()
    ms = 10.0 * (r + 1)  # the ranks report different times
    slowest = bench.reduce_max(ms, dist)
    out[r] = (w, r, lr, int(keys[0]), res.n_peeled, slowest,
              bench.aggregate_medges(2000, w, slowest))
    dist.destroy_process_group()


def test_two_gloo_ranks_independent_key_sets_and_max_timing():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        got = dict(out)
    assert sorted(got) == [0, 1]
    (w0, r0, l0, k0, p0, s0, v0), (w1, r1, l1, k1, p1, s1, v1) = got[0], got[1]
    assert (w0, w1, r0, r1, l0, l1) == (2, 2, 0, 1, 0, 1)
    assert k0 != k1                     # independent key sets
    assert s0 == s1 == 20.0             # both ranks take the slowest time
    assert v0 == v1 == pytest.approx(2000 * 2 / 0.020 / 1e6)
    assert p0 > 0 and p1 > 0
