"""Sharding a batch over GPUs by tet (ilu_partition), without a GPU.

The partition is checked for what the longest-processing-time rule
guarantees (every tet on exactly one rank, the largest load within 4/3 of
the optimum's lower bound), and the sharded run is exercised as two gloo
ranks on the CPU: each rank sweeps only its own tets (the oracle stands in
for the GPU batch), the results are gathered on rank 0 over the host, and
they equal a single-process run tet for tet."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import seeded_inputs as si  # noqa: E402


@pytest.fixture(scope="module")
def g():
    import paper_2210_15280_gb300 as g
    g.build()
    return g


@pytest.mark.parametrize("nranks", [1, 2, 3, 8])
def test_partition_covers_every_tet_once_and_balances(g, nranks):
    levels = si.batch_levels(7, 256, 5, 8)
    cost = np.array([bench.interior(int(L)) for L in levels], dtype=np.float64)
    rank_of, load = g.partition(cost, nranks)
    assert rank_of.shape == (256,) and rank_of.min() >= 0 and rank_of.max() < nranks
    for r in range(nranks):
        assert np.isclose(load[r], cost[rank_of == r].sum())
    assert np.isclose(load.sum(), cost.sum())
    bound = max(cost.sum() / nranks, cost.max())  # no split does better than this
    assert load.max() <= 4.0 / 3.0 * bound + 1e-9
    again, _ = g.partition(cost, nranks)
    assert np.array_equal(rank_of, again)  # deterministic: every rank computes the same split


def test_partition_rejects_bad_input(g):
    with pytest.raises(g.IluError):
        g.partition([1.0, -2.0], 2)
    with pytest.raises(g.IluError):
        g.partition([1.0], 0)
    rank_of, load = g.partition([], 4)
    assert rank_of.size == 0 and not load.any()


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    results = bench.sharded_oracle_sweeps(rank, world, dist)
    dist.destroy_process_group()
    if rank == 0:
        np.save(os.path.join(out, "gathered.npy"), np.array(results, dtype=object), allow_pickle=True)


def test_two_gloo_ranks_shard_and_gather(tmp_path):
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    code = ("import sys; sys.path.insert(0, %r); sys.path.insert(0, %r); import test_shard_host as t; "
            "t._rank(%%d, 2, %d, %r)" % (ROOT, os.path.join(ROOT, "tests"), port, str(tmp_path)))
    procs = [subprocess.Popen([sys.executable, "-c", code % r], cwd=ROOT) for r in range(2)]
    for p in procs:
        assert p.wait(timeout=600) == 0
    gathered = np.load(tmp_path / "gathered.npy", allow_pickle=True)
    single = bench.sharded_oracle_sweeps(0, 1, None)
    assert len(gathered) == len(single)
    for a, b in zip(gathered, single):
        assert a[0] == b[0] and np.array_equal(a[1], b[1])
