"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): the
native shard planner gives each rank a contiguous block range, the ranges
cover every block once, and the cross-rank reductions (max time, summed
entries) are what the benchmark reports.  No GPU is involved."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, ws, port, out):
    import torch.distributed as tdist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    w = synth.workloads.config2(levels=3)
    lo, hi = bench.shard_range(w.near, rank, ws)
    mine = int(bench.block_costs(w.near)[lo:hi].sum())
    total = bench.reduce_over_ranks(mine, "sum")
    slowest = bench.reduce_over_ranks(10.0 + rank, "max")
    # the default line's sharding: contiguous cost-balanced ranges of a batch's meshes
    batch = synth.workloads.config4(count=6, lo=200.0, hi=800.0)
    ids = [id(it) for it in bench.shard_items(batch.items, rank, ws)]
    pos = [k for k, it in enumerate(batch.items) if id(it) in ids]
    out[rank] = (lo, hi, mine, total, slowest, pos)
    tdist.barrier()
    tdist.destroy_process_group()


def test_two_rank_sharding_and_reductions():
    import bench  # noqa: F401  (imports without a GPU)
    ws = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(ws, _free_port(), out), nprocs=ws, join=True,
                       start_method="spawn")
    w = synth.workloads.config2(levels=3)
    costs = bench.block_costs(w.near)
    r0, r1 = out[0], out[1]
    assert r0[0] == 0 and r0[1] == r1[0] and r1[1] == len(costs)      # contiguous cover
    assert r0[2] + r1[2] == costs.sum() == r0[3] == r1[3]                # summed entries
    assert r0[4] == r1[4] == 11.0                                         # max over ranks
    assert abs(r0[2] - r1[2]) <= costs.max()                              # balanced
    assert r0[5] + r1[5] == list(range(6)) and r0[5] and r1[5]           # meshes split, once


def test_shard_planner_properties():
    import paper_1510_07244_gb300 as pkg
    from paper_1510_07244_gb300 import build as libbuild
    libbuild.build()
    rng = np.random.default_rng(3)
    for n_shards in (1, 2, 3, 8):
        cost = rng.integers(0, 1000, 500)
        b = pkg.bem_shard_blocks(cost, n_shards)
        assert b[0] == 0 and b[-1] == len(cost) and np.all(np.diff(b) >= 0)
        sums = np.array([cost[b[k]:b[k + 1]].sum() for k in range(n_shards)])
        assert sums.sum() == cost.sum()
        assert np.all(np.abs(sums - cost.sum() / n_shards) <= cost.max())
    with pytest.raises(pkg.BemError):
        pkg.bem_shard_blocks([1, -1], 2)
