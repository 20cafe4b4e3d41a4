"""The multi-rank paths on CPU (gloo, world size 2).

Designs are independent, so ranks shard them with no data-path collective.
The benchmark runs replicas: each rank evaluates its own copy of the grid
with its own stream keys (weak scaling), and the only collectives are the
timing barrier and the max of the per-rank times.  A batch can also be
split into contiguous design ranges balanced by N d^2 and the per-design
hit counts all-gathered afterwards (paper_2005_10494_gb300.partition).
This checks those host-side pieces; no GPU is used.
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import workloads


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prob = workloads.c2(n_scen=1, g1=2, g2=3, n_draws=1000)
    keys = bench.rank_keys(prob.keys, rank)
    t_max = bench.max_over_ranks(0.5 + rank, device="cpu")
    out[rank] = (keys.tolist(), t_max)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_ranks_shard_keys_and_reduce_time():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn")
        k0, t0 = out[0]
        k1, t1 = out[1]
    assert t0 == t1 == 1.5                       # max over ranks
    assert not set(k0) & set(k1)                 # independent streams per rank
    base = workloads.c2(n_scen=1, g1=2, g2=3, n_draws=1000).keys
    np.testing.assert_array_equal(k0, base)      # rank 0 keeps the workload's keys


# ------------------------------------------------ design-range sharding
def test_design_ranges_cover_every_design_once_and_balance_cost():
    from paper_2005_10494_gb300 import partition
    rng = np.random.default_rng(3)
    for J, world in ((1, 1), (5, 8), (37, 2), (1000, 3), (4096, 8)):
        n = rng.integers(1, 10_000_000, J)
        d = rng.integers(1, 21, J)
        cost = partition.design_cost(n, d)
        ranges = partition.design_ranges(cost, world)
        assert len(ranges) == world
        assert ranges[0][0] == 0 and ranges[-1][1] == J
        for (lo, hi), (lo2, _) in zip(ranges, ranges[1:]):
            assert lo <= hi == lo2                       # contiguous, disjoint, in order
        loads = [cost[lo:hi].sum() for lo, hi in ranges]
        # a contiguous split is within one design's cost of the even share
        assert max(loads) <= cost.sum() / world + cost.max() + 1e-6
    assert partition.design_ranges(np.zeros(6), 4) == [(0, 1), (1, 3), (3, 4), (4, 6)]
    with pytest.raises(ValueError):
        partition.design_ranges([1.0, -1.0], 2)


def _shard_worker(rank, world, port, out):
    import torch

    from oracle import mc as omc
    from paper_2005_10494_gb300 import partition
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prob = workloads.c3(n_scen=3, draws_range=(2e3, 2e4))
    lo, hi, sub = partition.shard_problem(prob, world, rank)
    cost = partition.design_cost(prob.n_draws, [prob.d_of(j) for j in range(prob.n_design)])
    ranges = partition.design_ranges(cost, world)
    assert (lo, hi) == ranges[rank]
    # the rank's hits (the oracle stands in for the rank's GPU here)
    designs = [{"Sigma": sub.sigmas[sub.design_scen[j]], "t": sub.t(j), "key": int(sub.keys[j]),
                "n_draws": int(sub.n_draws[j])} for j in range(sub.n_design)]
    hits = omc.mc_batch(designs, 9)["hits"].astype(np.int64) if designs else np.zeros(0, np.int64)
    full = partition.gather_designs(torch.as_tensor(hits), ranges)
    out[rank] = (full.numpy().tolist(), (lo, hi))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_ranks_shard_designs_and_gather_hits():
    """Two gloo ranks each evaluate their contiguous range of a batched
    uneven problem and all-gather the u64 hit counts; every rank then holds
    exactly the counts of one process evaluating all designs."""
    from oracle import mc as omc
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_shard_worker, args=(2, port, out), nprocs=2, start_method="spawn")
        h0, r0 = out[0]
        h1, r1 = out[1]
    prob = workloads.c3(n_scen=3, draws_range=(2e3, 2e4))
    designs = [{"Sigma": prob.sigmas[prob.design_scen[j]], "t": prob.t(j), "key": int(prob.keys[j]),
                "n_draws": int(prob.n_draws[j])} for j in range(prob.n_design)]
    ref = omc.mc_batch(designs, 9)["hits"].astype(np.int64)
    np.testing.assert_array_equal(h0, ref)
    np.testing.assert_array_equal(h1, ref)
    assert r0[0] == 0 and r0[1] == r1[0] and r1[1] == prob.n_design
    assert 0 < r0[1] < prob.n_design
