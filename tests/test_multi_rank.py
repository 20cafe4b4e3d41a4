"""The multi-replica path on CPU (gloo, world size 2).

Designs are independent, so ranks shard them with no data-path collective:
each rank evaluates its own copy of the grid with its own stream keys (weak
scaling), and the only collectives are the timing barrier and the max of
the per-rank times.  This checks those host-side pieces; no GPU is used.
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
