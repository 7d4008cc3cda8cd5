"""Multi-GPU host logic on CPU: ranks shard independent streams (disjoint
seeds, no data-path collective) and the benchmark reduces only its timing
(max over ranks) and counts (sum over ranks).  world_size 2, gloo backend."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seeds = bench.stream_seeds(rank, 4)
    elapsed = 1.0 + rank          # rank 1 is the slow one
    cells = 100.0 * (rank + 1)
    mx = bench.reduce_over_ranks(elapsed, "max", world)
    sm = bench.reduce_over_ranks(cells, "sum", world)
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    out[rank] = (mx, sm, gathered)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_streams_and_reduce_timing():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        mx, sm, gathered = res[rank]
        assert mx == 2.0 and sm == 300.0
        assert not set(gathered[0]) & set(gathered[1])      # disjoint streams
        assert len(gathered[0]) == len(gathered[1]) == 4     # same work per rank: weak scaling


def test_single_rank_reduction_is_identity():
    import bench
    assert bench.reduce_over_ranks(3.5, "max", 1) == 3.5
    assert bench.stream_seeds(0, 3) == [1000, 1001, 1002]
