"""The multi-GPU path is replicas only: ranks share no data, and the benchmark adds the
ranks' voxel-iterations and takes the slowest rank's time.  Checked with two gloo ranks
on the CPU."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    work, ms = bench.aggregate_ranks(dist, 1000.0 * (rank + 1), 10.0 + 5.0 * rank)
    out[rank] = (work, ms)
    # replicas draw different realizations (seed offset by rank) of the same workload recipe
    inp = bench.make_workload(rank)
    out[10 + rank] = float(inp.seeds[0, 0])
    members = bench.ensemble_members(rank)
    out[20 + rank] = (len(members), tuple(m.shape[0] for m in members), float(members[5].seeds[0, 0]))
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    import torch.multiprocessing as mp

    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == (3000.0, 15.0) and out[1] == (3000.0, 15.0)
    assert out[10] != out[11]
    # each rank steps its own 16-member ensemble of the same sizes
    assert out[20][:2] == out[21][:2] == (16, (64,) * 4 + (96,) * 4 + (128,) * 4 + (160,) * 4)
    assert out[20][2] != out[21][2]


def test_aggregate_without_process_group():
    import bench

    assert bench.aggregate_ranks(None, 5.0, 2.0) == (5.0, 2.0)
    with pytest.raises(SystemExit):
        bench.main_args(["--warmup", "1"])
