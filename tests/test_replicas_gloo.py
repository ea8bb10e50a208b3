"""The N > 1 path of bench.py (independent replicas): two gloo ranks on the CPU check that the
job rate uses the slowest rank's time and the sum of the ranks' work."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 100.0 + 50.0 * rank
    res = bench.combine_ranks(world, pu_step=1000, steps=10, ms=ms_local, ms_e2e=2 * ms_local, device="cpu")
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_combine():
    world, port = 2, 29517
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms, ms_e2e, value, e2e = res[r]
        assert ms == 150.0 and ms_e2e == 300.0
        assert value == pytest.approx(2 * 1000 * 10 / 0.150)
        assert e2e == pytest.approx(2 * 1000 / 0.300)
