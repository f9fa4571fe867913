"""The multi-rank path of bench.py on CPU (gloo, world size 2): the process
group comes up without a GPU, every rank passes the barrier, the timing is
the maximum over ranks, and the job throughput counts every rank's units
over that maximum.  Each rank processes independent images (weak scaling);
no collective touches the data path."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, local = bench.dist_setup(world)
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    mine = 10.0 + 5.0 * rank                      # this rank's timed milliseconds
    got = bench.reduce_max(mine, w, torch.device("cpu"))
    out[rank] = got
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_rank():
    world, port = 2, 29500 + os.getpid() % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        assert dict(out) == {0: 15.0, 1: 15.0}
    sys.path.insert(0, ROOT)
    import bench
    # 2 ranks x 20 steps x 4 Mpx each over the slowest rank's 15 ms
    assert abs(bench.job_throughput(2, 20, 4.0e6, 15.0) - 2 * 20 * 4.0 / 15e-3) < 1e-6
