"""The replicas-only multi-GPU path of bench.py, on CPU: two gloo ranks, each
with its own elapsed time; the job's rate must use the slowest rank's time
and count every rank's work (weak scaling, no data-path collective)."""
import os

import pytest
import torch.multiprocessing as mp


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    elapsed = [1.5, 2.0][rank]
    mx = bench.reduce_max(elapsed)
    out[rank] = bench.job_rate(100, world, mx)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    port = 29500 + os.getpid() % 1000
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    # 2 ranks x 100 units over the slower rank's 2.0 s
    assert out[0] == pytest.approx(100.0) and out[1] == pytest.approx(100.0)


def test_single_rank_is_a_no_op():
    import bench
    assert bench.reduce_max(3.25) == 3.25
    assert bench.job_rate(10, 1, 2.0) == 5.0
