"""The multi-GPU path of bench.py is independent replicas: every rank renders
its own copy of the workload, the job's time is the slowest rank's (max over
ranks) and its throughput the units of all ranks over that time.  Checked with
two gloo ranks on the CPU (no GPU, no collective on the data path)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [2.5, 4.0, 3.0][rank]  # rank 1 is the slowest
    ms_max = bench.max_over_ranks(ms, world, torch.device("cpu"))
    value = bench.job_throughput(1000.0, world, ms_max)
    w, r, l = bench.dist_setup()
    out.put((rank, ms_max, value, (w, r, l)))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_max_over_ranks_and_job_throughput(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slowest = max([2.5, 4.0, 3.0][:world])
    for rank, ms_max, value, env in res:
        assert ms_max == slowest
        assert value == pytest.approx(world * 1000.0 / (slowest * 1e-3))
        assert env == (world, rank, rank)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1, torch.device("cpu")) == 3.5
    assert bench.job_throughput(10.0, 1, 2.0) == pytest.approx(5000.0)


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the oracle arm runs on rank 0 alone; other ranks return
    at once without work."""
    import bench

    class Args:
        warmup, steps = 3, 5
    assert bench.run_reference(Args(), world=2, rank=1) is None
