"""The multi-rank (replica) path of bench.py on CPU ranks with gloo (world size 2)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # each replica reports its own time and units; the job takes the slowest rank
    tmax, usum, rate = bench.reduce_job(10.0 + 5.0 * rank, 1000 * (rank + 1), world)
    dist.barrier()
    dist.destroy_process_group()
    out[rank] = (tmax, usum, rate)


def test_replicas_take_max_time_and_sum_units():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    for r in range(world):
        tmax, usum, rate = out[r]
        assert tmax == pytest.approx(15.0)
        assert usum == pytest.approx(3000.0)
        assert rate == pytest.approx(3000.0 / 15e-3)


def test_reference_arm_other_ranks_do_no_work(monkeypatch):
    import bench
    called = []
    monkeypatch.setattr(bench, "oracle_sample", lambda *a, **k: called.append(1))
    monkeypatch.setattr(bench, "make_problem", lambda: None)

    class A:
        steps, warmup, gpus = 2, 1, 2
    bench.run_reference(A(), rank=1, world=2)
    assert not called


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_batch_shards_partition_the_members(world):
    """The independent plates of the batched workload are sharded over the
    ranks: every member on exactly one rank, and the work (PD nodes x m per
    round) balanced so that the slowest rank, which sets the job's time,
    carries little more than its share."""
    import bench
    from paper_2403_03605_gb300 import workloads as W
    work = [float(N) * 2 * m for N, _, _, m in W.batch_plates_draws(3605, 64)]
    shards = [bench.shard(work, r, world) for r in range(world)]
    flat = sorted(i for s in shards for i in s)
    assert flat == list(range(64))
    loads = [sum(work[i] for i in s) for s in shards]
    assert max(loads) <= 1.02 * sum(work) / world
    assert max(loads) / min(loads) <= 1.04
