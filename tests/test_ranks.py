"""The N > 1 bench path on CPU: world_size-2 gloo process groups (no GPU).
Replicas report the slowest rank's time and the sum of all ranks' checks;
the reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _aggregate_worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, checks = bench.aggregate_over_ranks(100.0 + 50.0 * rank, 1000 * (rank + 1), world, "cpu")
    out.put((rank, ms, checks))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_report_slowest_time_and_all_checks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    mp.start_processes(_aggregate_worker, args=(2, port, q), nprocs=2, join=True, start_method="spawn")
    got = sorted(q.get() for _ in range(2))
    for rank, ms, checks in got:
        assert ms == 150.0 and checks == 3000.0


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.aggregate_over_ranks(12.5, 7, 1, "cpu") == (12.5, 7.0)


def _reference_worker(rank, world, out):
    import contextlib
    import io
    import bench

    class A:
        pass
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(A(), rank, world)       # rank 1 returns at once
    out.put((rank, buf.getvalue()))


def test_reference_arm_runs_on_rank_zero_only():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_reference_worker, args=(1, 2, q))
    p.start()
    p.join(60)
    assert p.exitcode == 0
    rank, text = q.get()
    assert rank == 1 and text == ""


def test_shard_bounds_cover_every_program_once():
    import bench
    for count in (0, 1, 7, 256, 257):
        for world in (1, 2, 3, 8):
            blocks = [bench.shard_bounds(count, r, world) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == count
            assert all(blocks[r][1] == blocks[r + 1][0] for r in range(world - 1))
            sizes = [hi - lo for lo, hi in blocks]
            assert max(sizes) - min(sizes) <= 1


def _batch_totals_worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi = bench.shard_bounds(10, rank, world)
    # a rank's batched-solve figures: its block's solved count and its time
    t, solved = bench.aggregate_over_ranks(1.5 + rank, hi - lo, world, "cpu")
    out.put((rank, t, solved))
    dist.barrier()
    dist.destroy_process_group()


def test_batched_blocks_aggregate_to_the_whole_job():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    mp.start_processes(_batch_totals_worker, args=(2, _free_port(), q), nprocs=2, join=True, start_method="spawn")
    for rank, t, solved in sorted(q.get() for _ in range(2)):
        assert t == 2.5 and solved == 10.0
