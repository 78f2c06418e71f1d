"""The multi-process path of bench.py, on CPU: two gloo ranks (the pool's
GPU machines hold one GPU, so the NCCL path cannot run there). Checks the
max-over-ranks time, the whole-job value of the replicas and that the
reference arm does no work on ranks other than 0."""
import argparse
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    got = bench.max_over_ranks(10.0 + rank, world, device="cpu")
    value = bench.replica_mlups(1000, 10, 2.0, world)
    ref = bench.run_reference(argparse.Namespace(steps=1, warmup=0), rank) if rank != 0 else "skipped"
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got, value, ref))


def test_two_gloo_ranks_aggregate_like_the_bench():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    assert [r[0] for r in res] == [0, 1]
    assert all(r[1] == 11.0 for r in res)  # the slowest rank's time on every rank
    assert all(abs(r[2] - 2 * 1000 * 10 / 2.0 / 1e6) < 1e-15 for r in res)
    assert res[1][3] is None  # rank 1 of the reference arm returns without work
    assert all(p.exitcode == 0 for p in procs)


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.replica_mlups(40_000_000, 400, 0.8, 1) == pytest.approx(20_000.0)
