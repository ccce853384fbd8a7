"""The multi-GPU mode is replicas only (the product needs no exchange between
the GPUs of one box): each rank runs the whole workload, the bench reports the
slowest rank's time and the work of all ranks.  This checks that host logic
(`bench.max_over_ranks`, `bench.job_gflops`) with world_size 2 on the gloo
backend, on CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as tdist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, "cpu")  # rank 1 is the slower one
        out.put((rank, ms, bench.job_gflops(1_000_000, ms, world)))
        tdist.barrier()
    finally:
        tdist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, gf in got:
        assert ms == 15.0  # every rank sees the slowest rank's time
        assert gf == pytest.approx(2.0 * 1_000_000 * 2 / 15e-3 / 1e9)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, "cpu") == 3.5
    assert bench.job_gflops(500, 1.0, 1) == pytest.approx(1e-3)
