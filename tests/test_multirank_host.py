"""The multi-rank (torchrun) path of bench.py on CPU: two gloo ranks, no GPU.

Each rank of a multi-GPU run advances its own replica of the grid (the path has no
data-path collective); the only exchange is the max-over-ranks of the timed region, and the
job's throughput counts every rank's updates over the slowest rank's time.
"""
import os
import socket

import pytest
import torch.multiprocessing as tmp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        t = bench.max_over_ranks(10.0 + 5.0 * rank)          # rank r took 10 + 5 r ms
        value = bench.job_mlups(world, 1000, 20, t / 1e3)
        ws, r, local = bench.dist_env()

        class A:
            workload = "tgv2d_4096"
            steps = 1
            warmup = 0
        # the reference arm runs on rank 0 only; other ranks return at once without work
        ref_rc = bench.run_reference(A()) if r != 0 else None
        q.put((rank, t, value, (ws, r, local), ref_rc))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(180)
def test_two_gloo_ranks_agree_on_max_time_and_job_value():
    ctx = tmp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(150)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(q.get() for _ in range(2))
    for rank, t, value, env, ref_rc in got:
        assert t == 15.0                                  # the slowest rank's time on every rank
        assert value == pytest.approx(2 * 1000 * 20 / 0.015 / 1e6)
        assert env == (2, rank, rank)
        assert ref_rc == (0 if rank == 1 else None)


def test_single_process_has_no_exchange():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_mlups(1, 4096 * 4096, 10, 1.0) == pytest.approx(4096 * 4096 * 10 / 1e6)
