"""The multi-GPU form of bench.py is N independent replicas: each rank times its own jobs, the
job time is the slowest rank's (max over ranks), and the whole-job value counts every rank's
units.  That host logic runs here as two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [120.0, 150.0][rank]  # rank 1 is the slow replica
        worst = bench.max_over_ranks(local_ms)
        dist.barrier()
        q.put((rank, bench.dist_env(), worst, bench.replica_throughput(1000.0, world, worst)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[1] for o in out] == [(0, 0, 2), (1, 1, 2)]
    assert all(o[2] == 150.0 for o in out)
    # 1000 units per rank, 2 ranks, 150 ms: 2000 / 0.15 s
    assert out[0][3] == pytest.approx(2000.0 / 0.150)


def test_single_process_is_its_own_maximum():
    import bench

    assert bench.max_over_ranks(42.5) == 42.5
    assert bench.replica_throughput(10.0, 1, 100.0) == pytest.approx(100.0)
