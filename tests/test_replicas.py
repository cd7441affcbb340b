"""The multi-GPU path is replicas only (tiles are independent; no data exchange): the
host logic that combines the ranks of `bench.py --gpus N` -- distinct seeds per rank, the
maximum of the timings over ranks, the whole-job rate -- run as two gloo processes on the
CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # rank r's step and binning times: the job is as slow as the slowest replica
        got = bench.max_over_ranks([10.0 + rank, 5.0 - rank], world)
        dist.barrier()
        q.put((rank, got, bench.replica_seed(2, rank)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_maximum_and_distinct_seeds():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    env_root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    old = os.environ.get("PYTHONPATH", "")
    os.environ["PYTHONPATH"] = env_root + (os.pathsep + old if old else "")
    try:
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
        for p in procs:
            p.start()
        res = sorted(q.get(timeout=120) for _ in procs)
        for p in procs:
            p.join(timeout=60)
            assert p.exitcode == 0
    finally:
        os.environ["PYTHONPATH"] = old
    assert [r[1] for r in res] == [[11.0, 5.0], [11.0, 5.0]]
    assert res[0][2] != res[1][2]


def test_single_rank_and_job_rate():
    import bench
    assert bench.max_over_ranks([3.0, 4.0], 1) == [3.0, 4.0]
    # 2 ranks x 256 tiles in 5 ms of the slowest rank
    assert bench.job_rate(2, 256, 5.0) == pytest.approx(102400.0)
