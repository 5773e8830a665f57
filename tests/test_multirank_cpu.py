"""The multi-rank timing of bench.py on CPU: two gloo ranks (each scanning its own data, no
data-path collective) agree on the slowest rank's time, and the job's throughput counts the
bytes of both ranks over that time."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 * (rank + 1)  # rank 1 is the slow one
        got = bench.max_over_ranks(local_ms, dist, "cpu")
        q.put((rank, got, bench.job_gbs(1 << 30, world, 4, got)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [20.0, 20.0]
    # 2 ranks x 4 steps x 1 GiB in 20 ms
    assert out[0][2] == pytest.approx(2 * 4 * (1 << 30) / 0.020 / 1e9)


def test_one_rank_needs_no_process_group():
    import bench

    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_gbs(10**9, 1, 2, 1000.0) == pytest.approx(2.0)
