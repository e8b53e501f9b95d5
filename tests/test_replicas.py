"""Host logic of runs on several GPUs, on CPU: two gloo ranks (one process each) stand in for
two GPUs; the shares of independent items and the timing reduction are checked on every rank."""
import os
import socket

import pytest

from paper_1812_11626_gb300 import replicas as R


def test_shard_covers_items_once():
    for n in (0, 1, 7, 256):
        for world in (1, 2, 3, 8):
            parts = [R.shard(n, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
            sizes = [e - b for b, e in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        R.shard(10, 2, 2)


def test_single_process_reduction_is_identity():
    assert R.reduce_timing(12.5, 400) == (12.5, 400.0)
    assert R.throughput(500.0, 1000) == pytest.approx(2000.0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b, e = R.shard(256, rank, world)
        elapsed = 100.0 + 50.0 * rank          # rank 1 is the slower one
        ms, units = R.reduce_timing(elapsed, e - b, dist, "cpu")
        thr = R.throughput(elapsed, e - b, dist, "cpu")
        out.put((rank, b, e, ms, units, thr))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_max_time_and_total_work():
    import torch.multiprocessing as mp
    world = 2
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
    (r0, b0, e0, ms0, u0, t0), (r1, b1, e1, ms1, u1, t1) = res
    assert (b0, e0, b1, e1) == (0, 128, 128, 256)
    assert ms0 == ms1 == 150.0           # the slowest rank's time on every rank
    assert u0 == u1 == 256.0             # all ranks' work
    assert t0 == t1 == pytest.approx(256.0 / 0.150)
