"""The bench's multi-rank path on CPU: two gloo ranks agree on the slowest
rank's time and the whole-job (weak-scaling) rate; the reference arm prints
on rank 0 only."""
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


def _rank(rank, world, port, out):
    import sys

    import torch.distributed as dist

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank)
    rate = bench.weak_scaling_rate(64, 100, ms, world)
    out.put((rank, ms, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time_and_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]
    # 2 ranks x 64 frames x 100 steps in the slowest rank's 15 ms
    assert res[0][2] == res[1][2] == pytest.approx(2 * 64 * 100 / 0.015)


def test_single_process_identity():
    import bench

    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.weak_scaling_rate(64, 10, 1000.0, 1) == pytest.approx(640.0)
