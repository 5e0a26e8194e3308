"""The multi-rank path of bench.py on CPU: two gloo ranks take the maximum
of their timings and report the steps of all ranks over the slowest time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    r, w, local, dist = bench.dist_setup()
    ms = 100.0 + 50.0 * r                       # rank 1 is the slow one
    mx = bench.reduce_max(ms, dist)
    bench.barrier(dist)
    steps = 7
    q.put((r, w, mx, w * steps / (mx * 1e-3)))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    for r, w, mx, value in res:
        assert w == 2 and mx == pytest.approx(150.0)
        assert value == pytest.approx(2 * 7 / 0.150)
