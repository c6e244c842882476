"""The benchmark's multi-rank host logic on CPU (gloo, world size 2).

Each rank resamples an independent instance, so the data path has no
collective; the only exchange is the timing reduction (max over ranks) that
makes the whole-job rate.  Checked here without a GPU.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        env = bench.dist_env()
        t = bench.max_over_ranks(10.0 + 5.0 * rank, dist, torch.device("cpu"))
        q.put((rank, env, bench.rank_instance(rank), t))
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_reduction_and_instances():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [(2, 0, 0), (2, 1, 1)]
    assert len({r[2] for r in res}) == ws          # independent Philox streams
    assert all(r[3] == 15.0 for r in res)          # every rank sees the slowest rank's time


def test_whole_job_rate_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, None, None) == 3.5
    # 2 ranks x 4096 samples x 10 steps in 20 ms
    assert bench.whole_job_rate(2, 4096, 10, 20.0) == pytest.approx(2 * 4096 * 10 / 0.02)
