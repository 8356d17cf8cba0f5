"""The multi-rank path of the benchmark (replicas, one process per GPU) on two CPU ranks with the
gloo backend: barriers, the max over ranks of the step time, and the whole-job throughput."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    from paper_2504_19163_gb300 import replicas as RP
    r, local, w = RP.rank_env()
    dist = RP.init("gloo")
    RP.barrier(dist)
    ms_local = 10.0 + 5.0 * r           # rank 1 is the slowest
    ms_max = RP.max_over_ranks(ms_local, dist)
    rate = RP.whole_job_rate(1000.0, w, ms_max)
    RP.barrier(dist)
    RP.finish(dist)
    out.put((r, w, ms_max, rate))


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, ms_max, rate in res:
        assert w == 2 and ms_max == 15.0
        assert rate == pytest.approx(1000.0 * 2 / 0.015)


def test_single_process_needs_no_group(monkeypatch):
    for k in ("RANK", "LOCAL_RANK", "WORLD_SIZE"):
        monkeypatch.delenv(k, raising=False)
    from paper_2504_19163_gb300 import replicas as RP
    assert RP.rank_env() == (0, 0, 1)
    assert RP.init("gloo") is None
    assert RP.max_over_ranks(3.5, None) == 3.5
    assert RP.whole_job_rate(100.0, 1, 50.0) == pytest.approx(2000.0)
