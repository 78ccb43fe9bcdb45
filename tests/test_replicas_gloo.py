"""The multi-rank (replicas) path of bench.py on CPU: two gloo ranks.  The
job's time is the slowest rank's, its value counts every rank's units, and the
reference arm prints from rank 0 only.  No GPU."""
import importlib.util
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        b = _bench()
        mine = [12.5, 40.0][rank]  # rank 1 is the slow one
        total = b.max_over_ranks(mine, world, "cpu")
        q.put((rank, total, b.job_value(1000.0, world, total / 10)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_value_with_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, total, value in got:
        assert total == 40.0  # every rank sees the slowest rank's time
        assert value == pytest.approx(1000.0 * 2 / (4.0 / 1e3))  # both ranks' units over that time


def test_single_rank_helpers():
    b = _bench()
    assert b.max_over_ranks(3.5, 1) == 3.5
    assert b.job_value(10.0, 1, 2.0) == pytest.approx(5000.0)


def test_reference_arm_prints_on_rank_zero_only(monkeypatch):
    b = _bench()
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--workload", "uniform64", "--steps", "1",
                                      "--warmup", "0"])
    out = io.StringIO()
    with redirect_stdout(out):
        assert b.main() == 0
    assert out.getvalue() == ""
