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


def test_oracle_sample_sizes():
    """The reference arm's volume crop shrinks with the number of timed calls
    (about 150 s of oracle work in all), never above the single-run crop and
    never below 32; batches and 2D images keep their samples."""
    import numpy as np
    b = _bench()
    sides = [b.volume_sample_side(c) for c in (1, 3, 8, 13, 23, 53, 103, 10 ** 6)]
    assert sides == sorted(sides, reverse=True)
    assert sides[0] == b.VOLUME_SAMPLE and sides[-1] == 32
    vol = np.zeros((64, 64, 64), np.float32)
    arrs, units, desc = b.oracle_sample("grf512cube", vol, side=40)
    assert arrs[0].shape == (40, 40, 40) and units == b.num_cells((40, 40, 40)) and "40^3" in desc
    img = np.zeros((16, 16), np.float32)
    arrs, units, _ = b.oracle_sample("grf1024", img)
    assert arrs[0] is img and units == b.num_cells(img.shape)
    imgs = np.zeros((8, 4, 4), np.float32)
    arrs, units, _ = b.oracle_sample("batch4096", imgs, batch_images=5)
    assert len(arrs) == 5 and units == 5


def test_traffic_lines_follow_the_source(tmp_path, monkeypatch):
    """bench.py quotes an ncu traffic figure only while the kernel's source file
    is the one the capture was taken on (its SHA-256 in the summary line)."""
    b = _bench()
    sha = b.kernel_source_sha("h1_scan")
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "dram_traffic_demo.md").write_text(
        "traffic h1_scan 1234 bytes per launch, source sha256 %s\n"
        "traffic h0_stencil 99 bytes per launch, source sha256 %s\n" % (sha, "0" * 64))
    src = tmp_path / "paper_2005_12692_gb300" / "csrc"
    src.mkdir(parents=True)
    for f in ("cr_h1.cu", "cr_uf.cu"):
        (src / f).write_bytes(open(os.path.join(ROOT, "paper_2005_12692_gb300", "csrc", f), "rb").read())
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    assert b.measured_traffic("h1_scan", "demo") == (1234, "profiles/dram_traffic_demo.md")
    val, why = b.measured_traffic("h0_stencil", "demo")
    assert val is None and why.startswith("stale")
    assert b.measured_traffic("dual_stencil", "demo") == (None, None)
    assert b.measured_traffic("h1_scan", "missing") == (None, None)
