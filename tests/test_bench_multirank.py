"""The bench's multi-GPU logic on CPU with two gloo ranks: replicas only,
the timed region of the job ends with the slowest rank, and the whole-job
throughput is world_size replicas' work over that time; the reference arm
prints only on rank 0.  CPU only (torch.distributed gloo, 127.0.0.1)."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    mine = [12.5, 30.0][rank]  # this rank's timed-region length (ms)
    ms = bench.max_over_ranks(mine, dist, device="cpu")
    value = bench.job_value(world, 1024 * 1024 * 1000, 5, ms)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, ms, value))


def test_two_gloo_ranks_agree_on_the_slowest_time_and_the_job_value():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [30.0, 30.0]
    want = 2 * 1024 * 1024 * 1000 * 5 / 30e-3 / 1e6
    assert all(abs(r[2] - want) < 1e-9 * want for r in res)


def test_single_rank_value_and_no_reduction():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.job_value(1, 100, 2, 1.0) == pytest.approx(0.2)


def test_reference_arm_prints_only_on_rank_zero(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    buf = io.StringIO()
    with redirect_stdout(buf):
        rc = bench.run_reference(type("A", (), {"steps": 1, "warmup": 3})())
    assert rc == 0 and buf.getvalue() == ""


@pytest.mark.slow
def test_reference_arm_line_on_rank_zero(monkeypatch):
    """The oracle arm's JSON line (a bounded sample: one bench step of two
    leap-frog steps at 1024^2)."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(type("A", (), {"steps": 1, "warmup": 0})())
    line = json.loads(buf.getvalue())
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
