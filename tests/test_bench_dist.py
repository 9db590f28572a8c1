"""The bench's replica path on CPU: two gloo ranks agree on the slowest
rank's time and the whole-job rate; ranks other than 0 leave the reference
arm without work."""
import contextlib
import io
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # rank r took 100 + 50 r ms for 9 fields of 1000 vertices
        total, value = bench.job_rate(dist, 100.0 + 50.0 * rank, 9, 1000, world)
        q.put((rank, total, value))
    finally:
        dist.destroy_process_group()


def test_job_rate_takes_the_slowest_rank_over_gloo():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, total, value in got:
        assert total == 150.0
        assert value == pytest.approx(2 * 9 * 1000 / 0.150 / 1e6)


def test_job_rate_one_rank():
    import bench

    total, value = bench.job_rate(None, 200.0, 3, 10 ** 6, 1)
    assert total == 200.0 and value == pytest.approx(15.0)


def test_reference_arm_on_other_ranks_does_nothing(monkeypatch):
    import bench

    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.dist_env() == (2, 1, 1)
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        assert bench.run_reference(None) == 0
    assert out.getvalue() == ""
