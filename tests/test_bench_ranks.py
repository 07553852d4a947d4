"""Host logic of bench.py's N-process run, on CPU with the gloo backend
(world size 2): the timed region's length is the maximum over ranks (the
job ends with its slowest rank), and under torchrun the reference arm
runs on rank 0 alone (the other ranks exit without work or output)."""

import contextlib
import io
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


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        out.put((rank, bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")))
    finally:
        dist.destroy_process_group()


def test_timed_region_is_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == {0: 15.0, 1: 15.0}


def test_one_process_keeps_its_time():
    import bench
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5


def test_reference_arm_runs_on_rank_0_only(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(bench.argparse.Namespace(workload="ellipsoid20480_bmbie_d2_hard_plane", cpu_rows=2,
                                                     warmup=1, steps=1, precision="split"))
    assert buf.getvalue() == ""
