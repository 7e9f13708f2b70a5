"""The host side of the multi-GPU launch of the benchmark, on CPU: two ranks
of a gloo process group (the path runs independent replicas, one per GPU,
with no collective on the data path).  Each rank times its own steps; the
job's time is the largest of them, every rank receives it, and the
whole-job rate counts the units of every rank.  The reference arm runs on
rank 0 only: the other ranks return without work."""
import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(times[rank], dist, device="cpu")
        out.put((rank, ms, bench.whole_job_rate(world, 1000, ms)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [12.5, 20.0]
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in got] == [0, 1]
    for _, ms, rate in got:
        assert ms == 20.0
        assert rate == pytest.approx(2 * 1000 / 0.020)


def test_single_process_keeps_its_own_time():
    assert bench.max_over_ranks(7.0, None) == 7.0
    assert bench.whole_job_rate(1, 500, 250.0) == pytest.approx(2000.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(bench, "cpu_baseline", lambda **kw: called.append(kw) or {})
    assert bench.run_reference(None) is None
    assert not called and capsys.readouterr().out == ""
