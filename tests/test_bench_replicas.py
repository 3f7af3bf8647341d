"""Multi-process path of the benchmark (replicas over ranks): the max-over-ranks reduction and
the whole-job throughput, on two gloo ranks on the CPU, and the reference arm's rank > 0 exit."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # Rank r reports a step of (r + 1) ms and a default-kind time of 10 (world - r) ms.
        step_ms, def_ms = bench.max_over_ranks([rank + 1.0, 10.0 * (world - rank)], world, device="cpu")
        q.put((rank, step_ms, def_ms, bench.replica_value(1000, def_ms, world)))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
@pytest.mark.parametrize("world", [2, 3])
def test_max_over_ranks_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=90) for _ in range(world))
    for p in procs:
        p.join(30)
        assert p.exitcode == 0
    for rank, step_ms, def_ms, value in got:
        assert step_ms == float(world)          # slowest step
        assert def_ms == 10.0 * world           # slowest default-kind run (rank 0)
        # 1000 units on each of `world` ranks in 10*world ms
        assert value == pytest.approx(1000 * world / (10.0 * world * 1e-3))


def test_single_rank_is_identity():
    assert bench.max_over_ranks([3, 4.5], 1) == [3.0, 4.5]
    assert bench.replica_value(500, 2.0, 1) == pytest.approx(250_000.0)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup, gpus = 1, 0, 2

    def boom(*a, **k):
        raise AssertionError("rank 1 must not run the oracle")

    monkeypatch.setattr(bench, "cpu_baseline", boom)
    bench.run_reference(Args())
    assert capsys.readouterr().out == ""
