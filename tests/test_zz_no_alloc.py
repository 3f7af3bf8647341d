"""gsync_bench_barrier_static: the barrier workload for callers that cannot allocate device
memory (a host callback, a loop that must not take cudaMalloc's implicit synchronization, a
plugin whose framework owns the device memory).  It keeps the barrier object and the slot
buffers in the library's own static device array and must produce exactly what the
allocating entry point gsync_bench_barrier produces, call after call, even though each call
finds the previous call's contents in that array.

This file is collected last on purpose, and each test builds its own reference, so it passes
both alone in a fresh process and after every other test."""
import numpy as np
import pytest
import torch

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def outputs(nblocks, rounds):
    z = lambda n: torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")
    return {"chk": z(rounds * nblocks), "mix": z(nblocks), "bad": z(nblocks), "status": z(1)}


def static_call(kind, nblocks, threads, rounds, param):
    from paper_1110_4623_gb300 import gsync as G
    o = outputs(nblocks, rounds)
    cluster = param if kind == "cluster" else 1
    w = G.gsync_barrier_work(G.BARRIER_KINDS[kind], nblocks, threads, rounds, 1, cluster, None,
                             G.ptr(o["chk"]), G.ptr(o["mix"]), G.ptr(o["bad"]), G.ptr(o["status"]))
    rc = G.gsync_bench_barrier_static(w, 0 if kind == "cluster" else param, 0)
    torch.cuda.synchronize()
    a = lambda t: t.cpu().numpy().view(np.uint32)
    return rc, {"chk": a(o["chk"])[:rounds * nblocks].reshape(rounds, nblocks), "mix": a(o["mix"]),
                "bad": a(o["bad"]), "status": int(a(o["status"])[0])}


def allocating_call(kind, nblocks, threads, rounds, param):
    from paper_1110_4623_gb300 import runner
    return runner.BarrierRun(kind, nblocks, threads, rounds, full=True, param=param).run()


@pytest.mark.parametrize("kind,param", [("atomic", 0), ("flag", 0), ("flag", 1), ("tree", 8), ("cluster", 4)])
def test_two_calls_in_a_row_match_the_allocating_entry_point(kind, param):
    nblocks, threads, rounds = 64, 128, 700
    want = allocating_call(kind, nblocks, threads, rounds, param)
    assert want["rc"] == 0 and want["status"] == 0
    for _ in range(2):
        rc, got = static_call(kind, nblocks, threads, rounds, param)
        assert rc == 0 and got["status"] == 0
        assert np.array_equal(got["chk"], want["chk"])
        assert np.array_equal(got["mix"], want["mix"])
        assert np.array_equal(got["bad"], want["bad"])


def test_consecutive_calls_with_different_shapes():
    # A larger call leaves epochs and slots behind; the next, smaller call must not see them.
    for nblocks, rounds in [(1184, 300), (16, 1000), (1184, 300)]:
        want = allocating_call("atomic", nblocks, 128, rounds, 0)
        rc, got = static_call("atomic", nblocks, 128, rounds, 0)
        assert rc == 0 and got["status"] == 0
        assert np.array_equal(got["chk"], want["chk"]) and np.array_equal(got["mix"], want["mix"])


def test_sizes_beyond_the_static_limit_are_rejected():
    from paper_1110_4623_gb300 import gsync as G
    o = outputs(4097, 1)
    w = G.gsync_barrier_work(G.BARRIER_KINDS["atomic"], 4097, 128, 1, 1, 1, None, G.ptr(o["chk"]),
                             G.ptr(o["mix"]), G.ptr(o["bad"]), G.ptr(o["status"]))
    assert G.gsync_bench_barrier_static(w, 0, 0) == G.GSYNC_EINVAL
    # A tree of fan-in 2 over 4096 blocks needs more than the 96 KiB object region.
    w.nblocks = 4096
    w.kind = G.BARRIER_KINDS["tree"]
    assert G.gsync_bench_barrier_static(w, 2, 0) == G.GSYNC_EINVAL
