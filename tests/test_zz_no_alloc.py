"""gsync_bench_barrier_static: the barrier workload for callers that cannot allocate device
memory (a host callback, a loop that must not take cudaMalloc's implicit synchronization, a
plugin whose framework owns the device memory).  It keeps the barrier object and the slot
buffers in the library's own static device array and must produce exactly what the oracle
computes, and what the allocating entry point gsync_bench_barrier produces, call after call,
even though each call finds the previous call's contents -- possibly an object of another
kind -- in that array.

This file is collected last on purpose, and each test builds its own reference, so it passes
both alone in a fresh process and after every other test."""
import numpy as np
import pytest
import torch

from gpu_util import require_gpu
from oracle import calc

pytestmark = pytest.mark.gpu

# Every kind the entry point accepts, with the parameters the library uses for it.
ACCEPTED = [("atomic", 0), ("flag", 0), ("flag", 1), ("tree", 8), ("tree", 2), ("cluster", 2), ("cluster", 4),
            ("cluster", 8), ("sharded", 8), ("sharded", 32), ("split", 16 | 16 << 8), ("split", 4 | 2 << 8),
            ("count", 0), ("count", 8), ("count", 8 | 4 << 16), ("cluster", 4 | 1 << 4 | 8 << 8),
            ("cluster", 8 | 2 << 4), ("tree", 8 | 1 << 16), ("exchange", 8)]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def outputs(nblocks, rounds):
    z = lambda n: torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")
    return {"chk": z(rounds * nblocks), "mix": z(nblocks), "bad": z(nblocks), "status": z(1)}


def static_call(kind, nblocks, threads, rounds, param, full=True):
    from paper_1110_4623_gb300 import gsync as G
    o = outputs(nblocks, rounds)
    cluster = param & 0xF if kind == "cluster" else 1
    w = G.gsync_barrier_work(G.BARRIER_KINDS[kind], nblocks, threads, rounds, int(full), cluster, None,
                             G.ptr(o["chk"]) if full else None, G.ptr(o["mix"]), G.ptr(o["bad"]), G.ptr(o["status"]))
    rc = G.gsync_bench_barrier_static(w, param, 10_000_000_000)
    torch.cuda.synchronize()
    a = lambda t: t.cpu().numpy().view(np.uint32)
    out = {"mix": a(o["mix"]), "bad": a(o["bad"]), "status": int(a(o["status"])[0])}
    if full:
        out["chk"] = a(o["chk"])[:rounds * nblocks].reshape(rounds, nblocks)
    return rc, out


def allocating_call(kind, nblocks, threads, rounds, param):
    from paper_1110_4623_gb300 import runner
    return runner.BarrierRun(kind, nblocks, threads, rounds, full=True, param=param,
                             timeout_ns=10_000_000_000).run()


def same(got, want, keys=("chk", "mix", "bad")):
    return all(np.array_equal(got[k], want[k]) for k in keys)


@pytest.mark.parametrize("kind,param", ACCEPTED)
def test_two_calls_in_a_row_match_the_oracle_and_the_allocating_entry_point(kind, param):
    nblocks, threads, rounds = 64, 128, 700
    want = calc.barrier_full(nblocks, rounds)
    alloc = allocating_call(kind, nblocks, threads, rounds, param)
    assert alloc["rc"] == 0 and alloc["status"] == 0
    assert same(alloc, want)
    for _ in range(2):
        rc, got = static_call(kind, nblocks, threads, rounds, param)
        assert rc == 0 and got["status"] == 0
        assert same(got, want)
        assert same(got, alloc)


def test_each_call_finds_another_kind_in_the_array():
    # The array keeps the last call's object: a tree's node counters, a counting barrier's
    # 64-bit counter past zero, flag epochs.  Each call must rewrite all of it for its own kind.
    seq = [("tree", 2, 96), ("count", 8, 96), ("flag", 0, 96), ("sharded", 8, 64), ("count", 8 | 4 << 16, 64),
           ("atomic", 0, 96), ("cluster", 4, 96), ("split", 4 | 2 << 8, 64), ("cluster", 2 | 1 << 4, 96),
           ("tree", 8, 64), ("cluster", 4 | 2 << 4 | 8 << 8, 64), ("tree", 2 | 1 << 16, 96), ("count", 0, 96),
           ("exchange", 8, 96), ("exchange", 0, 64), ("count", 8, 96), ("exchange", 8, 96)]
    rounds = 300
    for kind, param, nblocks in seq:
        rc, got = static_call(kind, nblocks, 128, rounds, param)
        assert rc == 0 and got["status"] == 0, (kind, param)
        assert same(got, calc.barrier_full(nblocks, rounds)), (kind, param)


def test_consecutive_calls_with_different_shapes():
    # A larger call leaves epochs and slots behind; the next, smaller call must not see them.
    for nblocks, rounds in [(1184, 300), (16, 1000), (1184, 300)]:
        want = calc.barrier_full(nblocks, rounds)
        rc, got = static_call("atomic", nblocks, 128, rounds, 0)
        assert rc == 0 and got["status"] == 0
        assert same(got, want)


def test_default_barrier_at_the_full_grid_sampled():
    # The library's GB300 default barrier (counting, sleep parameter 8) at 1184 blocks in the
    # sampled fold that the bench times.
    nblocks, rounds = 1184, 1000
    want = calc.barrier_sampled(nblocks, rounds)
    for _ in range(2):
        rc, got = static_call("count", nblocks, 128, rounds, 8, full=False)
        assert rc == 0 and got["status"] == 0
        assert same(got, want, keys=("mix", "bad"))


def test_sizes_beyond_the_static_limit_and_the_two_die_kind_are_rejected():
    from paper_1110_4623_gb300 import gsync as G
    o = outputs(4097, 1)
    w = G.gsync_barrier_work(G.BARRIER_KINDS["atomic"], 4097, 128, 1, 1, 1, None, G.ptr(o["chk"]),
                             G.ptr(o["mix"]), G.ptr(o["bad"]), G.ptr(o["status"]))
    assert G.gsync_bench_barrier_static(w, 0, 0) == G.GSYNC_EINVAL
    # A tree of fan-in 2 over 4096 blocks needs more than the 96 KiB object region.
    w.nblocks = 4096
    w.kind = G.BARRIER_KINDS["tree"]
    assert G.gsync_bench_barrier_static(w, 2, 0) == G.GSYNC_EINVAL
    # The two-die barrier's init synchronizes the stream: refused before anything is enqueued.
    w.nblocks = 64
    w.kind = G.BARRIER_KINDS["die"]
    for param in (0, 1):
        assert G.gsync_bench_barrier_static(w, param, 0) == G.GSYNC_EINVAL
    torch.cuda.synchronize()
    assert int(o["status"].cpu()[0]) == 0
