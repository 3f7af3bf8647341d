"""Mutex workload on the GPU against the oracle (Section 5, "Mutex"): exact final counters
and data words, a valid grant log, and ticket-order grants for the fair kinds."""
import numpy as np
import pytest

from gpu_util import require_gpu
from oracle import calc
from paper_1110_4623_gb300 import inputs

pytestmark = pytest.mark.gpu

KINDS = ["cas_spin", "cas_backoff", "ticket", "sleep_queue", "cohort", "ring"]
FAIR = {"ticket", "sleep_queue", "ring"}


def grant_problems(kind, got, nblocks, acq, base=0, die_bases=(0, 0)):
    fifo = kind in FAIR
    return calc.check_grant_log(got["log"], got["ticket"] if fifo or kind == "cohort" else None, nblocks, acq,
                                fifo, ticket_base=base, per_die=kind == "cohort", die_bases=die_bases)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def backoff_for(kind):
    from paper_1110_4623_gb300 import runner
    return runner.backoff(min_ns=32, max_ns=2048) if kind == "cas_backoff" else None


def check(kind, nblocks, threads, acq, cs_words, max_delay=2000):
    from paper_1110_4623_gb300 import gsync as G
    from paper_1110_4623_gb300 import runner
    seed = inputs.mutex_seed(G.MUTEX_KINDS[kind], nblocks, cs_words)
    delay, add = inputs.mutex_inputs(nblocks, acq, seed, max_delay=max_delay)
    got = runner.MutexRun(kind, nblocks, threads, acq, cs_words, delay, add, bo=backoff_for(kind),
                          timeout_ns=10_000_000_000).run()
    want = calc.mutex_final(nblocks, acq, cs_words, add)
    assert got["rc"] == 0 and got["status"] == 0, got["status"]
    assert got["total"] == want["total"]
    assert np.array_equal(got["count"], want["count"])
    assert np.array_equal(got["data"], want["data"])
    assert grant_problems(kind, got, nblocks, acq) == []


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("nblocks", [148, 296, 592, 1184])
@pytest.mark.parametrize("cs_words", [0, 64, 1024])
def test_contention_sweep_full_size(kind, nblocks, cs_words):
    # 256 threads per block, 100 acquisitions per block, delays U{0..2000} cycles.
    check(kind, nblocks, 256, 100, cs_words)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("nblocks,threads,acq,cs_words", [(1, 32, 50, 7), (3, 64, 17, 33), (37, 96, 9, 1000),
                                                            (151, 256, 5, 1025), (5, 128, 20, 128), (9, 128, 20, 129),
                                                            (23, 256, 10, 600)])
def test_ragged_shapes(kind, nblocks, threads, acq, cs_words):
    # A section wider than the block (cs_words > threads) runs the kernel that batches up to
    # four loads per thread: exactly one word per thread, one word more, and partial passes.
    check(kind, nblocks, threads, acq, cs_words, max_delay=300)


@pytest.mark.parametrize("kind", KINDS)
def test_no_acquisitions(kind):
    from paper_1110_4623_gb300 import runner
    got = runner.MutexRun(kind, 8, 128, 0, 16, None, np.zeros(0, np.uint32)).run()
    assert got["status"] == 0 and got["total"] == 0 and not got["count"].any() and not got["data"].any()


@pytest.mark.parametrize("kind", KINDS)
def test_state_reused_across_launches(kind):
    # After a launch every lock is free again (ticket == turn, queue flag advanced), so the
    # same object serves the next launch.
    from paper_1110_4623_gb300 import runner
    delay, add = inputs.mutex_inputs(296, 20, 77, max_delay=100)
    mr = runner.MutexRun(kind, 296, 256, 20, 64, delay, add, bo=backoff_for(kind))
    want = calc.mutex_final(296, 20, 64, add)
    die_bases = (0, 0)
    for rep in range(3):
        got = mr.run()
        assert got["status"] == 0 and np.array_equal(got["data"], want["data"])
        base = rep * 296 * 20 if kind in FAIR else 0
        assert grant_problems(kind, got, 296, 20, base, die_bases) == []
        if kind == "cohort":
            c = calc.die_grant_counts(got["ticket"])
            die_bases = (die_bases[0] + c[0], die_bases[1] + c[1])


def test_host_buffer_entry_point():
    import ctypes
    import torch
    from paper_1110_4623_gb300 import gsync as G
    B, A, K = 592, 30, 64
    delay, add = inputs.mutex_inputs(B, A, 12345)
    n = B * A
    data = np.zeros(K, np.uint32); total = np.zeros(1, np.uint32); log = np.zeros(n, np.uint32)
    tick = np.zeros(n, np.uint32); count = np.zeros(B, np.uint32); status = np.zeros(1, np.uint32)
    p = lambda a: a.ctypes.data
    w = G.gsync_mutex_work(G.MUTEX_KINDS["ticket"], B, 256, A, K, 0, p(delay), p(add), p(data), p(total), p(log),
                           p(tick), p(count), p(status))
    nbytes = G.gsync_bench_mutex_workspace_bytes(w.kind, B, A, K)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    rc = G.gsync_bench_mutex_host(w, None, ws, nbytes)
    assert rc == 0 and status[0] == 0
    want = calc.mutex_final(B, A, K, add)
    assert total[0] == want["total"] and np.array_equal(data, want["data"])
    assert calc.check_grant_log(log, tick, B, A, fifo=True) == []


@pytest.mark.parametrize("cluster", [2, 4, 8])
@pytest.mark.parametrize("nblocks,cs_words", [(1184, 0), (1184, 64), (1184, 1024), (592, 64), (16, 7)])
def test_cluster_cohort_mutex(cluster, nblocks, cs_words):
    # The cohort protocol over thread-block clusters: the local lock lives in distributed
    # shared memory; each cluster's grants follow its own tickets.  At 1184 blocks this is the
    # contention sweep's full shape: 256 threads, 100 acquisitions per block, delays
    # U{0..2000} cycles, on the inputs the bench times (their seed), with the bench's backoff.
    from paper_1110_4623_gb300 import gsync as G
    from paper_1110_4623_gb300 import runner
    nb = nblocks - nblocks % cluster
    acq = 100 if nb == 1184 else 50
    seed = (inputs.mutex_seed(G.MUTEX_KINDS["cluster"], nb, cs_words) if nb == 1184
            else 31_000 + cluster + nb + cs_words)
    delay, add = inputs.mutex_inputs(nb, acq, seed)
    got = runner.MutexRun("cluster", nb, 256, acq, cs_words, delay, add, cluster=cluster, timeout_ns=10_000_000_000,
                          bo=runner.backoff(min_ns=128, max_ns=4000)).run()
    want = calc.mutex_final(nb, acq, cs_words, add)
    assert got["rc"] == 0 and got["status"] == 0, got["status"]
    assert got["total"] == want["total"] and np.array_equal(got["data"], want["data"])
    assert np.array_equal(got["count"], want["count"])
    assert calc.check_grant_log(got["log"], got["ticket"], nb, acq, False, group_bits=12) == []


@pytest.mark.parametrize("budget", [1, 3, 32767])
def test_cluster_cohort_budgets(budget):
    from paper_1110_4623_gb300 import runner
    delay, add = inputs.mutex_inputs(1184, 20, 41_000 + budget, max_delay=300)
    got = runner.MutexRun("cluster", 1184, 256, 20, 64, delay, add, cluster=8, budget=budget,
                          timeout_ns=10_000_000_000).run()
    want = calc.mutex_final(1184, 20, 64, add)
    assert got["status"] == 0 and np.array_equal(got["data"], want["data"])
    assert calc.check_grant_log(got["log"], got["ticket"], 1184, 20, False, group_bits=12) == []


@pytest.mark.parametrize("cluster", [2, 4, 8])
@pytest.mark.parametrize("nblocks,cs_words", [(1184, 0), (1184, 64), (1184, 1024), (592, 64), (16, 7), (8, 1025)])
def test_cluster_mcs_mutex(cluster, nblocks, cs_words):
    # The cluster cohort lock with an MCS queue per cluster (grants pushed into each waiter's
    # own shared memory), at the contention sweep's full shape and on ragged ones; its queue
    # order is the order of the tail swaps, so no ticket order is recorded.
    from paper_1110_4623_gb300 import gsync as G
    from paper_1110_4623_gb300 import runner
    nb = nblocks - nblocks % cluster
    acq = 100 if nb == 1184 else 50
    seed = (inputs.mutex_seed(G.MUTEX_KINDS["cluster_mcs"], nb, cs_words) if nb == 1184
            else 32_000 + cluster + nb + cs_words)
    delay, add = inputs.mutex_inputs(nb, acq, seed)
    got = runner.MutexRun("cluster_mcs", nb, 256, acq, cs_words, delay, add, cluster=cluster,
                          timeout_ns=10_000_000_000, bo=runner.backoff(min_ns=128, max_ns=4000)).run()
    want = calc.mutex_final(nb, acq, cs_words, add)
    assert got["rc"] == 0 and got["status"] == 0, got["status"]
    assert got["total"] == want["total"] and np.array_equal(got["data"], want["data"])
    assert np.array_equal(got["count"], want["count"])
    assert calc.check_grant_log(got["log"], None, nb, acq, False) == []


@pytest.mark.parametrize("budget", [1, 2, 3, 32767])
def test_cluster_mcs_budgets_and_reuse(budget):
    # Budgets from "always release the global lock" to the maximum, and the same object and
    # launch run twice: nodes live in shared memory and start afresh, the global lock goes on.
    from paper_1110_4623_gb300 import runner
    delay, add = inputs.mutex_inputs(1184, 20, 42_000 + budget, max_delay=300)
    mr = runner.MutexRun("cluster_mcs", 1184, 256, 20, 64, delay, add, cluster=8, budget=budget,
                         timeout_ns=10_000_000_000)
    want = calc.mutex_final(1184, 20, 64, add)
    for _ in range(2):
        got = mr.run()
        assert got["rc"] == 0 and got["status"] == 0 and np.array_equal(got["data"], want["data"])
        assert calc.check_grant_log(got["log"], None, 1184, 20, False) == []


def test_cluster_mcs_mutex_needs_a_cluster_size():
    from paper_1110_4623_gb300 import gsync as G
    from paper_1110_4623_gb300 import runner
    delay, add = inputs.mutex_inputs(64, 2, 5)
    mr = runner.MutexRun("cluster_mcs", 64, 128, 2, 8, delay, add, cluster=8)
    for bad in (1, 3, 16):  # not a cluster, does not divide 64, above 8
        mr.work.cluster = bad
        assert mr.launch() == G.GSYNC_EINVAL


def test_cluster_mutex_needs_a_cluster_size():
    from paper_1110_4623_gb300 import gsync as G
    from paper_1110_4623_gb300 import runner
    delay, add = inputs.mutex_inputs(64, 2, 5)
    mr = runner.MutexRun("cluster", 64, 128, 2, 8, delay, add, cluster=8)
    for bad in (1, 3, 16):  # not a cluster, does not divide 64, above 8
        mr.work.cluster = bad
        assert mr.launch() == G.GSYNC_EINVAL


def test_cohort_host_buffer_entry_point():
    import torch
    from paper_1110_4623_gb300 import gsync as G
    B, A, K = 1184, 20, 64
    delay, add = inputs.mutex_inputs(B, A, 4242)
    n = B * A
    data = np.zeros(K, np.uint32); total = np.zeros(1, np.uint32); log = np.zeros(n, np.uint32)
    tick = np.zeros(n, np.uint32); count = np.zeros(B, np.uint32); status = np.zeros(1, np.uint32)
    p = lambda a: a.ctypes.data
    w = G.gsync_mutex_work(G.MUTEX_KINDS["cohort"], B, 256, A, K, 0, p(delay), p(add), p(data), p(total), p(log),
                           p(tick), p(count), p(status))
    nbytes = G.gsync_bench_mutex_workspace_bytes(w.kind, B, A, K)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    assert G.gsync_bench_mutex_host(w, None, ws, nbytes) == 0 and status[0] == 0
    want = calc.mutex_final(B, A, K, add)
    assert total[0] == want["total"] and np.array_equal(data, want["data"])
    assert calc.check_grant_log(log, tick, B, A, fifo=False, per_die=True) == []


@pytest.mark.parametrize("budget", [1, 2, 64, 32767])
def test_cohort_budgets(budget):
    # budget 1: every acquisition goes through the global lock; 32767: passes stay on a die
    # for as long as it has waiters.
    from paper_1110_4623_gb300 import runner
    B, A, K = 592, 30, 64
    delay, add = inputs.mutex_inputs(B, A, 900 + budget, max_delay=500)
    mr = runner.MutexRun("cohort", B, 256, A, K, delay, add, budget=budget, timeout_ns=10_000_000_000)
    got = mr.run()
    want = calc.mutex_final(B, A, K, add)
    assert got["status"] == 0 and got["total"] == want["total"] and np.array_equal(got["data"], want["data"])
    assert grant_problems("cohort", got, B, A) == []


def test_cohort_local_locks_are_homed_on_their_dies():
    # Each die's local lock sits on a page that is near (short atomic round trip) to the SMs
    # of that die and far from the other die's SMs.
    import torch
    from paper_1110_4623_gb300 import gsync as G
    from paper_1110_4623_gb300 import runner
    die, ndies = runner.device_topology()
    if ndies < 2:
        pytest.skip("one-die GPU")
    mr = runner.MutexRun("cohort", 8, 128, 1, 1, None, np.zeros(8, np.uint32))
    hdr = mr.state[:64].view(torch.int32).cpu().numpy()
    sm = {d: int(np.flatnonzero(die == d)[0]) for d in (0, 1)}
    for d, word in ((0, hdr[10]), (1, hdr[11])):
        line = mr.state[4 * int(word):]
        near = runner.probe_rtt_by_line(sm[d], line, 1)[0]
        far = runner.probe_rtt_by_line(sm[1 - d], line, 1)[0]
        assert near + 60 < far, (d, near, far)


@pytest.mark.parametrize("spin", [1, 32, 4096])
def test_spin_then_sleep_policy(spin):
    # Section 5's futex stand-in: the CAS lock spins `spin` failed attempts, then backs off.
    from paper_1110_4623_gb300 import gsync as G
    from paper_1110_4623_gb300 import runner
    B, A, K = 1184, 30, 64
    delay, add = inputs.mutex_inputs(B, A, 700 + spin, max_delay=800)
    bo = runner.backoff(policy=G.BACKOFF_SPIN_THEN_SLEEP, min_ns=16, max_ns=512, spin=spin)
    got = runner.MutexRun("cas_backoff", B, 256, A, K, delay, add, bo=bo, timeout_ns=10_000_000_000).run()
    want = calc.mutex_final(B, A, K, add)
    assert got["status"] == 0 and got["total"] == want["total"] and np.array_equal(got["data"], want["data"])
    assert grant_problems("cas_backoff", got, B, A) == []


def test_ring_refuses_more_blocks_than_entries():
    # The ring holds one entry per waiting block: a grid larger than the ring is a config error.
    import torch
    from paper_1110_4623_gb300 import gsync as G
    from paper_1110_4623_gb300 import runner
    delay, add = inputs.mutex_inputs(64, 2, 5)
    mr = runner.MutexRun("ring", 64, 128, 2, 8, delay, add)
    small = torch.zeros(G.gsync_mutex_bytes(G.MUTEX_KINDS["ring"], 16), dtype=torch.uint8, device="cuda")
    G.check("init", G.gsync_mutex_init(small, small.numel(), G.MUTEX_KINDS["ring"], 16, None, 0))
    mr.state = small
    mr.reset()
    assert mr.launch() == 0
    assert mr.results()["status"] & G.GSYNC_STATUS_CONFIG
