"""Batched many-mutex kernel on the GPU against the oracle: per-key int64 sums and counts
exact (mutex definition applied to 4096 instances), and every barrier group's sampled slot
check exact (barrier definition applied per group)."""
import numpy as np
import pytest

from gpu_util import require_gpu
from oracle import calc
from paper_1110_4623_gb300 import inputs

pytestmark = pytest.mark.gpu

NKEYS, NB = 4096, 1184


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def make(nacq, cluster=1, rounds=100, policy=None, plain_launch=False, ncohort=64, block_threads=128):
    from paper_1110_4623_gb300 import autotune
    keys, adds, _ = inputs.batched_inputs(nacq, NKEYS, 1.1)
    cls = autotune.classify_keys(keys, NKEYS, NB)
    run = autotune.make_run(keys, adds, NKEYS, NB, 64, rounds, cluster, cls, block_threads=block_threads,
                            plain_launch=plain_launch, ncohort=ncohort)
    run.set_policy(policy or autotune.DEFAULT_POLICY)
    return run, keys, adds


def check(run, keys, adds, got, rounds):
    want = calc.batched_final(keys, adds, NKEYS)
    assert got["status"] == 0, got["status"]
    assert np.array_equal(got["sum"], want["sum"])
    assert np.array_equal(got["count"], want["count"])
    assert not got["bad"].any()
    for g, (st, sz) in enumerate(zip(run.group_start, run.group_sizes)):
        assert np.array_equal(got["mix"][st:st + sz], calc.barrier_sampled(int(sz), rounds)["mix"]), g
    covered = int(run.group_sizes.sum())
    assert not got["mix"][covered:].any()


@pytest.mark.parametrize("cluster", [1, 2, 4, 8])
def test_full_size_one_million_acquisitions(cluster):
    run, keys, adds = make(1_000_000, cluster=cluster)
    got = run.run()
    assert got["rc"] == 0
    check(run, keys, adds, got, 100)


@pytest.mark.parametrize("policy", [[("cas_spin", 0, 0)] * 3, [("cas_backoff", 64, 2048)] * 3,
                                    [("ticket", 128, 4000)] * 3,
                                    [("ticket", 0, 0), ("cas_backoff", 32, 1024), ("cas_spin", 0, 0)]])
def test_policies(policy):
    run, keys, adds = make(200_000, policy=policy, rounds=37)
    got = run.run()
    assert got["rc"] == 0
    check(run, keys, adds, got, 37)


@pytest.mark.parametrize("cluster,policy", [
    (4, [("cluster", 128, 4000), ("ticket", 256, 4000), ("ticket", 64, 2000)]),
    (2, [("cluster", 0, 0, 3), ("cluster", 128, 4000), ("cas_spin", 0, 0)]),
    (8, [("cluster", 128, 4000, 32767)] * 3),
    (1, [("cluster", 128, 4000)] * 3)])  # no clusters: the policy acts as the ticket lock
def test_cluster_cohort_policy(cluster, policy):
    # The cluster cohort lock for keys below 256 (the hot and warm keys of the Zipf stream),
    # with budgets 3, the default and the maximum; keys at or above 256 fall back to the
    # ticket lock.
    run, keys, adds = make(1_000_000 if cluster == 4 else 200_000, cluster=cluster, policy=policy, rounds=23)
    got = run.run()
    assert got["rc"] == 0
    check(run, keys, adds, got, 23)


@pytest.mark.parametrize("cluster,policy", [
    (1, [("ticket_carry", 0, 0)] * 3),
    (1, [("ticket_carry", 128, 4000)] * 3),
    (1, [("ticket_carry", 0, 0), ("cas_backoff", 32, 1024), ("ticket", 64, 2000)]),
    (4, [("ticket_carry", 0, 0), ("cluster", 128, 4000), ("ticket_carry", 64, 2000)])])
def test_ticket_carry_policy(cluster, policy):
    # The ticket lock whose turn record carries each key's count and sum, alone and beside
    # the other kinds, twice in a row on the same objects: the second launch starts from the
    # records the collect pass left (turns kept, counts and sums back at zero).
    run, keys, adds = make(1_000_000 if cluster == 1 and policy[1][0] == "ticket_carry" else 200_000,
                           cluster=cluster, policy=policy, rounds=29)
    for _ in range(2):
        got = run.run()
        assert got["rc"] == 0
        check(run, keys, adds, got, 29)


@pytest.mark.parametrize("cluster,policy,nacq,ncohort", [
    (1, [("cohort_carry", 0, 0)] * 3, 1_000_000, 64),
    (8, [("cohort_carry", 0, 0), ("cohort_carry", 8, 2000), ("ticket_carry", 0, 0)], 1_000_000, 64),
    (1, [("cohort_carry", 0, 0, 1), ("cohort_carry", 64, 2000, 3), ("cas_spin", 0, 0)], 200_000, 64),
    (4, [("cohort_carry", 0, 0, 32767), ("cluster", 128, 4000), ("ticket", 64, 2000)], 200_000, 64),
    (1, [("cohort_carry", 0, 0)] * 3, 200_000, 1),
    (2, [("cohort_carry", 0, 0)] * 3, 200_000, 0)])
def test_cohort_carry_policy(cluster, policy, nacq, ncohort):
    # The two-die cohort lock with carrying records on the hottest keys (keys below ncohort;
    # the rest of such a class use the carrying ticket lock): budgets 1 (every holder releases
    # the global lock), 3, the default and the maximum; beside the other kinds; one cohort
    # object, and none.  Twice in a row on the same objects: the collect pass returns every
    # counter and record to zero.
    run, keys, adds = make(nacq, cluster=cluster, policy=policy, rounds=31, ncohort=ncohort)
    for _ in range(2):
        got = run.run()
        assert got["rc"] == 0
        check(run, keys, adds, got, 31)


@pytest.mark.parametrize("cluster,policy,nacq", [
    (8, [("cluster_carry", 0, 0), ("cluster_carry", 8, 2000), ("ticket_carry", 0, 0)], 1_000_000),
    (2, [("cluster_carry", 0, 0, 1), ("cohort_carry", 0, 0), ("cas_spin", 0, 0)], 200_000),
    (4, [("cluster_carry", 64, 2000, 3), ("cluster", 128, 4000), ("cluster_carry", 0, 0, 32767)], 200_000),
    (1, [("cluster_carry", 0, 0)] * 3, 200_000)])  # no clusters: the carrying ticket lock
def test_cluster_carry_policy(cluster, policy, nacq):
    # The carrying cohort lock over thread-block clusters for keys below 256 (its local ticket
    # and record in block 0's shared memory; the rest fall back to the carrying ticket lock):
    # budgets 1, 3, the default and the maximum, beside the other kinds, twice in a row.
    run, keys, adds = make(nacq, cluster=cluster, policy=policy, rounds=27)
    for _ in range(2):
        got = run.run()
        assert got["rc"] == 0
        check(run, keys, adds, got, 27)


@pytest.mark.parametrize("cluster,policy,nacq,ncohort", [
    (8, [("cluster_die_carry", 0, 0), ("cluster_die_carry", 8, 2000), ("ticket_carry", 0, 0)], 1_000_000, 128),
    (2, [("cluster_die_carry", 0, 0, 1), ("cluster_carry", 0, 0), ("cas_spin", 0, 0)], 200_000, 64),
    (4, [("cluster_die_carry", 0, 0, 3), ("cohort_carry", 0, 0), ("cluster_die_carry", 64, 2000, 32767)],
     200_000, 128),
    (8, [("cluster_die_carry", 0, 0)] * 3, 200_000, 1),
    (1, [("cluster_die_carry", 0, 0)] * 3, 200_000, 64)])  # no clusters: the carrying ticket lock
def test_cluster_die_carry_policy(cluster, policy, nacq, ncohort):
    # The carrying lock over three levels (cluster, die, global) for keys below 256 and below
    # ncohort in a cluster launch, the rest on the carrying ticket lock: budgets 1, 3, the
    # default and the maximum (127 passes in a cluster, 255 on a die), beside the other kinds,
    # one cohort object, no clusters; twice in a row on the same objects.
    run, keys, adds = make(nacq, cluster=cluster, policy=policy, rounds=23, ncohort=ncohort)
    for _ in range(2):
        got = run.run()
        assert got["rc"] == 0
        check(run, keys, adds, got, 23)


@pytest.mark.parametrize("threads", [32, 160, 256])
@pytest.mark.parametrize("cluster", [1, 8])
def test_block_sizes(threads, cluster):
    # Blocks of up to 128 threads run the instantiation with 64 registers a thread, larger
    # ones the one with 32; both, with every carrying kind and the plain kinds beside them.
    pol = [("cluster_die_carry", 0, 0), ("cluster_carry", 0, 0), ("cohort_carry", 8, 2000)]
    run, keys, adds = make(200_000, cluster=cluster, policy=pol, rounds=19, block_threads=threads, ncohort=256)
    got = run.run()
    assert got["rc"] == 0
    check(run, keys, adds, got, 19)


def test_cluster_carry_graph_replay():
    import torch
    run, keys, adds = make(300_000, rounds=20, cluster=8,
                           policy=[("cluster_die_carry", 0, 0), ("cluster_carry", 0, 0), ("cohort_carry", 0, 0)])
    run.capture()
    for _ in range(3):
        run.replay()
        torch.cuda.synchronize()
        check(run, keys, adds, run.results(), 20)


def test_cohort_carry_graph_replay_and_policy_change():
    # Captured with clusters of 8 (the tuned launch's shape) and replayed; then the hot class
    # moves to the carrying ticket lock and back, which re-initialises the cohort objects.
    import torch
    pol = [("cohort_carry", 0, 0), ("cohort_carry", 8, 2000), ("ticket_carry", 0, 0)]
    run, keys, adds = make(300_000, rounds=20, cluster=8, policy=pol)
    run.capture()
    for _ in range(3):
        run.replay()
        torch.cuda.synchronize()
        check(run, keys, adds, run.results(), 20)
    run.set_policy([("ticket_carry", 0, 0)] * 3)
    check(run, keys, adds, run.run(), 20)
    run.set_policy(pol)
    check(run, keys, adds, run.run(), 20)


def test_ticket_carry_policy_change_and_graph_replay():
    # Switching a class from the plain ticket lock to the carrying one (and back) re-zeroes
    # the objects; a captured graph of the two kernels replays exactly.
    import torch
    run, keys, adds = make(300_000, rounds=20, plain_launch=True, policy=[("ticket", 0, 0)] * 3)
    check(run, keys, adds, run.run(), 20)
    run.set_policy([("ticket_carry", 0, 0), ("ticket_carry", 64, 2000), ("cas_spin", 0, 0)])
    run.capture()
    for _ in range(3):
        run.replay()
        torch.cuda.synchronize()
        check(run, keys, adds, run.results(), 20)
    run.set_policy([("ticket", 0, 0)] * 3)
    check(run, keys, adds, run.run(), 20)


def test_graph_capture_replays_exactly():
    import torch
    run, keys, adds = make(300_000, rounds=20, plain_launch=True)
    run.capture()
    for _ in range(2):
        run.replay()
        torch.cuda.synchronize()
        check(run, keys, adds, run.results(), 20)


@pytest.mark.parametrize("cluster", [2, 8])
def test_cluster_launch_graph_capture_replays_exactly(cluster):
    # The tuned configuration of the batched workload is a cluster launch (clusters of 8 for the
    # group barriers, the carrying ticket lock): captured as it is into a CUDA graph, with the
    # kernel that collects the carried sums, it replays exactly, launch after launch.
    import torch
    run, keys, adds = make(300_000, rounds=20, cluster=cluster,
                           policy=[("ticket_carry", 0, 0), ("ticket_carry", 64, 2000), ("ticket_carry", 0, 0)])
    run.capture()
    for _ in range(3):
        run.replay()
        torch.cuda.synchronize()
        check(run, keys, adds, run.results(), 20)


def test_cooperative_launch_in_capture_or_refused_cleanly():
    # Either the cooperative launch captures and replays exactly, or capture is refused with
    # an error status and the context stays usable.
    import torch
    from paper_1110_4623_gb300 import gsync as G
    run, keys, adds = make(100_000, rounds=10)
    try:
        run.capture()
    except G.GsyncError:
        torch.cuda.synchronize()
        got = run.run()
        check(run, keys, adds, got, 10)
        return
    run.replay()
    torch.cuda.synchronize()
    check(run, keys, adds, run.results(), 10)


def test_misaligned_cluster_groups_are_refused_on_device():
    from paper_1110_4623_gb300 import gsync as G
    from paper_1110_4623_gb300 import autotune, runner
    keys, adds, _ = inputs.batched_inputs(50_000, NKEYS, 1.1)
    cls = autotune.classify_keys(keys, NKEYS, NB)
    sizes = np.array([6, 10, 3, 8], dtype=np.int32)  # not multiples of 4
    run = runner.BatchedRun(keys, adds, NKEYS, NB, sizes, 10, cls, 3, cluster=4)
    run.set_policy(autotune.DEFAULT_POLICY)
    got = run.run()
    assert got["rc"] == 0 and got["status"] & G.GSYNC_STATUS_CONFIG
    want = calc.batched_final(keys, adds, NKEYS)
    assert np.array_equal(got["sum"], want["sum"])  # the lock work still completes


def test_cohort_objects_argument_checks():
    # A negative cohort count, or cohort objects asked for without a (128-byte aligned) buffer,
    # is refused before anything launches.
    from paper_1110_4623_gb300 import gsync as G
    run, _, _ = make(10_000, rounds=2)
    base = G.ptr(run.cohort_state)
    for n, ptr in ((-1, base), (4, None), (4, base + 64)):
        w = G.gsync_batched_work.from_buffer_copy(run.work)
        w.ncohort, w.cohort_state = n, ptr
        assert G.gsync_bench_batched(w) == G.GSYNC_EINVAL, (n, ptr)
    assert run.run()["rc"] == 0
