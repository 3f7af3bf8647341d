"""Condition variables on the GPU (future work in Section 7): a bounded producer/consumer
queue under one mutex and two condition variables.  Every item must be taken exactly once,
and the consumers' int64 sums must add up to the oracle's total."""
import numpy as np
import pytest

from gpu_util import require_gpu
from oracle import calc
from paper_1110_4623_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def check(producers, consumers, items, capacity, threads=128, bo=None, mutex="ticket", cluster=0):
    from paper_1110_4623_gb300 import runner
    n = producers * items
    value = inputs.condvar_inputs(n, inputs.SEED_CONDVAR ^ producers ^ (consumers << 12) ^ (capacity << 24))
    got = runner.CondVarRun(producers, consumers, items, capacity, value, block_threads=threads, bo=bo,
                            mutex=mutex, cluster=cluster).run()
    want = calc.condvar_final(value, producers, items, consumers)
    assert got["rc"] == 0 and got["status"] == 0, got["status"]
    assert np.array_equal(got["seen"], want["seen"]), int((got["seen"] != 1).sum())
    assert int(got["sum"].sum()) == want["total"]
    assert np.array_equal(got["count"], want["count"])
    # every item is put under one acquisition and taken under another; waits add re-locks
    assert got["acquisitions"] >= 2 * n


@pytest.mark.parametrize("producers,consumers,items,capacity", [
    (1, 1, 200, 1), (1, 1, 200, 7), (4, 4, 50, 2), (16, 4, 20, 3), (4, 16, 40, 1), (100, 10, 20, 8),
    (592, 592, 100, 16), (592, 592, 100, 1), (1000, 184, 92, 64)])
def test_producer_consumer_exactly_once(producers, consumers, items, capacity):
    check(producers, consumers, items, capacity)


@pytest.mark.parametrize("producers,consumers,items,capacity", [(1, 1, 100, 1), (592, 592, 100, 16), (16, 4, 20, 3)])
def test_producer_consumer_on_the_cohort_lock(producers, consumers, items, capacity):
    from paper_1110_4623_gb300 import runner
    check(producers, consumers, items, capacity, mutex="cohort", bo=runner.backoff(min_ns=128, max_ns=4000))


@pytest.mark.parametrize("mutex", ["cluster", "cluster_mcs"])
@pytest.mark.parametrize("producers,consumers,items,capacity,cluster", [
    (1, 1, 100, 1, 2), (592, 592, 100, 16, 4), (592, 592, 100, 1, 8), (16, 4, 20, 3, 4), (37, 11, 33, 5, 2)])
def test_producer_consumer_on_the_cluster_lock(mutex, producers, consumers, items, capacity, cluster):
    # Clusters mix producer and consumer blocks wherever producers is not a multiple of the
    # cluster size; the cohort passes the mutex between them inside the cluster (through block
    # 0's ticket lock, or the MCS queue's pushed grants).
    from paper_1110_4623_gb300 import runner
    check(producers, consumers, items, capacity, mutex=mutex, cluster=cluster,
          bo=runner.backoff(min_ns=128, max_ns=4000))


@pytest.mark.parametrize("mutex", ["cluster", "cluster_mcs"])
def test_cluster_lock_needs_a_cluster_size_that_divides_the_grid(mutex):
    from paper_1110_4623_gb300 import gsync as G
    from paper_1110_4623_gb300 import runner
    for bad in (1, 3, 16):  # not a cluster, does not divide 8 blocks, above 8
        r = runner.CondVarRun(4, 4, 4, 4, np.zeros(16, np.uint32), mutex=mutex, cluster=bad)
        assert r.launch() == G.GSYNC_EINVAL


def test_other_mutex_kinds_are_refused():
    from paper_1110_4623_gb300 import gsync as G
    from paper_1110_4623_gb300 import runner
    r = runner.CondVarRun(2, 2, 4, 4, np.zeros(8, np.uint32), mutex="cas_spin")
    assert r.launch() == G.GSYNC_EINVAL


def test_sleeping_waiters_and_ragged_threads():
    from paper_1110_4623_gb300 import runner
    check(37, 11, 33, 5, threads=96, bo=runner.backoff(min_ns=64, max_ns=2000))


def test_no_items():
    from paper_1110_4623_gb300 import runner
    got = runner.CondVarRun(8, 8, 0, 4, np.zeros(0, np.uint32)).run()
    assert got["rc"] == 0 and got["status"] == 0 and not got["count"].any()


def test_uneven_split_is_refused():
    from paper_1110_4623_gb300 import gsync as G
    from paper_1110_4623_gb300 import runner
    r = runner.CondVarRun(3, 2, 5, 4, np.zeros(15, np.uint32))  # 15 items over 2 consumers
    assert r.launch() == G.GSYNC_EINVAL


def test_critical_section_probe():
    # The probe of the queue's critical section: positive, longer than its frame, and refused
    # for a workspace that is too small.
    from paper_1110_4623_gb300 import gsync as G
    from paper_1110_4623_gb300 import runner
    body = runner.probe_condvar_cs(128, 1000)["ns_per_cs"]
    frame = runner.probe_condvar_cs(128, 1000, frame_only=True)["ns_per_cs"]
    assert 0 < frame < body < 100_000
    small = runner._state(256)
    assert G.gsync_probe_condvar_cs(128, 10, 0, small, 256)[0] == G.GSYNC_EINVAL
