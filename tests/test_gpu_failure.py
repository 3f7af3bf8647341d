"""Failure detection without a GPU fault: waits that can never succeed (a lock word that
nothing releases, a barrier counter that can never reach its target) end at the object's
timeout, or sooner when the host-side watchdog aborts the object, report it in the status
word, and leave the context usable."""
import numpy as np
import pytest
import torch

from gpu_util import require_gpu
from oracle import calc
from paper_1110_4623_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


# Lock word held by nobody (CAS kinds); a turn no ticket reaches (ticket); the first queue
# slot holding a ticket nobody has (queue lock).
@pytest.mark.parametrize("kind,line,value", [("cas_spin", 1, 1), ("cas_backoff", 1, 1), ("ticket", 2, 0x40000000),
                                             ("sleep_queue", 3, 99)])
def test_lock_that_is_never_released_times_out(kind, line, value):
    from paper_1110_4623_gb300 import gsync as G
    from paper_1110_4623_gb300 import runner
    delay, add = inputs.mutex_inputs(64, 4, 1, max_delay=0)
    mr = runner.MutexRun(kind, 64, 128, 4, 8, delay, add, bo=runner.backoff(min_ns=100, max_ns=1000),
                         timeout_ns=200_000_000)
    words = mr.state.view(torch.int32)
    words[line * 32] = value  # held by nobody / a turn that is never reached
    got = mr.run()
    assert got["rc"] == 0
    assert got["status"] & (G.GSYNC_STATUS_TIMEOUT | G.GSYNC_STATUS_ABORTED)
    assert got["status"] & G.GSYNC_STATUS_TIMEOUT
    assert got["total"] == 0 and not got["count"].any()
    assert G.gsync_object_abort_flag(mr.state)[1] != 0
    # The context is still usable: a fresh object runs to completion.
    ok = runner.MutexRun(kind, 64, 128, 4, 8, delay, add).run()
    assert ok["status"] == 0 and ok["total"] == 256


# The cluster forms compare the low 16 bits of the global turn with a cluster head's ticket:
# 0x8000 is a turn that none of the 256 acquisitions' tickets reaches.  The heads wait on the
# global lock; the blocks queued behind them in the cluster (on the shared-memory ticket or on
# the MCS queue) wait on a grant their head never passes.  Every wait must end.
@pytest.mark.parametrize("kind", ["cluster", "cluster_mcs"])
def test_cluster_lock_whose_global_turn_is_never_reached_times_out(kind):
    from paper_1110_4623_gb300 import gsync as G
    from paper_1110_4623_gb300 import runner
    delay, add = inputs.mutex_inputs(64, 4, 1, max_delay=0)
    mr = runner.MutexRun(kind, 64, 128, 4, 8, delay, add, timeout_ns=200_000_000, cluster=8)
    mr.state.view(torch.int32)[2 * 32] = 0x8000
    got = mr.run()
    assert got["rc"] == 0 and got["status"] & G.GSYNC_STATUS_TIMEOUT
    assert got["total"] == 0 and not got["count"].any()
    assert G.gsync_object_abort_flag(mr.state)[1] != 0
    ok = runner.MutexRun(kind, 64, 128, 4, 8, delay, add, cluster=8).run()
    assert ok["status"] == 0 and ok["total"] == 256


@pytest.mark.parametrize("kind", ["atomic", "cluster"])
def test_barrier_that_can_never_complete_times_out(kind):
    from paper_1110_4623_gb300 import gsync as G
    from paper_1110_4623_gb300 import runner
    br = runner.BarrierRun(kind, 64, 128, 10, full=False, param=2 if kind == "cluster" else 0,
                           timeout_ns=200_000_000)
    words = br.state.view(torch.int32)
    words[32] = 1_000_000  # arrival counter already past every target: nobody is last
    got = br.run()
    assert got["rc"] == 0 and got["status"] & G.GSYNC_STATUS_TIMEOUT
    ok = runner.BarrierRun(kind, 64, 128, 10, full=False, param=2 if kind == "cluster" else 0).run()
    assert ok["status"] == 0 and np.array_equal(ok["mix"], calc.barrier_sampled(64, 10)["mix"])


def test_semaphore_with_no_free_slot_times_out():
    from paper_1110_4623_gb300 import gsync as G
    from paper_1110_4623_gb300 import runner
    hold, add = inputs.sem_inputs(32, 2, 5, 0, 10)
    sr = runner.SemRun("ticket", 32, 128, 2, 1, hold, add, timeout_ns=200_000_000)
    sr.state.view(torch.int32)[32] = 1000  # count says 1000 holders: every wait must queue
    got = sr.run()
    assert got["status"] & G.GSYNC_STATUS_TIMEOUT


def _timed_watch(wd):
    import time
    t0 = time.monotonic()
    fired = wd.wait()
    return fired, time.monotonic() - t0


def test_watchdog_aborts_a_lock_that_is_never_released():
    # The object's own timeout is 3 s; the watchdog gives up after 0.1 s and the kernel must
    # return well before the timeout could end it.
    from paper_1110_4623_gb300 import gsync as G
    from paper_1110_4623_gb300 import runner
    delay, add = inputs.mutex_inputs(64, 4, 2, max_delay=0)
    mr = runner.MutexRun("ticket", 64, 128, 4, 8, delay, add, bo=runner.backoff(min_ns=100, max_ns=1000),
                         timeout_ns=3_000_000_000)
    mr.reset()
    mr.state.view(torch.int32)[2 * 32] = 0x40000000  # a turn no ticket reaches
    wd = runner.Watchdog([mr.state], 0.1)
    assert mr.launch() == 0
    fired, elapsed = _timed_watch(wd)
    got = mr.results()
    assert fired and elapsed < 1.5, elapsed
    assert got["status"] & G.GSYNC_STATUS_ABORTED and got["total"] == 0
    assert G.gsync_object_abort_flag(mr.state)[1] & 2  # set by the host
    ok = runner.MutexRun("ticket", 64, 128, 4, 8, delay, add).run()
    assert ok["status"] == 0 and ok["total"] == 256


def test_watchdog_aborts_a_cluster_queue_lock():
    # Heads wait on a global turn that is never reached, their MCS successors on records that
    # are never pushed; the watchdog's abort must end both kinds of wait.
    from paper_1110_4623_gb300 import gsync as G
    from paper_1110_4623_gb300 import runner
    delay, add = inputs.mutex_inputs(64, 4, 2, max_delay=0)
    mr = runner.MutexRun("cluster_mcs", 64, 128, 4, 8, delay, add, timeout_ns=3_000_000_000, cluster=8)
    mr.reset()
    mr.state.view(torch.int32)[2 * 32] = 0x8000
    wd = runner.Watchdog([mr.state], 0.1)
    assert mr.launch() == 0
    fired, elapsed = _timed_watch(wd)
    got = mr.results()
    assert fired and elapsed < 1.5, elapsed
    assert got["status"] & G.GSYNC_STATUS_ABORTED and got["total"] == 0
    ok = runner.MutexRun("cluster_mcs", 64, 128, 4, 8, delay, add, cluster=8).run()
    assert ok["status"] == 0 and ok["total"] == 256


def test_watchdog_aborts_a_barrier_that_cannot_complete():
    from paper_1110_4623_gb300 import gsync as G
    from paper_1110_4623_gb300 import runner
    br = runner.BarrierRun("atomic", 64, 128, 10, full=False, timeout_ns=3_000_000_000)
    br.status.zero_()
    br.state.view(torch.int32)[32] = 1_000_000  # arrival counter already past every target: nobody is last
    wd = runner.Watchdog([br.state], 0.1)
    assert br.launch() == 0
    fired, elapsed = _timed_watch(wd)
    torch.cuda.synchronize()
    assert fired and elapsed < 1.5, elapsed
    assert int(br.status.cpu()[0]) & G.GSYNC_STATUS_ABORTED


def test_watchdog_stays_quiet_on_work_that_finishes():
    from paper_1110_4623_gb300 import runner
    delay, add = inputs.mutex_inputs(296, 20, 3)
    mr = runner.MutexRun("cluster", 296, 256, 20, 64, delay, add, cluster=4)
    mr.reset()
    wd = runner.Watchdog([mr.state], 10.0)
    assert mr.launch() == 0
    fired, _ = _timed_watch(wd)
    got = mr.results()
    assert not fired and got["status"] == 0 and got["total"] == 296 * 20
