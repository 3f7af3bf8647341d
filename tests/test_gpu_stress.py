"""Seeded repetitions of the GB300 designs across shapes and parameters (cohort and cluster
cohort mutexes in both forms, counting barrier and the counting forms of the tree and cluster
barriers, the exchange barrier, ticket-window semaphore, condition variables, serving loop),
each checked exactly against the oracle: a net for races that one shape per test could miss."""
import numpy as np
import pytest

from gpu_util import require_gpu
from oracle import calc
from paper_1110_4623_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.mark.parametrize("i", range(30))
def test_cohort_mutex_repeated(i):
    from paper_1110_4623_gb300 import runner
    B = [148, 296, 592, 1184, 1216][i % 5]
    K = [0, 64, 1024][i % 3]
    budget = [1, 2, 16, 64, 4096][i % 5]
    delay, add = inputs.mutex_inputs(B, 20, 10_000 + i, max_delay=[0, 300, 2000][i % 3])
    got = runner.MutexRun("cohort", B, 256, 20, K, delay, add, budget=budget, timeout_ns=10**10,
                          bo=runner.backoff(min_ns=[0, 128][i % 2], max_ns=4000)).run()
    want = calc.mutex_final(B, 20, K, add)
    assert got["status"] == 0 and got["total"] == want["total"] and np.array_equal(got["data"], want["data"])
    assert calc.check_grant_log(got["log"], got["ticket"], B, 20, False, per_die=True) == []


@pytest.mark.parametrize("i", range(30))
def test_cluster_mutex_repeated(i):
    from paper_1110_4623_gb300 import runner
    c = [2, 4, 8][i % 3]
    B = [16, 296, 592, 1184, 1184][i % 5] // c * c
    K = [0, 64, 1024, 7][i % 4]
    budget = [1, 2, 64, 4096, 32767][i % 5]
    delay, add = inputs.mutex_inputs(B, 20, 20_000 + i, max_delay=[0, 300, 2000][i % 3])
    got = runner.MutexRun("cluster", B, 256, 20, K, delay, add, budget=budget, cluster=c, timeout_ns=10**10,
                          bo=runner.backoff(min_ns=[0, 128][i % 2], max_ns=4000)).run()
    want = calc.mutex_final(B, 20, K, add)
    assert got["status"] == 0 and got["total"] == want["total"] and np.array_equal(got["data"], want["data"])
    assert calc.check_grant_log(got["log"], got["ticket"], B, 20, False, group_bits=12) == []


@pytest.mark.parametrize("i", range(30))
def test_cluster_mcs_mutex_repeated(i):
    # The MCS form of the cluster cohort lock over grids, sections, budgets, delays and sleeps
    # (its queue order is the tail swaps', so only the grant log's validity is checked).
    from paper_1110_4623_gb300 import runner
    c = [8, 2, 4][i % 3]
    B = [16, 296, 592, 1184, 1184][i % 5] // c * c
    K = [0, 64, 1024, 7][i % 4]
    budget = [1, 2, 64, 4096, 32767][i % 5]
    delay, add = inputs.mutex_inputs(B, 20, 21_000 + i, max_delay=[0, 300, 2000][i % 3])
    got = runner.MutexRun("cluster_mcs", B, 256, 20, K, delay, add, budget=budget, cluster=c, timeout_ns=10**10,
                          bo=runner.backoff(min_ns=[0, 128][i % 2], max_ns=4000)).run()
    want = calc.mutex_final(B, 20, K, add)
    assert got["status"] == 0 and got["total"] == want["total"] and np.array_equal(got["data"], want["data"])
    assert calc.check_grant_log(got["log"], None, B, 20, False) == []


@pytest.mark.parametrize("i", range(30))
def test_window_semaphore_repeated(i):
    from paper_1110_4623_gb300 import runner
    B = [1, 37, 296, 592, 1184][i % 5]
    n = [1, 2, 4, 16, 64, 1000][i % 6]
    hold, add = inputs.sem_inputs(B, 30, 30_000 + i, [0, 100][i % 2], [500, 5000][i % 2])
    bo = runner.backoff(min_ns=[0, 16, 128][i % 3], max_ns=2000) if i % 3 else None
    got = runner.SemRun("window", B, 128, 30, n, hold, add, bo=bo, timeout_ns=10**10).run()
    want = calc.sem_final(B, 30, n, add)
    assert got["status"] == 0 and np.array_equal(got["count"], want["count"]) and got["tally"] == want["tally"]
    assert 1 <= got["max_occ"] <= min(n, B) and got["occupancy"] == 0
    if n == 1:
        assert got["total"] == want["total"]


@pytest.mark.parametrize("i", range(30))
def test_counting_barrier_repeated(i):
    from paper_1110_4623_gb300 import runner
    B = [2, 7, 64, 148, 600, 1184, 1216][i % 7]
    param = [0, 8, 16, 8 | 4 << 16, 1023][i % 5]
    got = runner.BarrierRun("count", B, 128, 300, full=True, param=param, timeout_ns=10**10).run()
    want = calc.barrier_full(B, 300)
    assert got["status"] == 0 and not got["bad"].any()
    assert np.array_equal(got["chk"], want["chk"]) and np.array_equal(got["mix"], want["mix"])


@pytest.mark.parametrize("i", range(24))
def test_counting_forms_of_tree_and_cluster_barriers_repeated(i):
    # The tree's counting form (node counters that only grow) and the cluster barrier's
    # counting forms (leaders on a growing counter; form 2 releases the cluster through a
    # second cluster barrier), over grids, fan-ins, cluster sizes and sleeps, full fold.
    from paper_1110_4623_gb300 import runner
    if i % 2:
        c = [1, 2, 4, 8][i // 2 % 4]
        B = [8, 64, 296, 1184][i // 2 % 4 if c != 8 else 3] // c * c
        kind, param = "cluster", c | (1 + (i // 2) % 2) << 4 | [0, 8, 64][i % 3] << 8
    else:
        B = [1, 3, 64, 150, 600, 1184][i // 2 % 6]
        kind, param = "tree", [2, 3, 8, 32, 64, 1024][i // 2 % 6] | 1 << 16
    got = runner.BarrierRun(kind, B, 128, 300, full=True, param=param, timeout_ns=10**10).run()
    want = calc.barrier_full(B, 300)
    assert got["status"] == 0 and not got["bad"].any(), (kind, hex(param), B)
    assert np.array_equal(got["chk"], want["chk"]) and np.array_equal(got["mix"], want["mix"])


@pytest.mark.parametrize("i", range(16))
def test_exchange_barrier_repeated(i):
    # The exchange barrier (slot values carried in fence-free arrivals) over grids and sleeps,
    # in the full fold (every block reads every record each round) and the sampled one, and
    # launched twice on the same object (global epochs keep growing).
    from paper_1110_4623_gb300 import runner
    B = [1, 2, 7, 64, 150, 296, 600, 1184][i % 8]
    param = [0, 8, 64, 1023][i % 4]
    full = B <= 296 or i % 2 == 0
    br = runner.BarrierRun("exchange", B, [32, 128, 256][i % 3], 200, full=full, param=param, timeout_ns=10**10)
    for _ in range(2):
        got = br.run()
        assert got["status"] == 0 and not got["bad"].any(), (B, param, full)
        want = calc.barrier_full(B, 200) if full else calc.barrier_sampled(B, 200)
        assert np.array_equal(got["mix"], want["mix"])
        if full:
            assert np.array_equal(got["chk"], want["chk"])


@pytest.mark.parametrize("i", range(20))
def test_condvar_repeated(i):
    from paper_1110_4623_gb300 import runner
    P, C, items = [(1, 1, 50), (8, 8, 20), (100, 50, 10), (592, 592, 40), (1100, 100, 10)][i % 5]
    v = inputs.condvar_inputs(P * items, 777 + i)
    mutex = ["ticket", "cohort", "cluster", "cluster_mcs"][i % 4]  # every grid here is even: clusters of 2 fit
    got = runner.CondVarRun(P, C, items, [1, 2, 16, 64][i % 4], v, mutex=mutex,
                            cluster=2 if mutex in ("cluster", "cluster_mcs") else 0,
                            bo=runner.backoff(min_ns=[0, 64][i % 2], max_ns=2000)).run()
    want = calc.condvar_final(v, P, items, C)
    assert got["rc"] == 0 and got["status"] == 0
    assert np.array_equal(got["seen"], want["seen"]) and int(got["sum"].sum()) == want["total"]


@pytest.mark.parametrize("i,rate,nslots,admitters,chunk", [
    (0, 1e4, 64, 16, 8192), (1, 1e5, 8, 4, 1024), (2, 5e5, 1, 1, 32768), (3, 1e6, 64, 16, 4096),
    (4, 2e6, 32, 8, 8192), (5, 1e5, 3, 2, 2048)])
def test_serving_repeated(i, rate, nslots, admitters, chunk):
    import torch
    from paper_1110_4623_gb300 import runner
    off, ln, pool = inputs.serve_inputs(3000, 16 << 20, seed=99)
    sched = inputs.poisson_arrivals(3000, rate, seed=500 + i)
    r = runner.ServeRun(off, ln, sched, torch.from_numpy(pool).cuda(), nslots=nslots, nblocks=304,
                        admitters=admitters, chunk_elems=chunk).run()
    assert r["rc"] == 0 and np.array_equal(r["res"], calc.serve_final(off, ln, pool))
