"""The grid-size sweep's small points, 1..64 blocks (the paper draws its Section 6 curves from
one block up): every mutex configuration, barrier kind and semaphore kind that the sweep
times there, run at the sweep's own sizes and inputs and checked bit-exactly against the
oracle."""
import numpy as np
import pytest

import bench
from gpu_util import require_gpu
from oracle import calc
from paper_1110_4623_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _points(cluster_of, items):
    out = []
    for item in items:
        seen = set()
        for B in bench.SWEEP_SMALL:
            nb = bench.sweep_grid(B, cluster_of(item))
            if nb and nb not in seen:
                seen.add(nb)
                out.append((item, nb))
    return out


MUTEX_POINTS = [((cfg, K), nb) for (cfg, K), nb in
                _points(lambda ck: bench.mutex_cluster(ck[0][1]),
                        [(cfg, K) for cfg in bench.MUTEX_CONFIGS for K in bench.CS_SIZES])]
BARRIER_POINTS = _points(lambda kp: kp[1] & 0xF if kp[0] == "cluster" else 0, bench.SWEEP_BARRIERS)
SEM_POINTS = [((kind, n), B) for kind in bench.SEM_STEP_KINDS for n in bench.SEM_COUNTS for B in bench.SWEEP_SMALL]


def test_points_cover_one_block_and_skip_grids_smaller_than_a_cluster():
    assert ((("atomic", 0)), 1) in BARRIER_POINTS
    assert all(nb % (kp[1] & 0xF) == 0 for kp, nb in BARRIER_POINTS if kp[0] == "cluster")
    assert min(nb for (ck, nb) in MUTEX_POINTS if ck[0][1] == "cluster_mcs") == bench.mutex_cluster("cluster_mcs")


@pytest.mark.parametrize("point", MUTEX_POINTS, ids=lambda p: f"{p[0][0][0]}-cs{p[0][1]}-b{p[1]}")
def test_mutex_sweep_point(point):
    from paper_1110_4623_gb300 import gsync as G
    from paper_1110_4623_gb300 import runner
    ((name, kind, policy, bo_ns, spin), K), nb = point
    delay, add = inputs.mutex_inputs(nb, bench.MUTEX_ACQ, inputs.mutex_seed(G.MUTEX_KINDS[kind], nb, K))
    bo = runner.backoff(policy=policy, min_ns=bo_ns[0], max_ns=bo_ns[1], spin=spin) if bo_ns else None
    got = runner.MutexRun(kind, nb, bench.MUTEX_THREADS, bench.MUTEX_ACQ, K, delay, add, bo=bo,
                          timeout_ns=bench.TIMEOUT_NS, cluster=bench.mutex_cluster(kind)).run()
    want = calc.mutex_final(nb, bench.MUTEX_ACQ, K, add)
    assert got["rc"] == 0 and got["status"] == 0, got["status"]
    assert got["total"] == want["total"] and np.array_equal(got["data"], want["data"])
    assert (got["count"] == bench.MUTEX_ACQ).all()


@pytest.mark.parametrize("point", BARRIER_POINTS, ids=lambda p: f"{bench.barrier_name(*p[0])}-b{p[1]}")
def test_barrier_sweep_point(point):
    from paper_1110_4623_gb300 import runner
    (kind, param), nb = point
    got = runner.BarrierRun(kind, nb, bench.BAR_THREADS, bench.BAR_ROUNDS, full=False, param=param,
                            timeout_ns=bench.TIMEOUT_NS).run()
    assert got["rc"] == 0 and got["status"] == 0, got["status"]
    assert not got["bad"].any()
    assert np.array_equal(got["mix"], calc.barrier_sampled(nb, bench.BAR_ROUNDS)["mix"])


@pytest.mark.parametrize("point", SEM_POINTS, ids=lambda p: f"{p[0][0]}-n{p[0][1]}-b{p[1]}")
def test_semaphore_sweep_point(point):
    from paper_1110_4623_gb300 import runner
    (kind, n), B = point
    hold, add = inputs.sem_inputs(B, bench.SEM_PAIRS, inputs.SEED_SEM ^ (n << 16) ^ B)
    got = runner.SemRun(kind, B, bench.SEM_THREADS, bench.SEM_PAIRS, n, hold, add,
                        bo=runner.backoff(min_ns=bench.SEM_BACKOFF[0], max_ns=bench.SEM_BACKOFF[1]),
                        timeout_ns=bench.TIMEOUT_NS).run()
    want = calc.sem_final(B, bench.SEM_PAIRS, n, add)
    assert got["rc"] == 0 and got["status"] == 0, got["status"]
    assert got["tally"] == want["tally"] and np.array_equal(got["count"], want["count"])
    assert 1 <= got["max_occ"] <= min(n, B)
    if n == 1:
        assert got["total"] == want["total"]
