"""The threaded CPU execution (real locks on host threads) reaches the final states that the
plain definitions in calc.py give: two independent computations of the same result."""
import numpy as np
import pytest

from oracle import calc, cpu
from paper_1110_4623_gb300 import inputs


@pytest.mark.parametrize("kind", list(cpu.MUTEX_KINDS))
@pytest.mark.parametrize("nblocks,acq,cs_words,threads", [(16, 25, 64, 4), (37, 9, 1024, 8), (5, 40, 0, 5), (64, 3, 7, 16)])
def test_mutex_exec_matches_definition(kind, nblocks, acq, cs_words, threads):
    delay, add = inputs.mutex_inputs(nblocks, acq, inputs.mutex_seed(cpu.MUTEX_KINDS[kind], nblocks, cs_words), max_delay=50)
    r = cpu.mutex_run(kind, nblocks, acq, cs_words, add, delay, nthreads=threads)
    want = calc.mutex_final(nblocks, acq, cs_words, add)
    assert r["total"] == want["total"]
    assert np.array_equal(r["data"], want["data"])
    assert np.array_equal(r["count"], want["count"])
    fifo = kind in ("ticket", "sleep_queue")
    assert calc.check_grant_log(r["log"], r["ticket"] if fifo else None, nblocks, acq, fifo) == []


@pytest.mark.parametrize("kind", list(cpu.SEM_KINDS))
@pytest.mark.parametrize("n_init", [1, 4, 16])
def test_sem_exec_matches_definition(kind, n_init):
    B, P = 24, 15
    hold, add = inputs.sem_inputs(B, P, 0x5EED0003 ^ n_init, hold_lo=0, hold_hi=200)
    r = cpu.sem_run(kind, B, P, n_init, add, hold, nthreads=8)
    want = calc.sem_final(B, P, n_init, add)
    assert np.array_equal(r["count"], want["count"])
    assert r["tally"] == want["tally"]
    assert 1 <= r["max_occ"] <= n_init
    if n_init == 1:
        assert r["total"] == want["total"]


@pytest.mark.parametrize("kind", list(cpu.BARRIER_KINDS))
def test_barrier_exec_full_matches_definition(kind):
    r = cpu.barrier_run(kind, 16, 300, full=True)
    want = calc.barrier_full(16, 300)
    assert np.array_equal(r["chk"], want["chk"])
    assert np.array_equal(r["mix"], want["mix"])
    assert not r["bad"].any()


@pytest.mark.parametrize("kind", list(cpu.BARRIER_KINDS))
@pytest.mark.parametrize("nblocks", [1, 2, 7, 33])
def test_barrier_exec_sampled_matches_definition(kind, nblocks):
    r = cpu.barrier_run(kind, nblocks, 200, full=False)
    want = calc.barrier_sampled(nblocks, 200)
    assert np.array_equal(r["mix"], want["mix"])
    assert not r["bad"].any()
