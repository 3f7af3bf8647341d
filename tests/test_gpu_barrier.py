"""Barrier workload on the GPU against the oracle, bit-exact (Section 5, "Barrier")."""
import numpy as np
import pytest

from gpu_util import require_gpu
from oracle import calc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


KINDS = [("atomic", 0), ("flag", 0), ("flag", 1), ("tree", 8), ("tree", 2), ("cluster", 2), ("cluster", 4),
         ("cluster", 8), ("sharded", 32), ("sharded", 8), ("sharded", 1), ("die", 0), ("die", 1), ("split", 1 | 1 << 8),
         ("split", 1 | 16 << 8), ("split", 16 | 16 << 8), ("split", 64 | 64 << 8), ("split", 7 | 3 << 8),
         ("count", 0), ("count", 8), ("count", 1023), ("count", 8 | 16 << 16), ("count", 2 << 16),
         ("count", 8 | 64 << 16), ("count", 7 << 16),
         # the counting form of the cluster barrier (param = c | form << 4 | sleep << 8)
         ("cluster", 2 | 1 << 4), ("cluster", 4 | 1 << 4 | 8 << 8), ("cluster", 8 | 1 << 4 | 8 << 8),
         ("cluster", 2 | 2 << 4), ("cluster", 4 | 2 << 4 | 8 << 8), ("cluster", 8 | 2 << 4 | 1023 << 8),
         # the counting form of the tree (param = fan | 1 << 16)
         ("tree", 2 | 1 << 16), ("tree", 8 | 1 << 16), ("tree", 32 | 1 << 16), ("tree", 1024 | 1 << 16),
         # the exchange barrier: the slot values carried in the arrivals (param = the sleep)
         ("exchange", 0), ("exchange", 8), ("exchange", 1023)]


@pytest.mark.parametrize("kind,param", KINDS)
def test_config1_full_fold_10000_rounds(kind, param):
    # 16 blocks x 128 threads, 10,000 rounds; per-round XOR checksum of all 16 slots.
    from paper_1110_4623_gb300 import runner
    if kind == "sharded":
        param = min(param, 16)
    got = runner.BarrierRun(kind, 16, 128, 10_000, full=True, param=param).run()
    want = calc.barrier_full(16, 10_000)
    assert got["rc"] == 0 and got["status"] == 0, got["status"]
    assert np.array_equal(got["chk"], want["chk"])
    assert np.array_equal(got["mix"], want["mix"])
    assert not got["bad"].any()


@pytest.mark.parametrize("kind,param", KINDS)
@pytest.mark.parametrize("nblocks", [148, 296, 592, 1184])
def test_sampled_sweep_1000_rounds(kind, param, nblocks):
    # A cluster launch needs the grid to be a multiple of the cluster size: 148 blocks run as
    # 144 with clusters of 8.
    from paper_1110_4623_gb300 import runner
    if kind == "cluster":
        nblocks -= nblocks % (param & 0xF)
    got = runner.BarrierRun(kind, nblocks, 128, 1000, full=False, param=param).run()
    want = calc.barrier_sampled(nblocks, 1000)
    assert got["rc"] == 0 and got["status"] == 0, got["status"]
    assert not got["bad"].any(), int(got["bad"].sum())
    assert np.array_equal(got["mix"], want["mix"])


@pytest.mark.parametrize("kind,param", [("atomic", 0), ("flag", 0), ("tree", 3), ("cluster", 1), ("sharded", 3),
                                        ("die", 0), ("die", 1), ("split", 5 | 3 << 8), ("count", 0),
                                        ("count", 8 | 5 << 16), ("cluster", 1 | 1 << 4), ("cluster", 1 | 2 << 4 | 8 << 8),
                                        ("tree", 3 | 1 << 16), ("exchange", 8)])
@pytest.mark.parametrize("nblocks,threads", [(1, 32), (2, 64), (37, 96), (151, 256)])
def test_ragged_grids_full_fold(kind, param, nblocks, threads):
    from paper_1110_4623_gb300 import runner
    if kind == "sharded":
        param = min(param, nblocks)
    got = runner.BarrierRun(kind, nblocks, threads, 300, full=True, param=param).run()
    want = calc.barrier_full(nblocks, 300)
    assert got["rc"] == 0 and got["status"] == 0
    assert np.array_equal(got["chk"], want["chk"]) and np.array_equal(got["mix"], want["mix"])
    assert not got["bad"].any()


def test_zero_rounds():
    from paper_1110_4623_gb300 import runner
    got = runner.BarrierRun("atomic", 8, 128, 0, full=False).run()
    assert got["rc"] == 0 and got["status"] == 0 and not got["mix"].any()


@pytest.mark.parametrize("kind,nblocks,param", [("flag", 64, 0), ("die", 64, 0), ("die", 1184, 0), ("die", 7, 0),
                                                ("split", 1184, 0), ("count", 1184, 0), ("count", 7, 0),
                                                ("cluster", 1184, 4 | 1 << 4 | 8 << 8), ("cluster", 1184, 8 | 2 << 4),
                                                ("cluster", 7, 1 | 1 << 4), ("tree", 1184, 8 | 1 << 16),
                                                ("tree", 7, 3 | 1 << 16), ("exchange", 1184, 8), ("exchange", 7, 0)])
def test_repeated_launches_continue_epochs(kind, nblocks, param):
    # The object keeps its epoch across launches: a second launch attaches at the new epoch
    # (DIE: and counts its blocks per die again in its first crossing; the counting kinds:
    # their counter rounded down to a multiple of the arrivals per crossing).
    from paper_1110_4623_gb300 import runner
    br = runner.BarrierRun(kind, nblocks, 128, 501, full=False, param=param)
    for _ in range(3):
        got = br.run()
        assert got["status"] == 0 and not got["bad"].any()
        assert np.array_equal(got["mix"], calc.barrier_sampled(nblocks, 501)["mix"])



def test_max_coresident_grid_runs():
    from paper_1110_4623_gb300 import gsync as G
    from paper_1110_4623_gb300 import runner
    rc, maxb = G.gsync_max_coresident_blocks(0, G.BARRIER_KINDS["atomic"], 128, 1)
    assert rc == 0 and maxb >= 1184
    got = runner.BarrierRun("atomic", maxb, 128, 200, full=False).run()
    assert got["status"] == 0 and np.array_equal(got["mix"], calc.barrier_sampled(maxb, 200)["mix"])


def test_grid_beyond_coresidency_is_refused():
    from paper_1110_4623_gb300 import gsync as G
    from paper_1110_4623_gb300 import runner
    rc, maxb = G.gsync_max_coresident_blocks(0, G.BARRIER_KINDS["atomic"], 256, 1)
    assert rc == 0
    br = runner.BarrierRun("atomic", maxb + 1, 256, 10, full=False)
    assert br.launch() == G.GSYNC_ENOTRESIDENT
