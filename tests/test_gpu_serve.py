"""Persistent serving loop against the oracle: every request's int64 segmented sum exact,
the same alone and in the mix (continuous batching must not change any result), and the
per-request-launch baseline exact too."""
import numpy as np
import pytest
import torch

from gpu_util import require_gpu
from oracle import calc
from paper_1110_4623_gb300 import inputs

pytestmark = pytest.mark.gpu

POOL = 1 << 24


@pytest.fixture(scope="module")
def pool():
    require_gpu()
    off, ln, p = inputs.serve_inputs(4000, POOL, seed=77)
    return off, ln, p, torch.from_numpy(p).cuda()


def make(pool, idx, rate, **kw):
    from paper_1110_4623_gb300 import runner
    off, ln, p, dp = pool
    sched = inputs.poisson_arrivals(len(idx), rate, seed=5)
    return runner.ServeRun(off[idx], ln[idx], sched, dp, **kw)


def test_results_exact_at_1e5_per_s(pool):
    off, ln, p, _ = pool
    idx = np.arange(2000)
    r = make(pool, idx, 1e5).run()
    assert r["rc"] == 0, r["stats"]
    assert np.array_equal(r["res"], calc.serve_final(off[idx], ln[idx], p))
    assert (r["latency_ns"] > 0).all()
    assert r["stats"][0] == 2000 and r["stats"][2] == 2000 and r["stats"][3] == 0


def test_same_result_alone_and_in_the_mix(pool):
    off, ln, p, _ = pool
    idx = np.arange(300)
    alone = make(pool, idx, 2e3, nslots=1).run()      # one request in flight at a time
    mixed = make(pool, idx, 5e6, nslots=64).run()     # a burst: requests overlap on the device
    assert alone["rc"] == 0 and mixed["rc"] == 0
    assert np.array_equal(alone["res"], mixed["res"])
    assert np.array_equal(mixed["res"], calc.serve_final(off[idx], ln[idx], p))


def test_ring_wraps(pool):
    off, ln, p, _ = pool
    idx = np.arange(4000)
    r = make(pool, idx, 1e6, ring_slots=64, nslots=16).run()
    assert r["rc"] == 0
    assert np.array_equal(r["res"], calc.serve_final(off[idx], ln[idx], p))


def test_per_request_launch_baseline_exact(pool):
    off, ln, p, _ = pool
    idx = np.arange(1000)
    r = make(pool, idx, 5e4).baseline(nstreams=4)
    assert r["rc"] == 0
    assert np.array_equal(r["res"], calc.serve_final(off[idx], ln[idx], p))


def test_extreme_lengths(pool):
    from paper_1110_4623_gb300 import runner
    _, _, p, dp = pool
    off = np.array([0, 1, POOL - (1 << 20), 3, 12345], dtype=np.int64)
    ln = np.array([1, 256, 1 << 20, (1 << 20) - 1, 32769], dtype=np.int64)
    sched = np.array([0, 1000, 2000, 3000, 4000], dtype=np.int64)
    r = runner.ServeRun(off, ln, sched, dp, nslots=2).run()
    assert r["rc"] == 0
    assert np.array_equal(r["res"], calc.serve_final(off, ln, p))


@pytest.mark.parametrize("rate,n,kw", [(1e5, 2000, {}), (1e6, 4000, {"ring_slots": 64, "nslots": 16})])
def test_device_resident_ring_exact(pool, rate, n, kw):
    # The ring in managed memory that the loop places in device memory (the host's producer
    # writes it in place): the same exact results, also when the ring wraps.
    off, ln, p, _ = pool
    idx = np.arange(n)
    r = make(pool, idx, rate, ring="device", **kw).run()
    assert r["rc"] == 0, r["stats"]
    assert np.array_equal(r["res"], calc.serve_final(off[idx], ln[idx], p))
    assert r["stats"][0] == n and r["stats"][2] == n and r["stats"][3] == 0


def test_device_resident_ring_same_alone_and_in_the_mix(pool):
    off, ln, p, _ = pool
    idx = np.arange(300)
    alone = make(pool, idx, 2e3, nslots=1, ring="device").run()
    mixed = make(pool, idx, 5e6, nslots=64, ring="device").run()
    assert alone["rc"] == 0 and mixed["rc"] == 0
    assert np.array_equal(alone["res"], mixed["res"])
    assert np.array_equal(mixed["res"], calc.serve_final(off[idx], ln[idx], p))
