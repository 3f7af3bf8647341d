"""Seeded input generators: determinism, ranges, distributions."""
import numpy as np

from paper_1110_4623_gb300 import inputs


def test_splitmix64_reference_values():
    # SplitMix64 with state 0: the first outputs are the published sequence of the
    # reference implementation (Vigna's splitmix64.c seeded with 0).
    z = inputs.splitmix64(0, 3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_deterministic_and_offset():
    a = inputs.splitmix64(123, 10)
    b = inputs.splitmix64(123, 5, offset=5)
    assert np.array_equal(a[5:], b)


def test_uniform_ranges():
    d, a = inputs.mutex_inputs(1184, 100, inputs.mutex_seed(0, 1184, 64))
    assert d.min() == 0 and d.max() == 2000 and d.dtype == np.uint32
    assert a.dtype == np.uint32 and a.max() > 2 ** 31
    h, _ = inputs.sem_inputs(296, 200, 1)
    assert h.min() >= 100 and h.max() <= 5000


def test_zipf_head_probability():
    # P(key 0) = 1 / H(4096, 1.1) ~ 0.1605 for Zipf s = 1.1 over 4096 keys.
    k = inputs.zipf_keys(7, 1_000_000, 4096, 1.1)
    h = (np.arange(1, 4097, dtype=np.float64) ** -1.1).sum()
    p0 = (k == 0).mean()
    assert abs(p0 - 1 / h) < 0.002
    assert k.min() == 0 and k.max() < 4096


def test_group_sizes_fit_grid():
    drawn, used = inputs.barrier_group_sizes(64, 2, 256, 1184)
    assert drawn.min() >= 2 and drawn.max() <= 256
    assert used.sum() <= 1184 and used.min() >= 2


def test_serve_inputs():
    off, ln, pool = inputs.serve_inputs(1000, 1 << 22, seed=9)
    assert ln.min() >= 256 and ln.max() <= 1 << 20
    assert (off + ln <= len(pool)).all() and off.min() >= 0
    assert pool.min() >= -(2 ** 20) and pool.max() <= 2 ** 20
    t = inputs.poisson_arrivals(10_000, 1e5, seed=1)
    assert abs(t[-1] / 1e9 - 0.1) < 0.01
