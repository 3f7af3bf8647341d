"""Pins the exact-state calculators to closed forms, special cases and invariants."""
import numpy as np
import pytest

from oracle import calc
from paper_1110_4623_gb300 import inputs


# ---- barrier ---------------------------------------------------------------------------

def test_config1_xor_checksum_is_zero_closed_form():
    # XOR_{b<16} (16 r + b) = XOR_{b<16} b = 0, for every round r.
    out = calc.barrier_full(16, 10_000)
    assert out["chk"].shape == (10_000, 16)
    assert not out["chk"].any()
    assert not out["bad"].any()


@pytest.mark.parametrize("nblocks", [4, 8, 148, 1184])
def test_xor_checksum_zero_when_grid_multiple_of_four(nblocks):
    # Four consecutive integers starting at a multiple of 4 XOR to 0.
    assert not calc.barrier_full(nblocks, 7)["chk"].any()


def test_xor_checksum_odd_grid_closed_form():
    # B = 3: XOR(3r, 3r+1, 3r+2); e.g. r = 0 -> 0^1^2 = 3, r = 1 -> 3^4^5 = 2.
    chk = calc.barrier_full(3, 2)["chk"]
    assert list(chk[:, 0]) == [3, 2]


def test_lowbias32_properties():
    assert calc.lowbias32(np.array([0]))[0] == 0
    # A composition of xor-shifts and odd multiplies is a bijection on 32-bit words.
    x = np.arange(1 << 20, dtype=np.uint32) * np.uint32(4093)
    assert len(np.unique(calc.lowbias32(x))) == len(np.unique(x))
    # Avalanche: flipping one input bit flips ~16 output bits on average.
    a = calc.lowbias32(x[:4096])
    b = calc.lowbias32(x[:4096] ^ np.uint32(1))
    flips = np.unpackbits((a ^ b).view(np.uint8)).sum() / 4096
    assert 14 < flips < 18


def test_rotl32():
    assert calc.rotl32(np.uint32(0x80000001), 5) == 0x30
    assert calc.rotl32(np.uint32(1), 31) == 0x80000000


def test_full_mix_single_round_by_hand():
    # One round, B = 2: slots 0 and 1; s = lowbias32(0) + lowbias32(1) = lowbias32(1).
    out = calc.barrier_full(2, 1)
    assert out["mix"][0] == calc.lowbias32(np.array([1]))[0]


def test_sampled_partner_sequence_by_hand():
    # B = 3, R = 2: block 0 reads partner 1 in round 0 (value 1), partner 2 in round 1
    # (value 3 + 2 = 5): mix = rotl(lowbias32(1), 5) ^ lowbias32(5).
    out = calc.barrier_sampled(3, 2)
    h1 = calc.lowbias32(np.array([1]))[0]
    want = calc.rotl32(np.uint32(h1), 5) ^ calc.lowbias32(np.array([5]))[0]
    assert out["mix"][0] == want
    assert not out["bad"].any()


def test_sampled_blocks_differ():
    # Every block reads a different partner sequence, so a mix that ignored b would match
    # across blocks; the definition gives distinct values.
    mix = calc.barrier_sampled(148, 50)["mix"]
    assert len(np.unique(mix)) == 148


# ---- mutex -----------------------------------------------------------------------------

def test_mutex_zero_addends_closed_form():
    B, A, K = 5, 7, 33
    out = calc.mutex_final(B, A, K, np.zeros(B * A, np.uint32))
    i = np.arange(K, dtype=np.uint64)
    want = ((B * A) * ((i * 0x9E3779B1) % 2 ** 32)) % 2 ** 32
    assert np.array_equal(out["data"].astype(np.uint64), want)
    assert out["total"] == B * A
    assert np.array_equal(out["count"], np.full(B, A))


def test_mutex_all_ones_addends_closed_form():
    B, A, K = 3, 4, 9
    out = calc.mutex_final(B, A, K, np.full(B * A, 0xFFFFFFFF, np.uint32))
    i = np.arange(K, dtype=np.uint64)
    c = (i * 0x9E3779B1) % 2 ** 32
    want = ((B * A) * (0xFFFFFFFF - c)) % 2 ** 32
    assert np.array_equal(out["data"].astype(np.uint64), want)


def test_mutex_word0_is_plain_sum():
    # c_0 = 0, so data[0] is the plain sum of the addends mod 2^32.
    _, add = inputs.mutex_inputs(37, 11, 99)
    out = calc.mutex_final(37, 11, 1, add)
    assert int(out["data"][0]) == int(sum(int(v) for v in add)) % 2 ** 32


def test_mutex_single_acquisition_is_xor():
    add = np.array([0xDEADBEEF], np.uint32)
    out = calc.mutex_final(1, 1, 130, add)
    for i in (0, 1, 64, 129):
        assert int(out["data"][i]) == 0xDEADBEEF ^ ((i * 0x9E3779B1) % 2 ** 32)


def test_mutex_empty_cs():
    out = calc.mutex_final(4, 3, 0, np.arange(12, dtype=np.uint32))
    assert out["data"].shape == (0,) and out["total"] == 12


def test_grant_log_checks():
    B, A = 3, 2
    good = np.array([0, 2, 4, 1, 3, 5])
    assert calc.check_grant_log(good, None, B, A, fifo=False) == []
    dup = good.copy(); dup[1] = 0
    assert calc.check_grant_log(dup, None, B, A, fifo=False)
    swapped = np.array([1, 0, 2, 3, 4, 5])  # block 0's second acquisition before its first
    assert "program order" in calc.check_grant_log(swapped, None, B, A, fifo=False)[0]
    tick = np.empty(6, np.uint32); tick[good] = np.arange(6)
    assert calc.check_grant_log(good, tick, B, A, fifo=True) == []
    tick2 = tick.copy(); tick2[[0, 2]] = tick2[[2, 0]]
    assert calc.check_grant_log(good, tick2, B, A, fifo=True)
    base = 2 ** 32 - 2
    tick3 = ((tick.astype(np.uint64) + base) % 2 ** 32).astype(np.uint32)
    assert calc.check_grant_log(good, tick3, B, A, fifo=True, ticket_base=base) == []


def test_grant_log_per_die():
    # Grants s = 0..5 of acquisitions good[s]; dies alternate 0,1,1,0,0,1; each die's tickets
    # count from its own base in grant order, with bit 31 marking die 1.
    B, A = 3, 2
    good = np.array([0, 2, 4, 1, 3, 5])
    die = np.array([0, 1, 1, 0, 0, 1])
    local = np.array([5, 9, 10, 6, 7, 11])  # die 0 from 5, die 1 from 9
    tick = np.empty(6, np.uint32)
    tick[good] = ((die.astype(np.uint64) << np.uint64(31)) | local.astype(np.uint64)).astype(np.uint32)
    assert calc.check_grant_log(good, tick, B, A, fifo=False, per_die=True, die_bases=(5, 9)) == []
    assert calc.die_grant_counts(tick) == (3, 3)
    assert calc.check_grant_log(good, tick, B, A, fifo=False, per_die=True, die_bases=(5, 8))
    bad = tick.copy(); bad[[good[0], good[3]]] = bad[[good[3], good[0]]]  # die 0 out of order
    assert "die 0" in calc.check_grant_log(good, bad, B, A, fifo=False, per_die=True, die_bases=(5, 9))[0]
    # a single global ticket order is not a per-die order once dies interleave
    assert calc.check_grant_log(good, tick, B, A, fifo=True)


# ---- semaphore, batched, serving --------------------------------------------------------

def test_sem_closed_forms():
    out = calc.sem_final(10, 20, 1, np.ones(200, np.uint32))
    assert out["tally"] == 200 and out["total"] == 200
    assert np.array_equal(out["count"], np.full(10, 20))
    out4 = calc.sem_final(10, 20, 4, np.full(200, 2 ** 31, np.uint32))
    assert out4["tally"] == 0 and "total" not in out4  # 200 * 2^31 = 0 mod 2^32


def test_batched_brute_force_small():
    keys = np.array([3, 0, 3, 1, 3], np.int32)
    adds = np.array([2 ** 63 - 1, 5, 1, -7, 2 ** 63 - 1], np.int64)
    out = calc.batched_final(keys, adds, 4)
    # key 3: (2^63-1) + 1 + (2^63-1) = 2^64 - 1 = -1 mod 2^64
    assert list(out["sum"]) == [5, -7, 0, -1]
    assert list(out["count"]) == [1, 1, 0, 3]


def test_batched_totals():
    keys, adds, _ = inputs.batched_inputs(10_000, 64, 1.1, seed=5)
    out = calc.batched_final(keys, adds, 64)
    assert int(out["count"].sum()) == 10_000
    assert (int(out["sum"].view(np.uint64).sum(dtype=np.uint64))
            == int(adds.view(np.uint64).sum(dtype=np.uint64)))


def test_serve_prefix_sum_identity():
    off, ln, pool = inputs.serve_inputs(50, 1 << 21, seed=3, len_lo=1, len_hi=1 << 20)
    res = calc.serve_final(off, ln, pool)
    cs = np.concatenate([[0], np.cumsum(pool.astype(np.int64))])
    assert np.array_equal(res, cs[off + ln] - cs[off])


def test_serve_constant_pool():
    pool = np.full(1 << 20, -(2 ** 20), np.int32)
    res = calc.serve_final(np.array([0, 5]), np.array([1 << 20, 256]), pool)
    assert list(res) == [-(2 ** 40), -(2 ** 28)]  # exceeds int32: accumulated in int64


def test_condvar_closed_form():
    # Values read as int32: 0xFFFFFFFF is -1, so [1, 2, 0xFFFFFFFF, 5] sums to 7.
    v = np.array([1, 2, 0xFFFFFFFF, 5], np.uint32)
    out = calc.condvar_final(v, 2, 2, 4)
    assert out["total"] == 7 and np.array_equal(out["count"], [1, 1, 1, 1])
    assert np.array_equal(out["seen"], [1, 1, 1, 1])
    # all-ones values over many items: n * (-1), beyond int32 range only in magnitude here
    out = calc.condvar_final(np.full(1 << 16, 0x80000000, np.uint32), 4, 1 << 14, 8)
    assert out["total"] == -(1 << 31) * (1 << 16)


def test_grant_log_per_group():
    # Two groups in the top 12 bits; each group's tickets count from 0 in grant order.
    B, A = 2, 3
    good = np.array([0, 3, 1, 4, 2, 5])        # grant order of acquisition ids
    grp = np.array([0, 1, 0, 1, 0, 1])
    local = np.array([0, 0, 1, 1, 2, 2])
    tick = np.empty(6, np.uint32)
    tick[good] = ((grp.astype(np.uint64) << np.uint64(20)) | local.astype(np.uint64)).astype(np.uint32)
    assert calc.check_grant_log(good, tick, B, A, fifo=False, group_bits=12) == []
    bad = tick.copy(); bad[[good[0], good[2]]] = bad[[good[2], good[0]]]
    assert "group 0" in calc.check_grant_log(good, bad, B, A, fifo=False, group_bits=12)[0]
