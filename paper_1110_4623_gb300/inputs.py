"""Seeded synthetic inputs for the synchronization workloads.

This module holds only random-number generation: it draws the per-acquisition delays,
addends, hold times, key streams, group sizes and request descriptors that the workloads
consume.  It contains none of the synchronization method's arithmetic and none of the
workloads' result arithmetic, so the CUDA path and the CPU oracle can both be fed from it
without sharing any computation.

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), used in counter mode: draw i of stream `seed` is
mix64(seed + (i + 1) * GAMMA).  Integers in [lo, hi] take the high 32 bits of a draw and
scale them with a 32x32->64 multiply (Lemire's multiply-shift; bias < 2^-32 * range).

The paper measures only synthetic loops of lock/unlock, wait/post and barrier calls
(Section 6, "Results & Discussion"), so no dataset stands behind any of these arrays.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Seeds of the five workload families.
SEED_BARRIER = 0x5EED0001
SEED_MUTEX = 0x5EED0002
SEED_SEM = 0x5EED0003
SEED_BATCHED = 0x5EED0004
SEED_SERVE = 0x5EED0005
SEED_CONDVAR = 0x5EED0006


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Draws offset..offset+n-1 of the counter-mode SplitMix64 stream `seed` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_u32(seed: int, n: int, lo: int, hi: int) -> np.ndarray:
    """n integers uniform on [lo, hi] (inclusive), 0 <= lo <= hi < 2^32, as uint32."""
    span = np.uint64(hi - lo + 1)
    hi32 = splitmix64(seed, n) >> np.uint64(32)
    with np.errstate(over="ignore"):
        v = (hi32 * span) >> np.uint64(32)
    return (v + np.uint64(lo)).astype(np.uint32)


def bits_u32(seed: int, n: int) -> np.ndarray:
    """n uniformly random 32-bit words (high half of each draw)."""
    return (splitmix64(seed, n) >> np.uint64(32)).astype(np.uint32)


def unit_f64(seed: int, n: int) -> np.ndarray:
    """n doubles uniform on (0, 1): 53 random bits, offset by half an ulp (never 0 or 1)."""
    z = splitmix64(seed, n) >> np.uint64(11)
    return (z.astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def mutex_seed(kind: int, nblocks: int, cs_words: int) -> int:
    return SEED_MUTEX ^ ((kind << 16) ^ nblocks ^ (cs_words << 24))


def mutex_inputs(nblocks: int, acq: int, seed: int, max_delay: int = 2000):
    """Per-acquisition inputs of the mutex contention workload.

    Acquisition id = b * acq + a.  Returns (delay, addend): delay[id] ~ U{0..max_delay}
    cycles spent before the lock call, addend[id] ~ U{0..2^32-1} the value the critical
    section adds.
    """
    n = nblocks * acq
    delay = uniform_u32(seed, n, 0, max_delay)
    addend = bits_u32(seed ^ 0xADD0ADD0, n)
    return delay, addend


def sem_inputs(nblocks: int, pairs: int, seed: int, hold_lo: int = 100, hold_hi: int = 5000):
    """Per-wait inputs of the counting-semaphore workload: (hold cycles, addend)."""
    n = nblocks * pairs
    hold = uniform_u32(seed, n, hold_lo, hold_hi)
    addend = bits_u32(seed ^ 0x5E3A5E3A, n)
    return hold, addend


def condvar_inputs(nitems: int, seed: int = SEED_CONDVAR) -> np.ndarray:
    """Per-item values of the condition-variable (producer/consumer) workload: uint32 bits,
    read as int32 on both sides."""
    return bits_u32(seed, nitems)


def zipf_keys(seed: int, n: int, nkeys: int, s: float) -> np.ndarray:
    """n keys in [0, nkeys) with P(key = k) proportional to (k + 1)^-s (rank 1 -> key 0).

    Inverse-CDF sampling on host doubles: key = first k with CDF[k] >= u.
    """
    w = np.arange(1, nkeys + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = unit_f64(seed, n)
    k = np.searchsorted(cdf, u, side="left")
    return np.minimum(k, nkeys - 1).astype(np.int32)


def batched_inputs(nacq: int, nkeys: int, s: float, seed: int = SEED_BATCHED):
    """Keys ~ Zipf(s) over nkeys mutexes and int64 addends for the batched workload."""
    keys = zipf_keys(seed, nacq, nkeys, s)
    adds = splitmix64(seed ^ 0xB47C4ED0, nacq).view(np.int64)
    delay = uniform_u32(seed ^ 0xDE1A7000, nacq, 0, 2000)
    return keys, adds, delay


def log_uniform_int(seed: int, n: int, lo: int, hi: int) -> np.ndarray:
    """n integers with log-uniform distribution on [lo, hi] (floor of exp(U[ln lo, ln(hi+1)]))."""
    u = unit_f64(seed, n)
    x = np.exp(np.log(lo) + u * (np.log(hi + 1) - np.log(lo)))
    return np.clip(np.floor(x), lo, hi).astype(np.int64)


def barrier_group_sizes(ngroups: int, lo: int, hi: int, grid: int, seed: int = SEED_BATCHED,
                        multiple: int = 1):
    """Drawn group sizes (log-uniform on [lo, hi]) and the sizes rescaled to fit `grid`.

    Rescaling multiplies every drawn size by grid / sum and floors it to a multiple of
    `multiple` (the cluster size when the groups use cluster barriers), with a floor of
    max(lo, multiple); it then trims the largest groups by `multiple` blocks at a time until
    the total fits the grid.
    """
    drawn = log_uniform_int(seed ^ 0x6A0B5, ngroups, lo, hi)
    floor_size = max(lo, multiple)
    floor_size += (-floor_size) % multiple
    total = int(drawn.sum())
    scale = min(1.0, grid / total)
    used = np.floor(drawn * scale / multiple).astype(np.int64) * multiple
    used = np.maximum(used, floor_size)
    while used.sum() > grid:
        j = int(np.argmax(used))
        if used[j] - multiple < floor_size:
            raise ValueError("grid too small for the barrier groups")
        used[j] -= multiple
    return drawn, used


def group_layout(sizes: np.ndarray, grid: int):
    """Consecutive group placement from block 0: (start[g], group_of_block[b] or -1)."""
    start = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int32)
    gob = np.full(grid, -1, dtype=np.int32)
    for g, (st, sz) in enumerate(zip(start, sizes)):
        gob[st:st + sz] = g
    return start, gob


def serve_inputs(nreq: int, pool_elems: int, seed: int = SEED_SERVE,
                 len_lo: int = 256, len_hi: int = 1 << 20):
    """Request descriptors and the value pool of the serving workload.

    Returns (offset int64[nreq], length int64[nreq], pool int32[pool_elems]):
    length ~ log-uniform on [len_lo, len_hi]; offset ~ U{0..pool_elems-length};
    pool values ~ U{-2^20..2^20}.
    """
    length = log_uniform_int(seed, nreq, len_lo, len_hi)
    if pool_elems < len_hi:
        raise ValueError("pool smaller than the longest request")
    u = unit_f64(seed ^ 0x0FF5E7, nreq)
    offset = np.floor(u * (pool_elems - length + 1)).astype(np.int64)
    pool = (uniform_u32(seed ^ 0x9001, pool_elems, 0, 1 << 21).astype(np.int64) - (1 << 20)).astype(np.int32)
    return offset, length, pool


def poisson_arrivals(nreq: int, rate_per_s: float, seed: int = SEED_SERVE) -> np.ndarray:
    """Scheduled arrival times in ns of a Poisson process of the given rate (open loop)."""
    u = unit_f64(seed ^ 0xA7712, nreq)
    gaps = -np.log(u) / rate_per_s * 1e9
    return np.cumsum(gaps).astype(np.int64)
