"""Exact final states of the synchronization workloads (oracle; test infrastructure only).

Every workload here is built so that, when the primitive is correct, its final state does not
depend on the order in which blocks were granted the primitive.  Each function below writes
that final state out from its definition with plain numpy on uint32 / uint64 words, with no
blocking, fusion or reordering beyond the definition.

Definitions (the paper's terms, Section 5 "Design"):
  barrier   - no block passes round r until every block has arrived at round r.
  mutex     - at most one block is inside the critical section at any time.
  semaphore - at most n blocks are inside the critical section at any time.
"""
from __future__ import annotations

import numpy as np

M32 = 0xFFFFFFFF
GOLDEN32 = 0x9E3779B1  # 2^32 / golden ratio, odd; the per-word constant of the mutex CS


def lowbias32(x: np.ndarray) -> np.ndarray:
    """The 32-bit integer hash "lowbias32" (C. Wellons, hash-prospector, 2018):
    x ^= x >> 16; x *= 0x7feb352d; x ^= x >> 15; x *= 0x846ca68b; x ^= x >> 16 (mod 2^32)."""
    x = np.asarray(x, dtype=np.uint64) & np.uint64(M32)
    x ^= x >> np.uint64(16)
    x = (x * np.uint64(0x7FEB352D)) & np.uint64(M32)
    x ^= x >> np.uint64(15)
    x = (x * np.uint64(0x846CA68B)) & np.uint64(M32)
    x ^= x >> np.uint64(16)
    return x.astype(np.uint32)


def rotl32(x: np.ndarray, k: int) -> np.ndarray:
    x = np.asarray(x, dtype=np.uint64) & np.uint64(M32)
    return (((x << np.uint64(k)) | (x >> np.uint64(32 - k))) & np.uint64(M32)).astype(np.uint32)


# --------------------------------------------------------------------------------------------
# Barrier workload (Section 5, "Barrier" definition; Section 6 "Results", barrier test)
# --------------------------------------------------------------------------------------------
# Round r: block b writes slot[r & 1][b] = r * B + b, crosses the barrier, then reads slots.
#  FULL    : block b reads every slot j < B of buffer r & 1 and records
#            chk[r][b] = XOR_j slot_j,   s_r = sum_j lowbias32(slot_j) mod 2^32,
#            mix[b]   <- rotl32(mix[b], 5) ^ s_r          (mix starts at 0),
#            bad[b]   += number of j with slot_j != r * B + j.
#  SAMPLED : block b reads one partner p = (b + r + 1) mod B and records
#            mix[b] <- rotl32(mix[b], 5) ^ lowbias32(slot_p), bad[b] += (slot_p != r*B + p).
# A correct barrier makes every read return the value written in the same round.


def barrier_full(nblocks: int, rounds: int) -> dict:
    r = np.arange(rounds, dtype=np.uint64)[:, None]
    j = np.arange(nblocks, dtype=np.uint64)[None, :]
    slots = ((r * np.uint64(nblocks) + j) & np.uint64(M32)).astype(np.uint32)   # [R, B]
    chk_row = np.bitwise_xor.reduce(slots, axis=1)                              # [R]
    s = (lowbias32(slots).astype(np.uint64).sum(axis=1) & np.uint64(M32)).astype(np.uint32)
    h = np.uint32(0)
    for rr in range(rounds):
        h = np.uint32(rotl32(h, 5) ^ s[rr])
    chk = np.repeat(chk_row[:, None], nblocks, axis=1).astype(np.uint32)
    return {
        "chk": chk,
        "mix": np.full(nblocks, h, dtype=np.uint32),
        "bad": np.zeros(nblocks, dtype=np.uint32),
    }


def barrier_sampled(nblocks: int, rounds: int) -> dict:
    b = np.arange(nblocks, dtype=np.uint64)
    mix = np.zeros(nblocks, dtype=np.uint32)
    for r in range(rounds):
        p = (b + np.uint64(r + 1)) % np.uint64(nblocks)
        x = ((np.uint64(r) * np.uint64(nblocks) + p) & np.uint64(M32)).astype(np.uint32)
        mix = rotl32(mix, 5) ^ lowbias32(x)
    return {"mix": mix.astype(np.uint32), "bad": np.zeros(nblocks, dtype=np.uint32)}


# --------------------------------------------------------------------------------------------
# Mutex workload (Section 5, "Mutex" definition; Section 6 "Results", mutex test)
# --------------------------------------------------------------------------------------------
# B blocks each make A acquisitions; acquisition id = b * A + a.  Inside the critical section
# the block appends id to a grant log at position `total` and increments `total` (plain
# load/store), and for every i < K adds  addend[id] XOR (i * GOLDEN32 mod 2^32)  to data[i]
# (plain load/store).  Lost updates under broken exclusion change `total`, `data` or the log.


def cs_word_constants(cs_words: int) -> np.ndarray:
    i = np.arange(cs_words, dtype=np.uint64)
    return ((i * np.uint64(GOLDEN32)) & np.uint64(M32)).astype(np.uint32)


def mutex_final(nblocks: int, acq: int, cs_words: int, addend: np.ndarray) -> dict:
    """Final total, data[K] and per-block counts of the mutex workload."""
    addend = np.asarray(addend, dtype=np.uint32)
    assert addend.shape == (nblocks * acq,)
    c = cs_word_constants(cs_words)
    data = np.zeros(cs_words, dtype=np.uint32)
    chunk = 64
    for lo in range(0, cs_words, chunk):
        cc = c[lo:lo + chunk]
        terms = (addend[:, None] ^ cc[None, :]).astype(np.uint64)
        data[lo:lo + chunk] = (terms.sum(axis=0) & np.uint64(M32)).astype(np.uint32)
    return {
        "total": np.uint32((nblocks * acq) & M32),
        "data": data,
        "count": np.full(nblocks, acq, dtype=np.uint32),
    }


def check_grant_log(log: np.ndarray, ticket: np.ndarray | None, nblocks: int, acq: int,
                    fifo: bool, ticket_base: int = 0, per_die: bool = False,
                    die_bases: tuple = (0, 0), group_bits: int = 0) -> list[str]:
    """Validity of a grant log (the parts of the result that are not unique).

    log[s] is the acquisition id granted s-th.  It must be a permutation of 0..B*A-1 in
    which each block's acquisitions appear in increasing order (a block acquires
    sequentially).  For the fair kinds (ticket and queue locks, Section 5: "gives access to
    the critical section to blocks in the order in which they request access") the ticket
    drawn by the acquisition granted s-th must be ticket_base + s.  per_die (the two-die
    cohort lock): ticket bit 31 is the die and bits 30..0 that die's ticket; each die's
    grants, in grant order, must carry die_bases[d] + 0, 1, 2, ...  group_bits = g (the
    cluster cohort lock): the top g bits are the group and the rest its ticket, and each
    group's grants, in grant order, must carry 0, 1, 2, ...
    """
    n = nblocks * acq
    log = np.asarray(log, dtype=np.int64)
    problems = []
    if log.shape != (n,):
        return [f"log has shape {log.shape}, expected ({n},)"]
    if not np.array_equal(np.sort(log), np.arange(n)):
        problems.append("grant log is not a permutation of the acquisition ids")
        return problems
    pos = np.empty(n, dtype=np.int64)
    pos[log] = np.arange(n)
    per_block = pos.reshape(nblocks, acq)
    if acq > 1 and not np.all(np.diff(per_block, axis=1) > 0):
        problems.append("a block's acquisitions are granted out of program order")
    if fifo:
        t = np.asarray(ticket, dtype=np.uint64)[log]
        want = (np.arange(n, dtype=np.uint64) + np.uint64(ticket_base)) & np.uint64(M32)
        if not np.array_equal(t, want):
            problems.append("grants are not in ticket order")
    if group_bits:
        t = np.asarray(ticket, dtype=np.uint64)[log]
        shift = np.uint64(32 - group_bits)
        grp, local = t >> shift, t & ((np.uint64(1) << shift) - np.uint64(1))
        for g in np.unique(grp):
            got = local[grp == g]
            if not np.array_equal(got, np.arange(len(got), dtype=np.uint64)):
                problems.append(f"group {int(g)}'s grants are not in its ticket order")
                break
    if per_die:
        t = np.asarray(ticket, dtype=np.uint64)[log]
        die, local = t >> np.uint64(31), t & np.uint64(0x7FFFFFFF)
        for d in (0, 1):
            got = local[die == d]
            want = (np.arange(len(got), dtype=np.uint64) + np.uint64(die_bases[d])) & np.uint64(0x7FFFFFFF)
            if not np.array_equal(got, want):
                problems.append(f"die {d}'s grants are not in its ticket order")
    return problems


def die_grant_counts(ticket: np.ndarray) -> tuple:
    """Grants per die in a cohort lock's ticket record (bit 31 = die)."""
    d = np.asarray(ticket, dtype=np.uint64) >> np.uint64(31)
    return int((d == 0).sum()), int((d == 1).sum())


# --------------------------------------------------------------------------------------------
# Counting-semaphore workload (Section 5, "Semaphore" definition)
# --------------------------------------------------------------------------------------------
# B blocks each make P wait/post pairs; pair id = b * P + p.  Inside, the block adds
# addend[id] to `tally` with an atomic add, and when n == 1 also increments `total` with a
# plain load/store (exclusion makes it exact).  The peak number of simultaneous holders is
# recorded and must not exceed n.


def sem_final(nblocks: int, pairs: int, n_init: int, addend: np.ndarray) -> dict:
    addend = np.asarray(addend, dtype=np.uint32)
    assert addend.shape == (nblocks * pairs,)
    out = {
        "count": np.full(nblocks, pairs, dtype=np.uint32),
        "tally": np.uint32(int(addend.astype(np.uint64).sum()) & M32),
        "occupancy_limit": n_init,
    }
    if n_init == 1:
        out["total"] = np.uint32((nblocks * pairs) & M32)
    return out


# --------------------------------------------------------------------------------------------
# Condition-variable workload (a bounded producer/consumer queue; condition variables are
# future work in Section 7): every item is put once and taken exactly once.
# --------------------------------------------------------------------------------------------


def condvar_final(value: np.ndarray, producers: int, items_per_producer: int, consumers: int) -> dict:
    """seen[i] = 1 for every item; the consumers' int64 sums add up to the sum of the values
    (read as int32); each consumer takes producers * items_per_producer / consumers items."""
    n = producers * items_per_producer
    v = np.asarray(value, dtype=np.uint32).view(np.int32).astype(np.int64)
    assert v.shape == (n,) and n % consumers == 0
    return {"seen": np.ones(n, dtype=np.uint32), "total": int(v.sum()),
            "count": np.full(consumers, n // consumers, dtype=np.uint32)}


# --------------------------------------------------------------------------------------------
# Batched many-mutex workload (mutex definition, applied per key)
# --------------------------------------------------------------------------------------------


def batched_final(keys: np.ndarray, adds: np.ndarray, nkeys: int) -> dict:
    """sum[k] = sum of adds[i] over i with keys[i] == k (mod 2^64); count[k] = #{i: keys[i]==k}."""
    keys = np.asarray(keys, dtype=np.int64)
    u = np.asarray(adds).view(np.uint64)
    s = np.zeros(nkeys, dtype=np.uint64)
    np.add.at(s, keys, u)
    cnt = np.bincount(keys, minlength=nkeys).astype(np.uint64)
    return {"sum": s.view(np.int64), "count": cnt}


# --------------------------------------------------------------------------------------------
# Serving workload: each request is an int32 segmented sum, accumulated in int64
# --------------------------------------------------------------------------------------------


def serve_final(offset: np.ndarray, length: np.ndarray, pool: np.ndarray) -> np.ndarray:
    pool = np.asarray(pool, dtype=np.int32)
    res = np.empty(len(offset), dtype=np.int64)
    for q, (o, n) in enumerate(zip(np.asarray(offset), np.asarray(length))):
        res[q] = pool[int(o):int(o) + int(n)].astype(np.int64).sum()
    return res
