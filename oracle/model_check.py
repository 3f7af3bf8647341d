"""Explicit-state model checker for the synchronization algorithms (oracle; test infra only).

Each algorithm runs as one step machine per block.  One step makes at most one shared-memory
access, and every access is atomic as a whole (sequential consistency, interleaving
semantics).  The checker enumerates every reachable state of `nproc` blocks that each perform
`ops` operations (lock/unlock pairs, wait/post pairs or barrier crossings), and reports:

  * safety: at most one block in a mutex's critical section, at most n in a semaphore's,
    no block past barrier round r before every block has arrived at round r, and, for the
    fair kinds, grants in ticket order;
  * progress: from every reachable state some state with all blocks done stays reachable
    (no deadlock, and no livelock that no schedule can escape).

Words are uint32 and wrap; ticket and epoch comparisons use the signed difference, so a run
can start its counters just below 2^32 to exercise wrap-around.

The algorithms follow Section 5 ("Design") and the pseudocode of the Appendix:
  SpinMutex     spin-lock mutex with optional backoff (Algorithm 1; "Spin-Lock Mutex")
  TicketMutex   fetch-and-add mutex ("FA Mutex"; Section 5, "Fetch-and-Add Mutex")
  QueueMutex    sleep-waiting queue lock: each waiter polls its own slot of a ring of flags
  RingMutex     the paper's ring-buffer sleeping mutex (Section 5, "design alternative")
  CohortMutex   two-die cohort lock: a ticket lock per die under a global ticket lock
  McsCohortMutex    the cluster cohort lock with an MCS queue per cluster (pushed grants)
  CarryCohortMutex  the cohort lock whose records carry the guarded data (batched kernel)
  CarryMcsHierMutex the same over three levels: an MCS queue per cluster, a ticket lock per
                    die, a global ticket lock (batched kernel)
  CondVarQueue  condition variables (ticket and signal counters) on a bounded buffer
  SpinSem       spin-lock semaphore with optional backoff ("Spin-Lock Semaphore")
  SleepSem      sleeping (FA) semaphore ("Sleeping Semaphore")
  AtomicBarrier two-stage atomic-counter barrier (Section 5, "Barrier")
  FlagBarrier   decentralized XF flag barrier (Section 5, "Barrier")
  TreeBarrier   combining-tree barrier (Section 2, hierarchical barriers)
  TreeCountBarrier  the same with node counters that only grow; the root's last add releases
  ShardedBarrier  arrivals counted on several counters, gathered by the master block
  ClusterBarrier  barrier inside groups of c blocks, then one leader per group globally
  ClusterCountBarrier  the same, with a growing counter over the leaders as the global stage
  DieBarrier    per-die counters and release words, a top counter between the dies
  SplitBarrier  S arrival counters under a top counter, R copies of the release word
  CountBarrier  one growing arrival counter that every block polls
  ExchangeBarrier  the counting barrier whose arrivals carry one value per block, no fence
  RingPublish   the serving ring's entry, written as two single-copy-atomic halves, no fence
  ServeSlot     a serving slot: generation-tagged chunk claims by fetch-and-add, reuse
Mutation variants with a planted mistake (`broken=...`) exist so that tests can show the
checker catches each kind of error.
"""
from __future__ import annotations

from dataclasses import dataclass, field

M32 = 0xFFFFFFFF
DONE = -1


def s_gt(a: int, b: int) -> bool:
    """a > b for wrapping uint32 counters: the signed 32-bit difference is positive."""
    d = (a - b) & M32
    return d != 0 and d < 0x80000000


def s_ge(a: int, b: int) -> bool:
    return ((a - b) & M32) < 0x80000000


def inc(x: int, k: int = 1) -> int:
    return (x + k) & M32


@dataclass
class Result:
    states: int = 0
    violation: str | None = None
    trace: list = field(default_factory=list)
    stuck_state: tuple | None = None

    @property
    def ok(self) -> bool:
        return self.violation is None


def _set(t: tuple, i: int, v) -> tuple:
    return t[:i] + (v,) + t[i + 1:]


# --------------------------------------------------------------------------------------------
# Mutexes
# --------------------------------------------------------------------------------------------
# Local state: (pc, ops_done, reg_a, reg_b).  Events: ("enter", ticket|None), ("exit",).
PC_ENTER, PC_EXIT = 50, 51


class SpinMutex:
    """Spin-lock mutex (Algorithm 1 and the Appendix's spin-lock mutex).

    lock: repeat OldVal <- atomicExch(M, 1) until OldVal = 0, with Backoff() after each
    failure when UseBackoff; unlock: M <- 0 (plain store; Algorithm 1 uses atomicExch(M, 0),
    selected with atomic_unlock).  cas=True replaces the exchange by atomicCAS(M, 0, 1).
    broken="test_then_set" splits the atomic into a load and a later store.
    """
    kind, capacity, fifo = "mutex", 1, False

    def __init__(self, backoff=False, cas=False, atomic_unlock=False, broken=None):
        self.backoff, self.cas, self.atomic_unlock, self.broken = backoff, cas, atomic_unlock, broken

    def init(self, nproc, ops):
        return (0,), tuple((0, 0, 0, 0) for _ in range(nproc))

    def step(self, p, loc, sh, nproc, ops):
        pc, k, a, b = loc
        M = sh[0]
        if pc == 0:
            if self.broken == "test_then_set":
                return ((9, k, a, b) if M == 0 else (0, k, a, b)), sh, None
            old = M
            if self.cas:
                if M == 0:
                    sh = (1,)
            else:
                sh = (1,)
            if old == 0:
                return (PC_ENTER, k, a, b), sh, None
            return ((1 if self.backoff else 0), k, a, b), sh, None
        if pc == 9:  # second half of the broken test-then-set
            return (PC_ENTER, k, a, b), (1,), None
        if pc == 1:  # Backoff(): no memory access
            return (0, k, a, b), sh, None
        if pc == PC_ENTER:
            return (PC_EXIT, k, a, b), sh, ("enter", None)
        if pc == PC_EXIT:
            return (2, k, a, b), sh, ("exit",)
        if pc == 2:  # unlock
            k += 1
            return ((0 if k < ops else DONE), k, a, b), (0,), None
        raise AssertionError(pc)


class TicketMutex:
    """Fetch-and-add (ticket) mutex.

    lock: TicketNumber <- fetch-and-add(ticket, 1); wait until turn = TicketNumber.
    unlock (literal=True): turn <- turn + 1 as a plain read then write (the Appendix's FA
    mutex); literal=False stores TicketNumber + 1, which is the same value because only the
    holder writes turn.  broken="no_advance" stores TicketNumber (the turn never moves on).
    """
    kind, capacity, fifo = "mutex", 1, True

    def __init__(self, literal=False, base=0, broken=None):
        self.literal, self.base, self.broken = literal, base & M32, broken

    def init(self, nproc, ops):
        return (self.base, self.base), tuple((0, 0, 0, 0) for _ in range(nproc))

    def step(self, p, loc, sh, nproc, ops):
        pc, k, t, r = loc
        ticket, turn = sh
        if pc == 0:
            return (1, k, ticket, r), (inc(ticket), turn), None
        if pc == 1:
            return ((PC_ENTER if turn == t else 1), k, t, r), sh, None
        if pc == PC_ENTER:
            return (PC_EXIT, k, t, r), sh, ("enter", t)
        if pc == PC_EXIT:
            return (2, k, t, r), sh, ("exit",)
        if pc == 2:
            if self.literal:
                return (3, k, t, turn), sh, None
            new = t if self.broken == "no_advance" else inc(t)
            k += 1
            return ((0 if k < ops else DONE), k, t, r), (ticket, new), None
        if pc == 3:
            k += 1
            return ((0 if k < ops else DONE), k, t, r), (ticket, inc(r)), None
        raise AssertionError(pc)


class CarryTicketMutex:
    """Ticket mutex whose turn word carries the guarded data (the batched kernel's
    GSYNC_BATCHED_TICKET_CARRY; a GB300 design, not in the paper).

    lock: t <- fetch-and-add(ticket, 1); read the record (turn, count, sum) as one access until
    turn = t.  The critical section adds f(t) = t + 1 to the sum it read and counts one more.
    unlock: write the record (t + 1, count + 1, sum + f(t)) as one access.  Each holder must
    see its predecessors' data: at entry, count = t - base and sum = the sum of f over the
    earlier tickets (mod 2^32 here), else a violation is reported.
    broken="split_read" reads the data first and the turn after, as two accesses (a stale
    read); broken="turn_only" publishes the turn without the data.
    The device reads and writes the record with relaxed 16-byte accesses.  The protocol
    communicates only through the ticket counter and this one record, each access to it is a
    single access, and a holder's write depends on the value its read returned.  So coherence
    on the record orders the hand-offs as the interleavings here do, and no fence is needed.
    """
    kind, capacity, fifo = "mutex", 1, True

    def __init__(self, base=0, broken=None):
        self.base, self.broken = base & M32, broken

    def _f(self, t):
        return (t + 1) & M32

    def _want_sum(self, t):
        s, u = 0, self.base
        while u != t:
            s = (s + self._f(u)) & M32
            u = inc(u)
        return s

    def init(self, nproc, ops):
        # shared: (ticket, turn, count, sum); local: (pc, k, t, count read, sum read)
        return (self.base, self.base, 0, 0), tuple((0, 0, 0, 0, 0) for _ in range(nproc))

    def step(self, p, loc, sh, nproc, ops):
        pc, k, t, c, sm = loc
        ticket, turn, count, total = sh
        if pc == 0:
            return (1, k, ticket, c, sm), (inc(ticket), turn, count, total), None
        if pc == 1:
            if self.broken == "split_read":  # data now, turn in the next step
                return (4, k, t, count, total), sh, None
            return ((PC_ENTER if turn == t else 1), k, t, count, total), sh, None
        if pc == 4:
            return ((PC_ENTER if turn == t else 1), k, t, c, sm), sh, None
        if pc == PC_ENTER:
            if c != ((t - self.base) & M32) or sm != self._want_sum(t):
                return loc, sh, ("violation", f"ticket {t:#x} entered with count {c} and sum {sm}")
            return (PC_EXIT, k, t, c, sm), sh, ("enter", t)
        if pc == PC_EXIT:
            return (2, k, t, c, sm), sh, ("exit",)
        if pc == 2:
            k += 1
            nxt = ((0 if k < ops else DONE), k, t, c, sm)
            if self.broken == "turn_only":
                return nxt, (ticket, inc(t), count, total), None
            return nxt, (ticket, inc(t), inc(c), (sm + self._f(t)) & M32), None
        raise AssertionError(pc)


class QueueMutex:
    """Sleep-waiting queue lock with one flag slot per waiter (ring of Q slots, Q a power of 2).

    lock: t <- fetch-and-add(tail, 1); wait until flag[t mod Q] = t.
    unlock: flag[(t + 1) mod Q] <- t + 1.  Every waiter polls its own slot, so one unlock is
    seen by exactly one waiter.  Initial state for a first ticket `base`: tail = base,
    flag[base mod Q] = base, and every other slot holds the latest ticket below base that
    maps to it, which no pending waiter can equal.

    Planted mistakes: broken="unsigned_ge" waits until flag >= t compared as plain unsigned
    numbers (after the tickets wrap past 2^32, a slot's old value looks larger than a small
    new ticket); broken="own_slot" makes unlock write t + 1 into the holder's own slot instead
    of its successor's; broken="no_ring_wrap" computes the successor's slot as
    (t mod Q) + 1 without wrapping, so the store meant for slot 0 lands past the ring.
    """
    kind, capacity, fifo = "mutex", 1, True

    def __init__(self, q=4, base=0, broken=None):
        assert q & (q - 1) == 0
        self.q, self.base, self.broken = q, base & M32, broken

    def init(self, nproc, ops):
        assert self.q >= nproc
        flags = []
        for i in range(self.q):
            back = (self.base - i) % self.q
            flags.append((self.base - back) & M32)
        return (self.base,) + tuple(flags), tuple((0, 0, 0, 0) for _ in range(nproc))

    def step(self, p, loc, sh, nproc, ops):
        pc, k, t, r = loc
        q = self.q
        if pc == 0:
            return (1, k, sh[0], r), _set(sh, 0, inc(sh[0])), None
        if pc == 1:
            f = sh[1 + (t % q)]
            mine = f >= t if self.broken == "unsigned_ge" else f == t
            return ((PC_ENTER if mine else 1), k, t, r), sh, None
        if pc == PC_ENTER:
            return (PC_EXIT, k, t, r), sh, ("enter", t)
        if pc == PC_EXIT:
            return (2, k, t, r), sh, ("exit",)
        if pc == 2:
            k += 1
            n = inc(t)
            nxt = (0 if k < ops else DONE)
            if self.broken == "own_slot":
                return (nxt, k, t, r), _set(sh, 1 + (t % q), n), None
            if self.broken == "no_ring_wrap":
                i = (t % q) + 1
                return (nxt, k, t, r), (sh if i == q else _set(sh, 1 + i, n)), None  # slot q: past the ring
            return (nxt, k, t, r), _set(sh, 1 + (n % q), n), None
        raise AssertionError(pc)


class RingMutex:
    """The paper's ring-buffer sleeping mutex (Section 5, design alternative to FA).

    An arriving block places itself at the end of a ring buffer and keeps checking whether the
    entry at the front is itself; unlock increments the head pointer.  Here the end slot is
    claimed with fetch-and-add on `tail` and then written with the block id; a waiter reads
    `head`, then ring[head mod Q], and enters when that entry is its own id.  Unlock clears the
    holder's entry before advancing `head`: without the clear (broken="no_clear") a block can
    match its own stale entry from an earlier lap of the ring.
    """
    kind, capacity, fifo = "mutex", 1, True
    EMPTY = M32

    def __init__(self, q=4, broken=None):
        self.q, self.broken = q, broken

    def init(self, nproc, ops):
        return (0, 0) + tuple([self.EMPTY] * self.q), tuple((0, 0, 0, 0) for _ in range(nproc))

    def step(self, p, loc, sh, nproc, ops):
        pc, k, t, h = loc
        q = self.q
        head, tail = sh[0], sh[1]
        if pc == 0:      # claim the end slot
            return (3, k, tail, h), _set(sh, 1, inc(tail)), None
        if pc == 3:      # place itself in the ring
            return (1, k, t, h), _set(sh, 2 + (t % q), p), None
        if pc == 1:      # read the head pointer
            return (4, k, t, head), sh, None
        if pc == 4:      # is the front entry this block?
            return ((PC_ENTER if sh[2 + (h % q)] == p else 1), k, t, h), sh, None
        if pc == PC_ENTER:
            return (PC_EXIT, k, t, h), sh, ("enter", t)
        if pc == PC_EXIT:
            return ((5 if self.broken == "no_clear" else 2), k, t, h), sh, ("exit",)
        if pc == 2:      # clear own entry
            return (5, k, t, h), _set(sh, 2 + (t % q), self.EMPTY), None
        if pc == 5:      # advance the head
            k += 1
            return ((0 if k < ops else DONE), k, t, h), _set(sh, 0, inc(t)), None
        raise AssertionError(pc)


class CondVarQueue:
    """Condition variables (the paper names them as future work, without an algorithm): a
    bounded buffer of capacity C guarded by one mutex and two condition variables, not_empty
    and not_full.  Blocks p < P produce, the rest consume; every block makes `ops` operations,
    so the producers' and consumers' operation totals must match.

    A condition variable is two counters: tickets (waiters so far) and signals (waiters
    released so far).  wait(cv): with the mutex held, t <- tickets; tickets <- t + 1; release
    the mutex; poll until signals > t (wrap-safe); take the mutex again.  signal(cv), with the
    mutex held: if signals != tickets then signals <- signals + 1 (release the oldest waiter;
    a signal with no waiter is lost, as usual).  broadcast: signals <- tickets.  The mutex is
    modelled as an atomic test-and-set word (its own correctness is checked elsewhere).

    Safety: one block at a time updates the buffer (the mutex), and the buffer never under-
    or overflows (a "violation" event); progress: every schedule can finish, which needs
    P x ops produced = (nproc - P) x ops consumed.  broken="signal_before_ticket": a waiter releases the mutex before
    taking its ticket (a signal in between is lost: deadlock).  broken="no_recheck": a woken
    waiter does not re-test the condition (another block can take the item first: underflow).
    """
    kind, capacity, fifo = "mutex", 1, False

    def __init__(self, P=1, C=1, broadcast=False, broken=None):
        self.P, self.C, self.broadcast, self.broken = P, C, broadcast, broken

    def init(self, nproc, ops):
        # (lock, count, ne_tickets, ne_signals, nf_tickets, nf_signals)
        return (0, 0, 0, 0, 0, 0), tuple((0, 0, 0, 0) for _ in range(nproc))

    def step(self, p, loc, sh, nproc, ops):
        pc, k, t, r = loc
        lock, count, net, nes, nft, nfs = sh
        producer = p < self.P
        # cv indices: the condition this block waits on, and the one it signals
        W = (4, 5) if producer else (2, 3)   # producers wait for not_full, consumers for not_empty
        S = (2, 3) if producer else (4, 5)

        if pc == 0:      # lock
            if lock:
                return loc, sh, None
            return (1, k, t, r), _set(sh, 0, 1), None
        if pc == 1:      # test the condition (under the mutex)
            ready = count < self.C if producer else count > 0
            return ((10 if ready else (2 if self.broken != "signal_before_ticket" else 20)), k, t, r), sh, None
        if pc == 2:      # wait: take a ticket (mutex held) ...
            tk = sh[W[0]]
            return (3, k, tk, r), _set(sh, W[0], inc(tk)), None
        if pc == 3:      # ... release the mutex ...
            return (4, k, t, r), _set(sh, 0, 0), None
        if pc == 4:      # ... wait for a signal past the ticket ...
            if not s_gt(sh[W[1]], t):
                return loc, sh, None
            return (5, k, t, r), sh, None
        if pc == 5:      # ... and take the mutex again
            if lock:
                return loc, sh, None
            return ((1 if self.broken != "no_recheck" else 10), k, t, r), _set(sh, 0, 1), None
        if pc == 20:     # broken: release first, then take the ticket
            return (21, k, t, r), _set(sh, 0, 0), None
        if pc == 21:
            tk = sh[W[0]]
            return (4, k, tk, r), _set(sh, W[0], inc(tk)), None
        if pc == 10:     # the buffer update (the critical section)
            return (11, k, t, r), sh, ("enter", None)
        if pc == 11:
            c2 = count + 1 if producer else count - 1
            if c2 < 0 or c2 > self.C:
                return loc, sh, ("violation", f"buffer count {c2} outside 0..{self.C}")
            return (12, k, t, r), _set(sh, 1, c2), ("exit",)
        if pc == 12:     # signal (or broadcast) the other side, mutex held
            tk, sg = sh[S[0]], sh[S[1]]
            if sg != tk:
                sg = tk if self.broadcast else inc(sg)
            return (13, k, t, r), _set(sh, S[1], sg), None
        if pc == 13:     # unlock
            k += 1
            return ((0 if k < ops else DONE), k, t, r), _set(sh, 0, 0), None
        raise AssertionError(pc)


# --------------------------------------------------------------------------------------------
# Semaphores
# --------------------------------------------------------------------------------------------


class CohortMutex:
    """Two-level cohort lock over two dies (lock cohorting: Dice, Marathe and Shavit, PPoPP
    2012), the library's GB300 design that keeps hand-offs inside a die.

    Block p sits on die p mod 2 (group p mod `groups`: the library also runs the protocol
    over thread-block clusters, with the local lock in distributed shared memory).  Each die d has a local ticket counter next_d and a local turn
    word (served_d, word_d) read and written as one 64-bit access; word_d's OWNED bit says the
    die's cohort already holds the global ticket lock (gnext, gturn; 16-bit ticket compare).
    lock: t <- FA(next_d); wait until served_d = t; if OWNED, inherit the global lock (passes
      and global ticket from word_d); else g <- FA(gnext) mod 2^16, wait until gturn = g.
    unlock: if next_d != t + 1 (a local waiter) and passes + 1 < budget: (served_d, word_d) <-
      (t + 1, OWNED | passes + 1 | g); else gturn <- g + 1 mod 2^16, then (served_d, word_d)
      <- (t + 1, 0).
    Grants are FIFO within a die (the event carries the die and the local ticket).
    broken="no_global": the first of a cohort enters without the global lock.
    broken="owned_on_release": the release path also marks the local turn OWNED.
    broken="skip_ticket": a pass within the die serves ticket t + 2 instead of t + 1.
    broken="pass_always": passes within the die whether or not a local waiter exists, and
    past the budget (the global lock is never released: the other die starves).
    """
    kind, capacity, fifo = "mutex", 1, False
    OWNED = 0x80000000

    def __init__(self, budget=2, base=0, gbase=0, broken=None, groups=2):
        self.budget, self.base, self.gbase, self.broken = budget, base & M32, gbase & M32, broken
        self.dies = groups  # dies, or thread-block clusters: the protocol is the same

    def init(self, nproc, ops):
        b, g = self.base, self.gbase
        # (next_d, served_d, word_d) per group, then (gnext, gturn)
        return (b, b, 0) * self.dies + (g, g & 0xFFFF), tuple((0, 0, 0, 0) for _ in range(nproc))

    def step(self, p, loc, sh, nproc, ops):
        pc, k, t, c = loc
        d = p % self.dies
        nx, sv, wd = sh[3 * d], sh[3 * d + 1], sh[3 * d + 2]
        G = 3 * self.dies
        gnext, gturn = sh[G], sh[G + 1]

        def put_local(nx2, sv2, wd2):
            return sh[:3 * d] + (nx2, sv2, wd2) + sh[3 * d + 3:]

        def finish():
            k2 = k + 1
            return (0 if k2 < ops else DONE), k2

        if pc == 0:
            return (1, k, nx, c), put_local(inc(nx), sv, wd), None
        if pc == 1:
            if sv != t:
                return loc, sh, None
            if wd & self.OWNED:
                return (PC_ENTER, k, t, wd & ~self.OWNED & M32), sh, None
            if self.broken == "no_global":
                return (PC_ENTER, k, t, 0), sh, None
            return (2, k, t, c), sh, None
        if pc == 2:
            return (3, k, t, gnext & 0xFFFF), sh[:G] + (inc(gnext), gturn), None
        if pc == 3:
            return ((PC_ENTER if (gturn & 0xFFFF) == c else 3), k, t, c), sh, None
        if pc == PC_ENTER:
            return (PC_EXIT, k, t, c), sh, ("enter", (d, t))
        if pc == PC_EXIT:
            return (4, k, t, c), sh, ("exit",)
        if pc == 4:
            passes = (c >> 16) & 0x7FFF
            if self.broken == "pass_always":
                return (5, k, t, c), sh, None
            waiter = nx != inc(t)
            return ((5 if waiter and passes + 1 < self.budget else 6), k, t, c), sh, None
        if pc == 5:
            passes, g = (c >> 16) & 0x7FFF, c & 0xFFFF
            pc2, k2 = finish()
            word = self.OWNED | ((passes + 1) << 16) | g
            return (pc2, k2, t, c), put_local(nx, inc(t, 2 if self.broken == "skip_ticket" else 1), word), None
        if pc == 6:
            g = c & 0xFFFF
            return (7, k, t, c), sh[:G + 1] + ((g + 1) & 0xFFFF,), None
        if pc == 7:
            pc2, k2 = finish()
            word = self.OWNED if self.broken == "owned_on_release" else 0
            return (pc2, k2, t, c), put_local(nx, inc(t), word), None
        raise AssertionError(pc)


class CarryCohortMutex:
    """The cohort lock (CohortMutex) whose records carry what it guards (the batched kernel's
    GSYNC_BATCHED_COHORT_CARRY; a GB300 design, not in the paper).

    Each group d has a local ticket counter next_d and a local record (served_d, word_d,
    sum_d), and the global lock a ticket counter gnext and a global record (gturn, gsum); each
    record is read and written as one access.  A holder takes the sum from the record that
    granted it the lock: the local record when word_d is OWNED (the cohort inherits the global
    lock), else the global record once gturn shows its global ticket.  It adds its own
    contribution, then passes the sum on in the record it releases: the local record with
    OWNED when a local waiter is queued and the budget allows, else the global record (then the
    local record, not OWNED).  A ghost total, updated as each holder leaves, checks that every
    holder enters with the sum of all earlier contributions.
    broken="global_reads_local": a holder granted by the global lock takes the sum from its
    local record; broken="pass_without_add": a local pass carries the sum the holder entered
    with, without its own contribution.
    """
    kind, capacity, fifo = "mutex", 1, False
    OWNED = 0x80000000

    def __init__(self, budget=2, groups=2, broken=None):
        self.budget, self.broken = budget, broken
        self.base = 0
        self.dies = groups

    def init(self, nproc, ops):
        # (next_d, served_d, word_d, sum_d) per group; (gnext, gturn, gsum); the ghost total
        return (0, 0, 0, 0) * self.dies + (0, 0, 0) + (0,), tuple((0, 0, 0, 0, 0) for _ in range(nproc))

    def step(self, p, loc, sh, nproc, ops):
        pc, k, t, c, s = loc
        d = p % self.dies
        nx, sv, wd, sd = sh[4 * d:4 * d + 4]
        G = 4 * self.dies
        gnext, gturn, gsum, truth = sh[G], sh[G + 1], sh[G + 2], sh[G + 3]
        f = (p + 1 + 16 * k) & M32  # this acquisition's contribution

        def put_local(rec):
            return sh[:4 * d] + (nx,) + rec + sh[4 * d + 4:]

        def finish():
            k2 = k + 1
            return (0 if k2 < ops else DONE), k2

        if pc == 0:
            return (1, k, nx, c, s), sh[:4 * d] + (inc(nx), sv, wd, sd) + sh[4 * d + 4:], None
        if pc == 1:  # one read of the local record
            if sv != t:
                return loc, sh, None
            if wd & self.OWNED:
                return (PC_ENTER, k, t, wd & ~self.OWNED & M32, sd), sh, None
            return (2, k, t, c, s), sh, None
        if pc == 2:
            return (3, k, t, gnext & 0xFFFF, s), sh[:G] + (inc(gnext), gturn, gsum, truth), None
        if pc == 3:  # one read of the global record
            if (gturn & 0xFFFF) != c:
                return loc, sh, None
            return (PC_ENTER, k, t, c, sd if self.broken == "global_reads_local" else gsum), sh, None
        if pc == PC_ENTER:
            if s != truth:
                return loc, sh, ("violation", f"block {p} entered with sum {s}, expected {truth}")
            return (PC_EXIT, k, t, c, s), sh, ("enter", (d, t))
        if pc == PC_EXIT:
            return (4, k, t, c, s), sh[:G + 3] + ((truth + f) & M32,), ("exit",)
        if pc == 4:
            passes = (c >> 16) & 0x7FFF
            waiter = nx != inc(t)
            return ((5 if waiter and passes + 1 < self.budget else 6), k, t, c, s), sh, None
        if pc == 5:  # pass within the group: the local record carries the sum
            passes, g = (c >> 16) & 0x7FFF, c & 0xFFFF
            out = s if self.broken == "pass_without_add" else (s + f) & M32
            pc2, k2 = finish()
            return (pc2, k2, t, c, s), put_local((inc(t), self.OWNED | ((passes + 1) << 16) | g, out)), None
        if pc == 6:  # release the global lock: the global record carries the sum
            g = c & 0xFFFF
            return (7, k, t, c, s), sh[:G + 1] + ((g + 1) & 0xFFFF, (s + f) & M32) + sh[G + 3:], None
        if pc == 7:
            pc2, k2 = finish()
            return (pc2, k2, t, c, s), put_local((inc(t), 0, (s + f) & M32)), None
        raise AssertionError(pc)


class CarryMcsHierMutex:
    """Three-level carrying cohort lock (the batched kernel's GSYNC_BATCHED_CLUSTER_DIE_CARRY;
    a GB300 design, not in the paper): an MCS queue (Mellor-Crummey and Scott, 1991) per
    cluster, under a ticket lock per die, under a global ticket lock, every level passing the
    guarded sum in its records.

    The cluster's tail holds (block, seq) of the last block to queue, or None when the cluster
    lock is free.  A block queues with seq = its own count of queueings plus one: it swaps
    itself into the tail; if the tail was None it holds the cluster lock at once (not owned:
    it continues at the die level); else it links itself into its predecessor's node, link =
    (block, seq, predecessor's seq), and polls its own node's record until the record's seq is
    its own.  A holder passes the lock by writing (successor's seq, owned word or None, sum)
    into its successor's node: the successor is the one whose link names the holder's current
    seq.  Without a successor it swaps the tail back to None if the tail still names it, and
    otherwise waits for the link.  Records and links are never reset: every one is checked
    against the seq it must carry.  Block p belongs to cluster cluster_of[p], cluster c to die
    die_of[c].  A die has a ticket counter and a record (served, word, sum) whose word, when
    owned, carries the global ticket and the die's pass count; the global lock a ticket counter
    and a record (turn, sum).  An owned cluster record carries the die ticket, the global ticket
    and both pass counts.  Served tickets, the global turn and record seqs are compared in 16
    bits, as on the device.  A holder takes the sum from the record that granted it the lock.
    It passes to its linked successor while the cluster budget allows; else to the next
    waiting cluster of its die (the die record owned) while the die budget allows, then frees
    its cluster; else it releases the global lock, then its die, then its cluster.  A ghost
    total checks that every holder enters with the sum of all earlier contributions.
    broken="no_seq_check": a block takes any record in its node as its grant;
    broken="stale_link": a holder trusts a link left by an earlier round; broken="no_cas": a
    holder without a linked successor leaves the tail as it is.
    """
    kind, capacity, fifo = "mutex", 1, False
    M16 = 0xFFFF

    def __init__(self, cluster_of=(0, 0, 1), die_of=(0, 0), cbudget=2, dbudget=2, broken=None):
        self.cluster_of, self.die_of = tuple(cluster_of), tuple(die_of)
        self.cbudget, self.dbudget, self.broken = cbudget, dbudget, broken
        self.nc, self.nd = len(self.die_of), max(self.die_of) + 1

    def init(self, nproc, ops):
        nodes = (None, None) * nproc                  # (link, record) per block
        tails = (None,) * self.nc
        dl = (0, 0, None, 0) * self.nd                # (next, served, word, sum) per die
        # loc: pc, k, seq, succ, td, cp, dp, g, s
        return nodes + tails + dl + (0, 0, 0) + (0,), tuple((0, 0, 0, None, 0, 0, 0, 0, 0) for _ in range(nproc))

    def step(self, p, loc, sh, nproc, ops):
        pc, k, seq, succ, td, cp, dp, g, s = loc
        c = self.cluster_of[p]
        d = self.die_of[c]
        N0 = 0
        T0 = 2 * nproc
        D0 = T0 + self.nc + 4 * d
        G = T0 + self.nc + 4 * self.nd
        link, rec = sh[N0 + 2 * p], sh[N0 + 2 * p + 1]
        tail = sh[T0 + c]
        dnext, dserved, dword, dsum = sh[D0:D0 + 4]
        gnext, gturn, gsum, truth = sh[G:G + 4]
        f = (p + 1 + 16 * k) & M32
        out = (s + f) & M32

        def put(i, vals):
            return sh[:i] + vals + sh[i + len(vals):]

        def L(**kw):
            v = dict(pc=pc, k=k, seq=seq, succ=succ, td=td, cp=cp, dp=dp, g=g, s=s)
            v.update(kw)
            return (v["pc"], v["k"], v["seq"], v["succ"], v["td"], v["cp"], v["dp"], v["g"], v["s"])

        def finish(**kw):
            k2 = k + 1
            return L(pc=(0 if k2 < ops else DONE), k=k2, succ=None, **kw)

        def linked():  # the successor named by this block's link for its current seq
            if link is None:
                return None
            sp, sseq, pseq = link
            if pseq != seq and self.broken != "stale_link":
                return None
            return (sp, sseq)

        if pc == 0:  # swap into the tail
            seq2 = seq + 1
            if tail is None:
                return L(pc=2, seq=seq2, cp=0), put(T0 + c, ((p, seq2),)), None
            return L(pc=1, seq=seq2, succ=tail), put(T0 + c, ((p, seq2),)), None
        if pc == 1:  # link into the predecessor's node (succ holds the predecessor here)
            pp, pseq = succ
            return L(pc=20, succ=None), put(N0 + 2 * pp, ((p, seq, pseq),)), None
        if pc == 20:  # poll this block's own record
            if rec is None or (rec[0] != seq & self.M16 and self.broken != "no_seq_check"):
                return loc, sh, None
            _, word, rsum = rec
            if word is not None:
                _, cp2, dp2, td2, g2 = word
                return L(pc=PC_ENTER, cp=cp2, dp=dp2, td=td2, g=g2, s=rsum), sh, None
            return L(pc=2, cp=0), sh, None
        if pc == 2:  # die ticket
            return L(pc=3, td=dnext), put(D0, (inc(dnext),)), None
        if pc == 3:
            if dserved != td & self.M16:
                return loc, sh, None
            if dword is not None:
                _, dp2, g2 = dword
                return L(pc=PC_ENTER, cp=0, dp=dp2, g=g2, s=dsum), sh, None
            return L(pc=4, cp=0, dp=0), sh, None
        if pc == 4:  # global ticket
            return L(pc=5, g=gnext & self.M16), put(G, (inc(gnext),)), None
        if pc == 5:
            if gturn != g:
                return loc, sh, None
            return L(pc=PC_ENTER, cp=0, dp=0, s=gsum), sh, None
        if pc == PC_ENTER:
            if s != truth:
                return loc, sh, ("violation", f"block {p} entered with sum {s}, expected {truth}")
            return L(pc=PC_EXIT), sh, ("enter", (c, seq))
        if pc == PC_EXIT:
            return L(pc=6), put(G + 3, ((truth + f) & M32,)), ("exit",)
        if pc == 6:  # one read of this block's link
            nxt = linked()
            if nxt is not None and cp + 1 < self.cbudget:
                return L(pc=7, succ=nxt), sh, None
            return L(pc=8, succ=nxt), sh, None
        if pc == 7:  # pass within the cluster: push an owned record to the successor
            sp, sseq = succ
            word = ("own", cp + 1, dp, td & self.M16, g)
            return finish(), put(N0 + 2 * sp + 1, ((sseq & self.M16, word, out),)), None
        if pc == 8:  # a waiter of this die?
            waiter = dnext != inc(td)
            return L(pc=(9 if waiter and dp + 1 < self.dbudget else 10)), sh, None
        if pc == 9:  # pass within the die
            return L(pc=11), put(D0 + 1, (inc(td) & self.M16, ("own", dp + 1, g), out)), None
        if pc == 10:  # release the global lock, then the die
            return L(pc=12), put(G + 1, ((g + 1) & self.M16, out)), None
        if pc == 12:
            return L(pc=11), put(D0 + 1, (inc(td) & self.M16, None, out)), None
        if pc == 11:  # release the cluster: push a record that is not owned, or free the tail
            nxt = succ if succ is not None else linked()
            if nxt is not None:
                sp, sseq = nxt
                return finish(), put(N0 + 2 * sp + 1, ((sseq & self.M16, None, out),)), None
            return L(pc=13), sh, None
        if pc == 13:  # compare-and-swap the tail back to None
            if tail == (p, seq) or self.broken == "no_cas":
                if self.broken == "no_cas":
                    return finish(), sh, None
                return finish(), put(T0 + c, (None,)), None
            return L(pc=14), sh, None
        if pc == 14:  # a successor swapped in: wait for its link
            nxt = linked()
            if nxt is None:
                return loc, sh, None
            sp, sseq = nxt
            return finish(), put(N0 + 2 * sp + 1, ((sseq & self.M16, None, out),)), None
        raise AssertionError(pc)


class McsCohortMutex:
    """Cluster cohort lock whose local level is an MCS queue (Mellor-Crummey and Scott, 1991)
    with pushed grants: the mutex kind GSYNC_MUTEX_CLUSTER_MCS (a GB300 design, not in the
    paper).  The global level is a ticket lock, as in CohortMutex.

    The cluster's tail holds (block, seq) of the last block to queue, or None when the cluster
    lock is free.  A block queues with seq = its own count of queueings plus one: it swaps
    itself into the tail; if the tail was None it holds the cluster lock (not owned) and takes
    a global ticket; else it links itself into its predecessor's node, link = (block, seq,
    predecessor's seq), and polls its own node's record until the record's seq is its own.  The
    holder passes the lock by writing (successor's seq, owned word or None) into its linked
    successor's node: owned (the global lock stays with the cluster) while the budget allows,
    else it releases the global lock first and pushes a record that is not owned.  Without a
    linked successor it releases the global lock and swaps the tail back to None if the tail
    still names it, else waits for the link.  Records and links are checked against the seq
    they carry and never reset.  Mutual exclusion is checked on the critical section.
    broken="no_seq_check", "stale_link" and "no_cas" as in CarryMcsHierMutex;
    broken="owned_after_release": a holder that released the global lock still pushes an
    owned record.
    """
    kind, capacity, fifo = "mutex", 1, False
    M16 = 0xFFFF

    def __init__(self, cluster_of=(0, 0, 1), budget=2, broken=None):
        self.cluster_of, self.budget, self.broken = tuple(cluster_of), budget, broken
        self.nc = max(self.cluster_of) + 1

    def init(self, nproc, ops):
        # nodes (link, record) per block; tails per cluster; (gnext, gturn)
        return (None, None) * nproc + (None,) * self.nc + (0, 0), \
            tuple((0, 0, 0, None, 0, 0) for _ in range(nproc))

    def step(self, p, loc, sh, nproc, ops):
        pc, k, seq, succ, cp, g = loc
        c = self.cluster_of[p]
        T0 = 2 * nproc
        G = T0 + self.nc
        link, rec = sh[2 * p], sh[2 * p + 1]
        tail = sh[T0 + c]
        gnext, gturn = sh[G], sh[G + 1]

        def put(i, vals):
            return sh[:i] + vals + sh[i + len(vals):]

        def L(**kw):
            v = dict(pc=pc, k=k, seq=seq, succ=succ, cp=cp, g=g)
            v.update(kw)
            return (v["pc"], v["k"], v["seq"], v["succ"], v["cp"], v["g"])

        def finish():
            k2 = k + 1
            return L(pc=(0 if k2 < ops else DONE), k=k2, succ=None)

        def linked():
            if link is None:
                return None
            sp, sseq, pseq = link
            if pseq != seq and self.broken != "stale_link":
                return None
            return (sp, sseq)

        if pc == 0:  # swap into the tail
            seq2 = seq + 1
            if tail is None:
                return L(pc=2, seq=seq2, cp=0), put(T0 + c, ((p, seq2),)), None
            return L(pc=1, seq=seq2, succ=tail), put(T0 + c, ((p, seq2),)), None
        if pc == 1:  # link into the predecessor's node
            pp, pseq = succ
            return L(pc=20, succ=None), put(2 * pp, ((p, seq, pseq),)), None
        if pc == 20:  # poll this block's own record
            if rec is None or (rec[0] != seq & self.M16 and self.broken != "no_seq_check"):
                return loc, sh, None
            if rec[1] is not None:
                _, cp2, g2 = rec[1]
                return L(pc=PC_ENTER, cp=cp2, g=g2), sh, None
            return L(pc=2, cp=0), sh, None
        if pc == 2:  # global ticket
            return L(pc=3, g=gnext & self.M16), put(G, (inc(gnext),)), None
        if pc == 3:
            if gturn & self.M16 != g:
                return loc, sh, None
            return L(pc=PC_ENTER, cp=0), sh, None
        if pc == PC_ENTER:
            return L(pc=PC_EXIT), sh, ("enter", None)
        if pc == PC_EXIT:
            return L(pc=6), sh, ("exit",)
        if pc == 6:  # one read of this block's link
            nxt = linked()
            if nxt is not None and cp + 1 < self.budget:
                return L(pc=7, succ=nxt), sh, None
            return L(pc=10, succ=nxt), sh, None
        if pc == 7:  # pass within the cluster: the global lock stays
            sp, sseq = succ
            return finish(), put(2 * sp + 1, ((sseq & self.M16, ("own", cp + 1, g)),)), None
        if pc == 10:  # release the global lock
            return L(pc=11), put(G + 1, (inc(gturn),)), None
        if pc == 11:  # free the cluster: push a record that is not owned, or free the tail
            nxt = succ if succ is not None else linked()
            if nxt is not None:
                sp, sseq = nxt
                word = ("own", cp + 1, g) if self.broken == "owned_after_release" else None
                return finish(), put(2 * sp + 1, ((sseq & self.M16, word),)), None
            return L(pc=13), sh, None
        if pc == 13:
            if self.broken == "no_cas":
                return finish(), sh, None
            if tail == (p, seq):
                return finish(), put(T0 + c, (None,)), None
            return L(pc=14), sh, None
        if pc == 14:
            nxt = linked()
            if nxt is None:
                return loc, sh, None
            sp, sseq = nxt
            return finish(), put(2 * sp + 1, ((sseq & self.M16, None),)), None
        raise AssertionError(pc)


class SpinSem:
    """Spin-lock semaphore (Section 5 and the Appendix's spin-lock semaphore).

    S starts at X + 1; 0 means another block holds the internal lock.  wait: V <- exch(S, 0);
    V > 1: exch(S, V - 1) and enter; V = 1 (at capacity): exch(S, 1) and retry; V = 0: retry.
    post: repeat V <- exch(S, 0) until V > 0, then exch(S, V + 1).  Backoff() after a failed
    wait attempt when UseBackoff (never in post).

    Planted mistakes: broken="keep_v" makes a successful wait write back V instead of V - 1
    (the permit is never taken); broken="post_no_inc" makes post write back V instead of
    V + 1 (the permit is never returned); broken="full_zero" makes a wait that finds the
    semaphore at capacity (V = 1) write back 0 instead of 1, which leaves the internal lock
    held.
    """
    kind, fifo = "sem", False

    def __init__(self, n=1, backoff=False, broken=None):
        self.capacity, self.backoff, self.broken = n, backoff, broken

    def init(self, nproc, ops):
        return (self.capacity + 1,), tuple((0, 0, 0, 0) for _ in range(nproc))

    def step(self, p, loc, sh, nproc, ops):
        pc, k, v, r = loc
        S = sh[0]
        retry = 7 if self.backoff else 0
        if pc == 0:
            if S > 1:
                return (1, k, S, r), (0,), None
            if S == 1:
                return (2, k, S, r), (0,), None
            return (retry, k, S, r), (0,), None
        if pc == 1:
            return (PC_ENTER, k, v, r), ((v if self.broken == "keep_v" else v - 1),), None
        if pc == 2:
            return (retry, k, v, r), ((0 if self.broken == "full_zero" else 1),), None
        if pc == 7:  # Backoff()
            return (0, k, v, r), sh, None
        if pc == PC_ENTER:
            return (PC_EXIT, k, v, r), sh, ("enter", None)
        if pc == PC_EXIT:
            return (3, k, v, r), sh, ("exit",)
        if pc == 3:
            if S > 0:
                return (4, k, S, r), (0,), None
            return (3, k, S, r), (0,), None
        if pc == 4:
            k += 1
            return ((0 if k < ops else DONE), k, v, r), ((v if self.broken == "post_no_inc" else v + 1),), None
        raise AssertionError(pc)


class SleepSem:
    """Sleeping (FA) semaphore (Section 5 and the Appendix's sleeping semaphore).

    wait: OldCount <- fetch-and-add(count, 1); if OldCount < maxCount enter; otherwise
    WaitIndex <- fetch-and-add(ticket, 1) and wait until turn > WaitIndex.
    post: OldCount <- fetch-and-add(count, -1); if OldCount > maxCount, fetch-and-add(turn, 1).
    The count is a signed 32-bit value; turn and WaitIndex compare by signed difference.
    broken="turn_ge" waits for turn >= WaitIndex instead (one grant too many).
    """
    kind, fifo = "sem", False

    def __init__(self, n=1, base=0, broken=None):
        self.capacity, self.base, self.broken = n, base & M32, broken

    def init(self, nproc, ops):
        return (0, self.base, self.base), tuple((0, 0, 0, 0) for _ in range(nproc))

    def step(self, p, loc, sh, nproc, ops):
        pc, k, w, r = loc
        count, ticket, turn = sh
        N = self.capacity
        if pc == 0:
            if count < N:
                return (PC_ENTER, k, w, r), (count + 1, ticket, turn), None
            return (1, k, w, r), (count + 1, ticket, turn), None
        if pc == 1:
            return (2, k, ticket, r), (count, inc(ticket), turn), None
        if pc == 2:
            ok = s_ge(turn, w) if self.broken == "turn_ge" else s_gt(turn, w)
            return ((PC_ENTER if ok else 2), k, w, r), sh, None
        if pc == PC_ENTER:
            return (PC_EXIT, k, w, r), sh, ("enter", None)
        if pc == PC_EXIT:
            return (3, k, w, r), sh, ("exit",)
        if pc == 3:
            k += 1
            nxt = 0 if k < ops else DONE
            if count > N:
                return (4, k, w, r), (count - 1, ticket, turn), None
            return (nxt, k, w, r), (count - 1, ticket, turn), None
        if pc == 4:
            return ((0 if k < ops else DONE), k, w, r), (count, ticket, inc(turn)), None
        raise AssertionError(pc)


class WindowSem:
    """Ticket-window semaphore (the library's GB300 alternative to the FA semaphore of Section 5):
    wait takes t <- fetch-and-add(ticket, 1) and enters once turn + N > t (signed difference),
    polling turn; post adds 1 to turn and nothing else.  Holders are tickets in
    [turn, turn + N), so at most N are inside, in ticket order of admission windows.  A stale
    read of turn is smaller, so it only delays an entry: the model reads turn after taking
    the ticket, the latest value it could see.
    broken="window_ge" enters once turn + N >= t (one holder too many)."""
    kind, fifo = "sem", False

    def __init__(self, n=1, base=0, broken=None):
        self.capacity, self.base, self.broken = n, base & M32, broken

    def init(self, nproc, ops):
        return (self.base, self.base), tuple((0, 0, 0) for _ in range(nproc))

    def step(self, p, loc, sh, nproc, ops):
        pc, k, t = loc
        ticket, turn = sh
        N = self.capacity
        if pc == 0:
            return (1, k, ticket), (inc(ticket), turn), None
        if pc == 1:
            edge = (turn + N) & M32
            ok = s_ge(edge, t) if self.broken == "window_ge" else s_gt(edge, t)
            return ((PC_ENTER if ok else 1), k, t), sh, None
        if pc == PC_ENTER:
            return (PC_EXIT, k, t), sh, ("enter", None)
        if pc == PC_EXIT:
            return (3, k, t), sh, ("exit",)
        if pc == 3:
            k += 1
            return ((0 if k < ops else DONE), k, t), (ticket, inc(turn)), None
        raise AssertionError(pc)


# --------------------------------------------------------------------------------------------
# Barriers.  Events: ("arrive",) when a block arrives, ("pass",) when it leaves the barrier.
# --------------------------------------------------------------------------------------------


class AtomicBarrier:
    """Two-stage atomic barrier: stage 1 counts arrivals with fetch-and-add; the last arriver
    resets the counter and advances the release epoch; stage 2 polls the epoch.  Each block
    keeps its expected epoch locally.  broken="no_wait": non-last arrivers leave at once.

    parity=True (the library's form): crossing e counts on counter e mod 2, and the last
    arriver advances the epoch first and resets that counter after, off the release path; the
    counter is next used two crossings later, which cannot start before the last arriver has
    arrived at the crossing in between.  broken="reset_one_counter": parity counting with the
    reset after the release but a single counter (a fast block can count into the next
    crossing before the reset)."""
    kind = "barrier"

    def __init__(self, base=0, broken=None, parity=False):
        self.base, self.broken = base & M32, broken
        self.parity = parity or broken == "reset_one_counter"

    def init(self, nproc, ops):
        return (0, 0, self.base), tuple((0, 0, self.base, 0) for _ in range(nproc))

    def step(self, p, loc, sh, nproc, ops):
        pc, k, e, r = loc
        counts, release = sh[:2], sh[2]
        c = (inc(e) & 1) if self.parity and self.broken != "reset_one_counter" else 0
        if pc == 0:
            last = counts[c] + 1 == nproc
            return ((1 if last else 3), k, e, r), _set(counts, c, counts[c] + 1) + (release,), ("arrive",)
        if not self.parity:
            if pc == 1:
                return (2, k, e, r), _set(counts, c, 0) + (release,), None
            if pc == 2:
                k += 1
                return ((0 if k < ops else DONE), k, inc(e), r), counts + (inc(e),), ("pass",)
        else:
            if pc == 1:  # release first ...
                return (2, k, e, r), counts + (inc(e),), ("pass",)
            if pc == 2:  # ... then reset the counter this crossing used
                k += 1
                return ((0 if k < ops else DONE), k, inc(e), r), _set(counts, c, 0) + (release,), None
        if pc == 3:
            if release == inc(e) or self.broken == "no_wait":
                k += 1
                return ((0 if k < ops else DONE), k, inc(e), r), sh, ("pass",)
            return loc, sh, None
        raise AssertionError(pc)


class CountBarrier:
    """Counting barrier: one arrival counter that only grows (64-bit on the device, so it never
    wraps in practice).  Every block adds 1 per crossing and then polls the counter until it
    reaches base + e x B for its e-th crossing: the last arrival's increment is itself the
    release, with no epoch word.  It cannot reach e x B before every block has made its e-th
    arrival, because no block arrives at crossing e + 1 before passing crossing e.
    broken="off_by_one": a block waits only for base + e x B - 1.

    S > 1 (two levels): block p counts in on sub-counter p mod S; the arrival that completes
    its sub-counter's e-th crossing (known from the value its fetch-and-add returns) adds 1 to
    the top counter without waiting for a return, and every block polls the top counter until
    it reaches base + e x G (G = min(S, B) sub-counters in use).  broken="top_early": the top
    counter gets its increment from the first arrival of a sub-counter, not the last."""
    kind = "barrier"

    def __init__(self, base=0, S=1, broken=None):
        self.base, self.S, self.broken = base, S, broken

    def init(self, nproc, ops):
        if self.S == 1:
            return (self.base * nproc,), tuple((0, 0, 0, 0) for _ in range(nproc))
        G = min(self.S, nproc)
        subs = tuple(self.base * len(range(c, nproc, self.S)) for c in range(self.S))
        return (self.base * G,) + subs, tuple((0, 0, 0, 0) for _ in range(nproc))

    def step(self, p, loc, sh, nproc, ops):
        pc, k, e, r = loc
        if self.S == 1:
            (count,) = sh
            if pc == 0:
                return (1, k, e + 1, r), (count + 1,), ("arrive",)
            if pc == 1:
                target = (self.base + e) * nproc - (1 if self.broken == "off_by_one" else 0)
                if count < target:
                    return loc, sh, None
                k += 1
                return ((0 if k < ops else DONE), k, e, r), sh, ("pass",)
            raise AssertionError(pc)
        G = min(self.S, nproc)
        c = p % self.S
        members = len(range(c, nproc, self.S))
        top = sh[0]
        if pc == 0:      # sub-counter fetch-and-add
            old = sh[1 + c]
            e1 = e + 1
            last = old + 1 == (self.base + e1) * members
            first = old == (self.base + e1 - 1) * members
            bump = first if self.broken == "top_early" else last
            return ((2 if bump else 1), k, e1, r), _set(sh, 1 + c, old + 1), ("arrive",)
        if pc == 2:      # completes the sub-counter: count in at the top (no return awaited)
            return (1, k, e, r), _set(sh, 0, top + 1), None
        if pc == 1:
            if top < (self.base + e) * G:
                return loc, sh, None
            k += 1
            return ((0 if k < ops else DONE), k, e, r), sh, ("pass",)
        raise AssertionError(pc)


class ExchangeBarrier:
    """Exchange barrier: the counting barrier whose arrival carries one value per block (a
    barrier and an all-gather in one; GSYNC_BAR_EXCHANGE, a GB300 design, not in the paper).

    For its e-th crossing block p writes a record (epoch, value) into slot (epoch mod 2, p) and
    adds 1 to the counter; there is no fence, so the device may make the two visible in either
    order: `late[p]` makes block p count in before its record is written.  The block polls the
    counter until it reaches (base + e) x B, then reads its partner's record of the same parity,
    polling until the record shows the crossing's epoch, and must find the value its partner
    published for it (value(q, epoch) = 16 q + epoch).  Records alternate by epoch parity: a
    block rewrites slot (e mod 2, p) for crossing e + 2 only after passing crossing e + 1, which
    needs every reader of crossing e to have arrived at e + 1.
    broken="single_buffer": one record per block (a fast block overwrites the record a slow one
    still has to read); broken="no_epoch_check": a reader takes the record without checking its
    epoch; broken="off_by_one": a block waits for one arrival less.
    """
    kind = "barrier"

    def __init__(self, base=0, late=(), broken=None):
        self.base, self.late, self.broken = base, tuple(late), broken

    def init(self, nproc, ops):
        recs = ((self.base, 0),) * (2 * nproc)  # (epoch, value) per (parity, block)
        return (self.base * nproc,) + recs, tuple((0, 0, 0, 0) for _ in range(nproc))

    def slot(self, epoch, q, nproc):
        return 1 + (0 if self.broken == "single_buffer" else (epoch & 1) * nproc) + q

    def step(self, p, loc, sh, nproc, ops):
        pc, k, e, r = loc
        count = sh[0]
        late = p < len(self.late) and self.late[p]
        ge = self.base + e + 1  # the epoch of the crossing this block is making (pc 0..2)
        if pc == 0:
            if late:
                return (1, k, e, r), _set(sh, 0, count + 1), ("arrive",)
            return (1, k, e, r), _set(sh, self.slot(ge, p, nproc), (ge, 16 * p + ge)), None
        if pc == 1:
            if late:
                return (2, k, e + 1, r), _set(sh, self.slot(ge, p, nproc), (ge, 16 * p + ge)), None
            return (2, k, e + 1, r), _set(sh, 0, count + 1), ("arrive",)
        if pc == 2:
            target = (self.base + e) * nproc - (1 if self.broken == "off_by_one" else 0)
            if count < target:
                return loc, sh, None
            return (3, k, e, r), sh, ("pass",)
        if pc == 3:  # the partner's record of this crossing
            ep = self.base + e
            q = (p + k + 1) % nproc
            rep, val = sh[self.slot(ep, q, nproc)]
            if rep != ep and self.broken != "no_epoch_check":
                return loc, sh, None
            if val != 16 * q + ep:
                return loc, sh, ("violation", f"block {p} read {val} from block {q} at epoch {ep}")
            k += 1
            return ((0 if k < ops else DONE), k, e, r), sh, None
        raise AssertionError(pc)


class SplitBarrier:
    """Split barrier: block p counts in on counter p mod S; the last arriver at a counter
    counts in on a top counter (skipped when S = 1), and the last arriver there writes the
    new epoch to R release copies; block p polls copy p mod R.  Counters alternate by epoch
    parity and the block that used one resets it (after the release when it released, before
    waiting otherwise).  broken="one_copy_early": the releaser passes after writing only the
    first copy and the rest never get written.  broken="no_top": the last arriver at any
    counter releases."""
    kind = "barrier"

    def __init__(self, S=2, R=2, base=0, broken=None):
        self.S, self.R, self.base, self.broken = S, R, base & M32, broken

    def init(self, nproc, ops):
        e = self.base
        # (counters[par][S] flattened: 2S, top[2], release[R])
        return (0,) * (2 * self.S + 2) + (e,) * self.R, tuple((0, 0, e, 0) for _ in range(nproc))

    def step(self, p, loc, sh, nproc, ops):
        pc, k, e, j = loc  # j: copy index being written by the releaser
        S, R = self.S, self.R
        e1 = inc(e)
        par = e1 & 1
        c = p % S
        ci, ti, rel0 = par * S + c, 2 * S + par, 2 * S + 2
        members = len(range(c, nproc, S))
        groups = min(S, nproc)

        def passed():
            k2 = k + 1
            return ((0 if k2 < ops else DONE), k2, e1, 0)

        if pc == 0:
            last = sh[ci] + 1 == members
            nxt = (1 if groups > 1 and self.broken != "no_top" else 3) if last else 6
            return (nxt, k, e, 0), _set(sh, ci, sh[ci] + 1), ("arrive",)
        if pc == 1:  # last at its counter: count in at the top
            last = sh[ti] + 1 == groups
            return ((3 if last else 2), k, e, 0), _set(sh, ti, sh[ti] + 1), None
        if pc == 2:  # not the releaser: reset the counter, then wait
            return (6, k, e, 0), _set(sh, ci, 0), None
        if pc == 3:  # releaser: write the copies one by one
            sh2 = _set(sh, rel0 + j, e1)
            if j + 1 < R and self.broken != "one_copy_early":
                return (3, k, e, j + 1), sh2, None
            return (4, k, e, 0), sh2, ("pass",)
        if pc == 4:
            sh2 = _set(sh, ci, 0)
            if groups > 1:
                sh2 = _set(sh2, ti, 0)
            return passed(), sh2, None
        if pc == 6:
            if sh[rel0 + p % R] != e1:
                return loc, sh, None
            return passed(), sh, ("pass",)
        raise AssertionError(pc)


class DieBarrier:
    """Two-die barrier: blocks count in on their own die's counter and poll their own die's
    release word (both homed on that die); the last arriver of each die counts in on a top
    counter, and the second die to finish releases both dies.

    The blocks per die are not known in advance: a block's first crossing of a launch is a
    registration crossing that counts all blocks on one flat counter while each block also
    counts itself into its die's membership word; the last arriver turns the membership into
    the dies' block counts and the number of dies with blocks, resets it, and releases both
    dies.  Later crossings use the per-die counters, two of each (and two top counters) by
    epoch parity: the releasing block resets the counters it used after the release, and a
    die leader that does not release resets its die counter before it waits.
    layout[p] is block p's die.
    broken="no_top": a die's last arriver releases without waiting for the other die.
    broken="no_reset": a die's last arriver does not reset its die's counter.
    """
    kind = "barrier"

    def __init__(self, layout=None, base=0, broken=None):
        self.layout, self.base, self.broken = layout, base & M32, broken

    def die(self, p):
        return self.layout[p] if self.layout is not None else p % 2

    def init(self, nproc, ops):
        if self.layout is not None:
            assert len(self.layout) == nproc
        e = self.base
        # (cnt_all, mem0, mem1, n0, n1, active, cnt[d=0,par=0], cnt[0,1], cnt[1,0], cnt[1,1],
        #  top[0], top[1], rel0, rel1)
        sh = (0,) * 12 + (e, e)
        return sh, tuple((0, 0, e, 0, 0) for _ in range(nproc))  # (pc, k, epoch, n_mine, active)

    def step(self, p, loc, sh, nproc, ops):
        pc, k, e, nm, act = loc
        d = self.die(p)
        e1 = inc(e)
        par = e1 & 1
        CNT_ALL, MEM, N, ACT, CNT, TOP, REL = 0, 1, 3, 5, 6, 10, 12
        ci, ti = CNT + 2 * d + par, TOP + par

        def passed(n_mine=nm, active=act):
            k2 = k + 1
            return ((0 if k2 < ops else DONE), k2, e1, n_mine, active)

        if pc == 0:
            return ((10 if nm == 0 else 20), k, e, nm, act), sh, None
        # registration crossing
        if pc == 10:
            return (11, k, e, nm, act), _set(sh, MEM + d, sh[MEM + d] + 1), None
        if pc == 11:
            last = sh[CNT_ALL] + 1 == nproc
            return ((12 if last else 16), k, e, nm, act), _set(sh, CNT_ALL, sh[CNT_ALL] + 1), ("arrive",)
        if pc == 12:
            return (13, k, e, nm, act), _set(sh, CNT_ALL, 0), None
        if pc == 13:
            m0, m1 = sh[MEM], sh[MEM + 1]
            sh2 = sh[:MEM] + (0, 0, m0, m1, int(m0 > 0) + int(m1 > 0)) + sh[ACT + 1:]
            return (14, k, e, nm, act), sh2, None
        if pc == 14:
            return (15, k, e, nm, act), _set(sh, REL, e1), None
        if pc == 15:
            return passed(sh[N + d], sh[ACT]), _set(sh, REL + 1, e1), ("pass",)
        if pc == 16:
            if sh[REL + d] != e1:
                return loc, sh, None
            return passed(sh[N + d], sh[ACT]), sh, ("pass",)
        # per-die crossing
        if pc == 20:
            last = sh[ci] + 1 == nm
            return ((21 if last else 26), k, e, nm, act), _set(sh, ci, sh[ci] + 1), ("arrive",)
        if pc == 21:
            return ((24 if act == 1 or self.broken == "no_top" else 22), k, e, nm, act), sh, None
        if pc == 22:
            last = sh[ti] == 1
            return ((24 if last else 27), k, e, nm, act), _set(sh, ti, sh[ti] + 1), None
        if pc == 27:  # leader of the first die to finish: reset, then wait
            sh2 = sh if self.broken == "no_reset" else _set(sh, ci, 0)
            return (26, k, e, nm, act), sh2, None
        if pc == 24:
            return (25, k, e, nm, act), _set(sh, REL, e1), None
        if pc == 25:
            return (28, k, e, nm, act), _set(sh, REL + 1, e1), ("pass",)
        if pc == 28:  # after the release: reset the counters this crossing used
            sh2 = sh if self.broken == "no_reset" else _set(sh, ci, 0)
            return ((29 if act == 2 and self.broken != "no_top" else 30), k, e, nm, act), sh2, None
        if pc == 29:
            return (30, k, e, nm, act), _set(sh, ti, 0), None
        if pc == 30:
            return passed(), sh, None
        if pc == 26:
            if sh[REL + d] != e1:
                return loc, sh, None
            return passed(), sh, ("pass",)
        raise AssertionError(pc)


class FlagBarrier:
    """Decentralized flag barrier of Xiao and Feng (Section 5, "Barrier").

    Each block writes its arrival flag; the master block (block 0) checks every flag, then
    writes the release flags, one per block (broadcast=True: one shared release word).
    Flags hold increasing epoch values, so no reset phase is needed.
    broken="skip_last": the master never checks the last block's flag.
    """
    kind = "barrier"

    def __init__(self, broadcast=False, base=0, broken=None):
        self.broadcast, self.base, self.broken = broadcast, base & M32, broken

    def init(self, nproc, ops):
        nrel = 1 if self.broadcast else nproc
        sh = tuple([self.base] * nproc) + tuple([self.base] * nrel)
        return sh, tuple((0, 0, self.base, 0) for _ in range(nproc))

    def _rel(self, p, nproc):
        return nproc + (0 if self.broadcast else p)

    def step(self, p, loc, sh, nproc, ops):
        pc, k, e, j = loc
        ne = inc(e)
        if p != 0:
            if pc == 0:
                return (1, k, e, j), _set(sh, p, ne), ("arrive",)
            if pc == 1:
                if sh[self._rel(p, nproc)] == ne:
                    k += 1
                    return ((0 if k < ops else DONE), k, ne, j), sh, ("pass",)
                return loc, sh, None
            raise AssertionError(pc)
        last = nproc - 1 if self.broken == "skip_last" else nproc
        if pc == 0:
            return (1, k, e, 1), _set(sh, 0, ne), ("arrive",)
        if pc == 1:  # check arrival flags 1..n-1, one load per step
            if j >= last:
                return (2, k, e, 1), sh, None
            if sh[j] == ne:
                return (1, k, e, j + 1), sh, None
            return loc, sh, None
        if pc == 2:  # write release flags, one store per step
            if self.broadcast:
                k += 1
                return ((0 if k < ops else DONE), k, ne, 0), _set(sh, nproc, ne), ("pass",)
            if j >= nproc:
                k += 1
                return ((0 if k < ops else DONE), k, ne, 0), sh, ("pass",)
            return (2, k, e, j + 1), _set(sh, nproc + j, ne), None
        raise AssertionError(pc)


class TreeBarrier:
    """Combining-tree barrier with fan-in `fan`: a block counts itself in at its leaf; the
    last arriver at a node resets that node and counts itself in at the parent; the last
    arriver at the root advances the release epoch, which every block polls.

    Planted mistakes: broken="no_reset": the last arriver at a node never resets it, so the
    next crossing's count overshoots the node's size; broken="release_at_leaf": the last
    arriver at a leaf releases at once instead of climbing to the root."""
    kind = "barrier"

    def __init__(self, fan=2, base=0, broken=None):
        self.fan, self.base, self.broken = fan, base & M32, broken

    def _tree(self, nproc):
        # nodes listed level by level: (size, parent index)
        nodes, level, width = [], [], nproc
        first = 0
        sizes = [min(self.fan, width - i) for i in range(0, width, self.fan)]
        levels = [sizes]
        while len(levels[-1]) > 1:
            w = len(levels[-1])
            levels.append([min(self.fan, w - i) for i in range(0, w, self.fan)])
        offs, off = [], 0
        for lv in levels:
            offs.append(off)
            off += len(lv)
        size, parent = [], []
        for li, lv in enumerate(levels):
            for i, s in enumerate(lv):
                size.append(s)
                parent.append(offs[li + 1] + i // self.fan if li + 1 < len(levels) else -1)
        return size, parent

    def init(self, nproc, ops):
        size, _ = self._tree(nproc)
        return tuple([0] * len(size)) + (self.base,), tuple((0, 0, self.base, p // self.fan) for p in range(nproc))

    def step(self, p, loc, sh, nproc, ops):
        size, parent = self._tree(nproc)
        pc, k, e, nd = loc
        rel = len(size)
        if pc in (0, 4):  # arrive at node nd (pc 0: the leaf, a block's own arrival)
            c = sh[nd] + 1
            ev = ("arrive",) if pc == 0 else None
            return ((1 if c == size[nd] else 3), k, e, nd), _set(sh, nd, c), ev
        if pc == 1:  # last arriver at nd: reset it, go up or release
            if self.broken != "no_reset":
                sh = _set(sh, nd, 0)
            if parent[nd] < 0 or self.broken == "release_at_leaf":
                return (2, k, e, nd), sh, None
            return (4, k, e, parent[nd]), sh, None
        if pc == 2:
            k += 1
            return ((0 if k < ops else DONE), k, inc(e), p // self.fan), _set(sh, rel, inc(e)), ("pass",)
        if pc == 3:
            if sh[rel] == inc(e):
                k += 1
                return ((0 if k < ops else DONE), k, inc(e), p // self.fan), sh, ("pass",)
            return loc, sh, None
        raise AssertionError(pc)


class TreeCountBarrier:
    """Combining tree of fan-in `fan` whose node counters only grow.  A block counts itself in
    at its leaf; the arrival whose fetch-and-add brings a node's counter to a multiple of the
    node's size is that node's last one for this crossing and counts in at the parent (counters
    start at multiples of their sizes, so no reset is needed); the root's last arrival is the
    release.  Every other arrival polls the root until it reaches base + e x (root's size).

    Planted mistakes: broken="first_climbs": the arrival whose add leaves a node at one past a
    multiple of its size climbs, instead of the one that completes it; broken="target_short":
    the root target is one short."""
    kind = "barrier"

    def __init__(self, fan=2, base=0, broken=None):
        self.fan, self.base, self.broken = fan, base, broken

    def init(self, nproc, ops):
        size, _ = TreeBarrier(self.fan)._tree(nproc)
        return tuple(self.base * z for z in size), tuple((0, 0, 0, p // self.fan) for p in range(nproc))

    def step(self, p, loc, sh, nproc, ops):
        size, parent = TreeBarrier(self.fan)._tree(nproc)
        root = len(size) - 1
        pc, k, e, nd = loc
        leaf = p // self.fan
        if pc in (0, 4):  # count in at node nd (pc 0: the leaf, the block's own arrival)
            c = sh[nd] + 1
            ev = ("arrive",) if pc == 0 else None
            if self.broken == "first_climbs":
                climbs = c % size[nd] == 1 % size[nd]
            else:
                climbs = c % size[nd] == 0
            if not climbs:
                return (3, k, e, leaf), _set(sh, nd, c), ev
            if nd == root:
                return (5, k, e, leaf), _set(sh, nd, c), ev  # the release itself
            return (4, k, e, parent[nd]), _set(sh, nd, c), ev
        if pc == 3:  # poll the root
            target = (self.base + e + 1) * size[root] - (1 if self.broken == "target_short" else 0)
            if sh[root] < target:
                return loc, sh, None
        if pc in (3, 5):
            k2 = k + 1
            return ((0 if k2 < ops else DONE), k2, e + 1, leaf), sh, ("pass",)
        raise AssertionError(pc)


class ShardedBarrier:
    """Sharded-counter barrier: block p counts itself into counter p mod S (fetch-and-add,
    counters never reset); the master block 0 checks that counter s holds
    (epoch + 1) x (blocks of shard s, master excluded), one counter per step, then writes
    each block's release flag.  broken="early": the master waits for one arrival fewer on
    shard 0; broken="counts_master": it also expects its own (never made) arrival."""
    kind = "barrier"

    def __init__(self, shards=2, base=0, broken=None):
        self.S, self.base, self.broken = shards, base & M32, broken

    def init(self, nproc, ops):
        # Consistent start at epoch `base`: counter s holds base x members (mod 2^32).
        assert self.S <= nproc
        true_members = [(nproc - s + self.S - 1) // self.S - (1 if s == 0 else 0) for s in range(self.S)]
        counters = tuple((self.base * m) & M32 for m in true_members)
        return counters + tuple([self.base] * nproc), tuple((0, 0, self.base, 0) for _ in range(nproc))

    def members(self, s, nproc):
        m = (nproc - s + self.S - 1) // self.S - (1 if s == 0 else 0)
        if s == 0 and self.broken == "early":
            m -= 1
        if s == 0 and self.broken == "counts_master":
            m += 1
        return m

    def step(self, p, loc, sh, nproc, ops):
        pc, k, e, j = loc
        ne = inc(e)
        S = self.S
        if p != 0:
            if pc == 0:
                return (1, k, e, j), _set(sh, p % S, inc(sh[p % S])), ("arrive",)
            if pc == 1:
                if sh[S + p] == ne:
                    k += 1
                    return ((0 if k < ops else DONE), k, ne, j), sh, ("pass",)
                return loc, sh, None
            raise AssertionError(pc)
        if pc == 0:
            return (1, k, e, 0), sh, ("arrive",)
        if pc == 1:  # check counter j
            if j >= S:
                return (2, k, e, 0), sh, None
            if sh[j] == (ne * self.members(j, nproc)) & M32:
                return (1, k, e, j + 1), sh, None
            return loc, sh, None
        if pc == 2:  # write release flags
            if j >= nproc:
                k += 1
                return ((0 if k < ops else DONE), k, ne, 0), sh, ("pass",)
            return (2, k, e, j + 1), _set(sh, S + j, ne), None
        raise AssertionError(pc)


class ClusterBarrier:
    """Hierarchical barrier over groups ("clusters") of c consecutive blocks.

    Phase 1 is a barrier inside the cluster (the hardware cluster barrier; modelled as a
    counter with a cluster epoch).  Phase 2: the cluster's leader (rank 0) arrives at a
    global two-stage atomic barrier of nproc / c leaders; every block polls the global release
    epoch.

    Planted mistakes: broken="leader_early": the leader counts in at the global counter as
    soon as it arrives itself, without waiting for its cluster; broken="all_count": every
    block of a cluster counts in at the global counter, not only the leader.
    """
    kind = "barrier"

    def __init__(self, c=2, base=0, broken=None):
        self.c, self.base, self.broken = c, base & M32, broken

    def init(self, nproc, ops):
        assert nproc % self.c == 0
        ncl = nproc // self.c
        sh = tuple([0] * ncl) + tuple([0] * ncl) + (0, self.base)
        return sh, tuple((0, 0, self.base, 0) for _ in range(nproc))

    def step(self, p, loc, sh, nproc, ops):
        c = self.c
        ncl = nproc // c
        cl, rank = p // c, p % c
        pc, k, e, ce = loc
        CC, CE, GC, REL = cl, ncl + cl, 2 * ncl, 2 * ncl + 1
        if pc == 0:
            n = sh[CC] + 1
            if self.broken == "leader_early" and rank == 0:
                # counts in globally now; the cluster barrier is crossed after the release
                return (3, k, e, ce), _set(sh, CC, n), ("arrive",)
            return ((1 if n == c else 2), k, e, ce), _set(sh, CC, n), ("arrive",)
        if pc == 1:
            sh = _set(sh, CC, 0)
            return (2, k, e, ce), _set(sh, CE, inc(sh[CE])), None
        if pc == 2:
            if sh[CE] == inc(ce):
                return ((3 if rank == 0 or self.broken == "all_count" else 6), k, e, inc(ce)), sh, None
            return loc, sh, None
        if pc == 3:
            n = sh[GC] + 1
            return ((4 if n == ncl else 6), k, e, ce), _set(sh, GC, n), None
        if pc == 4:
            return (5, k, e, ce), _set(sh, GC, 0), None
        if pc == 5:
            k += 1
            return ((0 if k < ops else DONE), k, inc(e), ce), _set(sh, REL, inc(e)), ("pass",)
        if pc == 6:
            if sh[REL] == inc(e):
                k += 1
                return ((0 if k < ops else DONE), k, inc(e), ce), sh, ("pass",)
            return loc, sh, None
        raise AssertionError(pc)


class ClusterCountBarrier:
    """Cluster barrier whose global stage is a counting barrier over the cluster leaders.

    A block first crosses the barrier of its cluster of c consecutive blocks (the hardware
    cluster barrier; modelled as a counter with a cluster epoch).  The cluster's leader (rank
    0) then adds 1 to a global counter that only grows and polls it until it reaches
    base + e x (nproc / c) for its e-th crossing: the last leader's increment is the release.
    release="poll": the other blocks of the cluster poll the global counter too.
    release="cluster": they wait at a second cluster barrier, which the leader reaches only
    after it has seen the counter reach its target.

    Planted mistakes: broken="off_by_one": the target is one short; broken="no_second": with
    release="cluster", the other blocks leave without the second cluster barrier.
    """
    kind = "barrier"

    def __init__(self, c=2, base=0, release="poll", broken=None):
        self.c, self.base, self.release, self.broken = c, base, release, broken

    def init(self, nproc, ops):
        assert nproc % self.c == 0
        ncl = nproc // self.c
        # per cluster: first barrier's counter and epoch, second barrier's counter and epoch
        sh = tuple([0] * (4 * ncl)) + (self.base * ncl,)
        return sh, tuple((0, 0, 0, 0, 0) for _ in range(nproc))

    def step(self, p, loc, sh, nproc, ops):
        c = self.c
        ncl = nproc // c
        cl, rank = p // c, p % c
        pc, k, e, ce, ce2 = loc
        CC, CE, CC2, CE2, GC = cl, ncl + cl, 2 * ncl + cl, 3 * ncl + cl, 4 * ncl
        second = self.release == "cluster"

        def passed(sh2, e2=e + 1, ce_=ce, ce2_=ce2):
            k2 = k + 1
            return ((0 if k2 < ops else DONE), k2, e2, ce_, ce2_), sh2, ("pass",)

        if pc == 0:  # arrive at the cluster barrier
            n = sh[CC] + 1
            return ((1 if n == c else 2), k, e, ce, ce2), _set(sh, CC, n), ("arrive",)
        if pc == 1:  # last of the cluster: reset and open the cluster barrier
            sh = _set(sh, CC, 0)
            return (2, k, e, ce, ce2), _set(sh, CE, sh[CE] + 1), None
        if pc == 2:
            if sh[CE] != ce + 1:
                return loc, sh, None
            if rank == 0:
                nxt = 3
            elif second:
                nxt = 5 if self.broken != "no_second" else 8
            else:
                nxt = 4
            return (nxt, k, e, ce + 1, ce2), sh, None
        if pc == 3:  # leader: count in on the global counter
            return (4, k, e, ce, ce2), _set(sh, GC, sh[GC] + 1), None
        if pc == 4:  # poll the global counter
            target = (self.base + e + 1) * ncl - (1 if self.broken == "off_by_one" else 0)
            if sh[GC] < target:
                return loc, sh, None
            if second:
                return (5, k, e, ce, ce2), sh, None
            return passed(sh)
        if pc == 5:  # second cluster barrier
            n = sh[CC2] + 1
            return ((6 if n == c else 7), k, e, ce, ce2), _set(sh, CC2, n), None
        if pc == 6:
            sh = _set(sh, CC2, 0)
            return (7, k, e, ce, ce2), _set(sh, CE2, sh[CE2] + 1), None
        if pc == 7:
            if sh[CE2] != ce2 + 1:
                return loc, sh, None
            return passed(sh, ce2_=ce2 + 1)
        if pc == 8:  # broken: leaves without the second cluster barrier
            return passed(sh)
        raise AssertionError(pc)


# --------------------------------------------------------------------------------------------
# Explorer
# --------------------------------------------------------------------------------------------


class RingPublish:
    """The serving ring's entry publication (the persistent serving loop; not in the paper).

    Block 0 is the host's producer, block 1 an admitter, over one ring slot that every request
    reuses.  The producer writes request i as two halves, lo = (seq, len) and hi = (off,
    seq_check), each one atomic store, in either order (`hi_first`) and with no fence, and
    reuses the slot only after the admitter has taken request i - 1.  The admitter reads the two
    halves with two separate reads (`read_hi_first` picks the order) and takes the entry when
    both sequence numbers equal i + 1; it must then hold request i's len (10 + i) and off
    (20 + i).
    broken="one_check": the admitter checks seq alone (a half of the previous lap slips in);
    broken="no_reuse_wait": the producer overwrites the slot before the admitter took the
    previous request (that request is lost and the admitter waits forever).
    """
    kind = "mutex"
    capacity = 1
    fifo = False

    def __init__(self, hi_first=False, read_hi_first=False, broken=None):
        self.hi_first, self.read_hi_first, self.broken = hi_first, read_hi_first, broken

    def init(self, nproc, ops):
        # shared: (lo, hi, requests taken); the slot starts empty (sequence numbers 0)
        locs = tuple((0, 0, None) if p < 2 else (DONE, 0, None) for p in range(nproc))
        return ((0, -1), (-1, 0), 0), locs

    def step(self, p, loc, sh, nproc, ops):
        pc, i, seen = loc
        lo, hi, taken = sh
        if p == 0:  # producer
            new_lo, new_hi = (i + 1, 10 + i), (20 + i, i + 1)
            if pc == 0:
                if taken < i and self.broken != "no_reuse_wait":
                    return loc, sh, None
                first = (lo, new_hi, taken) if self.hi_first else (new_lo, hi, taken)
                return (1, i, None), first, None
            second = (new_lo, hi, taken) if self.hi_first else (lo, new_hi, taken)
            i += 1
            return ((0 if i < ops else DONE), i, None), second, None
        # admitter
        if pc == 0:
            return (1, i, hi if self.read_hi_first else lo), sh, None
        got_lo, got_hi = (lo, seen) if self.read_hi_first else (seen, hi)
        (seq, ln), (off, chk) = got_lo, got_hi
        if seq != i + 1 or (chk != i + 1 and self.broken != "one_check"):
            return (0, i, None), sh, None  # not published yet: poll again
        if ln != 10 + i or off != 20 + i:
            return loc, sh, ("violation", f"request {i} taken with len {ln}, off {off}")
        i += 1
        return ((0 if i < ops else DONE), i, None), (lo, hi, i), None


class ServeSlot:
    """One slot of the persistent serving loop (not in the paper): an admitter publishes
    requests into the slot one after another, and workers claim the requests' chunks.

    Block 0 is the admitter.  For request r it takes the free slot (compare-and-swap of the
    state 0 -> 1), reads the generation and writes generation + 1, the chunk count NCH[r], the
    done count 0 and the accumulator 0, resets the claim counter to (generation, chunk 0),
    publishes the slot (state 2) and sets its bit in the active mask.  Blocks 1.. are workers.
    A worker that finds the bit set claims with one fetch-and-add on the (generation, chunk)
    counter, then reads (state, generation, chunk count) in one access: the claim is taken when
    the slot is active in the claim's generation and the chunk exists, dropped when the slot
    has moved on or the chunk is past the last, and waits while the slot is being set up.  The
    worker that takes the last chunk clears the bit.  A taken chunk adds its value (1 << chunk)
    to the accumulator and counts itself done; the block whose count completes the request
    reads the accumulator, which must hold every chunk, frees the slot (state 0) and counts
    the request completed.  Workers stop once every request is completed.  Each shared access
    is one step (sequential consistency).  The counter's chunk field stops growing one past the
    largest chunk count (a 16-bit field on the device, which the few claims made between a
    last chunk's hand-out and the clearing of the bit cannot carry into the generation).
    broken="no_gen_check": a worker takes any claim whose chunk exists in the active request,
    whatever the claim's generation (a chunk is then processed twice);
    broken="no_done_reset": the admitter leaves the done count of the previous request (the
    next request never completes).
    """
    kind = "mutex"
    capacity = 1 << 30
    fifo = False

    def __init__(self, nch=(1, 2), broken=None):
        self.nch, self.broken = tuple(nch), broken

    def init(self, nproc, ops):
        # shared: state, gen, nchunks, claim counter (gen, chunk), done, acc, completed, active
        # bit, and a ghost: the (generation, chunk) pairs processed so far
        sh = (0, 0, 0, (0, 0), 0, 0, 0, 0, frozenset())
        return sh, tuple((0, 0, 0, 0) for _ in range(nproc))

    @staticmethod
    def _put(sh, i, v):
        return sh[:i] + (v,) + sh[i + 1:]

    def step(self, p, loc, sh, nproc, ops):
        state, gen, nch, ctr, done, acc, completed, active, seen = sh
        pc, a, b, c = loc
        put = self._put
        R = len(self.nch)
        if p == 0:  # admitter; a = request, b = its generation
            if pc == 0:
                if state != 0:
                    return loc, sh, None
                return (1, a, b, c), put(sh, 0, 1), None
            if pc == 1:
                return (2, a, gen + 1, c), sh, None
            if pc == 2:
                return (3, a, b, c), put(sh, 1, b), None
            if pc == 3:
                return (4, a, b, c), put(sh, 2, self.nch[a]), None
            if pc == 4:
                return (5, a, b, c), put(sh, 4, done if self.broken == "no_done_reset" else 0), None
            if pc == 5:
                return (6, a, b, c), put(sh, 5, 0), None
            if pc == 6:
                return (7, a, b, c), put(sh, 3, (b, 0)), None
            if pc == 7:
                return (8, a, b, c), put(sh, 0, 2), None
            a += 1
            return ((0 if a < R else DONE), a, 0, 0), put(sh, 7, 1), None
        # worker; a, b = the claim's (generation, chunk), c = the request's chunk count
        if pc == 0:
            if completed == R:
                return (DONE, 0, 0, 0), sh, None
            return (10, 0, 0, 0), sh, None
        if pc == 10:
            return ((1 if active else 0), 0, 0, 0), sh, None
        if pc == 1:
            g, k = ctr
            # the chunk field stops at max(NCH) + 1: every claim past a request's last chunk is
            # dropped alike, and the bound keeps the state space finite
            return (2, g, k, 0), put(sh, 3, (g, min(k + 1, max(self.nch) + 1))), None
        if pc == 2:
            g, k = a, b
            if state == 2 and (gen == g or self.broken == "no_gen_check"):
                if k >= nch:
                    return (0, 0, 0, 0), sh, None  # past the last chunk: dropped
                return (3, gen, k, nch), sh, None
            if gen > g or (gen == g and state == 0):
                return (0, 0, 0, 0), sh, None  # the slot has moved on: dropped
            return loc, sh, None  # generation g is being set up: wait
        if pc == 3:  # the last chunk handed out: the slot leaves the active mask
            if b + 1 == c:
                return (4, a, b, c), put(sh, 7, 0), None
            return (4, a, b, c), sh, None
        if pc == 4:
            if (a, b) in seen:
                return loc, sh, ("violation", f"chunk {b} of generation {a} processed twice")
            return (5, a, b, c), put(put(sh, 5, acc | (1 << b)), 8, seen | {(a, b)}), None
        if pc == 5:
            return ((6 if done + 1 == c else 0), a, b, c), put(sh, 4, done + 1), None
        if pc == 6:
            if acc != (1 << c) - 1:
                return loc, sh, ("violation", f"generation {a} completed with chunks {acc:#b} of {c}")
            return (7, a, b, c), sh, None
        if pc == 7:
            return (8, a, b, c), put(sh, 0, 0), None
        return (0, 0, 0, 0), put(sh, 6, completed + 1), None


def _ghost0(model, nproc):
    if model.kind == "barrier":
        return (tuple([0] * nproc), tuple([0] * nproc))
    if getattr(model, "dies", 0):
        return (0, 0, (0,) * model.dies)  # (blocks inside, grants, grants per die)
    return (0, 0)  # (blocks inside, grants so far)


def _apply(model, ghost, p, ev, nproc):
    """Updates the ghost bookkeeping for an event; returns (ghost, violation or None)."""
    if ev is None:
        return ghost, None
    if ev[0] == "violation":
        return ghost, ev[1]
    if model.kind == "barrier":
        arrived, passed = ghost
        if ev[0] == "arrive":
            return (_set(arrived, p, arrived[p] + 1), passed), None
        r = passed[p]  # the round p is leaving
        if min(arrived) < r + 1:
            return ghost, f"block {p} passed round {r} before every block arrived"
        return (arrived, _set(passed, p, r + 1)), None
    inside, grants = ghost[0], ghost[1]
    rest = ghost[2:]
    if ev[0] == "enter":
        inside += 1
        if inside > model.capacity:
            return ghost, f"{inside} blocks inside a critical section of capacity {model.capacity}"
        if model.fifo and ev[1] is not None:
            want = (getattr(model, "base", 0) + grants) & M32
            if ev[1] != want:
                return ghost, f"grant {grants} went to ticket {ev[1]:#x}, expected {want:#x}"
        if rest:  # FIFO within each die: the die's grants follow its local tickets
            d, t = ev[1]
            per = rest[0]
            want = (model.base + per[d]) & M32
            if t != want:
                return ghost, f"die {d} grant {per[d]} went to local ticket {t:#x}, expected {want:#x}"
            rest = (_set(per, d, per[d] + 1),)
        return (inside, grants + 1) + rest, None
    return (inside - 1, grants) + rest, None


def check(model, nproc: int, ops: int, max_states: int = 2_000_000) -> Result:
    """Explores every interleaving of `nproc` blocks doing `ops` operations each."""
    sh0, loc0 = model.init(nproc, ops)
    s0 = (sh0, loc0, _ghost0(model, nproc))
    index = {s0: 0}
    states = [s0]
    parent = [-1]
    succ: list[list[int]] = [[]]
    stack = [0]
    res = Result()
    while stack:
        i = stack.pop()
        sh, locs, g = states[i]
        for p in range(nproc):
            if locs[p][0] == DONE:
                continue
            loc2, sh2, ev = model.step(p, locs[p], sh, nproc, ops)
            g2, bad = _apply(model, g, p, ev, nproc)
            s2 = (sh2, _set(locs, p, loc2), g2)
            if bad:
                res.violation = bad
                res.states = len(states)
                tr, j = [s2], i
                while j >= 0:
                    tr.append(states[j])
                    j = parent[j]
                res.trace = tr[::-1]
                return res
            j = index.get(s2)
            if j is None:
                j = len(states)
                index[s2] = j
                states.append(s2)
                parent.append(i)
                succ.append([])
                stack.append(j)
                if len(states) > max_states:
                    raise RuntimeError("state space larger than max_states")
            succ[i].append(j)
    res.states = len(states)
    # progress: every state must reach a final state (all blocks done)
    pred: list[list[int]] = [[] for _ in states]
    for i, ss in enumerate(succ):
        for j in ss:
            pred[j].append(i)
    final = [i for i, (_, locs, _) in enumerate(states) if all(l[0] == DONE for l in locs)]
    if not final:
        res.violation = "no final state is reachable"
        return res
    reach = set(final)
    work = list(final)
    while work:
        j = work.pop()
        for i in pred[j]:
            if i not in reach:
                reach.add(i)
                work.append(i)
    if len(reach) != len(states):
        stuck = next(i for i in range(len(states)) if i not in reach)
        res.violation = "a reachable state cannot reach completion (deadlock or livelock)"
        res.stuck_state = states[stuck]
    return res
