"""Machine-abstraction arithmetic (oracle; test infrastructure only).

Section 3 ("Benchmarks") times, per GPU, 1000 accesses per master thread on a saturated
GPU for: {volatile, atomic} x {contentious, noncontentious} x {read, write} plus the four
volatile tests preceded by one atomic (Table 1).  Table 2 divides every contentious time by
the matching noncontentious time; Table 3 divides every atomic and volatile-after-atomic
time by the volatile time of the same contention and direction.  Section 4 ("Machine
Abstraction") reduces them to three parameters:
  1. the Atomic:Volatile ratio (contentious atomic / contentious volatile),
  2. the Contentious:Noncontentious volatile ratio,
  3. whether an atomic unit with a non-empty queue holds the line hostage, visible as
     contentious volatile accesses slowed down by one preceding atomic.
Section 6 (Table "best implementation for each primitive") reports the resulting choices.
"""
from __future__ import annotations

ROWS = ("cont_volatile", "noncont_volatile", "cont_atomic", "noncont_atomic",
        "cont_vol_after_atomic", "noncont_vol_after_atomic")
DIRS = ("read", "write")


def table2(t: dict) -> dict:
    """Contentious : noncontentious time ratios (Table 2), per access direction."""
    out = {}
    for d in DIRS:
        out[("volatile", d)] = t[("cont_volatile", d)] / t[("noncont_volatile", d)]
        out[("atomic", d)] = t[("cont_atomic", d)] / t[("noncont_atomic", d)]
        out[("vol_after_atomic", d)] = t[("cont_vol_after_atomic", d)] / t[("noncont_vol_after_atomic", d)]
    return out


def table3(t: dict) -> dict:
    """Time ratios against volatile accesses of the same contention (Table 3)."""
    out = {}
    for d in DIRS:
        out[("cont_atomic", d)] = t[("cont_atomic", d)] / t[("cont_volatile", d)]
        out[("noncont_atomic", d)] = t[("noncont_atomic", d)] / t[("noncont_volatile", d)]
        out[("cont_vol_after_atomic", d)] = t[("cont_vol_after_atomic", d)] / t[("cont_volatile", d)]
        out[("noncont_vol_after_atomic", d)] = t[("noncont_vol_after_atomic", d)] / t[("noncont_volatile", d)]
    return out


# A preceding atomic that slows contentious volatile accesses by more than this factor is
# read as "the atomic unit holds the line hostage" (Tesla: 1.08/1.10, read as no; Fermi:
# 2.98/4.71, read as yes; Section 3 "Benchmark Results").
HOSTAGE_THRESHOLD = 1.5
# Atomic:Volatile above this is read as "contentious atomics are prohibitive" (Tesla ~92x,
# Fermi ~3-8x; Section 4).
PROHIBITIVE_ATOMIC_RATIO = 20.0


def abstraction(t: dict) -> dict:
    """The three parameters of Section 4, from a Table-1-shaped dict of times."""
    r3 = table3(t)
    r2 = table2(t)
    atomic_volatile = max(r3[("cont_atomic", "read")], r3[("cont_atomic", "write")])
    cont_noncont_vol = max(r2[("volatile", "read")], r2[("volatile", "write")])
    hostage = max(r3[("cont_vol_after_atomic", "read")], r3[("cont_vol_after_atomic", "write")]) > HOSTAGE_THRESHOLD
    return {"atomic_volatile": atomic_volatile, "cont_noncont_volatile": cont_noncont_vol,
            "line_hostage": bool(hostage)}


def design_choice(params: dict) -> dict:
    """Design per primitive from the abstraction (Section 4 strategies; Section 6 table).

    Prohibitive contentious atomics: move every atomic up front and sleep on volatile polls
    (FA mutex, sleeping semaphore).  Cheap atomics with a line-hostage atomic unit: spin with
    backoff for the mutex and for low-count semaphores, sleeping semaphore for high counts.
    The barrier is the decentralized flag (XF) barrier in both cases.
    """
    if params["atomic_volatile"] > PROHIBITIVE_ATOMIC_RATIO:
        return {"barrier": "flag", "mutex": "ticket", "sem_low": "ticket", "sem_high": "ticket"}
    if params["line_hostage"]:
        return {"barrier": "flag", "mutex": "cas_backoff", "sem_low": "spin_backoff", "sem_high": "ticket"}
    return {"barrier": "flag", "mutex": "cas_backoff", "sem_low": "ticket", "sem_high": "ticket"}
