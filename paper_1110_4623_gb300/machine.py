"""Machine abstraction of the GPU this runs on (Section 3 "Benchmarks", Section 4 "Machine
Abstraction"), measured with the library's probe kernels.

measure_table() times the paper's probe matrix: one master thread per block issues `iters`
accesses -- volatile or atomic, read or write, to one shared word (contentious) or to its own
word 256 bytes from the next block's (noncontentious), and the volatile ones also after one
preceding atomic -- on a saturated grid.  ratios() turns those times into the paper's two
ratio tables, abstraction() into its three parameters, and design() into the choice of
primitive each parameter set favours.
"""
from __future__ import annotations

from . import runner

ROWS = ("cont_volatile", "noncont_volatile", "cont_atomic", "noncont_atomic",
        "cont_vol_after_atomic", "noncont_vol_after_atomic")
# (probe op for reads, probe op for writes, contentious, preceded by one atomic)
_PROBES = {
    "cont_volatile": ("volatile_load", "volatile_store", True, False),
    "noncont_volatile": ("volatile_load", "volatile_store", False, False),
    "cont_atomic": ("atomic_read", "atomic_write", True, False),
    "noncont_atomic": ("atomic_read", "atomic_write", False, False),
    "cont_vol_after_atomic": ("volatile_load", "volatile_store", True, True),
    "noncont_vol_after_atomic": ("volatile_load", "volatile_store", False, True),
}


def measure_table(nblocks: int, block_threads: int = 128, iters: int = 1000, reps: int = 3) -> dict:
    """{(row, 'read'|'write'): milliseconds} for the paper's twelve + four probes."""
    out = {}
    for row, (rd, wr, cont, pre) in _PROBES.items():
        for d, op in (("read", rd), ("write", wr)):
            ns = sorted(runner.probe_throughput(op, cont, pre, nblocks, block_threads, iters)["ns"] for _ in range(reps))
            out[(row, d)] = ns[len(ns) // 2] / 1e6
    return out


def ratios(t: dict) -> tuple[dict, dict]:
    """Table 2 (contentious / noncontentious) and Table 3 (against the volatile access of the
    same contention), per access direction."""
    t2, t3 = {}, {}
    for d in ("read", "write"):
        t2[("volatile", d)] = t[("cont_volatile", d)] / t[("noncont_volatile", d)]
        t2[("atomic", d)] = t[("cont_atomic", d)] / t[("noncont_atomic", d)]
        t2[("vol_after_atomic", d)] = t[("cont_vol_after_atomic", d)] / t[("noncont_vol_after_atomic", d)]
        t3[("cont_atomic", d)] = t[("cont_atomic", d)] / t[("cont_volatile", d)]
        t3[("noncont_atomic", d)] = t[("noncont_atomic", d)] / t[("noncont_volatile", d)]
        t3[("cont_vol_after_atomic", d)] = t[("cont_vol_after_atomic", d)] / t[("cont_volatile", d)]
        t3[("noncont_vol_after_atomic", d)] = t[("noncont_vol_after_atomic", d)] / t[("noncont_volatile", d)]
    return t2, t3


# Thresholds of the reading of Section 4: a preceding atomic that slows contentious volatile
# accesses by more than 1.5x holds the line hostage; contentious atomics more than 20x slower
# than volatile accesses make every spinning design prohibitive.
HOSTAGE_THRESHOLD = 1.5
PROHIBITIVE_ATOMIC_RATIO = 20.0


def abstraction(t: dict) -> dict:
    t2, t3 = ratios(t)
    return {
        "atomic_volatile": max(t3[("cont_atomic", "read")], t3[("cont_atomic", "write")]),
        "atomic_volatile_read": t3[("cont_atomic", "read")],
        "cont_noncont_volatile": max(t2[("volatile", "read")], t2[("volatile", "write")]),
        "line_hostage": max(t3[("cont_vol_after_atomic", "read")], t3[("cont_vol_after_atomic", "write")])
        > HOSTAGE_THRESHOLD,
    }


def design(params: dict) -> dict:
    """The Section 4 strategy for a parameter set (Section 6's best-per-GPU table)."""
    if params["atomic_volatile"] > PROHIBITIVE_ATOMIC_RATIO:
        return {"barrier": "flag", "mutex": "ticket", "sem_low": "ticket", "sem_high": "ticket"}
    if params["line_hostage"]:
        return {"barrier": "flag", "mutex": "cas_backoff", "sem_low": "spin_backoff", "sem_high": "ticket"}
    return {"barrier": "flag", "mutex": "cas_backoff", "sem_low": "ticket", "sem_high": "ticket"}


# ---- GB300 extensions of the abstraction ------------------------------------------------
# Section 4 rates a GPU by how its atomics compare with its volatile accesses.  On GB300 two
# more things decide the design: a hand-off's cost depends on the dies of the two SMs and of
# the line (a two-die part), and a same-word atomic at the L2 slice (~0.6 ns) is cheap next to
# a release fence or an SM-to-SM hand-off (~160-480 ns), so serialized arrivals can cost less
# than an extra hand-off stage.

# A cross-die hand-off this much slower than an on-die one makes keeping hand-offs on a die pay.
DIE_GAP_NS = 100.0


def measure_extended(nblocks: int = 1184) -> dict:
    """Dies, near and far hand-off, release-fence cost and same-word atomic time, measured."""
    import numpy as np
    die, nd = runner.device_topology()
    near = runner.near_handoff(2000)["handoff_ns"]
    far = near
    if nd == 2:
        a, b = int(np.flatnonzero(die == 0)[0]), int(np.flatnonzero(die == 1)[0])
        far = runner.probe_pingpong(a, b, 2000)["handoff_ns"]
    fence = runner.probe_fence(0)["ns_per_fence"]
    r_same = runner.probe_throughput("red_add", True, False, nblocks, 128, 2000)["ops_per_s"]
    dsmem = runner.probe_cluster(1, 2, 2000)["ns"]
    return {"dies": nd, "handoff_near_ns": near, "handoff_far_ns": far, "handoff_dsmem_ns": dsmem,
            "fence_ns": fence, "atomic_same_ns": 1e9 / r_same}


def design_extended(params: dict, ext: dict, nblocks: int = 1184) -> dict:
    """The Section 4 choice, then the GB300 extensions: a cohort lock on a two-die part whose
    cross-die hand-off is DIE_GAP_NS slower (mutex_without_clusters), and over thread-block
    clusters when a hand-off through distributed shared memory beats the on-die L2 one and the
    kernel can launch in clusters (mutex); the counting barrier when `nblocks` serialized
    same-word atomics cost less than the two hand-offs of the flag barrier's extra stage."""
    choice = dict(design(params))
    if ext["dies"] == 2 and ext["handoff_far_ns"] - ext["handoff_near_ns"] > DIE_GAP_NS:
        choice["mutex"] = "cohort"
    choice["mutex_without_clusters"] = choice["mutex"]
    if ext.get("handoff_dsmem_ns", float("inf")) < ext["handoff_near_ns"]:
        choice["mutex"] = "cluster"
    if nblocks * ext["atomic_same_ns"] < 2.0 * ext["handoff_near_ns"]:
        choice["barrier"] = "count"
    return choice
