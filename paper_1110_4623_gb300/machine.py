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
        "line_hostage": bool(max(t3[("cont_vol_after_atomic", "read")], t3[("cont_vol_after_atomic", "write")])
                             > HOSTAGE_THRESHOLD),
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
    # the atomic round trip to a line homed on the probe's own die (fastest of eight pages)
    pages = runner._state(8 * 4096)
    rtt = min(runner.probe_latency("atomic_read", 1000, scratch=pages.data_ptr() + i * 4096)["ns_per_op"]
              for i in range(8))
    return {"dies": nd, "handoff_near_ns": near, "handoff_far_ns": far, "handoff_dsmem_ns": dsmem,
            "fence_ns": fence, "atomic_same_ns": 1e9 / r_same, "atomic_rtt_ns": rtt}


# An atomic round trip this large a part of a hand-off makes the ticket-window semaphore pay:
# its post advances the turn without the FA semaphore's round trip to the count.
WINDOW_RTT_FRACTION = 0.25


def design_extended(params: dict, ext: dict, nblocks: int = 1184) -> dict:
    """The Section 4 choice, then the GB300 extensions: a cohort lock on a two-die part whose
    cross-die hand-off is DIE_GAP_NS slower (mutex_without_clusters), and over thread-block
    clusters when a hand-off through distributed shared memory (a flag pushed into the peer's
    shared memory) beats the on-die L2 one and the kernel can launch in clusters (mutex: the
    cluster cohort lock whose MCS queue pushes each grant that way); the counting barrier
    when `nblocks` serialized
    same-word atomics cost less than the two hand-offs of the flag barrier's extra stage; the
    ticket-window semaphore when an atomic round trip exceeds WINDOW_RTT_FRACTION of the
    on-die hand-off."""
    choice = dict(design(params))
    if ext["dies"] == 2 and ext["handoff_far_ns"] - ext["handoff_near_ns"] > DIE_GAP_NS:
        choice["mutex"] = "cohort"
    choice["mutex_without_clusters"] = choice["mutex"]
    if ext.get("handoff_dsmem_ns", float("inf")) < ext["handoff_near_ns"]:
        choice["mutex"] = "cluster_mcs"
    if nblocks * ext["atomic_same_ns"] < 2.0 * ext["handoff_near_ns"]:
        choice["barrier"] = "count"
    if ext.get("atomic_rtt_ns", 0.0) > WINDOW_RTT_FRACTION * ext["handoff_near_ns"]:
        choice["sem_low"] = choice["sem_high"] = "window"
    return choice


# ---- the whole description -----------------------------------------------------------------

LATENCY_OPS = ("volatile_load", "load_relaxed", "load_acquire", "atomic_read", "atomic_add64", "atomic_acqrel")
SWEEP_BLOCKS = (1, 8, 38, 76, 152, 304, 608, 1184)
SLEEP_NS = (0, 20, 40, 100, 200, 500, 1000, 2000, 4000, 8000)
CLUSTER_SIZES = (2, 4, 8)
FENCE_OPS = {"alone": 0, "after_relaxed_store": 1, "after_four_stores": 2, "cluster_scope": 3}


def measure_all(nblocks: int = 1184, quick: bool = False) -> dict:
    """Everything the probes measure, as one JSON-ready description of this GPU:
    - the paper's probe matrix (Table 1 shape), its two ratio tables, the three Section 4
      parameters and the primitives they favour;
    - dependent-chain latency of one thread per access kind (32- and 64-bit atomics, relaxed
      and acquire loads);
    - same-word and distinct-word throughput of `red` and `atom` against the number of blocks;
    - the two dies: SMs per die and the atomic round trip to a line homed on the SM's own die
      and on the other;
    - SM-to-SM hand-offs (near, far, inside a cluster through distributed shared memory or an
      mbarrier), the hardware cluster barrier, release fences, __nanosleep accuracy and the
      host-to-GPU hand-off through pinned memory;
    - the GB300 extension of the design rule.
    quick: fewer accesses per probe (a check that everything runs, not a measurement)."""
    import numpy as np
    iters = 100 if quick else 1000
    reps = 1 if quick else 3
    table = measure_table(nblocks, 128, iters, reps)
    t2, t3 = ratios(table)
    params = abstraction(table)
    out = {
        "sm_count": runner.sm_count(),
        "table1_ms": {row: {d: table[(row, d)] for d in ("read", "write")} for row in ROWS},
        "table2": {f"{a}_{d}": v for (a, d), v in t2.items()},
        "table3": {f"{a}_{d}": v for (a, d), v in t3.items()},
        "parameters": params,
        "design_section4": design(params),
    }
    # The chained word at eight successive 4 KB pages: line homes alternate between the dies by
    # page, so the fastest is the round trip to the probe SM's own die and the slowest to the
    # other die (equal on a one-die part).
    n_lat = 256 if quick else 4096
    pages = runner._state(8 * 4096)
    out["latency_ns"] = {}
    for op in LATENCY_OPS:
        t = [runner.probe_latency(op, n_lat, scratch=pages.data_ptr() + i * 4096)["ns_per_op"] for i in range(8)]
        out["latency_ns"][op] = {"near": min(t), "far": max(t)}
    sweep = {}
    for op in ("red_add", "atomic_read"):
        for cont in (True, False):
            key = f"{op}_{'same' if cont else 'distinct'}_word_ops_per_s"
            sweep[key] = {str(b): runner.probe_throughput(op, cont, False, b, 128, iters)["ops_per_s"]
                          for b in SWEEP_BLOCKS if b <= nblocks}
    out["throughput_vs_blocks"] = sweep
    die, nd = runner.device_topology()
    sms = out["sm_count"]
    line = runner._state(128)
    rtt = runner.probe_rtt_by_sm(line, 16 if quick else 64)["rtt_ns"]
    by_die = [rtt[:sms][die[:sms] == d] for d in range(nd)]
    # one line, homed on one of the dies: the SMs of that die see the near round trip
    out["dies"] = {"count": nd, "sms_per_die": [int(len(x)) for x in by_die],
                   "atomic_rtt_ns_to_one_line_by_die_of_sm": [float(np.median(x)) for x in by_die]}
    ext = measure_extended(nblocks)
    n_hand = 500 if quick else 2000
    out["handoff_ns"] = {
        "near": ext["handoff_near_ns"], "far": ext["handoff_far_ns"],
        "dsmem": {str(c): runner.probe_cluster(1, c, n_hand)["ns"] for c in CLUSTER_SIZES},
        "mbarrier": {str(c): runner.probe_cluster(2, c, n_hand)["ns"] for c in CLUSTER_SIZES},
        # a relaxed 16-byte record with no fence, pushed into the peer's shared memory or
        # pulled from one's own (the hand-offs of the carrying locks over clusters)
        "dsmem_relaxed_push": {str(c): runner.probe_cluster(3, c, n_hand)["ns"] for c in CLUSTER_SIZES},
        "dsmem_relaxed_pull": {str(c): runner.probe_cluster(4, c, n_hand)["ns"] for c in CLUSTER_SIZES},
        "relaxed_near": runner.near_handoff_relaxed(n_hand)["handoff_ns"],
        "host": runner.probe_host_pingpong(200 if quick else 2000)["handoff_ns"],
    }
    out["cluster_barrier_ns"] = {str(c): runner.probe_cluster(0, c, n_hand)["ns"] for c in (1,) + CLUSTER_SIZES}
    out["fence_ns"] = {k: runner.probe_fence(op, n_hand)["ns_per_fence"] for k, op in FENCE_OPS.items()}
    slept = runner.probe_nanosleep(list(SLEEP_NS), 8 if quick else 64)
    out["nanosleep_ns"] = {str(r): float(s) for r, s in zip(SLEEP_NS, slept)}
    out["extended"] = ext
    out["design_extended"] = design_extended(params, ext, nblocks)
    return out


def main(argv=None) -> int:
    import argparse
    import json
    p = argparse.ArgumentParser(description="Measure this GPU's machine description (Sections 3-4, extended).")
    p.add_argument("--out", default="machine.json", help="where to write the JSON description")
    p.add_argument("--blocks", type=int, default=1184, help="grid of the saturated probes")
    p.add_argument("--quick", action="store_true", help="short probes: checks that everything runs")
    a = p.parse_args(argv)
    desc = measure_all(a.blocks, a.quick)
    with open(a.out, "w") as f:
        json.dump(desc, f, indent=1, default=float)
    print(json.dumps({"design_section4": desc["design_section4"], "design_extended": desc["design_extended"]}))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
