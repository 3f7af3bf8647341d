"""The GB300 extension of the Section 4 design rule (host logic, no GPU): it keeps the paper's
choices on the machines the paper measured, and picks the cohort lock and the counting
barrier from the two-die hand-off gap and the cheap same-word atomics that GB300 shows."""
from golden_io import read_table
from paper_1110_4623_gb300 import machine

COLS = [("tesla", "read"), ("tesla", "write"), ("fermi", "read"), ("fermi", "write")]


def times(gpu):
    out = {}
    for row, vals in read_table("table1_times_ms.txt").items():
        for (g, d), v in zip(COLS, vals):
            if g == gpu:
                out[(row, d)] = float(v)
    return out


# A one-die GPU whose contentious atomic costs about a microsecond (a Tesla-class DRAM atomic).
ONE_DIE_SLOW_ATOMICS = {"dies": 1, "handoff_near_ns": 1500.0, "handoff_far_ns": 1500.0, "fence_ns": 300.0,
                        "atomic_same_ns": 1000.0}
# GB300 as measured: 477 ns on-die hand-off, ~770 ns across dies, 385 ns inside a cluster
# through distributed shared memory, 0.64 ns same-word atomics.
GB300 = {"dies": 2, "handoff_near_ns": 477.0, "handoff_far_ns": 770.0, "handoff_dsmem_ns": 385.0, "fence_ns": 160.0,
         "atomic_same_ns": 0.64, "atomic_rtt_ns": 197.0}


def test_paper_machines_keep_the_paper_choice():
    for gpu in ("tesla", "fermi"):
        params = machine.abstraction(times(gpu))
        got = machine.design_extended(params, ONE_DIE_SLOW_ATOMICS)
        assert got.pop("mutex_without_clusters") == got["mutex"]
        assert got == machine.design(params)


def test_gb300_measurements_pick_cohort_and_count():
    params = machine.abstraction(times("tesla"))  # the atomic:volatile class GB300 falls in
    got = machine.design_extended(params, GB300, nblocks=1184)
    assert got["mutex"] == "cluster_mcs" and got["mutex_without_clusters"] == "cohort" and got["barrier"] == "count"
    assert got["sem_low"] == got["sem_high"] == "window"


def test_each_extension_needs_its_own_condition():
    params = machine.abstraction(times("fermi"))
    one_die_fast = dict(GB300, dies=1, handoff_far_ns=477.0, handoff_dsmem_ns=600.0)
    got = machine.design_extended(params, one_die_fast)
    assert got["mutex"] == machine.design(params)["mutex"] and got["barrier"] == "count"
    # 4096 blocks x 0.64 ns = 2.6 us > 2 x 477 ns: the flag barrier's extra stage is cheaper
    got = machine.design_extended(params, GB300, nblocks=4096)
    assert got["mutex"] == "cluster_mcs" and got["barrier"] == machine.design(params)["barrier"]
    # a cluster hand-off no faster than the on-die one: the die cohort stays the choice
    got = machine.design_extended(params, dict(GB300, handoff_dsmem_ns=500.0))
    assert got["mutex"] == "cohort"
    # an atomic round trip small next to a hand-off: the paper's semaphore stays
    got = machine.design_extended(params, dict(GB300, atomic_rtt_ns=100.0))
    assert got["sem_high"] == machine.design(params)["sem_high"] and got["sem_low"] == machine.design(params)["sem_low"]
