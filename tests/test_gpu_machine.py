"""Machine abstraction on the GPU: the library's ratio arithmetic over its own measured
Table-1 times agrees with the oracle's arithmetic over the same times (the measured times
themselves are hardware facts: parity unpinned, only sanity-checked)."""
import math

import pytest

from gpu_util import require_gpu
from oracle import classify

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def table():
    require_gpu()
    from paper_1110_4623_gb300 import machine
    return machine.measure_table(1184, 128, 1000, reps=1)


def test_all_sixteen_probes_measured(table):
    assert len(table) == 12
    assert all(v > 0 and math.isfinite(v) for v in table.values())


def test_ratio_arithmetic_matches_oracle(table):
    from paper_1110_4623_gb300 import machine
    t2, t3 = machine.ratios(table)
    o2, o3 = classify.table2(table), classify.table3(table)
    assert t2.keys() == o2.keys() and t3.keys() == o3.keys()
    for k in o2:
        assert math.isclose(t2[k], o2[k], rel_tol=1e-12)
    for k in o3:
        assert math.isclose(t3[k], o3[k], rel_tol=1e-12)
    assert machine.design(machine.abstraction(table)) == classify.design_choice(classify.abstraction(table))


def test_contentious_atomics_slower_than_noncontentious(table):
    assert table[("cont_atomic", "read")] > table[("noncont_atomic", "read")]


def test_extended_abstraction_measured_on_this_gpu():
    from paper_1110_4623_gb300 import machine
    ext = machine.measure_extended(1184)
    assert ext["dies"] in (1, 2)
    assert 0 < ext["atomic_same_ns"] < 100 and 50 < ext["handoff_near_ns"] < 5000 and ext["fence_ns"] > 0
    if ext["dies"] == 2:
        # the cross-die hand-off is the slower one, and the rule then keeps hand-offs on a die
        assert ext["handoff_far_ns"] > ext["handoff_near_ns"]
        params = machine.abstraction(machine.measure_table(1184, 128, 1000, reps=1))
        got = machine.design_extended(params, ext)
        assert got["mutex_without_clusters"] == "cohort"
        assert got["mutex"] == ("cluster_mcs" if ext["handoff_dsmem_ns"] < ext["handoff_near_ns"] else "cohort")
        window = ext["atomic_rtt_ns"] > machine.WINDOW_RTT_FRACTION * ext["handoff_near_ns"]
        assert got["sem_high"] == ("window" if window else machine.design(params)["sem_high"])


def test_machine_description_cli(tmp_path):
    # The whole description (python -m paper_1110_4623_gb300.machine) in its short form: every
    # section present, every time finite and positive, and its Section 4 choice the oracle's
    # choice for the Table 1 times it wrote.
    import json
    from paper_1110_4623_gb300 import machine
    out = tmp_path / "machine.json"
    assert machine.main(["--quick", "--out", str(out)]) == 0
    d = json.loads(out.read_text())
    sms = d["sm_count"]
    assert set(d["table1_ms"]) == set(machine.ROWS)
    table = {(row, k): v for row, rw in d["table1_ms"].items() for k, v in rw.items()}
    assert all(v > 0 and math.isfinite(v) for v in table.values())
    assert d["design_section4"] == classify.design_choice(classify.abstraction(table))
    assert set(d["latency_ns"]) == set(machine.LATENCY_OPS)
    assert all(0 < v["near"] <= v["far"] for v in d["latency_ns"].values())
    for key, per_blocks in d["throughput_vs_blocks"].items():
        assert list(per_blocks) == [str(b) for b in machine.SWEEP_BLOCKS], key
        assert all(v > 0 for v in per_blocks.values()), key
    assert sum(d["dies"]["sms_per_die"]) == sms and d["dies"]["count"] in (1, 2)
    if d["dies"]["count"] == 2:
        near, far = sorted(d["dies"]["atomic_rtt_ns_to_one_line_by_die_of_sm"])
        assert far > near
    hand = d["handoff_ns"]
    assert hand["near"] > 0 and hand["far"] > 0 and hand["host"] > 0
    assert all(v > 0 for v in list(hand["dsmem"].values()) + list(hand["mbarrier"].values()))
    assert all(v > 0 for v in list(hand["dsmem_relaxed_push"].values()) + list(hand["dsmem_relaxed_pull"].values()))
    assert hand["relaxed_near"] > 0
    assert all(v > 0 for v in d["cluster_barrier_ns"].values()) and all(v > 0 for v in d["fence_ns"].values())
    assert list(d["nanosleep_ns"]) == [str(n) for n in machine.SLEEP_NS]
    assert d["nanosleep_ns"]["8000"] > d["nanosleep_ns"]["100"]
    assert d["design_extended"]["mutex"] in ("cluster_mcs", "cohort", "ticket", "cas_backoff")
