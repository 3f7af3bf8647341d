"""The bench line's results log (--jsonl): one row per measured configuration, with the
rate or time, its roofline and fraction (host logic on a synthetic line, no GPU)."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def test_rows_cover_every_measured_configuration():
    import bench
    out = {
        "config": {"nblocks": 1184}, "n_gpus": 1, "clocks": {"sm_mhz": 2070.0},
        "mutex": {"ticket": {"0": {"acq_per_s": 8e5, "roof_acq_per_s": 1e6, "frac": 0.8},
                             "64": {"acq_per_s": 7e5, "roof_acq_per_s": 1e6, "frac": 0.7}}},
        "barrier": {"kinds": {"count8": {"ns_per_crossing": 2200.0, "roof_ns": 1200.0, "frac": 0.545}}},
        "semaphore": {"kinds": {"window": {"1": {"ops_per_s": 3e5, "roof_ops_per_s": 4e5, "frac": 0.75}}}},
        "condvar": {"mutex": {"cohort": {"items_per_s": 3e5, "frac": 0.48}}},
        "batched": {"default": {"acq_per_s": 4.8e6, "cluster": 1}, "tuned": {"acq_per_s": 5.2e6, "cluster": 4}},
        "serving": {"rates": {"1000": {"persistent": {"achieved_req_s": 1000.0, "p50_us": 8.0, "p99_us": 11.0},
                                       "per_request_launch": {"achieved_req_s": 1000.0, "p50_us": 12.0,
                                                              "p99_us": 18.0}}}},
    }
    rows = bench.result_rows(out)
    sections = [r["section"] for r in rows]
    assert sections.count("mutex") == 2 and sections.count("barrier") == 1 and sections.count("semaphore") == 1
    assert sections.count("condvar") == 1 and sections.count("batched") == 2 and sections.count("serving") == 2
    m = [r for r in rows if r["section"] == "mutex" and r["cs_words"] == 64][0]
    assert m["kind"] == "ticket" and m["frac"] == 0.7 and m["nblocks"] == 1184
    s = [r for r in rows if r["section"] == "serving" and r["kind"] == "persistent"][0]
    assert s["offered_req_s"] == 1000.0 and s["p99_us"] == 11.0
    assert all(r["clocks_sm_mhz"] == 2070.0 and r["n_gpus"] == 1 for r in rows)


def test_rows_of_a_line_without_optional_sections():
    import bench
    assert bench.result_rows({"config": {}, "n_gpus": 1}) == []


def test_sweep_rows():
    import bench
    out = {"config": {"nblocks": 1184}, "n_gpus": 1,
           "sweep": {"mutex_acq_per_s": {"cluster": {"64": {"148": 9e5, "1184": 8.9e5}}},
                     "barrier_ns_per_crossing": {"count8": {"148": 1700.0, "1184": 2100.0}, "cluster8": {"144": 2500.0}},
                     "semaphore_ops_per_s": {"window": {"4": {"296": 1.5e6}}}}}
    rows = bench.result_rows(out)
    m = [r for r in rows if r["section"] == "sweep_mutex"]
    assert len(m) == 2 and {r["nblocks"] for r in m} == {148, 1184} and all(r["cs_words"] == 64 for r in m)
    b = [r for r in rows if r["section"] == "sweep_barrier"]
    assert len(b) == 3 and {(r["kind"], r["nblocks"]) for r in b} >= {("cluster8", 144), ("count8", 148)}
    s = [r for r in rows if r["section"] == "sweep_semaphore"]
    assert s == [dict(s[0], section="sweep_semaphore", kind="window", n=4, nblocks=296, ops_per_s=1.5e6)]


def test_sweep_grids_start_at_one_block_and_round_cluster_grids_down():
    import bench
    assert bench.SWEEP_GRIDS[0] == 1 and bench.SWEEP_GRIDS[-1] == bench.NBLOCKS
    assert list(bench.SWEEP_GRIDS) == sorted(set(bench.SWEEP_GRIDS))
    assert bench.sweep_grid(148, 0) == 148 and bench.sweep_grid(148, 8) == 144 and bench.sweep_grid(148, 4) == 148
    assert bench.sweep_grid(4, 8) == 0 and bench.sweep_grid(8, 8) == 8 and bench.sweep_grid(1, 0) == 1
    # every cluster grid the sweep runs divides into whole clusters
    for c in (2, 4, 8):
        assert all(bench.sweep_grid(B, c) % c == 0 for B in bench.SWEEP_GRIDS)
