"""Pins the machine-abstraction arithmetic to the numbers the paper prints (Tables 1-3 and
the best-implementation table of Section 6)."""
import pytest

from golden_io import read_table
from oracle import classify

COLS = [("tesla", "read"), ("tesla", "write"), ("fermi", "read"), ("fermi", "write")]


def times(gpu):
    t1 = read_table("table1_times_ms.txt")
    out = {}
    for row, vals in t1.items():
        for (g, d), v in zip(COLS, vals):
            if g == gpu:
                out[(row, d)] = float(v)
    return out


def interval(t, num, den, d):
    """Range of num/den when every Table 1 entry is known only to +-0.0005 ms."""
    n, m = t[(num, d)], t[(den, d)]
    return (n - 5e-4) / (m + 5e-4), (n + 5e-4) / (m - 5e-4)


T2_PAIRS = {"volatile": ("cont_volatile", "noncont_volatile"),
            "atomic": ("cont_atomic", "noncont_atomic"),
            "vol_after_atomic": ("cont_vol_after_atomic", "noncont_vol_after_atomic")}
T3_PAIRS = {"cont_atomic": "cont_volatile", "noncont_atomic": "noncont_volatile",
            "cont_vol_after_atomic": "cont_volatile",
            "noncont_vol_after_atomic": "noncont_volatile"}


@pytest.mark.parametrize("gpu", ["tesla", "fermi"])
def test_table2_reproduces_printed_ratios(gpu):
    t = times(gpu)
    r = classify.table2(t)
    printed = read_table("table2_cont_noncont_ratios.txt")
    for row, vals in printed.items():
        for (g, d), v in zip(COLS, vals):
            if g != gpu:
                continue
            lo, hi = interval(t, *T2_PAIRS[row], d)
            assert lo - 0.01 <= float(v) <= hi + 0.01, (row, d, v, lo, hi)
            assert lo <= r[(row, d)] <= hi


@pytest.mark.parametrize("gpu", ["tesla", "fermi"])
def test_table3_reproduces_printed_ratios(gpu):
    t = times(gpu)
    r = classify.table3(t)
    printed = read_table("table3_vs_volatile_ratios.txt")
    for row, vals in printed.items():
        for (g, d), v in zip(COLS, vals):
            if g != gpu:
                continue
            lo, hi = interval(t, row, T3_PAIRS[row], d)
            assert lo - 0.01 <= float(v) <= hi + 0.01, (row, d, v, lo, hi)
            assert abs(r[(row, d)] - float(v)) <= 0.011  # printed to 2 decimals
            assert lo <= r[(row, d)] <= hi


def test_swapped_denominator_is_caught():
    # A plausible slip (dividing the contentious atomic time by the noncontentious volatile
    # time) lands far outside the printed Table 3 value.
    t = times("tesla")
    wrong = t[("cont_atomic", "read")] / t[("noncont_volatile", "read")]
    assert abs(wrong - 92.46) > 1.0


def test_abstraction_parameters_match_section4():
    tesla = classify.abstraction(times("tesla"))
    fermi = classify.abstraction(times("fermi"))
    # Tesla: contentious atomics ~90x volatile, no line hostage; Fermi: ~3-8x, hostage.
    assert tesla["atomic_volatile"] > 90 and not tesla["line_hostage"]
    assert 2 < fermi["atomic_volatile"] < 10 and fermi["line_hostage"]
    # Fermi's contentious:noncontentious volatile ratio is worse than Tesla's.
    assert fermi["cont_noncont_volatile"] > tesla["cont_noncont_volatile"]


@pytest.mark.parametrize("gpu", ["tesla", "fermi"])
def test_design_choice_matches_best_per_gpu_table(gpu):
    best = read_table("best_per_gpu.txt")
    col = 0 if gpu == "tesla" else 1
    choice = classify.design_choice(classify.abstraction(times(gpu)))
    for prim, vals in best.items():
        assert choice[prim] == vals[col], (gpu, prim)
