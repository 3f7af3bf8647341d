"""Host-side planning of the batched workload (no GPU): group sizes, layout, key classes."""
import numpy as np
import pytest

from paper_1110_4623_gb300 import inputs


@pytest.mark.parametrize("multiple", [1, 2, 4, 8])
def test_group_sizes_fit_and_align(multiple):
    drawn, used = inputs.barrier_group_sizes(64, 2, 256, 1184, multiple=multiple)
    assert used.sum() <= 1184
    assert (used % multiple == 0).all() and used.min() >= max(2, multiple)
    start, gob = inputs.group_layout(used, 1184)
    assert (start % multiple == 0).all()
    for g, (st, sz) in enumerate(zip(start, used)):
        assert (gob[st:st + sz] == g).all()
    assert (gob[used.sum():] == -1).all()


def test_key_classes():
    torch = pytest.importorskip("torch")  # autotune imports the runner (torch)
    from paper_1110_4623_gb300 import autotune
    keys, _, _ = inputs.batched_inputs(1_000_000, 4096, 1.1)
    cls = autotune.classify_keys(keys, 4096, 1184)
    counts = np.bincount(keys, minlength=4096)
    assert cls[0] == autotune.HOT and cls[4095] == autotune.COLD
    assert (counts[cls == autotune.HOT] >= 1_000_000 / 1184).all()
    # every hot key is drawn more often than every cold key
    assert counts[cls == autotune.HOT].min() > counts[cls == autotune.COLD].max()


def test_tuner_tries_the_cluster_kinds_at_every_cluster_size(monkeypatch):
    # The tuner's search, run against a cost table instead of the GPU: the cluster-only kinds
    # must be tried at every cluster size, and the fastest (cluster, policy) must win even when
    # the cluster size that was best before them is a different one.
    pytest.importorskip("torch")
    from paper_1110_4623_gb300 import autotune

    class FakeRun:
        def __init__(self, c):
            self.c, self.policy = c, None

        def set_policy(self, table):
            self.policy = [tuple(p) for p in table]

    def cost(run, reps=2):
        hot, warm, cold = run.policy
        ms = 100.0 - (3.0 if hot[0] == "cohort_carry" else 0.0)
        ms -= {1: 0.0, 2: 1.0, 4: 2.0, 8: 1.5}[run.c]  # clusters of 4 win with the plain policies
        if hot[0] == "cluster_die_carry":
            ms -= {2: 2.0, 4: 5.0, 8: 12.0}[run.c]  # ... but clusters of 8 win with this kind
        return ms

    monkeypatch.setattr(autotune, "make_run", lambda *a, **k: FakeRun(a[6]))
    monkeypatch.setattr(autotune, "_time", cost)
    keys, adds, _ = inputs.batched_inputs(20_000, 4096, 1.1)
    got = autotune.tune(keys, adds, 4096, 1184, 64, 10)
    assert got["cluster"] == 8 and got["policy"][0][0] == "cluster_die_carry"
    assert got["best_ms"] == pytest.approx(100.0 - 1.5 - 12.0)
    tried = {(t["cluster"], t["policy"][0]) for t in got["trials"] if t["policy"] and t["class"] == autotune.HOT}
    assert {(c, "cluster_die_carry") for c in (2, 4, 8)} <= tried
