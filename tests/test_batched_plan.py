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
