"""Topology probes and the SM-to-die map (the two-die extension of Section 4's machine
abstraction): round trips to a line split the SMs into the dies, the split is the same for
every line up to which die is near, and line homes alternate between the dies."""
import numpy as np
import pytest

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def test_device_topology_partitions_the_sms():
    from paper_1110_4623_gb300 import runner
    die, nd = runner.device_topology()
    assert nd in (1, 2)
    assert len(die) == runner.sm_count() and set(np.unique(die)) <= {0, 1}
    if nd == 2:
        assert 0 < int((die == 1).sum()) < len(die)
    die2, nd2 = runner.device_topology()  # cached: the same answer
    assert nd2 == nd and np.array_equal(die, die2)


def test_rtt_by_sm_matches_the_die_map_for_any_line():
    import torch
    from paper_1110_4623_gb300 import runner
    die, nd = runner.device_topology()
    if nd < 2:
        pytest.skip("one-die GPU")
    buf = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    for off in (0, 4096, 8192, 12288, 40960):
        r = runner.probe_rtt_by_sm(buf[off:], 32)
        assert r["status"] == 0
        rtt = r["rtt_ns"]
        near = rtt < (rtt.min() + rtt.max()) / 2
        assert np.array_equal(near, die == 0) or np.array_equal(near, die == 1), off
        assert rtt[~near].mean() > rtt[near].mean() + 60


def test_line_homes_alternate_in_pages():
    import torch
    from paper_1110_4623_gb300 import runner
    die, nd = runner.device_topology()
    if nd < 2:
        pytest.skip("one-die GPU")
    buf = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    sm0, sm1 = int(np.flatnonzero(die == 0)[0]), int(np.flatnonzero(die == 1)[0])
    a = runner.probe_rtt_by_line(sm0, buf, 256, 4096, 8)
    b = runner.probe_rtt_by_line(sm1, buf, 256, 4096, 8)
    home0 = a < b  # nearer to die 0's SM than to die 1's
    assert 0.25 < home0.mean() < 0.75  # both dies home a share of the pages
    # lines inside one 4 KB page share its home
    inner = runner.probe_rtt_by_line(sm0, buf, 32, 128, 8) < (a.min() + a.max()) / 2
    assert inner.all() or not inner.any()


def test_probe_argument_checks():
    import torch
    from paper_1110_4623_gb300 import gsync as G
    from paper_1110_4623_gb300 import runner
    buf = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    out = torch.zeros(256, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert G.gsync_probe_rtt_by_sm(buf, 0, buf, out, st) == G.GSYNC_EINVAL
    assert G.gsync_probe_rtt_by_sm(buf, 4, buf[4:], out, st) == G.GSYNC_EINVAL  # scratch misaligned
    assert G.gsync_probe_rtt_by_line(runner.sm_count(), buf, 1, 128, 4, out) == G.GSYNC_EINVAL
    assert G.gsync_probe_rtt_by_line(0, buf, 1, 2, 4, out) == G.GSYNC_EINVAL
    assert G.gsync_probe_rtt_by_line(0, buf, 0, 128, 4, out) == G.GSYNC_EINVAL
