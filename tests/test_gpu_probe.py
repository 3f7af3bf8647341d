"""Memory-system probes run, stay bounded and report sane values (Section 3, "Benchmarks")."""
import pytest

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


OPS = ["volatile_load", "volatile_store", "atomic_read", "atomic_write", "load_acquire", "load_relaxed",
       "store_release", "red_add", "atomic_add64", "atomic_acqrel"]


@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("contentious", [True, False])
def test_throughput_probe_runs(op, contentious):
    from paper_1110_4623_gb300 import runner
    r = runner.probe_throughput(op, contentious, False, 296, 128, 200)
    assert 0 < r["ns"] < 1e9


def test_contentious_atomics_are_not_faster_than_distinct_words():
    from paper_1110_4623_gb300 import runner
    same = runner.probe_throughput("atomic_read", True, False, 1184, 128, 1000)
    dist = runner.probe_throughput("atomic_read", False, False, 1184, 128, 1000)
    assert same["ns"] >= 0.5 * dist["ns"]


def test_latency_and_handoff_probes():
    from paper_1110_4623_gb300 import runner
    lat = runner.probe_latency("atomic_read", 2000)
    ld = runner.probe_latency("load_relaxed", 2000)
    assert 50 < lat["ns_per_op"] < 10_000 and 50 < ld["ns_per_op"] < 10_000
    sms = runner.sm_count()
    pp = runner.probe_pingpong(0, sms - 1, 1000)
    assert pp["status"] == 0 and 50 < pp["handoff_ns"] < 20_000


@pytest.mark.parametrize("op", ["volatile_load", "load_acquire", "atomic_write", "atomic_add64", "atomic_acqrel"])
def test_latency_probe_every_value_returning_access(op):
    # a dependent chain costs at least an L1 hit and less than a far-die round trip plus slack
    from paper_1110_4623_gb300 import runner
    assert 5 < runner.probe_latency(op, 1000)["ns_per_op"] < 10_000


@pytest.mark.parametrize("op", ["volatile_store", "store_release", "red_add"])
def test_latency_probe_refuses_accesses_without_a_result(op):
    from paper_1110_4623_gb300 import gsync as G
    from paper_1110_4623_gb300 import runner
    with pytest.raises(G.GsyncError):
        runner.probe_latency(op, 10)


def test_nanosleep_probe_monotone_on_average():
    from paper_1110_4623_gb300 import runner
    out = runner.probe_nanosleep([0, 1000, 10000], 32)
    assert out[2] > out[0]


def test_cs_probe():
    from paper_1110_4623_gb300 import runner
    a = runner.probe_cs(0, 256, 5000)["ns_per_cs"]
    b = runner.probe_cs(1024, 256, 5000)["ns_per_cs"]
    assert 0 < a and 0 < b


@pytest.mark.parametrize("cluster", [2, 8])
def test_cluster_handoff_probes(cluster):
    # The hardware cluster barrier and the hand-offs through distributed shared memory
    # (release/acquire flag, remote mbarrier arrive, relaxed 128-bit record pushed and pulled)
    # run and report sane times; malformed requests are refused.
    from paper_1110_4623_gb300 import gsync as G, runner
    import torch
    for op in (0, 1, 2, 3, 4):
        r = runner.probe_cluster(op, cluster, 1000)
        assert r["status"] == 0 and 10 < r["ns"] < 20_000, (op, r)
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    assert G.gsync_probe_cluster(5, cluster, 10, out) == G.GSYNC_EINVAL
    assert G.gsync_probe_cluster(3, 1, 10, out) == G.GSYNC_EINVAL
