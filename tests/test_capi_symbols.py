"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every function that
include/gsync.h declares (no compute calls: this runs on the CPU-only machine too)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in os.listdir(os.path.join(ROOT, "include")) if h.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:int|size_t|void|uint32_t|uint64_t)\s+\**\s*(gsync_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib_path():
    from paper_1110_4623_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["gsync_mutex_bytes", "gsync_mutex_init", "gsync_barrier_bytes", "gsync_barrier_init",
                     "gsync_sem_bytes", "gsync_sem_init", "gsync_bench_barrier", "gsync_bench_mutex",
                     "gsync_bench_sem", "gsync_probe_throughput", "gsync_max_coresident_blocks"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binding_signatures_match(lib_path):
    from paper_1110_4623_gb300 import gsync
    lib = gsync.lib()
    for name in declared_functions():
        assert hasattr(lib, name)
        assert name in gsync._SIG, f"binding has no signature for {name}"


def test_size_queries_without_gpu(lib_path):
    from paper_1110_4623_gb300 import gsync as G
    # Pure host arithmetic: no CUDA call is made.
    assert G.gsync_mutex_bytes(G.MUTEX_KINDS["cas_spin"], 1184) == 3 * 128
    assert G.gsync_mutex_bytes(G.MUTEX_KINDS["sleep_queue"], 1184) == (3 + 2048) * 128
    assert G.gsync_mutex_bytes(9, 4) == 0 and G.gsync_mutex_bytes(0, 0) == 0
    # two arrival counters (by epoch parity) and the release epoch
    assert G.gsync_barrier_bytes(G.BARRIER_KINDS["atomic"], 1184, 0) == 4 * 128
    assert G.gsync_barrier_bytes(G.BARRIER_KINDS["flag"], 1184, 0) == (1 + 37 + 37) * 128
    assert G.gsync_barrier_bytes(G.BARRIER_KINDS["flag"], 1184, 1) == (1 + 37 + 1) * 128
    # fan-in 8 over 1184 blocks: 148 + 19 + 3 + 1 nodes
    assert G.gsync_barrier_bytes(G.BARRIER_KINDS["tree"], 1184, 8) == (2 + 148 + 19 + 3 + 1) * 128
    assert G.gsync_barrier_bytes(G.BARRIER_KINDS["tree"], 16, 1) == 0
    # the tree's counting form has the same nodes; forms above 1 and fan-ins past 1024 are refused
    assert G.gsync_barrier_bytes(G.BARRIER_KINDS["tree"], 1184, 8 | 1 << 16) == (2 + 148 + 19 + 3 + 1) * 128
    assert G.gsync_barrier_bytes(G.BARRIER_KINDS["tree"], 1184, 8 | 2 << 16) == 0
    assert G.gsync_barrier_bytes(G.BARRIER_KINDS["tree"], 1184, 1025 | 1 << 16) == 0
    # the cluster barrier: c | form << 4 | sleep << 8
    assert G.gsync_barrier_bytes(G.BARRIER_KINDS["cluster"], 1184, 8 | 2 << 4 | 8 << 8) == 4 * 128
    assert G.gsync_barrier_bytes(G.BARRIER_KINDS["cluster"], 1184, 8 | 3 << 4) == 0
    assert G.gsync_barrier_bytes(G.BARRIER_KINDS["cluster"], 1184, 8 | 1024 << 8) == 0
    assert G.gsync_barrier_bytes(G.BARRIER_KINDS["cluster"], 1184, 8) == 4 * 128
    # two-die objects: 32 KB, room for a 4 KB page homed on each die
    assert G.gsync_barrier_bytes(G.BARRIER_KINDS["die"], 1184, 0) == 32768
    assert G.gsync_barrier_bytes(G.BARRIER_KINDS["die"], 1184, 1) == 32768
    assert G.gsync_barrier_bytes(G.BARRIER_KINDS["die"], 1184, 2) == 0
    # split: header, R release copies, 2S counters, 2 top counters
    assert G.gsync_barrier_bytes(G.BARRIER_KINDS["split"], 1184, 16 | 8 << 8) == (1 + 8 + 32 + 2) * 128
    assert G.gsync_barrier_bytes(G.BARRIER_KINDS["split"], 1184, 65 | 8 << 8) == 0
    assert G.gsync_barrier_bytes(G.BARRIER_KINDS["split"], 1184, 16) == 0  # R = 0
    assert G.gsync_barrier_bytes(G.BARRIER_KINDS["count"], 1184, 0) == 2 * 128
    # exchange: header, counter, then two 16-byte records per block
    assert G.gsync_barrier_bytes(G.BARRIER_KINDS["exchange"], 1184, 8) == (2 + 296) * 128
    assert G.gsync_barrier_bytes(G.BARRIER_KINDS["exchange"], 5, 0) == (2 + 2) * 128
    assert G.gsync_barrier_bytes(G.BARRIER_KINDS["exchange"], 1184, 1024) == 0
    assert G.gsync_barrier_bytes(G.BARRIER_KINDS["count"], 1184, 1024) == 0
    assert G.gsync_barrier_bytes(G.BARRIER_KINDS["count"], 1184, 8 | 16 << 16) == (2 + 16) * 128
    assert G.gsync_barrier_bytes(G.BARRIER_KINDS["count"], 1184, 8 | 65 << 16) == 0
    assert G.gsync_mutex_bytes(G.MUTEX_KINDS["cohort"], 1) == 32768
    # ring: header, tail, head, one line per entry (a power of two >= the waiters)
    assert G.gsync_mutex_bytes(G.MUTEX_KINDS["ring"], 1184) == (3 + 2048) * 128
    assert G.gsync_mutex_bytes(G.MUTEX_KINDS["cluster"], 4) == 3 * 128  # the global lock; local locks live in smem
    assert G.gsync_mutex_bytes(G.MUTEX_KINDS["cluster_mcs"], 4) == 3 * 128  # nodes live in smem
    assert G.gsync_mutex_bytes(8, 4) == 0
    assert G.gsync_barrier_bytes(G.BARRIER_KINDS["cluster"], 1183, 8) == 0
    assert G.gsync_sem_bytes(0) == 4 * 128 and G.gsync_sem_bytes(3) == 4 * 128 and G.gsync_sem_bytes(4) == 0
    assert G.gsync_bench_mutex_workspace_bytes(2, 1184, 100, 1024) > 4 * 1184 * 100 * 4
    assert G.gsync_probe_cs_scratch_bytes(64, 1000) > 0


def test_invalid_arguments_rejected_without_gpu(lib_path):
    import ctypes
    from paper_1110_4623_gb300 import gsync as G
    # Null / misaligned state is rejected before any CUDA call.
    assert G.lib().gsync_mutex_init(None, 384, 0, 4, None, 0, None) == G.GSYNC_EINVAL
    # cohort: null state, budget outside 1..32767, too small a state
    assert G.lib().gsync_mutex_init_cohort(None, 32768, 64, None, 0, None) == G.GSYNC_EINVAL
    assert G.lib().gsync_mutex_init_cohort(256, 32768, 0, None, 0, None) == G.GSYNC_EINVAL
    assert G.lib().gsync_mutex_init_cohort(256, 32768, 32768, None, 0, None) == G.GSYNC_EINVAL
    assert G.lib().gsync_mutex_init_cohort(256, 4096, 64, None, 0, None) == G.GSYNC_EINVAL
    assert G.lib().gsync_device_topology(None, None, None) == G.GSYNC_EINVAL
    # the host-side abort: null or misaligned state
    assert G.lib().gsync_object_abort(None, None) == G.GSYNC_EINVAL
    assert G.lib().gsync_object_abort(0x1004, None) == G.GSYNC_EINVAL
    # the caller-kernel gate rejects a null kernel or a bad shape before any CUDA call
    lib = G.lib()
    n = ctypes.c_int(0)
    assert lib.gsync_check_coresident(None, 1, 128, 0, 1, ctypes.byref(n)) == G.GSYNC_EINVAL
    assert lib.gsync_check_coresident(8, 0, 128, 0, 1, ctypes.byref(n)) == G.GSYNC_EINVAL
    assert lib.gsync_check_coresident(8, 1, 128, 0, 17, ctypes.byref(n)) == G.GSYNC_EINVAL
    # backoff policies 0..2 only (checked before any CUDA call)
    import ctypes
    bad = G.gsync_backoff(3, 16, 512, 0)
    assert G.lib().gsync_mutex_init(256, 384, G.MUTEX_KINDS["cas_backoff"], 4, ctypes.byref(bad), 0,
                                    None) == G.GSYNC_EINVAL
    assert G.lib().gsync_mutex_init(0x1001, 384, 0, 4, None, 0, None) == G.GSYNC_EINVAL
    assert G.lib().gsync_barrier_init(0x1000, 10, 0, 4, 0, 0, None) == G.GSYNC_EINVAL  # too small
    w = G.gsync_mutex_work(0, 0, 256, 1, 1, 0, None, None, None, None, None, None, None, None)
    assert G.lib().gsync_bench_mutex(0x1000, ctypes.byref(w), None) == G.GSYNC_EINVAL
