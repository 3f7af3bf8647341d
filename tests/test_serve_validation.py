"""The serving entry points reject malformed requests on the host, before any CUDA call
(runs without a GPU)."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def G():
    from paper_1110_4623_gb300 import build, gsync
    build.build()
    return gsync


def buffers(G, off, ln, sched, pool_elems):
    off = np.asarray(off, np.int64); ln = np.asarray(ln, np.int64); sched = np.asarray(sched, np.int64)
    keep = [off, ln, sched, np.zeros(64 * 128, np.uint8), np.zeros(64, np.uint32), np.zeros(len(off), np.int64),
            np.zeros(len(off), np.uint32), np.zeros(len(off), np.int64)]
    b = G.gsync_serve_buffers(0x1000, pool_elems, off.ctypes.data, ln.ctypes.data, sched.ctypes.data,
                              keep[3].ctypes.data, keep[4].ctypes.data, keep[5].ctypes.data, keep[6].ctypes.data,
                              keep[7].ctypes.data, None, None, (ctypes.c_uint32 * 4)())
    return b, keep


@pytest.mark.parametrize("off,ln,sched", [([0, 10], [5, 0], [0, 1]),           # empty request
                                           ([-1], [5], [0]),                     # negative offset
                                           ([90], [20], [0]),                    # past the pool end
                                           ([0, 0], [4, 4], [5, 1]),             # arrivals out of order
                                           ([0], [(1 << 15) * 1024 + 1], [0])])  # too many chunks
def test_bad_requests_rejected(G, off, ln, sched):
    pool = 100 if max(ln) < 1 << 20 else 1 << 40
    b, keep = buffers(G, off, ln, sched, pool)
    cfg = G.gsync_serve_cfg(len(off), 4, 8, 2, 1024, 64, 0, 1, 0)
    ws = (ctypes.c_uint8 * 4096)()
    addr = (ctypes.addressof(ws) + 255) & ~255
    assert G.gsync_serve_run(cfg, b, addr, 2048, stream=0) == G.GSYNC_EINVAL
    assert G.gsync_serve_baseline(cfg, b, addr, 2048, [1]) == G.GSYNC_EINVAL


def test_bad_config_rejected(G):
    b, keep = buffers(G, [0], [5], [0], 100)
    ws = (ctypes.c_uint8 * 4096)()
    addr = (ctypes.addressof(ws) + 255) & ~255
    for cfg in [G.gsync_serve_cfg(1, 65, 8, 2, 1024, 64, 0, 1, 0),   # too many slots
                G.gsync_serve_cfg(1, 4, 8, 8, 1024, 64, 0, 1, 0),    # no worker blocks
                G.gsync_serve_cfg(1, 4, 8, 2, 1024, 48, 0, 1, 0),    # ring not a power of two
                G.gsync_serve_cfg(1, 4, 8, 2, 512, 64, 0, 1, 0)]:    # chunk too small
        assert G.gsync_serve_run(cfg, b, addr, 2048, stream=0) == G.GSYNC_EINVAL
