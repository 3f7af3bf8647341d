"""Python binding of the gsync C ABI (include/gsync.h): the same entry-point names, argument
marshalling only.  Every operation runs in the CUDA library; if libgsync.so is missing or
fails to load, every call raises -- there is no fallback.

Pointer arguments accept a torch tensor (its data_ptr), a ctypes object, an int address or
None; `stream` accepts a torch.cuda.Stream, an int handle or None (the current torch stream).
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgsync.so")

# Enums of gsync.h
GSYNC_OK, GSYNC_EINVAL, GSYNC_ENOTRESIDENT, GSYNC_ETIMEDOUT, GSYNC_ECUDA, GSYNC_EABORTED = range(6)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOTRESIDENT", 3: "ETIMEDOUT", 4: "ECUDA", 5: "EABORTED"}
GSYNC_STATUS_TIMEOUT, GSYNC_STATUS_ABORTED, GSYNC_STATUS_VIOLATION, GSYNC_STATUS_CONFIG = 1, 2, 4, 8

MUTEX_KINDS = {"cas_spin": 0, "cas_backoff": 1, "ticket": 2, "sleep_queue": 3, "cohort": 4, "ring": 5, "cluster": 6,
               "cluster_mcs": 7}
# Policy kinds of the batched kernel: the mutex kinds it runs, plus the ticket lock whose turn
# line carries the guarded count and sum (GSYNC_BATCHED_TICKET_CARRY), and the cohort locks
# with carrying records over the two dies (GSYNC_BATCHED_COHORT_CARRY), over thread-block
# clusters (GSYNC_BATCHED_CLUSTER_CARRY), and over clusters within dies
# (GSYNC_BATCHED_CLUSTER_DIE_CARRY).
BATCHED_TICKET_CARRY = 16
BATCHED_COHORT_CARRY = 17
BATCHED_CLUSTER_CARRY = 18
BATCHED_CLUSTER_DIE_CARRY = 19
BATCHED_POLICY_KINDS = {**MUTEX_KINDS, "ticket_carry": BATCHED_TICKET_CARRY,
                        "cohort_carry": BATCHED_COHORT_CARRY, "cluster_carry": BATCHED_CLUSTER_CARRY,
                        "cluster_die_carry": BATCHED_CLUSTER_DIE_CARRY}
COHORT_DEFAULT_BUDGET = 64
BARRIER_KINDS = {"atomic": 0, "flag": 1, "tree": 2, "cluster": 3, "sharded": 4, "die": 5, "split": 6, "count": 7,
                 "exchange": 8}
SEM_KINDS = {"ticket": 0, "spin": 1, "spin_backoff": 2, "window": 3}
BACKOFF_EXPONENTIAL, BACKOFF_LINEAR_CYCLIC, BACKOFF_SPIN_THEN_SLEEP = 0, 1, 2
PROBE_OPS = {"volatile_load": 0, "volatile_store": 1, "atomic_read": 2, "atomic_write": 3,
             "load_acquire": 4, "load_relaxed": 5, "store_release": 6, "red_add": 7,
             "atomic_add64": 8, "atomic_acqrel": 9}

u32p = ctypes.c_void_p


class gsync_backoff(ctypes.Structure):
    _fields_ = [("policy", ctypes.c_uint32), ("min_ns", ctypes.c_uint32),
                ("max_ns", ctypes.c_uint32), ("spin", ctypes.c_uint32)]


class gsync_condvar_work(ctypes.Structure):
    _fields_ = [("producers", ctypes.c_int32), ("consumers", ctypes.c_int32), ("items_per_producer", ctypes.c_int32),
                ("capacity", ctypes.c_int32), ("block_threads", ctypes.c_int32), ("mutex_kind", ctypes.c_int32),
                ("cluster", ctypes.c_int32), ("value", u32p), ("seen", u32p), ("sum", u32p), ("count", u32p), ("status", u32p),
                ("acquisitions", u32p)]


class gsync_barrier_work(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("nblocks", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("rounds", ctypes.c_int32), ("full", ctypes.c_int32), ("cluster", ctypes.c_int32),
                ("slots", u32p), ("chk", u32p), ("mix", u32p), ("bad", u32p), ("status", u32p)]


class gsync_mutex_work(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("nblocks", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("acq", ctypes.c_int32), ("cs_words", ctypes.c_int32), ("cluster", ctypes.c_int32),
                ("delay", u32p), ("addend", u32p), ("data", u32p), ("total", u32p), ("grant_log", u32p),
                ("ticket", u32p), ("count", u32p), ("status", u32p)]


class gsync_sem_work(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("nblocks", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("pairs", ctypes.c_int32), ("initial_count", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("hold", u32p), ("addend", u32p), ("occupancy", u32p), ("max_occupancy", u32p),
                ("total", u32p), ("tally", u32p), ("count", u32p), ("status", u32p)]


class gsync_batched_work(ctypes.Structure):
    _fields_ = [("nkeys", ctypes.c_int32), ("nacq", ctypes.c_int32), ("nblocks", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("ngroups", ctypes.c_int32), ("rounds", ctypes.c_int32),
                ("cluster", ctypes.c_int32), ("nclasses", ctypes.c_int32), ("plain_launch", ctypes.c_int32),
                ("ncohort", ctypes.c_int32), ("timeout_ns", ctypes.c_uint64),
                ("mutex_state", u32p), ("key_class", u32p), ("policy", u32p), ("keys", u32p), ("adds", u32p),
                ("sum", u32p), ("count", u32p), ("group_start", u32p), ("group_size", u32p),
                ("group_of_block", u32p), ("group_state", u32p), ("slots", u32p), ("mix", u32p), ("bad", u32p),
                ("status", u32p), ("cohort_state", u32p)]


class gsync_serve_req(ctypes.Structure):
    _fields_ = [("seq", ctypes.c_uint32), ("len", ctypes.c_uint32), ("off", ctypes.c_uint32),
                ("seq_check", ctypes.c_uint32)]


class gsync_serve_cfg(ctypes.Structure):
    _fields_ = [("nreq", ctypes.c_int32), ("nslots", ctypes.c_int32), ("nblocks", ctypes.c_int32),
                ("admitters", ctypes.c_int32), ("chunk_elems", ctypes.c_int32), ("ring_slots", ctypes.c_int32),
                ("start_delay_us", ctypes.c_int32), ("drain_timeout_s", ctypes.c_int32),
                ("timeout_ns", ctypes.c_uint64)]


class gsync_serve_buffers(ctypes.Structure):
    _fields_ = [("pool", u32p), ("pool_elems", ctypes.c_int64), ("offset", u32p), ("length", u32p),
                ("sched_ns", u32p), ("ring", u32p),
                ("ctrl", u32p), ("res", u32p), ("done", u32p), ("latency_ns", u32p), ("publish_ns", u32p),
                ("trace", u32p),
                ("stats", ctypes.c_uint32 * 4)]


# name -> (restype, argtypes)
_SIG = {
    "gsync_mutex_bytes": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int]),
    "gsync_mutex_init": (ctypes.c_int, [u32p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(gsync_backoff), ctypes.c_uint64, u32p]),
    "gsync_mutex_init_cohort": (ctypes.c_int, [u32p, ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(gsync_backoff),
                                               ctypes.c_uint64, u32p]),
    "gsync_device_topology": (ctypes.c_int, [u32p, ctypes.POINTER(ctypes.c_int), u32p]),
    "gsync_mutex_init_cluster": (ctypes.c_int, [u32p, ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(gsync_backoff),
                                                ctypes.c_uint64, u32p]),
    "gsync_mutex_init_cluster_mcs": (ctypes.c_int, [u32p, ctypes.c_size_t, ctypes.c_int,
                                                    ctypes.POINTER(gsync_backoff), ctypes.c_uint64, u32p]),
    "gsync_check_coresident": (ctypes.c_int, [u32p, ctypes.c_int, ctypes.c_int, ctypes.c_size_t, ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_int)]),
    "gsync_launch_coresident": (ctypes.c_int, [u32p, ctypes.c_int, ctypes.c_int, ctypes.c_size_t, ctypes.c_int, u32p,
                                               u32p]),
    "gsync_cond_bytes": (ctypes.c_size_t, []),
    "gsync_cond_init": (ctypes.c_int, [u32p, ctypes.c_size_t, ctypes.POINTER(gsync_backoff), ctypes.c_uint64, u32p]),
    "gsync_bench_condvar_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int]),
    "gsync_probe_condvar_cs": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, u32p, ctypes.c_size_t,
                                              ctypes.POINTER(ctypes.c_uint64), u32p]),
    "gsync_bench_condvar": (ctypes.c_int, [ctypes.POINTER(gsync_condvar_work), ctypes.POINTER(gsync_backoff), u32p,
                                           ctypes.c_size_t, u32p]),
    "gsync_barrier_bytes": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "gsync_barrier_init": (ctypes.c_int, [u32p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_uint64, u32p]),
    "gsync_sem_bytes": (ctypes.c_size_t, [ctypes.c_int]),
    "gsync_sem_init": (ctypes.c_int, [u32p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int,
                                      ctypes.POINTER(gsync_backoff), ctypes.c_uint64, u32p]),
    "gsync_object_abort_flag": (ctypes.c_int, [u32p, ctypes.POINTER(ctypes.c_uint32), u32p]),
    "gsync_object_abort": (ctypes.c_int, [u32p, u32p]),
    "gsync_max_coresident_blocks": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                   ctypes.POINTER(ctypes.c_int)]),
    "gsync_device_sm_count": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int)]),
    "gsync_last_cuda_error": (ctypes.c_int, []),
    "gsync_bench_barrier": (ctypes.c_int, [u32p, ctypes.POINTER(gsync_barrier_work), u32p]),
    "gsync_bench_barrier_static": (ctypes.c_int, [ctypes.POINTER(gsync_barrier_work), ctypes.c_int, ctypes.c_uint64,
                                                  u32p]),
    "gsync_probe_barrier_trace": (ctypes.c_int, [u32p, ctypes.POINTER(gsync_barrier_work), u32p, u32p]),
    "gsync_bench_mutex": (ctypes.c_int, [u32p, ctypes.POINTER(gsync_mutex_work), u32p]),
    "gsync_bench_mutex_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "gsync_bench_mutex_host": (ctypes.c_int, [ctypes.POINTER(gsync_mutex_work), ctypes.POINTER(gsync_backoff),
                                              u32p, ctypes.c_size_t, u32p]),
    "gsync_bench_sem": (ctypes.c_int, [u32p, ctypes.POINTER(gsync_sem_work), u32p]),
    "gsync_bench_batched": (ctypes.c_int, [ctypes.POINTER(gsync_batched_work), u32p]),
    "gsync_serve_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int]),
    "gsync_serve_run": (ctypes.c_int, [ctypes.POINTER(gsync_serve_cfg), ctypes.POINTER(gsync_serve_buffers), u32p,
                                       ctypes.c_size_t, u32p]),
    "gsync_serve_baseline_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int]),
    "gsync_probe_host_pingpong": (ctypes.c_int, [u32p, ctypes.c_int, u32p, u32p]),
    "gsync_serve_baseline": (ctypes.c_int, [ctypes.POINTER(gsync_serve_cfg), ctypes.POINTER(gsync_serve_buffers),
                                            u32p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]),
    "gsync_probe_throughput": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int, u32p, u32p, u32p]),
    "gsync_probe_latency": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, u32p, u32p, u32p]),
    "gsync_probe_pingpong": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, u32p, u32p, u32p]),
    "gsync_probe_nanosleep": (ctypes.c_int, [u32p, ctypes.c_int, ctypes.c_int, u32p, u32p]),
    "gsync_probe_cs": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, u32p, u32p, u32p]),
    "gsync_probe_cs_scratch_bytes": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int]),
    "gsync_probe_handoff": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           u32p, u32p, u32p]),
    "gsync_probe_cluster": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, u32p, u32p]),
    "gsync_probe_fence": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, u32p, u32p, u32p]),
    "gsync_probe_sem_cs": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, u32p, u32p, u32p, u32p, u32p]),
    "gsync_probe_rtt_by_sm": (ctypes.c_int, [u32p, ctypes.c_int, u32p, u32p, u32p, u32p]),
    "gsync_probe_rtt_by_line": (ctypes.c_int, [ctypes.c_int, u32p, ctypes.c_int, ctypes.c_int, ctypes.c_int, u32p,
                                               u32p]),
}
SIGNAL_MODES = {"st_release": 0, "fence_st_relaxed": 1, "st_relaxed": 2, "red_release": 3, "exch_release": 4}
WAIT_MODES = {"ld_acquire": 0, "ld_relaxed_fence": 1, "ld_relaxed": 2, "ld_relaxed_then_acquire": 3,
              "ld_volatile_fence": 4, "ld_relaxed_x2": 5}

_lib = None


def lib():
    """Loads libgsync.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1110_4623_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIG.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def ptr(x):
    """Address of a torch tensor / int / ctypes object / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return ctypes.addressof(x)


def stream_handle(stream=None):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class GsyncError(RuntimeError):
    def __init__(self, fn, rc):
        extra = f" (cudaError {lib().gsync_last_cuda_error()})" if rc == GSYNC_ECUDA else ""
        super().__init__(f"{fn} returned {STATUS_NAMES.get(rc, rc)}{extra}")
        self.rc = rc


def check(fn, rc):
    if rc != GSYNC_OK:
        raise GsyncError(fn, rc)
    return rc


# ---- objects --------------------------------------------------------------------------

def gsync_mutex_bytes(kind: int, max_waiters: int) -> int:
    return lib().gsync_mutex_bytes(kind, max_waiters)


def gsync_mutex_init(state, nbytes, kind, max_waiters, backoff=None, timeout_ns=0, stream=None) -> int:
    bo = ctypes.byref(backoff) if backoff is not None else None
    return lib().gsync_mutex_init(ptr(state), nbytes, kind, max_waiters, bo, timeout_ns, stream_handle(stream))


def gsync_barrier_bytes(kind: int, nblocks: int, param: int) -> int:
    return lib().gsync_barrier_bytes(kind, nblocks, param)


def gsync_barrier_init(state, nbytes, kind, nblocks, param, timeout_ns=0, stream=None) -> int:
    return lib().gsync_barrier_init(ptr(state), nbytes, kind, nblocks, param, timeout_ns, stream_handle(stream))


def gsync_sem_bytes(kind: int) -> int:
    return lib().gsync_sem_bytes(kind)


def gsync_sem_init(state, nbytes, kind, initial_count, backoff=None, timeout_ns=0, stream=None) -> int:
    bo = ctypes.byref(backoff) if backoff is not None else None
    return lib().gsync_sem_init(ptr(state), nbytes, kind, initial_count, bo, timeout_ns, stream_handle(stream))


def gsync_object_abort_flag(state, stream=None) -> tuple[int, int]:
    v = ctypes.c_uint32(0)
    rc = lib().gsync_object_abort_flag(ptr(state), ctypes.byref(v), stream_handle(stream))
    return rc, v.value


def gsync_object_abort(state, stream=None) -> int:
    return lib().gsync_object_abort(ptr(state), stream_handle(stream))


def gsync_max_coresident_blocks(workload: int, kind: int, block_threads: int, cluster: int = 1) -> tuple[int, int]:
    v = ctypes.c_int(0)
    rc = lib().gsync_max_coresident_blocks(workload, kind, block_threads, cluster, ctypes.byref(v))
    return rc, v.value


def gsync_mutex_init_cohort(state, nbytes, budget, backoff=None, timeout_ns=0, stream=None) -> int:
    bo = ctypes.byref(backoff) if backoff is not None else None
    return lib().gsync_mutex_init_cohort(ptr(state), nbytes, budget, bo, timeout_ns, stream_handle(stream))


def gsync_mutex_init_cluster(state, nbytes, budget, backoff=None, timeout_ns=0, stream=None) -> int:
    bo = ctypes.byref(backoff) if backoff is not None else None
    return lib().gsync_mutex_init_cluster(ptr(state), nbytes, budget, bo, timeout_ns, stream_handle(stream))


def gsync_mutex_init_cluster_mcs(state, nbytes, budget, backoff=None, timeout_ns=0, stream=None) -> int:
    bo = ctypes.byref(backoff) if backoff is not None else None
    return lib().gsync_mutex_init_cluster_mcs(ptr(state), nbytes, budget, bo, timeout_ns, stream_handle(stream))


def gsync_device_topology(die_of_sm, stream=None) -> tuple[int, int]:
    """die_of_sm: a writable host buffer (numpy uint8) of at least sm_count bytes."""
    nd = ctypes.c_int(0)
    rc = lib().gsync_device_topology(die_of_sm.ctypes.data, ctypes.byref(nd), stream_handle(stream))
    return rc, nd.value


def gsync_cond_bytes() -> int:
    return lib().gsync_cond_bytes()


def gsync_cond_init(state, nbytes, backoff=None, timeout_ns=0, stream=None) -> int:
    bo = ctypes.byref(backoff) if backoff is not None else None
    return lib().gsync_cond_init(ptr(state), nbytes, bo, timeout_ns, stream_handle(stream))


def gsync_bench_condvar_workspace_bytes(capacity) -> int:
    return lib().gsync_bench_condvar_workspace_bytes(capacity)


def gsync_probe_condvar_cs(block_threads, iters, frame_only, workspace, nbytes, stream=None) -> tuple[int, int]:
    out = (ctypes.c_uint64 * 1)()
    rc = lib().gsync_probe_condvar_cs(block_threads, iters, int(frame_only), ptr(workspace), nbytes, out,
                                      stream_handle(stream))
    return rc, out[0]


def gsync_bench_condvar(work, backoff, workspace, nbytes, stream=None) -> int:
    bo = ctypes.byref(backoff) if backoff is not None else None
    return lib().gsync_bench_condvar(ctypes.byref(work), bo, ptr(workspace), nbytes, stream_handle(stream))


def gsync_device_sm_count() -> tuple[int, int]:
    v = ctypes.c_int(0)
    rc = lib().gsync_device_sm_count(ctypes.byref(v))
    return rc, v.value


def gsync_last_cuda_error() -> int:
    return lib().gsync_last_cuda_error()


# ---- workloads ------------------------------------------------------------------------

def gsync_bench_barrier(state, work: gsync_barrier_work, stream=None) -> int:
    return lib().gsync_bench_barrier(ptr(state), ctypes.byref(work), stream_handle(stream))


def gsync_bench_barrier_static(work: gsync_barrier_work, param: int = 0, timeout_ns: int = 0, stream=None) -> int:
    """The barrier workload in the library's own static device scratch (no allocation)."""
    return lib().gsync_bench_barrier_static(ctypes.byref(work), param, timeout_ns, stream_handle(stream))


def gsync_bench_mutex(state, work: gsync_mutex_work, stream=None) -> int:
    return lib().gsync_bench_mutex(ptr(state), ctypes.byref(work), stream_handle(stream))


def gsync_bench_mutex_workspace_bytes(kind, nblocks, acq, cs_words) -> int:
    return lib().gsync_bench_mutex_workspace_bytes(kind, nblocks, acq, cs_words)


def gsync_bench_mutex_host(work: gsync_mutex_work, backoff, workspace, workspace_bytes, stream=None) -> int:
    bo = ctypes.byref(backoff) if backoff is not None else None
    return lib().gsync_bench_mutex_host(ctypes.byref(work), bo, ptr(workspace), workspace_bytes,
                                        stream_handle(stream))


def gsync_bench_sem(state, work: gsync_sem_work, stream=None) -> int:
    return lib().gsync_bench_sem(ptr(state), ctypes.byref(work), stream_handle(stream))


def gsync_bench_batched(work: gsync_batched_work, stream=None) -> int:
    return lib().gsync_bench_batched(ctypes.byref(work), stream_handle(stream))


def gsync_serve_workspace_bytes(nslots: int) -> int:
    return lib().gsync_serve_workspace_bytes(nslots)


def gsync_serve_run(cfg: gsync_serve_cfg, buf: gsync_serve_buffers, workspace, workspace_bytes, stream=None) -> int:
    return lib().gsync_serve_run(ctypes.byref(cfg), ctypes.byref(buf), ptr(workspace), workspace_bytes,
                                 stream_handle(stream))


def gsync_serve_baseline_workspace_bytes(nreq: int) -> int:
    return lib().gsync_serve_baseline_workspace_bytes(nreq)


def gsync_serve_baseline(cfg: gsync_serve_cfg, buf: gsync_serve_buffers, workspace, workspace_bytes, streams) -> int:
    arr = (ctypes.c_void_p * len(streams))(*[stream_handle(s) for s in streams])
    return lib().gsync_serve_baseline(ctypes.byref(cfg), ctypes.byref(buf), ptr(workspace), workspace_bytes, arr,
                                      len(streams))


# ---- probes ---------------------------------------------------------------------------

def gsync_probe_throughput(op, contentious, pre_atomic, nblocks, block_threads, iters, scratch, times,
                           stream=None) -> int:
    return lib().gsync_probe_throughput(op, contentious, pre_atomic, nblocks, block_threads, iters, ptr(scratch),
                                        ptr(times), stream_handle(stream))


def gsync_probe_latency(op, iters, scratch, out, stream=None) -> int:
    return lib().gsync_probe_latency(op, iters, ptr(scratch), ptr(out), stream_handle(stream))


def gsync_probe_pingpong(sm_a, sm_b, iters, scratch, out, stream=None) -> int:
    return lib().gsync_probe_pingpong(sm_a, sm_b, iters, ptr(scratch), ptr(out), stream_handle(stream))


def gsync_probe_nanosleep(req_ns, n, iters, out_ns, stream=None) -> int:
    return lib().gsync_probe_nanosleep(ptr(req_ns), n, iters, ptr(out_ns), stream_handle(stream))


def gsync_probe_cs(cs_words, block_threads, iters, scratch, out, stream=None) -> int:
    return lib().gsync_probe_cs(cs_words, block_threads, iters, ptr(scratch), ptr(out), stream_handle(stream))


def gsync_probe_cs_scratch_bytes(cs_words, iters) -> int:
    return lib().gsync_probe_cs_scratch_bytes(cs_words, iters)


def gsync_probe_handoff(signal_mode, wait_mode, sm_a, sm_b, iters, scratch, out, stream=None) -> int:
    return lib().gsync_probe_handoff(signal_mode, wait_mode, sm_a, sm_b, iters, ptr(scratch), ptr(out),
                                     stream_handle(stream))


def gsync_probe_cluster(op, cluster, iters, out, stream=None) -> int:
    return lib().gsync_probe_cluster(op, cluster, iters, ptr(out), stream_handle(stream))


def gsync_probe_fence(op, iters, scratch, out, stream=None) -> int:
    return lib().gsync_probe_fence(op, iters, ptr(scratch), ptr(out), stream_handle(stream))


def gsync_probe_rtt_by_sm(line, iters, scratch, out_ns, status, stream=None) -> int:
    return lib().gsync_probe_rtt_by_sm(ptr(line), iters, ptr(scratch), ptr(out_ns), ptr(status), stream_handle(stream))


def gsync_probe_rtt_by_line(sm, base, nlines, stride_bytes, iters, out_ns, stream=None) -> int:
    return lib().gsync_probe_rtt_by_line(sm, ptr(base), nlines, stride_bytes, iters, ptr(out_ns), stream_handle(stream))


def gsync_probe_sem_cs(block_threads, iters, hold, addend, scratch, out, stream=None) -> int:
    return lib().gsync_probe_sem_cs(block_threads, iters, ptr(hold), ptr(addend), ptr(scratch), ptr(out),
                                    stream_handle(stream))


def gsync_probe_barrier_trace(state, work: gsync_barrier_work, trace, stream=None) -> int:
    return lib().gsync_probe_barrier_trace(ptr(state), ctypes.byref(work), ptr(trace), stream_handle(stream))


def gsync_probe_host_pingpong(words, iters, out_ns, stream=None) -> int:
    return lib().gsync_probe_host_pingpong(ptr(words), iters, ptr(out_ns), stream_handle(stream))
