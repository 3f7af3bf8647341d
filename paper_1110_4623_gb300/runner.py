"""Device-memory plumbing around the C ABI: allocates the objects and the workload buffers
as torch tensors, calls the entry points and copies results back as numpy arrays.  Every
synchronization step runs in the CUDA library (gsync.py raises if it is not built).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import gsync as G


def _u32(a) -> torch.Tensor:
    """Host uint32 array -> int32 device tensor with the same bits."""
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _zeros(n: int) -> torch.Tensor:
    return torch.zeros(max(int(n), 1), dtype=torch.int32, device="cuda")


def _np(t: torch.Tensor, n: int | None = None) -> np.ndarray:
    a = t.cpu().numpy().view(np.uint32)
    return a if n is None else a[:n]


def _state(nbytes: int) -> torch.Tensor:
    if nbytes <= 0:
        raise G.GsyncError("size query", G.GSYNC_EINVAL)
    t = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    assert t.data_ptr() % 256 == 0
    return t


def backoff(policy: int = G.BACKOFF_EXPONENTIAL, min_ns: int = 0, max_ns: int = 0, spin: int = 0) -> G.gsync_backoff:
    return G.gsync_backoff(policy, min_ns, max_ns, spin)


@dataclass
class StatusView:
    rc: int
    bits: int

    @property
    def ok(self) -> bool:
        return self.rc == G.GSYNC_OK and self.bits == 0


# ---------------------------------------------------------------------------------------

class Watchdog:
    """Host-side watchdog on a stream (the host half of failure detection; the device half is
    every wait's own deadline).  wait() records an event on `stream` and polls it; if the work
    queued before it has not finished within `deadline_s`, it sets the abort word of every
    object in `objects` (gsync_object_abort, on a stream of its own that is not ordered after
    the watched one), so their waits return GSYNC_EABORTED within a few polls, and then waits
    for the stream to drain.  Returns True if it had to abort.

    Construct it before launching the work it watches: it creates its own stream and event
    here, because creating a stream while a kernel runs on the legacy default stream can wait
    for that kernel -- the very wait the watchdog exists to cut short."""

    def __init__(self, objects, deadline_s: float, stream=None):
        self.objects = list(objects)
        self.deadline_s = deadline_s
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.side = torch.cuda.Stream()  # torch creates its pool streams non-blocking
        self.done = torch.cuda.Event()
        self.fired = False

    def wait(self, poll_s: float = 0.001) -> bool:
        import time
        self.done.record(self.stream)
        t_end = time.monotonic() + self.deadline_s
        while not self.done.query():
            if time.monotonic() > t_end:
                for obj in self.objects:
                    G.check("gsync_object_abort", G.gsync_object_abort(obj, self.side))
                self.fired = True
                self.side.synchronize()
                break
            time.sleep(poll_s)
        self.done.synchronize()
        return self.fired


class BarrierRun:
    """A barrier object plus the buffers of the barrier workload (gsync_bench_barrier)."""

    def __init__(self, kind: str, nblocks: int, block_threads: int, rounds: int, full: bool,
                 param: int = 0, timeout_ns: int = 0):
        self.kind, self.k = kind, G.BARRIER_KINDS[kind]
        self.nblocks, self.rounds, self.full = nblocks, rounds, full
        if kind == "tree" and param == 0:
            param = 8
        if kind == "cluster" and param == 0:
            param = 2
        if kind == "sharded" and param == 0:
            param = min(32, nblocks)
        if kind == "split" and param == 0:
            param = 8 | 8 << 8
        self.param = param
        nbytes = G.gsync_barrier_bytes(self.k, nblocks, param)
        self.state = _state(nbytes)
        G.check("gsync_barrier_init", G.gsync_barrier_init(self.state, nbytes, self.k, nblocks, param, timeout_ns))
        self.slots = _zeros(2 * nblocks)
        self.chk = _zeros(rounds * nblocks) if full else None
        self.mix = _zeros(nblocks)
        self.bad = _zeros(nblocks)
        self.status = _zeros(1)
        self.work = G.gsync_barrier_work(self.k, nblocks, block_threads, rounds, int(full),
                                         param & 0xF if kind == "cluster" else 1,
                                         G.ptr(self.slots), G.ptr(self.chk), G.ptr(self.mix), G.ptr(self.bad),
                                         G.ptr(self.status))

    def launch(self, stream=None) -> int:
        return G.gsync_bench_barrier(self.state, self.work, stream)

    def trace(self) -> np.ndarray:
        """Per-block, per-round (before, after) globaltimer of each barrier_wait: [B, R, 2] ns."""
        t = torch.zeros(2 * self.nblocks * self.rounds, dtype=torch.int64, device="cuda")
        self.status.zero_()
        G.check("gsync_probe_barrier_trace", G.gsync_probe_barrier_trace(self.state, self.work, t))
        torch.cuda.synchronize()
        return t.cpu().numpy().reshape(self.nblocks, self.rounds, 2)

    def run(self) -> dict:
        self.status.zero_()
        rc = self.launch()
        torch.cuda.synchronize()
        out = {"rc": rc, "status": int(_np(self.status)[0]), "mix": _np(self.mix), "bad": _np(self.bad)}
        if self.full:
            out["chk"] = _np(self.chk).reshape(self.rounds, self.nblocks)
        return out


class MutexRun:
    """A mutex object plus the buffers of the mutex workload (gsync_bench_mutex)."""

    def __init__(self, kind: str, nblocks: int, block_threads: int, acq: int, cs_words: int,
                 delay: np.ndarray | None, addend: np.ndarray, bo: G.gsync_backoff | None = None,
                 timeout_ns: int = 0, budget: int | None = None, cluster: int = 8):
        self.kind, self.k = kind, G.MUTEX_KINDS[kind]
        self.cluster = cluster if kind in ("cluster", "cluster_mcs") else 0
        self.nblocks, self.acq, self.cs_words = nblocks, acq, cs_words
        self.bo = bo
        n = nblocks * acq
        self.nbytes = G.gsync_mutex_bytes(self.k, nblocks)
        self.state = _state(self.nbytes)
        if budget is not None and kind == "cluster":
            G.check("gsync_mutex_init_cluster", G.gsync_mutex_init_cluster(self.state, self.nbytes, budget, bo,
                                                                          timeout_ns))
        elif budget is not None and kind == "cluster_mcs":
            G.check("gsync_mutex_init_cluster_mcs", G.gsync_mutex_init_cluster_mcs(self.state, self.nbytes, budget, bo,
                                                                                  timeout_ns))
        elif budget is not None:
            G.check("gsync_mutex_init_cohort", G.gsync_mutex_init_cohort(self.state, self.nbytes, budget, bo, timeout_ns))
        else:
            G.check("gsync_mutex_init", G.gsync_mutex_init(self.state, self.nbytes, self.k, nblocks, bo, timeout_ns))
        self.delay = _u32(delay) if delay is not None else None
        self.addend = _u32(addend)
        self.data = _zeros(cs_words)
        self.total = _zeros(1)
        self.log = _zeros(n)
        self.ticket = _zeros(n)
        self.count = _zeros(nblocks)
        self.status = _zeros(1)
        self.work = G.gsync_mutex_work(self.k, nblocks, block_threads, acq, cs_words, self.cluster,
                                       G.ptr(self.delay), G.ptr(self.addend), G.ptr(self.data), G.ptr(self.total),
                                       G.ptr(self.log), G.ptr(self.ticket), G.ptr(self.count), G.ptr(self.status))

    def reset(self):
        self.data.zero_()
        self.total.zero_()
        self.status.zero_()

    def launch(self, stream=None) -> int:
        return G.gsync_bench_mutex(self.state, self.work, stream)

    def results(self) -> dict:
        torch.cuda.synchronize()
        n = self.nblocks * self.acq
        return {"status": int(_np(self.status)[0]), "data": _np(self.data, self.cs_words),
                "total": _np(self.total)[0], "log": _np(self.log, n), "ticket": _np(self.ticket, n),
                "count": _np(self.count)}

    def run(self) -> dict:
        self.reset()
        rc = self.launch()
        out = self.results()
        out["rc"] = rc
        return out


class CondVarRun:
    """The condition-variable workload (gsync_bench_condvar): a bounded producer/consumer
    queue under one mutex and two condition variables."""

    def __init__(self, producers: int, consumers: int, items_per_producer: int, capacity: int,
                 value: np.ndarray, block_threads: int = 128, bo: G.gsync_backoff | None = None,
                 mutex: str = "ticket", cluster: int = 0):
        n = producers * items_per_producer
        self.producers, self.consumers, self.n, self.bo = producers, consumers, n, bo
        self.value = _u32(value) if n else _zeros(1)
        self.seen = _zeros(n)
        self.sum = torch.zeros(consumers, dtype=torch.int64, device="cuda")
        self.count = _zeros(consumers)
        self.status = _zeros(1)
        self.acq = _zeros(1)
        self.nbytes = G.gsync_bench_condvar_workspace_bytes(capacity)
        self.ws = _state(self.nbytes)
        self.work = G.gsync_condvar_work(producers, consumers, items_per_producer, capacity, block_threads,
                                         G.MUTEX_KINDS[mutex], cluster,
                                         G.ptr(self.value), G.ptr(self.seen), G.ptr(self.sum), G.ptr(self.count),
                                         G.ptr(self.status), G.ptr(self.acq))

    def reset(self):
        self.seen.zero_()
        self.sum.zero_()
        self.count.zero_()
        self.status.zero_()
        self.acq.zero_()

    def launch(self, stream=None) -> int:
        return G.gsync_bench_condvar(self.work, self.bo, self.ws, self.nbytes, stream)

    def run(self) -> dict:
        self.reset()
        rc = self.launch()
        torch.cuda.synchronize()
        return {"rc": rc, "status": int(_np(self.status)[0]), "seen": _np(self.seen, self.n),
                "sum": self.sum.cpu().numpy(), "count": _np(self.count, self.consumers),
                "acquisitions": int(_np(self.acq)[0])}


class SemRun:
    """A counting semaphore plus the buffers of the semaphore workload (gsync_bench_sem)."""

    def __init__(self, kind: str, nblocks: int, block_threads: int, pairs: int, initial_count: int,
                 hold: np.ndarray | None, addend: np.ndarray, bo: G.gsync_backoff | None = None,
                 timeout_ns: int = 0):
        self.kind, self.k = kind, G.SEM_KINDS[kind]
        self.nblocks, self.pairs, self.n = nblocks, pairs, initial_count
        nbytes = G.gsync_sem_bytes(self.k)
        self.state = _state(nbytes)
        G.check("gsync_sem_init", G.gsync_sem_init(self.state, nbytes, self.k, initial_count, bo, timeout_ns))
        self.hold = _u32(hold) if hold is not None else None
        self.addend = _u32(addend)
        self.scalars = _zeros(5 * 32)  # occupancy, max_occupancy, total, tally, status on separate lines
        self.count = _zeros(nblocks)
        s = self.scalars
        self.work = G.gsync_sem_work(self.k, nblocks, block_threads, pairs, initial_count, 0,
                                     G.ptr(self.hold), G.ptr(self.addend), s.data_ptr(), s.data_ptr() + 128,
                                     s.data_ptr() + 256, s.data_ptr() + 384, G.ptr(self.count), s.data_ptr() + 512)

    def reset(self):
        self.scalars.zero_()

    def launch(self, stream=None) -> int:
        return G.gsync_bench_sem(self.state, self.work, stream)

    def results(self) -> dict:
        torch.cuda.synchronize()
        s = _np(self.scalars)
        return {"occupancy": int(s[0]), "max_occ": int(s[32]), "total": s[64], "tally": s[96],
                "status": int(s[128]), "count": _np(self.count)}

    def run(self) -> dict:
        self.reset()
        rc = self.launch()
        out = self.results()
        out["rc"] = rc
        return out


# ---- probes ---------------------------------------------------------------------------

def probe_throughput(op: str, contentious: bool, pre_atomic: bool, nblocks: int, block_threads: int = 128,
                     iters: int = 1000) -> dict:
    """Runs one probe; returns the span of the blocks' globaltimer windows (ns) and ops/s."""
    scratch = _state(256 * nblocks)
    times = torch.zeros(2 * nblocks, dtype=torch.int64, device="cuda")
    G.check("gsync_probe_throughput", G.gsync_probe_throughput(G.PROBE_OPS[op], int(contentious), int(pre_atomic),
                                                               nblocks, block_threads, iters, scratch, times))
    torch.cuda.synchronize()
    t = times.cpu().numpy().reshape(nblocks, 2)
    span = int(t[:, 1].max() - t[:, 0].min())
    return {"ns": span, "ops_per_s": nblocks * iters / (span * 1e-9) if span > 0 else float("inf"),
            "mean_block_ns": float((t[:, 1] - t[:, 0]).mean())}


def probe_latency(op: str, iters: int = 4096, scratch=None) -> dict:
    """Dependent-chain latency of one access kind; scratch: None (a fresh buffer) or the
    device address of 128 bytes, 128-byte aligned (where the chained word lives)."""
    if scratch is None:
        scratch = _state(256)
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    G.check("gsync_probe_latency", G.gsync_probe_latency(G.PROBE_OPS[op], iters, scratch, out))
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    return {"ns_per_op": o[0] / iters, "cycles_per_op": o[1] / iters}


def probe_pingpong(sm_a: int, sm_b: int, iters: int = 2000, scratch: torch.Tensor | None = None) -> dict:
    """Half a release/acquire ping-pong between SMs sm_a and sm_b on the flag lines at the start
    of `scratch` (512 bytes, 128-byte aligned; a fresh buffer when None)."""
    scratch = _state(512) if scratch is None else scratch
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    G.check("gsync_probe_pingpong", G.gsync_probe_pingpong(sm_a, sm_b, iters, scratch, out))
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    return {"handoff_ns": o[0] / (2 * iters), "status": int(o[3]), "sm_a": int(o[1]), "sm_b": int(o[2])}


def probe_handoff(signal: str, wait: str, sm_a: int, sm_b: int, iters: int = 2000) -> dict:
    scratch = _state(512)
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    G.check("gsync_probe_handoff", G.gsync_probe_handoff(G.SIGNAL_MODES[signal], G.WAIT_MODES[wait], sm_a, sm_b,
                                                         iters, scratch, out))
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    return {"handoff_ns": o[0] / (2 * iters), "status": int(o[3])}


def probe_cluster(op: int, cluster: int, iters: int = 2000) -> dict:
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    G.check("gsync_probe_cluster", G.gsync_probe_cluster(op, cluster, iters, out))
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    per = o[0] / iters if op == 0 else o[0] / (2 * iters)
    return {"ns": per, "status": int(o[3])}


def _near_pair() -> tuple[int, int]:
    """Two SMs of die 0 (any two SMs on a one-die GPU)."""
    die, _ = device_topology()
    d0 = np.flatnonzero(die == 0)
    return int(d0[0]), int(d0[len(d0) // 2])


def _fastest_page(measure, pages: int) -> dict:
    """The fastest of `measure(flag_lines)` over `pages` consecutive 4 KB pages of one buffer
    (line homes alternate between the dies by page, so some page is homed on the pair's own
    die); the result dict gets its page."""
    buf = _state((pages + 1) * 4096)
    best = None
    for page in range(pages):
        r = measure(buf[page * 4096:])
        r["page"] = page
        if r["status"] == 0 and (best is None or r["handoff_ns"] < best["handoff_ns"]):
            best = r
    return best if best is not None else r


def near_handoff(iters: int = 4000, pages: int = 8) -> dict:
    """The shortest SM-to-SM hand-off on this GPU: a release/acquire ping-pong between two SMs
    of one die, at the fastest of `pages` page placements of the flag lines (the placement
    homed on that die)."""
    sm_a, sm_b = _near_pair()
    r = _fastest_page(lambda lines: probe_pingpong(sm_a, sm_b, iters, scratch=lines), pages)
    r["sms"] = (sm_a, sm_b)
    return r


def near_handoff_relaxed(iters: int = 4000, pages: int = 8) -> dict:
    """The same near-die hand-off with a relaxed store observed by relaxed polls: no fence on
    either side, the floor of a hand-off that orders nothing but its own location (the
    carrying locks' hand-off, whose guarded data travel in the flag's own access)."""
    sm_a, sm_b = _near_pair()

    def measure(lines):
        out = torch.zeros(4, dtype=torch.int64, device="cuda")
        G.check("gsync_probe_handoff", G.gsync_probe_handoff(G.SIGNAL_MODES["st_relaxed"], G.WAIT_MODES["ld_relaxed"],
                                                             sm_a, sm_b, iters, lines, out))
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        return {"handoff_ns": o[0] / (2 * iters), "status": int(o[3])}

    r = _fastest_page(measure, pages)
    r["sms"] = (sm_a, sm_b)
    return r


def device_topology() -> tuple[np.ndarray, int]:
    """(die of every SM id, number of dies) as the library measured and cached it."""
    die = np.zeros(256, dtype=np.uint8)
    rc, nd = G.gsync_device_topology(die)
    G.check("gsync_device_topology", rc)
    return die[:sm_count()].copy(), nd


def probe_rtt_by_sm(line: torch.Tensor, iters: int = 64) -> dict:
    """ns per dependent atomic round trip from every SM to the line at line.data_ptr()."""
    scratch = _state(128)
    out = torch.zeros(sm_count(), dtype=torch.int64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    G.check("gsync_probe_rtt_by_sm", G.gsync_probe_rtt_by_sm(line, iters, scratch, out, status))
    torch.cuda.synchronize()
    return {"rtt_ns": out.cpu().numpy() / iters, "status": int(status.item())}


def probe_rtt_by_line(sm: int, buf: torch.Tensor, nlines: int, stride_bytes: int = 128, iters: int = 16) -> np.ndarray:
    """ns per dependent atomic round trip from SM `sm` to each line buf + i * stride_bytes."""
    if (nlines - 1) * stride_bytes + 4 > buf.numel() * buf.element_size():
        raise ValueError("line range exceeds the buffer")
    out = torch.zeros(nlines, dtype=torch.int64, device="cuda")
    G.check("gsync_probe_rtt_by_line", G.gsync_probe_rtt_by_line(sm, buf, nlines, stride_bytes, iters, out))
    torch.cuda.synchronize()
    return out.cpu().numpy() / iters


def probe_fence(op: int, iters: int = 2000) -> dict:
    scratch = _state(1024)
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    G.check("gsync_probe_fence", G.gsync_probe_fence(op, iters, scratch, out))
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    return {"ns_per_fence": o[0] / iters, "cycles_per_fence": o[1] / iters}


def probe_nanosleep(req_ns, iters: int = 64) -> np.ndarray:
    req = _u32(np.asarray(req_ns, dtype=np.uint32))
    out = torch.zeros(len(req_ns), dtype=torch.int64, device="cuda")
    G.check("gsync_probe_nanosleep", G.gsync_probe_nanosleep(req, len(req_ns), iters, out))
    torch.cuda.synchronize()
    return out.cpu().numpy()


def probe_cs(cs_words: int, block_threads: int = 256, iters: int = 20000, scratch=None) -> dict:
    """scratch: None (a fresh buffer) or the device address of gsync_probe_cs_scratch_bytes
    bytes, 256-byte aligned (lets the caller choose where the probe's hot lines live)."""
    if scratch is None:
        scratch = _state(G.gsync_probe_cs_scratch_bytes(cs_words, iters))
    out = (G.ctypes.c_uint64 * 1)()
    G.check("gsync_probe_cs", G.gsync_probe_cs(cs_words, block_threads, iters, scratch, out))
    return {"ns_per_cs": out[0] / iters}


def probe_sem_cs(hold: np.ndarray | None, addend: np.ndarray | None, block_threads: int = 128,
                 iters: int | None = None, scratch=None) -> dict:
    """Mean time of one semaphore critical section with the workload's hold times, alone
    (hold and addend None: the frame alone, with an empty critical section).  scratch: None
    or the device address of 1024 bytes, 256-byte aligned."""
    iters = iters if iters is not None else len(hold)
    h = _u32(hold) if hold is not None else None
    a = _u32(addend) if addend is not None else None
    if scratch is None:
        scratch = _state(1024)
    out = (G.ctypes.c_uint64 * 1)()
    G.check("gsync_probe_sem_cs", G.gsync_probe_sem_cs(block_threads, iters, h, a, scratch, out))
    return {"ns_per_cs": out[0] / iters}


def probe_condvar_cs(block_threads: int = 128, iters: int = 4000, frame_only: bool = False, scratch=None) -> dict:
    """Mean time of one critical section of the condition-variable queue, alone (frame_only:
    the frame around an empty body).  scratch: None or the device address of
    gsync_bench_condvar_workspace_bytes(16) bytes, 256-byte aligned."""
    nbytes = G.gsync_bench_condvar_workspace_bytes(16)
    if scratch is None:
        scratch = _state(nbytes)
    rc, ns = G.gsync_probe_condvar_cs(block_threads, iters, frame_only, scratch, nbytes)
    G.check("gsync_probe_condvar_cs", rc)
    return {"ns_per_cs": ns / iters}


def sm_count() -> int:
    rc, n = G.gsync_device_sm_count()
    G.check("gsync_device_sm_count", rc)
    return n


COHORT_OBJ_BYTES = 32 * 1024  # one two-die cohort object (gsync_mutex_bytes of COHORT)


class BatchedRun:
    """The batched many-mutex workload (gsync_bench_batched): 4096 mutexes with Zipf keys,
    barrier groups, a per-class policy table; optional capture into a CUDA graph."""

    def __init__(self, keys: np.ndarray, adds: np.ndarray, nkeys: int, nblocks: int, group_sizes: np.ndarray,
                 rounds: int, key_class: np.ndarray, nclasses: int, block_threads: int = 128, cluster: int = 1,
                 timeout_ns: int = 10_000_000_000, plain_launch: bool = False, ncohort: int = 128):
        """ncohort: how many of the lowest keys (the hottest, for Zipf keys) get a two-die cohort
        object for the cohort_carry policy kind (32 KB each)."""
        from .inputs import group_layout
        self.nkeys, self.nacq, self.nblocks = nkeys, len(keys), nblocks
        self.group_sizes = np.asarray(group_sizes, dtype=np.int32)
        self.rounds, self.cluster = rounds, cluster
        start, gob = group_layout(self.group_sizes, nblocks)
        self.group_start, self.group_of_block = start, gob
        ng = len(self.group_sizes)
        self.mutex_state = torch.zeros(nkeys * 384, dtype=torch.uint8, device="cuda")
        self.group_state = torch.zeros(max(ng, 1) * 512, dtype=torch.uint8, device="cuda")
        self.key_class = torch.from_numpy(np.ascontiguousarray(key_class, dtype=np.uint8)).cuda()
        self.policy = torch.zeros(nclasses * 4, dtype=torch.int32, device="cuda")
        self.keys = torch.from_numpy(np.ascontiguousarray(keys, dtype=np.int32)).cuda()
        self.adds = torch.from_numpy(np.ascontiguousarray(adds, dtype=np.int64)).cuda()
        self.sum = torch.zeros(nkeys, dtype=torch.int64, device="cuda")
        self.count = _zeros(nkeys)
        self.gstart = torch.from_numpy(np.ascontiguousarray(start, dtype=np.int32)).cuda() if ng else _zeros(1)
        self.gsize = torch.from_numpy(self.group_sizes).cuda() if ng else _zeros(1)
        self.gob = torch.from_numpy(gob).cuda()
        self.slots = _zeros(2 * nblocks)
        self.mix = _zeros(nblocks)
        self.bad = _zeros(nblocks)
        self.status = _zeros(1)
        self.ncohort = max(0, min(int(ncohort), nkeys))
        self.cohort_state = torch.zeros(max(self.ncohort, 1) * COHORT_OBJ_BYTES, dtype=torch.uint8, device="cuda")
        self.work = G.gsync_batched_work(nkeys, self.nacq, nblocks, block_threads, ng, rounds, cluster, nclasses,
                                         int(plain_launch), self.ncohort, timeout_ns, G.ptr(self.mutex_state),
                                         G.ptr(self.key_class), G.ptr(self.policy), G.ptr(self.keys),
                                         G.ptr(self.adds), G.ptr(self.sum), G.ptr(self.count), G.ptr(self.gstart),
                                         G.ptr(self.gsize), G.ptr(self.gob), G.ptr(self.group_state),
                                         G.ptr(self.slots), G.ptr(self.mix), G.ptr(self.bad), G.ptr(self.status),
                                         G.ptr(self.cohort_state))
        self.graph = None

    def set_policy(self, table):
        """table: list of (kind, min_ns, max_ns[, budget]) per class (budget: the cohort locks'
        passes per cohort, 0 = default).  Zeroes the mutexes (kinds may change) and, when a
        class uses cohort_carry or cluster_die_carry, places and initialises the cohort
        objects."""
        flat = []
        for entry in table:
            kind, mn, mx = entry[:3]
            budget = entry[3] if len(entry) > 3 else 0
            flat += [G.BATCHED_POLICY_KINDS[kind] if isinstance(kind, str) else int(kind), int(mn), int(mx), int(budget)]
        self.policy.copy_(torch.tensor(flat, dtype=torch.int32))
        self.mutex_state.zero_()
        if {G.BATCHED_COHORT_CARRY, G.BATCHED_CLUSTER_DIE_CARRY} & set(flat[0::4]):
            base = G.ptr(self.cohort_state)
            for k in range(self.ncohort):
                G.check("gsync_mutex_init_cohort",
                        G.gsync_mutex_init_cohort(base + k * COHORT_OBJ_BYTES, COHORT_OBJ_BYTES, 1))
        self.graph = None

    def reset(self):
        self.sum.zero_()
        self.count.zero_()
        self.status.zero_()

    def launch(self, stream=None) -> int:
        return G.gsync_bench_batched(self.work, stream)

    def capture(self) -> None:
        """Captures reset + launch into one CUDA graph (replayed by replay())."""
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.reset()
            G.check("gsync_bench_batched", self.launch())  # warm-up outside the graph
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        with torch.cuda.graph(g):
            self.reset()
            rc = self.launch()
        G.check("gsync_bench_batched (capture)", rc)
        self.graph = g

    def replay(self):
        self.graph.replay()

    def results(self) -> dict:
        torch.cuda.synchronize()
        return {"status": int(_np(self.status)[0]), "sum": self.sum.cpu().numpy(),
                "count": self.count.cpu().numpy().view(np.uint32).astype(np.uint64),
                "mix": _np(self.mix), "bad": _np(self.bad)}

    def run(self) -> dict:
        self.reset()
        rc = self.launch()
        out = self.results()
        out["rc"] = rc
        return out


def _cudart():
    """The CUDA runtime library that torch loaded (by its soname), else the toolkit's."""
    import ctypes
    import glob
    names = ["libcudart.so.13", "libcudart.so"] + sorted(glob.glob("/usr/local/cuda/lib64/libcudart.so*"))
    for name in names:
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    raise RuntimeError("no CUDA runtime library found for a managed allocation")


class ManagedBuffer:
    """Managed memory (cudaMallocManaged, one address for host and device), freed on collection.
    The serving loop places a ring held here in device memory, written in place by the host."""

    def __init__(self, nbytes: int):
        import ctypes
        self._rt = _cudart()
        p = ctypes.c_void_p()
        rc = self._rt.cudaMallocManaged(ctypes.byref(p), ctypes.c_size_t(nbytes), ctypes.c_uint(1))
        if rc != 0 or not p.value:
            raise RuntimeError(f"cudaMallocManaged({nbytes}) failed: {rc}")
        self.ptr, self.nbytes = p.value, nbytes
        self._handle = ctypes.c_void_p(p.value)  # kept for __del__, which may run at shutdown

    def data_ptr(self) -> int:
        return self.ptr

    def free(self):
        if getattr(self, "ptr", None):
            torch.cuda.synchronize()
            self._rt.cudaFree(self._handle)
            self.ptr = None

    def __del__(self):
        try:
            self.free()
        except Exception:  # interpreter shutdown: the process exit releases the memory
            pass


class ServeRun:
    """The serving workload: a device value pool, request descriptors and Poisson arrival times,
    run through the persistent loop (gsync_serve_run) or one launch per request
    (gsync_serve_baseline).  Pinned host buffers carry the ring, results and flags."""

    def __init__(self, offset, length, sched_ns, pool: torch.Tensor, nslots: int = 32, nblocks: int = 304,
                 admitters: int = 8, chunk_elems: int = 32768, ring_slots: int = 65536, timeout_ns: int = 0,
                 drain_timeout_s: int = 30, ring: str = "host"):
        self.nreq = len(offset)
        self.offset = np.ascontiguousarray(offset, dtype=np.int64)
        self.length = np.ascontiguousarray(length, dtype=np.int64)
        self.sched = np.ascontiguousarray(sched_ns, dtype=np.int64)
        self.pool = pool
        self.cfg = G.gsync_serve_cfg(self.nreq, nslots, nblocks, admitters, chunk_elems, ring_slots, 2000,
                                     drain_timeout_s, timeout_ns)
        # ring="host": pinned host memory, polled by the admitters across the host link;
        # ring="device": managed memory that the loop places in device memory, written in place
        # by the host's producer thread
        if ring not in ("host", "device"):
            raise ValueError(ring)
        self.ring = (torch.zeros(ring_slots * 128, dtype=torch.uint8).pin_memory() if ring == "host"
                     else ManagedBuffer(ring_slots * 128))
        self.ctrl = torch.zeros(64, dtype=torch.int32).pin_memory()
        self.res = torch.zeros(self.nreq, dtype=torch.int64).pin_memory()
        self.done = torch.zeros(self.nreq, dtype=torch.int32).pin_memory()
        self.latency = np.zeros(self.nreq, dtype=np.int64)
        self.publish = np.zeros(self.nreq, dtype=np.int64)
        self.ws_bytes = G.gsync_serve_workspace_bytes(nslots)
        self.ws = torch.zeros(max(self.ws_bytes, 256), dtype=torch.uint8, device="cuda")
        self.bws_bytes = G.gsync_serve_baseline_workspace_bytes(self.nreq)
        self.bws = torch.zeros(self.bws_bytes, dtype=torch.uint8, device="cuda")
        self.trace = None

    def _buffers(self):
        return G.gsync_serve_buffers(G.ptr(self.pool), self.pool.numel(), self.offset.ctypes.data,
                                     self.length.ctypes.data,
                                     self.sched.ctypes.data, G.ptr(self.ring), G.ptr(self.ctrl), G.ptr(self.res),
                                     G.ptr(self.done), self.latency.ctypes.data, self.publish.ctypes.data,
                                     G.ptr(self.trace),
                                     (G.ctypes.c_uint32 * 4)())

    def _out(self, rc, buf, wall):
        return {"rc": rc, "res": self.res.numpy().copy(), "latency_ns": self.latency.copy(),
                "publish_delay_ns": self.publish - self.sched, "stats": list(buf.stats), "wall_s": wall}

    def enable_trace(self):
        self.trace = torch.zeros(4 * self.nreq, dtype=torch.int64, device="cuda")

    def trace_ns(self) -> np.ndarray:
        """[nreq, 4] globaltimer: entry seen, slot published, first chunk claimed, last chunk done."""
        torch.cuda.synchronize()
        return self.trace.cpu().numpy().reshape(self.nreq, 4)

    def run(self) -> dict:
        import time
        buf = self._buffers()
        t0 = time.perf_counter()
        rc = G.gsync_serve_run(self.cfg, buf, self.ws, self.ws_bytes)
        return self._out(rc, buf, time.perf_counter() - t0)

    def baseline(self, nstreams: int = 4) -> dict:
        import time
        streams = [torch.cuda.Stream() for _ in range(nstreams)]
        buf = self._buffers()
        t0 = time.perf_counter()
        rc = G.gsync_serve_baseline(self.cfg, buf, self.bws, self.bws_bytes, streams)
        return self._out(rc, buf, time.perf_counter() - t0)


def probe_host_pingpong(iters: int = 2000) -> dict:
    """One host <-> device hand-off through pinned host memory (release/acquire, system scope)."""
    words = torch.zeros(64, dtype=torch.int32).pin_memory()
    out = (G.ctypes.c_uint64 * 1)()
    G.check("gsync_probe_host_pingpong", G.gsync_probe_host_pingpong(words, iters, out))
    return {"handoff_ns": out[0] / (2 * iters)}
