"""ctypes binding of cpu_exec.c, the threaded CPU execution of the workloads.

ORACLE -- TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg of the benchmark).
`build()` compiles cpu_exec.c with the host C compiler into oracle/_build/.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cpu_exec.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle_cpu.so")

MUTEX_KINDS = {"cas_spin": 0, "cas_backoff": 1, "ticket": 2, "sleep_queue": 3}
SEM_KINDS = {"ticket": 0, "spin": 1, "spin_backoff": 2}
BARRIER_KINDS = {"atomic": 0, "flag": 1}

_lib = None


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    stamp = os.path.join(OUT_DIR, "HOST_ARCH")
    arch = platform.machine()
    if not os.path.exists(stamp) or open(stamp).read().strip() != arch:
        force = True
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               "-Wall", "-o", tmp, SRC])
        os.replace(tmp, LIB)
        with open(stamp, "w") as f:
            f.write(arch + "\n")
    return LIB


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        u32p = ctypes.POINTER(ctypes.c_uint32)
        dp = ctypes.POINTER(ctypes.c_double)
        i = ctypes.c_int
        _lib.oracle_mutex_run.argtypes = [i, i, i, i, i, u32p, u32p, u32p, u32p, u32p, u32p, u32p, dp]
        _lib.oracle_sem_run.argtypes = [i, i, i, i, i, u32p, u32p, u32p, u32p, u32p, u32p, dp]
        _lib.oracle_barrier_run.argtypes = [i, i, i, i, u32p, u32p, u32p, dp]
        for f in (_lib.oracle_mutex_run, _lib.oracle_sem_run, _lib.oracle_barrier_run):
            f.restype = ctypes.c_int
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.uint32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def default_threads() -> int:
    return os.cpu_count() or 1


def mutex_run(kind: str, nblocks: int, acq: int, cs_words: int, addend, delay=None,
              nthreads: int | None = None) -> dict:
    lib = _load()
    nthreads = min(nthreads or default_threads(), nblocks)
    n = nblocks * acq
    addend = np.ascontiguousarray(addend, dtype=np.uint32)
    delay = None if delay is None else np.ascontiguousarray(delay, dtype=np.uint32)
    data = np.zeros(max(cs_words, 1), dtype=np.uint32)
    total = np.zeros(1, dtype=np.uint32)
    log = np.zeros(max(n, 1), dtype=np.uint32)
    ticket = np.zeros(max(n, 1), dtype=np.uint32)
    count = np.zeros(nblocks, dtype=np.uint32)
    sec = ctypes.c_double(0.0)
    rc = lib.oracle_mutex_run(MUTEX_KINDS[kind], nblocks, acq, cs_words, nthreads, _p(addend),
                              _p(delay), _p(data), _p(total), _p(log), _p(ticket), _p(count),
                              ctypes.byref(sec))
    if rc:
        raise RuntimeError(f"oracle_mutex_run failed with {rc}")
    return {"data": data[:cs_words], "total": total[0], "log": log[:n], "ticket": ticket[:n],
            "count": count, "seconds": sec.value, "threads": nthreads}


def sem_run(kind: str, nblocks: int, pairs: int, n_init: int, addend, hold=None,
            nthreads: int | None = None) -> dict:
    lib = _load()
    nthreads = min(nthreads or default_threads(), nblocks)
    addend = np.ascontiguousarray(addend, dtype=np.uint32)
    hold = None if hold is None else np.ascontiguousarray(hold, dtype=np.uint32)
    count = np.zeros(nblocks, dtype=np.uint32)
    total = np.zeros(1, dtype=np.uint32)
    tally = np.zeros(1, dtype=np.uint32)
    max_occ = np.zeros(1, dtype=np.uint32)
    sec = ctypes.c_double(0.0)
    rc = lib.oracle_sem_run(SEM_KINDS[kind], nblocks, pairs, n_init, nthreads, _p(hold),
                            _p(addend), _p(count), _p(total), _p(tally), _p(max_occ),
                            ctypes.byref(sec))
    if rc:
        raise RuntimeError(f"oracle_sem_run failed with {rc}")
    return {"count": count, "total": total[0], "tally": tally[0], "max_occ": int(max_occ[0]),
            "seconds": sec.value, "threads": nthreads}


def barrier_run(kind: str, nblocks: int, rounds: int, full: bool) -> dict:
    lib = _load()
    chk = np.zeros(max(rounds * nblocks, 1), dtype=np.uint32) if full else None
    mix = np.zeros(nblocks, dtype=np.uint32)
    bad = np.zeros(nblocks, dtype=np.uint32)
    sec = ctypes.c_double(0.0)
    rc = lib.oracle_barrier_run(BARRIER_KINDS[kind], nblocks, rounds, int(full), _p(chk),
                                _p(mix), _p(bad), ctypes.byref(sec))
    if rc:
        raise RuntimeError(f"oracle_barrier_run failed with {rc}")
    out = {"mix": mix, "bad": bad, "seconds": sec.value, "threads": nblocks}
    if full:
        out["chk"] = chk[:rounds * nblocks].reshape(rounds, nblocks)
    return out
