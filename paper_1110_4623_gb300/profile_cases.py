"""Runs one named workload launch once, for capturing it under a profiler.

    python -m paper_1110_4623_gb300.profile_cases <case> [<case> ...]

Each case launches a single workload kernel at the bench's grid (1184 blocks) with fewer
operations per block than the bench, so that a multi-pass profiler capture stays short
(mutex_cluster_bench runs the bench's own three launches of the default kind, for one-pass
counters).
The result is checked against nothing; the parity tests do that.
"""
from __future__ import annotations

import sys

import torch

from . import gsync as G
from . import inputs, runner

NB = 1184


# Backoff as the bench runs each kind (ticket kinds: ns per waiter ahead, capped).
_BACKOFF = {"cas_backoff": (32, 2048), "cohort": (128, 4000), "cluster": (128, 4000)}


def _mutex(kind, K, acq=20):
    delay, add = inputs.mutex_inputs(NB, acq, inputs.mutex_seed(G.MUTEX_KINDS[kind], NB, K))
    bo = runner.backoff(min_ns=_BACKOFF[kind][0], max_ns=_BACKOFF[kind][1]) if kind in _BACKOFF else None
    r = runner.MutexRun(kind, NB, 256, acq, K, delay, add, bo=bo, timeout_ns=10_000_000_000, cluster=4)
    return lambda: G.check("gsync_bench_mutex", r.launch())


def _chain(launches):
    def run():
        for f in launches:
            f()
    return run


def _barrier(kind, param, rounds=200):
    r = runner.BarrierRun(kind, NB, 128, rounds, full=False, param=param, timeout_ns=10_000_000_000)
    return lambda: G.check("gsync_bench_barrier", r.launch())


def _sem(n, pairs=20, kind="ticket"):
    hold, add = inputs.sem_inputs(NB, pairs, inputs.SEED_SEM ^ (n << 16) ^ NB)
    r = runner.SemRun(kind, NB, 128, pairs, n, hold, add, bo=runner.backoff(min_ns=16, max_ns=2000),
                      timeout_ns=10_000_000_000)
    return lambda: G.check("gsync_bench_sem", r.launch())


def _batched(nacq=200_000, rounds=20, policy=None):
    from . import autotune
    keys, adds, _ = inputs.batched_inputs(nacq, 4096, 1.1)
    cls = autotune.classify_keys(keys, 4096, NB)
    r = autotune.make_run(keys, adds, 4096, NB, 64, rounds, 1, cls)
    r.set_policy(policy or autotune.DEFAULT_POLICY)
    return lambda: G.check("gsync_bench_batched", r.launch())


def _condvar(mutex="cohort", items=20):
    v = inputs.condvar_inputs(592 * items)
    r = runner.CondVarRun(592, 592, items, 16, v, bo=runner.backoff(min_ns=128, max_ns=4000), mutex=mutex)
    return lambda: G.check("gsync_bench_condvar", r.launch())


CASES = {
    "mutex_sleep_queue": lambda: _mutex("sleep_queue", 64),
    "mutex_ticket": lambda: _mutex("ticket", 64),
    "mutex_cas_spin": lambda: _mutex("cas_spin", 64),
    "mutex_cas_backoff": lambda: _mutex("cas_backoff", 64),
    "mutex_cohort": lambda: _mutex("cohort", 64),
    "mutex_cluster": lambda: _mutex("cluster", 64),
    # the bench step's launches of the default kind, at full size: CS 0, 64 and 1024 words,
    # 100 acquisitions per block (for per-launch DRAM traffic without scaling)
    "mutex_cluster_bench": lambda: _chain([_mutex("cluster", K, acq=100) for K in (0, 64, 1024)]),
    "barrier_atomic": lambda: _barrier("atomic", 0),
    "barrier_flag": lambda: _barrier("flag", 0),
    "barrier_cluster2": lambda: _barrier("cluster", 2),
    "barrier_count8": lambda: _barrier("count", 8),
    "sem_ticket_n4": lambda: _sem(4),
    "sem_window_n4": lambda: _sem(4, kind="window"),
    "batched_200k": lambda: _batched(),
    "batched_200k_carry": lambda: _batched(policy=[("ticket_carry", 0, 0), ("ticket_carry", 64, 2000),
                                                   ("cas_spin", 0, 0)]),
    "condvar_cohort": lambda: _condvar(),
}


def main(argv):
    if not argv or any(a not in CASES for a in argv):
        print(f"usage: python -m paper_1110_4623_gb300.profile_cases {{{','.join(CASES)}}} ...")
        return 2
    torch.cuda.set_device(0)
    launches = [CASES[a]() for a in argv]
    for f in launches:
        f()
    torch.cuda.synchronize()
    return 0


if __name__ == "__main__":
    raise SystemExit(main(sys.argv[1:]))
