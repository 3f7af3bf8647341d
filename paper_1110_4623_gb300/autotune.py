"""Autotuner for the batched many-mutex kernel (Section 7 names autotuning the backoff
variables per GPU and contention level as future work).

Keys are put in contention classes by their share of the acquisition stream: a key is *hot*
when it expects at least one waiter per hand-off (count >= acquisitions / blocks), *warm*
when it expects one sixteenth of that, *cold* otherwise.  For each class in turn (hot first,
since it bounds the makespan), the tuner times every candidate policy -- mutex kind, backoff
constants, spinning (min_ns = 0) or __nanosleep -- with the other classes fixed, keeps the
fastest, and then picks the cluster size of the barrier groups; with clusters, it last tries
the cluster cohort lock for the hot and warm classes.  Every trial is one real
launch of the batched kernel through the C ABI, timed with CUDA events on the launching
stream; results are verified against nothing here (the parity tests do that).
"""
from __future__ import annotations

import numpy as np
import torch

from . import inputs as I
from . import runner

HOT, WARM, COLD = 0, 1, 2
NCLASSES = 3

# (kind, min_ns, max_ns): min_ns = 0 means spin without sleeping.  ticket_carry is the ticket
# lock whose turn record carries the key's count and sum through each hand-off; cohort_carry
# the two-die cohort lock with carrying records (the hottest keys only, the rest of the class
# on ticket_carry).
CANDIDATES = [
    ("cas_spin", 0, 0),
    ("cas_backoff", 32, 1024),
    ("cas_backoff", 128, 4096),
    ("ticket", 0, 0),
    ("ticket", 64, 2000),
    ("ticket", 256, 4000),
    ("ticket_carry", 0, 0),
    ("ticket_carry", 8, 2000),
    ("ticket_carry", 64, 2000),
    ("cohort_carry", 0, 0),
]
CLUSTERS = [1, 2, 4, 8]
# Tried last, for the hot and warm classes, once a cluster size above 1 is chosen: the cluster
# cohort lock and the carrying locks over clusters (keys below 256) need a cluster launch.
CLUSTER_CANDIDATES = [("cluster", 128, 4000), ("cluster_carry", 0, 0), ("cluster_die_carry", 0, 0)]
DEFAULT_POLICY = [("ticket", 0, 0)] * NCLASSES


def classify_keys(keys: np.ndarray, nkeys: int, nblocks: int) -> np.ndarray:
    counts = np.bincount(np.asarray(keys, dtype=np.int64), minlength=nkeys)
    per_block = len(keys) / nblocks
    cls = np.full(nkeys, COLD, dtype=np.uint8)
    cls[counts >= per_block / 16.0] = WARM
    cls[counts >= per_block] = HOT
    return cls


def _time(run: runner.BatchedRun, reps: int = 2) -> float:
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(reps):
        run.reset()
        s.record()
        rc = run.launch()
        e.record()
        torch.cuda.synchronize()
        if rc != 0 or run.results()["status"] != 0:
            return float("inf")
        ts.append(s.elapsed_time(e))
    return float(np.median(ts))


def make_run(keys, adds, nkeys, nblocks, ngroups, rounds, cluster, key_class, block_threads=128, seed=I.SEED_BATCHED,
             plain_launch=False, ncohort=128):
    _, sizes = I.barrier_group_sizes(ngroups, 2, 256, nblocks, seed=seed, multiple=cluster)
    return runner.BatchedRun(keys, adds, nkeys, nblocks, sizes, rounds, key_class, NCLASSES,
                             block_threads=block_threads, cluster=cluster, plain_launch=plain_launch, ncohort=ncohort)


def tune(keys, adds, nkeys: int, nblocks: int, ngroups: int, rounds: int, block_threads: int = 128,
         reps: int = 2) -> dict:
    """Coordinate descent over the classes' policies, then over the group cluster size, then,
    at every cluster size above 1, over the cluster-only kinds for the hot and warm classes;
    the fastest combination wins."""
    key_class = classify_keys(keys, nkeys, nblocks)
    policy = list(DEFAULT_POLICY)
    trials = []
    run = make_run(keys, adds, nkeys, nblocks, ngroups, rounds, 1, key_class, block_threads)
    for cls in (HOT, WARM, COLD):
        best = None
        for cand in CANDIDATES:
            trial = list(policy)
            trial[cls] = cand
            run.set_policy(trial)
            ms = _time(run, reps)
            trials.append({"class": cls, "policy": cand, "cluster": 1, "ms": ms})
            if best is None or ms < best[0]:
                best = (ms, cand)
        policy[cls] = best[1]
    best_cluster = (None, 1)
    for c in CLUSTERS:
        r = run if c == 1 else make_run(keys, adds, nkeys, nblocks, ngroups, rounds, c, key_class, block_threads)
        r.set_policy(policy)
        ms = _time(r, reps)
        trials.append({"class": None, "policy": None, "cluster": c, "ms": ms})
        if best_cluster[0] is None or ms < best_cluster[0]:
            best_cluster = (ms, c)
    # The cluster-only kinds (the cluster cohort lock, the carrying locks over clusters) depend
    # on the cluster size as much as the group barriers do: try them at every size above 1.
    best = (best_cluster[0], best_cluster[1], list(policy))
    for c in CLUSTERS:
        if c == 1:
            continue
        r = make_run(keys, adds, nkeys, nblocks, ngroups, rounds, c, key_class, block_threads)
        pol_c = list(policy)
        ms_c = next(t["ms"] for t in trials if t["class"] is None and t["cluster"] == c)
        for cls in (HOT, WARM):
            for cand in CLUSTER_CANDIDATES:
                trial = list(pol_c)
                trial[cls] = cand
                r.set_policy(trial)
                ms = _time(r, reps)
                trials.append({"class": cls, "policy": cand, "cluster": c, "ms": ms})
                if ms < ms_c:
                    ms_c, pol_c = ms, trial
        if ms_c < best[0]:
            best = (ms_c, c, pol_c)
    best_cluster, policy = (best[0], best[1]), best[2]
    return {"policy": policy, "cluster": best_cluster[1], "best_ms": best_cluster[0],
            "class_sizes": [int((key_class == c).sum()) for c in range(NCLASSES)], "trials": trials,
            "key_class": key_class}
