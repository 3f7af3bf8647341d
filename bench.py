"""Benchmark of the inter-block synchronization hot path on GB300.

One step = one pass over every row of the hot path at 1184 blocks:
  * mutex contention (the paper's 4 kinds, its ring-buffer mutex and spin-then-sleep policy,
    and the two cohort locks x critical sections of 0/64/1024 words, 256 threads per block,
    100 acquisitions per block, seeded delays U{0..2000} cycles),
  * grid barriers (atomic, flag, tree and its counting form, cluster 2/4/8 and its counting form,
    sharded, two-die, split, counting; 128 threads, 1000 rounds each),
  * counting semaphores (sleeping FA kind, n in {1, 4, 16, 64}; 128 threads, 200 pairs each,
    hold U{100..5000} cycles).
`value` is lock acquisitions per second of the library's default mutex kind over its three
critical-section sizes; the other rows are reported beside it (barrier ns per crossing,
semaphore ops/s), each against a roofline whose terms (SM-to-SM hand-off latency,
critical-section time, same-word atomic throughput, atomic round trip) the probe kernels
measure in the same run.  After the timed steps, the batched many-mutex workload (4096 Zipf
keys, 1e6 acquisitions, 64 barrier groups) is autotuned and replayed from a CUDA graph.
`--impl reference` times the CPU oracle (threaded C execution of the same mutex workload on
the host cores).  Under torchrun every rank runs the same workload on its own GPU (replicas).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NBLOCKS = 1184
MUTEX_THREADS, MUTEX_ACQ, CS_SIZES = 256, 100, (0, 64, 1024)
BAR_THREADS, BAR_ROUNDS = 128, 1000
SEM_THREADS, SEM_PAIRS, SEM_COUNTS = 128, 200, (1, 4, 16, 64)
# Library defaults for GB300, chosen from 1184-block sweeps (the paper's API serves the
# fastest implementation of each primitive for the GPU as the default, Section 5 "API").
DEFAULT_MUTEX = "cluster_mcs"
DEFAULT_BARRIER = ("count", 8)
# cluster params: c | form << 4 (form 0: atomic stage over the leaders; 2: counting stage, the
# rest of the cluster released by a second cluster barrier -- the fastest cluster form measured)
# tree params: fan | form << 16 (form 1: counting tree, node counters that only grow)
BARRIERS = [("atomic", 0), ("flag", 0), ("flag", 1), ("tree", 8), ("tree", 8 | 1 << 16), ("tree", 64 | 1 << 16),
            ("cluster", 2), ("cluster", 4), ("cluster", 8),
            ("cluster", 4 | 2 << 4), ("cluster", 8 | 2 << 4), ("sharded", 32), ("sharded", 8), ("die", 0),
            ("die", 1), ("split", 16 | 16 << 8), ("count", 0), ("count", 8), ("exchange", 8)]
# Backoff (min_ns, max_ns) per kind; the ticket kinds sleep min_ns per waiter ahead, capped.
MUTEX_BACKOFF = {"cas_backoff": (16, 512), "ticket": (128, 4000), "cohort": (128, 4000), "cluster": (128, 4000),
                 "cluster_mcs": (128, 4000)}
# Blocks per cluster of the cluster cohort locks (sweeps of 2 / 4 / 8 picked 4 for the ticket
# form and 8 for the MCS form).
MUTEX_CLUSTERS = {"cluster": 4, "cluster_mcs": 8}


def mutex_cluster(kind):
    return MUTEX_CLUSTERS.get(kind, 0)



# The measured mutex configurations: (name, kind, backoff policy, (min_ns, max_ns), spin).
# cas_spin_then_sleep is Section 5's futex stand-in: the CAS lock spins, then backs off.
MUTEX_CONFIGS = [("cas_spin", "cas_spin", 0, None, 0), ("cas_backoff", "cas_backoff", 0, (16, 512), 0),
                 ("cas_spin_then_sleep", "cas_backoff", 2, (16, 512), 32), ("ticket", "ticket", 0, (128, 4000), 0),
                 ("sleep_queue", "sleep_queue", 0, None, 0), ("ring", "ring", 0, None, 0),
                 ("cohort", "cohort", 0, (128, 4000), 0), ("cluster", "cluster", 0, (128, 4000), 0),
                 ("cluster_mcs", "cluster_mcs", 0, (128, 4000), 0)]
SEM_BACKOFF = (16, 2000)
SEM_STEP_KINDS = ("window", "ticket")  # the library's default (the ticket window), then the paper's FA semaphore
DEFAULT_SEM = "window"
# Batched many-mutex workload: 4096 keys, Zipf(1.1), 1e6 acquisitions, 64 barrier groups.
BATCH_KEYS, BATCH_ACQ, BATCH_GROUPS, BATCH_ROUNDS, BATCH_THREADS = 4096, 1_000_000, 64, 100, 128
METRIC = "lock acquires/s & barrier ns at 1184 blocks vs L2-atomic roofline; p99 latency"
# DRAM bytes per launch of the default mutex kind's workload kernel from an ncu capture, or
# None while the kernel has changed since the last capture.
ROOF_TRAFFIC = 1_676_459
ROOF_TRAFFIC_NOTE = ("DRAM bytes (read + write) per launch of the dominant kernel (the MCS cluster cohort mutex "
                     "workload, clusters of 8), mean over the step's three launches (CS 0/64/1024: 1.73/2.10/1.20 MB), "
                     "one-pass ncu capture of the same launches in profiles/; algorithmic bytes 1.89 MB "
                     "(16 B per acquisition)")
TIMEOUT_NS = 10_000_000_000


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gsync", choices=["gsync", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-batched", action="store_true", help="skip the batched and serving sections")
    p.add_argument("--no-sweep", action="store_true", help="skip the grid-size sweep (148..1184 blocks)")
    p.add_argument("--jsonl", default=None, help="also append one JSON row per measured configuration to this file")
    return p.parse_args()


def result_rows(out):
    """The bench line flattened into one row per measured configuration (section, kind, grid,
    parameter): rate or time, roofline and its fraction, latency percentiles."""
    grid = out["config"].get("nblocks")
    rows = []
    for kind, per_cs in out.get("mutex", {}).items():
        for cs, r in per_cs.items():
            rows.append({"section": "mutex", "kind": kind, "nblocks": grid, "cs_words": int(cs),
                         "acq_per_s": r["acq_per_s"], "roof_acq_per_s": r["roof_acq_per_s"], "frac": r["frac"]})
    for kind, r in out.get("barrier", {}).get("kinds", {}).items():
        rows.append({"section": "barrier", "kind": kind, "nblocks": grid, "ns_per_crossing": r["ns_per_crossing"],
                     "roof_ns": r["roof_ns"], "frac": r["frac"]})
    for kind, per_n in out.get("semaphore", {}).get("kinds", {}).items():
        for n, r in per_n.items():
            rows.append({"section": "semaphore", "kind": kind, "nblocks": grid, "n": int(n),
                         "ops_per_s": r["ops_per_s"], "roof_ops_per_s": r["roof_ops_per_s"], "frac": r["frac"]})
    for kind, r in out.get("condvar", {}).get("mutex", {}).items():
        rows.append({"section": "condvar", "kind": kind, "items_per_s": r["items_per_s"], "frac": r["frac"]})
    for arm in ("default", "tuned"):
        r = out.get("batched", {}).get(arm)
        if r:
            rows.append({"section": "batched", "kind": arm, "acq_per_s": r["acq_per_s"], "frac": r.get("frac"),
                         "cluster": r["cluster"]})
    for rate, r in out.get("serving", {}).get("rates", {}).items():
        for arm in ("persistent", "persistent_device_ring", "per_request_launch"):
            if arm not in r:
                continue
            a = r[arm]
            rows.append({"section": "serving", "kind": arm, "offered_req_s": float(rate),
                         "achieved_req_s": a["achieved_req_s"], "p50_us": a["p50_us"], "p99_us": a["p99_us"]})
    sw = out.get("sweep", {})
    for kind, per_cs in sw.get("mutex_acq_per_s", {}).items():
        for cs, per_b in per_cs.items():
            for B, v in per_b.items():
                rows.append({"section": "sweep_mutex", "kind": kind, "cs_words": int(cs), "nblocks": int(B), "acq_per_s": v})
    for kind, per_b in sw.get("barrier_ns_per_crossing", {}).items():
        for B, v in per_b.items():
            rows.append({"section": "sweep_barrier", "kind": kind, "nblocks": int(B), "ns_per_crossing": v})
    for kind, per_n in sw.get("semaphore_ops_per_s", {}).items():
        for n, per_b in per_n.items():
            for B, v in per_b.items():
                rows.append({"section": "sweep_semaphore", "kind": kind, "n": int(n), "nblocks": int(B), "ops_per_s": v})
    stamp = {"clocks_sm_mhz": out.get("clocks", {}).get("sm_mhz"), "n_gpus": out.get("n_gpus")}
    return [dict(row, **stamp) for row in rows]


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(vals, world, device="cuda"):
    """Elementwise maximum of a list of floats over all ranks of the default process group
    (the identity for a single process)."""
    vals = [float(v) for v in vals]
    if world == 1:
        return vals
    import torch
    import torch.distributed as dist
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def replica_value(units_per_rank, ms_max, world):
    """Whole-job throughput of `world` independent replicas: every rank processes
    `units_per_rank`, and the job takes as long as its slowest rank."""
    return units_per_rank * world / (ms_max * 1e-3)


def br_param(kind, param):
    """The parameter a BarrierRun of this kind actually uses (its defaults for 0)."""
    if kind == "tree" and param == 0:
        return 8
    if kind == "cluster" and param == 0:
        return 2
    if kind == "sharded" and param == 0:
        return min(32, NBLOCKS)
    if kind == "split" and param == 0:
        return 8 | 8 << 8
    return param


def barrier_name(kind, param):
    if kind == "flag":
        return "flag_broadcast" if param else "flag"
    if kind == "cluster":
        c, form, sleep = param & 0xF, (param >> 4) & 0xF, param >> 8
        name = f"cluster{c}" + ("", "_count", "_count_cb")[form]
        return name + (f"_s{sleep}" if sleep else "")
    if kind == "tree":
        return f"tree{param & 0xFFFF}" + ("_count" if param >> 16 else "")
    if kind == "sharded" or (kind in ("count", "exchange") and param):
        return f"{kind}{param}"
    if kind == "split":
        return f"split{param & 0xFF}x{param >> 8}"
    if kind == "die":
        return "die_flat" if param else "die"
    return kind


# ------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------
# roofline terms (probe kernels)
# ------------------------------------------------------------------------------------------

PROBE_PAGES = 8  # 4 KB placements tried for each critical-section probe


def best_placement(probe, nbytes, runner):
    """The critical-section probes run one block, whose L2 accesses cost ~150 ns on lines
    homed on its own die and ~350 ns on the other's (line homes alternate between the dies in
    4 KB pages).  A fresh buffer lands on either, which moved T_cs and T_frame by ~200 ns
    from run to run.  The probe's hot lines sit at the start of its scratch, so running it at
    PROBE_PAGES successive 4 KB offsets of one buffer and keeping the fastest gives the
    near-die body on every run: the stricter bound, and a stable one."""
    buf = runner._state(nbytes + PROBE_PAGES * 4096)
    return float(min(probe(buf.data_ptr() + i * 4096) for i in range(PROBE_PAGES)))


def measure_roofline_terms(runner, inputs):
    """L_handoff, T_cs(K), T_cs_sem(n), R_same and L_rt from the probe kernels (medians)."""
    sms = runner.sm_count()
    # The bound is the shortest hand-off the machine offers: two SMs of one die, on lines homed
    # on that die.  Five fixed pairs on lines homed wherever are reported beside it.
    near = [runner.near_handoff(4000) for _ in range(3)]
    near_ns = [h["handoff_ns"] for h in near if h["status"] == 0]
    # the same pair with no fence on either side (a relaxed store seen by relaxed polls): the
    # hand-off of the carrying locks, whose guarded data travel in the flag's own access
    relaxed = [runner.near_handoff_relaxed(4000) for _ in range(3)]
    relaxed_ns = [h["handoff_ns"] for h in relaxed if h["status"] == 0]
    # ... or inside a thread-block cluster, through distributed shared memory
    dsm = [runner.probe_cluster(1, 2, 4000) for _ in range(3)]
    dsm_ns = [h["ns"] for h in dsm if h["status"] == 0]
    # ... and with no fence: a relaxed 16-byte record in the peer's shared memory (the hand-off
    # of the carrying lock over clusters)
    dsm_rx = [runner.probe_cluster(3, 2, 4000) for _ in range(3)]
    dsm_rx_ns = [h["ns"] for h in dsm_rx if h["status"] == 0]
    pairs = [(0, 1), (0, sms // 2), (0, sms - 1), (sms // 4, 3 * sms // 4), (2, sms - 3)]
    hand = [runner.probe_pingpong(a, b, 4000) for a, b in pairs if a != b and 0 <= a < sms and 0 <= b < sms]
    hand_ns = [h["handoff_ns"] for h in hand if h["status"] == 0]
    T_cs = {K: best_placement(lambda a, K=K: runner.probe_cs(K, MUTEX_THREADS, 20000, scratch=a)["ns_per_cs"],
                              runner.G.gsync_probe_cs_scratch_bytes(K, 20000), runner)
            for K in CS_SIZES}
    # the hardware cluster barrier, per crossing, for the cluster sizes the cluster barrier uses
    T_cb = {c: float(np.median([runner.probe_cluster(0, c, 4000)["ns"] for _ in range(3)])) for c in (2, 4, 8)}
    rs = [runner.probe_throughput("red_add", True, False, NBLOCKS, 128, 2000)["ops_per_s"] for _ in range(3)]
    ra = [runner.probe_throughput("atomic_read", True, False, NBLOCKS, 128, 1000)["ops_per_s"] for _ in range(3)]
    # dependent chains of one thread: atomic round trip and L2 load, on a line homed on the
    # probe's own die (a fresh buffer lands on either die: ~190 or ~390 ns for the atomic)
    L_rt = best_placement(lambda a: runner.probe_latency("atomic_read", 4000, scratch=a)["ns_per_op"], 256, runner)
    L_ld = best_placement(lambda a: runner.probe_latency("load_relaxed", 4000, scratch=a)["ns_per_op"], 256, runner)
    T_cs_sem = {}
    for n in SEM_COUNTS:
        hold, add = inputs.sem_inputs(NBLOCKS, SEM_PAIRS, inputs.SEED_SEM ^ (n << 16) ^ NBLOCKS)
        T_cs_sem[n] = best_placement(
            lambda a: runner.probe_sem_cs(hold[:4000], add[:4000], SEM_THREADS, scratch=a)["ns_per_cs"], 1024, runner)
    # The probes' frame (acquire load, barriers, release) is what a hand-off already costs:
    # subtract it so that hand-off + body does not count it twice.
    T_frame = best_placement(lambda a: runner.probe_cs(-1, MUTEX_THREADS, 20000, scratch=a)["ns_per_cs"],
                             runner.G.gsync_probe_cs_scratch_bytes(-1, 20000), runner)
    T_frame_sem = best_placement(
        lambda a: runner.probe_sem_cs(None, None, SEM_THREADS, iters=4000, scratch=a)["ns_per_cs"], 1024, runner)
    return {"sms": sms, "L_handoff_ns": float(min(np.median(near_ns), np.median(dsm_ns))),
            "L_handoff_l2_near_ns": float(np.median(near_ns)), "L_handoff_dsmem_ns": float(np.median(dsm_ns)),
            "L_handoff_relaxed_near_ns": float(np.median(relaxed_ns)),
            "L_handoff_relaxed_dsmem_ns": float(np.median(dsm_rx_ns)),
            "L_handoff_pairs_ns": hand_ns, "T_cs_ns": T_cs,
            "T_frame_ns": T_frame, "T_cs_sem_ns": T_cs_sem, "T_frame_sem_ns": T_frame_sem,
            "R_same_red_ops_s": float(np.median(rs)), "R_same_atom_ops_s": float(np.median(ra)), "L_rt_ns": L_rt,
            "L_ld_ns": L_ld, "T_cluster_bar_ns": T_cb}


def merge_terms(a, b):
    """The stricter roof of two measurements: lower latencies, higher throughputs."""
    out = dict(a)
    for k in ("L_handoff_ns", "L_handoff_l2_near_ns", "L_handoff_dsmem_ns", "L_handoff_relaxed_near_ns",
              "L_handoff_relaxed_dsmem_ns", "L_rt_ns",
              "L_ld_ns"):
        out[k] = min(a[k], b[k])
    for k in ("R_same_red_ops_s", "R_same_atom_ops_s"):
        out[k] = max(a[k], b[k])
    out["T_cs_ns"] = {K: min(a["T_cs_ns"][K], b["T_cs_ns"][K]) for K in a["T_cs_ns"]}
    out["T_cluster_bar_ns"] = {c: min(a["T_cluster_bar_ns"][c], b["T_cluster_bar_ns"][c]) for c in a["T_cluster_bar_ns"]}
    out["T_cs_sem_ns"] = {n: min(a["T_cs_sem_ns"][n], b["T_cs_sem_ns"][n]) for n in a["T_cs_sem_ns"]}
    # body = probe - frame, taken from the same measurement, then the smaller of the two
    out["T_body_ns"] = {K: min(a["T_cs_ns"][K] - a["T_frame_ns"], b["T_cs_ns"][K] - b["T_frame_ns"])
                        for K in a["T_cs_ns"]}
    out["T_body_sem_ns"] = {n: min(a["T_cs_sem_ns"][n] - a["T_frame_sem_ns"], b["T_cs_sem_ns"][n] - b["T_frame_sem_ns"])
                            for n in a["T_cs_sem_ns"]}
    out["before_after"] = {"before": {k: a[k] for k in ("L_handoff_ns", "T_cs_ns", "T_cs_sem_ns")},
                           "after": {k: b[k] for k in ("L_handoff_ns", "T_cs_ns", "T_cs_sem_ns")}}
    return out


def mutex_roof_acq_s(terms, K):
    """A perfect lock still pays one SM-to-SM hand-off (release, transit, observation) plus the
    critical-section body per acquisition, and two lock-word operations at the atomic unit."""
    return min(terms["R_same_atom_ops_s"] / 2.0, 1e9 / (terms["L_handoff_ns"] + max(terms["T_body_ns"][K], 0.0)))


def sem_roof_ops_s(terms, n):
    """Under capacity a wait is one atomic; at capacity n holders each hand off per op."""
    return min(terms["R_same_atom_ops_s"],
               n * 1e9 / (terms["L_handoff_l2_near_ns"] + max(terms["T_body_sem_ns"][n], 0.0)))


def tree_levels(B, fan):
    """Levels of a combining tree of fan-in `fan` over B leaves (1 for B <= fan)."""
    levels, width = 1, -(-B // fan)
    while width > 1:
        width = -(-width // fan)
        levels += 1
    return levels


def barrier_roof_ns(terms, kind, param, B):
    """The serial steps of one crossing, each at its measured cost, plus the workload's own
    share of a round: the partner slot each block reads after a crossing is a dependent L2 load
    (L_ld) on the critical path to its next arrival.  A grid-wide release reaches every block
    through L2, so the on-die L2 hand-off (L_h) bounds it; same-word arrivals serialize at the
    atomic unit (R_same).
      atomic : last arrival's round trip, B serialized arrivals, release hand-off
      count  : B serialized arrivals, whose last is the release (no round trip back)
      tree   : per level a round trip of the last arriver and fan serialized arrivals, then
               the root's release hand-off (counting form: no round trip at the root)
      flag   : (XF) two hand-offs in series -- the last arrival flag to the master block, the
               release flags to every block -- plus the master's second gather pass (a thread
               watches two or three of the 16-byte flag vectors, so some need two loads)
      sharded: two hand-offs in series (counters to the master warp, release flags to every
               block) and B/S serialized arrivals per counter
      cluster: the hardware cluster barrier (T_cb(c), measured), then over the B/c leaders:
               form 0 as atomic; form 1 as count; form 2 as count plus a second cluster barrier
      die    : B/2 arrivals per die, and with per-die counters one more round trip (the top)
      split  : B/S per counter plus S at the top, two round trips (S > 1)
      exchange: as count, but the arrival has no fence and the pollers' loads are relaxed, so
               the hand-off is the fence-free one (L_handoff_relaxed_near); the partner value
               is one load of its record (L_ld)"""
    L_rt, L_h, L_ld = terms["L_rt_ns"], terms["L_handoff_l2_near_ns"], terms.get("L_ld_ns", 0.0)
    t_atom = 1e9 / terms["R_same_atom_ops_s"]
    if kind == "atomic":
        ns = L_rt + B * t_atom + L_h
    elif kind == "count":
        ns = B * t_atom + L_h
    elif kind == "exchange":
        ns = B * t_atom + terms.get("L_handoff_relaxed_near_ns", L_h)
    elif kind == "tree":
        fan, form = param & 0xFFFF, param >> 16
        lv = tree_levels(B, fan)
        # form 1: the root's completing add is the release (no round trip back at the top)
        ns = (lv - form) * L_rt + lv * fan * t_atom + L_h
    elif kind == "flag":
        ns = 2 * L_h + L_ld
    elif kind == "sharded":
        ns = 2 * L_h + -(-B // param) * t_atom
    elif kind == "cluster":
        c, form = param & 0xF, (param >> 4) & 0xF
        t_cb = terms.get("T_cluster_bar_ns", {}).get(c, 0.0)
        leaders = B / c
        if form == 0:
            ns = t_cb + L_rt + leaders * t_atom + L_h
        else:
            ns = t_cb + leaders * t_atom + L_h + (t_cb if form == 2 else 0.0)
    elif kind == "die":
        ns = (L_rt + B * t_atom + L_h) if param == 1 else (2 * L_rt + B / 2 * t_atom + L_h)
    elif kind == "split":
        S = param & 0xFF
        ns = (2 * L_rt + (-(-B // S) + S) * t_atom + L_h) if S > 1 else (L_rt + B * t_atom + L_h)
    else:
        raise ValueError(kind)
    return ns + L_ld


# ------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------

class GpuStep:
    """All buffers of one step, allocated once; launch() enqueues the whole step."""

    def __init__(self, runner, G, inputs):
        import torch
        self.mutex = {}
        for name, kind, policy, bo_ns, spin in MUTEX_CONFIGS:
            for K in CS_SIZES:
                delay, add = inputs.mutex_inputs(NBLOCKS, MUTEX_ACQ, inputs.mutex_seed(G.MUTEX_KINDS[kind], NBLOCKS, K))
                bo = runner.backoff(policy=policy, min_ns=bo_ns[0], max_ns=bo_ns[1], spin=spin) if bo_ns else None
                self.mutex[(name, K)] = (runner.MutexRun(kind, NBLOCKS, MUTEX_THREADS, MUTEX_ACQ, K, delay, add, bo=bo,
                                                         timeout_ns=TIMEOUT_NS, cluster=mutex_cluster(kind)), add)
        self.barrier = {(k, p): runner.BarrierRun(k, NBLOCKS, BAR_THREADS, BAR_ROUNDS, full=False, param=p,
                                                  timeout_ns=TIMEOUT_NS) for k, p in BARRIERS}
        self.sem = {}
        for kind in SEM_STEP_KINDS:
            for n in SEM_COUNTS:
                hold, add = inputs.sem_inputs(NBLOCKS, SEM_PAIRS, inputs.SEED_SEM ^ (n << 16) ^ NBLOCKS)
                bo = runner.backoff(min_ns=SEM_BACKOFF[0], max_ns=SEM_BACKOFF[1])
                self.sem[(kind, n)] = (runner.SemRun(kind, NBLOCKS, SEM_THREADS, SEM_PAIRS, n, hold, add, bo=bo,
                                                     timeout_ns=TIMEOUT_NS), add)
        ev = lambda: torch.cuda.Event(enable_timing=True)
        self.ev = {key: (ev(), ev()) for key in list(self.mutex) + list(self.barrier) + [("sem",) + k for k in self.sem]}
        self.launches = 0

    def launch(self):
        """Enqueues one step; per-launch events on the launching (current) stream."""
        launches = 0
        for key, (mr, _) in self.mutex.items():
            mr.reset()
            a, b = self.ev[key]
            a.record()
            rc = mr.launch()
            b.record()
            assert rc == 0, (key, rc)
            launches += 1
        for key, br in self.barrier.items():
            br.status.zero_()
            a, b = self.ev[key]
            a.record()
            rc = br.launch()
            b.record()
            assert rc == 0, (key, rc)
            launches += 1
        for key, (sr, _) in self.sem.items():
            sr.reset()
            a, b = self.ev[("sem",) + key]
            a.record()
            rc = sr.launch()
            b.record()
            assert rc == 0, (key, rc)
            launches += 1
        self.launches = launches

    def times_ms(self):
        return {k: a.elapsed_time(b) for k, (a, b) in self.ev.items()}

    def verify(self, calc):
        """Checks every workload's final state against the oracle (after a step)."""
        bad = []
        for (kind, K), (mr, add) in self.mutex.items():
            got = mr.results()
            want = calc.mutex_final(NBLOCKS, MUTEX_ACQ, K, add)
            if got["status"] or got["total"] != want["total"] or not np.array_equal(got["data"], want["data"]):
                bad.append(f"mutex {kind} K={K}")
        want_mix = calc.barrier_sampled(NBLOCKS, BAR_ROUNDS)["mix"]
        for key, br in self.barrier.items():
            st = int(br.status.cpu()[0])
            mix = br.mix.cpu().numpy().view(np.uint32)
            if st or br.bad.cpu().numpy().any() or not np.array_equal(mix, want_mix):
                bad.append(f"barrier {key}")
        for (kind, n), (sr, add) in self.sem.items():
            got = sr.results()
            want = calc.sem_final(NBLOCKS, SEM_PAIRS, n, add)
            if got["status"] or got["tally"] != want["tally"] or got["max_occ"] > n:
                bad.append(f"sem {kind} n={n}")
        return bad


def e2e_mutex(G, inputs, kind, reps=3):
    """Default-kind mutex workload through gsync_bench_mutex_host with pinned host buffers:
    host->device copies of the inputs and device->host copies of every output are inside the
    timed call."""
    import torch
    total_acq, total_s = 0, 0.0
    h2d = d2h = 0
    n = NBLOCKS * MUTEX_ACQ
    bo = G.gsync_backoff(0, *MUTEX_BACKOFF[kind], 0) if kind in MUTEX_BACKOFF else None
    for K in CS_SIZES:
        delay, add = inputs.mutex_inputs(NBLOCKS, MUTEX_ACQ, inputs.mutex_seed(G.MUTEX_KINDS[kind], NBLOCKS, K))
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).pin_memory()
        hd, ha = pin(delay), pin(add)
        outs = {nm: torch.zeros(sz, dtype=torch.int32).pin_memory()
                for nm, sz in (("data", max(K, 1)), ("total", 1), ("log", n), ("ticket", n), ("count", NBLOCKS),
                               ("status", 1))}
        w = G.gsync_mutex_work(G.MUTEX_KINDS[kind], NBLOCKS, MUTEX_THREADS, MUTEX_ACQ, K,
                               mutex_cluster(kind), hd.data_ptr(),
                               ha.data_ptr(), outs["data"].data_ptr(), outs["total"].data_ptr(),
                               outs["log"].data_ptr(), outs["ticket"].data_ptr(), outs["count"].data_ptr(),
                               outs["status"].data_ptr())
        nbytes = G.gsync_bench_mutex_workspace_bytes(w.kind, NBLOCKS, MUTEX_ACQ, K)
        ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        G.check("gsync_bench_mutex_host", G.gsync_bench_mutex_host(w, bo, ws, nbytes))  # warm-up
        for _ in range(reps):
            t0 = time.perf_counter()
            G.check("gsync_bench_mutex_host", G.gsync_bench_mutex_host(w, bo, ws, nbytes))
            total_s += time.perf_counter() - t0
            total_acq += n
            assert int(outs["status"][0]) == 0 and int(outs["total"][0]) == n
        h2d += 8 * n
        d2h += 4 * (K + 1 + 2 * n + NBLOCKS + 1)
    k = len(CS_SIZES)
    return {"value": total_acq / total_s, "unit": "acq/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "kind": kind, "note": f"{k} host-buffer calls (one per CS size) per step; bytes summed over them"}


def batched_section(G, calc, inputs, runner, autotune, terms):
    """Autotunes the batched many-mutex workload, then times its CUDA-graph replay.  Roofline:
    the hottest key's acquisitions are serial, each at least one hand-off.  The carrying locks'
    hand-off is a relaxed 16-byte store seen by relaxed polls, with no fence; the carrying
    cohort locks pass on one die (through L2) or inside a cluster (through distributed shared
    memory).  So the strict roof charges the shorter of the two fence-free hand-offs:
    acq/s <= nacq / (n_hot * min(L_handoff_relaxed_near, L_handoff_relaxed_dsmem)).  Reported
    beside it: the roof with the fence-free L2 hand-off alone, with a release/acquire hand-off
    (what a lock that orders other data pays), and with a dependent L2 load added (a lock whose
    critical section loads the key's sum and count)."""
    import torch
    keys, adds, _ = inputs.batched_inputs(BATCH_ACQ, BATCH_KEYS, 1.1)
    want = calc.batched_final(keys, adds, BATCH_KEYS)
    t0 = time.perf_counter()
    tuned = autotune.tune(keys, adds, BATCH_KEYS, NBLOCKS, BATCH_GROUPS, BATCH_ROUNDS, BATCH_THREADS)
    tune_s = time.perf_counter() - t0
    out = {"workload": f"{BATCH_ACQ} acquisitions over {BATCH_KEYS} mutexes, Zipf(1.1) keys, {NBLOCKS} blocks x "
                       f"{BATCH_THREADS} threads, {BATCH_GROUPS} barrier groups x {BATCH_ROUNDS} rounds",
           "class_sizes": tuned["class_sizes"], "tuned_policy": tuned["policy"], "tuned_cluster": tuned["cluster"],
           "autotune_s": tune_s, "trials": len(tuned["trials"]), "l2": "flushed (512 MiB write) before each timed run"}
    n_hot = int(np.bincount(np.asarray(keys, dtype=np.int64), minlength=BATCH_KEYS).max())
    # The hottest key's acquisitions form one serial chain of at least one hand-off each (the
    # carrying locks move the guarded data with a fence-free hand-off, so no load and no fence
    # is added).  The looser bounds -- the fence-free L2 hand-off alone, a release/acquire
    # hand-off, and that plus one dependent load per acquisition (the critical section of the
    # other kinds) -- are reported beside it.
    l_free = min(terms["L_handoff_relaxed_near_ns"], terms["L_handoff_relaxed_dsmem_ns"])
    roof = BATCH_ACQ / (n_hot * l_free * 1e-9)
    roof_l2 = BATCH_ACQ / (n_hot * terms["L_handoff_relaxed_near_ns"] * 1e-9)
    roof_rel = BATCH_ACQ / (n_hot * terms["L_handoff_l2_near_ns"] * 1e-9)
    roof_ld = BATCH_ACQ / (n_hot * (terms["L_handoff_l2_near_ns"] + terms["L_ld_ns"]) * 1e-9)
    out.update({"hottest_key_acquisitions": n_hot, "roof_acq_per_s": roof, "roof_l2_relaxed_acq_per_s": roof_l2,
                "roof_release_acquire_acq_per_s": roof_rel, "roof_with_load_acq_per_s": roof_ld})
    results = {}
    for label, policy, cluster in (("default", autotune.DEFAULT_POLICY, 1), ("tuned", tuned["policy"], tuned["cluster"])):
        # Without clusters the kernel is captured as an ordinary launch after the co-residency
        # check (a cooperative launch is not captured); a cluster launch is captured as it is.
        run = autotune.make_run(keys, adds, BATCH_KEYS, NBLOCKS, BATCH_GROUPS, BATCH_ROUNDS, cluster,
                                tuned["key_class"], BATCH_THREADS, plain_launch=cluster == 1)
        run.set_policy(policy)
        graph, capture_error = False, None
        try:
            run.capture()
            graph = True
        except Exception as exc:  # capture refused: time plain launches instead, and say why
            capture_error = f"{type(exc).__name__}: {exc}"[:300]
            torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ts = []
        for _ in range(3):
            flush_l2()  # the inputs (12 MB) would otherwise stay in L2 from the run before
            if graph:
                s.record()
                run.replay()
                e.record()
            else:
                run.reset()
                s.record()
                G.check("gsync_bench_batched", run.launch())
                e.record()
            torch.cuda.synchronize()
            ts.append(s.elapsed_time(e))
        got = run.results()
        ok = (got["status"] == 0 and np.array_equal(got["sum"], want["sum"])
              and np.array_equal(got["count"], want["count"]) and not got["bad"].any())
        ms = float(np.median(ts))
        results[label] = {"ms": ms, "acq_per_s": BATCH_ACQ / (ms * 1e-3), "frac": BATCH_ACQ / (ms * 1e-3) / roof,
                          "cuda_graph": graph, "cluster": cluster, "parity": "ok" if ok else "FAILED"}
        if capture_error:
            results[label]["capture_error"] = capture_error
    out.update(results)
    return out


SERVE_POOL = 256 << 20           # 1 GiB of int32 values (8x the L2)
SERVE_RATES = (1e3, 1e4, 1e5, 1e6)
SERVE_SECONDS, SERVE_MAX_REQ = 0.5, 100_000
SERVE_CHUNK = 8192                # values per chunk (one block's share), both arms
SERVE_ADMITTERS = 16             # admitter blocks of the persistent loop (the other 288 blocks work)


CV_PRODUCERS, CV_CONSUMERS, CV_ITEMS, CV_CAPACITY = 592, 592, 100, 16


_FLUSH = []


def flush_l2():
    """Writes 512 MiB (four times the 129 MB L2) on the current stream, outside any timed
    region, so that the next timed launch finds its inputs in DRAM."""
    import torch
    if not _FLUSH:
        _FLUSH.append(torch.empty(512 << 20, dtype=torch.uint8, device="cuda"))
    _FLUSH[0].zero_()


# The paper draws its Section 6 curves from one block up to the most the GPU holds; the
# configurations' own grids start at 148 (one block per SM).
SWEEP_SMALL = (1, 2, 4, 8, 16, 32, 64)
SWEEP_GRIDS = SWEEP_SMALL + (148, 296, 592, 1184)
SWEEP_SEM_GRIDS = SWEEP_SMALL + (296, 592)


def sweep_grid(B, c):
    """The grid a sweep point of B blocks runs: rounded down to a multiple of the cluster size c
    for a cluster launch (0: no such grid, the point is skipped)."""
    return B - B % c if c else B

SWEEP_BARRIERS = [("atomic", 0), ("flag", 0), ("tree", 8), ("tree", 64 | 1 << 16), ("cluster", 2), ("cluster", 4),
                  ("cluster", 8), ("cluster", 8 | 2 << 4), ("count", 8), ("exchange", 8)]


def _time_launch(launch, reset, reps=3):
    """Median device time (ms) of `reps` launches after one untimed one, L2 flushed before each."""
    import torch
    ts = []
    for i in range(reps + 1):
        reset()
        flush_l2()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        rc = launch()
        e.record()
        torch.cuda.synchronize()
        assert rc == 0, rc
        if i:
            ts.append(s.elapsed_time(e))
    return float(np.median(ts))


def sweep_section(G, calc, inputs, runner, step):
    """Configs 2 and 3 over their grid sizes, as the paper's Section 6 curves are drawn (ops/s
    against the number of blocks, from one block up).  The mutex configurations at 1..64 and
    148, 296 and 592 blocks (1184 is the timed step's), the barrier kinds at 1..64 and
    148..1184 blocks, both semaphore kinds at 1..64, 296 and 592 blocks.  A cluster grid is
    rounded down to a multiple of its cluster size (144 blocks in clusters of 8 at 148), and a
    point smaller than one cluster is skipped.  Each point is a median of 3 launches with L2
    flushed before each, and each result is checked against the oracle."""
    out = {"grids": list(SWEEP_GRIDS), "mutex_acq_per_s": {}, "barrier_ns_per_crossing": {}, "semaphore_ops_per_s": {},
           "l2": "flushed (512 MiB write) before each launch", "parity": "ok"}
    bad = []
    for name, kind, policy, bo_ns, spin in MUTEX_CONFIGS:
        for K in CS_SIZES:
            row = out["mutex_acq_per_s"].setdefault(name, {}).setdefault(str(K), {})
            for B in SWEEP_GRIDS[:-1]:
                c = mutex_cluster(kind)
                nb = sweep_grid(B, c)
                if not nb or str(nb) in row:
                    continue
                delay, add = inputs.mutex_inputs(nb, MUTEX_ACQ, inputs.mutex_seed(G.MUTEX_KINDS[kind], nb, K))
                bo = runner.backoff(policy=policy, min_ns=bo_ns[0], max_ns=bo_ns[1], spin=spin) if bo_ns else None
                mr = runner.MutexRun(kind, nb, MUTEX_THREADS, MUTEX_ACQ, K, delay, add, bo=bo, timeout_ns=TIMEOUT_NS,
                                     cluster=c)
                ms = _time_launch(mr.launch, mr.reset)
                got, want = mr.results(), calc.mutex_final(nb, MUTEX_ACQ, K, add)
                if got["status"] or got["total"] != want["total"] or not np.array_equal(got["data"], want["data"]):
                    bad.append(f"mutex {name} K={K} B={nb}")
                row[str(nb)] = nb * MUTEX_ACQ / (ms * 1e-3)
    for kind, param in SWEEP_BARRIERS:
        row = out["barrier_ns_per_crossing"].setdefault(barrier_name(kind, param), {})
        for B in SWEEP_GRIDS:
            nb = sweep_grid(B, param & 0xF if kind == "cluster" else 0)
            if not nb or str(nb) in row:
                continue
            br = runner.BarrierRun(kind, nb, BAR_THREADS, BAR_ROUNDS, full=False, param=param, timeout_ns=TIMEOUT_NS)
            ms = _time_launch(br.launch, br.status.zero_)
            mix = br.mix.cpu().numpy().view(np.uint32)
            if int(br.status.cpu()[0]) or br.bad.cpu().numpy().any() or \
                    not np.array_equal(mix, calc.barrier_sampled(nb, BAR_ROUNDS)["mix"]):
                bad.append(f"barrier {kind} {param:#x} B={nb}")
            row[str(nb)] = ms * 1e6 / BAR_ROUNDS
    for kind in SEM_STEP_KINDS:
        for n in SEM_COUNTS:
            row = out["semaphore_ops_per_s"].setdefault(kind, {}).setdefault(str(n), {})
            for B in SWEEP_SEM_GRIDS:
                hold, add = inputs.sem_inputs(B, SEM_PAIRS, inputs.SEED_SEM ^ (n << 16) ^ B)
                sr = runner.SemRun(kind, B, SEM_THREADS, SEM_PAIRS, n, hold, add,
                                   bo=runner.backoff(min_ns=SEM_BACKOFF[0], max_ns=SEM_BACKOFF[1]), timeout_ns=TIMEOUT_NS)
                ms = _time_launch(sr.launch, sr.reset)
                got, want = sr.results(), calc.sem_final(B, SEM_PAIRS, n, add)
                if got["status"] or got["tally"] != want["tally"] or got["max_occ"] > n:
                    bad.append(f"sem {kind} n={n} B={B}")
                row[str(B)] = B * SEM_PAIRS / (ms * 1e-3)
    # the 1184-block points are the timed step's
    med = step
    for (name, K), ms in med["mutex"].items():
        out["mutex_acq_per_s"][name][str(K)]["1184"] = NBLOCKS * MUTEX_ACQ / (ms * 1e-3)
    for (kind, n), ms in med["sem"].items():
        out["semaphore_ops_per_s"][kind][str(n)]["1184"] = NBLOCKS * SEM_PAIRS / (ms * 1e-3)
    if bad:
        out["parity"] = bad
    return out


def condvar_section(calc, inputs, runner, terms):
    """Condition variables (future work in Section 7): bounded producer/consumer queue at 1184
    blocks.  Every item takes at least two lock acquisitions (the put and the take), each a
    hand-off plus the queue's own critical section, so the roof is half of
    1e9 / (L_handoff + T_body_cv), with T_body_cv from the single-block probe of that critical
    section minus its frame (the fastest of PROBE_PAGES placements)."""
    import torch
    n = CV_PRODUCERS * CV_ITEMS
    value = inputs.condvar_inputs(n)
    want = calc.condvar_final(value, CV_PRODUCERS, CV_ITEMS, CV_CONSUMERS)
    nbytes = runner.G.gsync_bench_condvar_workspace_bytes(16)
    t_cs = best_placement(lambda a: runner.probe_condvar_cs(128, 4000, False, scratch=a)["ns_per_cs"], nbytes, runner)
    t_frame = best_placement(lambda a: runner.probe_condvar_cs(128, 4000, True, scratch=a)["ns_per_cs"], nbytes, runner)
    t_body = max(t_cs - t_frame, 0.0)
    acq_roof = min(terms["R_same_atom_ops_s"] / 2.0, 1e9 / (terms["L_handoff_ns"] + t_body))
    roof = acq_roof / 2
    out = {"workload": f"{CV_PRODUCERS} producer + {CV_CONSUMERS} consumer blocks x 128 threads, {CV_ITEMS} items "
                       f"per producer, queue capacity {CV_CAPACITY}, one mutex + two condition variables",
           "roof_items_per_s": roof, "T_cs_cv_ns": t_cs, "T_frame_cv_ns": t_frame, "mutex": {},
           "l2": "flushed (512 MiB write) before each timed run"}
    for mutex, bo in (("ticket", (64, 2000)), ("cohort", (128, 4000)), ("cluster", (128, 4000)),
                      ("cluster_mcs", (128, 4000))):
        run = runner.CondVarRun(CV_PRODUCERS, CV_CONSUMERS, CV_ITEMS, CV_CAPACITY, value,
                                bo=runner.backoff(min_ns=bo[0], max_ns=bo[1]), mutex=mutex,
                                cluster=mutex_cluster(mutex))
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms, ok = [], True
        for _ in range(4):
            run.reset()
            flush_l2()
            s.record()
            rc = run.launch()
            e.record()
            torch.cuda.synchronize()
            st = int(run.status.cpu()[0])
            seen = run.seen.cpu().numpy().view(np.uint32)
            ok = ok and rc == 0 and st == 0 and np.array_equal(seen, want["seen"]) and \
                int(run.sum.sum().item()) == want["total"]
            ms.append(s.elapsed_time(e))
        t = float(np.median(ms[1:]))
        items_s = n / (t * 1e-3)
        acq = int(run.acq.cpu()[0])  # acquisitions of the last launch, re-locks after waits included
        out["mutex"][mutex] = {"ms": t, "items_per_s": items_s, "frac": items_s / roof,
                               "acquisitions_per_item": acq / n if n else 0.0,
                               "lock_acq_per_s": acq / (t * 1e-3), "lock_frac": acq / (t * 1e-3) / acq_roof,
                               "parity": "ok" if ok else "FAILED"}
    return out


def serve_section(calc, inputs, runner):
    """Persistent serving loop vs one launch per request at swept Poisson arrival rates."""
    import torch
    off_all, len_all, pool = inputs.serve_inputs(SERVE_MAX_REQ, SERVE_POOL)
    dpool = torch.from_numpy(pool).cuda()
    rng = np.random.default_rng(0)
    out = {"workload": f"int32 segmented sums, length log-uniform 256..1048576, pool {SERVE_POOL} values "
                       f"({SERVE_POOL * 4 >> 20} MiB), Poisson arrivals, open loop (latency from the scheduled arrival "
                       f"to the host seeing the completion flag); persistent loop: 304 blocks of which "
                       f"{SERVE_ADMITTERS} admit, 64 slots; both arms: chunks of {SERVE_CHUNK} values", "rates": {}}
    for rate in SERVE_RATES:
        nreq = int(min(SERVE_MAX_REQ, max(500, rate * SERVE_SECONDS)))
        off, ln = off_all[:nreq], len_all[:nreq]
        sched = inputs.poisson_arrivals(nreq, rate)
        sample = rng.choice(nreq, size=min(nreq, 300), replace=False)
        want = calc.serve_final(off[sample], ln[sample], pool)
        row = {"nreq": nreq, "chunk_values": SERVE_CHUNK}
        # persistent: the ring in pinned host memory; persistent_device_ring: the ring in managed
        # memory placed in device memory, written in place by the host
        for arm in ("persistent", "persistent_device_ring", "per_request_launch"):
            sr = runner.ServeRun(off, ln, sched, dpool, nslots=64, nblocks=304, admitters=SERVE_ADMITTERS,
                                 chunk_elems=SERVE_CHUNK, ring="device" if arm == "persistent_device_ring" else "host")
            r = sr.baseline(nstreams=8) if arm == "per_request_launch" else sr.run()
            lat = r["latency_ns"] / 1e3
            span = (sched[-1] + r["latency_ns"][-1]) / 1e9
            row[arm] = {"rc": r["rc"], "p50_us": float(np.percentile(lat, 50)), "p99_us": float(np.percentile(lat, 99)),
                        "mean_us": float(lat.mean()), "achieved_req_s": nreq / max(span, 1e-9),
                        "host_publish_delay_max_us": float(r["publish_delay_ns"].max() / 1e3),
                        "parity_sample": "ok" if np.array_equal(r["res"][sample], want) else "FAILED"}
        out["rates"][f"{rate:g}"] = row
    return out


def cpu_baseline(inputs, kind):
    """The CPU oracle (threaded C execution) on the host cores, same workload, one pass."""
    from oracle import cpu
    from paper_1110_4623_gb300 import gsync as G
    acq, secs, threads = 0, 0.0, 0
    # The host has no dies to keep hand-offs on: the oracle runs the cohort workload (same
    # inputs, same result) with its ticket lock.
    cpu_kind = kind if kind in cpu.MUTEX_KINDS else "ticket"
    for K in CS_SIZES:
        delay, add = inputs.mutex_inputs(NBLOCKS, MUTEX_ACQ, inputs.mutex_seed(G.MUTEX_KINDS[kind], NBLOCKS, K))
        r = cpu.mutex_run(cpu_kind, NBLOCKS, MUTEX_ACQ, K, add, delay)
        acq += NBLOCKS * MUTEX_ACQ
        secs += r["seconds"]
        threads = r["threads"]
    return {"value": acq / secs, "unit": "acq/s", "cores": threads, "kind": "oracle",
            "sample": f"{kind} mutex workload, {NBLOCKS} blocks x {MUTEX_ACQ} acquisitions x CS {list(CS_SIZES)} "
                      f"words (the full step's mutex workload of the default kind; the oracle's {cpu_kind} lock), "
                      f"blocks round-robin on {threads} threads"}


# The paper's own figures (context only, other hardware): same-word atomic throughput from
# Table 1 (1000 contentious atomics per block on a saturated GPU: Tesla GTX295, 240 blocks,
# 78.4 ms; Fermi GTX580, 128 blocks, 1.47 ms) and the relative results of Section 6.
PAPER_CONTEXT = {
    "same_word_atomics_per_s": {"tesla_gtx295": 240_000 / 78.407e-3, "fermi_gtx580": 128_000 / 1.479e-3},
    "kernel_relaunch_as_barrier_us": {"gt200_quoted": "10-14 synchronous, 3-7 asynchronous (Volkov and Demmel)"},
    "atomic_barrier_vs_xf": {"tesla_gtx295": "< 0.05 at 60 blocks", "fermi_gtx580": "~0.30 at 128 blocks"},
    "fa_mutex_vs_spin_backoff": {"tesla_gtx295": "> 20 (spin+backoff < 5 % of FA)", "fermi_gtx580": "~0.5"},
}


def relaunch_barrier_us(runner, reps=200):
    """The alternative the paper sets its grid barrier against (Section 2): ending the kernel and
    launching the next one.  An empty launch of the barrier workload's 1184-block grid (zero
    rounds; a cooperative launch, as the workload's), back to back on one stream (asynchronous:
    one launch's cost as a barrier) and with the host waiting for each (synchronous), in
    microseconds per relaunch."""
    import torch
    br = runner.BarrierRun("count", NBLOCKS, BAR_THREADS, 0, full=False, param=8)
    for _ in range(10):
        assert br.launch() == 0
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        br.launch()
    e.record()
    torch.cuda.synchronize()
    asyn = s.elapsed_time(e) * 1e3 / reps
    t0 = time.perf_counter()
    for _ in range(reps):
        br.launch()
        torch.cuda.synchronize()
    syn = (time.perf_counter() - t0) * 1e6 / reps
    return {"asynchronous": asyn, "synchronous": syn}


def paper_context(terms, barrier, mutex, relaunch=None):
    """The paper's figures beside the same quantities measured on this GPU in this run."""
    return {"paper": PAPER_CONTEXT,
            "gb300": {"kernel_relaunch_as_barrier_us": relaunch,
                      "grid_barrier_us": barrier[barrier_name(*DEFAULT_BARRIER)]["ns_per_crossing"] / 1e3,
                      "same_word_atomics_per_s": terms["R_same_atom_ops_s"],
                      "atomic_barrier_vs_xf": barrier["flag"]["ns_per_crossing"] / barrier["atomic"]["ns_per_crossing"],
                      "fa_mutex_vs_spin_backoff": float(np.mean([mutex["ticket"][k]["acq_per_s"] /
                                                                 mutex["cas_backoff"][k]["acq_per_s"]
                                                                 for k in mutex["ticket"]]))},
            "note": "speed ratios (higher = the first design is faster); the paper's figures are for its "
                    "hardware, quoted as context, not targets"}


def run_gpu(args):
    import torch
    from oracle import calc
    from paper_1110_4623_gb300 import autotune, gsync as G, inputs, runner

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    G.lib()
    terms_before = measure_roofline_terms(runner, inputs)
    step = GpuStep(runner, G, inputs)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        step.launch()
        torch.cuda.synchronize()
    bad = step.verify(calc)
    if bad:
        raise SystemExit(f"parity failure after warm-up: {bad}")

    per_step, per_kernel = [], []
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()  # 512 MiB write: evicts the 129 MB L2 between steps (outside the step's events)
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        step.launch()
        s1.record()
        torch.cuda.synchronize()
        per_step.append(s0.elapsed_time(s1))
        per_kernel.append(step.times_ms())
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    bad = step.verify(calc)
    terms = merge_terms(terms_before, measure_roofline_terms(runner, inputs))

    med = {k: float(np.median([pk[k] for pk in per_kernel])) for k in per_kernel[0]}
    def_ms = sum(med[(DEFAULT_MUTEX, K)] for K in CS_SIZES)
    step_ms, def_ms = max_over_ranks([float(np.mean(per_step)), def_ms], world)
    mutex = {}
    for (kind, K) in step.mutex:
        ms = med[(kind, K)]
        acq_s = NBLOCKS * MUTEX_ACQ / (ms * 1e-3)
        roof = mutex_roof_acq_s(terms, K)
        mutex.setdefault(kind, {})[str(K)] = {"ms": ms, "acq_per_s": acq_s, "roof_acq_per_s": roof, "frac": acq_s / roof}
    def_acq = NBLOCKS * MUTEX_ACQ * len(CS_SIZES)
    value = replica_value(def_acq, def_ms, world)
    roof_ms = sum(NBLOCKS * MUTEX_ACQ / mutex_roof_acq_s(terms, K) * 1e3 for K in CS_SIZES)
    peak = def_acq / (roof_ms * 1e-3)
    barrier = {}
    for (k, p) in step.barrier:
        ns = med[(k, p)] * 1e6 / BAR_ROUNDS
        roof = barrier_roof_ns(terms, k, br_param(k, p), NBLOCKS)
        barrier[barrier_name(k, p)] = {"ns_per_crossing": ns, "roof_ns": roof, "frac": roof / ns}
    bkey = barrier_name(*DEFAULT_BARRIER)
    sem_kinds = {}
    for kind in SEM_STEP_KINDS:
        sem_kinds[kind] = {}
        for n in SEM_COUNTS:
            ms = med[("sem", kind, n)]
            ops = NBLOCKS * SEM_PAIRS / (ms * 1e-3)
            roof = sem_roof_ops_s(terms, n)
            sem_kinds[kind][str(n)] = {"ops_per_s": ops, "roof_ops_per_s": roof, "frac": ops / roof}
    sem = sem_kinds[DEFAULT_SEM]

    # Section 4's rule plus its GB300 extensions (dies, hand-off gap, same-word atomic cost),
    # applied to this GPU's measurements, beside the defaults the sweeps chose.
    from paper_1110_4623_gb300 import machine
    ext = machine.measure_extended(NBLOCKS)
    params = machine.abstraction(machine.measure_table(NBLOCKS, 128, 1000, reps=1))
    design_rule = {"section4": machine.design(params), "extended": machine.design_extended(params, ext, NBLOCKS),
                   "measured": ext, "defaults": {"mutex": DEFAULT_MUTEX, "barrier": barrier_name(*DEFAULT_BARRIER),
                                                  "sem": DEFAULT_SEM}}
    out = {
        "metric": METRIC, "value": value, "unit": "acq/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic (seeded SplitMix64 delays/addends/hold times)",
        "config": step_config(world),
        "roofline": {"bound": "l2_handoff_latency", "achieved": value / world, "peak": peak, "unit": "acq/s",
                     "frac": (value / world) / peak, "traffic": ROOF_TRAFFIC,
                     "traffic_note": ROOF_TRAFFIC_NOTE,
                     "peak_source": "measured live: sum over CS sizes of 1e9 / (L_handoff + T_body(K)); L_handoff "
                                    "= the shortest hand-off the GPU offers: min of a ping-pong of two SMs of one "
                                    "die on lines homed on that die and a ping-pong inside a thread-block cluster "
                                    "through distributed shared memory; T_body = critical-section probe minus its "
                                    "frame, each at the fastest of 8 page placements (lines homed on the "
                                    "probe's own die); min with R_same/2; MEASURED_PEAKS.json's HBM and bf16 peaks do not "
                                    "bound this path"},
        "barrier": {"default": bkey, "ns_per_crossing": barrier[bkey]["ns_per_crossing"],
                    "frac": barrier[bkey]["frac"], "kinds": barrier},
        "mutex": mutex,
        "semaphore": {"kind": DEFAULT_SEM, "backoff_ns": list(SEM_BACKOFF), "n": sem, "kinds": sem_kinds},
        "roofline_terms": terms,
        "design_rule": design_rule,
        "paper_context": paper_context(terms, barrier, mutex, relaunch_barrier_us(runner)),
        "clocks": clk,
        "gpu_launches": step.launches * args.steps,
        "wall_s_timed_loop": wall,
        "parity_after_timing": "ok" if not bad else bad,
    }
    e2e = e2e_mutex(G, inputs, DEFAULT_MUTEX)
    # Every rank ran the same number of acquisitions; the job's time is the slowest rank's.
    (ms_per_acq,) = max_over_ranks([1e3 / e2e["value"]], world)
    e2e["value"] = replica_value(1, ms_per_acq, world)
    if rank == 0:
        out["e2e"] = e2e
        out["condvar"] = condvar_section(calc, inputs, runner, terms)
        if not args.no_sweep:
            step_ms = {"mutex": {key: med[key] for key in step.mutex},
                       "sem": {key: med[("sem",) + key] for key in step.sem}}
            out["sweep"] = sweep_section(G, calc, inputs, runner, step_ms)
        if not args.no_batched:
            out["batched"] = batched_section(G, calc, inputs, runner, autotune, terms)
            out["serving"] = serve_section(calc, inputs, runner)
            r5 = out["serving"]["rates"].get("100000")
            if r5:
                out["p99_latency_us"] = {"persistent_at_1e5_req_s": r5["persistent"]["p99_us"],
                                         "per_request_launch_at_1e5_req_s": r5["per_request_launch"]["p99_us"]}
        if not args.no_cpu_baseline and world == 1:
            out["cpu_baseline"] = cpu_baseline(inputs, DEFAULT_MUTEX)
        if args.jsonl:
            with open(args.jsonl, "a") as f:
                for row in result_rows(out):
                    f.write(json.dumps(row, default=float) + "\n")
        print(json.dumps(out, default=float))
    if world > 1:
        torch.distributed.destroy_process_group()


def step_config(world):
    """The workload the bench line is quoted on; both arms print it."""
    c = mutex_cluster(DEFAULT_MUTEX)
    return {"workload": f"mutex contention, {NBLOCKS} blocks x {MUTEX_THREADS} threads"
                        f"{f' in clusters of {c}' if c else ''}, {MUTEX_ACQ} "
                        f"acquisitions/block, CS {list(CS_SIZES)} int32 words, delays U{{0..2000}} cycles; "
                        f"+ barriers ({BAR_ROUNDS} rounds) and semaphores ({SEM_PAIRS} pairs) at {NBLOCKS} blocks",
            "default_mutex": f"{DEFAULT_MUTEX} (backoff {MUTEX_BACKOFF.get(DEFAULT_MUTEX)} ns)",
            "default_barrier": barrier_name(*DEFAULT_BARRIER), "nblocks": NBLOCKS,
            "l2": "flushed (512 MiB write) before every timed step", "parallelism": f"replicas x{world}"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_1110_4623_gb300 import inputs
    vals = []
    base = None
    t_all = time.perf_counter()
    for _ in range(args.warmup):
        cpu_baseline(inputs, DEFAULT_MUTEX)
    for _ in range(args.steps):
        base = cpu_baseline(inputs, DEFAULT_MUTEX)
        vals.append(base["value"])
    value = float(np.median(vals))
    step_ms = NBLOCKS * MUTEX_ACQ * len(CS_SIZES) / value * 1e3
    out = {"metric": METRIC, "impl": "reference", "value": value, "unit": "acq/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
           "config": step_config(world),
           "cpu_baseline": {"value": value, "unit": "acq/s", "cores": base["cores"], "kind": "oracle",
                            "sample": base["sample"]},
           "e2e": {"value": value, "unit": "acq/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "wall_s": time.perf_counter() - t_all}
    print(json.dumps(out, default=float))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
