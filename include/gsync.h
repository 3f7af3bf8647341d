/*
 * gsync.h -- C ABI of the inter-block GPU synchronization library (sm_103a).
 *
 * Implements the primitives of Stuart & Owens, "Efficient Synchronization Primitives for
 * GPUs": the grid barrier, the mutex (spin lock, spin lock with backoff, fetch-and-add
 * ticket lock, sleep-waiting queue lock) and the counting semaphore (sleeping FA semaphore,
 * spin-lock semaphore with and without backoff), plus the memory-system probes that
 * classify a GPU under the paper's machine abstraction.  Device-side calls are in
 * gsync_device.cuh; this header holds the host entry points.
 *
 * Conventions shared by every entry point:
 *  - Memory: the library never allocates.  Every pointer named "device" is caller-owned
 *    device memory; "host" pointers are caller-owned host memory.  Objects (the `state`
 *    buffers) must be 128-byte aligned and sized with the matching gsync_*_bytes().
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Entry points enqueue work and return without synchronizing, except the *_host
 *    variants, which copy host buffers in and out and synchronize `stream`.
 *  - Errors: every entry point returns a gsync_status; nothing throws or exits.  Device
 *    waits are bounded by the object's timeout; a timed-out or aborted wait is reported in
 *    the caller's `status` word (bit GSYNC_STATUS_TIMEOUT / GSYNC_STATUS_ABORTED) and in
 *    the object's abort word, and the kernel returns instead of hanging.
 *  - Block semantics (Section 3): one request per block; every thread of a block calls the
 *    device function, thread 0 acts, __syncthreads arbitrates inside the block.
 */
#ifndef GSYNC_H
#define GSYNC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gsync_status {
  GSYNC_OK = 0,
  GSYNC_EINVAL = 1,        /* bad argument: size, alignment, kind, or a buffer too small */
  GSYNC_ENOTRESIDENT = 2,  /* the grid cannot be co-resident, so a barrier could deadlock */
  GSYNC_ETIMEDOUT = 3,     /* a device wait exceeded the object's timeout */
  GSYNC_ECUDA = 4,         /* a CUDA runtime call failed (see gsync_last_cuda_error) */
  GSYNC_EABORTED = 5       /* a device wait gave up because another wait on the object timed
                              out, or the host aborted the object (gsync_object_abort) */
} gsync_status;

/* Bits of the device `status` word that the workload kernels OR in. */
enum {
  GSYNC_STATUS_TIMEOUT = 1u,
  GSYNC_STATUS_ABORTED = 2u,
  GSYNC_STATUS_VIOLATION = 4u, /* a workload saw an impossible state (e.g. a grant index past the end) */
  GSYNC_STATUS_CONFIG = 8u     /* launch shape does not match the object (e.g. grid != nblocks) */
};

/* Mutex kinds (Section 5, "Mutex"; Appendix, spin-lock and FA mutex pseudocode). */
typedef enum gsync_mutex_kind {
  GSYNC_MUTEX_CAS_SPIN = 0,    /* spin on atomicCAS(0 -> 1); unlock = release store 0 */
  GSYNC_MUTEX_CAS_BACKOFF = 1, /* the same with __nanosleep backoff after each failure */
  GSYNC_MUTEX_TICKET = 2,      /* fetch-and-add ticket; poll turn; unlock stores turn + 1 */
  GSYNC_MUTEX_SLEEP_QUEUE = 3, /* queue lock: each waiter polls its own padded flag slot */
  GSYNC_MUTEX_COHORT = 4,      /* two-die cohort lock: a ticket lock per die (homed on that
                                  die) under a global ticket lock; hand-offs stay on a die
                                  for up to `budget` acquisitions in a row */
  GSYNC_MUTEX_RING = 5,        /* the paper's ring-buffer sleeping mutex (Section 5, design
                                  alternative): a waiter writes its block id at the ring's
                                  end and polls the head pointer and the entry it names */
  GSYNC_MUTEX_CLUSTER = 6,     /* cohort lock over thread-block clusters: a ticket lock per
                                  cluster in distributed shared memory under a global ticket
                                  lock; needs a cluster launch (see gsync_mutex_init_cluster) */
  GSYNC_MUTEX_CLUSTER_MCS = 7  /* the same with an MCS queue per cluster: each waiter spins in
                                  its own shared memory and its predecessor pushes the grant
                                  into it; needs a cluster launch (see
                                  gsync_mutex_init_cluster_mcs) */
} gsync_mutex_kind;

/* Barrier kinds (Section 5, "Barrier"). */
typedef enum gsync_barrier_kind {
  GSYNC_BAR_ATOMIC = 0,  /* two-stage atomic counter + release epoch */
  GSYNC_BAR_FLAG = 1,    /* decentralized flag barrier of Xiao and Feng (XF) */
  GSYNC_BAR_TREE = 2,    /* combining tree of atomic counters (param = fan | form << 16) */
  GSYNC_BAR_CLUSTER = 3, /* hardware cluster barrier, then one leader per cluster on a counter
                            (param = c | form << 4 | sleep << 8; see gsync_barrier_bytes) */
  GSYNC_BAR_SHARDED = 4, /* arrivals spread over param counters, gathered by one warp (XF-style release) */
  GSYNC_BAR_DIE = 5,     /* two-die barrier: a release word per die, homed on that die; param 0:
                            a counter per die, the dies' last arrivers meet on a top counter;
                            param 1: one flat counter */
  GSYNC_BAR_SPLIT = 6,   /* S arrival counters under a top counter, R copies of the release
                            word (param = S | R << 8) */
  GSYNC_BAR_COUNT = 7,   /* a growing 64-bit arrival counter that every block polls: the last
                            arrival is the release (no epoch word); optionally two levels */
  GSYNC_BAR_EXCHANGE = 8 /* the counting barrier whose arrivals carry one 64-bit value per
                            block, read by any block after the crossing (gsync::barrier_exchange
                            and barrier_exchange_read): no fence, and only the exchanged values
                            are ordered; param = the sleep of COUNT (0..1023) */
} gsync_barrier_kind;

/* Semaphore kinds (Section 5, "Semaphore"; Appendix, spin-lock and sleeping semaphores). */
typedef enum gsync_sem_kind {
  GSYNC_SEM_TICKET = 0,       /* sleeping FA semaphore: <= 2 atomics per wait and per post */
  GSYNC_SEM_SPIN = 1,         /* spin-lock semaphore: S = X + 1, swap with 0 to update */
  GSYNC_SEM_SPIN_BACKOFF = 2, /* the same with backoff in wait (not in post) */
  GSYNC_SEM_WINDOW = 3        /* ticket window (GB300 alternative): wait takes a ticket t and
                                 enters once turn + n > t; post is one fire-and-forget add to
                                 turn, with no round trip */
} gsync_sem_kind;

/* Backoff policy (Section 5: "Backoff"; the paper's counter I runs from Imin to Imax by +1
 * and wraps; exponential doubling is the other common policy). */
enum {
  GSYNC_BACKOFF_EXPONENTIAL = 0,
  GSYNC_BACKOFF_LINEAR_CYCLIC = 1,
  /* Section 5's GPU stand-in for a futex: spin aggressively (no sleep) for `spin` failed
   * attempts, then fall back to exponential backoff from min_ns (CAS kinds). */
  GSYNC_BACKOFF_SPIN_THEN_SLEEP = 2
};

typedef struct gsync_backoff {
  uint32_t policy; /* GSYNC_BACKOFF_* */
  uint32_t min_ns; /* first sleep (and, for ticket locks, sleep per waiter ahead); 0 = no sleeping */
  uint32_t max_ns; /* cap */
  uint32_t spin;   /* SPIN_THEN_SLEEP: failed attempts before the first sleep (0 selects 32) */
} gsync_backoff;

/* ------------------------------------------------------------------------------------ */
/* Objects: size query and initialisation (Algorithm 1: CreateSpinLock allocates a word  */
/* and zeroes it; here the caller allocates and the library writes the initial state).   */
/* ------------------------------------------------------------------------------------ */

/* Bytes of a mutex for at most `max_waiters` blocks waiting at once; 0 if invalid.
 * COHORT takes 32 KB whatever the waiters. */
size_t gsync_mutex_bytes(int kind, int max_waiters);
/* Writes the initial state of a mutex into `state` (device) on `stream`.  `backoff` (host,
 * may be NULL for no sleeping) is copied; timeout_ns = 0 selects 2 s.  COHORT: as
 * gsync_mutex_init_cohort with GSYNC_COHORT_DEFAULT_BUDGET. */
int gsync_mutex_init(void* state, size_t bytes, int kind, int max_waiters,
                     const gsync_backoff* backoff, uint64_t timeout_ns, void* stream);

/* Cohort mutex (GSYNC_MUTEX_COHORT) with a chosen budget (1..32767): the lock passes from a
 * holder to the next waiter on the same die at most budget - 1 times in a row before the
 * global lock goes to the other die, so a block waits behind at most its own die's queue
 * plus `budget` acquisitions per other-die turn.  Measures the device's SM-to-die map (once
 * per device and process: the gsync_probe_rtt_by_sm probe, ~3 ms) and the home die of the
 * state's 4 KB pages, then places each die's local lock on a page homed on that die;
 * synchronizes `stream`.  On a one-die GPU both local locks serve every SM.  state: device,
 * 128-byte aligned, bytes >= gsync_mutex_bytes(GSYNC_MUTEX_COHORT, 1).  gsync_mutex_init with
 * COHORT or CLUSTER uses GSYNC_COHORT_DEFAULT_BUDGET. */
enum { GSYNC_COHORT_DEFAULT_BUDGET = 64 };
int gsync_mutex_init_cohort(void* state, size_t bytes, int budget, const gsync_backoff* backoff,
                            uint64_t timeout_ns, void* stream);

/* Cluster mutex (GSYNC_MUTEX_CLUSTER): the cohort protocol with the thread-block cluster as the
 * group (a holder passes to a waiter of its own cluster through distributed shared memory, at
 * most budget - 1 times in a row).  state holds only the global ticket lock (3 lines); each
 * cluster's local lock is a gsync::ClusterLocal the kernel declares __shared__ and hands to
 * gsync::mutex_attach_cluster at its start (all threads), and the kernel calls
 * gsync::mutex_cluster_end() before exiting.  The kernel must be launched with clusters
 * (gsync_launch_coresident with cluster > 1).  budget 1..32767; asynchronous on `stream`. */
int gsync_mutex_init_cluster(void* state, size_t bytes, int budget, const gsync_backoff* backoff,
                             uint64_t timeout_ns, void* stream);

/* Cluster MCS mutex (GSYNC_MUTEX_CLUSTER_MCS): the cluster cohort lock whose local lock is an
 * MCS queue (Mellor-Crummey and Scott, 1991).  Each block's node is a gsync::McsNode the kernel
 * declares __shared__ and hands to gsync::mutex_attach_cluster_mcs at its start (all threads);
 * the kernel calls gsync::mutex_cluster_end() before exiting and is launched with clusters.
 * A waiter spins on its own node; its predecessor writes the grant into it.  state holds the
 * global ticket lock (3 lines); budget 1..32767 as for CLUSTER; asynchronous on `stream`. */
int gsync_mutex_init_cluster_mcs(void* state, size_t bytes, int budget, const gsync_backoff* backoff,
                                 uint64_t timeout_ns, void* stream);

/* The device's SM-to-die map: die_of_sm (host, >= sm_count bytes) receives 0 or 1 per SM id
 * (die 0 = the SMs near a fixed line of the library's static memory), *ndies_out 1 or 2.
 * Measured once per device and process with gsync_probe_rtt_by_sm (the atomic round trip to
 * a line homed on the other die is ~2x longer), then cached; synchronizes `stream` on first
 * use. */
int gsync_device_topology(uint8_t* die_of_sm, int* ndies_out, void* stream);

/* Bytes of a barrier for `nblocks` blocks.  param: fan | form << 16 (TREE: fan-in 2..1024;
 * form 0: the last arriver at a node resets it and climbs, and the root's last arriver
 * advances a release epoch that every block polls; form 1: node counters that only grow, the
 * arrival that completes a node's crossing climbs, and the root's completing add is the
 * release that every block polls for), c | form << 4 |
 * sleep << 8 (CLUSTER: c the cluster size, 1..8, dividing nblocks; form 0: the cluster
 * leaders meet on an atomic barrier whose release epoch every block polls; form 1: the
 * leaders add to a growing counter, the last add is the release, and every block polls the
 * counter; form 2: as 1, but only the leaders poll and the other blocks wait at a second
 * hardware cluster barrier; sleep 0..1023 = ns a leader sleeps per 16 leader arrivals still
 * missing before its first poll, forms 1 and 2), release mode (FLAG: 0 one flag per block, 1 one word;
 * FLAG takes at most 8192 blocks), number of arrival counters (SHARDED, 1..32), S | R << 8
 * (SPLIT: S arrival counters and R release copies, 1..64 each), 0 or 1 (DIE: per-die counters,
 * or one flat counter with a release word on each die), sleep | S << 16 (COUNT: sleep 0..1023 =
 * ns of sleep before the first poll per 16 arrivals still missing, 0 polls at once; S 0..64,
 * S > 1 counts in through S sub-counters), 0 (ATOMIC).  FLAG and SHARDED need blockDim.x >= 32 (warp 0 of block 0 gathers the arrivals).
 * DIE takes 32 KB; its init measures the SM-to-die map and the home die of the state's
 * 4 KB pages as gsync_mutex_init_cohort does (and synchronizes `stream`); the first
 * crossing of each launch counts the blocks per die (a flat crossing), later ones run per
 * die.  On a one-die GPU DIE behaves as ATOMIC. */
size_t gsync_barrier_bytes(int kind, int nblocks, int param);
int gsync_barrier_init(void* state, size_t bytes, int kind, int nblocks, int param,
                       uint64_t timeout_ns, void* stream);

/* Condition variable (named as future work in Section 7; the paper gives no algorithm):
 * two counters, waiters so far and waiters released so far.  Device side (gsync_device.cuh):
 * cond_wait(cv, mutex, token) called by the whole block while it holds the mutex takes a
 * ticket, releases the mutex, waits until the releases pass its ticket and takes the mutex
 * again; cond_signal_thread / cond_broadcast_thread, called by thread 0 while it holds the
 * mutex, release the oldest waiter / every waiter.  `backoff` (may be NULL) sets the sleep
 * between polls of a waiting block; timeout_ns = 0 selects 2 s. */
size_t gsync_cond_bytes(void);
int gsync_cond_init(void* state, size_t bytes, const gsync_backoff* backoff, uint64_t timeout_ns,
                    void* stream);

/* Bytes of a counting semaphore. */
size_t gsync_sem_bytes(int kind);
/* Initial count n >= 1 (Section 5: at most n blocks inside at once). */
int gsync_sem_init(void* state, size_t bytes, int kind, int initial_count,
                   const gsync_backoff* backoff, uint64_t timeout_ns, void* stream);

/* Reads an object's abort word (device -> host, synchronous on `stream`): 0 when no wait
 * on the object has timed out and the host has not aborted it; bit 0 set by a device wait
 * that timed out, bit 1 by gsync_object_abort. */
int gsync_object_abort_flag(const void* state, uint32_t* flag_out, void* stream);

/* Host-side abort (the watchdog's lever): sets the object's abort word, so that every wait on
 * it -- running now or later -- returns GSYNC_EABORTED within a few polls instead of running
 * to the object's timeout.  A 32-bit stream write (cuStreamWriteValue32) enqueued on
 * `stream`, asynchronous: the GPU's front end performs it, so it needs no SM (it lands while
 * a co-resident grid holds every SM) and no host staging.  `stream` must not be ordered after
 * the kernel that waits: a stream created with cudaStreamNonBlocking, other than the
 * kernel's.  (Where the driver lacks stream memory operations, a host-to-device copy is used
 * instead, which lands only if the waiting kernel is not on the legacy default stream.)
 * gsync_*_init clears the word.  GSYNC_EINVAL for a NULL or misaligned state. */
int gsync_object_abort(void* state, void* stream);

/* ------------------------------------------------------------------------------------ */
/* Co-residency (Section 5: the barrier needs every block resident, "persistent threads") */
/* ------------------------------------------------------------------------------------ */

/* Largest grid of the given workload kernel that is co-resident on the current device
 * with `block_threads` threads per block (and `cluster` blocks per cluster when > 1).
 * workload: 0 barrier, 1 mutex, 2 semaphore; kind: that workload's kind enum. */
int gsync_max_coresident_blocks(int workload, int kind, int block_threads, int cluster,
                                int* max_blocks_out);

/* The same gate for the caller's own kernels (the ones that call barrier_wait and the other
 * device primitives of gsync_device.cuh).  `kernel` is the kernel's cudaFunction_t handle,
 * from cudaGetFuncBySymbol(&f, (const void*)my_kernel) in the caller's program (a host-stub
 * pointer would be unknown to the library's own CUDA runtime); smem_bytes its dynamic shared
 * memory (over 48 KB the caller sets the kernel's attribute first); cluster its blocks per
 * cluster (1 = no clusters).  Driver calls are made through cudaGetDriverEntryPointByVersion;
 * GSYNC_ECUDA if the driver lacks them, GSYNC_EINVAL if the handle is not a kernel.
 * gsync_check_coresident: *max_blocks_out = the largest co-resident grid; returns GSYNC_OK,
 *   or GSYNC_ENOTRESIDENT when grid exceeds it.
 * gsync_launch_coresident: launches the kernel on grid x block_threads (1-D), smem_bytes and
 *   `stream`, with args (an array of pointers to the arguments, as for cudaLaunchKernel), so
 *   that every block
 *   is resident at once (a cooperative launch; an occupancy-checked cluster launch when
 *   cluster > 1), or refuses with GSYNC_ENOTRESIDENT before anything runs.  Asynchronous. */
int gsync_check_coresident(const void* kernel, int grid, int block_threads, size_t smem_bytes,
                           int cluster, int* max_blocks_out);
int gsync_launch_coresident(const void* kernel, int grid, int block_threads, size_t smem_bytes,
                            int cluster, void** args, void* stream);

/* Number of SMs of the current device. */
int gsync_device_sm_count(int* sms_out);

/* Last CUDA error code seen by the library on this thread (cudaError_t as int). */
int gsync_last_cuda_error(void);

/* ------------------------------------------------------------------------------------ */
/* Workloads (Section 6, "Results": one kernel, a loop of operations per block).          */
/* All launches are cooperative (or occupancy-checked cluster launches): a grid that     */
/* cannot be co-resident returns GSYNC_ENOTRESIDENT before anything runs.                */
/* ------------------------------------------------------------------------------------ */

/* Barrier workload.  Round r: block b writes slots[(r&1)*nblocks + b] = r*nblocks + b,
 * crosses the barrier, then reads slots of the same half:
 *   full = 1: every slot j; chk[r*nblocks + b] = XOR_j slot_j; mix[b] = rotl(mix[b],5) ^
 *             (sum_j lowbias32(slot_j)); bad[b] += #(slot_j != r*nblocks + j)
 *   full = 0: partner p = (b + r + 1) mod nblocks; mix[b] = rotl(mix[b],5) ^ lowbias32(slot_p);
 *             bad[b] += (slot_p != r*nblocks + p)
 * Buffers (device): slots [2*nblocks] (scratch), chk [rounds*nblocks] (full only, else NULL),
 * mix [nblocks], bad [nblocks], status [1] (OR of GSYNC_STATUS_*; caller zeroes).
 * `state` must be a barrier initialised for nblocks (and `cluster` for CLUSTER). */
typedef struct gsync_barrier_work {
  int32_t kind, nblocks, block_threads, rounds, full, cluster;
  uint32_t* slots;
  uint32_t* chk;
  uint32_t* mix;
  uint32_t* bad;
  uint32_t* status;
} gsync_barrier_work;
int gsync_bench_barrier(void* state, const gsync_barrier_work* w, void* stream);

/* Phase trace of the sampled barrier workload (w->full must be 0): as gsync_bench_barrier,
 * and block b also writes its %globaltimer just before and just after its round-r barrier
 * into trace[2 * (b * rounds + r)] and trace[2 * (b * rounds + r) + 1] (device,
 * 2 x nblocks x rounds u64).  A diagnostic: it shows how long the last arrival takes to
 * release the first and the last waiter. */
int gsync_probe_barrier_trace(void* state, const gsync_barrier_work* w, uint64_t* trace,
                              void* stream);

/* The barrier workload for callers that cannot allocate device memory.  The paper has no
 * counterpart; this is a library convenience.  Some callers cannot call cudaMalloc: code
 * running where a device allocation is not allowed or would stall (a host callback, a loop
 * that must not take cudaMalloc's implicit device synchronization, a plugin whose framework
 * owns all device memory).  This variant allocates nothing.  The barrier object and the
 * slot buffers live in one 128 KiB file-scope device array inside the library, which every
 * GPU that loads the library holds until the process exits.  The caller still passes the
 * outputs in `w` (chk, mix, bad, status; w->slots is ignored).
 *  - Kinds: ATOMIC, FLAG, TREE, CLUSTER, SHARDED, SPLIT, COUNT and EXCHANGE, with `param`
 *    as for gsync_barrier_bytes (CLUSTER takes its size from w->cluster and its form and
 *    sleep from the other bits of `param`; EXCHANGE carries the slot values in its records
 *    and does not use the slot buffers).  DIE returns GSYNC_EINVAL: its init measures the die
 *    map and synchronizes the stream.
 *  - Limits: nblocks <= GSYNC_STATIC_MAX_BLOCKS (4096), and the object for (kind, nblocks,
 *    param) must fit in 96 KiB (gsync_barrier_bytes); anything larger returns GSYNC_EINVAL.
 *  - Every call looks up the array's device address (cudaGetSymbolAddress) with the
 *    caller's device current; nothing is cached, so the address stays right after a
 *    cudaDeviceReset.  The first call on a device (and the first after a reset) loads the
 *    library's module there: make it before any stream capture.
 *  - Every call shares the one array and each call rewrites the object and clears the
 *    slots, so calls whose work overlaps on the GPU (other streams, other threads) race and
 *    must be serialized by the caller. */
#define GSYNC_STATIC_MAX_BLOCKS 4096
int gsync_bench_barrier_static(const gsync_barrier_work* w, int param, uint64_t timeout_ns,
                               void* stream);

/* Mutex workload.  Block b makes `acq` acquisitions (id = b*acq + a): it waits delay[id]
 * SM cycles, locks, and inside the critical section its thread 0 reads total (the position
 * of this grant) and increments it (plain load/store), and its threads add addend[id] XOR
 * (i * 0x9E3779B1) to data[i] for every i < cs_words (plain loads/stores); then it unlocks,
 * and thread 0 writes id to grant_log[position] and the lock ticket to ticket[id]
 * (0xFFFFFFFF for the CAS kinds and CLUSTER_MCS): each is the grant's own slot, read by the
 * host only after the launch, so neither needs the lock.  count[b] receives the number of completed acquisitions.  The per-group kinds record a
 * ticket of their group's lock: COHORT as (die << 31) | ticket, CLUSTER as (cluster << 20) |
 * ticket (ticket below 2^20).
 * Buffers (device): delay, addend, grant_log, ticket [nblocks*acq]; data [cs_words];
 * total [1]; count [nblocks]; status [1].  data, total and status must start at zero, and no
 * two of the buffers may overlap. */
typedef struct gsync_mutex_work {
  int32_t kind, nblocks, block_threads, acq, cs_words;
  int32_t cluster; /* CLUSTER, CLUSTER_MCS: blocks per cluster (2..8, divides nblocks); else 0 or 1 */
  const uint32_t* delay;
  const uint32_t* addend;
  uint32_t* data;
  uint32_t* total;
  uint32_t* grant_log;
  uint32_t* ticket;
  uint32_t* count;
  uint32_t* status;
} gsync_mutex_work;
int gsync_bench_mutex(void* state, const gsync_mutex_work* w, void* stream);

/* The mutex workload from host buffers: copies delay and addend (host) into `workspace`
 * (device, >= gsync_bench_mutex_workspace_bytes bytes), initialises the mutex there, runs
 * the workload, and copies data, total, grant_log, ticket, count and status back into the
 * host buffers of `w` (whose pointers are host pointers here), then synchronizes `stream`. */
size_t gsync_bench_mutex_workspace_bytes(int kind, int nblocks, int acq, int cs_words);
int gsync_bench_mutex_host(const gsync_mutex_work* w, const gsync_backoff* backoff,
                           void* workspace, size_t workspace_bytes, void* stream);

/* Semaphore workload.  Block b makes `pairs` wait/post pairs (id = b*pairs + p); inside,
 * for hold[id] SM cycles from its entry, thread 0 counts itself into `occupancy` (atomic),
 * raises max_occupancy, increments total with a plain load/store when the initial count is
 * 1 and adds addend[id] to tally (atomic); at the end of the hold it counts itself out, then
 * posts.
 * Buffers (device): hold, addend [nblocks*pairs]; occupancy, max_occupancy, total, tally,
 * status [1] (zeroed by the caller); count [nblocks]. */
typedef struct gsync_sem_work {
  int32_t kind, nblocks, block_threads, pairs, initial_count, reserved;
  const uint32_t* hold;
  const uint32_t* addend;
  uint32_t* occupancy;
  uint32_t* max_occupancy;
  uint32_t* total;
  uint32_t* tally;
  uint32_t* count;
  uint32_t* status;
} gsync_sem_work;
int gsync_bench_sem(void* state, const gsync_sem_work* w, void* stream);

/* Condition-variable workload: a bounded buffer (producer/consumer queue) of `capacity` item
 * ids guarded by one mutex (TICKET, COHORT or CLUSTER) and two condition variables
 * (not_full, not_empty).  Blocks
 * 0 .. producers-1 each put items_per_producer items (item id = block * items_per_producer +
 * i); the next `consumers` blocks each take producers * items_per_producer / consumers items
 * (which must divide exactly).  A producer waits on not_full while the buffer is full and
 * signals not_empty after each put; a consumer the other way round.  A consumer adds value[id]
 * to sum[c] (int64) and seen[id] += 1 outside the mutex; count[c] = items it took.
 * Results: seen[i] = 1 for every item, sum over consumers = sum of value[] (int64).
 * Host entry: copies nothing; value, seen, sum, count, status are device buffers; the mutex,
 * the two condition variables and the buffer live in `workspace` (device, 256-byte aligned,
 * >= gsync_bench_condvar_workspace_bytes(capacity)), initialised by the call.  backoff (host,
 * may be NULL) sets the waiters' sleep; one co-resident launch of producers + consumers
 * blocks (in clusters of `cluster` for CLUSTER); GSYNC_ENOTRESIDENT if it does not fit.
 * status bits as for the other workloads. */
typedef struct gsync_condvar_work {
  int32_t producers, consumers, items_per_producer, capacity, block_threads;
  int32_t mutex_kind; /* the queue's mutex: GSYNC_MUTEX_TICKET, GSYNC_MUTEX_COHORT,
                         GSYNC_MUTEX_CLUSTER or GSYNC_MUTEX_CLUSTER_MCS */
  int32_t cluster;    /* CLUSTER, CLUSTER_MCS: blocks per cluster, 2..8, dividing producers +
                         consumers (0 = 4); ignored by the other kinds */
  const uint32_t* value;
  uint32_t* seen;
  int64_t* sum;
  uint32_t* count;
  uint32_t* status;
  uint32_t* acquisitions; /* optional (device, 1 word, zeroed by the caller, or NULL): mutex
                             acquisitions made, the re-locks after condition waits included */
} gsync_condvar_work;
size_t gsync_bench_condvar_workspace_bytes(int capacity);
/* Critical-section probe of the condition-variable queue (its roofline's T_cs): one block of
 * block_threads alternates a put and a take -- the workload's test of the queue under block
 * barriers, the slot and the queue's state, the signal -- framed like a hand-off (an acquire
 * load and a barrier before it, a barrier and a release store after it), `iters` times, with
 * no mutex and no waits; frame_only != 0 runs the frame around an empty body.  workspace
 * (device, 256-byte aligned) >= gsync_bench_condvar_workspace_bytes(16), initialised by the
 * call; out[0] (host) = elapsed ns.  Synchronizes `stream`. */
int gsync_probe_condvar_cs(int block_threads, int iters, int frame_only, void* workspace,
                           size_t workspace_bytes, uint64_t* out, void* stream);
int gsync_bench_condvar(const gsync_condvar_work* w, const gsync_backoff* backoff, void* workspace,
                        size_t workspace_bytes, void* stream);

/* Batched many-mutex workload (Section 5's mutex applied to many independent instances;
 * the paper measures one instance per kernel, and names autotuning of the backoff constants
 * as future work, Section 7).  One co-resident launch of nblocks blocks; acquisition i
 * (i < nacq) belongs to block i mod nblocks and runs, in order, on that block's thread 0:
 * lock mutex keys[i] with the policy of its contention class, sum[key] += adds[i] and
 * count[key] += 1 with plain loads and stores, unlock.  Blocks of barrier group g (blocks
 * group_start[g] .. + group_size[g] - 1; group_of_block[b] = g, or -1) also cross `rounds`
 * group barriers spread evenly over their acquisitions, with the sampled slot check of the
 * barrier workload (partner (j + r + 1) mod size inside the group); mix[b] and bad[b] as
 * there.
 *  - mutex_state (device, 128-byte aligned): nkeys x 384 bytes; zero it before the first
 *    launch and whenever a key's policy kind changes (the objects are left consistent by
 *    every completed launch otherwise).
 *  - key_class (device, nkeys bytes): class of each key, < nclasses.
 *  - policy (device, nclasses x 4 x u32): {kind (CAS_SPIN, CAS_BACKOFF, TICKET, CLUSTER,
 *    GSYNC_BATCHED_TICKET_CARRY, GSYNC_BATCHED_COHORT_CARRY, GSYNC_BATCHED_CLUSTER_CARRY or
 *    GSYNC_BATCHED_CLUSTER_DIE_CARRY; others act as TICKET), min_ns, max_ns, budget}: backoff of the CAS kind, or sleep per waiter ahead of the ticket kinds;
 *    min_ns = 0 spins without sleeping.  CLUSTER (the cluster cohort lock) applies in a cluster launch (cluster > 1) to
 *    keys below 256, whose local locks live in the blocks' shared memory, with `budget` passes
 *    per cohort (0 = the default, 64); elsewhere it acts as TICKET.  budget is ignored by the
 *    other kinds.  GSYNC_BATCHED_TICKET_CARRY is the ticket lock whose turn line carries the
 *    key's count and sum: one 16-byte record {turn, count, sum} read by the waiter's relaxed
 *    128-bit load and written by the holder's relaxed 128-bit store, so a hand-off moves the
 *    guarded data with it; a second kernel on the same stream copies such keys' count and sum
 *    to count[] and sum[] after the launch and zeroes them in the record.
 *    GSYNC_BATCHED_COHORT_CARRY is the two-die cohort lock with carrying records (a record
 *    {served, cohort word, sum} per die on a page homed on that die, and a global record
 *    {turn, -, sum}), `budget` passes inside a die per cohort (0 = the default, 64).  It
 *    applies to keys below ncohort, whose objects are in cohort_state; other keys of such a
 *    class use GSYNC_BATCHED_TICKET_CARRY.  The second kernel moves their count and sum out
 *    and returns their counters and records to zero.  GSYNC_BATCHED_CLUSTER_CARRY is the
 *    same carrying cohort protocol with the thread-block cluster as the group: in a cluster
 *    launch (cluster > 1), keys below 256 keep the cluster's ticket counter and record in
 *    the shared memory of the cluster's block 0 and pass the lock inside the cluster through
 *    distributed shared memory; the key's own object holds the global ticket and record.  The
 *    launch adds each cluster's count to count[] as it ends, and the second kernel moves the
 *    sum out.  Elsewhere it acts as GSYNC_BATCHED_TICKET_CARRY.
 *    GSYNC_BATCHED_CLUSTER_DIE_CARRY nests the two: cluster cohorts under die cohorts (on
 *    the die's page of the key's cohort object) under the global lock (the cohort object's
 *    lines 1-2), for keys below 256 and below ncohort in a cluster launch.  Its cluster level
 *    is an MCS queue whose holder pushes the record into its successor's shared memory.
 *    `budget` bounds the passes at both levels (at most 127 in a cluster, 255 on a die).
 *    The launch adds each block's count to count[] as it ends.  Elsewhere it acts as
 *    GSYNC_BATCHED_TICKET_CARRY.
 *  - keys (device, nacq x i32), adds (device, nacq x i64); sum (device, nkeys x i64) and
 *    count (device, nkeys x u32) zeroed by the caller.
 *  - group_state (device, 128-byte aligned): ngroups x 512 bytes, zeroed before the first
 *    launch; slots (device, 2 x nblocks u32) scratch; mix, bad (device, nblocks u32);
 *    status (device u32, zeroed).
 *  - cluster > 1 launches clusters of that size and uses the cluster-hierarchical barrier
 *    for the groups: every group must start at and span a multiple of `cluster` blocks
 *    (checked on the device; a violation sets GSYNC_STATUS_CONFIG and skips the barriers).
 *  - plain_launch = 1 uses an ordinary launch after the co-residency check instead of a
 *    cooperative one (for stream capture into a CUDA graph); cluster must then be 1.
 *  - cohort_state (device, 128-byte aligned; may be NULL when ncohort = 0): ncohort objects
 *    of 32768 bytes, object k for key k, each initialised by gsync_mutex_init_cohort (its
 *    budget is not used: the class policy's is) before the first launch and again whenever a
 *    key's policy kind changes.  ncohort < 0, or > 0 with cohort_state NULL or unaligned,
 *    returns GSYNC_EINVAL; values above nkeys act as nkeys. */
#define GSYNC_BATCHED_TICKET_CARRY 16u
#define GSYNC_BATCHED_COHORT_CARRY 17u
#define GSYNC_BATCHED_CLUSTER_CARRY 18u
#define GSYNC_BATCHED_CLUSTER_DIE_CARRY 19u
typedef struct gsync_batched_work {
  int32_t nkeys, nacq, nblocks, block_threads, ngroups, rounds, cluster, nclasses;
  int32_t plain_launch, ncohort;
  uint64_t timeout_ns;
  void* mutex_state;
  const uint8_t* key_class;
  const uint32_t* policy;
  const int32_t* keys;
  const int64_t* adds;
  int64_t* sum;
  uint32_t* count;
  const int32_t* group_start;
  const int32_t* group_size;
  const int32_t* group_of_block;
  void* group_state;
  uint32_t* slots;
  uint32_t* mix;
  uint32_t* bad;
  uint32_t* status;
  void* cohort_state;
} gsync_batched_work;
/* Launches the batched kernel and then batched_collect_kernel (two kernels, one stream). */
int gsync_bench_batched(const gsync_batched_work* w, void* stream);

/* Persistent serving loop with continuous batching (the paper motivates its primitives
 * with task queues, Section 1, and wishes for hardware enqueue/dequeue, Section 7).  Each
 * request q is an int32 segmented sum res[q] = sum of pool[offset[q] .. + length[q]) in
 * int64.  gsync_serve_run launches one co-resident kernel of nblocks x 256 threads, then
 * (host threads inside the call) publishes request q into the ring at time sched_ns[q]
 * after the start and records latency_ns[q] = the host time its completion flag was first
 * seen minus sched_ns[q] (open loop: latency counts from the scheduled arrival).
 *  - On the device, each of the `admitters` blocks first waits on the admission semaphore
 *    (n = nslots in-flight requests), then takes the next request index (its ticket of the
 *    ring's ticket lock), then waits for that ring entry to be published, claims a free slot and
 *    publishes the request in it; every other block claims chunks of chunk_elems values of
 *    any active request; the block that finishes a request's last chunk writes res[q] and
 *    done[q] = 1 into pinned host memory, frees the slot and posts the semaphore.  The
 *    semaphore and the lock are taken before the request arrives, off its latency path.
 *  - ring (ring_slots entries of 128 bytes, ring_slots a power of two), ctrl (64 words:
 *    ctrl[32] = shutdown), res
 *    (nreq x i64) and done (nreq x u32) are caller-owned pinned host memory
 *    (cudaHostAlloc or registered); pool is device memory; offset, length, sched_ns and
 *    latency_ns are ordinary host arrays.  The ring may instead be managed memory
 *    (cudaMallocManaged): on a GPU whose host reaches managed memory in place
 *    (cudaDevAttrDirectManagedMemAccessFromHost), the call advises it to live in device
 *    memory and to stay mapped for the host, and moves it there before it starts (the
 *    host's stores then land in device memory, and the admitters poll it through L2).  workspace (device, 256-byte aligned) holds
 *    gsync_serve_workspace_bytes(nslots) bytes.
 *  - Requires 0 <= offset[q], 1 <= length[q], offset[q] + length[q] <= pool_elems <= 2^32,
 *    at most 32767 chunks per request, nslots <= 64, non-decreasing sched_ns.
 *  - Returns GSYNC_ETIMEDOUT if not every request completed within drain_timeout_s after the
 *    last scheduled arrival, or if a device wait timed out (stats[3] = device status).
 *    Synchronizes `stream` before returning.
 * gsync_serve_baseline runs the same requests as one kernel launch each (block j sums chunk
 * j; the last block writes res and done), issued at the scheduled times round-robin over
 * `nstreams` caller streams, completions observed the same way.  workspace: device, 16-byte
 * aligned, gsync_serve_baseline_workspace_bytes(nreq) bytes. */
/* One ring entry (16 bytes), at the start of its own 128-byte line of the ring (entry i at
 * byte 128 * i).  Request q is in the ring when seq == seq_check == q + 1; the host writes
 * the entry as two aligned 8-byte stores, {seq, len} and {off, seq_check}, each single-copy
 * atomic, with no fence between them, and the device reads the entry with one 16-byte acquire
 * load: both sequence numbers current means both halves are. */
typedef struct gsync_serve_req {
  uint32_t seq;
  uint32_t len;
  uint32_t off;
  uint32_t seq_check;
} gsync_serve_req;
typedef struct gsync_serve_cfg {
  int32_t nreq, nslots, nblocks, admitters, chunk_elems, ring_slots;
  int32_t start_delay_us, drain_timeout_s;
  uint64_t timeout_ns;
} gsync_serve_cfg;
typedef struct gsync_serve_buffers {
  const int32_t* pool;
  int64_t pool_elems; /* every request must satisfy 0 <= offset, offset + length <= pool_elems */
  const int64_t* offset;
  const int64_t* length;
  const int64_t* sched_ns;
  gsync_serve_req* ring;
  uint32_t* ctrl;
  int64_t* res;
  uint32_t* done;
  int64_t* latency_ns;
  int64_t* publish_ns; /* optional (host, nreq, or NULL): host time request q was published
                          (persistent loop) or launched (baseline), ns from the start */
  uint64_t* trace;   /* optional (device, 4 x nreq u64, or NULL): %globaltimer when request q's
                        entry was seen, its slot published, its first chunk claimed, its last
                        chunk finished (persistent loop only) */
  uint32_t stats[4]; /* out: requests admitted, chunks processed, requests completed, device status */
} gsync_serve_buffers;
size_t gsync_serve_workspace_bytes(int nslots);
int gsync_serve_run(const gsync_serve_cfg* cfg, gsync_serve_buffers* buf, void* workspace,
                    size_t workspace_bytes, void* stream);
size_t gsync_serve_baseline_workspace_bytes(int nreq);
int gsync_serve_baseline(const gsync_serve_cfg* cfg, gsync_serve_buffers* buf, void* workspace,
                         size_t workspace_bytes, void* const* streams, int nstreams);

/* Host <-> device hand-off probe: one GPU thread and one host thread ping-pong a counter
 * through two words of pinned host memory (`words`, 64 u32, caller-owned, from cudaHostAlloc)
 * with system-scope release stores and acquire loads, `iters` times.  out_ns[0] (host) =
 * elapsed host ns for the whole exchange (one hand-off = out_ns[0] / (2 * iters)).
 * Synchronizes `stream`. */
int gsync_probe_host_pingpong(uint32_t* words, int iters, uint64_t* out_ns, void* stream);

/* ------------------------------------------------------------------------------------ */
/* Memory-system probes (Section 3, "Benchmarks"; Section 4 machine abstraction).        */
/* ------------------------------------------------------------------------------------ */

/* Access patterns of the paper's twelve + four probes and of the GB300 additions. */
typedef enum gsync_probe_op {
  GSYNC_PROBE_VOLATILE_LOAD = 0,   /* ld.volatile                          (paper: volatile read) */
  GSYNC_PROBE_VOLATILE_STORE = 1,  /* st.volatile                          (paper: volatile write) */
  GSYNC_PROBE_ATOMIC_READ = 2,     /* atomicAdd(p, 0)                      (paper: atomic read) */
  GSYNC_PROBE_ATOMIC_WRITE = 3,    /* atomicExch(p, 0)                     (paper: atomic write) */
  GSYNC_PROBE_LOAD_ACQUIRE = 4,    /* ld.acquire.gpu */
  GSYNC_PROBE_LOAD_RELAXED = 5,    /* ld.relaxed.gpu */
  GSYNC_PROBE_STORE_RELEASE = 6,   /* st.release.gpu */
  GSYNC_PROBE_RED_ADD = 7,         /* red.relaxed.gpu.add (no return) */
  GSYNC_PROBE_ATOMIC_ADD64 = 8,    /* atom.add.u64 */
  GSYNC_PROBE_ATOMIC_ACQREL = 9    /* atom.acq_rel.gpu.add */
} gsync_probe_op;

/* Throughput probe: `nblocks` blocks of `block_threads` threads; the master thread of each
 * block performs `iters` accesses of `op` to one shared word (contentious = 1) or to its own
 * word 256 bytes from the next block's (contentious = 0); pre_atomic = 1 issues one atomic
 * on the word first (the paper's "volatile preceded by atomic").  Each block writes its
 * start and end %globaltimer to times[2*b], times[2*b+1].  scratch (device) needs
 * 256 * nblocks bytes and is overwritten. */
int gsync_probe_throughput(int op, int contentious, int pre_atomic, int nblocks,
                           int block_threads, int iters, void* scratch, uint64_t* times,
                           void* stream);

/* Latency probe: one thread performs `iters` dependent accesses (each address depends on
 * the previous result) of one kind that returns a value: VOLATILE_LOAD, LOAD_RELAXED,
 * LOAD_ACQUIRE (L2 load round trips), ATOMIC_READ (atom.add of 0: L_rt), ATOMIC_WRITE,
 * ATOMIC_ADD64 or ATOMIC_ACQREL (each adds 0 or swaps in 0); the stores and red are refused
 * (GSYNC_EINVAL).  scratch (device, 128-byte aligned, 128 bytes) is overwritten.
 * out (device) [0] = elapsed ns, [1] = elapsed SM cycles. */
int gsync_probe_latency(int op, int iters, void* scratch, uint64_t* out, void* stream);

/* Ping-pong probe: the blocks on SMs sm_a and sm_b pass a token back and forth `iters`
 * times through release stores and acquire loads on separate lines; out[0] = elapsed ns
 * for the whole exchange (a hand-off is out[0] / (2 * iters)), out[1] = the SM of side A,
 * out[2] = the SM of side B, out[3] = status (0 ok).  Launches one block per SM.
 * scratch needs 512 bytes. */
int gsync_probe_pingpong(int sm_a, int sm_b, int iters, void* scratch, uint64_t* out,
                         void* stream);

/* Sleep probe: for each requested duration req_ns[i] (device, n entries) one thread calls
 * __nanosleep `iters` times and writes the mean measured ns per call to out_ns[i]. */
int gsync_probe_nanosleep(const uint32_t* req_ns, int n, int iters, uint64_t* out_ns,
                          void* stream);

/* Critical-section probe (T_cs): one block runs the mutex workload's critical-section body
 * `iters` times with no lock and no delay, framed like a hand-off (an acquire load and a
 * barrier before it, a barrier and a release store after it), timed with CUDA events;
 * out[0] (host) = elapsed ns.  cs_words = -1 runs the frame alone (no body), so that
 * T_cs(K) - T_frame is the body's own cost.  Synchronizes `stream`.  scratch (device,
 * 256-byte aligned) needs gsync_probe_cs_scratch_bytes(cs_words, iters) bytes. */
int gsync_probe_cs(int cs_words, int block_threads, int iters, void* scratch, uint64_t* out,
                   void* stream);
size_t gsync_probe_cs_scratch_bytes(int cs_words, int iters);

/* Semaphore critical-section probe (the semaphore roofline's T_cs): one block runs the
 * semaphore workload's critical section -- hold[p] SM cycles with the occupancy bookkeeping
 * and the tally inside them -- framed like a hand-off (an acquire load and a barrier before it, a barrier and a
 * release fence and store after it) for p < iters, with no semaphore.  hold, addend
 * (device) hold >= iters entries (hold may be NULL: no hold; both NULL: the frame alone,
 * with an empty critical section).  scratch (device, 256-byte aligned, 1024 bytes).
 * out[0] (host) = elapsed ns.  Synchronizes `stream`. */
int gsync_probe_sem_cs(int block_threads, int iters, const uint32_t* hold, const uint32_t* addend,
                       void* scratch, uint64_t* out, void* stream);

/* Hand-off probe: the ping-pong of gsync_probe_pingpong with a choice of how a side
 * releases (signal) and how the other side observes (wait); modes below.  Same buffers and
 * outputs as gsync_probe_pingpong. */
enum {
  GSYNC_SIGNAL_ST_RELEASE = 0,       /* st.release.gpu */
  GSYNC_SIGNAL_FENCE_ST_RELAXED = 1, /* fence.acq_rel.gpu; st.relaxed.gpu */
  GSYNC_SIGNAL_ST_RELAXED = 2,       /* st.relaxed.gpu (no ordering: a latency floor only) */
  GSYNC_SIGNAL_RED_RELEASE = 3,      /* red.release.gpu.add 1 */
  GSYNC_SIGNAL_EXCH_RELEASE = 4      /* atom.release.gpu.exch */
};
enum {
  GSYNC_WAIT_LD_ACQUIRE = 0,              /* poll with ld.acquire.gpu */
  GSYNC_WAIT_LD_RELAXED_FENCE = 1,        /* poll with ld.relaxed.gpu, then fence.acq_rel.gpu */
  GSYNC_WAIT_LD_RELAXED = 2,              /* poll with ld.relaxed.gpu (no ordering: floor only) */
  GSYNC_WAIT_LD_RELAXED_THEN_ACQUIRE = 3, /* poll relaxed, then one ld.acquire.gpu */
  GSYNC_WAIT_LD_VOLATILE_FENCE = 4,       /* poll with ld.volatile, then fence.acq_rel.gpu */
  GSYNC_WAIT_LD_RELAXED_X2 = 5            /* two relaxed polls in flight ~40 ns apart, then fence */
};
int gsync_probe_handoff(int signal_mode, int wait_mode, int sm_a, int sm_b, int iters,
                        void* scratch, uint64_t* out, void* stream);

/* Cluster probe: one cluster of `cluster` blocks (2..8; 1..8 for op 0) x 128 threads.
 * op 0: every thread runs `iters` hardware cluster barriers (out[0] / iters per barrier);
 * op 1: ranks 0 and cluster-1 ping-pong a flag in each other's shared memory with
 *       st.release.cluster / ld.acquire.cluster; op 2: the same with remote mbarrier arrives
 *       and mbarrier.try_wait; op 3: as op 1 with a 16-byte record written into the peer's
 *       shared memory and polled in one's own, relaxed 128-bit accesses, no fence; op 4: the
 *       same pulled (each writes its own record and polls the peer's); hand-off =
 *       out[0] / (2 * iters) for ops 1-4.  cluster < 2 with op > 0, or op outside 0..4,
 *       returns GSYNC_EINVAL.  out (device, 4 x u64):
 *       out[0] elapsed ns, out[3] status (0 ok, 1 timed out after 1 s). */
int gsync_probe_cluster(int op, int cluster, int iters, uint64_t* out, void* stream);

/* Fence probe: one thread runs `iters` gpu-scope fences; op 0 alone, op 1 after a relaxed
 * store, op 2 after four plain stores, op 3 cluster-scope fences.  out (device, 2 x u64):
 * elapsed ns and SM cycles.  scratch (device, 256-byte aligned) needs 1024 bytes. */
int gsync_probe_fence(int op, int iters, void* scratch, uint64_t* out, void* stream);

/* Topology probes (extends Section 4's machine abstraction to a two-die GPU: the distance
 * from an SM to a line's home die).  Both time chains of `iters` dependent atomic exchanges
 * (plus 4 untimed warm-up exchanges) from one thread and clobber the lines they touch.
 *
 * gsync_probe_rtt_by_sm: one block per SM, taking turns (the line is never contended);
 *   out_ns[s] (device, sm_count x u64) = ns for the chain from SM s to `line` (device,
 *   4-byte aligned).  scratch: device, 128-byte aligned, >= 128 bytes (the turn word).
 *   *status (device u32) = 0, or bit 0 if a turn wait ran past 1 s (entries left 0).
 * gsync_probe_rtt_by_line: from SM `sm`, out_ns[i] (device, nlines x u64) = ns for the chain
 *   to base + i * stride_bytes, for i < nlines (<= 65536); the caller owns that range.
 * Both are asynchronous on `stream`; GSYNC_EINVAL on bad arguments. */
int gsync_probe_rtt_by_sm(void* line, int iters, void* scratch, uint64_t* out_ns, uint32_t* status,
                          void* stream);
int gsync_probe_rtt_by_line(int sm, void* base, int nlines, int stride_bytes, int iters,
                            uint64_t* out_ns, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GSYNC_H */
